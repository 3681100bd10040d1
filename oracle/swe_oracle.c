/*
 * swe_oracle.c -- plain, slow FP64 CPU oracle for the two-step (Richtmyer)
 * Lax-Wendroff shallow-water step of "ForOpenCL: Transformations Exploiting
 * Array Syntax in Fortran for Accelerator Programming" (Sec. 3).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this file's library.  It shares
 * no code, header or constant with the CUDA library.
 *
 * Grid convention: arrays hold the interior plus a one-cell ghost ring,
 * (nx+2) x (ny+2) doubles, x fastest: element (i, j) at j*(nx+2) + i with
 * i = 0..nx+1, j = 0..ny+1; the interior is i = 1..nx, j = 1..ny.
 * H is the water height h, U = hu and V = hv (Sec. 3.1 names the state
 * arrays H, U, V with U, V the momenta).
 *
 * Compiled with -ffp-contract=off: every + - * / is one IEEE FP64 operation
 * in the order written, so the invariants pinned in tests hold bitwise.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX(i, j) ((size_t)(j) * (size_t)(nx + 2) + (size_t)(i))
/* x-face arrays: face i+1/2 for i = 0..nx on rows j = 1..ny */
#define FX(i, j) ((size_t)((j) - 1) * (size_t)(nx + 1) + (size_t)(i))
/* y-face arrays: face j+1/2 for j = 0..ny on columns i = 1..nx */
#define FY(i, j) ((size_t)(j) * (size_t)(nx) + (size_t)((i) - 1))

enum { WALL_LEFT = 1, WALL_RIGHT = 2, WALL_BOTTOM = 4, WALL_TOP = 8, WALL_ALL = 15 };

static int g_threads = 1;

/* Number of host threads the row loops of the step may use (>= 1). */
void oracle_set_threads(int n) { g_threads = n < 1 ? 1 : n; }

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Reflective walls.  The paper leaves the global boundary conditions to the
 * programmer, outside the kernel (Sec. 2.3); the walls here are reflective:
 * the ghost cell mirrors the adjacent interior cell, with the momentum
 * normal to the wall negated and the tangential momentum copied.  Only the
 * sides named in ``walls`` are filled; the other ghost cells keep whatever
 * they hold.  Corner ghosts are never read by the scheme (the x-face index
 * sets of Sec. 3.1 cover rows 1..ny only, the y-face sets columns 1..nx);
 * they are set to NaN so that any read of them would poison the result.
 */
void oracle_fill_halo(int nx, int ny, int walls, double *H, double *U, double *V)
{
    for (int j = 1; j <= ny; ++j) {
        if (walls & WALL_LEFT) {
            H[IDX(0, j)] = H[IDX(1, j)];
            U[IDX(0, j)] = -U[IDX(1, j)];
            V[IDX(0, j)] = V[IDX(1, j)];
        }
        if (walls & WALL_RIGHT) {
            H[IDX(nx + 1, j)] = H[IDX(nx, j)];
            U[IDX(nx + 1, j)] = -U[IDX(nx, j)];
            V[IDX(nx + 1, j)] = V[IDX(nx, j)];
        }
    }
    for (int i = 1; i <= nx; ++i) {
        if (walls & WALL_BOTTOM) {
            H[IDX(i, 0)] = H[IDX(i, 1)];
            U[IDX(i, 0)] = U[IDX(i, 1)];
            V[IDX(i, 0)] = -V[IDX(i, 1)];
        }
        if (walls & WALL_TOP) {
            H[IDX(i, ny + 1)] = H[IDX(i, ny)];
            U[IDX(i, ny + 1)] = U[IDX(i, ny)];
            V[IDX(i, ny + 1)] = -V[IDX(i, ny)];
        }
    }
    const double nan = NAN;
    const size_t corners[4] = {IDX(0, 0), IDX(nx + 1, 0), IDX(0, ny + 1), IDX(nx + 1, ny + 1)};
    for (int c = 0; c < 4; ++c) {
        H[corners[c]] = nan;
        U[corners[c]] = nan;
        V[corners[c]] = nan;
    }
}

/* Physical fluxes of the conservation laws (Sec. 3, the three PDEs):
 *   x-direction F = (hu, hu^2 + g h^2 / 2, huv),
 *   y-direction G = (hv, huv, hv^2 + g h^2 / 2),
 * written in the conserved variables H = h, U = hu, V = hv. */
static double flux_x_u(double H, double U, double g) { return U * U / H + 0.5 * g * H * H; }
static double flux_x_v(double H, double U, double V) { return U * V / H; }
static double flux_y_u(double H, double U, double V) { return U * V / H; }
static double flux_y_v(double H, double V, double g) { return V * V / H + 0.5 * g * H * H; }

/*
 * Size in doubles of the face workspace for oracle_step: the six face arrays
 * Hx, Ux, Vx ((nx+1) x ny) and Hy, Uy, Vy (nx x (ny+1)) of Sec. 3.1.
 */
size_t oracle_face_workspace(int nx, int ny)
{
    return 3 * (size_t)(nx + 1) * (size_t)ny + 3 * (size_t)nx * (size_t)(ny + 1);
}

/*
 * One two-step Lax-Wendroff step (Sec. 3, the two step equations; Sec. 3.1,
 * the Fortran statements for Hx and pH).  Reads H, U, V including the ghost
 * ring (which the caller fills), writes the interior of oH, oU, oV
 * (intent(out), double buffered as Sec. 2.5 requires).
 *
 * Step 1 (face states at t + dt/2).  For an x-face between the cell on its
 * left ("lt", index i) and on its right ("rt", index i+1):
 *     Qx = 0.5*(Q_lt + Q_rt) + (0.5*dt/dx)*(Fq_lt - Fq_rt),
 * which is the Fortran Hx statement of Sec. 3.1 (the printed equation's
 * "+ (F_{i+1} - F_i)" sign is read as the Fortran's "+ (F_i - F_{i+1})",
 * i.e. the standard Richtmyer minus).  y-faces likewise with dy and G.
 *
 * Step 2 (full step, dimensionally unsplit): for cell (i, j) with x-faces
 * i-1/2 ("face_lt") and i+1/2 ("face_rt"), y-faces j-1/2 ("face_dn") and
 * j+1/2 ("face_up"):
 *     Q' = Q + (dt/dx)*(F(face_lt) - F(face_rt)) + (dt/dy)*(G(face_dn) - G(face_up)),
 * the pH statement of Sec. 3.1, with the momentum rows using the physical
 * fluxes F, G evaluated at the face states.
 */
void oracle_step(int nx, int ny, double dx, double dy, double dt, double g,
                 const double *H, const double *U, const double *V,
                 double *oH, double *oU, double *oV, double *faces)
{
    const size_t nfx = (size_t)(nx + 1) * (size_t)ny;
    const size_t nfy = (size_t)nx * (size_t)(ny + 1);
    double *Hx = faces, *Ux = Hx + nfx, *Vx = Ux + nfx;
    double *Hy = Vx + nfx, *Uy = Hy + nfy, *Vy = Uy + nfy;

    const double hx = 0.5 * dt / dx; /* Fortran (0.5*dt/dx): (0.5*dt)/dx */
    const double hy = 0.5 * dt / dy;
    const double lx = dt / dx;
    const double ly = dt / dy;

    /* Step 1, x-faces i+1/2, i = 0..nx, rows j = 1..ny. */
#pragma omp parallel for schedule(static) num_threads(g_threads)
    for (int j = 1; j <= ny; ++j) {
        for (int i = 0; i <= nx; ++i) {
            const double Hl = H[IDX(i, j)], Ul = U[IDX(i, j)], Vl = V[IDX(i, j)];
            const double Hr = H[IDX(i + 1, j)], Ur = U[IDX(i + 1, j)], Vr = V[IDX(i + 1, j)];
            Hx[FX(i, j)] = 0.5 * (Hl + Hr) + hx * (Ul - Ur);
            Ux[FX(i, j)] = 0.5 * (Ul + Ur) + hx * (flux_x_u(Hl, Ul, g) - flux_x_u(Hr, Ur, g));
            Vx[FX(i, j)] = 0.5 * (Vl + Vr) + hx * (flux_x_v(Hl, Ul, Vl) - flux_x_v(Hr, Ur, Vr));
        }
    }
    /* Step 1, y-faces j+1/2, j = 0..ny, columns i = 1..nx. */
#pragma omp parallel for schedule(static) num_threads(g_threads)
    for (int j = 0; j <= ny; ++j) {
        for (int i = 1; i <= nx; ++i) {
            const double Hd = H[IDX(i, j)], Ud = U[IDX(i, j)], Vd = V[IDX(i, j)];
            const double Hu = H[IDX(i, j + 1)], Uu = U[IDX(i, j + 1)], Vu = V[IDX(i, j + 1)];
            Hy[FY(i, j)] = 0.5 * (Hd + Hu) + hy * (Vd - Vu);
            Uy[FY(i, j)] = 0.5 * (Ud + Uu) + hy * (flux_y_u(Hd, Ud, Vd) - flux_y_u(Hu, Uu, Vu));
            Vy[FY(i, j)] = 0.5 * (Vd + Vu) + hy * (flux_y_v(Hd, Vd, g) - flux_y_v(Hu, Vu, g));
        }
    }
    /* Step 2, cells i = 1..nx, j = 1..ny. */
#pragma omp parallel for schedule(static) num_threads(g_threads)
    for (int j = 1; j <= ny; ++j) {
        for (int i = 1; i <= nx; ++i) {
            /* x-faces i-1/2 (lt) and i+1/2 (rt) */
            const double Hxl = Hx[FX(i - 1, j)], Uxl = Ux[FX(i - 1, j)], Vxl = Vx[FX(i - 1, j)];
            const double Hxr = Hx[FX(i, j)], Uxr = Ux[FX(i, j)], Vxr = Vx[FX(i, j)];
            /* y-faces j-1/2 (dn) and j+1/2 (up) */
            const double Hyd = Hy[FY(i, j - 1)], Uyd = Uy[FY(i, j - 1)], Vyd = Vy[FY(i, j - 1)];
            const double Hyu = Hy[FY(i, j)], Uyu = Uy[FY(i, j)], Vyu = Vy[FY(i, j)];

            oH[IDX(i, j)] = H[IDX(i, j)] + lx * (Uxl - Uxr) + ly * (Vyd - Vyu);
            oU[IDX(i, j)] = U[IDX(i, j)]
                            + lx * (flux_x_u(Hxl, Uxl, g) - flux_x_u(Hxr, Uxr, g))
                            + ly * (flux_y_u(Hyd, Uyd, Vyd) - flux_y_u(Hyu, Uyu, Vyu));
            oV[IDX(i, j)] = V[IDX(i, j)]
                            + lx * (flux_x_v(Hxl, Uxl, Vxl) - flux_x_v(Hxr, Uxr, Vxr))
                            + ly * (flux_y_v(Hyd, Vyd, g) - flux_y_v(Hyu, Vyu, g));
        }
    }
}

/*
 * n_steps steps on the state held in H, U, V (arrays with ghost ring; the
 * result is left in them).  Each step: fill the ghosts of the sides named in
 * ``walls``, take one step into a second buffer, swap.  Returns 0, or -1 if
 * memory could not be allocated.
 */
int oracle_run(int nx, int ny, int walls, double dx, double dy, double dt, double g,
               int n_steps, double *H, double *U, double *V)
{
    const size_t n = (size_t)(nx + 2) * (size_t)(ny + 2);
    double *buf = (double *)malloc(3 * n * sizeof(double));
    double *faces = (double *)malloc(oracle_face_workspace(nx, ny) * sizeof(double));
    if (!buf || !faces) {
        free(buf);
        free(faces);
        return -1;
    }
    double *a[3] = {H, U, V};
    double *b[3] = {buf, buf + n, buf + 2 * n};
    /* ghost ring of the second buffer starts as a copy, so sides that are not
     * walls keep their (stale) neighbour data in both buffers */
    memcpy(b[0], H, n * sizeof(double));
    memcpy(b[1], U, n * sizeof(double));
    memcpy(b[2], V, n * sizeof(double));
    for (int s = 0; s < n_steps; ++s) {
        oracle_fill_halo(nx, ny, walls, a[0], a[1], a[2]);
        oracle_step(nx, ny, dx, dy, dt, g, a[0], a[1], a[2], b[0], b[1], b[2], faces);
        for (int k = 0; k < 3; ++k) {
            double *t = a[k];
            a[k] = b[k];
            b[k] = t;
        }
    }
    if (a[0] != H) {
        memcpy(H, a[0], n * sizeof(double));
        memcpy(U, a[1], n * sizeof(double));
        memcpy(V, a[2], n * sizeof(double));
    }
    free(buf);
    free(faces);
    return 0;
}

/*
 * Mass M = sum over interior cells of H * dx * dy.  Sec. 3 takes h as the
 * mass of a cell of unit size and uniform density; a cell of size dx x dy
 * holds h dx dy.  Neumaier-compensated summation in row-major order, so the
 * result is the exact sum to within about one rounding.
 */
double oracle_mass(int nx, int ny, double dx, double dy, const double *H)
{
    double s = 0.0, c = 0.0;
    for (int j = 1; j <= ny; ++j) {
        for (int i = 1; i <= nx; ++i) {
            const double x = H[IDX(i, j)];
            const double t = s + x;
            if (fabs(s) >= fabs(x))
                c += (s - t) + x;
            else
                c += (x - t) + s;
            s = t;
        }
    }
    return (s + c) * dx * dy;
}

/*
 * CFL time step.  Sec. 3 requires dt <= dx / (sqrt(g h) + |u|) (stated in
 * 1D).  In 2D the bound is taken per direction and per cell:
 *     dt = cfl * min over cells of min(dx / (sqrt(g H) + |U/H|),
 *                                      dy / (sqrt(g H) + |V/H|)).
 */
double oracle_cfl_dt(int nx, int ny, double dx, double dy, double g, double cfl,
                     const double *H, const double *U, const double *V)
{
    double best = INFINITY;
    for (int j = 1; j <= ny; ++j) {
        for (int i = 1; i <= nx; ++i) {
            const double h = H[IDX(i, j)];
            const double c = sqrt(g * h);
            const double tx = dx / (c + fabs(U[IDX(i, j)] / h));
            const double ty = dy / (c + fabs(V[IDX(i, j)] / h));
            if (tx < best) best = tx;
            if (ty < best) best = ty;
        }
    }
    return cfl * best;
}
