/*
 * swe_oracle_bathy.c -- FP64 oracle for two variants of the shallow-water
 * problem that the paper leaves open.  Sec. 2.3 leaves the global boundary
 * conditions to the programmer, outside the kernel; Sec. 3 takes a flat
 * bottom.  TEST INFRASTRUCTURE ONLY, like swe_oracle.c, and sharing nothing
 * with the CUDA library.  Arrays and index sets as in swe_oracle.c.
 *
 * Open (transmissive) sides.  Zero-gradient extrapolation: the ghost cell
 * copies the adjacent interior cell, all three components (no sign change),
 * so a wave leaves without the mirror image a wall sends back.
 *
 * Bottom topography.  With a bed elevation B(x, y) and H the water depth
 * (free surface H + B) the momentum equations gain the bed-slope source:
 *     (hu)_t + (hu^2 + g h^2/2)_x + (huv)_y = -g h B_x
 *     (hv)_t + (huv)_x + (hv^2 + g h^2/2)_y = -g h B_y.
 * Discretisation (this oracle's reading; the paper has no source term): in
 * each Lax-Wendroff step the source is taken at the same points as the
 * pressure-flux difference it balances, with the depth averaged over the
 * same two points:
 *   step 1, x-face between cells l, r:  + (dt/2dx) * g * (H_l + H_r)/2 * (B_l - B_r)
 *   step 2, cell i between x-faces L, R: + (dt/dx) * g * (Hx_L + Hx_R)/2 * (Bx_L - Bx_R),
 *                                       Bx = (B_i + B_i+1)/2 on the face,
 * and the same in y on the V rows.  For a lake at rest (H + B constant,
 * U = V = 0) each pair cancels exactly in real arithmetic, because
 * (g/2)(H_l^2 - H_r^2) = g (H_l + H_r)/2 (H_l - H_r) and H_l - H_r = B_r - B_l:
 * the scheme is well balanced.  The step reads B on the ghost ring too
 * (corners excepted); the caller fills it (a copy of the edge cell on walls
 * and open sides alike).
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#define IDX(i, j) ((size_t)(j) * (size_t)(nx + 2) + (size_t)(i))
#define FX(i, j) ((size_t)((j) - 1) * (size_t)(nx + 1) + (size_t)(i))
#define FY(i, j) ((size_t)(j) * (size_t)(nx) + (size_t)((i) - 1))

enum { B_LEFT = 1, B_RIGHT = 2, B_BOTTOM = 4, B_TOP = 8 };

/* from swe_oracle.c */
void oracle_fill_halo(int nx, int ny, int walls, double *H, double *U, double *V);
void oracle_step(int nx, int ny, double dx, double dy, double dt, double g, const double *H, const double *U,
                 const double *V, double *oH, double *oU, double *oV, double *faces);
size_t oracle_face_workspace(int nx, int ny);

/* Open sides named in ``sides``: ghost = adjacent interior cell (H, U, V). */
void oracle_fill_open(int nx, int ny, int sides, double *H, double *U, double *V)
{
    double *F[3] = {H, U, V};
    for (int k = 0; k < 3; ++k) {
        double *A = F[k];
        for (int j = 1; j <= ny; ++j) {
            if (sides & B_LEFT) A[IDX(0, j)] = A[IDX(1, j)];
            if (sides & B_RIGHT) A[IDX(nx + 1, j)] = A[IDX(nx, j)];
        }
        for (int i = 1; i <= nx; ++i) {
            if (sides & B_BOTTOM) A[IDX(i, 0)] = A[IDX(i, 1)];
            if (sides & B_TOP) A[IDX(i, ny + 1)] = A[IDX(i, ny)];
        }
    }
}

static double fxu(double H, double U, double g) { return U * U / H + 0.5 * g * H * H; }
static double fxv(double H, double U, double V) { return U * V / H; }
static double fyu(double H, double U, double V) { return U * V / H; }
static double fyv(double H, double V, double g) { return V * V / H + 0.5 * g * H * H; }

/* One step with the bed-slope source; B is (nx+2) x (ny+2) with its ghost
 * ring filled; ``faces`` holds oracle_face_workspace(nx, ny) doubles. */
void oracle_step_bathy(int nx, int ny, double dx, double dy, double dt, double g, const double *H, const double *U,
                       const double *V, const double *B, double *oH, double *oU, double *oV, double *faces)
{
    const size_t nfx = (size_t)(nx + 1) * (size_t)ny;
    const size_t nfy = (size_t)nx * (size_t)(ny + 1);
    double *Hx = faces, *Ux = Hx + nfx, *Vx = Ux + nfx;
    double *Hy = Vx + nfx, *Uy = Hy + nfy, *Vy = Uy + nfy;
    const double hx = 0.5 * dt / dx, hy = 0.5 * dt / dy, lx = dt / dx, ly = dt / dy;

    for (int j = 1; j <= ny; ++j) {
        for (int i = 0; i <= nx; ++i) {
            const double Hl = H[IDX(i, j)], Ul = U[IDX(i, j)], Vl = V[IDX(i, j)], Bl = B[IDX(i, j)];
            const double Hr = H[IDX(i + 1, j)], Ur = U[IDX(i + 1, j)], Vr = V[IDX(i + 1, j)], Br = B[IDX(i + 1, j)];
            Hx[FX(i, j)] = 0.5 * (Hl + Hr) + hx * (Ul - Ur);
            Ux[FX(i, j)] = 0.5 * (Ul + Ur) + hx * (fxu(Hl, Ul, g) - fxu(Hr, Ur, g)) + hx * (g * (0.5 * (Hl + Hr)) * (Bl - Br));
            Vx[FX(i, j)] = 0.5 * (Vl + Vr) + hx * (fxv(Hl, Ul, Vl) - fxv(Hr, Ur, Vr));
        }
    }
    for (int j = 0; j <= ny; ++j) {
        for (int i = 1; i <= nx; ++i) {
            const double Hd = H[IDX(i, j)], Ud = U[IDX(i, j)], Vd = V[IDX(i, j)], Bd = B[IDX(i, j)];
            const double Hu = H[IDX(i, j + 1)], Uu = U[IDX(i, j + 1)], Vu = V[IDX(i, j + 1)], Bu = B[IDX(i, j + 1)];
            Hy[FY(i, j)] = 0.5 * (Hd + Hu) + hy * (Vd - Vu);
            Uy[FY(i, j)] = 0.5 * (Ud + Uu) + hy * (fyu(Hd, Ud, Vd) - fyu(Hu, Uu, Vu));
            Vy[FY(i, j)] = 0.5 * (Vd + Vu) + hy * (fyv(Hd, Vd, g) - fyv(Hu, Vu, g)) + hy * (g * (0.5 * (Hd + Hu)) * (Bd - Bu));
        }
    }
    for (int j = 1; j <= ny; ++j) {
        for (int i = 1; i <= nx; ++i) {
            const double Hxl = Hx[FX(i - 1, j)], Uxl = Ux[FX(i - 1, j)], Vxl = Vx[FX(i - 1, j)];
            const double Hxr = Hx[FX(i, j)], Uxr = Ux[FX(i, j)], Vxr = Vx[FX(i, j)];
            const double Hyd = Hy[FY(i, j - 1)], Uyd = Uy[FY(i, j - 1)], Vyd = Vy[FY(i, j - 1)];
            const double Hyu = Hy[FY(i, j)], Uyu = Uy[FY(i, j)], Vyu = Vy[FY(i, j)];
            /* bed elevation on the four faces of the cell */
            const double Bxl = 0.5 * (B[IDX(i - 1, j)] + B[IDX(i, j)]), Bxr = 0.5 * (B[IDX(i, j)] + B[IDX(i + 1, j)]);
            const double Byd = 0.5 * (B[IDX(i, j - 1)] + B[IDX(i, j)]), Byu = 0.5 * (B[IDX(i, j)] + B[IDX(i, j + 1)]);

            oH[IDX(i, j)] = H[IDX(i, j)] + lx * (Uxl - Uxr) + ly * (Vyd - Vyu);
            oU[IDX(i, j)] = U[IDX(i, j)] + lx * (fxu(Hxl, Uxl, g) - fxu(Hxr, Uxr, g))
                            + ly * (fyu(Hyd, Uyd, Vyd) - fyu(Hyu, Uyu, Vyu))
                            + lx * (g * (0.5 * (Hxl + Hxr)) * (Bxl - Bxr));
            oV[IDX(i, j)] = V[IDX(i, j)] + lx * (fxv(Hxl, Uxl, Vxl) - fxv(Hxr, Uxr, Vxr))
                            + ly * (fyv(Hyd, Vyd, g) - fyv(Hyu, Vyu, g))
                            + ly * (g * (0.5 * (Hyd + Hyu)) * (Byd - Byu));
        }
    }
}

/* n_steps in place: fill reflective ``walls`` sides and ``open`` sides, then
 * step (with the source if B is not NULL, else the flat-bottom step of
 * swe_oracle.c).  0, or -1 if memory could not be allocated. */
int oracle_run_bc(int nx, int ny, int walls, int open, double dx, double dy, double dt, double g, int n_steps,
                  double *H, double *U, double *V, const double *B)
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
    memcpy(b[0], H, n * sizeof(double));
    memcpy(b[1], U, n * sizeof(double));
    memcpy(b[2], V, n * sizeof(double));
    for (int s = 0; s < n_steps; ++s) {
        oracle_fill_halo(nx, ny, walls, a[0], a[1], a[2]);
        oracle_fill_open(nx, ny, open, a[0], a[1], a[2]);
        if (B)
            oracle_step_bathy(nx, ny, dx, dy, dt, g, a[0], a[1], a[2], B, b[0], b[1], b[2], faces);
        else
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
