/*
 * swe_oracle_f32.c -- the oracle's step at the paper's own precision: the
 * same two-step Lax-Wendroff step, wall fill and run as swe_oracle.c, with
 * every value and operation in IEEE binary32 (the paper declares its
 * arrays `real` and its OpenCL kernel arguments `float`, Sec. 3.1 and Sec.
 * 4.2).  TEST INFRASTRUCTURE ONLY, like swe_oracle.c, and sharing nothing
 * with the CUDA library.
 *
 * Precision rules: the coefficients 0.5 dt/dx, 0.5 dt/dy, dt/dx, dt/dy are
 * formed in FP64 from the FP64 arguments and rounded once to binary32, g is
 * rounded once; every other operation is one binary32 operation in the order
 * written (float constants, no promotion to double: the build uses
 * -ffp-contract=off and a target whose float arithmetic is evaluated in
 * float, FLT_EVAL_METHOD == 0).  Arrays and index sets as in swe_oracle.c.
 */
#include <float.h>
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#if FLT_EVAL_METHOD != 0
#error "binary32 expressions must be evaluated in binary32"
#endif

#define IDX(i, j) ((size_t)(j) * (size_t)(nx + 2) + (size_t)(i))
#define FX(i, j) ((size_t)((j) - 1) * (size_t)(nx + 1) + (size_t)(i))
#define FY(i, j) ((size_t)(j) * (size_t)(nx) + (size_t)((i) - 1))

enum { F32_WALL_LEFT = 1, F32_WALL_RIGHT = 2, F32_WALL_BOTTOM = 4, F32_WALL_TOP = 8 };

/* Reflective ghost fill (the rule of oracle_fill_halo): the ghost copies the
 * adjacent interior cell with the wall-normal momentum negated; corners NaN. */
void oracle_fill_halo_f32(int nx, int ny, int walls, float *H, float *U, float *V)
{
    for (int j = 1; j <= ny; ++j) {
        if (walls & F32_WALL_LEFT) {
            H[IDX(0, j)] = H[IDX(1, j)];
            U[IDX(0, j)] = -U[IDX(1, j)];
            V[IDX(0, j)] = V[IDX(1, j)];
        }
        if (walls & F32_WALL_RIGHT) {
            H[IDX(nx + 1, j)] = H[IDX(nx, j)];
            U[IDX(nx + 1, j)] = -U[IDX(nx, j)];
            V[IDX(nx + 1, j)] = V[IDX(nx, j)];
        }
    }
    for (int i = 1; i <= nx; ++i) {
        if (walls & F32_WALL_BOTTOM) {
            H[IDX(i, 0)] = H[IDX(i, 1)];
            U[IDX(i, 0)] = U[IDX(i, 1)];
            V[IDX(i, 0)] = -V[IDX(i, 1)];
        }
        if (walls & F32_WALL_TOP) {
            H[IDX(i, ny + 1)] = H[IDX(i, ny)];
            U[IDX(i, ny + 1)] = U[IDX(i, ny)];
            V[IDX(i, ny + 1)] = -V[IDX(i, ny)];
        }
    }
    const size_t corners[4] = {IDX(0, 0), IDX(nx + 1, 0), IDX(0, ny + 1), IDX(nx + 1, ny + 1)};
    for (int c = 0; c < 4; ++c) {
        H[corners[c]] = NAN;
        U[corners[c]] = NAN;
        V[corners[c]] = NAN;
    }
}

/* Physical fluxes (Sec. 3): F = (U, U^2/H + g H^2/2, UV/H), G = (V, UV/H, V^2/H + g H^2/2). */
static float f32_flux_x_u(float H, float U, float g) { return U * U / H + 0.5f * g * H * H; }
static float f32_flux_x_v(float H, float U, float V) { return U * V / H; }
static float f32_flux_y_u(float H, float U, float V) { return U * V / H; }
static float f32_flux_y_v(float H, float V, float g) { return V * V / H + 0.5f * g * H * H; }

/* One step (the statements of oracle_step, in binary32).  ``faces`` holds
 * oracle_face_workspace(nx, ny) floats. */
void oracle_step_f32(int nx, int ny, double dx, double dy, double dt, double g64, const float *H, const float *U,
                     const float *V, float *oH, float *oU, float *oV, float *faces)
{
    const size_t nfx = (size_t)(nx + 1) * (size_t)ny;
    const size_t nfy = (size_t)nx * (size_t)(ny + 1);
    float *Hx = faces, *Ux = Hx + nfx, *Vx = Ux + nfx;
    float *Hy = Vx + nfx, *Uy = Hy + nfy, *Vy = Uy + nfy;

    const float hx = (float)(0.5 * dt / dx);
    const float hy = (float)(0.5 * dt / dy);
    const float lx = (float)(dt / dx);
    const float ly = (float)(dt / dy);
    const float g = (float)g64;

    for (int j = 1; j <= ny; ++j) {
        for (int i = 0; i <= nx; ++i) {
            const float Hl = H[IDX(i, j)], Ul = U[IDX(i, j)], Vl = V[IDX(i, j)];
            const float Hr = H[IDX(i + 1, j)], Ur = U[IDX(i + 1, j)], Vr = V[IDX(i + 1, j)];
            Hx[FX(i, j)] = 0.5f * (Hl + Hr) + hx * (Ul - Ur);
            Ux[FX(i, j)] = 0.5f * (Ul + Ur) + hx * (f32_flux_x_u(Hl, Ul, g) - f32_flux_x_u(Hr, Ur, g));
            Vx[FX(i, j)] = 0.5f * (Vl + Vr) + hx * (f32_flux_x_v(Hl, Ul, Vl) - f32_flux_x_v(Hr, Ur, Vr));
        }
    }
    for (int j = 0; j <= ny; ++j) {
        for (int i = 1; i <= nx; ++i) {
            const float Hd = H[IDX(i, j)], Ud = U[IDX(i, j)], Vd = V[IDX(i, j)];
            const float Hu = H[IDX(i, j + 1)], Uu = U[IDX(i, j + 1)], Vu = V[IDX(i, j + 1)];
            Hy[FY(i, j)] = 0.5f * (Hd + Hu) + hy * (Vd - Vu);
            Uy[FY(i, j)] = 0.5f * (Ud + Uu) + hy * (f32_flux_y_u(Hd, Ud, Vd) - f32_flux_y_u(Hu, Uu, Vu));
            Vy[FY(i, j)] = 0.5f * (Vd + Vu) + hy * (f32_flux_y_v(Hd, Vd, g) - f32_flux_y_v(Hu, Vu, g));
        }
    }
    for (int j = 1; j <= ny; ++j) {
        for (int i = 1; i <= nx; ++i) {
            const float Hxl = Hx[FX(i - 1, j)], Uxl = Ux[FX(i - 1, j)], Vxl = Vx[FX(i - 1, j)];
            const float Hxr = Hx[FX(i, j)], Uxr = Ux[FX(i, j)], Vxr = Vx[FX(i, j)];
            const float Hyd = Hy[FY(i, j - 1)], Uyd = Uy[FY(i, j - 1)], Vyd = Vy[FY(i, j - 1)];
            const float Hyu = Hy[FY(i, j)], Uyu = Uy[FY(i, j)], Vyu = Vy[FY(i, j)];

            oH[IDX(i, j)] = H[IDX(i, j)] + lx * (Uxl - Uxr) + ly * (Vyd - Vyu);
            oU[IDX(i, j)] = U[IDX(i, j)]
                            + lx * (f32_flux_x_u(Hxl, Uxl, g) - f32_flux_x_u(Hxr, Uxr, g))
                            + ly * (f32_flux_y_u(Hyd, Uyd, Vyd) - f32_flux_y_u(Hyu, Uyu, Vyu));
            oV[IDX(i, j)] = V[IDX(i, j)]
                            + lx * (f32_flux_x_v(Hxl, Uxl, Vxl) - f32_flux_x_v(Hxr, Uxr, Vxr))
                            + ly * (f32_flux_y_v(Hyd, Vyd, g) - f32_flux_y_v(Hyu, Vyu, g));
        }
    }
}

/* n_steps of (fill the ``walls`` sides, step) in place; 0 or -1 (no memory). */
int oracle_run_f32(int nx, int ny, int walls, double dx, double dy, double dt, double g, int n_steps, float *H,
                   float *U, float *V)
{
    const size_t n = (size_t)(nx + 2) * (size_t)(ny + 2);
    const size_t nf = 3 * (size_t)(nx + 1) * (size_t)ny + 3 * (size_t)nx * (size_t)(ny + 1);
    float *buf = (float *)malloc(3 * n * sizeof(float));
    float *faces = (float *)malloc(nf * sizeof(float));
    if (!buf || !faces) {
        free(buf);
        free(faces);
        return -1;
    }
    float *a[3] = {H, U, V};
    float *b[3] = {buf, buf + n, buf + 2 * n};
    memcpy(b[0], H, n * sizeof(float));
    memcpy(b[1], U, n * sizeof(float));
    memcpy(b[2], V, n * sizeof(float));
    for (int s = 0; s < n_steps; ++s) {
        oracle_fill_halo_f32(nx, ny, walls, a[0], a[1], a[2]);
        oracle_step_f32(nx, ny, dx, dy, dt, g, a[0], a[1], a[2], b[0], b[1], b[2], faces);
        for (int k = 0; k < 3; ++k) {
            float *t = a[k];
            a[k] = b[k];
            b[k] = t;
        }
    }
    if (a[0] != H) {
        memcpy(H, a[0], n * sizeof(float));
        memcpy(U, a[1], n * sizeof(float));
        memcpy(V, a[2], n * sizeof(float));
    }
    free(buf);
    free(faces);
    return 0;
}
