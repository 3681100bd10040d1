// swe_region.cu -- the two-step Lax-Wendroff step of Sec. 3 and the wall
// ghost fill written as region statements (Sec. 2.3, Sec. 3.1) in the front
// end of swe_region.cuh, and the C ABI around them (swe_region_*).
//
// Arrays carry their ghost ring: (nx + 2) x (ny + 2) elements, interior
// cells at (1..nx, 1..ny).  As in Sec. 2.3, boundary conditions are not part
// of the step: the step reads the ghosts as they are, and the wall fill is a
// separate set of region statements the caller runs between steps.
//
// Lowering (Sec. 4.2.1).  One CTA owns a TX x TY tile of interior cells.
// The intent(in) arrays H, U, V are staged with their one-cell halo into
// shared memory by three TMA tile loads; the face arrays are shared-memory
// tiles; the output statements store straight to global memory.  Each
// statement group is one loop of the CTA's threads over its region.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <new>

#include "swe_device.cuh"
#include "swe_region.cuh"

namespace swe {
namespace region {

template <class T>
struct LwCoef {
    T hx, hy;  // 0.5 dt/dx, 0.5 dt/dy (step 1)
    T lx, ly;  // dt/dx, dt/dy (step 2)
    T g;
};

// Physical fluxes of Sec. 3 as elemental functions of regions:
//   F = (U, U^2/H + g H^2/2, U V/H),   G = (V, U V/H, V^2/H + g H^2/2).
template <class EH, class EU, class T>
__host__ __device__ __forceinline__ auto flux_x_u(const EH &H, const EU &U, T g)
{
    return U * U / H + 0.5 * g * H * H;
}
template <class EH, class EU, class EV>
__host__ __device__ __forceinline__ auto flux_x_v(const EH &H, const EU &U, const EV &V)
{
    return U * V / H;
}
template <class EH, class EU, class EV>
__host__ __device__ __forceinline__ auto flux_y_u(const EH &H, const EU &U, const EV &V)
{
    return U * V / H;
}
template <class EH, class EV, class T>
__host__ __device__ __forceinline__ auto flux_y_v(const EH &H, const EV &V, T g)
{
    return V * V / H + 0.5 * g * H * H;
}

// One Lax-Wendroff step (Sec. 3) on arrays with a one-cell halo.  H, U, V
// are (nx + 2) x (ny + 2) with their ghosts filled, and oH, oU, oV of that
// shape receive the interior.  The temporaries: Fu, Fuv, Gv, the cell
// fluxes U^2/H + gH^2/2, UV/H (both F's third and G's second component) and
// V^2/H + gH^2/2, of the cell arrays' shape; on the (nx + 1) x ny x-faces
// (face i between cells i and i + 1) Ux and the face fluxes FXu, FXv; on
// the nx x (ny + 1) y-faces Vy, GYu, GYv.
//
// Step 1 takes the half step to every face from the two cells beside it; a
// face array's region is the cell arrays' with one cell fewer left out on
// the face's side, so the face arrays are one longer than the interior in
// their direction.  The face states Hx, Vx (Hy, Uy) are only needed through
// the face fluxes, which are formed in the same statement group, so they are
// not stored.  Step 2 updates each interior cell from its four faces, the
// face regions now leaving one face out on the far side.  Each flux value is
// computed once per cell or face, by the same operations in the same order as
// the textbook per-face form, so the bits do not change.
#pragma nv_exec_check_disable
template <class T, class Run, class A, class F, class X, class Y, class O>
__host__ __device__ __forceinline__ void lw_statements(Run &run, const A &H, const A &U, const A &V, const F &Fu,
                                                       const F &Fuv, const F &Gv, const X &Ux, const X &FXu,
                                                       const X &FXv, const Y &Vy, const Y &GYu, const Y &GYv,
                                                       const O &oH, const O &oU, const O &oV, const LwCoef<T> &k)
{
    const Halo interior{1, 1, 1, 1}, whole{0, 0, 0, 0};
    // cells on the left / right of the x-faces, below / above the y-faces
    const Halo lt{0, 1, 1, 1}, rt{1, 0, 1, 1}, dn{1, 1, 0, 1}, up{1, 1, 1, 0};

    // Cell fluxes (Sec. 3: F = (U, U^2/H + gH^2/2, UV/H), G = (V, UV/H, V^2/H + gH^2/2)).
    {
        const auto Hc = region_cpy(H, whole), Uc = region_cpy(U, whole), Vc = region_cpy(V, whole);
        run(region_ptr(Fu, whole) = flux_x_u(Hc, Uc, k.g), region_ptr(Fuv, whole) = flux_x_v(Hc, Uc, Vc),
            region_ptr(Gv, whole) = flux_y_v(Hc, Vc, k.g));
    }
    // Step 1, x-faces: Q_face = (Q_lt + Q_rt) / 2 + (dt / 2dx) (F_lt - F_rt).
    {
        const auto Hf = 0.5 * (region_cpy(H, lt) + region_cpy(H, rt)) + k.hx * (region_cpy(U, lt) - region_cpy(U, rt));
        const auto Uf = 0.5 * (region_cpy(U, lt) + region_cpy(U, rt)) + k.hx * (region_cpy(Fu, lt) - region_cpy(Fu, rt));
        const auto Vf = 0.5 * (region_cpy(V, lt) + region_cpy(V, rt)) + k.hx * (region_cpy(Fuv, lt) - region_cpy(Fuv, rt));
        // the y-face group reads neither of these: no barrier in between
        run.independent(region_ptr(Ux, whole) = Uf, region_ptr(FXu, whole) = flux_x_u(Hf, Uf, k.g),
                        region_ptr(FXv, whole) = flux_x_v(Hf, Uf, Vf));
    }
    // Step 1, y-faces with G and dt / 2dy.
    {
        const auto Hf = 0.5 * (region_cpy(H, dn) + region_cpy(H, up)) + k.hy * (region_cpy(V, dn) - region_cpy(V, up));
        const auto Uf = 0.5 * (region_cpy(U, dn) + region_cpy(U, up)) + k.hy * (region_cpy(Fuv, dn) - region_cpy(Fuv, up));
        const auto Vf = 0.5 * (region_cpy(V, dn) + region_cpy(V, up)) + k.hy * (region_cpy(Gv, dn) - region_cpy(Gv, up));
        run(region_ptr(Vy, whole) = Vf, region_ptr(GYu, whole) = flux_y_u(Hf, Uf, Vf),
            region_ptr(GYv, whole) = flux_y_v(Hf, Vf, k.g));
    }
    // Step 2: Q' = Q + (dt/dx) (F(face left) - F(face right))
    //                + (dt/dy) (G(face below) - G(face above)).
    {
        const Halo fl{0, 1, 0, 0}, fr{1, 0, 0, 0}, fd{0, 0, 0, 1}, fu{0, 0, 1, 0};
        run(region_ptr(oH, interior) = region_cpy(H, interior) + k.lx * (region_cpy(Ux, fl) - region_cpy(Ux, fr)) +
                                       k.ly * (region_cpy(Vy, fd) - region_cpy(Vy, fu)),
            region_ptr(oU, interior) = region_cpy(U, interior) + k.lx * (region_cpy(FXu, fl) - region_cpy(FXu, fr)) +
                                       k.ly * (region_cpy(GYu, fd) - region_cpy(GYu, fu)),
            region_ptr(oV, interior) = region_cpy(V, interior) + k.lx * (region_cpy(FXv, fl) - region_cpy(FXv, fr)) +
                                       k.ly * (region_cpy(GYv, fd) - region_cpy(GYv, fu)));
    }
}

// The step over a bottom topography B (bed elevation; H the depth, H + B the
// free surface): the momentum rows gain the bed-slope source -g H B_x
// (-g H B_y), taken at the points of the pressure-flux difference it
// balances with the depth averaged over the same two points, so that a lake
// at rest (H + B constant, U = V = 0) cancels term by term:
//   step 1 on a face between cells a, b:   + (dt/2dx) g (H_a + H_b)/2 (B_a - B_b)
//   step 2 on a cell between faces L, R:   + (dt/dx) g (Hx_L + Hx_R)/2 (Bx_L - Bx_R),
//   with Bx = (B_i + B_i+1)/2 on each face, and likewise in y.
// B has the cell arrays' shape, ghosts included.  The face depths Hx, Hy are
// now stored for step 2; everything else is lw_statements'.
#pragma nv_exec_check_disable
template <class T, class Run, class A, class F, class X, class Y, class O>
__host__ __device__ __forceinline__ void bed_statements(Run &run, const A &H, const A &U, const A &V, const A &B,
                                                        const F &Fu, const F &Fuv, const F &Gv, const X &Hx,
                                                        const X &Ux, const X &FXu, const X &FXv, const Y &Hy,
                                                        const Y &Vy, const Y &GYu, const Y &GYv, const O &oH,
                                                        const O &oU, const O &oV, const LwCoef<T> &k)
{
    const Halo interior{1, 1, 1, 1}, whole{0, 0, 0, 0};
    const Halo lt{0, 1, 1, 1}, rt{1, 0, 1, 1}, dn{1, 1, 0, 1}, up{1, 1, 1, 0};
    {
        const auto Hc = region_cpy(H, whole), Uc = region_cpy(U, whole), Vc = region_cpy(V, whole);
        run(region_ptr(Fu, whole) = flux_x_u(Hc, Uc, k.g), region_ptr(Fuv, whole) = flux_x_v(Hc, Uc, Vc),
            region_ptr(Gv, whole) = flux_y_v(Hc, Vc, k.g));
    }
    {
        const auto Hl = region_cpy(H, lt), Hr = region_cpy(H, rt);
        const auto Hf = 0.5 * (Hl + Hr) + k.hx * (region_cpy(U, lt) - region_cpy(U, rt));
        const auto Uf = 0.5 * (region_cpy(U, lt) + region_cpy(U, rt)) + k.hx * (region_cpy(Fu, lt) - region_cpy(Fu, rt)) +
                        k.hx * (k.g * (0.5 * (Hl + Hr)) * (region_cpy(B, lt) - region_cpy(B, rt)));
        const auto Vf = 0.5 * (region_cpy(V, lt) + region_cpy(V, rt)) + k.hx * (region_cpy(Fuv, lt) - region_cpy(Fuv, rt));
        run.independent(region_ptr(Hx, whole) = Hf, region_ptr(Ux, whole) = Uf,
                        region_ptr(FXu, whole) = flux_x_u(Hf, Uf, k.g), region_ptr(FXv, whole) = flux_x_v(Hf, Uf, Vf));
    }
    {
        const auto Hd = region_cpy(H, dn), Hu = region_cpy(H, up);
        const auto Hf = 0.5 * (Hd + Hu) + k.hy * (region_cpy(V, dn) - region_cpy(V, up));
        const auto Uf = 0.5 * (region_cpy(U, dn) + region_cpy(U, up)) + k.hy * (region_cpy(Fuv, dn) - region_cpy(Fuv, up));
        const auto Vf = 0.5 * (region_cpy(V, dn) + region_cpy(V, up)) + k.hy * (region_cpy(Gv, dn) - region_cpy(Gv, up)) +
                        k.hy * (k.g * (0.5 * (Hd + Hu)) * (region_cpy(B, dn) - region_cpy(B, up)));
        run(region_ptr(Hy, whole) = Hf, region_ptr(Vy, whole) = Vf, region_ptr(GYu, whole) = flux_y_u(Hf, Uf, Vf),
            region_ptr(GYv, whole) = flux_y_v(Hf, Vf, k.g));
    }
    {
        const Halo fl{0, 1, 0, 0}, fr{1, 0, 0, 0}, fd{0, 0, 0, 1}, fu{0, 0, 1, 0};
        // the bed on the four faces of each interior cell
        const auto Bc = region_cpy(B, interior);
        const auto Bxl = 0.5 * (region_cpy(B, Halo{0, 2, 1, 1}) + Bc), Bxr = 0.5 * (Bc + region_cpy(B, Halo{2, 0, 1, 1}));
        const auto Byd = 0.5 * (region_cpy(B, Halo{1, 1, 0, 2}) + Bc), Byu = 0.5 * (Bc + region_cpy(B, Halo{1, 1, 2, 0}));
        run(region_ptr(oH, interior) = region_cpy(H, interior) + k.lx * (region_cpy(Ux, fl) - region_cpy(Ux, fr)) +
                                       k.ly * (region_cpy(Vy, fd) - region_cpy(Vy, fu)),
            region_ptr(oU, interior) = region_cpy(U, interior) + k.lx * (region_cpy(FXu, fl) - region_cpy(FXu, fr)) +
                                       k.ly * (region_cpy(GYu, fd) - region_cpy(GYu, fu)) +
                                       k.lx * (k.g * (0.5 * (region_cpy(Hx, fl) + region_cpy(Hx, fr))) * (Bxl - Bxr)),
            region_ptr(oV, interior) = region_cpy(V, interior) + k.lx * (region_cpy(FXv, fl) - region_cpy(FXv, fr)) +
                                       k.ly * (region_cpy(GYv, fd) - region_cpy(GYv, fu)) +
                                       k.ly * (k.g * (0.5 * (region_cpy(Hy, fd) + region_cpy(Hy, fu))) * (Byd - Byu)));
    }
}

// Boundary conditions as region statements on the whole (nx + 2) x (ny + 2)
// arrays, one group per side: each ghost strip gets the strip of interior
// cells beside it, with the wall-normal momentum negated on a reflective
// wall (kind 1) and copied unchanged on an open, zero-gradient side (kind 2);
// kind 0 leaves the side alone.  Sides: left, right, bottom, top.  Corner
// ghosts are not written (the step never reads them).
struct Sides {
    int kind[4];
};

#pragma nv_exec_check_disable
template <class Run, class A>
__host__ __device__ __forceinline__ void boundary_statements(Run &run, const A &H, const A &U, const A &V,
                                                             const Sides &sd)
{
    const int nx = H.nx - 2, ny = H.ny - 2;
    const Halo ghost[4] = {{0, nx + 1, 1, 1}, {nx + 1, 0, 1, 1}, {1, 1, 0, ny + 1}, {1, 1, ny + 1, 0}};
    const Halo edge[4] = {{1, nx, 1, 1}, {nx, 1, 1, 1}, {1, 1, 1, ny}, {1, 1, ny, 1}};
#pragma unroll
    for (int side = 0; side < 4; ++side) {
        const Halo g = ghost[side], e = edge[side];
        if (sd.kind[side] == 2) {
            run(region_ptr(H, g) = region_cpy(H, e), region_ptr(U, g) = region_cpy(U, e),
                region_ptr(V, g) = region_cpy(V, e));
        } else if (sd.kind[side] == 1 && side < 2) {
            run(region_ptr(H, g) = region_cpy(H, e), region_ptr(U, g) = -region_cpy(U, e),
                region_ptr(V, g) = region_cpy(V, e));
        } else if (sd.kind[side] == 1) {
            run(region_ptr(H, g) = region_cpy(H, e), region_ptr(U, g) = region_cpy(U, e),
                region_ptr(V, g) = -region_cpy(V, e));
        }
    }
}

// Launch shape of the step kernel: TX x TY interior cells per CTA, NT
// threads.  The staged inputs are (TX + 2) x (TY + 2) with rows padded to a
// 16-byte multiple (the TMA box); each staged array starts on 128 bytes (a
// TMA destination must) and the temporaries follow them.
template <class T, int TX_, int TY_, int NT_>
struct Shape {
    static constexpr int TX = TX_, TY = TY_, NT = NT_;
    static constexpr int VEC = 16 / (int)sizeof(T);
    static constexpr int BX = (TX + 2 + VEC - 1) / VEC * VEC;
    static constexpr int BY = TY + 2;
    static constexpr int ALIGN = 128 / (int)sizeof(T);
    static constexpr int IN = (BX * BY + ALIGN - 1) / ALIGN * ALIGN;
    static constexpr int CF = (TX + 2) * (TY + 2);  // cell fluxes
    static constexpr int FX = (TX + 1) * TY;        // x-face arrays
    static constexpr int FY = TX * (TY + 1);        // y-face arrays
    static constexpr size_t SMEM = 128 + (size_t)(3 * IN + 3 * CF + 3 * FX + 3 * FY) * sizeof(T);
    // with a bed: B staged too, and the face depths Hx, Hy kept
    static constexpr size_t SMEM_BED = SMEM + (size_t)(IN + FX + FY) * sizeof(T);
    static_assert(TX % VEC == 0, "TMA x coordinate must be a 16-byte multiple");
    static_assert((IN * sizeof(T)) % 128 == 0, "each staged input starts on 128 bytes");
    static_assert(BX <= 256 && BY <= 256, "TMA box limit");
};

struct Maps4 {
    CUtensorMap m[4];  // H, U, V and (the bed step only) B
};

template <class T>
struct Out3 {
    T *h, *u, *v;
    long long pitch;
};

template <class S, class T, bool BED>
__global__ void __launch_bounds__(S::NT) region_lw_kernel(const __grid_constant__ Maps4 maps, Out3<T> out, int nx,
                                                          int ny, LwCoef<T> k, int *err)
{
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm);
    // staged inputs first, each on a 128-byte boundary (the TMA destination
    // rule), then the temporaries
    T *sH = reinterpret_cast<T *>(sm + 128);
    T *sU = sH + S::IN, *sV = sU + S::IN;
    T *sB = sV + S::IN;  // BED only
    T *cf = sV + (BED ? 2 : 1) * S::IN;
    T *fx = cf + 3 * S::CF;
    T *fy = fx + 3 * S::FX;
    T *hxy = fy + 3 * S::FY;  // BED only: Hx, Hy
    const int x0 = blockIdx.x * S::TX, y0 = blockIdx.y * S::TY;  // tile corner, ghosted coordinates

    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(bar, (BED ? 4u : 3u) * S::BX * S::BY * (uint32_t)sizeof(T));
        tma_load_2d(sH, &maps.m[0], bar, x0, y0);
        tma_load_2d(sU, &maps.m[1], bar, x0, y0);
        tma_load_2d(sV, &maps.m[2], bar, x0, y0);
        if (BED) tma_load_2d(sB, &maps.m[3], bar, x0, y0);
    }
    const bool ok = mbar_wait_bounded(bar, 0, err);
    if (!__syncthreads_and(ok)) return;

    // The tile's cells at or past (vx, vy) belong to the right / top ghosts
    // or lie outside the arrays: the output statements store below them.
    constexpr int CX = S::TX + 2, CY = S::TY + 2;
    const int vx = min(CX, nx + 1 - x0), vy = min(CY, ny + 1 - y0);
    const auto H = array<int>(sH, CX, CY, S::BX), U = array<int>(sU, CX, CY, S::BX), V = array<int>(sV, CX, CY, S::BX);
    const auto Fu = array<int>(cf, CX, CY, CX), Fuv = array<int>(cf + S::CF, CX, CY, CX),
               Gv = array<int>(cf + 2 * S::CF, CX, CY, CX);
    const auto Ux = array<int>(fx, S::TX + 1, S::TY, S::TX + 1), FXu = array<int>(fx + S::FX, S::TX + 1, S::TY, S::TX + 1),
               FXv = array<int>(fx + 2 * S::FX, S::TX + 1, S::TY, S::TX + 1);
    const auto Vy = array<int>(fy, S::TX, S::TY + 1, S::TX), GYu = array<int>(fy + S::FY, S::TX, S::TY + 1, S::TX),
               GYv = array<int>(fy + 2 * S::FY, S::TX, S::TY + 1, S::TX);
    // output windows: (TY + 2) rows of the planes from the tile's corner (32-bit offsets within them)
    const long long o = (long long)y0 * out.pitch + x0;
    const int op = (int)out.pitch;
    const Window<T, int> oH{out.h + o, CX, CY, op, vx, vy};
    const Window<T, int> oU{out.u + o, CX, CY, op, vx, vy};
    const Window<T, int> oV{out.v + o, CX, CY, op, vx, vy};
    // (-0, -0) for the packed products, as -0 * g (g > 0 is checked on the
    // host): a run-time value, which the compiler cannot fold into a multiply
    const float nz0 = __fmul_rn(-0.0f, (float)k.g);
    CtaRun<S::NT> run{err, pack2(nz0, nz0)};
    if constexpr (BED) {
        const auto B = array<int>(sB, CX, CY, S::BX);
        const auto Hx = array<int>(hxy, S::TX + 1, S::TY, S::TX + 1);
        const auto Hy = array<int>(hxy + S::FX, S::TX, S::TY + 1, S::TX);
        bed_statements<T>(run, H, U, V, B, Fu, Fuv, Gv, Hx, Ux, FXu, FXv, Hy, Vy, GYu, GYv, oH, oU, oV, k);
    } else {
        lw_statements<T>(run, H, U, V, Fu, Fuv, Gv, Ux, FXu, FXv, Vy, GYu, GYv, oH, oU, oV, k);
    }
}

__global__ void div_probe_kernel(const float *a, const float *b, float *out, int n, int which)
{
    if (which == 4) {  // the stencil kernels' approximate reciprocal
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = rcp(b[i]);
        return;
    }
    if (which == 3) {  // the fast division's reciprocal step alone
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
            out[i] = rcp_rn_fast(b[i]);
        return;
    }
    if (which == 2) {  // elements 2m, 2m + 1 as one pair (n even)
        for (int m = blockIdx.x * blockDim.x + threadIdx.x; 2 * m < n; m += gridDim.x * blockDim.x) {
            F2 q;
            if (!fdiv_fast2(pack2(a[2 * m], a[2 * m + 1]), pack2(b[2 * m], b[2 * m + 1]), q))
                q = pack2(__fdiv_rn(a[2 * m], b[2 * m]), __fdiv_rn(a[2 * m + 1], b[2 * m + 1]));
            unpack2(q, out[2 * m], out[2 * m + 1]);
        }
        return;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = which == 0 ? fdiv_rn(a[i], b[i]) : __fdiv_rn(a[i], b[i]);
}

template <class T>
__global__ void __launch_bounds__(256) region_walls_kernel(Array<T> H, Array<T> U, Array<T> V, Sides sd, int *err)
{
    GridRun run{err};
    boundary_statements(run, H, U, V, sd);
}

// Step-kernel shapes (variant 1.. of swe_region_create).
using F32A = Shape<float, 64, 16, 256>;
using F32B = Shape<float, 128, 8, 256>;
using F32C = Shape<float, 32, 32, 256>;
using F32D = Shape<float, 64, 16, 128>;
using F32E = Shape<float, 32, 16, 128>;
using F64A = Shape<double, 64, 8, 256>;
using F64B = Shape<double, 32, 16, 256>;
using F64C = Shape<double, 32, 8, 128>;

}  // namespace region
}  // namespace swe

using namespace swe;
using namespace swe::region;

struct swe_region {
    int dtype = SWE_F32;
    int nx = 0, ny = 0;
    long long pitch = 0;
    int variant = 1;
    int *d_err = nullptr;
    long long launches = 0;
};

static swe_status rst(cudaError_t e)
{
    if (e == cudaSuccess) return SWE_OK;
    return e == cudaErrorMemoryAllocation ? SWE_ENOMEM : SWE_ECUDA;
}

template <class S>
static void shape_of(int *tx, int *ty, int *nt, size_t *smem)
{
    *tx = S::TX;
    *ty = S::TY;
    *nt = S::NT;
    *smem = S::SMEM;
}

// Tile shape of (dtype, variant); false if there is none.
static bool variant_shape(int dtype, int variant, int *tx, int *ty, int *nt, size_t *smem, int *bx, int *by)
{
    if (dtype == SWE_F32) {
        switch (variant) {
            case 1: shape_of<F32A>(tx, ty, nt, smem); *bx = F32A::BX; *by = F32A::BY; return true;
            case 2: shape_of<F32B>(tx, ty, nt, smem); *bx = F32B::BX; *by = F32B::BY; return true;
            case 3: shape_of<F32C>(tx, ty, nt, smem); *bx = F32C::BX; *by = F32C::BY; return true;
            case 4: shape_of<F32D>(tx, ty, nt, smem); *bx = F32D::BX; *by = F32D::BY; return true;
            case 5: shape_of<F32E>(tx, ty, nt, smem); *bx = F32E::BX; *by = F32E::BY; return true;
        }
    } else if (dtype == SWE_F64) {
        switch (variant) {
            case 1: shape_of<F64A>(tx, ty, nt, smem); *bx = F64A::BX; *by = F64A::BY; return true;
            case 2: shape_of<F64B>(tx, ty, nt, smem); *bx = F64B::BX; *by = F64B::BY; return true;
            case 3: shape_of<F64C>(tx, ty, nt, smem); *bx = F64C::BX; *by = F64C::BY; return true;
        }
    }
    return false;
}

template <class S, bool BED, class T>
static cudaError_t launch_step(const Maps4 &maps, const Out3<T> &out, int nx, int ny, const LwCoef<T> &k, int *err,
                               cudaStream_t s)
{
    constexpr size_t smem = BED ? S::SMEM_BED : S::SMEM;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(region_lw_kernel<S, T, BED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    if (attr != cudaSuccess) return attr;
    const dim3 grid((nx + S::TX - 1) / S::TX, (ny + S::TY - 1) / S::TY);
    region_lw_kernel<S, T, BED><<<grid, S::NT, smem, s>>>(maps, out, nx, ny, k, err);
    return cudaGetLastError();
}

template <class S, class T>
static cudaError_t launch_any(bool bed, const Maps4 &maps, const Out3<T> &out, int nx, int ny, const LwCoef<T> &k,
                              int *err, cudaStream_t s)
{
    return bed ? launch_step<S, true>(maps, out, nx, ny, k, err, s) : launch_step<S, false>(maps, out, nx, ny, k, err, s);
}

template <class T>
static LwCoef<T> lw_coef(double dx, double dy, double dt, double g)
{
    LwCoef<T> k;
    k.hx = (T)(0.5 * dt / dx);
    k.hy = (T)(0.5 * dt / dy);
    k.lx = (T)(dt / dx);
    k.ly = (T)(dt / dy);
    k.g = (T)g;
    return k;
}

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

static swe_status region_step(swe_region *r, const void *const in[3], const void *bed, void *const out[3], double dx,
                              double dy, double dt, double g, cudaStream_t s)
{
    for (double v : {dx, dy, dt, g})
        if (!(v > 0.0) || !std::isfinite(v)) return SWE_EINVAL;
    for (int f = 0; f < 3; ++f)
        if (!in[f] || !out[f] || !aligned16(in[f])) return SWE_EINVAL;
    const bool use_bed = bed != nullptr;
    if (use_bed && !aligned16(bed)) return SWE_EINVAL;
    int tx, ty, nt, bx, by;
    size_t smem;
    if (!variant_shape(r->dtype, r->variant, &tx, &ty, &nt, &smem, &bx, &by)) return SWE_EINVAL;
    Maps4 maps;
    for (int f = 0; f < (use_bed ? 4 : 3); ++f)
        if (!encode_plane_map(&maps.m[f], r->dtype, f < 3 ? in[f] : bed, r->nx + 2, r->ny + 2, r->pitch, bx, by))
            return SWE_ECUDA;
    cudaError_t e;
    if (r->dtype == SWE_F32) {
        const Out3<float> o{(float *)out[0], (float *)out[1], (float *)out[2], r->pitch};
        const LwCoef<float> k = lw_coef<float>(dx, dy, dt, g);
        switch (r->variant) {
            case 1: e = launch_any<F32A>(use_bed, maps, o, r->nx, r->ny, k, r->d_err, s); break;
            case 2: e = launch_any<F32B>(use_bed, maps, o, r->nx, r->ny, k, r->d_err, s); break;
            case 3: e = launch_any<F32C>(use_bed, maps, o, r->nx, r->ny, k, r->d_err, s); break;
            case 4: e = launch_any<F32D>(use_bed, maps, o, r->nx, r->ny, k, r->d_err, s); break;
            default: e = launch_any<F32E>(use_bed, maps, o, r->nx, r->ny, k, r->d_err, s); break;
        }
    } else {
        const Out3<double> o{(double *)out[0], (double *)out[1], (double *)out[2], r->pitch};
        const LwCoef<double> k = lw_coef<double>(dx, dy, dt, g);
        switch (r->variant) {
            case 1: e = launch_any<F64A>(use_bed, maps, o, r->nx, r->ny, k, r->d_err, s); break;
            case 2: e = launch_any<F64B>(use_bed, maps, o, r->nx, r->ny, k, r->d_err, s); break;
            default: e = launch_any<F64C>(use_bed, maps, o, r->nx, r->ny, k, r->d_err, s); break;
        }
    }
    if (e != cudaSuccess) return rst(e);
    ++r->launches;
    return SWE_OK;
}

static swe_status region_bound(swe_region *r, void *const st[3], const Sides &sd, cudaStream_t s)
{
    for (int f = 0; f < 3; ++f)
        if (!st[f]) return SWE_EINVAL;
    bool any = false;
    for (int side = 0; side < 4; ++side) {
        if (sd.kind[side] < 0 || sd.kind[side] > 2) return SWE_EINVAL;
        any = any || sd.kind[side] != 0;
    }
    if (!any) return SWE_OK;
    const int blocks = (int)std::min<long long>((std::max(r->nx, r->ny) + 255) / 256, 1024);
    const int ax = r->nx + 2, ay = r->ny + 2;
    if (r->dtype == SWE_F32) {
        region_walls_kernel<float><<<blocks, 256, 0, s>>>(array((float *)st[0], ax, ay, r->pitch),
                                                          array((float *)st[1], ax, ay, r->pitch),
                                                          array((float *)st[2], ax, ay, r->pitch), sd, r->d_err);
    } else {
        region_walls_kernel<double><<<blocks, 256, 0, s>>>(array((double *)st[0], ax, ay, r->pitch),
                                                           array((double *)st[1], ax, ay, r->pitch),
                                                           array((double *)st[2], ax, ay, r->pitch), sd, r->d_err);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return rst(e);
    ++r->launches;
    return SWE_OK;
}

static Sides sides_of_walls(int walls)
{
    Sides sd;
    for (int side = 0; side < 4; ++side) sd.kind[side] = (walls >> side) & 1;
    return sd;
}

extern "C" {

void swe_region_destroy(swe_region *r)
{
    if (!r) return;
    cudaDeviceSynchronize();
    cudaFree(r->d_err);
    delete r;
}

swe_status swe_region_create(int dtype, int nx, int ny, long long pitch, int variant, swe_region **out)
{
    if (!out) return SWE_EINVAL;
    *out = nullptr;
    if (dtype != SWE_F32 && dtype != SWE_F64) return SWE_EINVAL;
    const long long es = dtype == SWE_F64 ? 8 : 4;
    if (nx < 1 || ny < 1 || nx > 65536 || ny > 65536 || pitch < nx + 2 || (pitch * es) % 16 != 0) return SWE_EINVAL;
    if (variant == 0) variant = dtype == SWE_F32 ? 3 : 2;  // the fastest shapes measured at 8192^2
    int tx, ty, nt, bx, by;
    size_t smem;
    if (!variant_shape(dtype, variant, &tx, &ty, &nt, &smem, &bx, &by)) return SWE_EINVAL;
    swe_region *r = new (std::nothrow) swe_region();
    if (!r) return SWE_ENOMEM;
    r->dtype = dtype;
    r->nx = nx;
    r->ny = ny;
    r->pitch = pitch;
    r->variant = variant;
    swe_status st = rst(cudaMalloc(&r->d_err, sizeof(int)));
    if (st == SWE_OK) st = rst(cudaMemset(r->d_err, 0, sizeof(int)));
    if (st != SWE_OK) {
        swe_region_destroy(r);
        return st;
    }
    *out = r;
    return SWE_OK;
}

swe_status swe_region_step(swe_region *r, const void *const in[3], void *const out[3], double dx, double dy,
                           double dt, double g, void *stream)
{
    if (!r || !in || !out) return SWE_EINVAL;
    return region_step(r, in, nullptr, out, dx, dy, dt, g, static_cast<cudaStream_t>(stream));
}

swe_status swe_region_step_bed(swe_region *r, const void *const in[3], const void *bed, void *const out[3], double dx,
                               double dy, double dt, double g, void *stream)
{
    if (!r || !in || !out || !bed) return SWE_EINVAL;
    return region_step(r, in, bed, out, dx, dy, dt, g, static_cast<cudaStream_t>(stream));
}

swe_status swe_region_walls(swe_region *r, void *const state[3], int walls, void *stream)
{
    if (!r || !state || walls < 0 || walls > 15) return SWE_EINVAL;
    return region_bound(r, state, sides_of_walls(walls), static_cast<cudaStream_t>(stream));
}

swe_status swe_region_boundary(swe_region *r, void *const state[3], const int kinds[4], void *stream)
{
    if (!r || !state || !kinds) return SWE_EINVAL;
    Sides sd;
    for (int side = 0; side < 4; ++side) sd.kind[side] = kinds[side];
    return region_bound(r, state, sd, static_cast<cudaStream_t>(stream));
}

swe_status swe_region_run(swe_region *r, void *const a[3], void *const b[3], int n_steps, int walls, double dx,
                          double dy, double dt, double g, void *stream, int *result_in_b)
{
    if (walls < 0 || walls > 15) return SWE_EINVAL;
    const int kinds[4] = {walls & 1, (walls >> 1) & 1, (walls >> 2) & 1, (walls >> 3) & 1};
    return swe_region_run_bc(r, a, b, nullptr, n_steps, kinds, dx, dy, dt, g, stream, result_in_b);
}

swe_status swe_region_run_bc(swe_region *r, void *const a[3], void *const b[3], const void *bed, int n_steps,
                             const int kinds[4], double dx, double dy, double dt, double g, void *stream,
                             int *result_in_b)
{
    if (!r || !a || !b || !kinds || n_steps < 0) return SWE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Sides sd;
    for (int side = 0; side < 4; ++side) sd.kind[side] = kinds[side];
    void *const *cur = a, *const *nxt = b;
    for (int i = 0; i < n_steps; ++i) {
        swe_status st = region_bound(r, cur, sd, s);
        if (st == SWE_OK) st = region_step(r, (const void *const *)cur, bed, nxt, dx, dy, dt, g, s);
        if (st != SWE_OK) return st;
        std::swap(cur, nxt);
    }
    if (result_in_b) *result_in_b = (cur == b) ? 1 : 0;
    return SWE_OK;
}

swe_status swe_region_query(swe_region *r, int key, long long *value)
{
    if (!r || !value) return SWE_EINVAL;
    int tx, ty, nt, bx, by;
    size_t smem;
    variant_shape(r->dtype, r->variant, &tx, &ty, &nt, &smem, &bx, &by);
    switch (key) {
        case SWE_RQ_LAUNCHES: *value = r->launches; break;
        case SWE_RQ_TILE_X: *value = tx; break;
        case SWE_RQ_TILE_Y: *value = ty; break;
        case SWE_RQ_SMEM: *value = (long long)smem; break;
        case SWE_RQ_ERROR: {
            int word = 0;
            if (cudaMemcpy(&word, r->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SWE_ECUDA;
            *value = word;
            break;
        }
        default: return SWE_EINVAL;
    }
    return SWE_OK;
}

swe_status swe_selftest_div(const float *a, const float *b, float *out, int n, int which, void *stream)
{
    if (!a || !b || !out || n < 0 || which < 0 || which > 4 || (which == 2 && n % 2)) return SWE_EINVAL;
    if (n == 0) return SWE_OK;
    div_probe_kernel<<<std::min((n + 255) / 256, 4096), 256, 0, static_cast<cudaStream_t>(stream)>>>(a, b, out, n,
                                                                                                       which);
    return rst(cudaGetLastError());
}

swe_status swe_region_shapes(int nx, int ny, int *ext, int max_groups, int *n_groups)
{
    if (!ext || !n_groups || nx < 1 || ny < 1 || nx > 65536 || ny > 65536 || max_groups < 0) return SWE_EINVAL;
    const ShapeArray<double> C{nx + 2, ny + 2}, X{nx + 1, ny}, Y{nx, ny + 1};
    ShapeRun run;
    lw_statements<double>(run, C, C, C, C, C, C, X, X, X, Y, Y, Y, C, C, C, lw_coef<double>(1.0, 1.0, 0.1, 9.8));
    boundary_statements(run, C, C, C, sides_of_walls(15));
    *n_groups = run.n;
    for (int i = 0; i < std::min(run.n, std::min(max_groups, 16)); ++i) {
        ext[2 * i] = run.ext[i].x;
        ext[2 * i + 1] = run.ext[i].y;
    }
    return SWE_OK;
}

}  // extern "C"
