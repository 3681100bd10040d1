// swe_step.cu -- single-grid Lax-Wendroff step kernels (Sec. 3 step
// equations; Sec. 3.1 statements), FP32 and FP64.
//
//  * lw_naive_kernel: one thread per cell, the five-point neighbourhood read
//    straight from global memory.  The plain GPU form of the scheme.
//  * lw_tiled_kernel: one CTA per output tile.  A single thread issues three
//    TMA loads (H, U, V) of the tile plus its halo into shared memory, the
//    CTA waits on an mbarrier, then each thread owns a 16-byte column vector
//    (4 FP32 or 2 FP64 cells) and marches down RY rows, keeping the y-face
//    flux of the row below in registers so every y-face is computed once.
//    Results are stored with 16-byte vector stores.
//
// Reflective walls (the ghost rule) are applied where the neighbours are
// formed: a neighbour outside the grid is the mirror of the cell next to the
// wall, with the wall-normal momentum negated.  No ghost cells are stored.
#include <mutex>

#include "swe_tile.cuh"

namespace swe {


// ---------------------------------------------------------------------------
// Naive kernel
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) lw_naive_kernel(const T *__restrict__ H, const T *__restrict__ U,
                                                       const T *__restrict__ V, T *__restrict__ oH,
                                                       T *__restrict__ oU, T *__restrict__ oV, int nx, int ny,
                                                       long long pitch, Coef<T> k, const DevCoef<T> *kd)
{
    if (!take_dev_coef(kd, k)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= nx || j >= ny) return;
    auto cell = [&](int ii, int jj) {
        const size_t o = (size_t)jj * (size_t)pitch + (size_t)ii;
        return make_cell<T>(H[o], U[o], V[o], k.hg);
    };
    const CellQ<T> c = cell(i, j);
    const CellQ<T> l = i > 0 ? cell(i - 1, j) : mirror_x(c);
    const CellQ<T> r = i < nx - 1 ? cell(i + 1, j) : mirror_x(c);
    const CellQ<T> d = j > 0 ? cell(i, j - 1) : mirror_y(c);
    const CellQ<T> u = j < ny - 1 ? cell(i, j + 1) : mirror_y(c);
    const Flux3<T> Fl = xface_flux(l, c, k), Fr = xface_flux(c, r, k);
    const Flux3<T> Gd = yface_flux(d, c, k), Gu = yface_flux(c, u, k);
    T h = c.h, hu = c.u, hv = c.v;
    lw_update(h, hu, hv, Fl, Fr, Gd, Gu, k);
    const size_t o = (size_t)j * (size_t)pitch + (size_t)i;
    oH[o] = h;
    oU[o] = hu;
    oV[o] = hv;
}

// ---------------------------------------------------------------------------
// Tiled TMA kernel
// ---------------------------------------------------------------------------
template <typename T, int NWARP, int RY>
__global__ void __launch_bounds__(NWARP * 32) lw_tiled_kernel(const __grid_constant__ CUtensorMap mH,
                                                              const __grid_constant__ CUtensorMap mU,
                                                              const __grid_constant__ CUtensorMap mV,
                                                              T *__restrict__ oH, T *__restrict__ oU,
                                                              T *__restrict__ oV, int nx, int ny,
                                                              long long pitch, Coef<T> k, int *err,
                                                              const DevCoef<T> *kd)
{
    if (!take_dev_coef(kd, k)) return;
    using C = TiledCfg<T, NWARP, RY>;
    extern __shared__ __align__(128) unsigned char smem[];
    T *sH = reinterpret_cast<T *>(smem);
    T *sU = reinterpret_cast<T *>(smem + C::BOX_STRIDE);
    T *sV = reinterpret_cast<T *>(smem + 2 * C::BOX_STRIDE);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 3 * C::BOX_STRIDE);
    const int x0 = blockIdx.x * C::TX;
    const int y0 = blockIdx.y * C::TY;
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        mbar_arrive_expect_tx(bar, (uint32_t)(3 * C::BOX_BYTES));
        tma_load_2d(sH, &mH, bar, x0 - C::AX, y0 - 1);
        tma_load_2d(sU, &mU, bar, x0 - C::AX, y0 - 1);
        tma_load_2d(sV, &mV, bar, x0 - C::AX, y0 - 1);
    }
    __syncthreads();
    if (!mbar_wait_bounded(bar, 0, err)) return;
    const bool xedge = (x0 == 0) || (x0 + C::TX >= nx);
    if (xedge)
        tiled_compute<T, NWARP, RY, true>(sH, sU, sV, oH, oU, oV, nx, ny, pitch, x0, y0, k);
    else
        tiled_compute<T, NWARP, RY, false>(sH, sU, sV, oH, oU, oV, nx, ny, pitch, x0, y0, k);
}

// Tile shapes of the tiled kernel: 4 warps x 8 rows; 128x32 FP32 cells or
// 64x32 FP64 cells per CTA, ~54 KB of shared memory (4 CTAs per SM).
constexpr int kTiledWarps = 4;
constexpr int kTiledRows = 8;
using CfgF = TiledCfg<float, kTiledWarps, kTiledRows>;
using CfgD = TiledCfg<double, kTiledWarps, kTiledRows>;

StepGeom tiled_geom(int dtype)
{
    if (dtype == SWE_F64) return StepGeom{CfgD::TX, CfgD::TY, kTiledWarps * 32, CfgD::SMEM};
    return StepGeom{CfgF::TX, CfgF::TY, kTiledWarps * 32, CfgF::SMEM};
}

// Box (BW, BH) the tiled kernel expects its tensor maps to carry.
void tiled_box(int dtype, int *bw, int *bh)
{
    if (dtype == SWE_F64) {
        *bw = CfgD::BW;
        *bh = CfgD::BH;
    } else {
        *bw = CfgF::BW;
        *bh = CfgF::BH;
    }
}

cudaError_t launch_naive(int dtype, const void *in, void *out, size_t plane, int nx, int ny, long long pitch,
                         double dx, double dy, double dt, double g, cudaStream_t s, const void *kd)
{
    const dim3 block(64, 4);
    const dim3 grid((nx + 63) / 64, (ny + 3) / 4);
    if (dtype == SWE_F64) {
        const double *a = static_cast<const double *>(in);
        double *b = static_cast<double *>(out);
        lw_naive_kernel<double><<<grid, block, 0, s>>>(a, a + plane, a + 2 * plane, b, b + plane, b + 2 * plane, nx,
                                                       ny, pitch, make_coef<double>(dx, dy, dt, g),
                                                       static_cast<const DevCoef<double> *>(kd));
    } else {
        const float *a = static_cast<const float *>(in);
        float *b = static_cast<float *>(out);
        lw_naive_kernel<float><<<grid, block, 0, s>>>(a, a + plane, a + 2 * plane, b, b + plane, b + 2 * plane, nx,
                                                      ny, pitch, make_coef<float>(dx, dy, dt, g),
                                                      static_cast<const DevCoef<float> *>(kd));
    }
    return cudaGetLastError();
}

template <typename T, typename Cfg>
static cudaError_t launch_tiled_t(const CUtensorMap *maps, void *out, size_t plane, int nx, int ny,
                                  long long pitch, double dx, double dy, double dt, double g, int *err,
                                  cudaStream_t s, const void *kd)
{
    auto kern = lw_tiled_kernel<T, kTiledWarps, kTiledRows>;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [&] {
        attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
    });
    if (attr_err != cudaSuccess) return attr_err;
    T *b = static_cast<T *>(out);
    const dim3 grid((nx + Cfg::TX - 1) / Cfg::TX, (ny + Cfg::TY - 1) / Cfg::TY);
    kern<<<grid, kTiledWarps * 32, Cfg::SMEM, s>>>(maps[0], maps[1], maps[2], b, b + plane, b + 2 * plane, nx, ny,
                                                   pitch, make_coef<T>(dx, dy, dt, g), err,
                                                   static_cast<const DevCoef<T> *>(kd));
    return cudaGetLastError();
}

cudaError_t launch_tiled(int dtype, const CUtensorMap *maps_in, void *out, size_t plane, int nx, int ny,
                         long long pitch, double dx, double dy, double dt, double g, int *err, cudaStream_t s,
                         const void *kd)
{
    if (dtype == SWE_F64)
        return launch_tiled_t<double, CfgD>(maps_in, out, plane, nx, ny, pitch, dx, dy, dt, g, err, s, kd);
    return launch_tiled_t<float, CfgF>(maps_in, out, plane, nx, ny, pitch, dx, dy, dt, g, err, s, kd);
}

}  // namespace swe
