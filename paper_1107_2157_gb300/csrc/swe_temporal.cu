// swe_temporal.cu -- the two-step (temporally blocked) Lax-Wendroff kernel.
// Two steps of Sec. 3 per launch: the tile is staged with a two-cell halo,
// the intermediate state of the tile plus a one-cell ring is computed into
// shared memory, and the second step is taken from there.  Same face and
// update functions as the one-step kernel (swe_tile.cuh), hence the same bits.
#include <mutex>

#include "swe_tile.cuh"

namespace swe {

template <typename T>
static Coef<T> make_coef(double dx, double dy, double dt, double g)
{
    Coef<T> k;
    k.hx = (T)(0.5 * dt / dx);
    k.hy = (T)(0.5 * dt / dy);
    k.lx = (T)(dt / dx);
    k.ly = (T)(dt / dy);
    k.hg = (T)(0.5 * g);
    return k;
}

// ---------------------------------------------------------------------------
// Two steps per launch (temporal blocking): one CTA per tile stages the
// tile with a two-cell halo and runs tb2_tile_compute (swe_tile.cuh); DRAM
// sees each cell read and written once per two steps.
// ---------------------------------------------------------------------------
template <typename T, int NWARP, int RY>
__global__ void __launch_bounds__(NWARP * 32) lw_tb2_kernel(const __grid_constant__ CUtensorMap mH,
                                                            const __grid_constant__ CUtensorMap mU,
                                                            const __grid_constant__ CUtensorMap mV,
                                                            T *__restrict__ oH, T *__restrict__ oU,
                                                            T *__restrict__ oV, int nx, int ny, long long pitch,
                                                            Coef<T> k, int *err)
{
    using B = Tb2Cfg<T, NWARP, RY>;
    using C = typename B::C;
    extern __shared__ __align__(128) unsigned char smem[];
    T *iH = reinterpret_cast<T *>(smem);
    T *iU = reinterpret_cast<T *>(smem + B::IN_STRIDE);
    T *iV = reinterpret_cast<T *>(smem + 2 * B::IN_STRIDE);
    T *mH_ = reinterpret_cast<T *>(smem + 3 * B::IN_STRIDE);
    T *mU_ = reinterpret_cast<T *>(smem + 3 * B::IN_STRIDE + C::BOX_STRIDE);
    T *mV_ = reinterpret_cast<T *>(smem + 3 * B::IN_STRIDE + 2 * C::BOX_STRIDE);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 3 * B::IN_STRIDE + 3 * C::BOX_STRIDE);
    const int x0 = blockIdx.x * C::TX;
    const int y0 = blockIdx.y * C::TY;
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        mbar_arrive_expect_tx(bar, (uint32_t)(3 * B::IN_BYTES));
        tma_load_2d(iH, &mH, bar, x0 - C::AX, y0 - 2);
        tma_load_2d(iU, &mU, bar, x0 - C::AX, y0 - 2);
        tma_load_2d(iV, &mV, bar, x0 - C::AX, y0 - 2);
    }
    __syncthreads();
    if (!__syncthreads_and(mbar_wait_bounded(bar, 0, err))) return;
    tb2_tile_compute<T, NWARP, RY>(iH, iU, iV, mH_, mU_, mV_, oH, oU, oV, nx, ny, pitch, x0, y0, k);
}

// Two-step kernel shapes (warps x rows per warp): 0: 4x8 (tile 128x32,
// ~112 KB smem), 1: 8x4 (128x32, 256 threads), 2: 4x4 (128x16, ~61 KB),
// 3: 8x2 (128x16, 256 threads).
template <typename T, int W, int R>
struct TbShape {
    using Cfg = Tb2Cfg<T, W, R>;
    static constexpr int WARPS = W, ROWS = R;
};

template <typename T, typename S>
static void tb2_box_t(int *bw, int *bh)
{
    *bw = S::Cfg::C::BW;
    *bh = S::Cfg::BH_IN;
}

void tb2_box(int dtype, int variant, int *bw, int *bh)
{
    const bool d = dtype == SWE_F64;
    switch (variant) {
        case 1: d ? tb2_box_t<double, TbShape<double, 8, 4>>(bw, bh) : tb2_box_t<float, TbShape<float, 8, 4>>(bw, bh); break;
        case 2: d ? tb2_box_t<double, TbShape<double, 4, 4>>(bw, bh) : tb2_box_t<float, TbShape<float, 4, 4>>(bw, bh); break;
        case 3: d ? tb2_box_t<double, TbShape<double, 8, 2>>(bw, bh) : tb2_box_t<float, TbShape<float, 8, 2>>(bw, bh); break;
        default: d ? tb2_box_t<double, TbShape<double, 4, 8>>(bw, bh) : tb2_box_t<float, TbShape<float, 4, 8>>(bw, bh); break;
    }
}

template <typename T, typename S>
static cudaError_t launch_tb2_t(const CUtensorMap *maps, void *out, size_t plane, int nx, int ny, long long pitch,
                                double dx, double dy, double dt, double g, int *err, cudaStream_t s)
{
    using Cfg = typename S::Cfg;
    auto kern = lw_tb2_kernel<T, S::WARPS, S::ROWS>;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [&] {
        attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
    });
    if (attr_err != cudaSuccess) return attr_err;
    T *b = static_cast<T *>(out);
    const dim3 grid((nx + Cfg::C::TX - 1) / Cfg::C::TX, (ny + Cfg::C::TY - 1) / Cfg::C::TY);
    kern<<<grid, S::WARPS * 32, Cfg::SMEM, s>>>(maps[0], maps[1], maps[2], b, b + plane, b + 2 * plane, nx, ny,
                                                pitch, make_coef<T>(dx, dy, dt, g), err);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_tb2_v(int variant, const CUtensorMap *maps, void *out, size_t plane, int nx, int ny,
                                long long pitch, double dx, double dy, double dt, double g, int *err, cudaStream_t s)
{
    switch (variant) {
        case 1: return launch_tb2_t<T, TbShape<T, 8, 4>>(maps, out, plane, nx, ny, pitch, dx, dy, dt, g, err, s);
        case 2: return launch_tb2_t<T, TbShape<T, 4, 4>>(maps, out, plane, nx, ny, pitch, dx, dy, dt, g, err, s);
        case 3: return launch_tb2_t<T, TbShape<T, 8, 2>>(maps, out, plane, nx, ny, pitch, dx, dy, dt, g, err, s);
        default: return launch_tb2_t<T, TbShape<T, 4, 8>>(maps, out, plane, nx, ny, pitch, dx, dy, dt, g, err, s);
    }
}

cudaError_t launch_tb2(int dtype, int variant, const CUtensorMap *maps_in, void *out, size_t plane, int nx, int ny,
                       long long pitch, double dx, double dy, double dt, double g, int *err, cudaStream_t s)
{
    if (dtype == SWE_F64)
        return launch_tb2_v<double>(variant, maps_in, out, plane, nx, ny, pitch, dx, dy, dt, g, err, s);
    return launch_tb2_v<float>(variant, maps_in, out, plane, nx, ny, pitch, dx, dy, dt, g, err, s);
}

}  // namespace swe
