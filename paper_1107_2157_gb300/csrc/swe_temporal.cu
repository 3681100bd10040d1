// swe_temporal.cu -- the two-step (temporally blocked) Lax-Wendroff kernel.
// Two steps of Sec. 3 per launch: the tile is staged with a two-cell halo,
// the intermediate state of the tile plus a one-cell ring is computed into
// shared memory, and the second step is taken from there.  Same face and
// update functions as the one-step kernel (swe_tile.cuh), hence the same bits.
#include <algorithm>
#include <mutex>

#include "swe_tile.cuh"

namespace swe {


// ---------------------------------------------------------------------------
// Two steps per launch (temporal blocking): each CTA takes tiles
// blockIdx.x, blockIdx.x + gridDim.x, ... in row-major tile order (one tile
// when the grid has a CTA per tile), stages a tile with a two-cell halo and
// runs the two phases of tb2_tile_compute (swe_tile.cuh); DRAM sees each
// cell read and written once per two steps.  Phase 2 reads only the
// intermediate box, so as soon as phase 1 is done a CTA with a next tile
// issues its TMA load into the input box, and the load runs under phase 2.
// ---------------------------------------------------------------------------
template <typename T, int NWARP, int RY>
__global__ void __launch_bounds__(NWARP * 32) lw_tb2_kernel(const __grid_constant__ CUtensorMap mH,
                                                            const __grid_constant__ CUtensorMap mU,
                                                            const __grid_constant__ CUtensorMap mV,
                                                            T *__restrict__ oH, T *__restrict__ oU,
                                                            T *__restrict__ oV, int nx, int ny, long long pitch,
                                                            Coef<T> k, int *err, const DevCoef<T> *kd)
{
    if (!take_dev_coef(kd, k)) return;
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
    const int tiles_x = (nx + C::TX - 1) / C::TX;
    const int ntiles = tiles_x * ((ny + C::TY - 1) / C::TY);
    auto load = [&](int tile) {
        const int x0 = (tile % tiles_x) * C::TX, y0 = (tile / tiles_x) * C::TY;
        mbar_arrive_expect_tx(bar, (uint32_t)(3 * B::IN_BYTES));
        tma_load_2d(iH, &mH, bar, x0 - C::AX, y0 - 2);
        tma_load_2d(iU, &mU, bar, x0 - C::AX, y0 - 2);
        tma_load_2d(iV, &mV, bar, x0 - C::AX, y0 - 2);
    };
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        if ((int)blockIdx.x < ntiles) load(blockIdx.x);
    }
    __syncthreads();
    uint32_t phase = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, phase ^= 1u) {
        const int x0 = (tile % tiles_x) * C::TX, y0 = (tile / tiles_x) * C::TY;
        if (!__syncthreads_and(mbar_wait_bounded(bar, phase, err))) return;
        tb2_phase1<T, NWARP, RY>(iH, iU, iV, mH_, mU_, mV_, nx, ny, x0, y0, k);
        __syncthreads();
        // the input box is free: fetch the next tile while phase 2 runs
        const int next = tile + gridDim.x;
        if (threadIdx.x == 0 && next < ntiles) {
            fence_proxy_async_smem();
            load(next);
        }
        tb2_phase2<T, NWARP, RY>(mH_, mU_, mV_, oH, oU, oV, nx, ny, pitch, x0, y0, k);
        __syncthreads();  // the intermediate box is rewritten by the next tile's phase 1
    }
}

// Two-step kernel shapes (warps x rows per warp): 0: 4x8 (tile 128x32,
// ~112 KB smem), 1: 8x4 (128x32, 256 threads), 2: 4x4 (128x16, ~61 KB),
// 3: 8x2 (128x16, 256 threads), all with one CTA per tile; 4: 8x4 with
// persistent CTAs (as many as fit on the device, each prefetching its next
// tile under phase 2).  5..8 (FP32; 5 and 6 also FP64): warps streaming up
// column strips (swe_stream.cu).
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

bool stream_box(int variant, int *bw, int *bh);
bool stream_box_d(int variant, int *bw, int *bh);
cudaError_t launch_stream_d(int variant, const CUtensorMap *maps, void *out, size_t plane, int nx, int ny,
                            long long pitch, double dx, double dy, double dt, double g, int *err, cudaStream_t s,
                            const void *kd);
cudaError_t launch_stream(int variant, const CUtensorMap *maps, void *out, size_t plane, int nx, int ny,
                          long long pitch, double dx, double dy, double dt, double g, int *err, cudaStream_t s,
                          const void *kd);

void tb2_box(int dtype, int variant, int *bw, int *bh)
{
    const bool d = dtype == SWE_F64;
    if (!d && stream_box(variant, bw, bh)) return;
    if (d && stream_box_d(variant, bw, bh)) return;
    switch (variant) {
        case 1:
        case 4: d ? tb2_box_t<double, TbShape<double, 8, 4>>(bw, bh) : tb2_box_t<float, TbShape<float, 8, 4>>(bw, bh); break;
        case 2: d ? tb2_box_t<double, TbShape<double, 4, 4>>(bw, bh) : tb2_box_t<float, TbShape<float, 4, 4>>(bw, bh); break;
        case 3: d ? tb2_box_t<double, TbShape<double, 8, 2>>(bw, bh) : tb2_box_t<float, TbShape<float, 8, 2>>(bw, bh); break;
        default: d ? tb2_box_t<double, TbShape<double, 4, 8>>(bw, bh) : tb2_box_t<float, TbShape<float, 4, 8>>(bw, bh); break;
    }
}

template <typename T, typename S>
static cudaError_t launch_tb2_t(const CUtensorMap *maps, void *out, size_t plane, int nx, int ny, long long pitch,
                                double dx, double dy, double dt, double g, int *err, cudaStream_t s, bool persistent,
                                const void *kd)
{
    using Cfg = typename S::Cfg;
    auto kern = lw_tb2_kernel<T, S::WARPS, S::ROWS>;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [&] {
        attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
    });
    if (attr_err != cudaSuccess) return attr_err;
    static int ctas = 0;  // CTAs of this shape resident on the device: the persistent grid
    if (!ctas) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, S::WARPS * 32, Cfg::SMEM);
        if (e != cudaSuccess) return e;
        ctas = sms * (per_sm > 0 ? per_sm : 1);
    }
    T *b = static_cast<T *>(out);
    const long long tiles =
        (long long)((nx + Cfg::C::TX - 1) / Cfg::C::TX) * (long long)((ny + Cfg::C::TY - 1) / Cfg::C::TY);
    const int grid = (int)(persistent ? std::min<long long>(tiles, ctas) : tiles);
    kern<<<grid, S::WARPS * 32, Cfg::SMEM, s>>>(maps[0], maps[1], maps[2], b, b + plane, b + 2 * plane, nx, ny,
                                                pitch, make_coef<T>(dx, dy, dt, g), err,
                                                static_cast<const DevCoef<T> *>(kd));
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_tb2_v(int variant, const CUtensorMap *maps, void *out, size_t plane, int nx, int ny,
                                long long pitch, double dx, double dy, double dt, double g, int *err, cudaStream_t s,
                                const void *kd)
{
    switch (variant) {
        case 1: return launch_tb2_t<T, TbShape<T, 8, 4>>(maps, out, plane, nx, ny, pitch, dx, dy, dt, g, err, s, false, kd);
        case 2: return launch_tb2_t<T, TbShape<T, 4, 4>>(maps, out, plane, nx, ny, pitch, dx, dy, dt, g, err, s, false, kd);
        case 3: return launch_tb2_t<T, TbShape<T, 8, 2>>(maps, out, plane, nx, ny, pitch, dx, dy, dt, g, err, s, false, kd);
        case 4: return launch_tb2_t<T, TbShape<T, 8, 4>>(maps, out, plane, nx, ny, pitch, dx, dy, dt, g, err, s, true, kd);
        default: return launch_tb2_t<T, TbShape<T, 4, 8>>(maps, out, plane, nx, ny, pitch, dx, dy, dt, g, err, s, false, kd);
    }
}

cudaError_t launch_tb2(int dtype, int variant, const CUtensorMap *maps_in, void *out, size_t plane, int nx, int ny,
                       long long pitch, double dx, double dy, double dt, double g, int *err, cudaStream_t s,
                       const void *kd)
{
    if (dtype == SWE_F64) {
        if (variant == 5 || variant == 6)
            return launch_stream_d(variant, maps_in, out, plane, nx, ny, pitch, dx, dy, dt, g, err, s, kd);
        return launch_tb2_v<double>(variant, maps_in, out, plane, nx, ny, pitch, dx, dy, dt, g, err, s, kd);
    }
    if (variant >= 5) return launch_stream(variant, maps_in, out, plane, nx, ny, pitch, dx, dy, dt, g, err, s, kd);
    return launch_tb2_v<float>(variant, maps_in, out, plane, nx, ny, pitch, dx, dy, dt, g, err, s, kd);
}

}  // namespace swe
