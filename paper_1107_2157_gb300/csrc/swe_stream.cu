// swe_stream.cu -- the single-grid streaming two-step kernel (two-step
// shapes 5..8): every warp takes one (strip, row range) segment of the grid
// through stream_segment (swe_stream.cuh).
#include <algorithm>
#include <mutex>
#include <type_traits>

#include "swe_stream.cuh"

namespace swe {

// The grid's NS strips are cut into row ranges: the interior strips
// 1 .. NS - 2 into K each, taken by warps gw < K (NS - 2) as strip
// 1 + gw % (NS - 2) of range gw / (NS - 2), so the warps running at the same
// time cover all strips of the same rows (DRAM sees whole grid rows, and a
// strip's overlap columns come from L2).  The first and last strips hold the
// walls and cost more per row (ghost columns); they are cut into Ke > K
// ranges, taken by the warps after those, so that their warps end with the
// others.  Keeping them together also keeps most CTAs on one copy of the row
// loop (0.4 % faster than interleaving them with the interior warps).
// Warp gw's segment (strip s, output rows [ya, yb)) of a grid of ns strips;
// false if the warp has none.
__device__ __forceinline__ bool segment_of(int gw, int ns, int ny, int K, int Ke, int &s, int &ya, int &yb)
{
    const int ne = ns == 1 ? 1 : 2;  // strips 0 and ns - 1
    const int ni = ns - ne;          // interior strips: 1 .. ns - 2
    int j, R;                        // row range, ranges of the strip
    if (gw < K * ni) {
        s = 1 + gw % ni;
        j = gw / ni;
        R = K;
    } else if (gw < K * ni + ne * Ke) {
        const int e = (gw - K * ni) / Ke;
        s = e == 0 ? 0 : ns - 1;
        j = (gw - K * ni) % Ke;
        R = Ke;
    } else {
        return false;
    }
    ya = (int)((long long)j * ny / R);
    yb = (int)((long long)(j + 1) * ny / R);
    return ya < yb;
}

template <int VP, int LO, int NO, int CR, int NSLOT, int WARPS, int MINB>
__global__ void __launch_bounds__(WARPS * 32, MINB)
    lw_stream_kernel(const __grid_constant__ CUtensorMap mH, const __grid_constant__ CUtensorMap mU,
                     const __grid_constant__ CUtensorMap mV, float *__restrict__ oH, float *__restrict__ oU,
                     float *__restrict__ oV, int nx, int ny, long long pitch, int K, int Ke, Coef<float> k,
                     int *err, const DevCoef<float> *kd)
{
    if (!take_dev_coef(kd, k)) return;
    using C = StreamCfg<VP, LO, NO, CR, NSLOT, WARPS>;
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int s, ya, yb;
    if (!segment_of(blockIdx.x * WARPS + warp, (nx + C::OUT - 1) / C::OUT, ny, K, Ke, s, ya, yb)) return;
    StreamWarp<VP, LO, NO, CR, NSLOT, WARPS> w;
    w.mH = &mH;
    w.mU = &mU;
    w.mV = &mV;
    w.ring = smem + (size_t)warp * C::WARP_BYTES;
    w.bars = reinterpret_cast<uint64_t *>(smem + WARPS * C::WARP_BYTES) + warp * NSLOT;
    w.phase = 0;
    w.err = err;
    if (lane == 0) {
        for (int i = 0; i < NSLOT; ++i) mbar_init(w.bars + i, 1);
        fence_mbar_init();
    }
    __syncwarp();
    const Coef2 k2 = coef2(k);
    const int xs = s * C::OUT;
    // the stored columns read input columns xs - 2 .. xs + OUT + 1: a strip
    // whose range reaches column -1 or nx fills that ghost column (held by
    // its overlap lane)
    const bool edge = xs == 0 || nx <= xs + C::OUT + 1;
    bool bad = false;  // the single-grid step reports no depth flags
    if (edge)
        (void)stream_segment<true>(w, oH, oU, oV, nx, ny, pitch, xs, ya, yb, k2, bad);
    else
        (void)stream_segment<false>(w, oH, oU, oV, nx, ny, pitch, xs, ya, yb, k2, bad);
}

// The same for scalar (FP64) lanes: two FP64 cells per lane, 60-column strips.
template <typename T, int LO, int NO, int CR, int NSLOT, int WARPS, int MINB>
__global__ void __launch_bounds__(WARPS * 32, MINB)
    lw_stream_s_kernel(const __grid_constant__ CUtensorMap mH, const __grid_constant__ CUtensorMap mU,
                       const __grid_constant__ CUtensorMap mV, T *__restrict__ oH, T *__restrict__ oU,
                       T *__restrict__ oV, int nx, int ny, long long pitch, int K, int Ke, Coef<T> k, int *err,
                       const DevCoef<T> *kd)
{
    if (!take_dev_coef(kd, k)) return;
    using C = StreamCfgS<T, LO, NO, CR, NSLOT, WARPS>;
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int s, ya, yb;
    if (!segment_of(blockIdx.x * WARPS + warp, (nx + C::OUT - 1) / C::OUT, ny, K, Ke, s, ya, yb)) return;
    StreamWarpS<C, CR, NSLOT> w;
    w.mH = &mH;
    w.mU = &mU;
    w.mV = &mV;
    w.ring = smem + (size_t)warp * C::WARP_BYTES;
    w.bars = reinterpret_cast<uint64_t *>(smem + WARPS * C::WARP_BYTES) + warp * NSLOT;
    w.phase = 0;
    w.err = err;
    if (lane == 0) {
        for (int i = 0; i < NSLOT; ++i) mbar_init(w.bars + i, 1);
        fence_mbar_init();
    }
    __syncwarp();
    const int xs = s * C::OUT;
    const bool edge = xs == 0 || nx <= xs + C::OUT + 1;
    bool bad = false;
    if (edge)
        (void)stream_segment_s<true, T, LO, NO, CR, NSLOT, WARPS>(w, oH, oU, oV, nx, ny, pitch, xs, ya, yb, k, bad);
    else
        (void)stream_segment_s<false, T, LO, NO, CR, NSLOT, WARPS>(w, oH, oU, oV, nx, ny, pitch, xs, ya, yb, k, bad);
}

// Launch shapes (two-step variants 5..8): pairs per lane, first stored
// lane, stored lanes, rows per TMA chunk, chunks per warp, warps per CTA,
// CTAs per SM the registers are capped for, and the wall strips' row ranges
// per interior strip's, in eighths.  Measured on GB300 at 8192^2 (ms per
// two-step launch, equal ranges for all strips): 5: 0.327, 6: 0.328, 7:
// 0.371, 8: 0.342; a 128-register cap for two pairs per lane spills 1.1 KB a
// thread.  The wall strips' warps are the last to finish with equal ranges:
// 1.125, 1.25 and 1.5 times as many ranges give shape 5 0.308, 0.307 and
// 0.305 ms; beyond 1.5 the resident warps no longer hold 26 ranges of every
// interior strip, and 25 give 0.316.  All strips on the wall code path (one
// copy of the row loop; the batched kernel's choice) give 0.329: here 67 of
// 69 strips hold no wall, and the ghost patch costs them more than the
// second copy of the loop does.
constexpr int kMinRows = 16;
template <int VARIANT>
struct StreamShape;
template <>
struct StreamShape<5> {  // the FP32 default: 120-column strips, two pairs per lane, two 4-row chunks
    static constexpr int VP = 2, LO = 1, NO = 30, CR = 4, SLOTS = 2, WARPS = 4, MINB = 3, EW8 = 12;
};
template <>
struct StreamShape<6> {  // as 5 with three chunks per warp
    static constexpr int VP = 2, LO = 1, NO = 30, CR = 4, SLOTS = 3, WARPS = 4, MINB = 3, EW8 = 12;
};
template <>
struct StreamShape<7> {  // 56-column strips (lanes 2..29), one pair per lane: 16 warps per SM
    static constexpr int VP = 1, LO = 2, NO = 28, CR = 4, SLOTS = 3, WARPS = 4, MINB = 4, EW8 = 12;
};
template <>
struct StreamShape<8> {  // as 5 with four 2-row chunks
    static constexpr int VP = 2, LO = 1, NO = 30, CR = 2, SLOTS = 4, WARPS = 4, MINB = 3, EW8 = 12;
};

template <int V>
using StreamCfgOf = StreamCfg<StreamShape<V>::VP, StreamShape<V>::LO, StreamShape<V>::NO, StreamShape<V>::CR,
                                StreamShape<V>::SLOTS, StreamShape<V>::WARPS>;

template <int V>
static void stream_box_t(int *bw, int *bh)
{
    *bw = StreamCfgOf<V>::BW;
    *bh = StreamCfgOf<V>::ROWS;
}

bool stream_box(int variant, int *bw, int *bh)
{
    switch (variant) {
        case 5: stream_box_t<5>(bw, bh); return true;
        case 6: stream_box_t<6>(bw, bh); return true;
        case 7: stream_box_t<7>(bw, bh); return true;
        case 8: stream_box_t<8>(bw, bh); return true;
        default: return false;
    }
}

// Resident CTAs of a streaming kernel on the device (its dynamic shared
// memory attribute set on the way).
template <typename K>
static cudaError_t stream_ctas(K kern, int warps, size_t smem, int *ctas)
{
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int dev = 0, sms = 0, per_sm = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem);
    *ctas = sms * std::max(per_sm, 1);
    return e;
}

// K row ranges of at least kMinRows rows for the interior strips and Ke =
// K EW8 / 8 (rounded up) for the wall strips, K as large as the resident
// warps (slots) allow; returns the warps to launch.
static int stream_ranges(int ns, int ny, int slots, int ew8, int *K_out, int *Ke_out)
{
    const int ne = ns == 1 ? 1 : 2;
    int K = std::max(1, std::min(slots / ns, (ny + kMinRows - 1) / kMinRows));
    auto walls = [&](int k) { return std::max(k, (k * ew8 + 7) / 8); };
    while (K > 1 && K * (ns - ne) + ne * walls(K) > slots) --K;
    *K_out = K;
    *Ke_out = walls(K);
    return K * (ns - ne) + ne * walls(K);
}

template <int V>
static cudaError_t launch_stream_t(const CUtensorMap *maps, void *out, size_t plane, int nx, int ny, long long pitch,
                                   double dx, double dy, double dt, double g, int *err, cudaStream_t s,
                                   const void *kd)
{
    using S = StreamShape<V>;
    using C = StreamCfgOf<V>;
    auto kern = lw_stream_kernel<S::VP, S::LO, S::NO, S::CR, S::SLOTS, S::WARPS, S::MINB>;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    static int ctas = 0;
    std::call_once(once, [&] { attr_err = stream_ctas(kern, S::WARPS, C::SMEM, &ctas); });
    if (attr_err != cudaSuccess) return attr_err;
    int K = 0, Ke = 0;
    const int warps = stream_ranges((nx + C::OUT - 1) / C::OUT, ny, ctas * S::WARPS, S::EW8, &K, &Ke);
    const int grid = (warps + S::WARPS - 1) / S::WARPS;
    float *b = static_cast<float *>(out);
    kern<<<grid, S::WARPS * 32, C::SMEM, s>>>(maps[0], maps[1], maps[2], b, b + plane, b + 2 * plane, nx, ny,
                                                   pitch, K, Ke, make_coef<float>(dx, dy, dt, g), err,
                                                   static_cast<const DevCoef<float> *>(kd));
    return cudaGetLastError();
}

// FP64 (two-step variants 5 and 6): two cells per lane, 60-column strips,
// two 4-row chunks per warp, 4 warps per CTA; registers uncapped (2 CTAs per
// SM) or capped for 3 CTAs per SM.
template <int MINB_>
struct StreamShapeD {
    static constexpr int LO = 1, NO = 30, CR = 4, SLOTS = 2, WARPS = 4, MINB = MINB_, EW8 = 12;
};
using StreamCfgD = StreamCfgS<double, 1, 30, 4, 2, 4>;

bool stream_box_d(int variant, int *bw, int *bh)
{
    if (variant != 5 && variant != 6) return false;
    *bw = StreamCfgD::BW;
    *bh = StreamCfgD::ROWS;
    return true;
}

template <int MINB>
static cudaError_t launch_stream_d_t(const CUtensorMap *maps, void *out, size_t plane, int nx, int ny,
                                     long long pitch, double dx, double dy, double dt, double g, int *err,
                                     cudaStream_t s, const void *kd)
{
    using S = StreamShapeD<MINB>;
    using C = StreamCfgD;
    auto kern = lw_stream_s_kernel<double, S::LO, S::NO, S::CR, S::SLOTS, S::WARPS, S::MINB>;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    static int ctas = 0;
    std::call_once(once, [&] { attr_err = stream_ctas(kern, S::WARPS, C::SMEM, &ctas); });
    if (attr_err != cudaSuccess) return attr_err;
    int K = 0, Ke = 0;
    const int warps = stream_ranges((nx + C::OUT - 1) / C::OUT, ny, ctas * S::WARPS, S::EW8, &K, &Ke);
    double *b = static_cast<double *>(out);
    kern<<<(warps + S::WARPS - 1) / S::WARPS, S::WARPS * 32, C::SMEM, s>>>(
        maps[0], maps[1], maps[2], b, b + plane, b + 2 * plane, nx, ny, pitch, K, Ke, make_coef<double>(dx, dy, dt, g),
        err, static_cast<const DevCoef<double> *>(kd));
    return cudaGetLastError();
}

cudaError_t launch_stream_d(int variant, const CUtensorMap *maps, void *out, size_t plane, int nx, int ny,
                            long long pitch, double dx, double dy, double dt, double g, int *err, cudaStream_t s,
                            const void *kd)
{
    if (variant == 6) return launch_stream_d_t<3>(maps, out, plane, nx, ny, pitch, dx, dy, dt, g, err, s, kd);
    return launch_stream_d_t<1>(maps, out, plane, nx, ny, pitch, dx, dy, dt, g, err, s, kd);
}

cudaError_t launch_stream(int variant, const CUtensorMap *maps, void *out, size_t plane, int nx, int ny,
                          long long pitch, double dx, double dy, double dt, double g, int *err, cudaStream_t s,
                          const void *kd)
{
    switch (variant) {
        case 5: return launch_stream_t<5>(maps, out, plane, nx, ny, pitch, dx, dy, dt, g, err, s, kd);
        case 6: return launch_stream_t<6>(maps, out, plane, nx, ny, pitch, dx, dy, dt, g, err, s, kd);
        case 7: return launch_stream_t<7>(maps, out, plane, nx, ny, pitch, dx, dy, dt, g, err, s, kd);
        case 8: return launch_stream_t<8>(maps, out, plane, nx, ny, pitch, dx, dy, dt, g, err, s, kd);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace swe
