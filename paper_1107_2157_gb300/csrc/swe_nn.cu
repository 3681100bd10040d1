// swe_nn.cu -- the learned coarse-grid corrector: a 3 -> 32 -> 32 -> 3
// network of zero-padded 3x3 convolutions with GELU (no counterpart in the
// paper; it corrects the coarse Lax-Wendroff step of Sec. 3), trained and
// run by this file's kernels.
//
// Activation layout ("row-chunked"): bf16 A[n][y][c][x][8], channel = 8c+k,
// so one image row holds CH strips of W pixels x 16 bytes.  A 5D TMA box
// {8 ch, 130 px, CH, R+2 rows, 1 image} of that tensor lands in shared memory
// as [R+2][CH][130][8]: for every output row and 3x3 tap the MMA's A operand
// (128 consecutive pixels x 16 channels) is then a K-major, unswizzled
// matrix at a shifted shared-memory address -- core matrices of 8 pixels x
// 16 bytes, 128 bytes apart along M and one channel strip (2080 bytes) apart
// along K.  No im2col copy is made; zero padding comes from the TMA's
// out-of-range fill.
//
// conv3x3_tc_kernel: one CTA computes 128 x R output pixels of one image.
// One thread issues R x 9 x (CH/2) tcgen05.mma (M=128, N=COUT, K=16, BF16
// in, FP32 accumulate in TMEM), one TMEM accumulator of COUT columns per
// output row; the epilogue reads TMEM with tcgen05.ld and applies bias,
// GELU, the loss or the GELU derivative.  Forward layers and the input
// gradients (transposed convolutions with flipped, transposed weights) all
// use this kernel.  Weight gradients run on the tensor cores too
// (wgrad_tc_kernel, pixels as the MMA's K).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "swe_gelu.cuh"
#include "swe_tc.cuh"
#include "swe_views.cuh"

namespace swe {

constexpr int kTileX = 128;                // output pixels per tile row (the MMA's M)
constexpr int kHaloX = kTileX + 2;         // 130
constexpr int kPixB = 16;                  // bytes per pixel strip (8 bf16)
constexpr int kStripB = kHaloX * kPixB;    // 2080: one channel strip of the halo tile
#ifndef SWE_CONV_ROWS
#define SWE_CONV_ROWS 4
#endif
constexpr int kConvRows = SWE_CONV_ROWS;   // output rows per CTA

__host__ __device__ constexpr size_t al128(size_t x) { return (x + 127) / 128 * 128; }
__host__ __device__ constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
__host__ __device__ constexpr uint32_t pow2_at_least(uint32_t x, uint32_t p = 32)
{
    return p >= x ? p : pow2_at_least(x, p * 2);
}

template <int CH, int COUT, int R>
struct ConvCfg {
    static constexpr int NKS = CH / 2;    // K steps of 16 channels per tap
    static constexpr int NC = COUT / 8;   // core matrices along N
    static constexpr size_t A_BYTES = (size_t)CH * (R + 2) * kStripB;
    static constexpr size_t B_BLOCK = (size_t)2 * NC * 128;  // one (tap, K step): 16 x COUT
    static constexpr size_t B_BYTES = (size_t)9 * NKS * B_BLOCK;
    static constexpr size_t OFF_B = al128(A_BYTES);
    static constexpr size_t OFF_BAR = al128(OFF_B + B_BYTES);
    static constexpr size_t USED = OFF_BAR + 64;
    static constexpr size_t SMEM = USED + 128;
    static constexpr uint32_t TMEM_COLS = pow2_at_least((uint32_t)(R * COUT));
};

enum { EPI_GELU = 0, EPI_GELU_BWD = 1, EPI_LOSS = 2, EPI_RESID = 3, EPI_APPLY = 4 };

struct EpiArgs {
    const float *bias;        // COUT floats (EPI_GELU, EPI_LOSS, EPI_RESID)
    bf16 *out;                // row-chunked output, COUT/8 strips (a, dz or dr)
    bf16 *zout;               // EPI_GELU: pre-activation (may be null)
    const bf16 *zin;          // EPI_GELU_BWD: pre-activation of the layer being differentiated
    const float *target;      // EPI_LOSS: FP32 [n][3][H][W] normalised targets
    float *resid;             // EPI_RESID: FP32 [n][3][H][W] output (scaled); EPI_LOSS: optional r
    float oscale[3];          // EPI_RESID / EPI_APPLY: per-channel output scale
    float *state;             // EPI_APPLY: state planes the scaled residual is added to
    long long st_img, st_plane, st_pitch;  // EPI_APPLY: their strides (floats)
    double *hsum;             // EPI_APPLY: per-image sum of the h correction (may be null)
    float loss_scale;         // EPI_LOSS: d loss / d r factor (2 / count)
    const float *img_w;       // EPI_LOSS: per-image loss weight (null = 1)
    double *loss_accum;       // EPI_LOSS: sum of squared errors
};

__device__ __forceinline__ void tma_load_5d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1, int c2,
                                            int c3, int c4)
{
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_addr(bar))
        : "memory");
}

// Evaluates erf (which = 0), gelu (1) or gelu' (2) of n values (self-test).
__global__ void gelu_probe_kernel(const float *__restrict__ z, float *__restrict__ out, int n, int which)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float g;
        out[i] = which == 0 ? erf_as(z[i], g) : (which == 1 ? gelu_f(z[i]) : gelu_grad_f(z[i]));
    }
}

__device__ __forceinline__ size_t rc_index(int n, int y, int c, int x, int H, int W, int CHO)
{
    return ((((size_t)n * H + y) * CHO + c) * W + x) * 8;
}

template <int CH, int COUT, int R, int EPI>
__global__ void __launch_bounds__(128) conv3x3_tc_kernel(const __grid_constant__ CUtensorMap mIn,
                                                         const bf16 *__restrict__ wimg, EpiArgs ea, int W, int H,
                                                         int *err)
{
    using C = ConvCfg<CH, COUT, R>;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *sA = smem;
    unsigned char *sB = smem + C::OFF_B;
    uint64_t *bar_tma = reinterpret_cast<uint64_t *>(smem + C::OFF_BAR);
    uint64_t *bar_mma = bar_tma + 1;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar_tma + 2);
    const int x0 = blockIdx.x * kTileX, y0 = blockIdx.y * R, n = blockIdx.z;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        mbar_init(bar_tma, 1);
        mbar_init(bar_mma, 1);
        fence_mbar_init();
        mbar_arrive_expect_tx(bar_tma, (uint32_t)C::A_BYTES);
        tma_load_5d(sA, &mIn, bar_tma, 0, x0 - 1, 0, y0 - 1, n);
    }
    {  // weights (already in the B-operand byte order) -> shared memory
        const uint4 *src = reinterpret_cast<const uint4 *>(wimg);
        uint4 *dst = reinterpret_cast<uint4 *>(sB);
        for (int i = tid; i < (int)(C::B_BYTES / 16); i += 128) dst[i] = __ldg(src + i);
    }
    fence_proxy_async_smem();  // make them visible to the tensor core's reads
    if (warp == 0) tc::tmem_alloc(tslot, C::TMEM_COLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;

    // Epilogue operands that do not depend on the MMA are fetched now, so
    // their latency overlaps the loads and the MMAs.
    const int px = x0 + warp * 32 + lane;
    constexpr int PF = (EPI == EPI_GELU_BWD) ? COUT / 8 : ((EPI == EPI_LOSS || EPI == EPI_APPLY) ? 3 : 1);
    uint4 zpre[R][EPI == EPI_GELU_BWD ? PF : 1];
    float fpre[R][(EPI == EPI_LOSS || EPI == EPI_APPLY) ? 3 : 1];
    if (px < W) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int y = y0 + r;
            if (y >= H) break;
            if constexpr (EPI == EPI_GELU_BWD) {
#pragma unroll
                for (int c = 0; c < PF; ++c)
                    zpre[r][c] = *reinterpret_cast<const uint4 *>(ea.zin + rc_index(n, y, c, px, H, W, PF));
            } else if constexpr (EPI == EPI_LOSS) {
                const size_t plane = (size_t)H * W;
                const size_t po = ((size_t)n * 3) * plane + (size_t)y * W + px;
#pragma unroll
                for (int c = 0; c < 3; ++c) fpre[r][c] = __ldg(ea.target + po + c * plane);
            } else if constexpr (EPI == EPI_APPLY) {
                const float *st = ea.state + n * ea.st_img + (long long)y * ea.st_pitch + px;
#pragma unroll
                for (int c = 0; c < 3; ++c) fpre[r][c] = st[c * ea.st_plane];
            }
        }
    }

    bool ok = __syncthreads_and(mbar_wait_bounded(bar_tma, 0, err));
    if (ok && tid == 0) {
        constexpr uint32_t idesc = tc::idesc_bf16(128, COUT);
#pragma unroll 1
        for (int r = 0; r < R; ++r) {
#pragma unroll 1
            for (int t = 0; t < 9; ++t) {
                const int ky = t / 3, kx = t % 3;
#pragma unroll
                for (int s = 0; s < C::NKS; ++s) {
                    const unsigned char *a = sA + ((size_t)(r + ky) * CH + 2 * s) * kStripB + kx * kPixB;
                    const unsigned char *b = sB + (size_t)(t * C::NKS + s) * C::B_BLOCK;
                    tc::mma_bf16(tmem + (uint32_t)(r * COUT), tc::smem_desc(a, kStripB, 128),
                                 tc::smem_desc(b, C::NC * 128, 128), idesc, (t | s) != 0);
                }
            }
        }
        tc::commit(bar_mma);
    }
    if (ok) ok = mbar_wait_bounded(bar_mma, 0, err);
    ok = __syncthreads_and(ok);
    tc::fence_after_sync();

    if (ok) {
        const int x = x0 + warp * 32 + lane;
        const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16);
        double lsum = 0.0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int y = y0 + r;
            float v[COUT];
            if constexpr (COUT == 32)
                tc::ld_x32(tbase + (uint32_t)(r * COUT), v);
            else
                tc::ld_x16(tbase + (uint32_t)(r * COUT), v);
            if (x >= W || y >= H) continue;
            if constexpr (EPI == EPI_GELU || EPI == EPI_GELU_BWD) {
                constexpr int CHO = COUT / 8;
#pragma unroll
                for (int c = 0; c < CHO; ++c) {
                    const size_t o = rc_index(n, y, c, x, H, W, CHO);
                    __align__(16) bf16 a8[8], z8[8];
                    if constexpr (EPI == EPI_GELU) {
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            const float z = v[8 * c + k] + __ldg(ea.bias + 8 * c + k);
                            z8[k] = __float2bfloat16_rn(z);
                            a8[k] = __float2bfloat16_rn(gelu_f(z));
                        }
                        *reinterpret_cast<uint4 *>(ea.out + o) = *reinterpret_cast<const uint4 *>(a8);
                        if (ea.zout) *reinterpret_cast<uint4 *>(ea.zout + o) = *reinterpret_cast<const uint4 *>(z8);
                    } else {
                        const uint4 zr = zpre[r][c];
                        const bf16 *zz = reinterpret_cast<const bf16 *>(&zr);
#pragma unroll
                        for (int k = 0; k < 8; ++k)
                            a8[k] = __float2bfloat16_rn(v[8 * c + k] * gelu_grad_f(__bfloat162float(zz[k])));
                        *reinterpret_cast<uint4 *>(ea.out + o) = *reinterpret_cast<const uint4 *>(a8);
                    }
                }
            } else {
                float rr[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) rr[c] = v[c] + __ldg(ea.bias + c);
                const size_t plane = (size_t)H * W;
                const size_t po = ((size_t)n * 3) * plane + (size_t)y * W + x;
                if constexpr (EPI == EPI_LOSS) {
                    __align__(16) bf16 d8[16];
#pragma unroll
                    for (int k = 0; k < 16; ++k) d8[k] = __float2bfloat16_rn(0.0f);
                    const float w = ea.img_w ? __ldg(ea.img_w + n) : 1.0f;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float d = rr[c] - fpre[r][c];
                        lsum += (double)w * ((double)d * (double)d);
                        d8[c] = __float2bfloat16_rn(ea.loss_scale * w * d);
                        if (ea.resid) ea.resid[po + c * plane] = rr[c];
                    }
                    *reinterpret_cast<uint4 *>(ea.out + rc_index(n, y, 0, x, H, W, 2)) =
                        *reinterpret_cast<const uint4 *>(d8);
                    *reinterpret_cast<uint4 *>(ea.out + rc_index(n, y, 1, x, H, W, 2)) =
                        *reinterpret_cast<const uint4 *>(d8 + 8);
                } else if constexpr (EPI == EPI_RESID) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) ea.resid[po + c * plane] = rr[c] * ea.oscale[c];
                } else {
                    float *st = ea.state + n * ea.st_img + (long long)y * ea.st_pitch + x;
#pragma unroll
                    for (int c = 0; c < 3; ++c) st[c * ea.st_plane] = __fmaf_rn(rr[c], ea.oscale[c], fpre[r][c]);
                    lsum += (double)(rr[0] * ea.oscale[0]);
                }
            }
        }
        if constexpr (EPI == EPI_LOSS || EPI == EPI_APPLY) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
            double *acc = EPI == EPI_LOSS ? ea.loss_accum : (ea.hsum ? ea.hsum + n : nullptr);
            if (lane == 0 && acc && lsum != 0.0) atomicAdd(acc, lsum);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tmem, C::TMEM_COLS);
}

// ---------------------------------------------------------------------------
// Weight gradients on the tensor cores.  dW[ky][kx][ci][co] = sum_p
// X[p + (ky-1, kx-1)][ci] dY[p][co] is a GEMM with the pixels as K: both
// activations are row-chunked, so for one image row a strip holds pixels at
// a 16-byte stride with 8 channels contiguous in each -- a 16-bit MN-major
// operand whose core matrices (8 channels x 8 pixels, 128 contiguous bytes)
// lie 128 bytes apart along K and one strip (2080 bytes) apart along M or N.
// In the staged box [rows][CHX][130][8] the strips of consecutive rows
// continue at that same stride, so the 16 core-matrix groups of an M = 128
// operand starting at output row r are (dy, strip) = (g / CHX, g % CHX),
// dy = 0 .. 16/CHX - 1: one MMA covers the three vertical taps at once (the
// groups with dy > 2 are computed and discarded).  The horizontal tap kx is
// a 16-byte shift of the A start address, and each kx has its own TMEM
// accumulator of N = COUT columns.
//
// wgrad_tc_kernel: persistent CTAs stride over tiles of 128 pixels x R rows
// of one image; per tile thread 0 issues R x 3 x 8 MMAs (M = 128, N = 8 CHY,
// K = 16 pixels, A and B MN-major) while all threads add the staged output
// gradient into the bias gradient; at the end the accumulators go to the
// CTA's partial row (the layout of the CUDA-core kernel's rows), which
// reduce_rows_kernel sums in a fixed order.
// ---------------------------------------------------------------------------
constexpr int kWgRows = 4;  // output rows per tile

template <int CHX, int CHY>
struct WgCfg {
    static constexpr int N = 8 * CHY;                 // MMA N: output-gradient channels (padded)
    static constexpr int DY = 16 / CHX;               // vertical taps one M = 128 operand spans
    static constexpr int XROWS = kWgRows + DY - 1;    // staged input rows
    static constexpr size_t X_BYTES = (size_t)XROWS * CHX * kStripB;
    static constexpr size_t Y_BYTES = (size_t)kWgRows * CHY * kStripB;
    static constexpr size_t OFF_Y = al128(X_BYTES);
    static constexpr size_t OFF_RED = al128(OFF_Y + Y_BYTES);
    static constexpr size_t OFF_BAR = al128(OFF_RED + (size_t)4 * 32 * 4);  // 4 warps x 32 bias partials
    static constexpr size_t SMEM = OFF_BAR + 64 + 128;
    static constexpr uint32_t TMEM_COLS = pow2_at_least((uint32_t)(3 * N));
};

template <int CHX, int CHY, int CIN, int COUT>
__global__ void __launch_bounds__(128) wgrad_tc_kernel(const __grid_constant__ CUtensorMap mX,
                                                       const __grid_constant__ CUtensorMap mY, int W, int H, int n,
                                                       float *__restrict__ partial, int *err)
{
    using C = WgCfg<CHX, CHY>;
    constexpr int N = C::N;
    constexpr int NOUT = 9 * CIN * COUT + COUT;
    static_assert(CIN <= 8 * CHX && COUT <= N && C::DY >= 3, "tile shape");
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *sX = smem;
    unsigned char *sY = smem + C::OFF_Y;
    float *red = reinterpret_cast<float *>(smem + C::OFF_RED);
    uint64_t *bar_tma = reinterpret_cast<uint64_t *>(smem + C::OFF_BAR);
    uint64_t *bar_mma = bar_tma + 1;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar_tma + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_x = (W + kTileX - 1) / kTileX, tiles_y = (H + kWgRows - 1) / kWgRows;
    const long long ntiles = (long long)tiles_x * tiles_y * n;

    if (tid == 0) {
        mbar_init(bar_tma, 1);
        mbar_init(bar_mma, 1);
        fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(tslot, C::TMEM_COLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;

    float bacc[COUT];
#pragma unroll
    for (int c = 0; c < COUT; ++c) bacc[c] = 0.0f;
    constexpr uint32_t idesc = tc::idesc_bf16(128, N) | (1u << 15) | (1u << 16);  // A and B MN-major
    bool ok = true, any = false;
    uint32_t phase = 0;
    for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, phase ^= 1u) {
        const int tx = (int)(tile % tiles_x);
        const int ty = (int)((tile / tiles_x) % tiles_y);
        const int img = (int)(tile / ((long long)tiles_x * tiles_y));
        const int x0 = tx * kTileX, y0 = ty * kWgRows;
        if (tid == 0) {
            mbar_arrive_expect_tx(bar_tma, (uint32_t)(C::X_BYTES + C::Y_BYTES));
            tma_load_5d(sX, &mX, bar_tma, 0, x0 - 1, 0, y0 - 1, img);
            tma_load_5d(sY, &mY, bar_tma, 0, x0, 0, y0, img);
        }
        ok = __syncthreads_and(mbar_wait_bounded(bar_tma, phase, err));
        if (!ok) break;
        tc::fence_after_sync();
        if (tid == 0) {
#pragma unroll 1
            for (int r = 0; r < kWgRows; ++r) {
#pragma unroll 1
                for (int kx = 0; kx < 3; ++kx) {
#pragma unroll
                    for (int ks = 0; ks < 8; ++ks) {
                        const unsigned char *a = sX + (size_t)r * CHX * kStripB + (size_t)(16 * ks + kx) * kPixB;
                        const unsigned char *b = sY + (size_t)r * CHY * kStripB + (size_t)(16 * ks) * kPixB;
                        tc::mma_bf16(tmem + (uint32_t)(kx * N), tc::smem_desc(a, 128, kStripB),
                                     tc::smem_desc(b, 128, kStripB), idesc, any || r > 0 || ks > 0);
                    }
                }
            }
            tc::commit(bar_mma);
        }
        any = true;
        // bias gradient: thread t adds pixel t of every staged row
        {
#pragma unroll
            for (int r = 0; r < kWgRows; ++r) {
#pragma unroll
                for (int c8 = 0; c8 < (COUT + 7) / 8; ++c8) {
                    const uint4 q = *reinterpret_cast<const uint4 *>(sY + ((size_t)r * CHY + c8) * kStripB +
                                                                     (size_t)tid * kPixB);
                    const bf16 *v = reinterpret_cast<const bf16 *>(&q);
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        if (8 * c8 + k < COUT) bacc[8 * c8 + k] += __bfloat162float(v[k]);
                }
            }
        }
        fence_proxy_async_smem();  // the generic reads above come before the next TMA write
        ok = mbar_wait_bounded(bar_mma, phase, err);
        ok = __syncthreads_and(ok);
        tc::fence_after_sync();
    }

    float *out = partial + (size_t)blockIdx.x * NOUT;
    // bias: warp sums, then warp 0 adds the four warps' values in order
#pragma unroll
    for (int c = 0; c < COUT; ++c) {
        float v = bacc[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp * 32 + c] = v;
    }
    __syncthreads();
    if (tid < COUT) out[9 * CIN * COUT + tid] = ok ? ((red[tid] + red[32 + tid]) + red[64 + tid]) + red[96 + tid] : 0.0f;
    // weights: TMEM lane m = row (dy, strip, channel) of the M = 128 operand
    const int g = (warp * 32 + lane) >> 3, ky = g / CHX, ci = (g % CHX) * 8 + (lane & 7);
    const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
    for (int kx = 0; kx < 3; ++kx) {
        float v[N];
        if (any && ok) {
            if constexpr (N == 32)
                tc::ld_x32(tbase + (uint32_t)(kx * N), v);
            else
                tc::ld_x16(tbase + (uint32_t)(kx * N), v);
        } else {
#pragma unroll
            for (int c = 0; c < N; ++c) v[c] = 0.0f;
        }
        if (ky < 3 && ci < CIN) {
            float *o = out + (size_t)((ky * 3 + kx) * CIN + ci) * COUT;
#pragma unroll
            for (int c = 0; c < COUT; ++c) o[c] = v[c];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tmem, C::TMEM_COLS);
}

// ---------------------------------------------------------------------------
// Small element-wise kernels
// ---------------------------------------------------------------------------

// FP32 state planes (3 per image, rows of ``pitch``) -> row-chunked bf16 input
// with 16 channels: (h - h0)/sh, hu/su, hv/su, then zeros.  With a second
// state ``base`` the input is the difference (state - base) instead:
// (dh/sh, dhu/su, dhv/su), formed in FP32 before the rounding to bf16.
__global__ void prep_input_kernel(const float *__restrict__ state, const float *__restrict__ base,
                                  long long img_stride, long long plane_stride, long long pitch, int W, int H, int n,
                                  float h0, float inv_sh, float inv_su, bf16 *__restrict__ x0)
{
    const long long total = (long long)n * H * W;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
         p += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(p % W);
        const int y = (int)((p / W) % H);
        const int i = (int)(p / ((long long)W * H));
        const long long o = i * img_stride + (long long)y * pitch + x;
        const float *s = state + o;
        float f0 = s[0] - h0, f1 = s[plane_stride], f2 = s[2 * plane_stride];
        if (base) {
            const float *b = base + o;
            f0 = s[0] - b[0];
            f1 -= b[plane_stride];
            f2 -= b[2 * plane_stride];
        }
        __align__(16) bf16 c8[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) c8[k] = __float2bfloat16_rn(0.0f);
        c8[0] = __float2bfloat16_rn(f0 * inv_sh);
        c8[1] = __float2bfloat16_rn(f1 * inv_su);
        c8[2] = __float2bfloat16_rn(f2 * inv_su);
        *reinterpret_cast<uint4 *>(x0 + rc_index(i, y, 0, x, H, W, 2)) = *reinterpret_cast<const uint4 *>(c8);
        *reinterpret_cast<uint4 *>(x0 + rc_index(i, y, 1, x, H, W, 2)) = *reinterpret_cast<const uint4 *>(c8 + 8);
    }
}

// F x F block average of FP32 planes: fine [n][3] planes (rows of fpitch) ->
// coarse planes (rows of cpitch).  The F*F values are summed row by row.
template <int F>
__global__ void downsample_kernel(const float *__restrict__ fine, long long f_img, long long f_plane, long long fpitch,
                                  float *__restrict__ coarse, long long c_img, long long c_plane, long long cpitch,
                                  int Wc, int Hc, int n)
{
    const long long total = (long long)n * 3 * Hc * Wc;
    const float inv = 1.0f / (float)(F * F);
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
         p += (long long)gridDim.x * blockDim.x) {
        const int X = (int)(p % Wc);
        const int Y = (int)((p / Wc) % Hc);
        const int f = (int)((p / ((long long)Wc * Hc)) % 3);
        const int i = (int)(p / ((long long)Wc * Hc * 3));
        const float *src = fine + i * f_img + f * f_plane + (long long)(F * Y) * fpitch + F * X;
        float s = 0.0f;
#pragma unroll
        for (int a = 0; a < F; ++a)
#pragma unroll
            for (int b = 0; b < F; ++b) s += src[a * fpitch + b];
        coarse[i * c_img + f * c_plane + (long long)Y * cpitch + X] = s * inv;
    }
}

// Area-weighted average of n images (3 planes each) of Hs x Ws cells onto
// Hd x Wd cells covering the same square (Wd <= Ws, Hd <= Hs): destination
// cell X spans [X fx, (X+1) fx) source cells, fx = Ws / Wd, and takes the
// mean of the source over that span, each source cell weighted by its
// overlap; separable in x and y.  The integral of every plane is kept, and
// an integer ratio is the plain block average.
__global__ void resample_kernel(const float *__restrict__ src, long long s_img, long long s_plane, long long s_pitch,
                                int Ws, int Hs, float *__restrict__ dst, long long d_img, long long d_plane,
                                long long d_pitch, int Wd, int Hd, int n)
{
    const long long total = (long long)n * 3 * Hd * Wd;
    const double fx = (double)Ws / Wd, fy = (double)Hs / Hd;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
         p += (long long)gridDim.x * blockDim.x) {
        const int X = (int)(p % Wd);
        const int Y = (int)((p / Wd) % Hd);
        const int f = (int)((p / ((long long)Wd * Hd)) % 3);
        const int i = (int)(p / ((long long)Wd * Hd * 3));
        const double x0 = X * fx, x1 = (X + 1) * fx, y0 = Y * fy, y1 = (Y + 1) * fy;
        const int i0 = (int)floor(x0), i1 = min(Ws, (int)ceil(x1));
        const int j0 = (int)floor(y0), j1 = min(Hs, (int)ceil(y1));
        const float *plane = src + i * s_img + f * s_plane;
        double acc = 0.0;
        for (int j = j0; j < j1; ++j) {
            const double wy = fmin(y1, (double)(j + 1)) - fmax(y0, (double)j);
            double row = 0.0;
            for (int c = i0; c < i1; ++c) {
                const double wx = fmin(x1, (double)(c + 1)) - fmax(x0, (double)c);
                row += wx * (double)plane[(long long)j * s_pitch + c];
            }
            acc += wy * row;
        }
        dst[i * d_img + f * d_plane + (long long)Y * d_pitch + X] = (float)(acc / (fx * fy));
    }
}

// Sums the per-CTA partial rows in a fixed order: grad[j] = sum_b partial[b][j].
__global__ void reduce_rows_kernel(const float *__restrict__ partial, int rows, int cols, float *__restrict__ out)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < cols; j += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < rows; ++b) s += (double)partial[(size_t)b * cols + j];
        out[j] = (float)s;
    }
}

// AdamW on FP32 master parameters (decoupled weight decay on every entry).
__global__ void adamw_kernel(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                             const float *__restrict__ g, int n, float lr, float b1, float b2, float eps, float wd,
                             float c1, float c2, float gscale)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i] * gscale;
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * ((mi * c1) / (sqrtf(vi * c2) + eps) + wd * w[i]);
    }
}

// Squared L2 norm of a vector into out[0] (one block).
__global__ void sqnorm_kernel(const float *__restrict__ g, int n, float *out)
{
    __shared__ double part[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += (double)g[i] * g[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += part[k];
        out[0] = (float)t;
    }
}

// Packs FP32 weights W[t][cin][cout] (t = 3*ky + kx) into the bf16 B-operand
// image of a conv with NKS K steps and NC N-cores.  With ``flip`` the image is
// that of the input gradient: tap t uses W[8 - t], K runs over cout and N
// over cin.
__global__ void pack_weights_kernel(const float *__restrict__ Wsrc, int cin, int cout, int NKS, int NC, int flip,
                                    bf16 *__restrict__ img)
{
    const int total = 9 * NKS * 2 * NC * 64;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int kk = e % 8;
        const int rr = (e / 8) % 8;
        const int ni = (e / 64) % NC;
        const int ki = (e / (64 * NC)) % 2;
        const int s = (e / (128 * NC)) % NKS;
        const int t = e / (128 * NC * NKS);
        const int k = s * 16 + ki * 8 + kk;  // K index
        const int nn = ni * 8 + rr;          // N index
        float v = 0.0f;
        if (!flip) {
            if (k < cin && nn < cout) v = Wsrc[(t * cin + k) * cout + nn];
        } else {
            if (k < cout && nn < cin) v = Wsrc[((8 - t) * cin + nn) * cout + k];
        }
        img[e] = __float2bfloat16_rn(v);
    }
}

// Bias padded to the accumulator width (zeros past the real channels).
__global__ void pad_bias_kernel(const float *__restrict__ b, int n, int npad, float *__restrict__ out)
{
    for (int i = threadIdx.x; i < npad; i += blockDim.x) out[i] = i < n ? b[i] : 0.0f;
}

// Per image: subtract the mean of the h correction (so the corrected step
// keeps the mass of the Lax-Wendroff step exactly, up to rounding) and add
// the correction to the state.  One block per image.
__global__ void __launch_bounds__(1024) apply_correction_kernel(float *__restrict__ state, long long img_stride,
                                                                long long plane_stride, long long pitch,
                                                                const float *__restrict__ resid, int W, int H,
                                                                int project_mass)
{
    __shared__ double part[32];
    const int i = blockIdx.x;
    const size_t plane = (size_t)H * W;
    const float *r = resid + (size_t)i * 3 * plane;
    double s = 0.0;
    if (project_mass)
        for (size_t p = threadIdx.x; p < plane; p += blockDim.x) s += (double)r[p];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    double tot = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) tot += part[k];
    const float mean = project_mass ? (float)(tot / (double)plane) : 0.0f;
    float *st = state + (size_t)i * img_stride;
    for (size_t p = threadIdx.x; p < plane; p += blockDim.x) {
        const size_t y = p / W, x = p % W;
        const size_t o = y * pitch + x;
        st[o] += r[p] - mean;
        st[plane_stride + o] += r[plane + p];
        st[2 * plane_stride + o] += r[2 * plane + p];
    }
}

// h[n] -= hsum[n] / (H W) over every cell of each image.
__global__ void subtract_mean_kernel(float *__restrict__ state, long long img_stride, long long pitch, int W, int H,
                                     int n, const double *__restrict__ hsum)
{
    const long long plane = (long long)H * W;
    const long long total = (long long)n * plane;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / plane);
        const long long p = e % plane;
        const float mean = (float)(hsum[i] / (double)plane);
        state[i * img_stride + (p / W) * pitch + (p % W)] -= mean;
    }
}

// target[n][c][y][x] = (next[n][c][y][x] - lw_c(y, x)) * inv_scale[c], clipped
// to [-clip, clip] when clip > 0.
__global__ void make_target_kernel(const float *__restrict__ next, const float *__restrict__ lw, long long img_stride,
                                   long long plane_stride, long long pitch, int W, int H, int n, float is_h,
                                   float is_u, float clip, float *__restrict__ target)
{
    const long long plane = (long long)H * W;
    const long long total = (long long)n * 3 * plane;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(e % W);
        const int y = (int)((e / W) % H);
        const int c = (int)((e / plane) % 3);
        const int i = (int)(e / (3 * plane));
        const float l = lw[i * img_stride + c * plane_stride + (long long)y * pitch + x];
        float t = (next[e] - l) * (c == 0 ? is_h : is_u);
        if (clip > 0.0f) t = fminf(fmaxf(t, -clip), clip);
        target[e] = t;
    }
}

// Per-image loss weight w[i] = max(ms_i, floor)^(-power/2), ms_i the mean
// square of image i's target over its three channels (one block per image,
// FP64 sums in a fixed order).
__global__ void __launch_bounds__(256) image_weight_kernel(const float *__restrict__ target, long long img_elems,
                                                           float power, float floor, float *__restrict__ w)
{
    __shared__ double part[8];
    const float *t = target + (size_t)blockIdx.x * img_elems;
    double s = 0.0;
    for (long long e = threadIdx.x; e < img_elems; e += blockDim.x) s += (double)t[e] * (double)t[e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int k = 0; k < 8; ++k) tot += part[k];
        const double ms = fmax(tot / (double)img_elems, (double)floor);
        w[blockIdx.x] = (float)pow(ms, -0.5 * (double)power);
    }
}

bool encode_act_map(CUtensorMap *map, const void *base, int W, int H, int CH, int N, int box_rows);

}  // namespace swe

// ===========================================================================
// Host side: the network object and its C ABI
// ===========================================================================
using namespace swe;

namespace {

constexpr int kHidden = 32;
// flat parameter layout: W1[9][3][32], b1[32], W2[9][32][32], b2[32], W3[9][32][3], b3[3]
constexpr int kOffW1 = 0, kOffB1 = 864, kOffW2 = 896, kOffB2 = 10112, kOffW3 = 10144, kOffB3 = 11008;
constexpr int kParams = 11011;
constexpr int kWgBlocks = 304;
constexpr int kWgMaxOut = 9 * 32 * 32 + 32;

using L1 = ConvCfg<2, 32, kConvRows>;  // layer 1 forward; layer 3 input gradient
using L2 = ConvCfg<4, 32, kConvRows>;  // layer 2 forward and input gradient
using L3 = ConvCfg<4, 16, kConvRows>;  // layer 3 forward

template <int CH, int COUT, int EPI>
cudaError_t launch_conv(const CUtensorMap &map, const bf16 *wimg, const EpiArgs &ea, int W, int H, int n, int *err,
                        cudaStream_t s)
{
    using C = ConvCfg<CH, COUT, kConvRows>;
    auto kern = conv3x3_tc_kernel<CH, COUT, kConvRows, EPI>;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [&] { attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM); });
    if (attr != cudaSuccess) return attr;
    const dim3 grid((W + kTileX - 1) / kTileX, (H + kConvRows - 1) / kConvRows, n);
    kern<<<grid, 128, C::SMEM, s>>>(map, wimg, ea, W, H, err);
    return cudaGetLastError();
}

template <int CHX, int CHY, int CIN, int COUT>
cudaError_t launch_wgrad(const CUtensorMap &mX, const CUtensorMap &mY, int W, int H, int n, float *partial,
                         float *grad_w, float *grad_b, int *err, cudaStream_t s)
{
    using C = WgCfg<CHX, CHY>;
    auto kern = wgrad_tc_kernel<CHX, CHY, CIN, COUT>;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [&] { attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM); });
    if (attr != cudaSuccess) return attr;
    const long long ntiles = (long long)((W + kTileX - 1) / kTileX) * ((H + kWgRows - 1) / kWgRows) * n;
    const int blocks = (int)std::min<long long>(ntiles, kWgBlocks);
    kern<<<blocks, 128, C::SMEM, s>>>(mX, mY, W, H, n, partial, err);
    constexpr int nw = 9 * CIN * COUT;
    reduce_rows_kernel<<<(nw + COUT + 255) / 256, 256, 0, s>>>(partial, blocks, nw + COUT, grad_w);
    // the bias part of each row sits right after the weights: copy it to grad_b
    cudaMemcpyAsync(grad_b, grad_w + nw, COUT * sizeof(float), cudaMemcpyDeviceToDevice, s);
    return cudaGetLastError();
}

}  // namespace

struct swe_net {
    int device = 0;
    int max_n = 0, H = 0, W = 0;
    float *params = nullptr, *m = nullptr, *v = nullptr, *grads = nullptr, *gtmp = nullptr, *partial = nullptr;
    float *bias_pad = nullptr;  // b1 (32) | b2 (32) | b3 padded (16)
    float *gnorm = nullptr;
    bf16 *w1f = nullptr, *w2f = nullptr, *w3f = nullptr, *w2d = nullptr, *w3d = nullptr;
    bf16 *x0 = nullptr, *z1 = nullptr, *a1 = nullptr, *z2 = nullptr, *a2 = nullptr, *dr = nullptr, *dz2 = nullptr,
         *dz1 = nullptr;
    float *resid = nullptr;
    CUtensorMap m_x0, m_a1, m_a2, m_dr, m_dz2;
    CUtensorMap g_x0, g_a1, g_a2, g_dr, g_dz2, g_dz1;  // boxes of the weight-gradient kernel
    float norm[5] = {1.0f, 1.0f, 1.0f, 1.0f, 1.0f};  // h0, sh, su, oh, ou
    double *loss = nullptr, *h_loss = nullptr;
    double *hsum = nullptr;
    float *img_w = nullptr;          // per-image loss weights (max_images)
    float loss_power = 0.0f, loss_floor = 1.0f;
    int *err = nullptr;
    long long step = 0;
};

namespace swe {

bool net_view(swe_net *t, NetView *v)
{
    if (!t || !v) return false;
    v->w1 = t->w1f;
    v->w2 = t->w2f;
    v->w3 = t->w3f;
    v->bias = t->bias_pad;
    for (int k = 0; k < 5; ++k) v->norm[k] = t->norm[k];
    v->d_err = t->err;
    return true;
}

}  // namespace swe

static swe_status nst(cudaError_t e)
{
    if (e == cudaSuccess) return SWE_OK;
    return e == cudaErrorMemoryAllocation ? SWE_ENOMEM : SWE_ECUDA;
}
#define N_TRY(x)                                 \
    do {                                         \
        cudaError_t e_ = (x);                    \
        if (e_ != cudaSuccess) return nst(e_);   \
    } while (0)

static cudaError_t repack(swe_net *t, cudaStream_t s)
{
    pack_weights_kernel<<<18, 256, 0, s>>>(t->params + kOffW1, 3, 32, 1, 4, 0, t->w1f);
    pack_weights_kernel<<<36, 256, 0, s>>>(t->params + kOffW2, 32, 32, 2, 4, 0, t->w2f);
    pack_weights_kernel<<<18, 256, 0, s>>>(t->params + kOffW3, 32, 3, 2, 2, 0, t->w3f);
    pack_weights_kernel<<<36, 256, 0, s>>>(t->params + kOffW2, 32, 32, 2, 4, 1, t->w2d);
    pack_weights_kernel<<<18, 256, 0, s>>>(t->params + kOffW3, 32, 3, 1, 4, 1, t->w3d);
    pad_bias_kernel<<<1, 32, 0, s>>>(t->params + kOffB1, 32, 32, t->bias_pad);
    pad_bias_kernel<<<1, 32, 0, s>>>(t->params + kOffB2, 32, 32, t->bias_pad + 32);
    pad_bias_kernel<<<1, 32, 0, s>>>(t->params + kOffB3, 3, 16, t->bias_pad + 64);
    return cudaGetLastError();
}

extern "C" {

size_t swe_net_param_count(void) { return kParams; }

void swe_net_destroy(swe_net *t)
{
    if (!t) return;
    cudaDeviceSynchronize();
    for (void *p : {(void *)t->params, (void *)t->m, (void *)t->v, (void *)t->grads, (void *)t->gtmp,
                    (void *)t->partial, (void *)t->bias_pad, (void *)t->gnorm, (void *)t->w1f, (void *)t->w2f,
                    (void *)t->w3f, (void *)t->w2d, (void *)t->w3d, (void *)t->x0, (void *)t->z1, (void *)t->a1,
                    (void *)t->z2, (void *)t->a2, (void *)t->dr, (void *)t->dz2, (void *)t->dz1, (void *)t->resid,
                    (void *)t->loss, (void *)t->err, (void *)t->hsum, (void *)t->img_w})
        cudaFree(p);
    cudaFreeHost(t->h_loss);
    delete t;
}

swe_status swe_net_create(int max_images, int H, int W, swe_net **out)
{
    if (!out) return SWE_EINVAL;
    *out = nullptr;
    if (max_images < 1 || H < 1 || W < 1 || H > 8192 || W > 8192) return SWE_EINVAL;
    swe_net *t = new (std::nothrow) swe_net();
    if (!t) return SWE_ENOMEM;
    auto fail = [&](swe_status st) {
        swe_net_destroy(t);
        return st;
    };
    cudaGetDevice(&t->device);
    t->max_n = max_images;
    t->H = H;
    t->W = W;
    const size_t px = (size_t)max_images * H * W;
    struct {
        void **p;
        size_t bytes;
    } allocs[] = {
        {(void **)&t->params, kParams * 4}, {(void **)&t->m, kParams * 4}, {(void **)&t->v, kParams * 4},
        {(void **)&t->grads, kParams * 4}, {(void **)&t->gtmp, kWgMaxOut * 4},
        {(void **)&t->partial, (size_t)kWgBlocks * kWgMaxOut * 4}, {(void **)&t->bias_pad, 80 * 4},
        {(void **)&t->gnorm, 16}, {(void **)&t->w1f, L1::B_BYTES}, {(void **)&t->w2f, L2::B_BYTES},
        {(void **)&t->w3f, L3::B_BYTES}, {(void **)&t->w2d, L2::B_BYTES}, {(void **)&t->w3d, L1::B_BYTES},
        {(void **)&t->x0, px * 16 * 2}, {(void **)&t->z1, px * 32 * 2}, {(void **)&t->a1, px * 32 * 2},
        {(void **)&t->z2, px * 32 * 2}, {(void **)&t->a2, px * 32 * 2}, {(void **)&t->dr, px * 16 * 2},
        {(void **)&t->dz2, px * 32 * 2}, {(void **)&t->dz1, px * 32 * 2}, {(void **)&t->resid, px * 3 * 4},
        {(void **)&t->loss, 16}, {(void **)&t->err, 16}, {(void **)&t->hsum, (size_t)max_images * 8},
        {(void **)&t->img_w, (size_t)max_images * 4},
    };
    for (auto &a : allocs) {
        swe_status st = nst(cudaMalloc(a.p, a.bytes));
        if (st != SWE_OK) return fail(st);
        if ((st = nst(cudaMemset(*a.p, 0, a.bytes))) != SWE_OK) return fail(st);
    }
    if (cudaMallocHost(&t->h_loss, 16) != cudaSuccess) return fail(SWE_ENOMEM);
    const int rows = kConvRows + 2;
    if (!encode_act_map(&t->m_x0, t->x0, W, H, 2, max_images, rows) ||
        !encode_act_map(&t->m_a1, t->a1, W, H, 4, max_images, rows) ||
        !encode_act_map(&t->m_a2, t->a2, W, H, 4, max_images, rows) ||
        !encode_act_map(&t->m_dr, t->dr, W, H, 2, max_images, rows) ||
        !encode_act_map(&t->m_dz2, t->dz2, W, H, 4, max_images, rows) ||
        !encode_act_map(&t->g_x0, t->x0, W, H, 2, max_images, WgCfg<2, 4>::XROWS) ||
        !encode_act_map(&t->g_a1, t->a1, W, H, 4, max_images, WgCfg<4, 4>::XROWS) ||
        !encode_act_map(&t->g_a2, t->a2, W, H, 4, max_images, WgCfg<4, 2>::XROWS) ||
        !encode_act_map(&t->g_dr, t->dr, W, H, 2, max_images, kWgRows) ||
        !encode_act_map(&t->g_dz2, t->dz2, W, H, 4, max_images, kWgRows) ||
        !encode_act_map(&t->g_dz1, t->dz1, W, H, 4, max_images, kWgRows))
        return fail(SWE_ECUDA);
    *out = t;
    return SWE_OK;
}

swe_status swe_net_set_params(swe_net *t, const float *params_host)
{
    if (!t || !params_host) return SWE_EINVAL;
    N_TRY(cudaMemcpy(t->params, params_host, kParams * 4, cudaMemcpyHostToDevice));
    N_TRY(cudaMemset(t->m, 0, kParams * 4));
    N_TRY(cudaMemset(t->v, 0, kParams * 4));
    t->step = 0;
    N_TRY(repack(t, nullptr));
    N_TRY(cudaDeviceSynchronize());
    return SWE_OK;
}

swe_status swe_net_get_params(swe_net *t, float *params_host)
{
    if (!t || !params_host) return SWE_EINVAL;
    N_TRY(cudaDeviceSynchronize());
    N_TRY(cudaMemcpy(params_host, t->params, kParams * 4, cudaMemcpyDeviceToHost));
    return SWE_OK;
}

swe_status swe_net_set_norm(swe_net *t, const float *norm5)
{
    if (!t || !norm5) return SWE_EINVAL;
    for (int k = 0; k < 5; ++k)
        if (!std::isfinite(norm5[k]) || (k > 0 && !(norm5[k] > 0.0f))) return SWE_EINVAL;
    std::memcpy(t->norm, norm5, sizeof(t->norm));
    return SWE_OK;
}

swe_status swe_net_prep_input(swe_net *t, int n, const float *state, const float *base, long long img_stride,
                              long long plane_stride, long long pitch, void *stream)
{
    if (!t || !state || n < 1 || n > t->max_n || pitch < t->W) return SWE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    prep_input_kernel<<<1184, 256, 0, s>>>(state, base, img_stride, plane_stride, pitch, t->W, t->H, n, t->norm[0],
                                           1.0f / t->norm[1], 1.0f / t->norm[2], t->x0);
    return nst(cudaGetLastError());
}

static swe_status forward_hidden(swe_net *t, int n, bool save_z, cudaStream_t s)
{
    EpiArgs e1 = {};
    e1.bias = t->bias_pad;
    e1.out = t->a1;
    e1.zout = save_z ? t->z1 : nullptr;
    N_TRY((launch_conv<2, 32, EPI_GELU>(t->m_x0, t->w1f, e1, t->W, t->H, n, t->err, s)));
    EpiArgs e2 = {};
    e2.bias = t->bias_pad + 32;
    e2.out = t->a2;
    e2.zout = save_z ? t->z2 : nullptr;
    N_TRY((launch_conv<4, 32, EPI_GELU>(t->m_a1, t->w2f, e2, t->W, t->H, n, t->err, s)));
    return SWE_OK;
}

swe_status swe_net_infer(swe_net *t, int n, float *resid_out, void *stream)
{
    if (!t || n < 1 || n > t->max_n) return SWE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    swe_status st = forward_hidden(t, n, false, s);
    if (st != SWE_OK) return st;
    EpiArgs e3 = {};
    e3.bias = t->bias_pad + 64;
    e3.resid = resid_out ? resid_out : t->resid;
    e3.oscale[0] = t->norm[3];
    e3.oscale[1] = t->norm[4];
    e3.oscale[2] = t->norm[4];
    N_TRY((launch_conv<4, 16, EPI_RESID>(t->m_a2, t->w3f, e3, t->W, t->H, n, t->err, s)));
    return SWE_OK;
}

swe_status swe_net_correct(swe_net *t, int n, float *state, long long img_stride, long long plane_stride,
                           long long pitch, int project_mass, void *stream)
{
    if (!t || !state || n < 1 || n > t->max_n || pitch < t->W) return SWE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    swe_status st = forward_hidden(t, n, false, s);
    if (st != SWE_OK) return st;
    if (project_mass) N_TRY(cudaMemsetAsync(t->hsum, 0, (size_t)n * sizeof(double), s));
    EpiArgs e3 = {};
    e3.bias = t->bias_pad + 64;
    e3.oscale[0] = t->norm[3];
    e3.oscale[1] = t->norm[4];
    e3.oscale[2] = t->norm[4];
    e3.state = state;
    e3.st_img = img_stride;
    e3.st_plane = plane_stride;
    e3.st_pitch = pitch;
    e3.hsum = project_mass ? t->hsum : nullptr;
    N_TRY((launch_conv<4, 16, EPI_APPLY>(t->m_a2, t->w3f, e3, t->W, t->H, n, t->err, s)));
    if (project_mass) {
        subtract_mean_kernel<<<1184, 256, 0, s>>>(state, img_stride, pitch, t->W, t->H, n, t->hsum);
        N_TRY(cudaGetLastError());
    }
    return SWE_OK;
}

swe_status swe_net_apply(swe_net *t, int n, float *state, long long img_stride, long long plane_stride,
                         long long pitch, int project_mass, void *stream)
{
    if (!t || !state || n < 1 || n > t->max_n) return SWE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    apply_correction_kernel<<<n, 1024, 0, s>>>(state, img_stride, plane_stride, pitch, t->resid, t->W, t->H,
                                                project_mass);
    return nst(cudaGetLastError());
}

swe_status swe_net_make_target(swe_net *t, int n, const float *next, const float *lw, long long img_stride,
                               long long plane_stride, long long pitch, float clip, float *target, void *stream)
{
    if (!t || !next || !lw || !target || n < 1 || !(clip >= 0.0f)) return SWE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    make_target_kernel<<<1184, 256, 0, s>>>(next, lw, img_stride, plane_stride, pitch, t->W, t->H, n,
                                            1.0f / t->norm[3], 1.0f / t->norm[4], clip, target);
    return nst(cudaGetLastError());
}

swe_status swe_net_train_step(swe_net *t, int n, const float *target, float lr, float wd, float clip, int update,
                              double *loss_out, float *grads_out, float *resid_out, void *stream)
{
    if (!t || !target || n < 1 || n > t->max_n) return SWE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int W = t->W, H = t->H;
    N_TRY(cudaMemsetAsync(t->loss, 0, sizeof(double), s));
    swe_status st = forward_hidden(t, n, true, s);
    if (st != SWE_OK) return st;
    const double count = (double)n * 3 * H * W;
    EpiArgs e3 = {};
    e3.bias = t->bias_pad + 64;
    e3.target = target;
    e3.out = t->dr;
    e3.resid = resid_out;
    e3.loss_scale = (float)(2.0 / count);
    e3.loss_accum = t->loss;
    if (t->loss_power != 0.0f) {
        image_weight_kernel<<<n, 256, 0, s>>>(target, (long long)3 * H * W, t->loss_power, t->loss_floor, t->img_w);
        N_TRY(cudaGetLastError());
        e3.img_w = t->img_w;
    }
    N_TRY((launch_conv<4, 16, EPI_LOSS>(t->m_a2, t->w3f, e3, W, H, n, t->err, s)));
    // input gradients: dz2 = conv^T(dr; W3) * gelu'(z2), dz1 = conv^T(dz2; W2) * gelu'(z1)
    EpiArgs b3 = {};
    b3.out = t->dz2;
    b3.zin = t->z2;
    N_TRY((launch_conv<2, 32, EPI_GELU_BWD>(t->m_dr, t->w3d, b3, W, H, n, t->err, s)));
    EpiArgs b2 = {};
    b2.out = t->dz1;
    b2.zin = t->z1;
    N_TRY((launch_conv<4, 32, EPI_GELU_BWD>(t->m_dz2, t->w2d, b2, W, H, n, t->err, s)));
    // weight gradients
    N_TRY((launch_wgrad<4, 2, 32, 3>(t->g_a2, t->g_dr, W, H, n, t->partial, t->grads + kOffW3, t->gtmp, t->err, s)));
    N_TRY(cudaMemcpyAsync(t->grads + kOffB3, t->gtmp, 3 * 4, cudaMemcpyDeviceToDevice, s));
    N_TRY((launch_wgrad<4, 4, 32, 32>(t->g_a1, t->g_dz2, W, H, n, t->partial, t->grads + kOffW2, t->gtmp, t->err, s)));
    N_TRY(cudaMemcpyAsync(t->grads + kOffB2, t->gtmp, 32 * 4, cudaMemcpyDeviceToDevice, s));
    N_TRY((launch_wgrad<2, 4, 3, 32>(t->g_x0, t->g_dz1, W, H, n, t->partial, t->grads + kOffW1, t->gtmp, t->err, s)));
    N_TRY(cudaMemcpyAsync(t->grads + kOffB1, t->gtmp, 32 * 4, cudaMemcpyDeviceToDevice, s));
    if (update) {
        t->step += 1;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.0f / (1.0f - std::pow(b1, (float)t->step));
        const float c2 = 1.0f / (1.0f - std::pow(b2, (float)t->step));
        float gscale = 1.0f;
        if (clip > 0.0f) {
            sqnorm_kernel<<<1, 1024, 0, s>>>(t->grads, kParams, t->gnorm);
            float gn2 = 0.0f;
            N_TRY(cudaMemcpyAsync(&gn2, t->gnorm, 4, cudaMemcpyDeviceToHost, s));
            N_TRY(cudaStreamSynchronize(s));
            const float gn = std::sqrt(gn2);
            if (gn > clip) gscale = clip / gn;
        }
        adamw_kernel<<<44, 256, 0, s>>>(t->params, t->m, t->v, t->grads, kParams, lr, b1, b2, 1e-8f, wd, c1, c2,
                                        gscale);
        N_TRY(repack(t, s));
    }
    if (grads_out) N_TRY(cudaMemcpyAsync(grads_out, t->grads, kParams * 4, cudaMemcpyDeviceToHost, s));
    N_TRY(cudaMemcpyAsync(t->h_loss, t->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    N_TRY(cudaStreamSynchronize(s));
    if (loss_out) *loss_out = t->h_loss[0] / count;
    int word = 0;
    N_TRY(cudaMemcpy(&word, t->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (word) {
        cudaMemset(t->err, 0, sizeof(int));
        return (swe_status)word;
    }
    return SWE_OK;
}

swe_status swe_net_set_loss_weighting(swe_net *t, float power, float floor)
{
    if (!t || !std::isfinite(power) || power < 0.0f || power > 4.0f || !(floor > 0.0f) || !std::isfinite(floor))
        return SWE_EINVAL;
    t->loss_power = power;
    t->loss_floor = floor;
    return SWE_OK;
}

swe_status swe_net_check(swe_net *t, void *stream)
{
    if (!t) return SWE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    N_TRY(cudaStreamSynchronize(s));
    int word = 0;
    N_TRY(cudaMemcpy(&word, t->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (word) {
        cudaMemset(t->err, 0, sizeof(int));
        return (swe_status)word;
    }
    return SWE_OK;
}

swe_status swe_selftest_gelu(const float *z, float *out, int n, int which, void *stream)
{
    if (!z || !out || n < 0 || which < 0 || which > 2) return SWE_EINVAL;
    gelu_probe_kernel<<<(n + 255) / 256 > 0 ? std::min((n + 255) / 256, 4096) : 1, 256, 0,
                        static_cast<cudaStream_t>(stream)>>>(z, out, n, which);
    return nst(cudaGetLastError());
}

swe_status swe_resample(const float *src, long long s_img, long long s_plane, long long s_pitch, int Ws, int Hs,
                        float *dst, long long d_img, long long d_plane, long long d_pitch, int Wd, int Hd, int n,
                        void *stream)
{
    if (!src || !dst || n < 1 || Wd < 1 || Hd < 1 || Wd > Ws || Hd > Hs || s_pitch < Ws || d_pitch < Wd)
        return SWE_EINVAL;
    resample_kernel<<<2368, 256, 0, static_cast<cudaStream_t>(stream)>>>(src, s_img, s_plane, s_pitch, Ws, Hs, dst,
                                                                        d_img, d_plane, d_pitch, Wd, Hd, n);
    return nst(cudaGetLastError());
}

swe_status swe_downsample(int factor, const float *fine, long long f_img, long long f_plane, long long f_pitch,
                          float *coarse, long long c_img, long long c_plane, long long c_pitch, int Wc, int Hc, int n,
                          void *stream)
{
    if (!fine || !coarse || Wc < 1 || Hc < 1 || n < 1 || factor < 1 || factor > 4) return SWE_EINVAL;
    if (f_pitch < (long long)factor * Wc || c_pitch < Wc) return SWE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    switch (factor) {
        case 1: downsample_kernel<1><<<1184, 256, 0, s>>>(fine, f_img, f_plane, f_pitch, coarse, c_img, c_plane, c_pitch, Wc, Hc, n); break;
        case 2: downsample_kernel<2><<<1184, 256, 0, s>>>(fine, f_img, f_plane, f_pitch, coarse, c_img, c_plane, c_pitch, Wc, Hc, n); break;
        case 3: downsample_kernel<3><<<1184, 256, 0, s>>>(fine, f_img, f_plane, f_pitch, coarse, c_img, c_plane, c_pitch, Wc, Hc, n); break;
        default: downsample_kernel<4><<<1184, 256, 0, s>>>(fine, f_img, f_plane, f_pitch, coarse, c_img, c_plane, c_pitch, Wc, Hc, n); break;
    }
    return nst(cudaGetLastError());
}

}  // extern "C"
