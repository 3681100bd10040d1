// swe_learned.cu -- the learned coarse step fused into one persistent
// launch: for every instance of a batch and every step, the coarse
// Lax-Wendroff step (Sec. 3), the corrector network (zero-padded 3x3
// convolutions 3 -> 32 -> 32 -> 3 with GELU, BF16 operands, FP32
// accumulation in tensor memory) on the normalised increment, and the
// corrected update with the mass projection, all on one SM per instance.
// The network has no counterpart in the paper.
//
// A CTA owns whole instances (up to 256 cells wide) and sweeps each one row
// by row.  Tick t of a sweep computes, in a software pipeline two rows deep
// per stage:
//   LW  row t      CUDA cores; the network input x0[t] (the normalised
//                  increment, 16 bf16 channels) goes to a 2-row ring
//   E1  row t-2    GELU of layer 1's accumulator -> a1 ring (2 rows)
//   E2  row t-4    GELU of layer 2's accumulator -> a2 ring (2 rows)
//   E3  row t-6    layer 3's output, scaled, added to the LW row -> HBM
// The MMAs run by input row: input row j of a layer feeds output rows j+1,
// j, j-1 through kernel rows ky = 0, 1, 2, so one MMA per (kx, K step, half
// row) with N = 3 x (output channels) -- the B operand is the three ky
// weight blocks side by side -- adds row j's contributions to the three
// output rows' accumulators at once.  Each layer keeps its accumulators in
// a ring of three TMEM blocks (output row r in block r mod 3); the weights
// are stored in three rotations so that block b of the MMA's output always
// meets the ky that row r = b (mod 3) needs.  An accumulator starts from
// the bias (the epilogue that reads output row r re-arms the block for row
// r+3), so every MMA accumulates.  Per tick a separate warp -- one elected
// lane -- issues layer 1 on x0[t] once E1 has re-armed its block, layer 2
// on a1[t-2] after E2, and layer 3 on a2[t-4] after E3; their results are
// read one tick later, so the tensor core runs under the next tick's CUDA
// work.  The A operand is a ring row at a shifted shared-memory address
// (kx): no im2col copy exists.  Pixels outside the grid are zero in the
// rings and rows outside it are never MMA inputs: the zero padding.
//
// Mass projection: the mean of the h correction over the instance is known
// only when the sweep ends, so it is kept as a pending offset m: the state
// written by a sweep is (true h) + m, the next sweep subtracts m as it
// loads, and after the last step every h is corrected in place.  The steps
// are the unfused path's (correct, then subtract the mean); the sum behind
// the mean is taken per pixel in FP32 over blocks of 16 rows and in FP64
// across blocks and pixels (the unfused path sums in FP64 throughout), so
// the two means agree to FP32 rounding of 16-term sums.
#include <algorithm>
#include <mutex>

#include "swe_gelu.cuh"
#include "swe_tc.cuh"
#include "swe_views.cuh"

#ifndef SWE_LEARN_NG
#define SWE_LEARN_NG 2
#endif
#ifndef SWE_LEARN_C0
#define SWE_LEARN_C0 8
#endif

namespace swe {

namespace {

__host__ __device__ constexpr size_t lal16(size_t x) { return (x + 15) / 16 * 16; }

template <int NH, int NG>
struct LearnCfg {
    static constexpr int PX = 128 * NH;      // pixels of a row (the MMA's M per half)
    static constexpr int PXB = PX + 2;       // with a zero pixel at each end
    static constexpr int STRIP = PXB * 16;   // one 8-channel strip of a ring row, bytes
    static constexpr int X0_ROW = 2 * STRIP; // 16 channels
    static constexpr int A_ROW = 4 * STRIP;  // 32 channels
    // LW_SLOTS: a thread of group 0 writes its pixel of the Lax-Wendroff
    // row t in tick t and reads it back in tick t+6 (rows t-6 .. t live)
    static constexpr int RING = 2, LW_SLOTS = 7;
    static constexpr int NCW = 4 * NH * NG;  // compute warps; one more issues the MMAs
    static constexpr int THREADS = (NCW + 1) * 32;
    // layer 1's channels per epilogue thread: group 0 (which also runs the
    // Lax-Wendroff row and the output stage) takes C0, group 1 the rest;
    // group 1 also takes all 32 channels of layer 2
    static_assert(NG == 2, "two compute groups: group 0 the Lax-Wendroff row and the output stage, group 1 layer 2");
    static constexpr int C0 = SWE_LEARN_C0;
    static constexpr int C1 = 32 - C0;
    static_assert(C0 % 8 == 0 && C0 >= 0 && C0 <= 32, "layer-1 channel split in 8-channel strips");
    // Weight images: per layer, rotation rho (0..2), kx, K step s, a 16 x 3C
    // K-major B operand [K core 2][N core 3C/8][8 x 16 B].
    static constexpr size_t IMG1 = 2 * 12 * 128, IMG2 = 2 * 12 * 128, IMG3 = 2 * 6 * 128;
    static constexpr size_t W1_B = 9 * 1 * IMG1, W2_B = 9 * 2 * IMG2, W3_B = 9 * 2 * IMG3;
    static constexpr size_t OFF_W1 = 0;
    static constexpr size_t OFF_W2 = OFF_W1 + W1_B;
    static constexpr size_t OFF_W3 = OFF_W2 + W2_B;
    static constexpr size_t OFF_X0 = OFF_W3 + W3_B;
    static constexpr size_t OFF_A1 = lal16(OFF_X0 + (size_t)RING * X0_ROW);
    static constexpr size_t OFF_A2 = lal16(OFF_A1 + (size_t)RING * A_ROW);
    static constexpr size_t OFF_LW = lal16(OFF_A2 + (size_t)RING * A_ROW);
    static constexpr size_t OFF_XR = OFF_LW + (size_t)LW_SLOTS * 3 * PX * 4;
    static constexpr size_t OFF_BIAS = OFF_XR + (size_t)2 * 5 * PXB * 4;
    static constexpr size_t OFF_RED = lal16(OFF_BIAS + 80 * 4);
    static constexpr size_t OFF_BAR = lal16(OFF_RED + 16 * 8);
    static constexpr size_t SMEM = OFF_BAR + 128;
    // TMEM per layer: per half-row of 128 pixels, three row blocks of C
    // columns (C = 32, 32, 16).
    static constexpr uint32_t ACC1 = 0, ACC2 = NH * 96, ACC3 = 2 * NH * 96;
    static constexpr uint32_t TMEM_USED = ACC3 + NH * 48;
    static constexpr uint32_t TMEM_COLS = TMEM_USED <= 256 ? 256 : 512;
};

struct LearnArgs {
    const BatchInst *inst;
    int n_inst;
    int n_steps;
    int parity0;
    const bf16 *w1, *w2, *w3;  // B-operand images (global)
    const float *bias;         // 80 floats
    float inv_sh, inv_su;      // input normalisation of the increment
    float os_h, os_u;          // output scales of the residual
    int project;               // zero-mean h correction
    int *flags;
    int *err;
};

// mbarriers (shared memory, in this order).  Each advances one phase per
// batch; no barrier runs two phases ahead of a waiter, because every
// arrival for batch t+1 follows its warp's wait on batch t.  B_RDY2 and B_L2
// concern group 1 only (layer 2's epilogue), B_RDY3 and B_L3 group 0 only
// (the output stage); the MMA warp waits for B_RDY1, B_RDY2 and B_RDY3 in
// turn, so each layer's MMAs also follow the epilogue that wrote their
// input row.
enum { B_RDY1 = 0, B_RDY2 = 1, B_RDY3 = 2, B_L1 = 3, B_L2 = 4, B_L3 = 5, B_FIN = 6, B_COUNT = 7 };

__device__ __forceinline__ void named_bar_sync(int id, int count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ uint4 zero4() { return make_uint4(0u, 0u, 0u, 0u); }

// True on exactly one lane of the (converged) warp.
__device__ __forceinline__ bool elect_one()
{
    uint32_t p;
    asm volatile(
        "{\n\t.reg .pred P;\n\t"
        "elect.sync _|P, 0xffffffff;\n\t"
        "selp.b32 %0, 1, 0, P;\n\t}"
        : "=r"(p));
    return p != 0;
}

// Two floats rounded to bf16 (nearest even), lo in the low half.
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// A warp hands its shared-memory writes (generic proxy) and its finished
// TMEM reads over to the MMA warp: every lane fences, lane 0 arrives.
__device__ __forceinline__ void publish(uint64_t *bar, int lane)
{
    fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncwarp();
    if (lane == 0) mbar_arrive(bar);
}

// The same for a hand-over of TMEM writes only (no shared-memory operand
// was written): no proxy fence.
__device__ __forceinline__ void publish_tmem(uint64_t *bar, int lane)
{
    tc::fence_before_sync();
    __syncwarp();
    if (lane == 0) mbar_arrive(bar);
}

__device__ __forceinline__ int mod3(int r) { return r - 3 * (r / 3); }

// Sixteen bias values (shared memory, 16-byte aligned) into registers.
__device__ __forceinline__ void load16(const float *p, float (&b)[16])
{
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float4 f = *reinterpret_cast<const float4 *>(p + 4 * k);
        b[4 * k] = f.x;
        b[4 * k + 1] = f.y;
        b[4 * k + 2] = f.z;
        b[4 * k + 3] = f.w;
    }
}

// Arms CPT accumulator columns at taddr with the bias (TMEM store); an odd
// 8 columns first, so that every 16-column store starts on a multiple of 16
// when taddr's column is a multiple of 16 or sits 8 past one.
// The stores are issued back to back and waited for once (WAIT), or the
// caller waits (tc::wait_st) before the columns are handed to the MMAs.
template <int CPT, bool WAIT = true>
__device__ __forceinline__ void arm(uint32_t taddr, const float *bias)
{
    static_assert(CPT % 8 == 0, "8-column granules");
    constexpr int LEAD = CPT % 16;
    if constexpr (LEAD == 8) {
        float b[16];
        load16(bias, b);  // 16 floats are readable: the bias block has 80
        tc::st_x8_async(taddr, b);
    }
#pragma unroll
    for (int c = 0; c < CPT / 16; ++c) {
        float b[16];
        load16(bias + LEAD + 16 * c, b);
        tc::st_x16_async(taddr + LEAD + 16 * c, b);
    }
    if constexpr (WAIT) tc::wait_st();
}

// CPT (8, 16 or 24) accumulator columns at taddr into v, in the same
// granules as arm: the loads are issued back to back and waited for once.
template <int CPT>
__device__ __forceinline__ void tmem_load(uint32_t taddr, float (&v)[CPT])
{
    static_assert(CPT == 8 || CPT == 16 || CPT == 24, "granules");
    if constexpr (CPT == 8) {
        uint32_t a[8];
        tc::ld_x8_async(taddr, a);
        tc::wait_ld(a);
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(a[i]);
    } else if constexpr (CPT == 16) {
        uint32_t b[16];
        tc::ld_x16_async(taddr, b);
        tc::wait_ld(b);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(b[i]);
    } else {
        uint32_t a[8], b[16];
        tc::ld_x8_async(taddr, a);
        tc::ld_x16_async(taddr + 8, b);
        tc::wait_ld(a, b);
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(a[i]);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[8 + i] = __uint_as_float(b[i]);
    }
}

// Hidden-layer epilogue of one pixel: CPT finished accumulator columns at
// taddr (bias included) -> GELU -> bf16 -> CPT/8 strips of a ring row at
// dst (strip stride ``strip``), zeros where the pixel is outside the grid;
// then the columns are re-armed with the bias.
template <int CPT>
__device__ __forceinline__ void hidden_epilogue(uint32_t taddr, const float *bias, unsigned char *dst, int strip,
                                                bool valid)
{
    if constexpr (CPT == 32) {  // 16 columns at a time (registers)
        hidden_epilogue<16>(taddr, bias, dst, strip, valid);
        hidden_epilogue<16>(taddr + 16, bias + 16, dst + 2 * strip, strip, valid);
    } else {
        float v[CPT];
        tmem_load<CPT>(taddr, v);
        arm<CPT, false>(taddr, bias);  // completes under the activations
#pragma unroll
        for (int c = 0; c < CPT / 8; ++c) {
            float y[8];
#pragma unroll
            for (int k = 0; k < 8; k += 2) gelu_f2(v[8 * c + k], v[8 * c + k + 1], y[k], y[k + 1]);
            const uint4 o = make_uint4(pack_bf16x2(y[0], y[1]), pack_bf16x2(y[2], y[3]), pack_bf16x2(y[4], y[5]),
                                       pack_bf16x2(y[6], y[7]));
            *reinterpret_cast<uint4 *>(dst + c * strip) = valid ? o : zero4();
        }
        tc::wait_st();
    }
}

// Copies the per-tap B images of one layer (global; block (tap, s) is
// [K core 2][N core NC][8 x 16 B]) into the rotated, concatenated images
// (shared): image (rho, kx, s) has N block b = the weights of tap
// (ky, kx) with ky = (rho - b + 1) mod 3, for an input row j = rho (mod 3)
// whose MMA output block b holds output row r = b (mod 3), ky = j - r + 1.
__device__ __forceinline__ void rotate_weights(const bf16 *src, unsigned char *dst, int NC, int NKS, int tid,
                                               int nthreads)
{
    const uint4 *s = reinterpret_cast<const uint4 *>(src);
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    const int cores_img = 2 * 3 * NC;
    const int total = 9 * NKS * cores_img * 8;
    for (int e = tid; e < total; e += nthreads) {
        const int u = e & 7, core = e >> 3;
        const int nip = core % (3 * NC), ki = (core / (3 * NC)) & 1, img = core / cores_img;
        const int sk = img % NKS, kx = (img / NKS) % 3, rho = img / (3 * NKS);
        const int b = nip / NC, ni = nip % NC;
        const int ky = (rho + 4 - b) % 3, tap = 3 * ky + kx;
        d[e] = __ldg(s + ((size_t)((tap * NKS + sk) * 2 * NC + ki * NC + ni) * 8 + u));
    }
}

template <int NH, int NG>
__global__ void __launch_bounds__(LearnCfg<NH, NG>::THREADS, 1) learned_step_kernel(const LearnArgs a)
{
    using C = LearnCfg<NH, NG>;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *sW1 = smem + C::OFF_W1;
    unsigned char *sW2 = smem + C::OFF_W2;
    unsigned char *sW3 = smem + C::OFF_W3;
    unsigned char *sX0 = smem + C::OFF_X0;
    unsigned char *sA1 = smem + C::OFF_A1;
    unsigned char *sA2 = smem + C::OFF_A2;
    float *sLW = reinterpret_cast<float *>(smem + C::OFF_LW);
    float *sXR = reinterpret_cast<float *>(smem + C::OFF_XR);
    float *sBias = reinterpret_cast<float *>(smem + C::OFF_BIAS);
    double *sRed = reinterpret_cast<double *>(smem + C::OFF_RED);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + C::OFF_BAR);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + B_COUNT);
    volatile int *sAbort = reinterpret_cast<volatile int *>(bars + B_COUNT) + 1;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        mbar_init(bars + B_RDY1, C::NCW);
        mbar_init(bars + B_RDY2, C::NCW - C::PX / 32);  // group 1: layer 2's epilogue
        mbar_init(bars + B_RDY3, C::PX / 32);            // group 0: the output stage
        mbar_init(bars + B_L1, 1);
        mbar_init(bars + B_L2, 1);
        mbar_init(bars + B_L3, 1);
        mbar_init(bars + B_FIN, 1);
        fence_mbar_init();
        *sAbort = 0;
    }
    // weights (rotated, concatenated), bias, and zeroed rings
    rotate_weights(a.w1, sW1, 4, 1, tid, C::THREADS);
    rotate_weights(a.w2, sW2, 4, 2, tid, C::THREADS);
    rotate_weights(a.w3, sW3, 2, 2, tid, C::THREADS);
    for (int i = tid; i < 80; i += C::THREADS) sBias[i] = a.bias[i];
    {
        uint4 *z = reinterpret_cast<uint4 *>(sX0);
        const int nz = (int)((C::OFF_LW - C::OFF_X0) / 16);
        for (int i = tid; i < nz; i += C::THREADS) z[i] = zero4();
    }
    fence_proxy_async_smem();
    if (warp == C::NCW) tc::tmem_alloc(tslot, C::TMEM_COLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;

    if (warp == C::NCW) {
        // ------------------------------------------------------------------
        // MMA issue.  Batch t of a sweep: layer 1 on input row t, layer 2 on
        // row t-2, layer 3 on row t-4 (rows outside the grid skipped).  The
        // whole warp runs the loop so that the operands stay warp-uniform;
        // one elected lane issues.
        // ------------------------------------------------------------------
        constexpr uint32_t id96 = tc::idesc_bf16(128, 96), id64 = tc::idesc_bf16(128, 64);
        constexpr uint32_t id48 = tc::idesc_bf16(128, 48), id32 = tc::idesc_bf16(128, 32);
        // Descriptors of the first byte of each operand region; an operand
        // at byte offset o has descriptor base + (o >> 4) (the address field
        // holds addr >> 4 and shared memory is < 256 KB, so the sum never
        // carries out of it).
        const uint64_t dX0 = tc::smem_desc(sX0, C::STRIP, 128), dA1 = tc::smem_desc(sA1, C::STRIP, 128),
                       dA2 = tc::smem_desc(sA2, C::STRIP, 128);
        const uint64_t dW1 = tc::smem_desc(sW1, 12 * 128, 128), dW2 = tc::smem_desc(sW2, 12 * 128, 128),
                       dW3 = tc::smem_desc(sW3, 6 * 128, 128);
        // All MMAs of input row j of one layer: kx, K steps, half rows.  Row
        // 0 has no output row -1 (whose block is row 2's): N covers blocks
        // 0 and 1 only.
        auto layer = [&](uint64_t dA, int row_bytes, int j, int nks, uint64_t dW, int img, uint32_t acc, int ncol3,
                         uint32_t idesc_full, uint32_t idesc_first) {
            const uint32_t idesc = j == 0 ? idesc_first : idesc_full;
            const int rho = mod3(j);
#pragma unroll
            for (int kx = 0; kx < 3; ++kx)
#pragma unroll
                for (int sk = 0; sk < 2; ++sk) {
                    if (sk >= nks) break;
                    const uint32_t ao = (uint32_t)((j & 1) * row_bytes) + (uint32_t)(2 * sk * C::STRIP) +
                                        (uint32_t)(kx * 16);
                    const uint32_t bo = (uint32_t)(((rho * 3 + kx) * nks + sk) * img);
#pragma unroll
                    for (int hh = 0; hh < NH; ++hh)
                        tc::mma_bf16(acc + (uint32_t)(hh * ncol3), dA + ((ao + (uint32_t)(2048 * hh)) >> 4),
                                     dW + (bo >> 4), idesc, true);
                }
        };
        // Waits (whole warp) for phase ``par`` of ``bar``; false once anything
        // has given up.
        auto wait_all = [&](uint64_t *bar, uint32_t par) {
            bool go = !*sAbort && mbar_wait_bounded(bar, par, a.err);
            go = __all_sync(0xffffffffu, go);
            if (!go && lane == 0) *sAbort = 1;
            tc::fence_after_sync();
            return go;
        };
        uint32_t nb = 0;
        for (int i = blockIdx.x; i < a.n_inst; i += gridDim.x) {
            const int H = a.inst[i].ny;
            const int T = H + 6;
            for (int k = 0; k < a.n_steps; ++k) {
                for (int t = 0; t + 1 < T; ++t, ++nb) {
                    const uint32_t par = nb & 1u;
                    if (!wait_all(bars + B_RDY1, par)) continue;
                    if (elect_one()) {
                        if (t < H) layer(dX0, C::X0_ROW, t, 1, dW1, (int)C::IMG1, tmem + C::ACC1, 96, id96, id64);
                        tc::commit(bars + B_L1);
                    }
                    __syncwarp();
                    if (!wait_all(bars + B_RDY2, par)) continue;
                    if (elect_one()) {
                        if (t - 2 >= 0 && t - 2 < H)
                            layer(dA1, C::A_ROW, t - 2, 2, dW2, (int)C::IMG2, tmem + C::ACC2, 96, id96, id64);
                        tc::commit(bars + B_L2);
                    }
                    __syncwarp();
                    if (!wait_all(bars + B_RDY3, par)) continue;
                    if (elect_one()) {
                        if (t - 4 >= 0 && t - 4 < H)
                            layer(dA2, C::A_ROW, t - 4, 2, dW3, (int)C::IMG3, tmem + C::ACC3, 48, id48, id32);
                        tc::commit(bars + B_L3);
                    }
                    __syncwarp();
                }
            }
        }
        // every MMA issued has completed before the accumulators are freed
        if (elect_one()) tc::commit(bars + B_FIN);
        __syncwarp();
        mbar_wait_bounded(bars + B_FIN, 0, a.err);
        __syncwarp();
    } else {
        // ------------------------------------------------------------------
        // Compute warps.  Warp w reads TMEM lanes 32 (w % 4) .. +31: pixel
        // px = 128 hh + 32 q + lane of half hh, channel group g.  Group 0
        // (PX threads, one per pixel) also runs the Lax-Wendroff step, the
        // output stage and the mass sums; group 1 all of layer 2's epilogue.
        // ------------------------------------------------------------------
        const int q = warp & 3, hh = (warp >> 2) % NH, g = warp / (4 * NH);
        const int px = 128 * hh + 32 * q + lane;
        const bool lw_thread = g == 0;
        const uint32_t tl = (uint32_t)(32 * q) << 16;
        // this thread's accumulator columns (block 0) of each layer
        const int ch = g == 0 ? 0 : C::C0;  // this thread's first hidden channel
        const uint32_t t1 = tmem + tl + C::ACC1 + hh * 96 + ch;
        const uint32_t t3 = tmem + tl + C::ACC3 + hh * 48;
        const int sw = (ch / 8) * C::STRIP + (px + 1) * 16;  // ring offset of this thread's layer-1 strips
        const uint32_t t2a = tmem + tl + C::ACC2 + hh * 96;   // layer 2, all 32 channels (group 1)
        const int sw2 = (px + 1) * 16;
        // the hidden-layer epilogue with this group's channel count
        auto epilogue = [&](uint32_t taddr, const float *bias, unsigned char *dst, bool valid) {
            if (g == 0) {
                if constexpr (C::C0 > 0) hidden_epilogue<C::C0>(taddr, bias, dst, C::STRIP, valid);
            } else {
                if constexpr (C::C1 > 0) hidden_epilogue<C::C1>(taddr, bias, dst, C::STRIP, valid);
            }
        };
        auto arm_hidden = [&](uint32_t taddr, const float *bias) {
            if (g == 0) {
                if constexpr (C::C0 > 0) arm<C::C0>(taddr, bias);
            } else {
                if constexpr (C::C1 > 0) arm<C::C1>(taddr, bias);
            }
        };
        uint32_t nb = 0;  // batches of the finished sweeps
        // waits for ``bar`` (per thread); records a give-up for everyone
        auto wait = [&](uint64_t *bar, uint32_t par) {
            if (!mbar_try_wait(bar, par) && !*sAbort && !mbar_wait_bounded(bar, par, a.err)) *sAbort = 1;
            __syncwarp();
            tc::fence_after_sync();
        };
        for (int i = blockIdx.x; i < a.n_inst; i += gridDim.x) {
            const BatchInst I = a.inst[i];
            const int W = I.nx, H = I.ny, T = H + 6;
            const long long pitch = I.pitch, plane = I.plane;
            const Coef<float> kc = I.k;
            const bool inside = px < W;
            float m = 0.0f;  // pending h offset of the state being read
            bool bad = false;
            for (int step = 0; step < a.n_steps; ++step) {
                const int cb = (a.parity0 + step) & 1;
                const float *src = cb ? I.buf[1] : I.buf[0];
                float *dst = cb ? I.buf[0] : I.buf[1];
                CellQ<float> cur = {}, nxt = {};
                Flux3<float> gd = {};
                float ph = 0.0f, pu = 0.0f, pv = 0.0f;  // prefetched raw row
                auto load_cell = [&](int r) {
                    const long long o = (long long)r * pitch + px;
                    const float h = src[o] - m;
                    bad |= !(h > 0.0f);
                    return make_cell<float>(h, src[o + plane], src[o + 2 * plane], kc.hg);
                };
                if (lw_thread && inside) {
                    cur = load_cell(0);
                    if (H > 1) nxt = load_cell(1);
                    if (H > 2) {
                        const long long o = 2 * pitch + px;
                        ph = src[o];
                        pu = src[o + plane];
                        pv = src[o + 2 * plane];
                    }
                    gd = yface_flux(mirror_y(cur), cur, kc);
                }
                // every accumulator block starts from the bias (all MMAs of
                // the previous sweep have completed: its last tick waited
                // for them)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    arm_hidden(t1 + b * 32, sBias + ch);
                    if (lw_thread) {
                        tc::st_x4_async(t3 + b * 16, sBias + 64);
                        tc::wait_st();
                    } else {
                        arm<32>(t2a + b * 32, sBias + 32);
                    }
                }
                double hs = 0.0;  // this pixel's h corrections: FP32 sums of 16 rows, added in FP64
                float hs16 = 0.0f;
                int lws = 0;  // lw ring slot of row t (t mod 7)
#pragma unroll 1
                for (int t = 0; t < T; ++t, lws = lws == C::LW_SLOTS - 1 ? 0 : lws + 1) {
                    const uint32_t parW = (nb + (uint32_t)t - 1u) & 1u;  // batch t-1
                    const bool publish_t = t + 1 < T;
                    // ---- Lax-Wendroff row t; network input x0[t] ----
                    if (lw_thread && t < H) {
                        // the row's cells (state and x-fluxes) for the
                        // neighbours' x-faces
                        float *xr = sXR + (t & 1) * 5 * C::PXB;
                        if (inside) {
                            xr[px + 1] = cur.h;
                            xr[C::PXB + px + 1] = cur.u;
                            xr[2 * C::PXB + px + 1] = cur.v;
                            xr[3 * C::PXB + px + 1] = cur.f2;
                            xr[4 * C::PXB + px + 1] = cur.f3;
                        }
                        named_bar_sync(1, C::PX);
                        uint4 x8 = zero4();
                        if (inside) {
                            // a neighbour's h, hu, hv, f2, f3 as its own thread
                            // formed them (g3 is not read by an x-face)
                            auto xcell = [&](int i) {
                                CellQ<float> c;
                                c.h = xr[i];
                                c.u = xr[C::PXB + i];
                                c.v = xr[2 * C::PXB + i];
                                c.f2 = xr[3 * C::PXB + i];
                                c.f3 = xr[4 * C::PXB + i];
                                c.g3 = 0.0f;
                                return c;
                            };
                            const CellQ<float> left = px == 0 ? mirror_x(cur) : xcell(px);
                            const CellQ<float> right = px == W - 1 ? mirror_x(cur) : xcell(px + 2);
                            const CellQ<float> up = t + 1 < H ? nxt : mirror_y(cur);
                            const Flux3<float> Fl = xface_flux(left, cur, kc);
                            const Flux3<float> Fr = xface_flux(cur, right, kc);
                            const Flux3<float> gu = yface_flux(cur, up, kc);
                            float oh = cur.h, ou = cur.u, ov = cur.v;
                            lw_update(oh, ou, ov, Fl, Fr, gd, gu, kc);
                            bad |= !(oh > 0.0f);
                            float *lw = sLW + lws * 3 * C::PX;
                            lw[px] = oh;
                            lw[C::PX + px] = ou;
                            lw[2 * C::PX + px] = ov;
                            x8.x = pack_bf16x2((oh - cur.h) * a.inv_sh, (ou - cur.u) * a.inv_su);
                            x8.y = pack_bf16x2((ov - cur.v) * a.inv_su, 0.0f);
                            gd = gu;
                            if (t + 1 < H) {
                                cur = nxt;
                                if (t + 2 < H) {
                                    const float h = ph - m;
                                    bad |= !(h > 0.0f);
                                    nxt = make_cell<float>(h, pu, pv, kc.hg);
                                    if (t + 3 < H) {
                                        const long long o = (long long)(t + 3) * pitch + px;
                                        ph = src[o];
                                        pu = src[o + plane];
                                        pv = src[o + 2 * plane];
                                    }
                                }
                            }
                        }
                        // slot t & 1 held x0[t-2], read by batch t-2 (waited in tick t-1)
                        *reinterpret_cast<uint4 *>(sX0 + (t & 1) * C::X0_ROW + (px + 1) * 16) = x8;
                    }
                    // ---- E1 of row t-2 (completed by batch t-1) ----
                    // Its a1 slot was last read by layer 2's batch t-2.  A
                    // commit tracks every MMA its thread issued before it
                    // (one lane issues them all: elect.sync on the converged
                    // MMA warp elects the same lane every time), so the wait
                    // on layer 1's batch t-1 (issued after layer 2's batch
                    // t-2) also covers that read: group 0 needs no wait on
                    // layer 2.  Likewise layer 2's wait on batch t-1
                    // covers layer 3's batch t-2, the last reader of the a2
                    // slot that E2 rewrites.
                    if (t >= 1) wait(bars + B_L1, parW);
                    const int r1 = t - 2;
                    if (r1 >= 0 && r1 < H)
                        epilogue(t1 + mod3(r1) * 32, sBias + ch, sA1 + (r1 & 1) * C::A_ROW + sw, inside);
                    if (publish_t) publish(bars + B_RDY1, lane);
                    // ---- E2 of row t-4 (group 1) ----
                    if (!lw_thread) {
                        if (t >= 1) wait(bars + B_L2, parW);
                        const int r2 = t - 4;
                        if (r2 >= 0 && r2 < H)
                            hidden_epilogue<32>(t2a + mod3(r2) * 32, sBias + 32, sA2 + (r2 & 1) * C::A_ROW + sw2,
                                                C::STRIP, inside);
                        if (publish_t) publish(bars + B_RDY2, lane);
                    }
                    // ---- E3: corrected row t-6 (group 0) ----
                    if (lw_thread && t >= 1) wait(bars + B_L3, parW);
                    const int r3 = t - 6;
                    if (lw_thread && r3 >= 0 && r3 < H) {
                        // only columns 0..2 of a layer-3 block are outputs
                        // (the padding columns are never read): four
                        // columns are read and re-armed
                        const uint32_t ta = t3 + mod3(r3) * 16;
                        uint32_t v4[4];
                        tc::ld_x4_async(ta, v4);
                        tc::wait_ld(v4);
                        tc::st_x4_async(ta, sBias + 64);
                        const float v[3] = {__uint_as_float(v4[0]), __uint_as_float(v4[1]), __uint_as_float(v4[2])};
                        if (inside) {
                            const int s3 = lws >= 6 ? lws - 6 : lws + 1;  // (t - 6) mod 7
                            const float *lw = sLW + s3 * 3 * C::PX;
                            const long long o = (long long)r3 * pitch + px;
                            dst[o] = __fmaf_rn(v[0], a.os_h, lw[px]);
                            dst[o + plane] = __fmaf_rn(v[1], a.os_u, lw[C::PX + px]);
                            dst[o + 2 * plane] = __fmaf_rn(v[2], a.os_u, lw[2 * C::PX + px]);
                            hs16 += v[0] * a.os_h;
                        }
                        if ((r3 & 15) == 15 || r3 == H - 1) {
                            hs += (double)hs16;
                            hs16 = 0.0f;
                        }
                        tc::wait_st();
                    }
                    if (lw_thread && publish_t) publish_tmem(bars + B_RDY3, lane);
                }
                nb += (uint32_t)(T - 1);
                // ---- mass projection: the mean h correction becomes the pending offset ----
                if (lw_thread) {
                    double s = hs;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                    if (lane == 0) sRed[warp] = s;
                    named_bar_sync(1, C::PX);
                    double tot = 0.0;
                    for (int w = 0; w < 4 * NH; ++w) tot += sRed[w];
                    m = a.project ? (float)(tot / ((double)W * (double)H)) : 0.0f;
                }
            }
            // ---- the final state: apply the pending offset, check the depth ----
            if (lw_thread && inside && a.n_steps > 0) {
                float *h = ((a.parity0 + a.n_steps) & 1) ? I.buf[1] : I.buf[0];
                for (int r = 0; r < H; ++r) {
                    const long long o = (long long)r * pitch + px;
                    const float v = h[o] - m;
                    if (m != 0.0f) h[o] = v;
                    bad |= !(v > 0.0f);
                }
            }
            if (lw_thread && bad) atomicOr(&a.flags[i], SWE_FLAG_NONPOSITIVE);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == C::NCW) tc::tmem_free(tmem, C::TMEM_COLS);
}

template <int NH, int NG>
cudaError_t launch_learned(const LearnArgs &a, int grid, cudaStream_t s)
{
    using C = LearnCfg<NH, NG>;
    static_assert(C::SMEM <= 232448, "shared memory of the fused learned step");
    static_assert(8 * B_COUNT + 8 <= 128, "barrier area");
    static_assert(C::TMEM_USED <= C::TMEM_COLS, "tensor memory");
    static_assert(C::OFF_BIAS % 16 == 0, "bias is read as float4");
    auto kern = learned_step_kernel<NH, NG>;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once,
                   [&] { attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM); });
    if (attr != cudaSuccess) return attr;
    kern<<<grid, C::THREADS, C::SMEM, s>>>(a);
    return cudaGetLastError();
}

}  // namespace
}  // namespace swe

using namespace swe;

extern "C" swe_status swe_batch_learned_step(swe_batch *b, swe_net *net, int n_steps, int project_mass, void *stream)
{
    BatchView bv;
    NetView nv;
    if (!batch_view(b, &bv) || !net_view(net, &nv) || n_steps < 0) return SWE_EINVAL;
    if (n_steps == 0) return SWE_OK;
    int wmax = 0;
    for (int i = 0; i < bv.n; ++i) wmax = std::max(wmax, bv.h_inst[i].nx);
    if (wmax > 256) return SWE_EUNSUPPORTED;
    LearnArgs a;
    a.inst = bv.d_inst;
    a.n_inst = bv.n;
    a.n_steps = n_steps;
    a.parity0 = bv.cur;
    a.w1 = nv.w1;
    a.w2 = nv.w2;
    a.w3 = nv.w3;
    a.bias = nv.bias;
    a.inv_sh = 1.0f / nv.norm[1];
    a.inv_su = 1.0f / nv.norm[2];
    a.os_h = nv.norm[3];
    a.os_u = nv.norm[4];
    a.project = project_mass ? 1 : 0;
    a.flags = bv.d_flags;
    a.err = bv.d_err;
    const int grid = std::min(bv.n, std::max(1, bv.sms));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const cudaError_t e = wmax <= 128 ? launch_learned<1, SWE_LEARN_NG>(a, grid, s)
                                      : launch_learned<2, SWE_LEARN_NG>(a, grid, s);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? SWE_ENOMEM : SWE_ECUDA;
    batch_advance(b, n_steps);
    return SWE_OK;
}
