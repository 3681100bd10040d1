// swe_batch.cu -- batched ensembles: many independent FP32 grids of
// different sizes, each with its own dx, dy and dt, advanced together by ONE
// persistent, cooperatively launched kernel that runs all requested steps.
//
// Work list: every instance is cut into tiles of TX x TY cells; the tiles of
// all instances form one flat list (instance-major, so the CTAs working at
// the same time share halo rows in L2).  CTAs stride over the list; each tile
// is staged by TMA (three box loads on one mbarrier, double buffered so the
// next tile's loads overlap this tile's arithmetic; each warp hands a stage
// back on a second mbarrier once it has read it, and only the thread that
// refills the stage waits for that) and computed by the same tile routine as
// the single-grid kernel (swe_tile.cuh).  A grid-wide barrier with a bounded
// wait separates the time steps; all instances step together.
//
// Streaming variants (two steps per pass): warps stream up 120-column strips
// of the instances as the single-grid default does (swe_stream.cuh), taking
// (instance, strip, row range) segments longest first from a pass counter.
//
// The launch is captured once per (step count, buffer parity) into a CUDA
// graph on a private stream and replayed on the caller's stream.  Tile shape,
// staging depth and CTAs per SM come from the autotuner (swe_batch_tune),
// which times each candidate on the batch itself and caches the winner in a
// JSON-lines file.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "swe_stream.cuh"
#include "swe_tile.cuh"
#include "swe_views.cuh"

namespace swe {

struct TileRec {
    int inst;
    unsigned short bx, by;  // tile column / row within the instance
};

// ---------------------------------------------------------------------------
// The persistent kernel
// ---------------------------------------------------------------------------
template <int NWARP, int RY, int STAGES>
struct BatchCfg {
    using C = TiledCfg<float, NWARP, RY>;
    static constexpr size_t STAGE_BYTES = 3 * C::BOX_STRIDE;
    static constexpr size_t SMEM = STAGES * STAGE_BYTES + 64;
};

// A warp's release of a staged tile: one arrival on the stage's "empty"
// barrier (NWARP arrivals complete a phase), after all its lanes have read
// the stage.
__device__ __forceinline__ void stage_release(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

template <int NWARP, int RY, int STAGES>
__global__ void __launch_bounds__(NWARP * 32) batch_lw_kernel(const BatchInst *__restrict__ inst,
                                                              const CUtensorMap *__restrict__ maps,
                                                              const TileRec *__restrict__ tiles, int ntiles,
                                                              int n_steps, int parity0, GridBarrier *gbar,
                                                              int *err, int *flags)
{
    using B = BatchCfg<NWARP, RY, STAGES>;
    using C = typename B::C;
    extern __shared__ __align__(128) unsigned char smem[];
    // per stage: "full" (the TMA boxes landed; one arrival + the bytes) and
    // "empty" (every warp is done with the boxes; NWARP arrivals)
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * B::STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NWARP);
        }
        fence_mbar_init();
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;

    auto box = [&](int stage, int f) {
        return reinterpret_cast<float *>(smem + stage * B::STAGE_BYTES + f * C::BOX_STRIDE);
    };
    // thread 0: once every warp has released ``stage``'s previous tile, start
    // the three TMA loads of tile t (buffer ``cur``) into it; false if that
    // wait gave up
    uint32_t used = 0, epar = 0;  // bit s: stage s was filled before / parity of its next release
    auto issue = [&](int t, int stage, int cur) -> bool {
        if ((used >> stage) & 1u) {
            if (!mbar_wait_bounded(&empty[stage], (epar >> stage) & 1u, err)) return false;
            epar ^= 1u << stage;
        }
        used |= 1u << stage;
        const TileRec r = tiles[t];
        const CUtensorMap *m = maps + ((size_t)r.inst * 2 + cur) * 3;
        const int x0 = (int)r.bx * C::TX, y0 = (int)r.by * C::TY;
        mbar_arrive_expect_tx(&full[stage], (uint32_t)(3 * C::BOX_BYTES));
        tma_load_2d(box(stage, 0), m + 0, &full[stage], x0 - C::AX, y0 - 1);
        tma_load_2d(box(stage, 1), m + 1, &full[stage], x0 - C::AX, y0 - 1);
        tma_load_2d(box(stage, 2), m + 2, &full[stage], x0 - C::AX, y0 - 1);
        return true;
    };

    uint32_t phases = 0;  // bit s = parity of the next completion of full[s]
    for (int step = 0; step < n_steps; ++step) {
        const int cur = (parity0 + step) & 1;
        if (threadIdx.x == 0 && (int)blockIdx.x < ntiles) {
            fence_proxy_async_global();  // other CTAs' stores of the last step -> TMA reads
            if (!issue(blockIdx.x, 0, cur)) return;
        }
        int it = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
            const int st = STAGES > 1 ? (it & 1) : 0;
            const int tn = t + gridDim.x;
            // the tile's record and its instance's parameters: two dependent
            // global loads, issued before the waits so that they overlap them
            const TileRec r = tiles[t];
            const BatchInst *I = inst + r.inst;
            float *o = I->buf[cur ^ 1];
            const long long plane = I->plane, pitch = I->pitch;
            const int nx = I->nx, ny = I->ny;
            const Coef<float> k = I->k;
            if (STAGES > 1 && threadIdx.x == 0 && tn < ntiles && !issue(tn, st ^ 1, cur)) return;
            if (!mbar_wait_bounded(&full[st], (phases >> st) & 1u, err)) {
                // give the other stage's prefetch (if any) a bounded chance to land
                if (STAGES > 1 && tn < ntiles) mbar_wait_bounded(&full[st ^ 1], (phases >> (st ^ 1)) & 1u, err);
                return;
            }
            phases ^= 1u << st;

            const int x0 = (int)r.bx * C::TX, y0 = (int)r.by * C::TY;
            bool bad;
            if (x0 == 0 || x0 + C::TX >= nx)
                bad = tiled_compute<float, NWARP, RY, true>(box(st, 0), box(st, 1), box(st, 2), o, o + plane,
                                                            o + 2 * plane, nx, ny, pitch, x0, y0, k);
            else
                bad = tiled_compute<float, NWARP, RY, false>(box(st, 0), box(st, 1), box(st, 2), o, o + plane,
                                                             o + 2 * plane, nx, ny, pitch, x0, y0, k);
            // the warp is done with this stage: flag, then release it (no
            // CTA barrier, so a warp may run one tile ahead of the slowest)
            if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&flags[r.inst], SWE_FLAG_NONPOSITIVE);
            __syncwarp();
            if (lane == 0) stage_release(&empty[st]);
            if (STAGES == 1 && threadIdx.x == 0 && tn < ntiles && !issue(tn, 0, cur)) return;
        }
        if (!grid_sync_bounded(gbar, gridDim.x, err)) return;
    }
}

// ---------------------------------------------------------------------------
// The same with temporal blocking: two steps per pass over the tile list.
// Each tile is staged with a two-cell y-halo (one TMA box of TY + 4 rows per
// field) and advanced twice by tb2_tile_compute into the other buffer; a
// grid barrier separates the passes.  An odd last step takes one step from
// the same box (tile row 0 at box row 2).  Same bits as the one-step
// kernels; DRAM sees each cell once per two steps (plus the halo rows).
// ---------------------------------------------------------------------------
template <int NWARP, int RY>
__global__ void __launch_bounds__(NWARP * 32) batch_tb2_kernel(const BatchInst *__restrict__ inst,
                                                               const CUtensorMap *__restrict__ maps,
                                                               const TileRec *__restrict__ tiles, int ntiles,
                                                               int n_steps, int parity0, GridBarrier *gbar, int *err,
                                                               int *flags)
{
    using B = Tb2Cfg<float, NWARP, RY>;
    using C = typename B::C;
    extern __shared__ __align__(128) unsigned char smem[];
    float *iH = reinterpret_cast<float *>(smem);
    float *iU = reinterpret_cast<float *>(smem + B::IN_STRIDE);
    float *iV = reinterpret_cast<float *>(smem + 2 * B::IN_STRIDE);
    float *mH_ = reinterpret_cast<float *>(smem + 3 * B::IN_STRIDE);
    float *mU_ = reinterpret_cast<float *>(smem + 3 * B::IN_STRIDE + C::BOX_STRIDE);
    float *mV_ = reinterpret_cast<float *>(smem + 3 * B::IN_STRIDE + 2 * C::BOX_STRIDE);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 3 * B::IN_STRIDE + 3 * C::BOX_STRIDE);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    int cur = parity0;
    const int pairs = n_steps / 2, passes = pairs + (n_steps & 1);
    for (int p = 0; p < passes; ++p, cur ^= 1) {
        const bool two = p < pairs;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const TileRec r = tiles[t];
            const int x0 = (int)r.bx * C::TX, y0 = (int)r.by * C::TY;
            // the instance's parameters, loaded before the barrier and the wait
            const BatchInst *I = inst + r.inst;
            float *o = I->buf[cur ^ 1];
            const long long plane = I->plane, pitch = I->pitch;
            const int nx = I->nx, ny = I->ny;
            const Coef<float> k = I->k;
            __syncthreads();  // the previous tile is done with the boxes
            if (threadIdx.x == 0) {
                const CUtensorMap *m = maps + ((size_t)r.inst * 2 + cur) * 3;
                fence_proxy_async_global();  // other CTAs' stores of the last pass -> TMA reads
                mbar_arrive_expect_tx(bar, (uint32_t)(3 * B::IN_BYTES));
                tma_load_2d(iH, m + 0, bar, x0 - C::AX, y0 - 2);
                tma_load_2d(iU, m + 1, bar, x0 - C::AX, y0 - 2);
                tma_load_2d(iV, m + 2, bar, x0 - C::AX, y0 - 2);
            }
            if (!__syncthreads_and(mbar_wait_bounded(bar, phase, err))) return;
            phase ^= 1u;
            bool bad;
            if (two)
                bad = tb2_tile_compute<float, NWARP, RY>(iH, iU, iV, mH_, mU_, mV_, o, o + plane, o + 2 * plane, nx,
                                                          ny, pitch, x0, y0, k);
            else if (x0 == 0 || x0 + C::TX >= nx)
                bad = tiled_compute<float, NWARP, RY, true, 2>(iH, iU, iV, o, o + plane, o + 2 * plane, nx, ny, pitch,
                                                               x0, y0, k);
            else
                bad = tiled_compute<float, NWARP, RY, false, 2>(iH, iU, iV, o, o + plane, o + 2 * plane, nx, ny,
                                                                pitch, x0, y0, k);
            if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&flags[r.inst], SWE_FLAG_NONPOSITIVE);
        }
        if (!grid_sync_bounded(gbar, gridDim.x, err)) return;
    }
}

// ---------------------------------------------------------------------------
// Two steps per pass by streaming warps (stream_segment, swe_stream.cuh):
// every instance is cut into column strips and the strips into row ranges;
// in every pass the warps take these segments, longest first, from a shared
// counter, one step in the last pass of an odd count.  The work buffer holds
// two pass counters (zeroed before each launch; pass p counts on p & 1 and
// resets the other for pass p + 1) and then the segments.
// ---------------------------------------------------------------------------
struct SegRec {
    int inst;
    int strip;  // column strip: columns strip * OUT ..
    int ya, yb; // output rows [ya, yb)
};
constexpr int kWorkHead = 4;  // ints before the segments: two counters, padded to 16 bytes
static_assert(sizeof(SegRec) == 4 * sizeof(int), "segments are four ints");

template <int VP, int LO, int NO, int CR, int NSLOT, int WARPS, int MINB>
__global__ void __launch_bounds__(WARPS * 32, MINB)
    batch_stream_kernel(const BatchInst *__restrict__ inst, const CUtensorMap *__restrict__ maps, void *work,
                        int nsegs, int n_steps, int parity0, GridBarrier *gbar, int *err, int *flags)
{
    using C = StreamCfg<VP, LO, NO, CR, NSLOT, WARPS>;
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    StreamWarp<VP, LO, NO, CR, NSLOT, WARPS> w;
    w.ring = smem + (size_t)warp * C::WARP_BYTES;
    w.bars = reinterpret_cast<uint64_t *>(smem + WARPS * C::WARP_BYTES) + warp * NSLOT;
    w.phase = 0;
    w.err = err;
    if (lane == 0) {
        for (int i = 0; i < NSLOT; ++i) mbar_init(w.bars + i, 1);
        fence_mbar_init();
    }
    __syncwarp();
    int *ctr = static_cast<int *>(work);
    const SegRec *segs = reinterpret_cast<const SegRec *>(ctr + kWorkHead);
    bool ok = true;
    int cur = parity0;
    const int pairs = n_steps / 2, passes = pairs + (n_steps & 1);
    for (int p = 0; p < passes; ++p, cur ^= 1) {
        const bool two = p < pairs;
        // the next pass's counter was last used two passes ago
        if (blockIdx.x == 0 && threadIdx.x == 0) ctr[(p + 1) & 1] = 0;
        // other warps' stores of the last pass -> this warp's TMA reads
        if (lane == 0) fence_proxy_async_global();
        for (;;) {
            int i = 0;
            if (lane == 0) i = atomicAdd(ctr + (p & 1), 1);
            i = __shfl_sync(kFull, i, 0);
            if (i >= nsegs || !ok) break;
            const SegRec r = segs[i];
            const BatchInst *I = inst + r.inst;
            const CUtensorMap *m = maps + ((size_t)r.inst * 2 + cur) * 3;
            w.mH = m;
            w.mU = m + 1;
            w.mV = m + 2;
            float *o = I->buf[cur ^ 1];
            const long long plane = I->plane, pitch = I->pitch;
            const int nx = I->nx, ny = I->ny;
            const Coef2 k2 = coef2(I->k);
            const int xs = r.strip * C::OUT;
            // Every strip takes the wall code path (the ghost patch changes
            // nothing where no ghost column is in reach).  With instances a
            // few strips wide, about 40 % of the strips hold a wall; one copy
            // of the row loop instead of two cuts instruction-fetch stalls
            // and spills and measured 18 % faster (0.468 against 0.568 ms per
            // step on the 512-grid ensemble at 3 CTAs/SM).
            // The cells are paired (c_0, c_2), (c_1, c_3) in each lane: the
            // x-face pairs then line up without regrouping, and this kernel
            // (one copy of the row loop, more live state than the
            // single-grid one) measured 3 % faster so; the single-grid
            // kernel keeps (c_0, c_1), (c_2, c_3), which its compiled code
            // favours.  Either pairing gives the same bits.
            bool bad = false;
            float *oh = o, *ou = o + plane, *ov = o + 2 * plane;
            if (two)
                ok = stream_segment<true, VP, LO, NO, CR, NSLOT, WARPS, false, true>(w, oh, ou, ov, nx, ny, pitch, xs,
                                                                                     r.ya, r.yb, k2, bad);
            else  // the one-step pass: an odd count's last
                ok = stream_segment<true, VP, LO, NO, CR, NSLOT, WARPS, true, true>(w, oh, ou, ov, nx, ny, pitch, xs,
                                                                                    r.ya, r.yb, k2, bad);
            if (__any_sync(kFull, bad) && lane == 0) atomicOr(&flags[r.inst], SWE_FLAG_NONPOSITIVE);
        }
        // every warp reaches the barrier, also after a timed-out wait
        if (!grid_sync_bounded(gbar, gridDim.x, err)) return;
    }
}

// ---------------------------------------------------------------------------
// Variants the autotuner chooses from
// ---------------------------------------------------------------------------
struct Variant {
    int nwarp, ry, stages, depth;
    int tile_x, tile_y, box_w, box_h;
    size_t smem;
    const void *func;
    int kind = 0;  // 0: tiles (tile list), 1: streaming warps (segment schedule)
};

template <int NWARP, int RY, int STAGES>
static Variant make_variant()
{
    using B = BatchCfg<NWARP, RY, STAGES>;
    using C = typename B::C;
    return Variant{NWARP, RY, STAGES, 1, C::TX, C::TY, C::BW, C::BH, B::SMEM,
                   reinterpret_cast<const void *>(&batch_lw_kernel<NWARP, RY, STAGES>)};
}

template <int NWARP, int RY>
static Variant make_variant_tb2()
{
    using B = Tb2Cfg<float, NWARP, RY>;
    using C = typename B::C;
    return Variant{NWARP, RY, 1, 2, C::TX, C::TY, C::BW, B::BH_IN, B::SMEM,
                   reinterpret_cast<const void *>(&batch_tb2_kernel<NWARP, RY>)};
}

// Streaming warps: two pairs per lane, 120-column strips, two 4-row chunks,
// 4 warps per CTA, registers for 3 CTAs per SM (as the single-grid default).
using BatchStreamC = StreamCfg<2, 1, 30, 4, 2, 4>;
template <int MINB>
static Variant make_variant_stream()
{
    using C = BatchStreamC;
    Variant v{4, C::ROWS, 2, 2, C::OUT, 0, C::BW, C::ROWS, C::SMEM,
              reinterpret_cast<const void *>(&batch_stream_kernel<2, 1, 30, 4, 2, 4, MINB>)};
    v.kind = 1;
    return v;
}

// Buffer swaps (= launches of a step pass) that n steps take with a variant.
static int swaps_of(const Variant &V, int n) { return V.depth == 2 ? n / 2 + (n & 1) : n; }

static const std::vector<Variant> &variants()
{
    static const std::vector<Variant> v = {
        make_variant<4, 8, 2>(),   // 128x32 tiles, double-buffered
        make_variant<4, 4, 2>(),   // 128x16 tiles, double-buffered
        make_variant<4, 8, 1>(),   // 128x32 tiles, single stage
        make_variant<8, 4, 2>(),   // 128x32 tiles, 8 warps, double-buffered
        make_variant<4, 16, 1>(),  // 128x64 tiles, single stage
        make_variant_tb2<8, 4>(),  // two steps per pass: 128x32 tiles, 8 warps
        make_variant_tb2<4, 4>(),  // two steps per pass: 128x16 tiles
        make_variant_tb2<8, 2>(),  // two steps per pass: 128x16 tiles, 8 warps
        make_variant_stream<3>(),  // two steps per pass: streaming warps, 120-column strips, 3 CTAs/SM
        make_variant_stream<2>(),  // the same without the register cap (2 CTAs/SM)
    };
    return v;
}

bool encode_plane_map(CUtensorMap *map, int dtype, const void *base, int nx, int ny, long long pitch, int box_x,
                      int box_y);
size_t reduce_scratch_doubles_many(int n, int B);

// Wait probes for swe_selftest_wait: which = 0 waits on an mbarrier that no
// one arrives at, which = 1 on a grid barrier that expects one CTA more than
// the launch has.  Both give up after limit_ns and record SWE_ETIMEOUT.
__global__ void wait_probe_kernel(int which, unsigned long long limit_ns, GridBarrier *bar, int *err)
{
    __shared__ uint64_t mbar;
    if (which == 0) {
        if (threadIdx.x == 0) {
            mbar_init(&mbar, 2);
            fence_mbar_init();
        }
        __syncthreads();
        mbar_wait_bounded(&mbar, 0, err, limit_ns);
    } else {
        grid_sync_bounded(bar, gridDim.x + 1, err, limit_ns);
    }
}

static cudaError_t launch_wait_probe(int which, unsigned long long limit_ns, GridBarrier *bar, int *err,
                                     cudaStream_t s)
{
    wait_probe_kernel<<<which == 0 ? 1 : 4, 64, 0, s>>>(which, limit_ns, bar, err);
    return cudaGetLastError();
}

}  // namespace swe

using namespace swe;

struct swe_batch {
    int device = 0;
    int n = 0;
    double g = 9.8;
    std::vector<int> nx, ny;
    std::vector<double> dx, dy, dt;
    std::vector<long long> pitch, off;  // elements; off[i] = first element of instance i in a half
    size_t half = 0;                    // elements per half (all buffers of one parity)
    float *pool = nullptr;
    int cur = 0;
    std::vector<BatchInst> h_inst;
    BatchInst *d_inst = nullptr;
    CUtensorMap *d_maps = nullptr;               // maps of the configured variant
    std::map<int, CUtensorMap *> maps_by_box;  // by box (w, h); written once each, never rewritten
    TileRec *d_tiles = nullptr;
    int ntiles = 0, tiles_ty = -1, tiles_cap = 0;
    void *d_work = nullptr;  // streaming variant: pass counters + segments
    size_t work_cap = 0;     // bytes
    int nwork = 0;           // segments
    GridBarrier *d_bar = nullptr;
    int *d_err = nullptr;
    int *d_flags = nullptr;
    RedGrid *d_red[2] = {nullptr, nullptr};
    double *d_scratch = nullptr;
    double *d_out = nullptr;
    double *h_out = nullptr;
    int red_blocks = 32;
    int variant = 0, ctas_per_sm = 1, blocks = 0, sms = 0;
    cudaStream_t cap = nullptr;
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;
    bool graph_ok = true;
    long long launches = 0;
    int tuned = 0;
};

namespace swe {

bool batch_view(swe_batch *b, BatchView *v)
{
    if (!b || !v) return false;
    v->n = b->n;
    v->cur = b->cur;
    v->sms = b->sms;
    v->d_inst = b->d_inst;
    v->h_inst = b->h_inst.data();
    v->d_flags = b->d_flags;
    v->d_err = b->d_err;
    return true;
}

void batch_advance(swe_batch *b, int n_steps)
{
    b->cur ^= (n_steps & 1);
    b->launches += 1;
}

}  // namespace swe

static swe_status st_of(cudaError_t e)
{
    if (e == cudaSuccess) return SWE_OK;
    if (e == cudaErrorMemoryAllocation) return SWE_ENOMEM;
    return SWE_ECUDA;
}

#define B_TRY(expr)                                   \
    do {                                              \
        cudaError_t e_ = (expr);                      \
        if (e_ != cudaSuccess) return st_of(e_);      \
    } while (0)

static Coef<float> coef_of(double dx, double dy, double dt, double g)
{
    const Coef<float> k = make_coef<float>(dx, dy, dt, g);
    return k;
}

static void drop_graphs(swe_batch *b)
{
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
}

// (Re)builds the tile list and tensor maps for variant v and sets the launch
// width; invalidates captured graphs.
// The streaming variant's segments for P warps: each instance's strips
// (OUT columns, all on the same code path, so a row costs the same
// everywhere) are cut into row ranges of about equal length, about four per
// warp, and listed longest first: the warps take them in this order from
// the pass counter.
static swe_status build_stream_schedule(swe_batch *b, int P)
{
    constexpr int OUT = BatchStreamC::OUT, kMinRows = 16;
    long long total = 0;
    for (int i = 0; i < b->n; ++i) total += (long long)((b->nx[i] + OUT - 1) / OUT) * b->ny[i];
    const double target = std::max(1.0, (double)total / (4.0 * P));
    std::vector<SegRec> segs;
    for (int i = 0; i < b->n; ++i) {
        const int ns = (b->nx[i] + OUT - 1) / OUT, ny = b->ny[i];
        const int K = std::max(1, std::min((int)std::lround(ny / target), std::max(1, ny / kMinRows)));
        for (int st = 0; st < ns; ++st)
            for (int j = 0; j < K; ++j)
                segs.push_back(SegRec{i, st, (int)((long long)j * ny / K), (int)((long long)(j + 1) * ny / K)});
    }
    std::stable_sort(segs.begin(), segs.end(),
                     [](const SegRec &a, const SegRec &c) { return a.yb - a.ya > c.yb - c.ya; });
    std::vector<int> buf(kWorkHead + 4 * segs.size(), 0);
    std::memcpy(buf.data() + kWorkHead, segs.data(), segs.size() * sizeof(SegRec));
    const size_t bytes = buf.size() * sizeof(int);
    if (bytes > b->work_cap) {
        cudaFree(b->d_work);
        b->d_work = nullptr;
        b->work_cap = 0;
        B_TRY(cudaMalloc(&b->d_work, bytes));
        b->work_cap = bytes;
    }
    B_TRY(cudaMemcpy(b->d_work, buf.data(), bytes, cudaMemcpyHostToDevice));
    b->nwork = (int)segs.size();
    return SWE_OK;
}

static swe_status configure(swe_batch *b, int v, int ctas_per_sm)
{
    const Variant &V = variants()[v];
    if (V.kind == 0 && b->tiles_ty != V.tile_y) {
        std::vector<TileRec> t;
        for (int i = 0; i < b->n; ++i) {
            const int tx = (b->nx[i] + V.tile_x - 1) / V.tile_x;
            const int ty = (b->ny[i] + V.tile_y - 1) / V.tile_y;
            for (int y = 0; y < ty; ++y)
                for (int x = 0; x < tx; ++x) t.push_back(TileRec{i, (unsigned short)x, (unsigned short)y});
        }
        if ((int)t.size() > b->tiles_cap) {
            cudaFree(b->d_tiles);
            b->d_tiles = nullptr;
            B_TRY(cudaMalloc(&b->d_tiles, t.size() * sizeof(TileRec)));
            b->tiles_cap = (int)t.size();
        }
        B_TRY(cudaMemcpy(b->d_tiles, t.data(), t.size() * sizeof(TileRec), cudaMemcpyHostToDevice));
        b->ntiles = (int)t.size();
        b->tiles_ty = V.tile_y;
    }
    // Tensor maps live in global memory.  The TMA unit may keep a descriptor
    // cached by address, so a map array is never rewritten in place: each
    // box height gets its own array, encoded once.
    const int box_key = V.box_w * 65536 + V.box_h;
    auto found = b->maps_by_box.find(box_key);
    if (found == b->maps_by_box.end()) {
        std::vector<CUtensorMap> m((size_t)b->n * 6);
        for (int i = 0; i < b->n; ++i)
            for (int c = 0; c < 2; ++c)
                for (int f = 0; f < 3; ++f) {
                    const float *base = b->h_inst[i].buf[c] + f * b->h_inst[i].plane;
                    if (!encode_plane_map(&m[((size_t)i * 2 + c) * 3 + f], SWE_F32, base, b->nx[i], b->ny[i],
                                          b->pitch[i], V.box_w, V.box_h))
                        return SWE_ECUDA;
                }
        CUtensorMap *d = nullptr;
        B_TRY(cudaMalloc(&d, m.size() * sizeof(CUtensorMap)));
        const cudaError_t e = cudaMemcpy(d, m.data(), m.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(d);
            return st_of(e);
        }
        found = b->maps_by_box.emplace(box_key, d).first;
    }
    b->d_maps = found->second;
    B_TRY(cudaFuncSetAttribute(V.func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)V.smem));
    int occ = 0;
    B_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, V.func, V.nwarp * 32, V.smem));
    if (occ < 1) return SWE_EUNSUPPORTED;
    b->variant = v;
    b->ctas_per_sm = std::max(1, std::min(ctas_per_sm, occ));
    b->blocks = b->sms * b->ctas_per_sm;
    if (V.kind == 1) {
        const swe_status st = build_stream_schedule(b, b->blocks * V.nwarp);
        if (st != SWE_OK) return st;
    }
    drop_graphs(b);
    return SWE_OK;
}

static int max_ctas(int v)
{
    const Variant &V = variants()[v];
    cudaFuncSetAttribute(V.func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)V.smem);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, V.func, V.nwarp * 32, V.smem);
    return occ;
}

static cudaError_t launch_direct(swe_batch *b, int n_steps, int parity0, cudaStream_t s)
{
    const Variant &V = variants()[b->variant];
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b->blocks);
    cfg.blockDim = dim3(V.nwarp * 32);
    cfg.dynamicSmemBytes = V.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // the tile list, or the streaming variant's segments (its pass counters
    // zeroed first)
    if (V.kind == 1) {
        const cudaError_t e = cudaMemsetAsync(b->d_work, 0, kWorkHead * sizeof(int), s);
        if (e != cudaSuccess) return e;
    }
    void *work = V.kind == 1 ? b->d_work : static_cast<void *>(b->d_tiles);
    int nwork = V.kind == 1 ? b->nwork : b->ntiles;
    void *args[] = {(void *)&b->d_inst, (void *)&b->d_maps, (void *)&work,    (void *)&nwork,
                    (void *)&n_steps,   (void *)&parity0,   (void *)&b->d_bar, (void *)&b->d_err,
                    (void *)&b->d_flags};
    return cudaLaunchKernelExC(&cfg, V.func, args);
}

// Enqueues n_steps on s: replays a captured graph when capture works.
static swe_status run_steps(swe_batch *b, int n_steps, cudaStream_t s)
{
    const int parity0 = b->cur;
    if (b->graph_ok) {
        auto key = std::make_pair(n_steps, parity0);
        auto it = b->graphs.find(key);
        if (it == b->graphs.end()) {
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ge = nullptr;
            bool ok = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                const cudaError_t le = launch_direct(b, n_steps, parity0, b->cap);
                const cudaError_t ee = cudaStreamEndCapture(b->cap, &g);
                ok = le == cudaSuccess && ee == cudaSuccess && g &&
                     cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
            }
            if (g) cudaGraphDestroy(g);
            if (!ok) {
                cudaGetLastError();  // capture is not supported here: launch directly from now on
                if (ge) cudaGraphExecDestroy(ge);
                b->graph_ok = false;
            } else {
                it = b->graphs.emplace(key, ge).first;
            }
        }
        if (b->graph_ok) {
            B_TRY(cudaGraphLaunch(it->second, s));
            b->cur ^= (swaps_of(variants()[b->variant], n_steps) & 1);
            b->launches += 1;
            return SWE_OK;
        }
    }
    B_TRY(launch_direct(b, n_steps, parity0, s));
    b->cur ^= (swaps_of(variants()[b->variant], n_steps) & 1);
    b->launches += 1;
    return SWE_OK;
}

static std::string tune_key(const swe_batch *b)
{
    cudaDeviceProp p;
    cudaGetDeviceProperties(&p, b->device);
    unsigned long long h = 1469598103934665603ull;  // FNV-1a over the sizes
    for (int i = 0; i < b->n; ++i) {
        h = (h ^ (unsigned long long)b->nx[i]) * 1099511628211ull;
        h = (h ^ (unsigned long long)b->ny[i]) * 1099511628211ull;
    }
    char buf[256];
    std::snprintf(buf, sizeof(buf), "%s|n=%d|sizes=%016llx", p.name, b->n, h);
    for (char *c = buf; *c; ++c)
        if (*c == '"') *c = '\'';
    return buf;
}

static bool cache_lookup(const char *path, const std::string &key, int *v, int *cps)
{
    if (!path || !*path) return false;
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    const std::string needle = "\"key\": \"" + key + "\"";
    while (std::fgets(line, sizeof(line), f)) {
        if (!std::strstr(line, needle.c_str())) continue;
        const char *pv = std::strstr(line, "\"variant\": ");
        const char *pc = std::strstr(line, "\"ctas_per_sm\": ");
        if (pv && pc) {
            *v = std::atoi(pv + 11);
            *cps = std::atoi(pc + 15);
            found = *v >= 0 && *v < (int)variants().size() && *cps >= 1;
        }
    }
    std::fclose(f);
    return found;
}

struct Trial {
    int v, cps;
    double ms;
};

// Appends the tuner's decision for ``key``: first a line with every trial
// (variant, CTAs per SM, depth, ms per step), then the winner's line, the
// one cache_lookup reads.
static void cache_store(const char *path, const std::string &key, int v, int cps, double ms,
                        const std::vector<Trial> &trials)
{
    if (!path || !*path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "{\"key\": \"%s\", \"trials\": [", key.c_str());
    for (size_t i = 0; i < trials.size(); ++i)
        std::fprintf(f, "%s{\"v\": %d, \"cps\": %d, \"depth\": %d, \"ms\": %.6f}", i ? ", " : "", trials[i].v,
                     trials[i].cps, variants()[trials[i].v].depth, trials[i].ms);
    std::fprintf(f, "]}\n");
    const Variant &V = variants()[v];
    std::fprintf(f,
                 "{\"key\": \"%s\", \"variant\": %d, \"ctas_per_sm\": %d, \"tile_x\": %d, \"tile_y\": %d, "
                 "\"stages\": %d, \"depth\": %d, \"ms_per_step\": %.6f}\n",
                 key.c_str(), v, cps, V.tile_x, V.tile_y, V.stages, V.depth, ms);
    std::fclose(f);
}

extern "C" {

void swe_batch_destroy(swe_batch *b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    drop_graphs(b);
    if (b->cap) cudaStreamDestroy(b->cap);
    cudaFree(b->pool);
    cudaFree(b->d_inst);
    for (auto &kv : b->maps_by_box) cudaFree(kv.second);
    cudaFree(b->d_tiles);
    cudaFree(b->d_work);
    cudaFree(b->d_bar);
    cudaFree(b->d_err);
    cudaFree(b->d_flags);
    cudaFree(b->d_red[0]);
    cudaFree(b->d_red[1]);
    cudaFree(b->d_scratch);
    cudaFree(b->d_out);
    cudaFreeHost(b->h_out);
    delete b;
}

swe_status swe_batch_create(int n, const int *nx, const int *ny, const double *dx, const double *dy,
                            const double *dt, double g, swe_batch **out)
{
    if (!out) return SWE_EINVAL;
    *out = nullptr;
    if (n < 1 || !nx || !ny || !dx || !dy || !dt || !(g > 0.0) || !std::isfinite(g)) return SWE_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (nx[i] < 1 || ny[i] < 1 || nx[i] > 65536 || ny[i] > 65536) return SWE_EINVAL;
        for (double v : {dx[i], dy[i], dt[i]})
            if (!(v > 0.0) || !std::isfinite(v)) return SWE_EINVAL;
    }
    swe_batch *b = new (std::nothrow) swe_batch();
    if (!b) return SWE_ENOMEM;
    auto fail = [&](swe_status s) {
        swe_batch_destroy(b);
        return s;
    };
    cudaGetDevice(&b->device);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    b->n = n;
    b->g = g;
    b->nx.assign(nx, nx + n);
    b->ny.assign(ny, ny + n);
    b->dx.assign(dx, dx + n);
    b->dy.assign(dy, dy + n);
    b->dt.assign(dt, dt + n);
    long long at = 0;
    for (int i = 0; i < n; ++i) {
        const long long p = plane_pitch(nx[i], 4);
        b->pitch.push_back(p);
        b->off.push_back(at);
        at += 3 * p * ny[i];
        at = (at + 63) / 64 * 64;  // 256-byte aligned instances
    }
    b->half = (size_t)at;
    swe_status s;
    if ((s = st_of(cudaMalloc(&b->pool, 2 * b->half * sizeof(float)))) != SWE_OK) return fail(s);
    if ((s = st_of(cudaMemset(b->pool, 0, 2 * b->half * sizeof(float)))) != SWE_OK) return fail(s);
    b->h_inst.resize(n);
    std::vector<RedGrid> red[2];
    for (int i = 0; i < n; ++i) {
        BatchInst &I = b->h_inst[i];
        I.buf[0] = b->pool + b->off[i];
        I.buf[1] = b->pool + b->half + b->off[i];
        I.pitch = b->pitch[i];
        I.plane = b->pitch[i] * ny[i];
        I.nx = nx[i];
        I.ny = ny[i];
        I.k = coef_of(dx[i], dy[i], dt[i], g);
        for (int c = 0; c < 2; ++c)
            red[c].push_back(RedGrid{I.buf[c], I.buf[c] + I.plane, I.buf[c] + 2 * I.plane, I.pitch, nx[i], ny[i],
                                     dx[i], dy[i]});
    }
    if ((s = st_of(cudaMalloc(&b->d_inst, n * sizeof(BatchInst)))) != SWE_OK) return fail(s);
    if ((s = st_of(cudaMemcpy(b->d_inst, b->h_inst.data(), n * sizeof(BatchInst), cudaMemcpyHostToDevice))) !=
        SWE_OK)
        return fail(s);
    for (int c = 0; c < 2; ++c) {
        if ((s = st_of(cudaMalloc(&b->d_red[c], n * sizeof(RedGrid)))) != SWE_OK) return fail(s);
        if ((s = st_of(cudaMemcpy(b->d_red[c], red[c].data(), n * sizeof(RedGrid), cudaMemcpyHostToDevice))) !=
            SWE_OK)
            return fail(s);
    }
    if ((s = st_of(cudaMalloc(&b->d_bar, sizeof(GridBarrier)))) != SWE_OK) return fail(s);
    if ((s = st_of(cudaMemset(b->d_bar, 0, sizeof(GridBarrier)))) != SWE_OK) return fail(s);
    if ((s = st_of(cudaMalloc(&b->d_err, sizeof(int)))) != SWE_OK) return fail(s);
    if ((s = st_of(cudaMemset(b->d_err, 0, sizeof(int)))) != SWE_OK) return fail(s);
    if ((s = st_of(cudaMalloc(&b->d_flags, n * sizeof(int)))) != SWE_OK) return fail(s);
    if ((s = st_of(cudaMemset(b->d_flags, 0, n * sizeof(int)))) != SWE_OK) return fail(s);
    const size_t sd = reduce_scratch_doubles_many(n, b->red_blocks);
    if ((s = st_of(cudaMalloc(&b->d_scratch, sd * sizeof(double)))) != SWE_OK) return fail(s);
    if ((s = st_of(cudaMalloc(&b->d_out, 2 * (size_t)n * sizeof(double)))) != SWE_OK) return fail(s);
    if ((s = st_of(cudaMallocHost(&b->h_out, 2 * (size_t)n * sizeof(double)))) != SWE_OK) return fail(s);
    if ((s = st_of(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking))) != SWE_OK) return fail(s);
    if ((s = configure(b, 0, 2)) != SWE_OK) return fail(s);
    *out = b;
    return SWE_OK;
}

static swe_status batch_copy(swe_batch *b, int i, void *const *user, long long ld, bool to_dev, cudaStream_t s)
{
    if (!b || i < 0 || i >= b->n || ld < b->nx[i]) return SWE_EINVAL;
    for (int k = 0; k < 3; ++k)
        if (!user[k]) return SWE_EINVAL;
    const BatchInst &I = b->h_inst[i];
    for (int k = 0; k < 3; ++k) {
        float *dev = I.buf[b->cur] + k * I.plane;
        const size_t w = (size_t)I.nx * sizeof(float);
        if (to_dev)
            B_TRY(cudaMemcpy2DAsync(dev, I.pitch * sizeof(float), user[k], ld * sizeof(float), w, I.ny,
                                    cudaMemcpyDefault, s));
        else
            B_TRY(cudaMemcpy2DAsync(user[k], ld * sizeof(float), dev, I.pitch * sizeof(float), w, I.ny,
                                    cudaMemcpyDefault, s));
    }
    return SWE_OK;
}

swe_status swe_batch_set_state(swe_batch *b, int i, const void *h, const void *hu, const void *hv, long long ld,
                               int on_device, void *stream)
{
    (void)on_device;
    void *p[3] = {const_cast<void *>(h), const_cast<void *>(hu), const_cast<void *>(hv)};
    return batch_copy(b, i, p, ld, true, static_cast<cudaStream_t>(stream));
}

swe_status swe_batch_get_state(swe_batch *b, int i, void *h, void *hu, void *hv, long long ld, int on_device,
                               void *stream)
{
    (void)on_device;
    void *p[3] = {h, hu, hv};
    return batch_copy(b, i, p, ld, false, static_cast<cudaStream_t>(stream));
}

swe_status swe_batch_set_dt(swe_batch *b, const double *dt, void *stream)
{
    if (!b || !dt) return SWE_EINVAL;
    for (int i = 0; i < b->n; ++i)
        if (!(dt[i] > 0.0) || !std::isfinite(dt[i])) return SWE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (int i = 0; i < b->n; ++i) {
        b->dt[i] = dt[i];
        b->h_inst[i].k = coef_of(b->dx[i], b->dy[i], dt[i], b->g);
    }
    // the pageable source is copied before cudaMemcpyAsync returns
    B_TRY(cudaMemcpyAsync(b->d_inst, b->h_inst.data(), b->n * sizeof(BatchInst), cudaMemcpyHostToDevice, s));
    return SWE_OK;
}

swe_status swe_batch_step(swe_batch *b, int n_steps, void *stream)
{
    if (!b || n_steps < 0) return SWE_EINVAL;
    if (n_steps == 0) return SWE_OK;
    return run_steps(b, n_steps, static_cast<cudaStream_t>(stream));
}

swe_status swe_batch_status(swe_batch *b, int *flags_out, void *stream)
{
    if (!b || !flags_out) return SWE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int err = 0;
    B_TRY(cudaMemcpyAsync(flags_out, b->d_flags, b->n * sizeof(int), cudaMemcpyDeviceToHost, s));
    B_TRY(cudaMemcpyAsync(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    B_TRY(cudaStreamSynchronize(s));
    if (err) {
        for (int i = 0; i < b->n; ++i) flags_out[i] |= SWE_FLAG_TIMEOUT;
    }
    B_TRY(cudaMemsetAsync(b->d_flags, 0, b->n * sizeof(int), s));
    B_TRY(cudaMemsetAsync(b->d_err, 0, sizeof(int), s));
    B_TRY(cudaMemsetAsync(b->d_bar, 0, sizeof(GridBarrier), s));
    B_TRY(cudaStreamSynchronize(s));
    return err ? (swe_status)err : SWE_OK;
}

swe_status swe_batch_mass(swe_batch *b, double *mass_out, void *stream)
{
    if (!b || !mass_out) return SWE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    B_TRY(launch_mass_many(b->d_red[b->cur], b->n, b->red_blocks, b->d_scratch, b->d_out, s));
    B_TRY(cudaMemcpyAsync(b->h_out, b->d_out, 2 * (size_t)b->n * sizeof(double), cudaMemcpyDeviceToHost, s));
    B_TRY(cudaStreamSynchronize(s));
    for (int i = 0; i < b->n; ++i) mass_out[i] = b->h_out[2 * i];
    return SWE_OK;
}

swe_status swe_batch_cfl_dt(swe_batch *b, double cfl, double *dt_out, void *stream)
{
    if (!b || !dt_out || !(cfl > 0.0) || !std::isfinite(cfl)) return SWE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    B_TRY(launch_cfl_many(b->d_red[b->cur], b->n, b->red_blocks, b->g, cfl, b->d_scratch, b->d_out, s));
    B_TRY(cudaMemcpyAsync(b->h_out, b->d_out, 2 * (size_t)b->n * sizeof(double), cudaMemcpyDeviceToHost, s));
    B_TRY(cudaStreamSynchronize(s));
    bool bad = false;
    for (int i = 0; i < b->n; ++i) {
        dt_out[i] = b->h_out[2 * i + 1] != 0.0 ? 0.0 : b->h_out[2 * i];
        bad |= b->h_out[2 * i + 1] != 0.0;
    }
    return bad ? SWE_ECHECK : SWE_OK;
}

swe_status swe_batch_tune(swe_batch *b, const char *cache_path, void *stream)
{
    if (!b) return SWE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const char *path = cache_path && *cache_path ? cache_path : std::getenv("SWE_TUNE_CACHE");
    const std::string key = tune_key(b);
    int v = 0, cps = 1;
    if (cache_lookup(path, key, &v, &cps)) {
        swe_status st = configure(b, v, cps);
        if (st == SWE_OK) b->tuned = 2;
        return st;
    }
    // keep the current state: trials run on it and it is restored afterwards
    float *saved = nullptr;
    B_TRY(cudaMalloc(&saved, b->half * sizeof(float)));
    B_TRY(cudaMemcpyAsync(saved, b->pool + (size_t)b->cur * b->half, b->half * sizeof(float),
                          cudaMemcpyDeviceToDevice, s));
    const int cur0 = b->cur;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best_ms = 1e30;
    int best_v = 0, best_c = 1;
    std::vector<Trial> trials;
    const int trial_steps = 8;
    swe_status st = SWE_OK;
    for (int vi = 0; vi < (int)variants().size() && st == SWE_OK; ++vi) {
        const int occ = max_ctas(vi);
        for (int c = 1; c <= occ && st == SWE_OK; ++c) {
            if ((st = configure(b, vi, c)) != SWE_OK) break;
            if ((st = run_steps(b, 2, s)) != SWE_OK) break;  // capture + warm-up
            float best = 1e30f;
            for (int rep = 0; rep < 2; ++rep) {
                cudaEventRecord(e0, s);
                if ((st = run_steps(b, trial_steps, s)) != SWE_OK) break;
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                best = std::min(best, ms);
            }
            const double per = best / trial_steps;
            trials.push_back(Trial{vi, c, per});
            if (per < best_ms) {
                best_ms = per;
                best_v = vi;
                best_c = c;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->cur = cur0;
    cudaMemcpyAsync(b->pool + (size_t)cur0 * b->half, saved, b->half * sizeof(float), cudaMemcpyDeviceToDevice, s);
    cudaStreamSynchronize(s);
    cudaFree(saved);
    cudaMemset(b->d_flags, 0, b->n * sizeof(int));
    if (st != SWE_OK) return st;
    st = configure(b, best_v, best_c);
    if (st == SWE_OK) {
        b->tuned = 1;
        cache_store(path, key, best_v, best_c, best_ms, trials);
    }
    return st;
}

swe_status swe_batch_query(swe_batch *b, int key, long long *value)
{
    if (!b || !value) return SWE_EINVAL;
    const Variant &V = variants()[b->variant];
    switch (key) {
        case SWE_BQ_VARIANT: *value = b->variant; break;
        case SWE_BQ_CTAS_PER_SM: *value = b->ctas_per_sm; break;
        case SWE_BQ_BLOCKS: *value = b->blocks; break;
        case SWE_BQ_TILES: *value = b->ntiles; break;
        case SWE_BQ_TILE_X: *value = V.tile_x; break;
        case SWE_BQ_TILE_Y: *value = V.tile_y; break;
        case SWE_BQ_STAGES: *value = V.stages; break;
        case SWE_BQ_DEPTH: *value = V.depth; break;
        case SWE_BQ_GRAPH: *value = b->graph_ok ? 1 : 0; break;
        case SWE_BQ_LAUNCHES: *value = b->launches; break;
        case SWE_BQ_TUNED: *value = b->tuned; break;
        case SWE_BQ_CELLS: {
            long long c = 0;
            for (int i = 0; i < b->n; ++i) c += (long long)b->nx[i] * b->ny[i];
            *value = c;
            break;
        }
        case SWE_BQ_VARIANT_COUNT: *value = (long long)variants().size(); break;
        case SWE_BQ_KIND: *value = V.kind; break;
        default: return SWE_EINVAL;
    }
    return SWE_OK;
}

swe_status swe_selftest_wait(int which, double limit_ms, void *stream)
{
    if ((which != 0 && which != 1) || !(limit_ms > 0.0) || limit_ms > 5000.0) return SWE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int *d_err = nullptr;
    GridBarrier *d_bar = nullptr;
    B_TRY(cudaMalloc(&d_err, sizeof(int)));
    cudaError_t e = cudaMalloc(&d_bar, sizeof(GridBarrier));
    if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_bar, 0, sizeof(GridBarrier), s);
    if (e == cudaSuccess) e = launch_wait_probe(which, (unsigned long long)(limit_ms * 1e6), d_bar, d_err, s);
    int word = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&word, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_err);
    cudaFree(d_bar);
    if (e != cudaSuccess) return st_of(e);
    return (swe_status)word;
}

swe_status swe_batch_state_ptr(swe_batch *b, int i, float **h, long long *plane_stride, long long *pitch)
{
    if (!b || !h || !plane_stride || !pitch || i < 0 || i >= b->n) return SWE_EINVAL;
    *h = b->h_inst[i].buf[b->cur];
    *plane_stride = b->h_inst[i].plane;
    *pitch = b->h_inst[i].pitch;
    return SWE_OK;
}

swe_status swe_batch_copy_states(swe_batch *b, float *dst, void *stream)
{
    if (!b || !dst) return SWE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    size_t at = 0;
    for (int i = 0; i < b->n; ++i) {
        const BatchInst &I = b->h_inst[i];
        for (int k = 0; k < 3; ++k) {
            B_TRY(cudaMemcpy2DAsync(dst + at, (size_t)I.nx * sizeof(float), I.buf[b->cur] + k * I.plane,
                                    (size_t)I.pitch * sizeof(float), (size_t)I.nx * sizeof(float), I.ny,
                                    cudaMemcpyDeviceToDevice, s));
            at += (size_t)I.nx * I.ny;
        }
    }
    return SWE_OK;
}

swe_status swe_batch_configure(swe_batch *b, int variant, int ctas_per_sm)
{
    if (!b || variant < 0 || variant >= (int)variants().size() || ctas_per_sm < 1) return SWE_EINVAL;
    return configure(b, variant, ctas_per_sm);
}

}  // extern "C"
