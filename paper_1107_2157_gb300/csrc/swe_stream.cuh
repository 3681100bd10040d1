// swe_stream.cuh -- two Lax-Wendroff steps per pass (Sec. 3 step equations)
// by warps that stream up column strips, FP32: the device code shared by the
// single-grid kernel (swe_stream.cu) and the batched one (swe_batch.cu).
//
// A warp owns a strip of OUT grid columns starting at xs and a range of its
// rows.  Each lane holds VX = 2 VP consecutive columns c_0 .. c_{VX-1} as VP
// cell pairs on the packed f32x2 pipe, pair p = (c_{2p}, c_{2p+1}), or with
// SPLIT pair p = (c_p, c_{p+VP}) (the same for VP = 1); lanes LO .. LO + NO
// - 1 hold the strip, lane LO - 1 and lane LO + NO the columns just outside
// it.  (The default shape: VP = 2, lane l holds xs - 4 + 4l .. xs - 1 + 4l,
// lanes 1..30 store 120 columns.)
// For each row q the warp takes the first step of row q (the intermediate
// state, from input rows q-1..q+1) and then the second step of row q-1 (from
// intermediate rows q-2..q).  The intermediate rows never leave registers:
// a lane's second step needs only its own intermediate cells, the rows above
// and below in the same lane, and the adjacent lanes' cells, which it reads
// with warp shuffles.  The x-face between two lanes is computed once, by the
// lane on its right, and handed to the lane on its left.  The overlap lanes
// compute the intermediate cells just outside the strip that the second step
// reads; their own second-step results are discarded.
//
// Strips are whole 32-byte sectors wide (OUT a multiple of 8 columns, xs a
// multiple of OUT): two warps never write parts of one sector, which would
// make L2 read it back from DRAM before writing it out.
//
// Input rows arrive by TMA, CR rows of the three planes at a time, into a
// ring of NSLOT chunks per warp; every input row is read from shared memory
// once.  Warps are independent (no CTA barrier): each waits only on its own
// chunks' mbarriers, with bounded waits.
//
// Against the tiled two-step kernel (swe_temporal.cu) the y-faces at the
// edges of a warp's rows and the ring of the intermediate box are not
// recomputed, and x-neighbour cells are not rebuilt from shared memory; the
// price is the two overlap lanes.  Every cell goes through the same face and
// update functions, in the same operand order, so the bits are those of two
// one-step passes.
#pragma once

#include <type_traits>

#include "swe_tile.cuh"

namespace swe {

template <int VP, int LO, int NO, int CR, int NSLOT, int WARPS>
struct StreamCfg {
    static constexpr int VX = 2 * VP;      // cells per lane: VP pairs
    static constexpr int BW = 32 * VX;     // columns a warp holds (the TMA box width)
    static constexpr int OUT = NO * VX;    // columns it stores: lanes LO .. LO + NO - 1
    static constexpr int ROWS = CR;        // rows per TMA chunk
    static constexpr uint32_t PLANE_BYTES = BW * CR * 4;
    static constexpr uint32_t CHUNK_BYTES = 3 * PLANE_BYTES;
    static constexpr size_t WARP_BYTES = (size_t)NSLOT * CHUNK_BYTES;
    static constexpr size_t SMEM = WARPS * WARP_BYTES + WARPS * NSLOT * sizeof(uint64_t);
    static_assert(VP == 1 || VP == 2, "one or two pairs per lane");
    static_assert(LO >= 1 && LO + NO <= 31, "an overlap lane on each side of the stored ones");
    static_assert(OUT % 8 == 0 && (LO * VX) % 4 == 0, "32-byte output rows, 16-byte aligned boxes");
};

constexpr unsigned kFull = 0xffffffffu;

// The x-face flux pairs of a lane's cells c_0 .. c_{2VP-1} (pairs
// c[p] = (c_{2p}, c_{2p+1})): Fl[p] = (c_{2p-1}|c_{2p}, c_{2p}|c_{2p+1}) and
// Fr[p] = (c_{2p}|c_{2p+1}, c_{2p+1}|c_{2p+2}), where c_{-1} is the lower
// lane's last cell and the face right of the last cell is the upper lane's
// first face.  Walls are in the data (stream_ghosts).
template <int VP, bool SPLIT = false>
__device__ __forceinline__ void stream_xfaces(const CellQ2 (&c)[VP], const Coef2 &k2, Flux2 (&Fl)[VP],
                                              Flux2 (&Fr)[VP])
{
    CellQ<float> L;
    L.h = __shfl_up_sync(kFull, hi2(c[VP - 1].h), 1);
    L.u = __shfl_up_sync(kFull, hi2(c[VP - 1].u), 1);
    L.v = __shfl_up_sync(kFull, hi2(c[VP - 1].v), 1);
    L.f2 = __shfl_up_sync(kFull, hi2(c[VP - 1].f2), 1);
    L.f3 = __shfl_up_sync(kFull, hi2(c[VP - 1].f3), 1);
    L.g3 = 0.0f;  // not read by an x-face
    if constexpr (SPLIT) {
        // pair p = (c_p, c_{p+VP}): the left cells of pair p >= 1 are pair
        // p - 1, those of pair 0 are (c_{-1}, c_{VP-1}); Fr[p] = Fl[p+1], and
        // the last pair's right faces are (c_VP's left face, the upper
        // lane's first face)
        Fl[0] = xface_flux2(pair_cells(L, cell_lo(c[VP - 1])), c[0], k2);
#pragma unroll
        for (int p = 1; p < VP; ++p) Fl[p] = xface_flux2(c[p - 1], c[p], k2);
        const float fa = __shfl_down_sync(kFull, lo2(Fl[0].a), 1);
        const float fb = __shfl_down_sync(kFull, lo2(Fl[0].b), 1);
        const float fc = __shfl_down_sync(kFull, lo2(Fl[0].c), 1);
#pragma unroll
        for (int p = 0; p + 1 < VP; ++p) Fr[p] = Fl[p + 1];
        Fr[VP - 1] = flux_pair(hi2(Fl[0].a), hi2(Fl[0].b), hi2(Fl[0].c), fa, fb, fc);
    } else {
        Fl[0] = xface_flux2(pair_cells(L, cell_lo(c[0])), c[0], k2);
#pragma unroll
        for (int p = 1; p < VP; ++p) Fl[p] = xface_flux2(pair_cells(cell_hi(c[p - 1]), cell_lo(c[p])), c[p], k2);
        const float fa = __shfl_down_sync(kFull, lo2(Fl[0].a), 1);
        const float fb = __shfl_down_sync(kFull, lo2(Fl[0].b), 1);
        const float fc = __shfl_down_sync(kFull, lo2(Fl[0].c), 1);
#pragma unroll
        for (int p = 0; p + 1 < VP; ++p)
            Fr[p] = flux_pair(hi2(Fl[p].a), hi2(Fl[p].b), hi2(Fl[p].c), lo2(Fl[p + 1].a), lo2(Fl[p + 1].b),
                              lo2(Fl[p + 1].c));
        Fr[VP - 1] = flux_pair(hi2(Fl[VP - 1].a), hi2(Fl[VP - 1].b), hi2(Fl[VP - 1].c), fa, fb, fc);
    }
}

// Reflective walls as ghost columns: in a strip that reaches a wall, the
// raw state (h, hu, hv) of column -1 becomes that of column 0 with hu
// negated, and column nx that of column nx - 1 likewise, before the cells
// are formed.  make_cell of (h, -hu, hv) has exactly the bits of mirror_x
// of make_cell(h, hu, hv) (every product involving hu changes sign and
// nothing else), so the faces next to a wall are those of the other
// kernels.  gx0 is the grid column of the lane's first cell.
template <int VP, bool SPLIT = false>
__device__ __forceinline__ void stream_ghosts(F2 (&h)[VP], F2 (&u)[VP], F2 (&v)[VP], int gx0, int nx)
{
    constexpr int VX = 2 * VP;
    float hs[VX], us[VX], vs[VX];
#pragma unroll
    for (int p = 0; p < VP; ++p) {
        const int j0 = SPLIT ? p : 2 * p, j1 = SPLIT ? p + VP : 2 * p + 1;  // the pair's columns
        unpack2(h[p], hs[j0], hs[j1]);
        unpack2(u[p], us[j0], us[j1]);
        unpack2(v[p], vs[j0], vs[j1]);
    }
    // the lower lane's last cell and the upper lane's first cell
    const float ph = __shfl_up_sync(kFull, hs[VX - 1], 1), pu = __shfl_up_sync(kFull, us[VX - 1], 1),
                pv = __shfl_up_sync(kFull, vs[VX - 1], 1);
    const float nh = __shfl_down_sync(kFull, hs[0], 1), nu = __shfl_down_sync(kFull, us[0], 1),
                nv = __shfl_down_sync(kFull, vs[0], 1);
    float gh[VX], gu[VX], gv[VX];
#pragma unroll
    for (int j = 0; j < VX; ++j) {
        gh[j] = hs[j];
        gu[j] = us[j];
        gv[j] = vs[j];
        const int col = gx0 + j;
        if (col == -1) {  // mirror of column 0: the next cell
            gh[j] = j + 1 < VX ? hs[j + 1] : nh;
            gu[j] = -(j + 1 < VX ? us[j + 1] : nu);
            gv[j] = j + 1 < VX ? vs[j + 1] : nv;
        } else if (col == nx) {  // mirror of column nx - 1: the previous cell
            gh[j] = j > 0 ? hs[j - 1] : ph;
            gu[j] = -(j > 0 ? us[j - 1] : pu);
            gv[j] = j > 0 ? vs[j - 1] : pv;
        }
    }
#pragma unroll
    for (int p = 0; p < VP; ++p) {
        const int j0 = SPLIT ? p : 2 * p, j1 = SPLIT ? p + VP : 2 * p + 1;
        h[p] = pack2(gh[j0], gh[j1]);
        u[p] = pack2(gu[j0], gu[j1]);
        v[p] = pack2(gv[j0], gv[j1]);
    }
}

// One step of a row of a lane's cells ``c`` (pairs), given the y-face fluxes
// below (gd) and above (gu); returns the updated (h, hu, hv) pairs.
template <int VP, bool SPLIT = false>
__device__ __forceinline__ void stream_update(const CellQ2 (&c)[VP], const Flux2 (&gd)[VP], const Flux2 (&gu)[VP],
                                              const Coef2 &k2, F2 (&oh)[VP], F2 (&ou)[VP], F2 (&ov)[VP])
{
    Flux2 Fl[VP], Fr[VP];
    stream_xfaces<VP, SPLIT>(c, k2, Fl, Fr);
#pragma unroll
    for (int p = 0; p < VP; ++p) {
        oh[p] = c[p].h;
        ou[p] = c[p].u;
        ov[p] = c[p].v;
        lw_update2(oh[p], ou[p], ov[p], Fl[p], Fr[p], gd[p], gu[p], k2);
    }
}

template <int VP, int LO, int NO, int CR, int NSLOT, int WARPS>
struct StreamWarp {
    using C = StreamCfg<VP, LO, NO, CR, NSLOT, WARPS>;
    const CUtensorMap *mH, *mU, *mV;
    unsigned char *ring;  // NSLOT chunks: planes h, hu, hv of CR rows x BW columns
    uint64_t *bars;       // one mbarrier per slot
    uint32_t phase;       // bit j: the parity of slot j's next completion
    int *err;

    __device__ __forceinline__ void issue(int c, int x, int first)
    {
        const int slot = c % NSLOT;
        unsigned char *dst = ring + (size_t)slot * C::CHUNK_BYTES;
        mbar_arrive_expect_tx(bars + slot, C::CHUNK_BYTES);
        tma_load_2d(dst, mH, bars + slot, x, first + c * CR);
        tma_load_2d(dst + C::PLANE_BYTES, mU, bars + slot, x, first + c * CR);
        tma_load_2d(dst + 2 * C::PLANE_BYTES, mV, bars + slot, x, first + c * CR);
    }
};

template <int VP, bool SPLIT = false>
__device__ __forceinline__ void store_cells(float *dst, const F2 (&x)[VP])
{
    if constexpr (VP == 2) {
        float4 t;
        if constexpr (SPLIT) {  // pairs (c_0, c_2), (c_1, c_3)
            unpack2(x[0], t.x, t.z);
            unpack2(x[1], t.y, t.w);
        } else {
            unpack2(x[0], t.x, t.y);
            unpack2(x[1], t.z, t.w);
        }
        *reinterpret_cast<float4 *>(dst) = t;
    } else {
        float2 t;
        unpack2(x[0], t.x, t.y);
        *reinterpret_cast<float2 *>(dst) = t;
    }
}

// Two steps (ONE: one step) of output rows [ya, yb) of the strip whose
// stored lanes start at column xs.  Returns false (with SWE_ETIMEOUT
// recorded) if a chunk did not arrive in time; sets bad if a stored depth is
// not positive (h <= 0 or NaN).
//
// The row loop is unrolled by two with the roles of the two state sets
// swapped between the halves (the cells and faces of the current row are
// the "next" ones of the row before), so nothing is copied from row to row;
// input rows and output rows are walked with running offsets.
template <bool EDGE, int VP, int LO, int NO, int CR, int NSLOT, int WARPS, bool ONE = false, bool SPLIT = false>
__device__ __forceinline__ bool stream_segment(StreamWarp<VP, LO, NO, CR, NSLOT, WARPS> &w, float *__restrict__ oH,
                                               float *__restrict__ oU, float *__restrict__ oV, int nx, int ny,
                                               long long pitch, int xs, int ya, int yb, const Coef2 &k2,
                                               bool &bad)
{
    using C = StreamCfg<VP, LO, NO, CR, NSLOT, WARPS>;
    constexpr int VX = C::VX;
    const int lane = threadIdx.x & 31;
    const int bx = xs - LO * VX;  // box column of lane 0's first cell
    const int gx0 = bx + VX * lane;
    const bool stores = lane >= LO && lane < LO + NO && gx0 < nx;
    // first-step rows q0..q1: the output rows and, for two steps, the ring
    // rows next to them
    const int q0 = ONE ? ya : max(ya - 1, 0), q1 = ONE ? yb - 1 : min(yb, ny - 1);
    const int first = q0 > 0 ? q0 - 1 : 0;                // input rows read: first..last
    const int last = min(q1 + 1, ny - 1);
    const int nch = (last - first) / CR + 1;
    int issued = min(NSLOT, nch);

    // the slots were last read before this point: order those reads before
    // the TMA writes that refill them
    __syncwarp();
    if (lane == 0) {
        fence_proxy_async_smem();
        for (int c = 0; c < issued; ++c) w.issue(c, bx, first);
    }
    bool ok = true;
    // The next input row's cells (rows first, first + 1, ... in turn).
    // Entering a chunk frees the previous one, which is refilled with the
    // chunk NSLOT on.  After a timeout the reads stay inside the ring and
    // their values are not stored.
    int rr = CR, ci = -1, slot = NSLOT - 1;
    const float *rp = reinterpret_cast<const float *>(w.ring) + VX * lane;
    auto next_row = [&](CellQ2(&c)[VP]) {
        if (rr == CR) {
            if (ok) {
                ++ci;
                slot = slot + 1 == NSLOT ? 0 : slot + 1;
                if (ci >= 1 && issued < nch) {
                    __syncwarp();
                    if (lane == 0) {
                        fence_proxy_async_smem();
                        w.issue(issued, bx, first);
                    }
                    ++issued;
                }
                if (__all_sync(kFull, mbar_wait_bounded(w.bars + slot, (w.phase >> slot) & 1u, w.err)))
                    w.phase ^= 1u << slot;
                else
                    ok = false;
                rp = reinterpret_cast<const float *>(w.ring + (size_t)slot * C::CHUNK_BYTES) + VX * lane;
            }
            rr = 0;
        }
        const float *p = rp + rr * C::BW;
        ++rr;
        F2 h[VP], u[VP], v[VP];
        if constexpr (VP == 2) {
            const float4 h4 = *reinterpret_cast<const float4 *>(p);
            const float4 u4 = *reinterpret_cast<const float4 *>(p + C::BW * CR);
            const float4 v4 = *reinterpret_cast<const float4 *>(p + 2 * C::BW * CR);
            if constexpr (SPLIT) {  // pairs (c_0, c_2), (c_1, c_3)
                h[0] = pack2(h4.x, h4.z);
                h[VP - 1] = pack2(h4.y, h4.w);
                u[0] = pack2(u4.x, u4.z);
                u[VP - 1] = pack2(u4.y, u4.w);
                v[0] = pack2(v4.x, v4.z);
                v[VP - 1] = pack2(v4.y, v4.w);
            } else {
                h[0] = pack2(h4.x, h4.y);
                h[VP - 1] = pack2(h4.z, h4.w);
                u[0] = pack2(u4.x, u4.y);
                u[VP - 1] = pack2(u4.z, u4.w);
                v[0] = pack2(v4.x, v4.y);
                v[VP - 1] = pack2(v4.z, v4.w);
            }
        } else {
            const float2 h2 = *reinterpret_cast<const float2 *>(p);
            const float2 u2 = *reinterpret_cast<const float2 *>(p + C::BW * CR);
            const float2 v2 = *reinterpret_cast<const float2 *>(p + 2 * C::BW * CR);
            h[0] = pack2(h2.x, h2.y);
            u[0] = pack2(u2.x, u2.y);
            v[0] = pack2(v2.x, v2.y);
        }
        if (EDGE) stream_ghosts<VP, SPLIT>(h, u, v, gx0, nx);
#pragma unroll
        for (int j = 0; j < VP; ++j) c[j] = make_cell2(h[j], u[j], v[j], k2);
    };
    // output rows ya, ya + 1, ... in turn
    long long orow = (long long)ya * pitch + gx0;
    auto store_next = [&](const F2(&oh)[VP], const F2(&ou)[VP], const F2(&ov)[VP]) {
        if (stores && ok) {
            store_cells<VP, SPLIT>(oH + orow, oh);
            store_cells<VP, SPLIT>(oU + orow, ou);
            store_cells<VP, SPLIT>(oV + orow, ov);
#pragma unroll
            for (int p = 0; p < VP; ++p) {
                float a, b;
                unpack2(oh[p], a, b);
                const int j0 = SPLIT ? p : 2 * p, j1 = SPLIT ? p + VP : 2 * p + 1;
                bad |= (gx0 + j0 < nx && !(a > 0.0f)) || (gx0 + j1 < nx && !(b > 0.0f));
            }
        }
        orow += pitch;
    };
    auto mirror_row = [](const CellQ2(&c)[VP], CellQ2(&m)[VP]) {
#pragma unroll
        for (int p = 0; p < VP; ++p) m[p] = mirror_y2(c[p]);
    };
    // The first step of row q: c = its input cells, d = the faces below;
    // n receives row q + 1's cells, u the faces between, m the intermediate
    // cells of row q.  TOP: row q may be the grid's last (its upper
    // neighbour the mirror).
    auto first_step = [&](auto top, int q, const CellQ2(&c)[VP], CellQ2(&n)[VP], const Flux2(&d)[VP],
                          Flux2(&u)[VP], CellQ2(&m)[VP]) {
        if (!decltype(top)::value || q + 1 < ny)
            next_row(n);
        else
            mirror_row(c, n);
#pragma unroll
        for (int p = 0; p < VP; ++p) u[p] = yface_flux2(c[p], n[p], k2);
        F2 oh[VP], ou[VP], ov[VP];
        stream_update<VP, SPLIT>(c, d, u, k2, oh, ou, ov);
        if (EDGE) stream_ghosts<VP, SPLIT>(oh, ou, ov, gx0, nx);
#pragma unroll
        for (int p = 0; p < VP; ++p) m[p] = make_cell2(oh[p], ou[p], ov[p], k2);
    };
    const std::true_type top;
    const std::false_type inner;
    // The second step of row q - 1 (c2, d2) once the first step of row q has
    // given n2.
    auto second_step = [&](const CellQ2(&c2)[VP], const CellQ2(&n2)[VP], const Flux2(&d2)[VP], Flux2(&u2)[VP]) {
#pragma unroll
        for (int p = 0; p < VP; ++p) u2[p] = yface_flux2(c2[p], n2[p], k2);
        F2 oh[VP], ou[VP], ov[VP];
        stream_update<VP, SPLIT>(c2, d2, u2, k2, oh, ou, ov);
        store_next(oh, ou, ov);
    };

    // A1/B1, dA1/dB1: first-step cells and faces; A2/B2, dA2/dB2: the same
    // for the second step.
    CellQ2 A1[VP], B1[VP], A2[VP], B2[VP];
    Flux2 dA1[VP], dB1[VP], dA2[VP], dB2[VP];
    if (q0 == 0) {
        next_row(A1);
        mirror_row(A1, B1);
    } else {
        next_row(B1);
        next_row(A1);
    }
#pragma unroll
    for (int p = 0; p < VP; ++p) dA1[p] = yface_flux2(B1[p], A1[p], k2);
    if constexpr (ONE) {
        // one step of rows ya..yb-1: the current row's cells in A1, the faces
        // below it in dA1 (a copy per row: this pass is taken at most once
        // per call)
#pragma unroll 1
        for (int q = ya; q < yb && ok; ++q) {
            if (q + 1 < ny)
                next_row(B1);
            else
                mirror_row(A1, B1);
#pragma unroll
            for (int p = 0; p < VP; ++p) dB1[p] = yface_flux2(A1[p], B1[p], k2);
            F2 oh[VP], ou[VP], ov[VP];
            stream_update<VP, SPLIT>(A1, dA1, dB1, k2, oh, ou, ov);
            store_next(oh, ou, ov);
#pragma unroll
            for (int p = 0; p < VP; ++p) {
                A1[p] = B1[p];
                dA1[p] = dB1[p];
            }
        }
    } else {
        // the intermediate rows ya - 1 (if any) and ya; afterwards the current
        // first-step row is ya + 1 in A1/dA1 and the current second-step row ya
        // in A2/dA2
        if (ya == 0) {
            first_step(top, 0, A1, B1, dA1, dB1, A2);
            mirror_row(A2, B2);
#pragma unroll
            for (int p = 0; p < VP; ++p) {
                A1[p] = B1[p];
                dA1[p] = dB1[p];
            }
        } else {
            first_step(top, ya - 1, A1, B1, dA1, dB1, B2);
            first_step(top, ya, B1, A1, dB1, dA1, A2);
        }
#pragma unroll
        for (int p = 0; p < VP; ++p) dA2[p] = yface_flux2(B2[p], A2[p], k2);

        // rows up to qr read their upper neighbour from the ring
        const int qr = min(q1, ny - 2);
        int q = ya + 1;
#pragma unroll 1
        for (; q + 1 <= qr && ok; q += 2) {
            first_step(inner, q, A1, B1, dA1, dB1, B2);
            second_step(A2, B2, dA2, dB2);
            first_step(inner, q + 1, B1, A1, dB1, dA1, A2);
            second_step(B2, A2, dB2, dA2);
        }
#pragma unroll 1
        for (; q <= q1 && ok; ++q) {  // at most two rows: an odd one and the grid's last
            first_step(top, q, A1, B1, dA1, dB1, B2);
            second_step(A2, B2, dA2, dB2);
#pragma unroll
            for (int p = 0; p < VP; ++p) {
                A1[p] = B1[p];
                dA1[p] = dB1[p];
                A2[p] = B2[p];
                dA2[p] = dB2[p];
            }
        }
        if (ok && yb == ny) {  // the top row: the row above is the mirror
            mirror_row(A2, B2);
            second_step(A2, B2, dA2, dB2);
        }
    }
    if (!ok) {
        // chunk ci timed out: wait (bounded) for it and the others in flight
        for (int c = ci; c < issued; ++c) {
            const int sl = c % NSLOT;
            (void)__all_sync(kFull, mbar_wait_bounded(w.bars + sl, (w.phase >> sl) & 1u, w.err, 100000000ull));
            w.phase ^= 1u << sl;
        }
    }
    return ok;
}

// ---------------------------------------------------------------------------
// Scalar lanes (FP64): a lane holds VX = 16 / sizeof(T) consecutive cells
// (one 16-byte vector per plane) as CellQ<T>; the strips, row ranges, TMA
// ring and two-phase row loop are those of the paired lanes above.  FP64
// runs at a small fraction of the FP32 rate on GB300, so what the streaming
// layout saves here is arithmetic: every cell's fluxes, x-face and y-face are
// formed once (the tiled one-step kernel forms two neighbour cells and one
// extra face for every two cells of a row).
// ---------------------------------------------------------------------------
template <typename T, int LO, int NO, int CR, int NSLOT, int WARPS>
struct StreamCfgS {
    static constexpr int VX = 16 / (int)sizeof(T);  // cells per lane
    static constexpr int BW = 32 * VX;              // columns a warp holds (the TMA box width)
    static constexpr int OUT = NO * VX;             // columns it stores: lanes LO .. LO + NO - 1
    static constexpr int ROWS = CR;
    static constexpr uint32_t PLANE_BYTES = BW * CR * sizeof(T);
    static constexpr uint32_t CHUNK_BYTES = 3 * PLANE_BYTES;
    static constexpr size_t WARP_BYTES = (size_t)NSLOT * CHUNK_BYTES;
    static constexpr size_t SMEM = WARPS * WARP_BYTES + WARPS * NSLOT * sizeof(uint64_t);
    static_assert(LO >= 1 && LO + NO <= 31, "an overlap lane on each side of the stored ones");
    static_assert((OUT * sizeof(T)) % 32 == 0 && (LO * VX * sizeof(T)) % 16 == 0,
                  "32-byte output rows, 16-byte aligned boxes");
};

template <typename Cfg, int CR, int NSLOT>
struct StreamWarpS {
    const CUtensorMap *mH, *mU, *mV;
    unsigned char *ring;
    uint64_t *bars;
    uint32_t phase;
    int *err;

    __device__ __forceinline__ void issue(int c, int x, int first)
    {
        const int slot = c % NSLOT;
        unsigned char *dst = ring + (size_t)slot * Cfg::CHUNK_BYTES;
        mbar_arrive_expect_tx(bars + slot, Cfg::CHUNK_BYTES);
        tma_load_2d(dst, mH, bars + slot, x, first + c * CR);
        tma_load_2d(dst + Cfg::PLANE_BYTES, mU, bars + slot, x, first + c * CR);
        tma_load_2d(dst + 2 * Cfg::PLANE_BYTES, mV, bars + slot, x, first + c * CR);
    }
};

// x-faces of a lane's cells: F[j] is the face left of cell j, F[VX] the face
// right of the last cell (the upper lane's F[0]); the left neighbour of cell
// 0 is the lower lane's last cell.  Walls are in the data (stream_ghosts_s).
template <typename T, int VX>
__device__ __forceinline__ void stream_xfaces_s(const CellQ<T> (&c)[VX], const Coef<T> &k, Flux3<T> (&F)[VX + 1])
{
    CellQ<T> L;
    L.h = __shfl_up_sync(kFull, c[VX - 1].h, 1);
    L.u = __shfl_up_sync(kFull, c[VX - 1].u, 1);
    L.v = __shfl_up_sync(kFull, c[VX - 1].v, 1);
    L.f2 = __shfl_up_sync(kFull, c[VX - 1].f2, 1);
    L.f3 = __shfl_up_sync(kFull, c[VX - 1].f3, 1);
    L.g3 = T(0);  // not read by an x-face
    F[0] = xface_flux(L, c[0], k);
#pragma unroll
    for (int j = 1; j < VX; ++j) F[j] = xface_flux(c[j - 1], c[j], k);
    F[VX].a = __shfl_down_sync(kFull, F[0].a, 1);
    F[VX].b = __shfl_down_sync(kFull, F[0].b, 1);
    F[VX].c = __shfl_down_sync(kFull, F[0].c, 1);
}

// stream_ghosts for scalar lanes: column -1 takes column 0's raw state with
// hu negated, column nx column nx - 1's (make_cell of the mirrored state has
// exactly the bits of mirror_x of the cell).
template <typename T, int VX>
__device__ __forceinline__ void stream_ghosts_s(T (&h)[VX], T (&u)[VX], T (&v)[VX], int gx0, int nx)
{
    const T ph = __shfl_up_sync(kFull, h[VX - 1], 1), pu = __shfl_up_sync(kFull, u[VX - 1], 1),
            pv = __shfl_up_sync(kFull, v[VX - 1], 1);
    const T nh = __shfl_down_sync(kFull, h[0], 1), nu = __shfl_down_sync(kFull, u[0], 1),
            nv = __shfl_down_sync(kFull, v[0], 1);
    T gh[VX], gu[VX], gv[VX];
#pragma unroll
    for (int j = 0; j < VX; ++j) {
        gh[j] = h[j];
        gu[j] = u[j];
        gv[j] = v[j];
        const int col = gx0 + j;
        if (col == -1) {
            gh[j] = j + 1 < VX ? h[j + 1] : nh;
            gu[j] = -(j + 1 < VX ? u[j + 1] : nu);
            gv[j] = j + 1 < VX ? v[j + 1] : nv;
        } else if (col == nx) {
            gh[j] = j > 0 ? h[j - 1] : ph;
            gu[j] = -(j > 0 ? u[j - 1] : pu);
            gv[j] = j > 0 ? v[j - 1] : pv;
        }
    }
#pragma unroll
    for (int j = 0; j < VX; ++j) {
        h[j] = gh[j];
        u[j] = gu[j];
        v[j] = gv[j];
    }
}

// stream_segment for scalar lanes: two steps (ONE: one step) of output rows
// [ya, yb) of the strip whose stored lanes start at column xs; false after a
// timed-out wait; bad set for a stored depth that is not positive.
template <bool EDGE, typename T, int LO, int NO, int CR, int NSLOT, int WARPS, bool ONE = false>
__device__ __forceinline__ bool stream_segment_s(StreamWarpS<StreamCfgS<T, LO, NO, CR, NSLOT, WARPS>, CR, NSLOT> &w,
                                                 T *__restrict__ oH, T *__restrict__ oU, T *__restrict__ oV, int nx,
                                                 int ny, long long pitch, int xs, int ya, int yb, const Coef<T> &k,
                                                 bool &bad)
{
    using C = StreamCfgS<T, LO, NO, CR, NSLOT, WARPS>;
    constexpr int VX = C::VX;
    using V = typename VecOf<T>::type;  // the 16-byte vector of a lane's cells
    const int lane = threadIdx.x & 31;
    const int bx = xs - LO * VX;
    const int gx0 = bx + VX * lane;
    const bool stores = lane >= LO && lane < LO + NO && gx0 < nx;
    const int q0 = ONE ? ya : max(ya - 1, 0), q1 = ONE ? yb - 1 : min(yb, ny - 1);
    const int first = q0 > 0 ? q0 - 1 : 0;
    const int last = min(q1 + 1, ny - 1);
    const int nch = (last - first) / CR + 1;
    int issued = min(NSLOT, nch);
    __syncwarp();
    if (lane == 0) {
        fence_proxy_async_smem();
        for (int c = 0; c < issued; ++c) w.issue(c, bx, first);
    }
    bool ok = true;
    int rr = CR, ci = -1, slot = NSLOT - 1;
    const T *rp = reinterpret_cast<const T *>(w.ring) + VX * lane;
    using Cells = CellQ<T>[VX];
    using Faces = Flux3<T>[VX];
    auto next_row = [&](Cells &c) {
        if (rr == CR) {
            if (ok) {
                ++ci;
                slot = slot + 1 == NSLOT ? 0 : slot + 1;
                if (ci >= 1 && issued < nch) {
                    __syncwarp();
                    if (lane == 0) {
                        fence_proxy_async_smem();
                        w.issue(issued, bx, first);
                    }
                    ++issued;
                }
                if (__all_sync(kFull, mbar_wait_bounded(w.bars + slot, (w.phase >> slot) & 1u, w.err)))
                    w.phase ^= 1u << slot;
                else
                    ok = false;
                rp = reinterpret_cast<const T *>(w.ring + (size_t)slot * C::CHUNK_BYTES) + VX * lane;
            }
            rr = 0;
        }
        const T *p = rp + rr * C::BW;
        ++rr;
        const V h4 = *reinterpret_cast<const V *>(p);
        const V u4 = *reinterpret_cast<const V *>(p + C::BW * CR);
        const V v4 = *reinterpret_cast<const V *>(p + 2 * C::BW * CR);
        T h[VX], u[VX], v[VX];
#pragma unroll
        for (int j = 0; j < VX; ++j) {
            h[j] = reinterpret_cast<const T *>(&h4)[j];
            u[j] = reinterpret_cast<const T *>(&u4)[j];
            v[j] = reinterpret_cast<const T *>(&v4)[j];
        }
        if (EDGE) stream_ghosts_s<T, VX>(h, u, v, gx0, nx);
#pragma unroll
        for (int j = 0; j < VX; ++j) c[j] = make_cell<T>(h[j], u[j], v[j], k.hg);
    };
    long long orow = (long long)ya * pitch + gx0;
    auto store_next = [&](const T(&oh)[VX], const T(&ou)[VX], const T(&ov)[VX]) {
        if (stores && ok) {
            store_vec<T, VX>(oH + orow, oh);
            store_vec<T, VX>(oU + orow, ou);
            store_vec<T, VX>(oV + orow, ov);
#pragma unroll
            for (int j = 0; j < VX; ++j) bad |= gx0 + j < nx && !(oh[j] > T(0));
        }
        orow += pitch;
    };
    auto mirror_row = [](const Cells &c, Cells &m) {
#pragma unroll
        for (int j = 0; j < VX; ++j) m[j] = mirror_y(c[j]);
    };
    auto update = [&](const Cells &c, const Faces &d, const Faces &u, T(&oh)[VX], T(&ou)[VX], T(&ov)[VX]) {
        Flux3<T> F[VX + 1];
        stream_xfaces_s<T, VX>(c, k, F);
#pragma unroll
        for (int j = 0; j < VX; ++j) {
            oh[j] = c[j].h;
            ou[j] = c[j].u;
            ov[j] = c[j].v;
            lw_update(oh[j], ou[j], ov[j], F[j], F[j + 1], d[j], u[j], k);
        }
    };
    auto first_step = [&](auto top, int q, const Cells &c, Cells &n, const Faces &d, Faces &u, Cells &m) {
        if (!decltype(top)::value || q + 1 < ny)
            next_row(n);
        else
            mirror_row(c, n);
#pragma unroll
        for (int j = 0; j < VX; ++j) u[j] = yface_flux(c[j], n[j], k);
        T oh[VX], ou[VX], ov[VX];
        update(c, d, u, oh, ou, ov);
        if (EDGE) stream_ghosts_s<T, VX>(oh, ou, ov, gx0, nx);
#pragma unroll
        for (int j = 0; j < VX; ++j) m[j] = make_cell<T>(oh[j], ou[j], ov[j], k.hg);
    };
    const std::true_type top;
    const std::false_type inner;
    auto second_step = [&](const Cells &c2, const Cells &n2, const Faces &d2, Faces &u2) {
#pragma unroll
        for (int j = 0; j < VX; ++j) u2[j] = yface_flux(c2[j], n2[j], k);
        T oh[VX], ou[VX], ov[VX];
        update(c2, d2, u2, oh, ou, ov);
        store_next(oh, ou, ov);
    };
    auto copy = [](const Cells &a, Cells &b, const Faces &fa, Faces &fb) {
#pragma unroll
        for (int j = 0; j < VX; ++j) {
            b[j] = a[j];
            fb[j] = fa[j];
        }
    };

    Cells A1, B1, A2, B2;
    Faces dA1, dB1, dA2, dB2;
    if (q0 == 0) {
        next_row(A1);
        mirror_row(A1, B1);
    } else {
        next_row(B1);
        next_row(A1);
    }
#pragma unroll
    for (int j = 0; j < VX; ++j) dA1[j] = yface_flux(B1[j], A1[j], k);
    if constexpr (ONE) {
#pragma unroll 1
        for (int q = ya; q < yb && ok; ++q) {
            if (q + 1 < ny)
                next_row(B1);
            else
                mirror_row(A1, B1);
#pragma unroll
            for (int j = 0; j < VX; ++j) dB1[j] = yface_flux(A1[j], B1[j], k);
            T oh[VX], ou[VX], ov[VX];
            update(A1, dA1, dB1, oh, ou, ov);
            store_next(oh, ou, ov);
            copy(B1, A1, dB1, dA1);
        }
    } else {
        if (ya == 0) {
            first_step(top, 0, A1, B1, dA1, dB1, A2);
            mirror_row(A2, B2);
            copy(B1, A1, dB1, dA1);
        } else {
            first_step(top, ya - 1, A1, B1, dA1, dB1, B2);
            first_step(top, ya, B1, A1, dB1, dA1, A2);
        }
#pragma unroll
        for (int j = 0; j < VX; ++j) dA2[j] = yface_flux(B2[j], A2[j], k);
        const int qr = min(q1, ny - 2);
        int q = ya + 1;
#pragma unroll 1
        for (; q + 1 <= qr && ok; q += 2) {
            first_step(inner, q, A1, B1, dA1, dB1, B2);
            second_step(A2, B2, dA2, dB2);
            first_step(inner, q + 1, B1, A1, dB1, dA1, A2);
            second_step(B2, A2, dB2, dA2);
        }
#pragma unroll 1
        for (; q <= q1 && ok; ++q) {
            first_step(top, q, A1, B1, dA1, dB1, B2);
            second_step(A2, B2, dA2, dB2);
            copy(B1, A1, dB1, dA1);
            copy(B2, A2, dB2, dA2);
        }
        if (ok && yb == ny) {
            mirror_row(A2, B2);
            second_step(A2, B2, dA2, dB2);
        }
    }
    if (!ok) {
        for (int c = ci; c < issued; ++c) {
            const int sl = c % NSLOT;
            (void)__all_sync(kFull, mbar_wait_bounded(w.bars + sl, (w.phase >> sl) & 1u, w.err, 100000000ull));
            w.phase ^= 1u << sl;
        }
    }
    return ok;
}

}  // namespace swe
