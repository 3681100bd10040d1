// swe_tile.cuh -- the tile computation shared by the single-grid and the
// batched step kernels: a CTA holds a tile of H, U, V plus its halo in
// shared memory (box layout below) and computes one Lax-Wendroff step of
// the tile's cells (Sec. 3 step equations), storing them to global memory.
#pragma once

#include <type_traits>

#include "swe_device.cuh"

namespace swe {

template <typename T>
struct VecOf;
template <>
struct VecOf<float> {
    static constexpr int N = 4;
    using type = float4;
};
template <>
struct VecOf<double> {
    static constexpr int N = 2;
    using type = double2;
};

template <typename T, int NWARP, int RY>
struct TiledCfg {
    static constexpr int VX = VecOf<T>::N;  // cells per thread in x (16 bytes)
    static constexpr int TX = 32 * VX;      // tile width (one warp across)
    static constexpr int TY = NWARP * RY;   // tile height (warps stacked)
    static constexpr int ROWS = RY;         // rows per warp
    static constexpr int AX = VX;           // x halo, rounded up to 16 bytes
    static constexpr int BW = TX + 2 * AX;  // TMA box width
    static constexpr int BH = TY + 2;       // TMA box height
    static constexpr size_t BOX_BYTES = (size_t)BW * BH * sizeof(T);
    static constexpr size_t BOX_STRIDE = (BOX_BYTES + 127) / 128 * 128;
    static constexpr size_t SMEM = 3 * BOX_STRIDE + 128;
};

template <typename T, int VX>
__device__ __forceinline__ void load_row(const T *sH, const T *sU, const T *sV, int idx, T hg, CellQ<T> (&c)[VX])
{
    using V = typename VecOf<T>::type;
    const V h = *reinterpret_cast<const V *>(sH + idx);
    const V u = *reinterpret_cast<const V *>(sU + idx);
    const V v = *reinterpret_cast<const V *>(sV + idx);
    const T *ph = reinterpret_cast<const T *>(&h);
    const T *pu = reinterpret_cast<const T *>(&u);
    const T *pv = reinterpret_cast<const T *>(&v);
#pragma unroll
    for (int p = 0; p < VX; ++p) c[p] = make_cell<T>(ph[p], pu[p], pv[p], hg);
}

// Shared-memory boxes as strip_compute reads them: three planes (SoA), or
// one array of (h, hu, hv, pad) cells (the packed layout, FP32).  idx is a
// cell index of the box.
template <typename T>
struct SoaBox {
    const T *h, *u, *v;
    template <int VX>
    __device__ __forceinline__ void row(int idx, T hg, CellQ<T> (&c)[VX]) const
    {
        load_row<T, VX>(h, u, v, idx, hg, c);
    }
    __device__ __forceinline__ CellQ<T> cell(int idx, T hg) const { return make_cell<T>(h[idx], u[idx], v[idx], hg); }
    // FP32: cells idx .. idx+3 as the pairs (0, 1), (2, 3); and two single
    // cells a, b as one pair
    __device__ __forceinline__ void row2(int idx, const Coef2 &k, CellQ2 (&c)[2]) const
    {
        const float4 hh = *reinterpret_cast<const float4 *>(h + idx);
        const float4 uu = *reinterpret_cast<const float4 *>(u + idx);
        const float4 vv = *reinterpret_cast<const float4 *>(v + idx);
        c[0] = make_cell2(pack2(hh.x, hh.y), pack2(uu.x, uu.y), pack2(vv.x, vv.y), k);
        c[1] = make_cell2(pack2(hh.z, hh.w), pack2(uu.z, uu.w), pack2(vv.z, vv.w), k);
    }
    __device__ __forceinline__ CellQ2 cell2(int a, int b, const Coef2 &k) const
    {
        return make_cell2(pack2(h[a], h[b]), pack2(u[a], u[b]), pack2(v[a], v[b]), k);
    }
};

struct PackedBox {
    const float4 *p;
    template <int VX>
    __device__ __forceinline__ void row(int idx, float hg, CellQ<float> (&c)[VX]) const
    {
#pragma unroll
        for (int q = 0; q < VX; ++q) {
            const float4 s = p[idx + q];
            c[q] = make_cell<float>(s.x, s.y, s.z, hg);
        }
    }
    __device__ __forceinline__ CellQ<float> cell(int idx, float hg) const
    {
        const float4 s = p[idx];
        return make_cell<float>(s.x, s.y, s.z, hg);
    }
    __device__ __forceinline__ void row2(int idx, const Coef2 &k, CellQ2 (&c)[2]) const
    {
        const float4 s0 = p[idx], s1 = p[idx + 1], s2 = p[idx + 2], s3 = p[idx + 3];
        c[0] = make_cell2(pack2(s0.x, s1.x), pack2(s0.y, s1.y), pack2(s0.z, s1.z), k);
        c[1] = make_cell2(pack2(s2.x, s3.x), pack2(s2.y, s3.y), pack2(s2.z, s3.z), k);
    }
    __device__ __forceinline__ CellQ2 cell2(int a, int b, const Coef2 &k) const
    {
        const float4 sa = p[a], sb = p[b];
        return make_cell2(pack2(sa.x, sb.x), pack2(sa.y, sb.y), pack2(sa.z, sb.z), k);
    }
};

template <typename T, int VX>
__device__ __forceinline__ void store_vec(T *dst, const T (&x)[VX])
{
    using V = typename VecOf<T>::type;
    *reinterpret_cast<V *>(dst) = *reinterpret_cast<const V *>(x);
}

// The arithmetic of one thread's VX-cell column vector over tile-local rows
// [r_begin, r_end): marching down, each y-face flux is computed once and
// carried to the next row; x-faces come from the thread's cells and the two
// neighbours in the same row.  The box holds the tile-local cell (c, r) at
// shared index (r + row_off) * BW + c + AX.  Reflective walls are applied
// where neighbours are formed (XEDGE: the tile touches an x-wall).  Rows
// must lie inside the grid (0 <= y0 + r < ny).  ``store(r, h, hu, hv)``
// receives each finished row.
// GHOSTED: the box's halo holds real neighbour cells everywhere (a
// partition's ghost ring), so no wall is formed; use with XEDGE = false.
// The FP32, four-cells-per-thread form of strip_compute_box for columns away
// from an x-wall, on the packed FP32 pipe: the thread's cells form the pairs
// (0, 1) and (2, 3); its five x-faces are computed as the pairs (F0, F1),
// (F2, F3) and F4 alone, its four y-faces and updates as two pairs.  Every
// value goes through the operations of the scalar routine, so the bits are
// the same.
template <bool GHOSTED, typename Box, typename Store>
__device__ __forceinline__ void strip_compute_pairs(const Box &box, int BW, int AX, int row_off, int r_begin,
                                                    int r_end, int cx, int ny, int y0, const Coef<float> &k,
                                                    Store &&store)
{
    auto sidx = [&](int c, int r) { return (r + row_off) * BW + c + AX; };
    const Coef2 k2 = coef2(k);
    CellQ2 ca[2], cb[2];
    Flux2 ga[2], gb[2];

    // One row: ``cur`` holds row r and ``gd`` its lower y-faces; row r + 1
    // goes to ``nxt`` and the faces between them to ``gu``.  The loop below
    // alternates the roles of the two sets, so nothing is copied per row.
    auto row = [&](int r, CellQ2(&cur)[2], CellQ2(&nxt)[2], const Flux2(&gd)[2], Flux2(&gu)[2]) {
        if (!GHOSTED && y0 + r + 1 == ny) {
            nxt[0] = mirror_y2(cur[0]);
            nxt[1] = mirror_y2(cur[1]);
        } else {
            box.row2(sidx(cx, r + 1), k2, nxt);
        }
        gu[0] = yface_flux2(cur[0], nxt[0], k2);
        gu[1] = yface_flux2(cur[1], nxt[1], k2);

        // (left, right) neighbours of the thread's four cells on row r
        const CellQ2 lr = box.cell2(sidx(cx - 1, r), sidx(cx + 4, r), k2);
        const CellQ<float> c1 = cell_hi(cur[0]), c2 = cell_lo(cur[1]), c3 = cell_hi(cur[1]);
        const Flux2 F01 = xface_flux2(pair_cells(cell_lo(lr), cell_lo(cur[0])), cur[0], k2);
        const Flux2 F23 = xface_flux2(pair_cells(c1, c2), cur[1], k2);
        const Flux3<float> F4 = xface_flux(c3, cell_hi(lr), k);
        const Flux2 F12 = flux_pair(hi2(F01.a), hi2(F01.b), hi2(F01.c), lo2(F23.a), lo2(F23.b), lo2(F23.c));
        const Flux2 F34 = flux_pair(hi2(F23.a), hi2(F23.b), hi2(F23.c), F4.a, F4.b, F4.c);

        F2 oh0 = cur[0].h, ou0 = cur[0].u, ov0 = cur[0].v;
        F2 oh1 = cur[1].h, ou1 = cur[1].u, ov1 = cur[1].v;
        lw_update2(oh0, ou0, ov0, F01, F12, gd[0], gu[0], k2);
        lw_update2(oh1, ou1, ov1, F23, F34, gd[1], gu[1], k2);
        float oh[4], ou[4], ov[4];
        unpack2(oh0, oh[0], oh[1]);
        unpack2(oh1, oh[2], oh[3]);
        unpack2(ou0, ou[0], ou[1]);
        unpack2(ou1, ou[2], ou[3]);
        unpack2(ov0, ov[0], ov[1]);
        unpack2(ov1, ov[2], ov[3]);
        store(r, oh, ou, ov);
    };

    box.row2(sidx(cx, r_begin), k2, ca);
    if (!GHOSTED && y0 + r_begin == 0) {
        cb[0] = mirror_y2(ca[0]);
        cb[1] = mirror_y2(ca[1]);
    } else {
        box.row2(sidx(cx, r_begin - 1), k2, cb);
    }
    ga[0] = yface_flux2(cb[0], ca[0], k2);
    ga[1] = yface_flux2(cb[1], ca[1], k2);

    int r = r_begin;
#pragma unroll 1
    for (; r + 1 < r_end; r += 2) {
        row(r, ca, cb, ga, gb);
        row(r + 1, cb, ca, gb, ga);
    }
    if (r < r_end) row(r, ca, cb, ga, gb);
}

template <typename T, int VX, bool XEDGE, typename Box, typename Store, bool GHOSTED = false>
__device__ __forceinline__ void strip_compute_box(const Box &box, int BW, int AX, int row_off, int r_begin, int r_end,
                                                  int cx, int gx, int nx, int ny, int y0, const Coef<T> &k,
                                                  Store &&store)
{
    if (r_begin >= r_end) return;
    if constexpr (std::is_same<T, float>::value && VX == 4 && !XEDGE) {
        strip_compute_pairs<GHOSTED>(box, BW, AX, row_off, r_begin, r_end, cx, ny, y0, k, store);
        return;
    }
    auto sidx = [&](int c, int r) { return (r + row_off) * BW + c + AX; };
    const int pw = nx - gx;  // window position of the right wall ghost, if in 1..VX

    CellQ<T> cur[VX], nxt[VX];
    Flux3<T> gd[VX], gu[VX];

    box.template row<VX>(sidx(cx, r_begin), k.hg, cur);
    if (!GHOSTED && y0 + r_begin == 0) {
#pragma unroll
        for (int p = 0; p < VX; ++p) nxt[p] = mirror_y(cur[p]);
    } else {
        box.template row<VX>(sidx(cx, r_begin - 1), k.hg, nxt);
    }
#pragma unroll
    for (int p = 0; p < VX; ++p) gd[p] = yface_flux(nxt[p], cur[p], k);

#pragma unroll 1
    for (int r = r_begin; r < r_end; ++r) {
        const int gy = y0 + r;
        if (!GHOSTED && gy + 1 == ny) {
#pragma unroll
            for (int p = 0; p < VX; ++p) nxt[p] = mirror_y(cur[p]);
        } else {
            box.template row<VX>(sidx(cx, r + 1), k.hg, nxt);
        }
#pragma unroll
        for (int p = 0; p < VX; ++p) gu[p] = yface_flux(cur[p], nxt[p], k);

        // x-neighbours of the thread's cells on row r
        CellQ<T> left = box.cell(sidx(cx - 1, r), k.hg);
        CellQ<T> right = box.cell(sidx(cx + VX, r), k.hg);
        if (XEDGE) {
            if (gx == 0) left = mirror_x(cur[0]);
            if (pw == VX) right = mirror_x(cur[VX - 1]);
        }
        Flux3<T> F[VX + 1];
        F[0] = xface_flux(left, cur[0], k);
#pragma unroll
        for (int p = 1; p < VX; ++p) {
            if (XEDGE && p == pw)
                F[p] = xface_flux(cur[p - 1], mirror_x(cur[p - 1]), k);
            else
                F[p] = xface_flux(cur[p - 1], cur[p], k);
        }
        F[VX] = xface_flux(cur[VX - 1], right, k);

        T oh[VX], ou[VX], ov[VX];
#pragma unroll
        for (int p = 0; p < VX; ++p) {
            oh[p] = cur[p].h;
            ou[p] = cur[p].u;
            ov[p] = cur[p].v;
            lw_update(oh[p], ou[p], ov[p], F[p], F[p + 1], gd[p], gu[p], k);
        }
        store(r, oh, ou, ov);
#pragma unroll
        for (int p = 0; p < VX; ++p) {
            cur[p] = nxt[p];
            gd[p] = gu[p];
        }
    }
}

template <typename T, int VX, bool XEDGE, typename Store>
__device__ __forceinline__ void strip_compute(const T *sH, const T *sU, const T *sV, int BW, int AX, int row_off,
                                              int r_begin, int r_end, int cx, int gx, int nx, int ny, int y0,
                                              const Coef<T> &k, Store &&store)
{
    strip_compute_box<T, VX, XEDGE>(SoaBox<T>{sH, sU, sV}, BW, AX, row_off, r_begin, r_end, cx, gx, nx, ny, y0, k,
                                    store);
}

// One cell of a box, computed on its own from the 5-point neighbourhood (the
// same face and update functions as strip_compute, so the same bits).
template <typename T>
__device__ __forceinline__ void box_cell(const T *sH, const T *sU, const T *sV, int BW, int AX, int row_off, int c,
                                         int r, int gx, int gy, int nx, int ny, const Coef<T> &k, T &h, T &hu, T &hv)
{
    auto cell = [&](int cc, int rr) {
        const int i = (rr + row_off) * BW + cc + AX;
        return make_cell<T>(sH[i], sU[i], sV[i], k.hg);
    };
    const CellQ<T> C = cell(c, r);
    const CellQ<T> L = gx == 0 ? mirror_x(C) : cell(c - 1, r);
    const CellQ<T> R = gx == nx - 1 ? mirror_x(C) : cell(c + 1, r);
    const CellQ<T> D = gy == 0 ? mirror_y(C) : cell(c, r - 1);
    const CellQ<T> U = gy == ny - 1 ? mirror_y(C) : cell(c, r + 1);
    const Flux3<T> Fl = xface_flux(L, C, k), Fr = xface_flux(C, R, k);
    const Flux3<T> Gd = yface_flux(D, C, k), Gu = yface_flux(C, U, k);
    h = C.h;
    hu = C.u;
    hv = C.v;
    lw_update(h, hu, hv, Fl, Fr, Gd, Gu, k);
}

// Which cells of a tile a thread computes.  A warp normally spans the tile's
// TX columns, VX cells per lane.  When the grid ends within TX/2 (TX/4)
// columns of the tile's left edge -- the last column strip of a grid whose
// width is not a multiple of TX -- the warp is cut into G = 2 (4) lane groups
// of TX/G columns that take different rows, so such a tile costs 1/G of the
// row iterations of a full one.  The rows [r0, r1) are cut into NWARP * G
// runs of (nearly) equal length, one per lane group: RY rows per warp for a
// full tile, fewer per warp for a tile cut short by the grid's last row.
// The cell arithmetic does not depend on which thread runs it, so the bits
// do not either.
struct TileWork {
    int cx;      // first tile column of the thread's VX cells
    int rb, re;  // its tile rows [rb, re)
};

template <int TX, int VX, int NWARP>
__device__ __forceinline__ TileWork tile_work(bool xedge, int x0, int nx, int r0, int r1)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int w = nx - x0;  // grid columns from the tile's left edge on
    const int G = !xedge ? 1 : (w <= TX / 4 ? 4 : (w <= TX / 2 ? 2 : 1));
    const int L = 32 / G;                   // lanes per group
    const int j = warp * G + lane / L;      // the group's index in the CTA
    const int n = max(r1 - r0, 0), W = NWARP * G;
    return TileWork{(lane % L) * VX, r0 + j * n / W, r0 + (j + 1) * n / W};
}

// Computes one output tile from the staged box (see TiledCfg; the box's
// first row is tile row -ROW_OFF) and stores it.  Returns true if some
// stored depth is not positive (h <= 0 or NaN).
template <typename T, int NWARP, int RY, bool XEDGE, int ROW_OFF = 1, bool GHOSTED = false>
__device__ __forceinline__ bool tiled_compute(const T *sH, const T *sU, const T *sV, T *__restrict__ oH,
                                              T *__restrict__ oU, T *__restrict__ oV, int nx, int ny,
                                              long long pitch, int x0, int y0, const Coef<T> &k)
{
    using C = TiledCfg<T, NWARP, RY>;
    constexpr int VX = C::VX;
    const TileWork tw = tile_work<C::TX, VX, NWARP>(XEDGE, x0, nx, 0, min(C::TY, ny - y0));
    const int cx = tw.cx;
    const int gx = x0 + cx;
    const int rb = tw.rb;
    const int re = tw.re;
    bool bad = false;
    auto store_fn = [&](int r, const T(&oh)[VX], const T(&ou)[VX], const T(&ov)[VX]) {
        if (gx < nx) {
#pragma unroll
            for (int p = 0; p < VX; ++p) bad |= (gx + p < nx) && !(oh[p] > T(0));
            // whole 16-byte vectors: columns past nx land in the row padding
            const size_t o = (size_t)(y0 + r) * (size_t)pitch + (size_t)gx;
            store_vec<T, VX>(oH + o, oh);
            store_vec<T, VX>(oU + o, ou);
            store_vec<T, VX>(oV + o, ov);
        }
    };
    strip_compute_box<T, VX, XEDGE, SoaBox<T>, decltype(store_fn) &, GHOSTED>(
        SoaBox<T>{sH, sU, sV}, C::BW, C::AX, ROW_OFF, rb, re, cx, gx, nx, ny, y0, k, store_fn);
    return bad;
}

// ---------------------------------------------------------------------------
// Two steps of one tile (temporal blocking).  The input box holds the tile
// with a two-cell y-halo (box origin (x0 - AX, y0 - 2), TY + 4 rows); the
// intermediate state of the tile plus a one-cell ring goes to a second box
// laid out like the one-step kernel's input box, and the one-step tile
// routine takes the second step from there.  Every cell goes through the
// same face and update functions as in the one-step kernel, so the result
// equals two one-step passes bit for bit.  All threads of the CTA call it.
// ---------------------------------------------------------------------------
template <typename T, int NWARP, int RY>
struct Tb2Cfg {
    using C = TiledCfg<T, NWARP, RY>;
    static constexpr int BH_IN = C::TY + 4;
    static constexpr size_t IN_BYTES = (size_t)C::BW * BH_IN * sizeof(T);
    static constexpr size_t IN_STRIDE = (IN_BYTES + 127) / 128 * 128;
    static constexpr size_t SMEM = 3 * IN_STRIDE + 3 * C::BOX_STRIDE + 128;
};

// Phase 1: the intermediate state on rows [-1, TY] of the tile's columns
// (the ring rows included) into the intermediate box, cut among the lane
// groups as phase 2 cuts them, so phase 2 finds every cell inside the grid
// that it reads here or in the ring columns.  All threads of the CTA call it.
template <typename T, int NWARP, int RY>
__device__ __forceinline__ void tb2_phase1(const T *iH, const T *iU, const T *iV, T *mH_, T *mU_, T *mV_, int nx,
                                           int ny, int x0, int y0, const Coef<T> &k)
{
    using C = TiledCfg<T, NWARP, RY>;
    constexpr int VX = C::VX;
    const bool xedge = (x0 == 0) || (x0 + C::TX >= nx);
    const TileWork tw = tile_work<C::TX, VX, NWARP>(xedge, x0, nx, max(-1, -y0), min(C::TY + 1, ny - y0));
    const int cx = tw.cx, gx = x0 + cx, r0 = tw.rb, r1 = tw.re;
    auto to_mid = [&](int r, const T(&h)[VX], const T(&u)[VX], const T(&v)[VX]) {
        const int o = (r + 1) * C::BW + cx + C::AX;
        store_vec<T, VX>(mH_ + o, h);
        store_vec<T, VX>(mU_ + o, u);
        store_vec<T, VX>(mV_ + o, v);
    };
    if (xedge)
        strip_compute<T, VX, true>(iH, iU, iV, C::BW, C::AX, 2, r0, r1, cx, gx, nx, ny, y0, k, to_mid);
    else
        strip_compute<T, VX, false>(iH, iU, iV, C::BW, C::AX, 2, r0, r1, cx, gx, nx, ny, y0, k, to_mid);
    // the ring columns -1 and TX, one cell at a time
    for (int idx = threadIdx.x; idx < 2 * (C::TY + 2); idx += blockDim.x) {
        const int c = (idx & 1) ? C::TX : -1;
        const int r = (idx >> 1) - 1;
        const int cgx = x0 + c, gy = y0 + r;
        if (cgx < 0 || cgx >= nx || gy < 0 || gy >= ny) continue;
        T h, hu, hv;
        box_cell<T>(iH, iU, iV, C::BW, C::AX, 2, c, r, cgx, gy, nx, ny, k, h, hu, hv);
        const int o = (r + 1) * C::BW + c + C::AX;
        mH_[o] = h;
        mU_[o] = hu;
        mV_[o] = hv;
    }
}

// Phase 2: the second step from the intermediate box to global memory.
// Returns true if some stored depth is not positive.
template <typename T, int NWARP, int RY>
__device__ __forceinline__ bool tb2_phase2(const T *mH_, const T *mU_, const T *mV_, T *__restrict__ oH,
                                           T *__restrict__ oU, T *__restrict__ oV, int nx, int ny, long long pitch,
                                           int x0, int y0, const Coef<T> &k)
{
    using C = TiledCfg<T, NWARP, RY>;
    const bool xedge = (x0 == 0) || (x0 + C::TX >= nx);
    if (xedge) return tiled_compute<T, NWARP, RY, true>(mH_, mU_, mV_, oH, oU, oV, nx, ny, pitch, x0, y0, k);
    return tiled_compute<T, NWARP, RY, false>(mH_, mU_, mV_, oH, oU, oV, nx, ny, pitch, x0, y0, k);
}

template <typename T, int NWARP, int RY>
__device__ __forceinline__ bool tb2_tile_compute(const T *iH, const T *iU, const T *iV, T *mH_, T *mU_, T *mV_,
                                                 T *__restrict__ oH, T *__restrict__ oU, T *__restrict__ oV,
                                                 int nx, int ny, long long pitch, int x0, int y0, const Coef<T> &k)
{
    tb2_phase1<T, NWARP, RY>(iH, iU, iV, mH_, mU_, mV_, nx, ny, x0, y0, k);
    __syncthreads();
    return tb2_phase2<T, NWARP, RY>(mH_, mU_, mV_, oH, oU, oV, nx, ny, pitch, x0, y0, k);
}

}  // namespace swe
