// swe_tile.cuh -- the tile computation shared by the single-grid and the
// batched step kernels: a CTA holds a tile of H, U, V plus its halo in
// shared memory (box layout below) and computes one Lax-Wendroff step of
// the tile's cells (Sec. 3 step equations), storing them to global memory.
#pragma once

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

template <typename T, int VX>
__device__ __forceinline__ void store_vec(T *dst, const T (&x)[VX])
{
    using V = typename VecOf<T>::type;
    *reinterpret_cast<V *>(dst) = *reinterpret_cast<const V *>(x);
}

// Computes one output tile from the staged box (see TiledCfg) and stores it.
// Returns true if some stored depth is not positive (h <= 0 or NaN).
template <typename T, int NWARP, int RY, bool XEDGE>
__device__ __forceinline__ bool tiled_compute(const T *sH, const T *sU, const T *sV, T *__restrict__ oH,
                                              T *__restrict__ oU, T *__restrict__ oV, int nx, int ny,
                                              long long pitch, int x0, int y0, const Coef<T> &k)
{
    bool bad = false;
    using C = TiledCfg<T, NWARP, RY>;
    constexpr int VX = C::VX;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int cx = lane * VX;  // tile-local first column of this thread
    const int gx = x0 + cx;
    const int rb = warp * RY;  // tile-local first row of this warp
    if (y0 + rb >= ny) return false;
    // shared-memory index of tile-local cell (c, r); the box starts at (-AX, -1)
    auto sidx = [](int c, int r) { return (r + 1) * C::BW + c + C::AX; };
    const int pw = nx - gx;  // window position of the right wall ghost, if in 1..VX

    CellQ<T> cur[VX], nxt[VX];
    Flux3<T> gd[VX], gu[VX];

    load_row<T, VX>(sH, sU, sV, sidx(cx, rb), k.hg, cur);
    if (y0 + rb == 0) {
#pragma unroll
        for (int p = 0; p < VX; ++p) nxt[p] = mirror_y(cur[p]);
    } else {
        load_row<T, VX>(sH, sU, sV, sidx(cx, rb - 1), k.hg, nxt);
    }
#pragma unroll
    for (int p = 0; p < VX; ++p) gd[p] = yface_flux(nxt[p], cur[p], k);

#pragma unroll
    for (int q = 0; q < RY; ++q) {
        const int r = rb + q;
        const int gy = y0 + r;
        if (gy >= ny) break;
        if (gy + 1 == ny) {
#pragma unroll
            for (int p = 0; p < VX; ++p) nxt[p] = mirror_y(cur[p]);
        } else {
            load_row<T, VX>(sH, sU, sV, sidx(cx, r + 1), k.hg, nxt);
        }
#pragma unroll
        for (int p = 0; p < VX; ++p) gu[p] = yface_flux(cur[p], nxt[p], k);

        // x-neighbours of the thread's cells on row r
        const int il = sidx(cx - 1, r), ir = sidx(cx + VX, r);
        CellQ<T> left = make_cell<T>(sH[il], sU[il], sV[il], k.hg);
        CellQ<T> right = make_cell<T>(sH[ir], sU[ir], sV[ir], k.hg);
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
        if (gx < nx) {
#pragma unroll
            for (int p = 0; p < VX; ++p) bad |= (gx + p < nx) && !(oh[p] > T(0));
            // whole 16-byte vectors: columns past nx land in the row padding
            const size_t o = (size_t)gy * (size_t)pitch + (size_t)gx;
            store_vec<T, VX>(oH + o, oh);
            store_vec<T, VX>(oU + o, ou);
            store_vec<T, VX>(oV + o, ov);
        }
#pragma unroll
        for (int p = 0; p < VX; ++p) {
            cur[p] = nxt[p];
            gd[p] = gu[p];
        }
    }
    return bad;
}


}  // namespace swe
