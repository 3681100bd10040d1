// swe_device.cuh -- device helpers shared by the stencil kernels: inline PTX
// for mbarriers and TMA tile loads, bounded waits, and the shallow-water flux
// algebra of the two-step Lax-Wendroff scheme (Sec. 3).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "swe_internal.h"

namespace swe {

// ---------------------------------------------------------------------------
// Bounded waits.  Every spin in this library gives up after this many
// nanoseconds of %globaltimer, records SWE_ETIMEOUT in the error word and
// lets the kernel return.
// ---------------------------------------------------------------------------
#ifndef SWE_WAIT_LIMIT_NS
#define SWE_WAIT_LIMIT_NS 2000000000ull
#endif

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes mbarrier initialisation visible to the async (TMA) proxy.
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for phase ``parity`` of ``bar`` to complete; gives up after
// SWE_WAIT_LIMIT_NS, records SWE_ETIMEOUT in *err and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int *err,
                                                  uint64_t limit_ns = SWE_WAIT_LIMIT_NS)
{
    for (int i = 0; i < 32; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer_ns() - t0 > limit_ns) {
            atomicExch(err, (int)SWE_ETIMEOUT);
            return false;
        }
    }
}

// 2D TMA tile load of the box at (x, y) of ``map`` into shared memory,
// completing on ``bar`` (transaction bytes).  x * element size must be a
// multiple of 16 bytes; out-of-range elements are filled with zeros.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

// 3D TMA tile load (box at (c0, c1, c2) of ``map``); c0 * element size must
// be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1, int c2)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap *map)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// Orders this thread's earlier generic-proxy view of global memory before its
// later async-proxy (TMA) reads: needed when a TMA load reads data that other
// CTAs stored in the same kernel.
__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Grid-wide barrier for a cooperatively launched kernel (all CTAs resident).
// ``count`` and ``gen`` are zero-initialised device words shared by every
// CTA.  Thread 0 of each CTA arrives; the last arrival resets the count and
// bumps the generation, the others wait for the generation to change.  The
// wait is bounded: after SWE_WAIT_LIMIT_NS it records SWE_ETIMEOUT in *err
// and the barrier returns false on every thread of the CTA.
struct GridBarrier {
    unsigned int count;
    unsigned int gen;
};

__device__ __forceinline__ bool grid_sync_bounded(GridBarrier *b, unsigned int nblocks, int *err,
                                                  uint64_t limit_ns = SWE_WAIT_LIMIT_NS)
{
    __shared__ int ok_shared;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned int *vgen = &b->gen;
        const unsigned int g0 = *vgen;
        __threadfence();
        if (atomicAdd(&b->count, 1u) == nblocks - 1) {
            atomicExch(&b->count, 0u);
            __threadfence();
            atomicAdd(&b->gen, 1u);
        } else {
            const uint64_t t0 = globaltimer_ns();
            while (*vgen == g0) {
                if (globaltimer_ns() - t0 > limit_ns) {
                    atomicExch(err, (int)SWE_ETIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok_shared = ok;
    }
    __syncthreads();
    return ok_shared != 0;
}

// ---------------------------------------------------------------------------
// Arithmetic.  rcp(): FP32 uses the hardware approximate reciprocal
// (rcp.approx, at most 1 ulp error); FP64 uses IEEE division.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rcp(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }

// Rounded products that the compiler may not fuse into a later add.  The
// flux products below feed subtractions (a - b*c); left to itself the
// compiler fuses such a pair into an FMA only where the product has a single
// use, which depends on the tile shape (a warp's first and last row).  With
// every product rounded, each cell's update is the same function of its
// neighbours for every tile shape, so all kernels give identical bits.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// Coefficients of the step.  The face functions below carry every face
// quantity doubled: with s = a + b and d a flux difference, the half step's
// 0.5 s + (0.5 dt/dx) d is evaluated as s + (dt/dx) d, which is exactly twice
// it in every rounding (a factor of two is exact, and lx = 2 hx exactly), and
// the update then takes (0.5 dt/dx) times the difference of doubled fluxes,
// which is exactly dt/dx times the difference of the fluxes.  This saves the
// three halvings of each face and gives the same bits as the plain form,
// provided the reciprocal of 2x is half the reciprocal of x: true of IEEE
// division and of rcp.approx (the latter checked on the GPU by the tests).
template <typename T>
struct Coef {
    T hx, hy;  // 0.5 dt/dx, 0.5 dt/dy: the update's factors on doubled fluxes
    T lx, ly;  // dt/dx, dt/dy: the doubled face states' factors
    T hg;      // g/2: the hydrostatic pressure g h^2 / 2 of a cell
    T qg;      // g/4 (= hg/2 exactly): the pressure of a doubled face state
};

template <typename T>
__host__ __device__ inline Coef<T> make_coef(double dx, double dy, double dt, double g)
{
    Coef<T> k;
    k.hx = (T)(0.5 * dt / dx);
    k.hy = (T)(0.5 * dt / dy);
    k.lx = (T)(dt / dx);
    k.ly = (T)(dt / dy);
    k.hg = (T)(0.5 * g);
    k.qg = k.hg * (T)0.5;
    return k;
}

// Coefficients a step kernel can read from device memory instead of its
// argument (swe_run): written on the device from the FP64 CFL step by the
// same make_coef, so they have the host's bits.  skip != 0 when the CFL pass
// found a non-positive depth; the step kernels then leave the state alone.
template <typename T>
struct DevCoef {
    Coef<T> k;
    int skip;
};

// Takes the device coefficients if kd is given; false when the step is to
// be skipped.  Every thread of a kernel calls it before any barrier.
template <typename T>
__device__ __forceinline__ bool take_dev_coef(const DevCoef<T> *kd, Coef<T> &k)
{
    if (!kd) return true;
    if (kd->skip) return false;
    k = kd->k;
    return true;
}

// A cell with its physical fluxes (Sec. 3 conservation laws):
//   F = (U, U^2/H + g H^2/2, U V/H),  G = (V, U V/H, V^2/H + g H^2/2).
// f3 doubles as G's second component (both are U V / H).
template <typename T>
struct CellQ {
    T h, u, v;
    T f2, f3, g3;
};

template <typename T>
__device__ __forceinline__ CellQ<T> make_cell(T h, T u, T v, T hg)
{
    CellQ<T> c;
    c.h = h;
    c.u = u;
    c.v = v;
    const T inv = rcp(h);
    const T p = mul_rn(mul_rn(hg, h), h);
    const T uu = mul_rn(u, inv);
    const T vv = mul_rn(v, inv);
    c.f2 = fma(u, uu, p);
    c.f3 = mul_rn(u, vv);
    c.g3 = fma(v, vv, p);
    return c;
}

// Mirror of a cell across an x-wall: U negated, H and V copied.
template <typename T>
__device__ __forceinline__ CellQ<T> mirror_x(const CellQ<T> &c)
{
    CellQ<T> m = c;
    m.u = -c.u;
    m.f3 = -c.f3;
    return m;
}

// Mirror of a cell across a y-wall: V negated, H and U copied.
template <typename T>
__device__ __forceinline__ CellQ<T> mirror_y(const CellQ<T> &c)
{
    CellQ<T> m = c;
    m.v = -c.v;
    m.f3 = -c.f3;
    return m;
}

template <typename T>
struct Flux3 {
    T a, b, c;
};

// Step 1 on an x-face between cells L (left) and R (right), then the
// x-flux F evaluated at the face state (step 2's input), both doubled (see
// Coef): the face state is 2 (0.5 (L + R) + (0.5 dt/dx) (F(L) - F(R))) and
// the result is 2 F of it.
template <typename T>
__device__ __forceinline__ Flux3<T> xface_flux(const CellQ<T> &L, const CellQ<T> &R, const Coef<T> &k)
{
    const T Hf = fma(k.lx, L.u - R.u, L.h + R.h);
    const T Uf = fma(k.lx, L.f2 - R.f2, L.u + R.u);
    const T Vf = fma(k.lx, L.f3 - R.f3, L.v + R.v);
    const T inv = rcp(Hf);
    const T uf = mul_rn(Uf, inv);
    Flux3<T> F;
    F.a = Uf;
    F.b = fma(Uf, uf, mul_rn(mul_rn(k.qg, Hf), Hf));
    F.c = mul_rn(Vf, uf);
    return F;
}

// Step 1 on a y-face between cells D (below) and U (above), then the
// y-flux G at the face state, both doubled as in xface_flux.
template <typename T>
__device__ __forceinline__ Flux3<T> yface_flux(const CellQ<T> &D, const CellQ<T> &U, const Coef<T> &k)
{
    const T Hf = fma(k.ly, D.v - U.v, D.h + U.h);
    const T Uf = fma(k.ly, D.f3 - U.f3, D.u + U.u);
    const T Vf = fma(k.ly, D.g3 - U.g3, D.v + U.v);
    const T inv = rcp(Hf);
    const T vf = mul_rn(Vf, inv);
    Flux3<T> G;
    G.a = Vf;
    G.b = mul_rn(Uf, vf);
    G.c = fma(Vf, vf, mul_rn(mul_rn(k.qg, Hf), Hf));
    return G;
}

// Step 2: conservative update of one cell from its four (doubled) face
// fluxes: u - (dt/dx)(F_r - F_l) - (dt/dy)(G_u - G_d).
template <typename T>
__device__ __forceinline__ void lw_update(T &h, T &u, T &v, const Flux3<T> &Fl, const Flux3<T> &Fr,
                                          const Flux3<T> &Gd, const Flux3<T> &Gu, const Coef<T> &k)
{
    h = fma(k.hy, Gd.a - Gu.a, fma(k.hx, Fl.a - Fr.a, h));
    u = fma(k.hy, Gd.b - Gu.b, fma(k.hx, Fl.b - Fr.b, u));
    v = fma(k.hy, Gd.c - Gu.c, fma(k.hx, Fl.c - Fr.c, v));
}

// ---------------------------------------------------------------------------
// The same arithmetic on two FP32 cells at once.  An F2 holds two floats in
// one 64-bit register pair; add/sub/mul/fma.rn.f32x2 perform on each lane
// exactly the IEEE operation the scalar functions above perform, and the
// reciprocal is taken per lane with the same instruction, so every lane of
// a paired result has the bits of the scalar computation, provided no packed
// product feeds a packed add or subtract (see mul2_nf).  Used by the tile
// routine for cells away from an x-wall.
// ---------------------------------------------------------------------------
struct F2 {
    unsigned long long v;
};

__device__ __forceinline__ F2 pack2(float lo, float hi)
{
    F2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpack2(F2 x, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x.v));
}
__device__ __forceinline__ float lo2(F2 x)
{
    float a, b;
    unpack2(x, a, b);
    return a;
}
__device__ __forceinline__ float hi2(F2 x)
{
    float a, b;
    unpack2(x, a, b);
    return b;
}
__device__ __forceinline__ F2 add2(F2 a, F2 b)
{
    F2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 sub2(F2 a, F2 b)
{
    F2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 mul2(F2 a, F2 b)
{
    F2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c)
{
    F2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}
// A product that a later add or subtract may not absorb.  Unlike the scalar
// mul.rn, a packed mul.rn.f32x2 whose result feeds an add/sub.rn.f32x2 is
// fused into one FMA by the compiler (measured on sm_103a, --fmad=false or
// not), which changes the rounding.  So the product is taken as the packed
// FMA a*b + nz with nz = (-0, -0).  RN(a*b + (-0)) = RN(a*b) for every a, b (a zero product keeps
// its sign: +0 + -0 = +0, -0 + -0 = -0), and an FMA is not absorbed into a
// later add.  nz must be a run-time value: given the constant -0 the
// compiler turns the FMA back into a multiply, and fuses that (measured).
__device__ __forceinline__ F2 mul2_nf(F2 a, F2 b, F2 nz)
{
    F2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(nz.v));
    return r;
}
__device__ __forceinline__ F2 rcp2(F2 x)
{
    float a, b;
    unpack2(x, a, b);
    return pack2(rcp(a), rcp(b));
}
__device__ __forceinline__ F2 neg2(F2 x)  // exact sign flip of both lanes
{
    F2 r;
    r.v = x.v ^ 0x8000000080000000ull;
    return r;
}

struct CellQ2 {
    F2 h, u, v;
    F2 f2, f3, g3;
};
struct Flux2 {
    F2 a, b, c;
};
// the coefficients broadcast to both lanes; nz = (-0, -0) for mul2_nf,
// formed at run time as -0 * g/2 (g > 0 is checked when a grid is created)
struct Coef2 {
    F2 hx, hy, lx, ly, hg, qg, nz;
};
__device__ __forceinline__ Coef2 coef2(const Coef<float> &k)
{
    const float z = __fmul_rn(-0.0f, k.hg);
    return {pack2(k.hx, k.hx), pack2(k.hy, k.hy), pack2(k.lx, k.lx), pack2(k.ly, k.ly), pack2(k.hg, k.hg),
            pack2(k.qg, k.qg), pack2(z, z)};
}

// make_cell on two cells
__device__ __forceinline__ CellQ2 make_cell2(F2 h, F2 u, F2 v, const Coef2 &k)
{
    CellQ2 c;
    c.h = h;
    c.u = u;
    c.v = v;
    const F2 inv = rcp2(h);
    const F2 p = mul2(mul2(k.hg, h), h);
    const F2 uu = mul2(u, inv);
    const F2 vv = mul2(v, inv);
    c.f2 = fma2(u, uu, p);
    c.f3 = mul2_nf(u, vv, k.nz);  // differenced by the face steps
    c.g3 = fma2(v, vv, p);
    return c;
}

__device__ __forceinline__ CellQ2 mirror_y2(const CellQ2 &c)
{
    CellQ2 m = c;
    m.v = neg2(c.v);
    m.f3 = neg2(c.f3);
    return m;
}

// two scalar cells as a pair, and back
__device__ __forceinline__ CellQ2 pair_cells(const CellQ<float> &a, const CellQ<float> &b)
{
    return {pack2(a.h, b.h), pack2(a.u, b.u), pack2(a.v, b.v), pack2(a.f2, b.f2), pack2(a.f3, b.f3),
            pack2(a.g3, b.g3)};
}
__device__ __forceinline__ CellQ<float> cell_lo(const CellQ2 &c)
{
    return {lo2(c.h), lo2(c.u), lo2(c.v), lo2(c.f2), lo2(c.f3), lo2(c.g3)};
}
__device__ __forceinline__ CellQ<float> cell_hi(const CellQ2 &c)
{
    return {hi2(c.h), hi2(c.u), hi2(c.v), hi2(c.f2), hi2(c.f3), hi2(c.g3)};
}

// xface_flux on two faces
__device__ __forceinline__ Flux2 xface_flux2(const CellQ2 &L, const CellQ2 &R, const Coef2 &k)
{
    const F2 Hf = fma2(k.lx, sub2(L.u, R.u), add2(L.h, R.h));
    const F2 Uf = fma2(k.lx, sub2(L.f2, R.f2), add2(L.u, R.u));
    const F2 Vf = fma2(k.lx, sub2(L.f3, R.f3), add2(L.v, R.v));
    const F2 inv = rcp2(Hf);
    const F2 uf = mul2(Uf, inv);
    Flux2 F;
    F.a = Uf;
    F.b = fma2(Uf, uf, mul2(mul2(k.qg, Hf), Hf));
    F.c = mul2_nf(Vf, uf, k.nz);  // differenced by the update
    return F;
}

// yface_flux on two faces
__device__ __forceinline__ Flux2 yface_flux2(const CellQ2 &D, const CellQ2 &U, const Coef2 &k)
{
    const F2 Hf = fma2(k.ly, sub2(D.v, U.v), add2(D.h, U.h));
    const F2 Uf = fma2(k.ly, sub2(D.f3, U.f3), add2(D.u, U.u));
    const F2 Vf = fma2(k.ly, sub2(D.g3, U.g3), add2(D.v, U.v));
    const F2 inv = rcp2(Hf);
    const F2 vf = mul2(Vf, inv);
    Flux2 G;
    G.a = Vf;
    G.b = mul2_nf(Uf, vf, k.nz);  // differenced by the update
    G.c = fma2(Vf, vf, mul2(mul2(k.qg, Hf), Hf));
    return G;
}

// lw_update on two cells
__device__ __forceinline__ void lw_update2(F2 &h, F2 &u, F2 &v, const Flux2 &Fl, const Flux2 &Fr, const Flux2 &Gd,
                                           const Flux2 &Gu, const Coef2 &k)
{
    h = fma2(k.hy, sub2(Gd.a, Gu.a), fma2(k.hx, sub2(Fl.a, Fr.a), h));
    u = fma2(k.hy, sub2(Gd.b, Gu.b), fma2(k.hx, sub2(Fl.b, Fr.b), u));
    v = fma2(k.hy, sub2(Gd.c, Gu.c), fma2(k.hx, sub2(Fl.c, Fr.c), v));
}

// (lo of a, lo of b) and (hi of a, hi of b) style regroupings of fluxes
__device__ __forceinline__ Flux2 flux_pair(float a0, float b0, float c0, float a1, float b1, float c1)
{
    return {pack2(a0, a1), pack2(b0, b1), pack2(c0, c1)};
}

}  // namespace swe
