// swe_internal.h -- library-internal declarations shared by the .cu files
// of the shallow-water library (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/swe.h"

namespace swe {

// Device planes: ny rows of ``pitch`` elements, interior cell (i, j) at
// j*pitch + i.  The pitch is a multiple of 128 bytes so that every row
// starts on a 128-byte boundary (TMA strides, 16-byte vector access).
inline long long plane_pitch(int nx, size_t esize)
{
    const long long per = 128 / (long long)esize;
    return ((long long)nx + per - 1) / per * per;
}

// Step-kernel launch geometry of one variant.
struct StepGeom {
    int tile_x, tile_y;  // output cells per CTA
    int threads;         // threads per CTA
    size_t smem;         // dynamic shared memory, bytes
};

// Launchers implemented in swe_step.cu.  ``in``/``out`` each point to three
// planes (H, U, V) of ``plane`` elements.  All return cudaError_t of the
// launch.  ``kd``, if given, is a device DevCoef<T> (swe_device.cuh) whose
// coefficients replace those made from (dx, dy, dt, g).
cudaError_t launch_naive(int dtype, const void *in, void *out, size_t plane, int nx, int ny, long long pitch,
                         double dx, double dy, double dt, double g, cudaStream_t s, const void *kd = nullptr);
cudaError_t launch_tiled(int dtype, const CUtensorMap *maps_in, void *out, size_t plane, int nx, int ny,
                         long long pitch, double dx, double dy, double dt, double g, int *err, cudaStream_t s,
                         const void *kd = nullptr);
cudaError_t launch_tb2(int dtype, int variant, const CUtensorMap *maps_in, void *out, size_t plane, int nx, int ny,
                       long long pitch, double dx, double dy, double dt, double g, int *err, cudaStream_t s,
                       const void *kd = nullptr);
void tb2_box(int dtype, int variant, int *bw, int *bh);  // TMA box of two-step kernel shape ``variant``
// Packed-state kernel (swe_packed.cu): state as (h, hu, hv, 0) float4 cells,
// ppitch cells per row.  launch_pack copies the planes into the packed
// buffer (unpack = false) or back (unpack = true).
cudaError_t launch_packed(const CUtensorMap *map, void *out, int nx, int ny, long long ppitch, double dx, double dy,
                          double dt, double g, int *err, cudaStream_t s, const void *kd = nullptr);
cudaError_t launch_pack(const void *h, const void *u, const void *v, long long pitch, void *out, long long ppitch,
                        int nx, int ny, bool unpack, cudaStream_t s);
void packed_box(int *bw, int *bh);  // TMA box (cells) of the packed kernel
StepGeom tiled_geom(int dtype);
void tiled_box(int dtype, int *bw, int *bh);  // TMA box the tiled kernel loads

// Reductions implemented in swe_reduce.cu.  ``scratch`` holds at least
// reduce_scratch_doubles() doubles; results land in out_dev[0..1]
// (value, bad-cell count).
size_t reduce_scratch_doubles();
size_t reduce_scratch_doubles_many(int n, int B);

// One grid of a batched reduction (device array of n of these).  dx, dy are
// used by the CFL step and as the cell area of the mass.
struct RedGrid {
    const void *h, *u, *v;
    long long pitch;
    int nx, ny;
    double dx, dy;
};
// Batched FP32 reductions over n grids with B blocks each; out_dev[2g] gets
// grid g's mass or dt, out_dev[2g+1] its bad-cell count (CFL only).
cudaError_t launch_mass_many(const RedGrid *grids_dev, int n, int B, double *scratch, double *out_dev,
                             cudaStream_t s);
cudaError_t launch_cfl_many(const RedGrid *grids_dev, int n, int B, double g, double cfl, double *scratch,
                            double *out_dev, cudaStream_t s);
cudaError_t launch_mass(int dtype, const void *H, int nx, int ny, long long pitch, double dxdy, double *scratch,
                        double *out_dev, cudaStream_t s);
cudaError_t launch_cfl(int dtype, const void *H, const void *U, const void *V, int nx, int ny, long long pitch,
                       double dx, double dy, double g, double cfl, double *scratch, double *out_dev,
                       cudaStream_t s);
// The step coefficients of a CFL result res_dev = (dt, bad-cell count) into
// the device DevCoef<T> at kd (T the context's dtype); kd->skip when bad.
cudaError_t launch_coef_from_cfl(int dtype, const double *res_dev, double dx, double dy, double g, void *kd,
                                 cudaStream_t s);

// TMA descriptor encoding through the driver entry point (no -lcuda link).
// Encodes a 2D map over an nx x ny plane with the given box; returns false
// if the driver entry point is unavailable or the encode fails.
bool encode_plane_map(CUtensorMap *map, int dtype, const void *base, int nx, int ny, long long pitch, int box_x,
                      int box_y);
// 3D map {4 components, nx, ny} over packed FP32 cells, ppitch cells per row.
bool encode_packed_map(CUtensorMap *map, const void *base, int nx, int ny, long long ppitch, int box_x, int box_y);

}  // namespace swe
