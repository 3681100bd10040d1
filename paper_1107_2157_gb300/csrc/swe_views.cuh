// swe_views.cuh -- library-internal views of the batch and network objects,
// for kernels that need both (the fused learned coarse step).
#pragma once

#include <cuda_bf16.h>

#include "swe_device.cuh"

namespace swe {

// One instance of a batch as the device sees it.
struct BatchInst {
    float *buf[2];       // three planes (H, U, V) per buffer
    long long plane;     // elements per plane
    long long pitch;     // elements per row
    int nx, ny;
    Coef<float> k;
};

struct BatchView {
    int n;                     // instances
    int cur;                   // buffer parity holding the current state
    int sms;                   // SMs of the batch's device
    const BatchInst *d_inst;   // device array of n
    const BatchInst *h_inst;   // host copy
    int *d_flags;              // per-instance SWE_FLAG_* words
    int *d_err;                // device error word
};

// Fills *v; false for a null batch.
bool batch_view(swe_batch *b, BatchView *v);
// Records that a launch advanced every instance by n_steps (buffer parity).
void batch_advance(swe_batch *b, int n_steps);

struct NetView {
    const __nv_bfloat16 *w1, *w2, *w3;  // B-operand images of the three forward convolutions
    const float *bias;                  // b1 (32) | b2 (32) | b3 padded to 16
    float norm[5];                      // h0, sh, su, oh, ou
    int *d_err;
};

bool net_view(swe_net *t, NetView *v);

}  // namespace swe
