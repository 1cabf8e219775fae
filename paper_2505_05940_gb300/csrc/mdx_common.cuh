// Small device helpers shared by the kernels of libmdx.
#pragma once

#include <cstdint>

#include "mdx_internal.h"

namespace mdx {

// Compensated accumulation (Knuth two-sum): (hi, lo) += x exactly up to the
// rounding of lo.  Used for the modal state q and the adjoint a, whose
// per-step increments are orders of magnitude below their value.
__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float x) {
    float s = hi + x;
    float bb = s - hi;
    float err = (hi - (s - bb)) + (x - bb);
    float l = lo + err;
    float h = s + l;
    lo = l - (h - s);
    hi = h;
}

// Kahan summation for long reductions over time (gradient sums).
__device__ __forceinline__ void kahan_add(float &sum, float &comp, float x) {
    float y = x - comp;
    float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One Stormer-Verlet step in difference form for one mode (see mdx_internal.h):
// d = r F - eps v - r omega^2 q, v += d, q += v, with q, v and r omega^2 as
// FP32 pairs (hi + lo).
__device__ __forceinline__ void sv_step(float &qhi, float &qlo, float &vhi, float &vlo, float eps,
                                        float rw2, float rw2lo, float r, float F) {
    const float rest = fmaf(rw2, qhi, fmaf(rw2lo, qhi, rw2 * qlo));
    const float d = fmaf(r, F, fmaf(-eps, vhi, -rest));
    two_sum_add(vhi, vlo, d);
    // q += (vhi + vlo)
    float s = qhi + vhi;
    float bb = s - qhi;
    float err = (qhi - (s - bb)) + (vhi - bb);
    float l = qlo + err + vlo;
    float h = s + l;
    qlo = l - (h - s);
    qhi = h;
}

// One adjoint step in the same difference form:
//   mu^n = (1 - eps) mu^{n+1} - r omega^2 a^{n+1} - (J w) + c ybar^{n-1},  a^n = a^{n+1} + mu^n
__device__ __forceinline__ void adj_step(float &ahi, float &alo, float &mu, float eps, float rw2,
                                         float Jw, float pick) {
    float t = fmaf(-eps, mu, mu);
    t = fmaf(-rw2, ahi, t);
    t = t - Jw;
    t = t + pick;
    mu = t;
    two_sum_add(ahi, alo, mu);
}

__device__ __forceinline__ void set_status(int *status, int inst, int code) {
    if (status) atomicCAS(status + inst, 0, code);
}

}  // namespace mdx
