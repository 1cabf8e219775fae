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

// Compensated pickup term: (s, e) += (c + c_lo) (q_hi + q_lo).  The product c q_hi is
// split exactly (its rounding error from an fma), the sum is a two-sum, and
// the small terms (product error, c q_lo, sum error) gather in e.  The pickup
// sum y = sum_mu c_mu q_mu can cancel strongly (a pickup near nodal lines of
// the dominant modes), so plain FP32 summation of the rounded q_hi would lose
// digits that the compensated state still holds.
__device__ __forceinline__ void pickup_add(float &s, float &e, float c, float clo, float qhi,
                                           float qlo) {
    const float p = c * qhi;
    const float pe = fmaf(c, qhi, -p);
    const float t = s + p;
    const float bb = t - s;
    const float err = (s - (t - bb)) + (p - bb);
    s = t;
    e += err + fmaf(c, qlo, fmaf(clo, qhi, pe));
}

// (s, e) += (s2, e2) with the sum's rounding error folded into e.
__device__ __forceinline__ void pickup_merge(float &s, float &e, float s2, float e2) {
    const float t = s + s2;
    const float bb = t - s;
    const float err = (s - (t - bb)) + (s2 - bb);
    s = t;
    e += e2 + err;
}

// Compensated warp reduction of (s, e); every lane receives the total s + e.
__device__ __forceinline__ float warp_pickup_sum(float s, float e) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
        const float e2 = __shfl_xor_sync(0xffffffffu, e, o);
        pickup_merge(s, e, s2, e2);
    }
    return s + e;
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
