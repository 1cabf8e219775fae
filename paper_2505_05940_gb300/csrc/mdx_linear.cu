// Linear modal response, parallel in time (Sec. 4.3.2).
//
// Without the nonlinear terms every mode obeys its own linear recursion
// (Sec. 3.2; Eq. 20-23 for Stormer-Verlet, Eq. 15-19 for the impulse-invariant
// scheme),
//     q^{n+1} = g q^n + p q^{n-1} + r b e^n,
// i.e. X^{n+1} = A X^n + (r b e^n, 0) with X^n = (q^n, q^{n-1}) and the
// companion matrix A = [[g, p], [1, 0]], whose eigenvalues are the discrete
// poles of the mode.  The paper evaluates such responses by repeated
// multiplication with the poles organised as a prefix scan over time; here
// the scan is blocked in time:
//   1. every chunk of L steps runs its inputs from a zero state (all chunks
//      and modes in parallel) and keeps only its final state E_j;
//   2. per mode, the chunk boundary states follow sequentially,
//      S_j = A^L S_{j-1} + E_j (A^L by repeated squaring), S_{-1} = X^0;
//   3. every chunk reruns from its true incoming state S_{j-1} and writes the
//      pickup y^n = sum_mu c_mu q_mu^{n+1} (warp reduction over modes).
// The arithmetic is FP64 (the linear solver is a reference-grade generator,
// not the hot path); audio is rounded to FP32 at the end.
#include <cuda_runtime.h>

#include "../../include/mdx.h"
#include "mdx_common.cuh"
#include "mdx_scheme.cuh"

namespace mdx {

namespace {

constexpr int kLinThreads = 256;

struct LinCoef {
    double g, p, rb, c;
};

__device__ __forceinline__ LinCoef lin_coef(const LinearParams &P, const InstDesc &d, int m) {
    const long long gm = d.mode_off + m;
    const SchemeCoef k = scheme_coef(P.scheme, P.omega2[gm], P.gamma[gm], P.dt[gm]);
    LinCoef o;
    o.p = k.eps - 1.0;             // eps = 1 + p
    o.g = 2.0 - k.eps - k.rho;     // rho = 1 - g - p
    o.rb = k.r * P.b[gm];
    o.c = P.c[gm];
    return o;
}

__global__ void __launch_bounds__(kLinThreads) lin_local_kernel(const LinearParams P) {
    const int j = blockIdx.x, inst = blockIdx.y;
    if (j >= P.n_chunks - 1) return;        // the last chunk's end state is not needed
    const InstDesc d = P.inst[inst];
    const int n0 = j * P.L, n1 = min(P.steps, n0 + P.L);
    const float *e = P.exc ? P.exc + (long long)inst * P.total_steps : nullptr;
    for (int m = threadIdx.x; m < d.N; m += blockDim.x) {
        const LinCoef k = lin_coef(P, d, m);
        double x0 = 0.0, x1 = 0.0;
        for (int n = n0; n < n1; ++n) {
            const double u = e ? k.rb * (double)e[n] : 0.0;
            const double qn = fma(k.g, x0, fma(k.p, x1, u));
            x1 = x0;
            x0 = qn;
        }
        double *E = P.E + ((long long)j * P.total_modes + d.mode_off + m) * 2;
        E[0] = x0;
        E[1] = x1;
    }
}

__global__ void lin_carry_kernel(const LinearParams P) {
    const long long gmode = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gmode >= P.total_modes) return;
    const int inst = P.mode_inst[gmode];
    const InstDesc d = P.inst[inst];
    const int m = (int)(gmode - d.mode_off);
    const LinCoef k = lin_coef(P, d, m);
    // A^L by repeated squaring
    double a00 = k.g, a01 = k.p, a10 = 1.0, a11 = 0.0;
    double r00 = 1.0, r01 = 0.0, r10 = 0.0, r11 = 1.0;
    for (int L = P.L; L > 0; L >>= 1) {
        if (L & 1) {
            const double t00 = r00 * a00 + r01 * a10, t01 = r00 * a01 + r01 * a11;
            const double t10 = r10 * a00 + r11 * a10, t11 = r10 * a01 + r11 * a11;
            r00 = t00, r01 = t01, r10 = t10, r11 = t11;
        }
        const double s00 = a00 * a00 + a01 * a10, s01 = a00 * a01 + a01 * a11;
        const double s10 = a10 * a00 + a11 * a10, s11 = a10 * a01 + a11 * a11;
        a00 = s00, a01 = s01, a10 = s10, a11 = s11;
    }
    double s0 = P.q0 ? P.q0[gmode] : 0.0, s1 = P.qm1 ? P.qm1[gmode] : 0.0;
    double *S = P.S + gmode * 2;
    S[0] = s0;
    S[1] = s1;
    for (int j = 0; j < P.n_chunks - 1; ++j) {
        const double *E = P.E + ((long long)j * P.total_modes + gmode) * 2;
        const double t0 = fma(r00, s0, fma(r01, s1, E[0]));
        const double t1 = fma(r10, s0, fma(r11, s1, E[1]));
        s0 = t0;
        s1 = t1;
        double *Sj = P.S + ((long long)(j + 1) * P.total_modes + gmode) * 2;
        Sj[0] = s0;
        Sj[1] = s1;
    }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kLinThreads) lin_out_kernel(const LinearParams P) {
    __shared__ double ypart[kLinThreads / 32][kLinChunk];
    const int j = blockIdx.x, inst = blockIdx.y;
    const InstDesc d = P.inst[inst];
    const int n0 = j * P.L, n1 = min(P.steps, n0 + P.L);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float *e = P.exc ? P.exc + (long long)inst * P.total_steps : nullptr;
    for (int k = threadIdx.x; k < (kLinThreads / 32) * kLinChunk; k += blockDim.x)
        (&ypart[0][0])[k] = 0.0;
    __syncthreads();
    // every warp walks whole rounds of 32 modes, so the shuffles stay converged
    for (int m0 = warp * 32; m0 < d.N; m0 += kLinThreads) {
        const int m = m0 + lane;
        const bool on = m < d.N;
        LinCoef k{0.0, 0.0, 0.0, 0.0};
        double x0 = 0.0, x1 = 0.0;
        if (on) {
            k = lin_coef(P, d, m);
            const double *S = P.S + ((long long)j * P.total_modes + d.mode_off + m) * 2;
            x0 = S[0];
            x1 = S[1];
        }
        for (int n = n0; n < n1; ++n) {
            const double u = e ? k.rb * (double)e[n] : 0.0;
            const double qn = fma(k.g, x0, fma(k.p, x1, u));
            x1 = x0;
            x0 = qn;
            const double y = warp_sum_d(on ? k.c * qn : 0.0);
            if (lane == 0) ypart[warp][n - n0] += y;
        }
        if (on && j == P.n_chunks - 1) {
            if (P.q_end) P.q_end[d.mode_off + m] = x0;
            if (P.qm1_end) P.qm1_end[d.mode_off + m] = x1;
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n1 - n0; t += blockDim.x) {
        double y = 0.0;
#pragma unroll
        for (int w = 0; w < kLinThreads / 32; ++w) y += ypart[w][t];
        if (P.audio) P.audio[(long long)inst * P.total_steps + n0 + t] = (float)y;
        if (!isfinite(y)) set_status(P.status, inst, MDX_ERR_NONFINITE);
    }
}

}  // namespace

cudaError_t launch_linear(const LinearParams &P, cudaStream_t s) {
    if (P.steps <= 0 || P.n_inst <= 0) return cudaSuccess;
    const dim3 grid(P.n_chunks, P.n_inst);
    lin_local_kernel<<<grid, kLinThreads, 0, s>>>(P);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int cb = 128;
    lin_carry_kernel<<<(int)((P.total_modes + cb - 1) / cb), cb, 0, s>>>(P);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    lin_out_kernel<<<grid, kLinThreads, 0, s>>>(P);
    return cudaGetLastError();
}

}  // namespace mdx
