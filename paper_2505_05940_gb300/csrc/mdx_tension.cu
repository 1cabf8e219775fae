// Strings (Kirchhoff-Carrier) and membranes (Berger): one warp per instance.
//
// Per step (Sec. 3.2, Eq. 20 in difference form; Sec. 3.1, Eq. 8):
//   S       = sum_nu lambda_nu q_nu^2                      (warp reduction)
//   fnl_mu  = tau' lambda_mu q_mu S
//   v, q    <- Stormer-Verlet difference-form update
//   y^n     = sum_mu c_mu q^{n+1}_mu                       (warp reduction)
// Lane l holds modes l, l+32, ...; the whole time loop runs inside the kernel
// with the state in registers.  The same kernel re-runs a segment from a
// checkpoint (storing every state) and sweeps a stored segment backwards
// (adjoint recursion, J symmetric because fnl = grad V, V = tau'/4 S^2).
#include <cuda_runtime.h>

#include "../../include/mdx.h"
#include "mdx_common.cuh"

namespace mdx {

template <int J>
__global__ void __launch_bounds__(32 * kTensionWarpsPerBlock)
tension_kernel(const TensionParams P) {
    const int lane = threadIdx.x & 31;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= P.n_list) return;
    const int inst = P.list[w];
    const InstDesc d = P.inst[inst];
    const int N = d.N;
    const long long mo = d.mode_off;
    const long long TM = P.total_modes;
    const float taup = d.taup;

    float eps[J], rw2[J], rw2l[J], r[J], b[J], c[J], clo[J], lam[J];
    float x0[J], x1[J], x2[J], x3[J];   // forward: q_hi, q_lo, v_hi, v_lo ; reverse: a_hi, a_lo, mu
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int m = lane + 32 * j;
        const bool ok = m < N;
        eps[j] = ok ? P.coef.eps[mo + m] : 0.f;
        rw2[j] = ok ? P.coef.rw2[mo + m] : 0.f;
        rw2l[j] = ok ? P.coef.rw2lo[mo + m] : 0.f;
        r[j] = ok ? P.coef.r[mo + m] : 0.f;
        b[j] = ok ? P.coef.b[mo + m] : 0.f;
        c[j] = ok ? P.coef.c[mo + m] : 0.f;
        clo[j] = ok ? P.coef.clo[mo + m] : 0.f;
        lam[j] = ok ? P.coef.lam[mo + m] : 0.f;
    }
    const float *exc = P.exc ? P.exc + (long long)inst * P.total_steps : nullptr;

    if (P.mode != MODE_REVERSE) {
        // ---------------------------------------------------------- forward / recompute
        const float *src = P.state_io;
        if (P.mode == MODE_RECOMPUTE) src = P.ckpt + (long long)(P.n_begin / P.ckpt_K) * kStateArrays * TM;
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int m = lane + 32 * j;
            const bool ok = m < N;
            x0[j] = ok ? src[mo + m] : 0.f;
            x1[j] = ok ? src[TM + mo + m] : 0.f;
            x2[j] = ok ? src[2 * TM + mo + m] : 0.f;
            x3[j] = ok ? src[3 * TM + mo + m] : 0.f;
        }
        float S = 0.f;
#pragma unroll
        for (int j = 0; j < J; ++j) S = fmaf(lam[j] * x0[j], x0[j], S);
        S = warp_sum(S);
        float *aud = P.audio ? P.audio + (long long)inst * P.total_steps : nullptr;
        float ybuf = 0.f, ebuf = 0.f;
        bool bad = false;
        for (int it = 0; it < P.steps; ++it) {
            const int n = P.n_begin + it;
            if ((it & 31) == 0) {
                const int nn = n + lane;
                ebuf = (exc && nn < P.total_steps) ? exc[nn] : 0.f;
            }
            const float e = __shfl_sync(0xffffffffu, ebuf, it & 31);
            if (P.mode == MODE_FORWARD && P.ckpt && (n % P.ckpt_K) == 0) {
                float *ck = P.ckpt + (long long)(n / P.ckpt_K) * kStateArrays * TM;
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    const int m = lane + 32 * j;
                    if (m < N) {
                        ck[mo + m] = x0[j];
                        ck[TM + mo + m] = x1[j];
                        ck[2 * TM + mo + m] = x2[j];
                        ck[3 * TM + mo + m] = x3[j];
                    }
                }
            }
            if (P.mode == MODE_RECOMPUTE) {
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    const int m = lane + 32 * j;
                    if (m < N) {
                        P.seg_q[(long long)it * TM + mo + m] = x0[j];
                        P.seg_v[(long long)it * TM + mo + m] = x2[j];
                    }
                }
            }
            float ys = 0.f, ye = 0.f, Sp = 0.f;
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const float f = taup * lam[j] * x0[j] * S;
                sv_step(x0[j], x1[j], x2[j], x3[j], eps[j], rw2[j], rw2l[j], r[j], fmaf(b[j], e, -f));
                pickup_add(ys, ye, c[j], clo[j], x0[j], x1[j]);
                Sp = fmaf(lam[j] * x0[j], x0[j], Sp);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float s2 = __shfl_xor_sync(0xffffffffu, ys, o);
                const float e2 = __shfl_xor_sync(0xffffffffu, ye, o);
                pickup_merge(ys, ye, s2, e2);
                Sp += __shfl_xor_sync(0xffffffffu, Sp, o);
            }
            const float yp = ys + ye;
            S = Sp;
            if (lane == (it & 31)) ybuf = yp;
            if (!isfinite(yp)) bad = true;
            if (aud && (((it & 31) == 31) || it == P.steps - 1)) {
                const int base = n - (it & 31);
                if (lane <= (it & 31)) aud[base + lane] = ybuf;
            }
        }
        if (P.mode == MODE_RECOMPUTE) {
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const int m = lane + 32 * j;
                if (m < N) {
                    P.seg_q[(long long)P.steps * TM + mo + m] = x0[j];
                    P.seg_v[(long long)P.steps * TM + mo + m] = x2[j];
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const int m = lane + 32 * j;
                if (m < N) {
                    P.state_io[mo + m] = x0[j];
                    P.state_io[TM + mo + m] = x1[j];
                    P.state_io[2 * TM + mo + m] = x2[j];
                    P.state_io[3 * TM + mo + m] = x3[j];
                }
            }
        }
        if (bad && lane == 0) set_status(P.status, inst, MDX_ERR_NONFINITE);
        return;
    }

    // ------------------------------------------------------------------ reverse sweep
    // seg_q[t], seg_v[t] hold q^{n0+t}, v^{n0+t} for t = 0..steps.
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int m = lane + 32 * j;
        const bool ok = m < N;
        x0[j] = ok ? P.adj[mo + m] : 0.f;
        x1[j] = ok ? P.adj[TM + mo + m] : 0.f;
        x2[j] = ok ? P.adj[2 * TM + mo + m] : 0.f;
    }
    float gs[GA_N][J], gc[GA_N][J];
#pragma unroll
    for (int g = 0; g < GA_N; ++g)
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int m = lane + 32 * j;
            const bool ok = m < N;
            gs[g][j] = ok ? P.gacc[(long long)(2 * g) * TM + mo + m] : 0.f;
            gc[g][j] = ok ? P.gacc[(long long)(2 * g + 1) * TM + mo + m] : 0.f;
        }
    float ts = 0.f, tc = 0.f;
    if (lane == 0) { ts = P.tacc[2 * inst]; tc = P.tacc[2 * inst + 1]; }
    const float *yb = P.ybar + (long long)inst * P.total_steps;
    bool bad = false;
    for (int it = P.steps - 1; it >= 0; --it) {
        const int n = P.n_begin + it;
        const float e = exc ? exc[n] : 0.f;
        const float ybn = yb[n];
        const float ybm = (n >= 1) ? yb[n - 1] : 0.f;
        float q[J], v[J], q1[J], wv[J];
        float S = 0.f, Pq = 0.f;
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int m = lane + 32 * j;
            const bool ok = m < N;
            q[j] = ok ? P.seg_q[(long long)it * TM + mo + m] : 0.f;
            v[j] = ok ? P.seg_v[(long long)it * TM + mo + m] : 0.f;
            q1[j] = ok ? P.seg_q[(long long)(it + 1) * TM + mo + m] : 0.f;
            wv[j] = r[j] * x0[j];
            S = fmaf(lam[j] * q[j], q[j], S);
            Pq = fmaf(lam[j] * q[j], wv[j], Pq);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            S += __shfl_xor_sync(0xffffffffu, S, o);
            Pq += __shfl_xor_sync(0xffffffffu, Pq, o);
        }
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const float a = x0[j];
            const float f = taup * lam[j] * q[j] * S;
            const float Jw = taup * lam[j] * fmaf(S, wv[j], 2.f * q[j] * Pq);
            kahan_add(gs[GA_A][j], gc[GA_A][j], a * q[j]);
            kahan_add(gs[GA_V][j], gc[GA_V][j], a * v[j]);
            kahan_add(gs[GA_F][j], gc[GA_F][j], a * fmaf(b[j], e, -f));
            kahan_add(gs[GA_E][j], gc[GA_E][j], a * e);
            kahan_add(gs[GA_C][j], gc[GA_C][j], ybn * q1[j]);
            adj_step(x0[j], x1[j], x2[j], eps[j], rw2[j], Jw, c[j] * ybm);
        }
        if (lane == 0) kahan_add(ts, tc, -S * Pq);
        if (!isfinite(x0[0])) bad = true;
    }
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int m = lane + 32 * j;
        if (m < N) {
            P.adj[mo + m] = x0[j];
            P.adj[TM + mo + m] = x1[j];
            P.adj[2 * TM + mo + m] = x2[j];
#pragma unroll
            for (int g = 0; g < GA_N; ++g) {
                P.gacc[(long long)(2 * g) * TM + mo + m] = gs[g][j];
                P.gacc[(long long)(2 * g + 1) * TM + mo + m] = gc[g][j];
            }
        }
    }
    if (lane == 0) { P.tacc[2 * inst] = ts; P.tacc[2 * inst + 1] = tc; }
    if (bad && lane == 0) set_status(P.status, inst, MDX_ERR_NONFINITE);
}

// J (modes per lane) buckets: 1, 2, 4, 8, 16, 32.
static int tension_bucket(int N) {
    int j = (N + 31) / 32;
    int b = 1;
    while (b < j) b <<= 1;
    return b;
}

template <int J>
static cudaError_t launch_j(const TensionParams &p, cudaStream_t s) {
    const int threads = 32 * kTensionWarpsPerBlock;
    const int blocks = (p.n_list + kTensionWarpsPerBlock - 1) / kTensionWarpsPerBlock;
    if (blocks == 0) return cudaSuccess;
    tension_kernel<J><<<blocks, threads, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_tension(const TensionParams &p, int max_n, cudaStream_t s) {
    switch (tension_bucket(max_n)) {
        case 1: return launch_j<1>(p, s);
        case 2: return launch_j<2>(p, s);
        case 4: return launch_j<4>(p, s);
        case 8: return launch_j<8>(p, s);
        case 16: return launch_j<16>(p, s);
        default: return launch_j<32>(p, s);
    }
}

}  // namespace mdx
