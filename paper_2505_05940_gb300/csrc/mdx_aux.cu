// Small element-wise kernels around the time loops: state conversion between
// the FP64 interface and the compensated FP32 device form, adjoint
// initialisation, and the FP64 gradient epilogue (chain rule from the
// difference-form sums to d omega^2, d gamma, d b, d c; Sec. 3.2, Eq. 21-23).
#include <cuda_runtime.h>

#include "mdx_common.cuh"
#include "mdx_scheme.cuh"

namespace mdx {

__global__ void init_state_kernel(const AuxInit a) {
    const long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (m >= a.total_modes) return;
    const double q0 = a.q0 ? a.q0[m] : 0.0;
    const double qm1 = a.qm1 ? a.qm1[m] : 0.0;
    const float hi = (float)q0;
    const double v = q0 - qm1;
    const float vhi = (float)v;
    a.state[m] = hi;
    a.state[a.total_modes + m] = (float)(q0 - (double)hi);
    a.state[2 * a.total_modes + m] = vhi;
    a.state[3 * a.total_modes + m] = (float)(v - (double)vhi);
}

cudaError_t launch_init_state(const AuxInit &a, cudaStream_t s) {
    if (a.total_modes == 0) return cudaSuccess;
    const int t = 256;
    init_state_kernel<<<(unsigned)((a.total_modes + t - 1) / t), t, 0, s>>>(a);
    return cudaGetLastError();
}

__global__ void finalize_state_kernel(const float *st, long long TM, double *q_end,
                                      double *qm1_end) {
    const long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (m >= TM) return;
    const double q = (double)st[m] + (double)st[TM + m];
    if (q_end) q_end[m] = q;
    if (qm1_end) qm1_end[m] = q - ((double)st[2 * TM + m] + (double)st[3 * TM + m]);
}

cudaError_t launch_finalize_state(const float *state, long long TM, double *q_end,
                                  double *qm1_end, cudaStream_t s) {
    if (TM == 0 || (!q_end && !qm1_end)) return cudaSuccess;
    const int t = 256;
    finalize_state_kernel<<<(unsigned)((TM + t - 1) / t), t, 0, s>>>(state, TM, q_end, qm1_end);
    return cudaGetLastError();
}

__global__ void init_adjoint_kernel(const InstDesc *inst, const float *c, const float *ybar,
                                    int steps, float *adj, long long TM) {
    const int i = blockIdx.x;
    const InstDesc d = inst[i];
    const float yl = (steps > 0) ? ybar[(long long)i * steps + steps - 1] : 0.f;
    for (int s = threadIdx.x; s < d.N; s += blockDim.x) {
        const long long m = d.mode_off + s;
        const float a = c[m] * yl;
        adj[m] = a;
        adj[TM + m] = 0.f;
        adj[2 * TM + m] = a;
    }
}

cudaError_t launch_init_adjoint(const InstDesc *inst, int n_inst, const float *c,
                                const float *ybar, int steps, float *adj, long long TM,
                                int max_n, cudaStream_t s) {
    if (n_inst == 0) return cudaSuccess;
    (void)max_n;
    init_adjoint_kernel<<<n_inst, 256, 0, s>>>(inst, c, ybar, steps, adj, TM);
    return cudaGetLastError();
}

__device__ __forceinline__ double kval(const float *p) {
    // Kahan pair (sum, compensation): value = sum - compensation
    return (double)p[0] - (double)p[1];
}

__global__ void grad_epilogue_kernel(const GradEpilogue g) {
    const int i = blockIdx.x;
    const InstDesc d = g.inst[i];
    const long long TM = g.total_modes;
    for (int s = threadIdx.x; s < d.N; s += blockDim.x) {
        const long long m = d.mode_off + s;
        const double T = g.dt[m], w2 = g.omega2[m], gm = g.gamma[m];
        const SchemeCoef k = scheme_coef(g.scheme, w2, gm, T);
        auto acc = [&](int idx) {
            return (double)g.gacc[(long long)(2 * idx) * TM + m] -
                   (double)g.gacc[(long long)(2 * idx + 1) * TM + m];
        };
        const double A = acc(GA_A), V = acc(GA_V), F = acc(GA_F), E = acc(GA_E), C = acc(GA_C);
        double dw2, dgm;
        scheme_grads(g.scheme, w2, gm, T, A, V, F, &dw2, &dgm);
        if (g.d_omega2) g.d_omega2[m] = dw2;
        if (g.d_gamma) g.d_gamma[m] = dgm;
        if (g.d_b) g.d_b[m] = k.r * E;
        if (g.d_c) g.d_c[m] = C;
        const double a0 = (double)g.adj[m] + (double)g.adj[TM + m];
        const double mu0 = (double)g.adj[2 * TM + m];
        if (g.d_q0) g.d_q0[m] = a0;
        // q^{-1} enters through v^0 = q^0 - q^{-1}, carried with factor 1 - eps
        if (g.d_qm1) g.d_qm1[m] = -(1.0 - k.eps) * (a0 - mu0);
    }
    if (threadIdx.x == 0) {
        if (g.d_tau) g.d_tau[i] = (d.kind == 0 && g.tacc) ? kval(g.tacc + 2 * i) : 0.0;
        double dir = 0.0;
        for (int k = 0; k < d.M; ++k) {
            if (g.d_kappa) g.d_kappa[d.k_off + g.kperm[d.k_off + k]] = kval(g.kacc + 2 * (d.k_off + k));
            if (d.has_dir)
                for (int a = 0; a < 4; ++a) dir += g.dir_acc[(d.k_off + k) * 4 + a];
        }
        if (g.d_dir) g.d_dir[i] = dir;
    }
}

cudaError_t launch_grad_epilogue(const GradEpilogue &g, int max_n, cudaStream_t s) {
    if (g.n_inst == 0) return cudaSuccess;
    (void)max_n;
    grad_epilogue_kernel<<<g.n_inst, 256, 0, s>>>(g);
    return cudaGetLastError();
}

}  // namespace mdx
