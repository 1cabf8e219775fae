// Learned-proposal network: a small MLP trained on simulator output.
//
// Layers d0 -> d1 -> ... -> dL with ReLU between hidden layers and a linear
// output.  Weights are BF16 (an FP32 master copy is kept for the optimiser);
// every product accumulates in FP32 on the tensor cores (mma.sync m16n8k16,
// BF16 x BF16 -> FP32).  Activations are stored in BF16 between layers.
//
// Kernels: one generic strided GEMM with fused epilogues (bias, ReLU, ReLU
// mask of the backward pass, FP32 or BF16 output), a column-sum for bias
// gradients, and the Adam update.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/mdx.h"
#include "mdx_internal.h"

namespace mdx {

namespace {

constexpr int BM = 64, BN = 64, BK = 32;
constexpr int kGemmThreads = 128;   // 4 warps, each a 32 x 32 tile

enum : int { EPI_NONE = 0, EPI_BIAS = 1, EPI_RELU = 2, EPI_MASK = 4, EPI_BF16 = 8, EPI_ACCUM = 16 };

struct GemmArgs {
    int M, N, K;
    const uint16_t *A;             // element (m, k) at A[m * sAm + k * sAk]  (BF16 bits)
    long long sAm, sAk;
    const uint16_t *B;             // element (k, n) at B[k * sBk + n * sBn]
    long long sBk, sBn;
    void *C;                       // element (m, n) at C[m * ldc + n] (FP32 or BF16)
    long long ldc;
    const float *bias;             // [N]
    const uint16_t *mask;          // BF16 [M][ldm]: keep where mask > 0 (ReLU derivative)
    long long ldm;
    int epi;
};

__device__ __forceinline__ uint32_t pack2(uint16_t lo, uint16_t hi) {
    return (uint32_t)lo | ((uint32_t)hi << 16);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint16_t f2bf(float x) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

__device__ __forceinline__ float bf2f(uint16_t x) { return __bfloat162float(__ushort_as_bfloat16(x)); }

}  // namespace

__global__ void __launch_bounds__(kGemmThreads) mlp_gemm_kernel(const GemmArgs g) {
    __shared__ uint16_t As[BM][BK + 8];   // [m][k]
    __shared__ uint16_t Bs[BN][BK + 8];   // [n][k]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int gr = lane >> 2, tq = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
    for (int k0 = 0; k0 < g.K; k0 += BK) {
        for (int e = tid; e < BM * BK; e += kGemmThreads) {
            const int mm = e / BK, kk = e % BK;
            const int m = m0 + mm, k = k0 + kk;
            As[mm][kk] = (m < g.M && k < g.K) ? g.A[m * g.sAm + k * g.sAk] : (uint16_t)0;
        }
        for (int e = tid; e < BN * BK; e += kGemmThreads) {
            const int nn = e / BK, kk = e % BK;
            const int n = n0 + nn, k = k0 + kk;
            Bs[nn][kk] = (n < g.N && k < g.K) ? g.B[k * g.sBk + n * g.sBn] : (uint16_t)0;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < BK; ks += 16) {
            uint32_t a[2][4], b[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + i * 16 + gr;
                a[i][0] = pack2(As[r][ks + 2 * tq], As[r][ks + 2 * tq + 1]);
                a[i][1] = pack2(As[r + 8][ks + 2 * tq], As[r + 8][ks + 2 * tq + 1]);
                a[i][2] = pack2(As[r][ks + 2 * tq + 8], As[r][ks + 2 * tq + 9]);
                a[i][3] = pack2(As[r + 8][ks + 2 * tq + 8], As[r + 8][ks + 2 * tq + 9]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = wn + j * 8 + gr;
                b[j][0] = pack2(Bs[c][ks + 2 * tq], Bs[c][ks + 2 * tq + 1]);
                b[j][1] = pack2(Bs[c][ks + 2 * tq + 8], Bs[c][ks + 2 * tq + 9]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
    // epilogue
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int m = m0 + wm + i * 16 + gr + ((e >> 1) ? 8 : 0);
                const int n = n0 + wn + j * 8 + 2 * tq + (e & 1);
                if (m >= g.M || n >= g.N) continue;
                float v = acc[i][j][e];
                if (g.epi & EPI_BIAS) v += g.bias[n];
                if (g.epi & EPI_RELU) v = fmaxf(v, 0.f);
                if ((g.epi & EPI_MASK) && !(bf2f(g.mask[m * g.ldm + n]) > 0.f)) v = 0.f;
                if (g.epi & EPI_BF16) {
                    static_cast<uint16_t *>(g.C)[m * g.ldc + n] = f2bf(v);
                } else {
                    float *C = static_cast<float *>(g.C);
                    if (g.epi & EPI_ACCUM) v += C[m * g.ldc + n];
                    C[m * g.ldc + n] = v;
                }
            }
}

static cudaError_t gemm(const GemmArgs &g, cudaStream_t s) {
    if (g.M <= 0 || g.N <= 0) return cudaSuccess;
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM);
    mlp_gemm_kernel<<<grid, kGemmThreads, 0, s>>>(g);
    return cudaGetLastError();
}

// db[n] = sum_m dz[m][n] (dz BF16 [M][N]), FP32 accumulation.
__global__ void col_sum_kernel(const uint16_t *dz, int M, int N, float *db) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int m = 0; m < M; ++m) s += bf2f(dz[(long long)m * N + n]);
    db[n] = s;
}

__global__ void f32_to_bf16_kernel(const float *x, long long n, uint16_t *y) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) y[i] = f2bf(x[i]);
}

// Adam (Kingma & Ba): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
// w -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps); BF16 copy refreshed.
__global__ void adam_kernel(long long n, float *w, uint16_t *wb, const float *g, float *m, float *v,
                            float lr, float b1, float b2, float eps, float c1, float c2) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (wb) wb[i] = f2bf(wi);
}

}  // namespace mdx

using namespace mdx;

static int mlp_check(const mdx_mlp *net, int batch) {
    if (!net || net->n_layers < 1 || net->n_layers > MDX_MLP_MAX_LAYERS)
        return set_last_error(MDX_ERR_ARG, "n_layers must be in 1..MDX_MLP_MAX_LAYERS");
    if (batch < 1) return set_last_error(MDX_ERR_ARG, "batch must be >= 1");
    for (int l = 0; l <= net->n_layers; ++l)
        if (net->dims[l] < 1) return set_last_error(MDX_ERR_ARG, "layer widths must be >= 1");
    for (int l = 0; l < net->n_layers; ++l)
        if (!net->W[l] || !net->b[l]) return set_last_error(MDX_ERR_ARG, "missing weights or biases");
    return MDX_OK;
}

static long long act_offset(const mdx_mlp *net, int batch, int l) {
    // activations of hidden layers 1..L-1, each [batch][d_l], concatenated
    long long off = 0;
    for (int j = 1; j < l; ++j) off += (long long)batch * net->dims[j];
    return off;
}

extern "C" size_t mdx_mlp_act_elems(const mdx_mlp *net, int batch) {
    if (mlp_check(net, batch)) return 0;
    return (size_t)act_offset(net, batch, net->n_layers);
}

extern "C" int mdx_mlp_forward(const mdx_mlp *net, int batch, const uint16_t *x, uint16_t *acts,
                               float *y, void *stream) {
    int rc = mlp_check(net, batch);
    if (rc) return rc;
    if (!x || !y || (net->n_layers > 1 && !acts)) return set_last_error(MDX_ERR_ARG, "null buffer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint16_t *in = x;
    for (int l = 0; l < net->n_layers; ++l) {
        const int K = net->dims[l], N = net->dims[l + 1];
        const bool last = l == net->n_layers - 1;
        GemmArgs g{};
        g.M = batch;
        g.N = N;
        g.K = K;
        g.A = in;
        g.sAm = K;
        g.sAk = 1;
        g.B = net->W[l];        // W[n][k] -> B(k, n) = W[n * K + k]
        g.sBk = 1;
        g.sBn = K;
        g.bias = net->b[l];
        if (last) {
            g.C = y;
            g.ldc = N;
            g.epi = EPI_BIAS;
        } else {
            uint16_t *out = acts + act_offset(net, batch, l + 1);
            g.C = out;
            g.ldc = N;
            g.epi = EPI_BIAS | EPI_RELU | EPI_BF16;
            in = out;
        }
        if (gemm(g, s) != cudaSuccess) return set_last_error(MDX_ERR_CUDA, "mlp forward launch failed");
    }
    return MDX_OK;
}

extern "C" size_t mdx_mlp_work_elems(const mdx_mlp *net, int batch) {
    if (mlp_check(net, batch)) return 0;
    int dmax = 0;
    for (int l = 0; l <= net->n_layers; ++l) dmax = net->dims[l] > dmax ? net->dims[l] : dmax;
    return (size_t)2 * batch * dmax;
}

extern "C" int mdx_mlp_backward(const mdx_mlp *net, int batch, const uint16_t *x,
                                const uint16_t *acts, const float *dy, float *const *dW,
                                float *const *db, uint16_t *work, void *stream) {
    int rc = mlp_check(net, batch);
    if (rc) return rc;
    if (!x || !dy || !dW || !db || !work) return set_last_error(MDX_ERR_ARG, "null buffer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dmax = 0;
    for (int l = 0; l <= net->n_layers; ++l) dmax = net->dims[l] > dmax ? net->dims[l] : dmax;
    uint16_t *dz = work;                              // BF16 [batch][d_{l+1}] of the current layer
    uint16_t *dz_next = work + (long long)batch * dmax;
    // output layer: dz = dy (linear), rounded to BF16 once
    {
        const long long n = (long long)batch * net->dims[net->n_layers];
        f32_to_bf16_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(dy, n, dz);
    }
    for (int l = net->n_layers - 1; l >= 0; --l) {
        const int K = net->dims[l], N = net->dims[l + 1];
        const uint16_t *in = (l == 0) ? x : acts + act_offset(net, batch, l);
        // dW[n][k] = sum_m dz[m][n] in[m][k]
        GemmArgs g{};
        g.M = N;
        g.N = K;
        g.K = batch;
        g.A = dz;               // A(n, m) = dz[m * N + n]
        g.sAm = 1;
        g.sAk = N;
        g.B = in;               // B(m, k) = in[m * K + k]
        g.sBk = K;
        g.sBn = 1;
        g.C = dW[l];
        g.ldc = K;
        g.epi = EPI_NONE;
        if (gemm(g, s) != cudaSuccess) return set_last_error(MDX_ERR_CUDA, "mlp backward launch failed");
        col_sum_kernel<<<(N + 127) / 128, 128, 0, s>>>(dz, batch, N, db[l]);
        if (l > 0) {
            // dz_prev[m][k] = (sum_n dz[m][n] W[n][k]) * [act_l[m][k] > 0], BF16
            GemmArgs h{};
            h.M = batch;
            h.N = K;
            h.K = N;
            h.A = dz;
            h.sAm = N;
            h.sAk = 1;
            h.B = net->W[l];    // B(n, k) = W[n * K + k]
            h.sBk = K;
            h.sBn = 1;
            h.C = dz_next;
            h.ldc = K;
            h.mask = in;
            h.ldm = K;
            h.epi = EPI_MASK | EPI_BF16;
            if (gemm(h, s) != cudaSuccess) return set_last_error(MDX_ERR_CUDA, "mlp backward launch failed");
            uint16_t *t = dz;
            dz = dz_next;
            dz_next = t;
        }
    }
    if (cudaGetLastError() != cudaSuccess) return set_last_error(MDX_ERR_CUDA, "mlp backward launch failed");
    return MDX_OK;
}

extern "C" int mdx_adam_step(long long n, float *w, uint16_t *w_bf16, const float *g, float *m,
                             float *v, float lr, float beta1, float beta2, float eps, int t,
                             void *stream) {
    if (n < 0 || !w || !g || !m || !v || t < 1) return set_last_error(MDX_ERR_ARG, "bad Adam arguments");
    if (n == 0) return MDX_OK;
    const float c1 = 1.f - powf(beta1, (float)t), c2 = 1.f - powf(beta2, (float)t);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, w, w_bf16, g, m, v, lr, beta1, beta2,
                                                            eps, c1, c2);
    if (cudaGetLastError() != cudaSuccess) return set_last_error(MDX_ERR_CUDA, "adam launch failed");
    return MDX_OK;
}

extern "C" int mdx_f32_to_bf16(long long n, const float *x, uint16_t *y, void *stream) {
    if (n < 0 || (n > 0 && (!x || !y))) return set_last_error(MDX_ERR_ARG, "bad conversion arguments");
    if (n == 0) return MDX_OK;
    f32_to_bf16_kernel<<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, n, y);
    if (cudaGetLastError() != cudaSuccess) return set_last_error(MDX_ERR_CUDA, "conversion launch failed");
    return MDX_OK;
}
