// Learned-proposal network: a small MLP trained on simulator output.
//
// Layers d0 -> d1 -> ... -> dL with ReLU between hidden layers and a linear
// output.  Weights are BF16 (an FP32 master copy is kept for the optimiser);
// every product accumulates in FP32 on the fifth-generation tensor cores
// (tcgen05.mma kind::f16, BF16 x BF16 -> FP32 in tensor memory).  Activations
// are stored in BF16 between layers.
//
// Kernels: one generic strided GEMM with fused epilogues (bias, ReLU, ReLU
// mask of the backward pass, FP32 or BF16 output), a column-sum for bias
// gradients, and the Adam update.  The GEMM computes one 128 x 128 output
// tile per CTA: 64-wide K chunks of both operands are staged (16-byte
// vectors where K is contiguous in memory, coalesced gathers where the
// operand is transposed) into K-major core-matrix images in two buffers, one
// thread issues four 128 x N x 16 MMAs per chunk and commits to the buffer's
// mbarrier, so the next chunk's staging overlaps the MMAs; four warps read
// the accumulator with tcgen05.ld (one lane quarter each, one output row per
// lane) and apply the epilogue.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/mdx.h"
#include "mdx_internal.h"
#include "mdx_tc.cuh"

namespace mdx {

namespace {

constexpr int TBM = 128, TBN = 128, TBK = 64;   // output tile, K chunk (BF16 elements)
constexpr int kGemmThreads = 128;                // 4 warps = the 4 tensor-memory lane quarters
constexpr int kTileBytes = TBM * TBK * 2;        // one operand chunk image (16 KB)
constexpr long long kGemmWait = 1LL << 24;

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

__device__ __forceinline__ uint16_t f2bf(float x) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

__device__ __forceinline__ float bf2f(uint16_t x) { return __bfloat162float(__ushort_as_bfloat16(x)); }

// Instruction descriptor of kind::f16 with BF16 A and B (both K-major) and an
// FP32 accumulator, shape M x N.
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16_tc(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Stages rows row0 .. row0+127 (valid below `rows`) and K columns k0 .. k0+63
// (valid below K) of a strided BF16 matrix, element (r, k) at
// src[r * s_r + k * s_k], into a K-major core-matrix image: 16-byte units of
// 8 K-adjacent elements, 8-row groups 8 units (1024 bytes) apart.
__device__ __forceinline__ void stage_operand(uint16_t *img, const uint16_t *src, long long s_r,
                                              long long s_k, int row0, int rows, int k0, int K) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool kvec = (s_k == 1) && ((s_r & 7) == 0) &&
                      ((reinterpret_cast<uintptr_t>(src) & 15) == 0);
    // each thread stages 8 units; all loads are issued before the stores
    constexpr int kU = 32 / (kGemmThreads / 32);
    uint4 v[kU];
    if (kvec) {
        // 32 units per warp: 8 rows x 4 K units (512 contiguous bytes of the image)
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int w = warp + u * (kGemmThreads / 32);
            const int r = (w >> 1) * 8 + (lane & 7), kg = (w & 1) * 4 + (lane >> 3);
            const int row = row0 + r, k = k0 + kg * 8;
            v[u] = make_uint4(0u, 0u, 0u, 0u);
            if (row < rows) {
                if (k + 8 <= K) {
                    v[u] = __ldg(reinterpret_cast<const uint4 *>(src + (long long)row * s_r + k));
                } else if (k < K) {
                    alignas(16) uint16_t t[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) t[e] = (k + e < K) ? src[(long long)row * s_r + k + e] : 0;
                    v[u] = *reinterpret_cast<const uint4 *>(t);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int w = warp + u * (kGemmThreads / 32);
            const int r = (w >> 1) * 8 + (lane & 7), kg = (w & 1) * 4 + (lane >> 3);
            *reinterpret_cast<uint4 *>(img + (((r >> 3) * 8 + kg) * 64 + (r & 7) * 8)) = v[u];
        }
    } else {
        // transposed operand: lanes walk 32 consecutive rows (coalesced when s_r = 1)
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int w = warp + u * (kGemmThreads / 32);
            const int r = (w & 3) * 32 + lane, kg = w >> 2;
            const int row = row0 + r, k = k0 + kg * 8;
            alignas(16) uint16_t t[8];
#pragma unroll
            for (int e = 0; e < 8; ++e)
                t[e] = (row < rows && k + e < K) ? src[(long long)row * s_r + (long long)(k + e) * s_k] : 0;
            v[u] = *reinterpret_cast<const uint4 *>(t);
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int w = warp + u * (kGemmThreads / 32);
            const int r = (w & 3) * 32 + lane, kg = w >> 2;
            *reinterpret_cast<uint4 *>(img + (((r >> 3) * 8 + kg) * 64 + (r & 7) * 8)) = v[u];
        }
    }
}

struct GemmCtrl {
    uint64_t bar[2];
    uint32_t tmem;
    int fail;
};

}  // namespace

__global__ void __launch_bounds__(kGemmThreads) mlp_gemm_kernel(const GemmArgs g) {
    using namespace tc;
    extern __shared__ __align__(1024) unsigned char gsm[];
    GemmCtrl &C = *reinterpret_cast<GemmCtrl *>(gsm);
    uint16_t *img = reinterpret_cast<uint16_t *>(gsm + 1024);   // [2 buffers][A, B] 16 KB each
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * TBN;
    const int nvalid = min(TBN, g.N - n0);
    const int NT = (nvalid + 15) & ~15;                         // MMA N (multiple of 16)
    const int chunks = (g.K + TBK - 1) / TBK;
    if (tid == 0) {
        bar_init(&C.bar[0], 1);
        bar_init(&C.bar[1], 1);
        C.fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(
                         su32(&C.tmem))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = C.tmem;
    const uint32_t idesc = idesc_bf16(TBM, NT);
    bool ok = true;
    int committed = 0;   // chunks whose MMAs thread 0 has committed
    for (int c = 0; c < chunks && ok; ++c) {
        const int b = c & 1;
        uint16_t *Ai = img + (size_t)b * 2 * (kTileBytes / 2);
        uint16_t *Bi = Ai + kTileBytes / 2;
        if (c >= 2) {
            // the MMAs of chunk c - 2 have read this buffer
            long long i = 0;
            while (!bar_try(&C.bar[b], (uint32_t)(((c - 2) >> 1) & 1)) && ++i < kGemmWait) {
            }
            if (i >= kGemmWait) C.fail = 1;
            __syncthreads();
            if (C.fail) {
                ok = false;
                break;
            }
        }
        stage_operand(Ai, g.A, g.sAm, g.sAk, m0, g.M, c * TBK, g.K);
        stage_operand(Bi, g.B, g.sBn, g.sBk, n0, g.N, c * TBK, g.K);
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a0 = su32(Ai), b0 = su32(Bi);
#pragma unroll
            for (int kk = 0; kk < TBK / 16; ++kk) {
                const uint64_t ad = smem_desc(a0 + kk * 256u, 128u, 1024u);
                const uint64_t bd = smem_desc(b0 + kk * 256u, 128u, 1024u);
                mma_bf16_tc(tmem, ad, bd, idesc, (c | kk) ? 1u : 0u);
            }
            mma_commit(&C.bar[b]);
            ++committed;
        }
    }
    // the last commit covers every MMA issued before it
    if (ok && chunks > 0) {
        const int c = chunks - 1;
        long long i = 0;
        while (!bar_try(&C.bar[c & 1], (uint32_t)((c >> 1) & 1)) && ++i < kGemmWait) {
        }
        if (i >= kGemmWait) ok = false;
    }
    tc_fence_after();
    // epilogue: warp q owns tensor-memory lanes 32 q .. 32 q + 31 (output rows)
    const int m = m0 + warp * 32 + lane;
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    for (int cb = 0; cb < NT; cb += 16) {
        float v[16];
        if (chunks > 0) {
            tmem_ld16(tmem + lane_base + (uint32_t)cb, v);
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = 0.f;
        }
        if (m >= g.M) continue;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int n = n0 + cb + j;
            if (cb + j >= nvalid) break;
            float x = ok ? v[j] : __int_as_float(0x7fc00000);
            if (g.epi & EPI_BIAS) x += g.bias[n];
            if (g.epi & EPI_RELU) x = fmaxf(x, 0.f);
            if ((g.epi & EPI_MASK) && !(bf2f(g.mask[(long long)m * g.ldm + n]) > 0.f)) x = 0.f;
            if (g.epi & EPI_BF16) {
                static_cast<uint16_t *>(g.C)[(long long)m * g.ldc + n] = f2bf(x);
            } else {
                float *Cp = static_cast<float *>(g.C);
                if (g.epi & EPI_ACCUM) x += Cp[(long long)m * g.ldc + n];
                Cp[(long long)m * g.ldc + n] = x;
            }
        }
    }
    if (!ok && tid == 0) {
        // a wait ran out: let the MMAs in flight finish before the memory is
        // released (the last commit on each buffer's barrier)
        for (int bb = 0; bb < 2; ++bb) {
            const int cnt = (committed + 1 - bb) / 2;
            if (cnt <= 0) continue;
            long long i = 0;
            while (!bar_try(&C.bar[bb], (uint32_t)((cnt - 1) & 1)) && ++i < kGemmWait) {
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem) : "memory");
}

namespace {

constexpr size_t kGemmSmem = 1024 + 4 * (size_t)kTileBytes;
std::once_flag g_gemm_attr;

}  // namespace

static cudaError_t gemm(const GemmArgs &g, cudaStream_t s) {
    if (g.M <= 0 || g.N <= 0) return cudaSuccess;
    std::call_once(g_gemm_attr, [] {
        cudaFuncSetAttribute(mlp_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kGemmSmem);
    });
    dim3 grid((g.N + TBN - 1) / TBN, (g.M + TBM - 1) / TBM);
    mlp_gemm_kernel<<<grid, kGemmThreads, kGemmSmem, s>>>(g);
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
