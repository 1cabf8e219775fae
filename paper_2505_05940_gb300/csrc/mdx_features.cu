// Log-mel features of simulated audio: the input of the learned proposal
// network (initial estimates for the inverse fits of Sec. 4.3).
//
// Per signal x of length T and segment s of S:
//   frames   f = 0 .. F-1, F = 1 + T / hop, frame f covers the signal extended
//            by reflection by n_fft / 2 on both sides (centred frames), times
//            the periodic Hann window w_j = (1 - cos(2 pi j / n_fft)) / 2;
//   power    P_f[k] = |sum_j w_j x_f[j] e^{-2 pi i j k / n_fft}|^2, k <= n_fft / 2;
//   mel      m_f[i] = log(sum_k W[i][k] P_f[k] + 1e-6), W the triangular filters
//            equally spaced on the HTK mel scale mel(f) = 2595 log10(1 + f / 700)
//            between fmin and fmax (n_mels + 2 points; filter i rises from
//            point i to point i+1 and falls to point i+2);
//   output   out[i][s] = mean of m_f[i] over frames floor(s F / S) .. floor((s+1) F / S) - 1
//            (at least one frame).
// One CTA per (segment, signal): an iterative radix-2 FFT in shared memory
// per frame (FP32, twiddles from FP64 sincospi), the filters evaluated in
// FP64 once per CTA and kept per bin (a bin lies in at most two adjacent
// triangles), the frame loop in order, so the result is deterministic.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/mdx.h"
#include "mdx_internal.h"

namespace mdx {

namespace {

constexpr int kFeatThreads = 512;

struct LogmelArgs {
    const float *audio;
    int batch, T, n_fft, log2n, hop, n_mels, segments;
    double fs, fmin, fmax;
    float *out;
};

__device__ __forceinline__ double hz_to_mel(double f) { return 2595.0 * log10(1.0 + f / 700.0); }
__device__ __forceinline__ double mel_to_hz(double m) { return 700.0 * (pow(10.0, m / 2595.0) - 1.0); }

__device__ __forceinline__ double tri_weight(const double *pts, int i, double f) {
    const double lo = pts[i], c = pts[i + 1], hi = pts[i + 2];
    const double up = (f - lo) / fmax(c - lo, 1e-9);
    const double dn = (hi - f) / fmax(hi - c, 1e-9);
    return fmax(0.0, fmin(up, dn));
}

// Byte offsets of the shared-memory arrays (one definition for the kernel and
// the launch): X [n] float2, tw [n/2] float2, P, w1, w2 [n/2 + 1] float,
// ifirst [n/2 + 1] int, pts [n_mels + 2] double (8-byte aligned).
struct FeatLayout {
    size_t tw, P, w1, w2, ifirst, pts, end;
};

__host__ __device__ inline FeatLayout feat_layout(int n_fft, int n_mels) {
    const size_t half = (size_t)n_fft / 2;
    FeatLayout L;
    L.tw = sizeof(float2) * (size_t)n_fft;
    L.P = L.tw + sizeof(float2) * half;
    L.w1 = L.P + sizeof(float) * (half + 1);
    L.w2 = L.w1 + sizeof(float) * (half + 1);
    L.ifirst = L.w2 + sizeof(float) * (half + 1);
    L.pts = (L.ifirst + sizeof(int) * (half + 1) + 7) & ~(size_t)7;
    L.end = L.pts + sizeof(double) * (size_t)(n_mels + 2);
    return L;
}

__global__ void __launch_bounds__(kFeatThreads) logmel_kernel(const LogmelArgs A) {
    extern __shared__ __align__(16) unsigned char fsm[];
    const int n = A.n_fft, half = n / 2;
    const FeatLayout FL = feat_layout(n, A.n_mels);
    float2 *X = reinterpret_cast<float2 *>(fsm);
    float2 *tw = reinterpret_cast<float2 *>(fsm + FL.tw);
    float *P = reinterpret_cast<float *>(fsm + FL.P);
    float *w1 = reinterpret_cast<float *>(fsm + FL.w1);
    float *w2 = reinterpret_cast<float *>(fsm + FL.w2);
    int *ifirst = reinterpret_cast<int *>(fsm + FL.ifirst);
    double *pts = reinterpret_cast<double *>(fsm + FL.pts);
    const int s = blockIdx.x, b = blockIdx.y, tid = threadIdx.x;
    const int T = A.T, hop = A.hop, S = A.segments, nm = A.n_mels;
    const int F = 1 + T / hop;
    const int f0 = (int)(((long long)s * F) / S);
    int f1 = (int)(((long long)(s + 1) * F) / S);
    f1 = min(max(f1, f0 + 1), F);
    const float *x = A.audio + (long long)b * T;

    // twiddles, mel points (numpy linspace: a + j step, the last point exact)
    for (int k = tid; k < half; k += blockDim.x) {
        double sn, cs;
        sincospi(-2.0 * k / n, &sn, &cs);
        tw[k] = make_float2((float)cs, (float)sn);
    }
    const double m_lo = hz_to_mel(A.fmin), m_hi = hz_to_mel(A.fmax);
    const double mstep = (m_hi - m_lo) / (nm + 1);
    for (int j = tid; j < nm + 2; j += blockDim.x)
        pts[j] = mel_to_hz(j == nm + 1 ? m_hi : m_lo + j * mstep);
    __syncthreads();
    // per bin: the two triangles that may contain it (i_first and i_first + 1)
    const double df = (A.fs / 2.0) / half;
    for (int k = tid; k <= half; k += blockDim.x) {
        const double f = (k == half) ? A.fs / 2.0 : k * df;
        int lo = -1, hi = nm + 2;                 // largest j with pts[j] < f
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (pts[mid] < f) lo = mid; else hi = mid;
        }
        const int i0 = lo - 1;
        ifirst[k] = i0;
        w1[k] = (i0 >= 0 && i0 < nm) ? (float)tri_weight(pts, i0, f) : 0.f;
        w2[k] = (i0 + 1 >= 0 && i0 + 1 < nm) ? (float)tri_weight(pts, i0 + 1, f) : 0.f;
    }
    __syncthreads();
    int kmin = 0, kmax = -1;
    if (tid < nm) {
        kmin = max(0, (int)floor(pts[tid] / df));
        kmax = min(half, (int)ceil(pts[tid + 2] / df));
    }
    float acc = 0.f;
    const int pad = n / 2;
    for (int f = f0; f < f1; ++f) {
        // windowed frame, stored in bit-reversed order
        for (int j = tid; j < n; j += blockDim.x) {
            int t = f * hop + j - pad;
            if (t < 0) t = -t;
            if (t >= T) t = 2 * (T - 1) - t;
            const float w = (float)(0.5 * (1.0 - cospi(2.0 * j / n)));
            const int r = (int)(__brev((unsigned)j) >> (32 - A.log2n));
            X[r] = make_float2(w * x[t], 0.f);
        }
        __syncthreads();
        for (int len = 2; len <= n; len <<= 1) {
            const int hl = len >> 1, stride = n / len;
            for (int t = tid; t < half; t += blockDim.x) {
                const int g = t / hl, pos = t - g * hl;
                const int i0 = g * len + pos, i1 = i0 + hl;
                const float2 w = tw[pos * stride];
                const float2 a = X[i0], c = X[i1];
                const float2 bw = make_float2(c.x * w.x - c.y * w.y, c.x * w.y + c.y * w.x);
                X[i0] = make_float2(a.x + bw.x, a.y + bw.y);
                X[i1] = make_float2(a.x - bw.x, a.y - bw.y);
            }
            __syncthreads();
        }
        for (int k = tid; k <= half; k += blockDim.x) P[k] = X[k].x * X[k].x + X[k].y * X[k].y;
        __syncthreads();
        if (tid < nm) {
            float v = 0.f;
            for (int k = kmin; k <= kmax; ++k) {
                const int i0 = ifirst[k];
                const float wt = (i0 == tid) ? w1[k] : ((i0 + 1 == tid) ? w2[k] : 0.f);
                v = fmaf(wt, P[k], v);
            }
            acc += logf(v + 1e-6f);
        }
        __syncthreads();
    }
    if (tid < nm) A.out[((long long)b * nm + tid) * S + s] = acc / (float)(f1 - f0);
}

size_t logmel_smem(int n_fft, int n_mels) { return feat_layout(n_fft, n_mels).end; }

}  // namespace

}  // namespace mdx

extern "C" int mdx_logmel(const float *audio, int batch, int T, double fs, int n_fft, int hop,
                          int n_mels, double fmin, double fmax, int segments, float *out,
                          void *stream) {
    using namespace mdx;
    if (!audio || !out) return set_last_error(MDX_ERR_ARG, "audio and out are required");
    if (batch < 1 || segments < 1) return set_last_error(MDX_ERR_ARG, "batch and segments must be >= 1");
    if (n_fft < 16 || n_fft > 2048 || (n_fft & (n_fft - 1)) != 0)
        return set_last_error(MDX_ERR_ARG, "n_fft must be a power of two in [16, 2048]");
    int log2n = 0;
    while ((1 << log2n) < n_fft) ++log2n;
    if (hop < 1) return set_last_error(MDX_ERR_ARG, "hop must be >= 1");
    if (T <= n_fft / 2) return set_last_error(MDX_ERR_ARG, "T must exceed n_fft / 2 (reflection padding)");
    if (1 + T / hop < segments) return set_last_error(MDX_ERR_ARG, "fewer frames than segments");
    if (n_mels < 1 || n_mels > kFeatThreads)
        return set_last_error(MDX_ERR_ARG, "n_mels must be in [1, 512]");
    if (!(fs > 0.0) || !(fmin >= 0.0) || !(fmax > fmin) || fmax > fs / 2.0)
        return set_last_error(MDX_ERR_ARG, "need 0 <= fmin < fmax <= fs / 2");
    LogmelArgs A{audio, batch, T, n_fft, log2n, hop, n_mels, segments, fs, fmin, fmax, out};
    const size_t smem = logmel_smem(n_fft, n_mels);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    logmel_kernel<<<dim3((unsigned)segments, (unsigned)batch), kFeatThreads, smem, s>>>(A);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_last_error(MDX_ERR_CUDA, cudaGetErrorString(e));
    return MDX_OK;
}
