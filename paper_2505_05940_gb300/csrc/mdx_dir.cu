// Directional derivative <dL/dH, dH> of one adjoint segment.
//
// With f_s = sum_k kappa_k eta_k (H^k q)_s (Sec. 3.1, Eq. 9) the loss
// gradient with respect to the (symmetric) coupling tensor, contracted with a
// direction tensor dH, is
//     -sum_k kappa_k sum_n (z_k^n)^T dH^k q^n,   z_k^n = xi_k^n q^n + eta_k^n w^n,
// where q^n is the forward state, w^n = r a^{n+1} the scaled adjoint and
// eta_k^n = q.H^k q, xi_k^n = w.H^k q the per-step scalars the reverse sweep
// stores.  Over one segment of L steps this is, per stress mode,
//     <dH^k, G_k>,  G_k = sum_n z_k^n (q^n)^T  (a GEMM over the segment),
// so dH is read once per segment instead of once per step.
//
// One CTA per (plate, stress mode).  G_k is formed only on the coupling
// blocks (all of H^k for the dense layout, the four symmetry-class blocks for
// the class layout) in 64 x 64 output tiles, 4 x 4 per thread, over step
// tiles of 32 held in shared memory.
//
// The same kernels give the full gradient dL/dH (WRITE = true): instead of
// the contraction with dH, -kappa_k G_k is added into an FP64 output in each
// plate's own mode order; after the last segment the output is symmetrised,
// dL/dH^k_ij = -kappa_k (G_k + G_k^T)_ij / 2, since H^k is symmetric.
#include <cuda_runtime.h>

#include "../../include/mdx.h"
#include "mdx_common.cuh"
#include "mdx_tc.cuh"

namespace mdx {

namespace {

constexpr int kTile = 64;     // output tile edge
constexpr int kStepTile = 32; // steps per shared-memory tile
constexpr int kDirThreads = 256;

__device__ __forceinline__ int pick4d(const int (&v)[4], int a) {
    return a == 0 ? v[0] : (a == 1 ? v[1] : (a == 2 ? v[2] : v[3]));
}

}  // namespace

template <bool WRITE>
__global__ void __launch_bounds__(kDirThreads) dir_contract_kernel(const DirParams P) {
    __shared__ float Zt[kTile][kStepTile + 1];
    __shared__ float Qt[kTile][kStepTile + 1];
    __shared__ float red[kDirThreads / 32];
    const DirUnit U = P.units[blockIdx.x];
    const InstDesc d = P.inst[U.inst];
    const int tid = threadIdx.x;
    const int tr = tid / 16, tc = tid % 16;        // 16 x 16 threads, 4 x 4 outputs each
    const long long TM = P.total_modes;
    const int kint = U.kl;                          // internal stress index within the plate
    const long long kk = d.k_off + kint;
    float part = 0.f;
    const int nblocks = d.parity ? 4 : 1;
    long long cursor = 0;                            // class layout: offset of super-block a
    for (int a = 0; a < nblocks; ++a) {
        int nr, nc, orow, ocol, nb4, mc = 1, kl = 0;
        if (d.parity) {
            const int bcl = a ^ U.c;
            nr = pick4d(d.ncls, a);
            nc = pick4d(d.ncls, bcl);
            orow = pick4d(d.ocls, a);
            ocol = pick4d(d.ocls, bcl);
            nb4 = (nc + 3) & ~3;
            mc = U.mc;
            kl = U.kpos;
        } else {
            nr = nc = d.N;
            orow = ocol = 0;
            nb4 = d.Npad;
        }
        const float *blk = d.parity ? P.dH + U.off + cursor
                                    : P.dH + d.dH_off + (long long)kint * d.N * d.Npad;
        if (d.parity) cursor += (long long)nr * mc * nb4;
        if (nr == 0 || nc == 0) continue;
        for (int r0 = 0; r0 < nr; r0 += kTile) {
            for (int c0 = 0; c0 < nc; c0 += kTile) {
                float acc[4][4];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
                for (int n0 = 0; n0 < P.steps; n0 += kStepTile) {
                    // z rows and q columns of this step tile (mode indices through the
                    // class permutation for the class layout)
                    for (int e = tid; e < kTile * kStepTile; e += kDirThreads) {
                        const int rr = e / kStepTile, nn = e % kStepTile;
                        const int n = n0 + nn;
                        float z = 0.f, qc = 0.f;
                        if (n < P.steps) {
                            const float xi = P.xe[((long long)n * 2 + 0) * P.total_k + kk];
                            const float eta = P.xe[((long long)n * 2 + 1) * P.total_k + kk];
                            if (r0 + rr < nr) {
                                const int pos = orow + r0 + rr;
                                const int m = d.parity ? P.perm[d.perm_off + pos] : pos;
                                const long long g = (long long)n * TM + d.mode_off + m;
                                z = fmaf(xi, P.seg_q[g], eta * P.seg_w[g]);
                            }
                            if (c0 + rr < nc) {
                                const int pos = ocol + c0 + rr;
                                const int m = d.parity ? P.perm[d.perm_off + pos] : pos;
                                qc = P.seg_q[(long long)n * TM + d.mode_off + m];
                            }
                        }
                        Zt[rr][nn] = z;
                        Qt[rr][nn] = qc;
                    }
                    __syncthreads();
#pragma unroll 4
                    for (int nn = 0; nn < kStepTile; ++nn) {
                        float zr[4], qv[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            zr[i] = Zt[tr * 4 + i][nn];
                            qv[i] = Qt[tc * 4 + i][nn];
                        }
#pragma unroll
                        for (int i = 0; i < 4; ++i)
#pragma unroll
                            for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(zr[i], qv[j], acc[i][j]);
                    }
                    __syncthreads();
                }
                if constexpr (WRITE) {
                    // -kappa_k G_k into the plate's [k][i][j] block (user order)
                    const double sc = -(double)P.kappa[kk];
                    const int ku = P.kperm[kk];
                    double *blkout = P.dH_out + P.dh_off[U.inst] + (long long)ku * d.N * d.N;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int rr = r0 + tr * 4 + i;
                        if (rr >= nr) continue;
                        const int mi = d.parity ? P.perm[d.perm_off + orow + rr] : orow + rr;
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int cc = c0 + tc * 4 + j;
                            if (cc >= nc) continue;
                            const int mj = d.parity ? P.perm[d.perm_off + ocol + cc] : ocol + cc;
                            blkout[(long long)mi * d.N + mj] += sc * (double)acc[i][j];
                        }
                    }
                } else {
                    // <dH block tile, G tile>
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int rr = r0 + tr * 4 + i;
                        if (rr >= nr) continue;
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int cc = c0 + tc * 4 + j;
                            if (cc >= nc) continue;
                            const float h = d.parity ? blk[((long long)rr * mc + kl) * nb4 + cc]
                                                     : blk[(long long)rr * d.Npad + cc];
                            part = fmaf(h, acc[i][j], part);
                        }
                    }
                }
            }
        }
    }
    if constexpr (!WRITE) {
        part = warp_sum(part);
        if ((tid & 31) == 0) red[tid >> 5] = part;
        __syncthreads();
        if (tid == 0) {
            float t = 0.f;
            for (int w = 0; w < kDirThreads / 32; ++w) t += red[w];
            const float kap = P.kappa[kk];
            P.dir_acc[kk * 4] += -(double)kap * (double)t;
        }
    }
}

// Class layout: one CTA per (plate, stress-mode class c, row class a).  For a
// batch of KB stress modes of class c, each thread accumulates a 4 x 4 tile of
// G_k = sum_n z_k^n (q_b^n)^T (rows p of class a, columns s of class b = a ^ c)
// over the segment's steps, with z_k^n = xi_k^n q_a^n + eta_k^n w_a^n formed on
// the fly from shared-memory state tiles; then <dH^k_ab, G_k> per mode.
constexpr int kDirKB = 4;
template <bool WRITE>
__global__ void __launch_bounds__(kDirThreads) dir_class_kernel(const DirParams P) {
    __shared__ float Qc[kTile][kStepTile + 1];
    __shared__ float Qr[kTile][kStepTile + 1];
    __shared__ float Wr[kTile][kStepTile + 1];
    __shared__ float XI[kDirKB][kStepTile], ET[kDirKB][kStepTile];
    __shared__ float red[kDirKB][kDirThreads / 32];
    const DirGroup Gp = P.groups[blockIdx.x];
    const InstDesc d = P.inst[Gp.inst];
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int tr = tid / 16, tc = tid % 16;
    const long long TM = P.total_modes;
    const int bcl = Gp.a ^ Gp.c;
    const int nr = pick4d(d.ncls, Gp.a), nc = pick4d(d.ncls, bcl);
    const int orow = pick4d(d.ocls, Gp.a), ocol = pick4d(d.ocls, bcl);
    const int nb4 = (nc + 3) & ~3;
    for (int kb = 0; kb < Gp.nk; kb += kDirKB) {
        const int nkb = min(kDirKB, Gp.nk - kb);
        float tot[kDirKB] = {0.f, 0.f, 0.f, 0.f};
        for (int r0 = 0; r0 < nr; r0 += kTile) {
            for (int c0 = 0; c0 < nc; c0 += kTile) {
                float acc[kDirKB][4][4];
#pragma unroll
                for (int q = 0; q < kDirKB; ++q)
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[q][i][j] = 0.f;
                for (int n0 = 0; n0 < P.steps; n0 += kStepTile) {
                    const int nst = min(kStepTile, P.steps - n0);
                    __syncthreads();
                    for (int e = tid; e < kTile * kStepTile; e += kDirThreads) {
                        const int rr = e / kStepTile, nn = e % kStepTile;
                        float qv = 0.f, wv = 0.f, cv = 0.f;
                        if (nn < nst) {
                            const long long rowoff = (long long)(n0 + nn) * TM + d.mode_off;
                            if (r0 + rr < nr) {
                                const int m = P.perm[d.perm_off + orow + r0 + rr];
                                qv = P.seg_q[rowoff + m];
                                wv = P.seg_w[rowoff + m];
                            }
                            if (c0 + rr < nc) cv = P.seg_q[rowoff + P.perm[d.perm_off + ocol + c0 + rr]];
                        }
                        Qr[rr][nn] = qv;
                        Wr[rr][nn] = wv;
                        Qc[rr][nn] = cv;
                    }
                    for (int e = tid; e < kDirKB * kStepTile; e += kDirThreads) {
                        const int q = e / kStepTile, nn = e % kStepTile;
                        float xv = 0.f, ev = 0.f;
                        if (q < nkb && nn < nst) {
                            const DirUnit u = P.units[Gp.unit0 + kb + q];
                            const long long kk = d.k_off + u.kl;
                            xv = P.xe[((long long)(n0 + nn) * 2 + 0) * P.total_k + kk];
                            ev = P.xe[((long long)(n0 + nn) * 2 + 1) * P.total_k + kk];
                        }
                        XI[q][nn] = xv;
                        ET[q][nn] = ev;
                    }
                    __syncthreads();
#pragma unroll 2
                    for (int nn = 0; nn < kStepTile; ++nn) {
                        float qr[4], wr[4], qc[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            qr[i] = Qr[tr * 4 + i][nn];
                            wr[i] = Wr[tr * 4 + i][nn];
                            qc[i] = Qc[tc * 4 + i][nn];
                        }
#pragma unroll
                        for (int q = 0; q < kDirKB; ++q) {
                            const float x = XI[q][nn], y = ET[q][nn];
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                const float z = fmaf(x, qr[i], y * wr[i]);
#pragma unroll
                                for (int j = 0; j < 4; ++j) acc[q][i][j] = fmaf(z, qc[j], acc[q][i][j]);
                            }
                        }
                    }
                }
                if constexpr (WRITE) {
                    // -kappa_k G_k into the plate's [k][i][j] block (user order)
                    for (int q = 0; q < kDirKB; ++q) {
                        if (q >= nkb) break;
                        const DirUnit u = P.units[Gp.unit0 + kb + q];
                        const long long kk = d.k_off + u.kl;
                        const double sc = -(double)P.kappa[kk];
                        double *blkout = P.dH_out + P.dh_off[Gp.inst] +
                                         (long long)P.kperm[kk] * d.N * d.N;
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int rr = r0 + tr * 4 + i;
                            if (rr >= nr) continue;
                            const int mi = P.perm[d.perm_off + orow + rr];
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const int cc = c0 + tc * 4 + j;
                                if (cc >= nc) continue;
                                const int mj = P.perm[d.perm_off + ocol + cc];
                                blkout[(long long)mi * d.N + mj] += sc * (double)acc[q][i][j];
                            }
                        }
                    }
                    continue;
                }
                // <dH^k tile, G_k tile>
#pragma unroll
                for (int q = 0; q < kDirKB; ++q) {
                    if (q >= nkb) break;
                    const DirUnit u = P.units[Gp.unit0 + kb + q];
                    long long sb = 0;
                    for (int a2 = 0; a2 < Gp.a; ++a2) {
                        const int nb2 = (pick4d(d.ncls, a2 ^ Gp.c) + 3) & ~3;
                        sb += (long long)pick4d(d.ncls, a2) * u.mc * nb2;
                    }
                    const float *blk = P.dH + u.off + sb + (long long)u.kpos * nb4;
                    const long long rstride = (long long)u.mc * nb4;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int rr = r0 + tr * 4 + i;
                        if (rr >= nr) continue;
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int cc = c0 + tc * 4 + j;
                            if (cc < nc) tot[q] = fmaf(__ldg(blk + rr * rstride + cc), acc[q][i][j], tot[q]);
                        }
                    }
                }
            }
        }
        if constexpr (WRITE) continue;
#pragma unroll
        for (int q = 0; q < kDirKB; ++q) {
            const float v = warp_sum(tot[q]);
            if (lane == 0) red[q][warp] = v;
        }
        __syncthreads();
        if (tid < nkb) {
            float t = 0.f;
            for (int w = 0; w < kDirThreads / 32; ++w) t += red[tid][w];
            const DirUnit u = P.units[Gp.unit0 + kb + tid];
            const long long kk = d.k_off + u.kl;
            P.dir_acc[kk * 4 + Gp.a] += -(double)P.kappa[kk] * (double)t;
        }
    }
}

// ---------------------------------------------------------------------------
// Tensor-core contraction (class layout).
//
// The contraction is reordered so that its inner product runs over the
// columns s of the coupling block:
//   <dH^k_ab, G_k> = sum_n xi_k^n (q_a^n . U^n_k) + eta_k^n (w_a^n . U^n_k),
//   U^n_k = dH^k_ab q_b^n,
// and all U for a tile of 128 steps and a chunk of (stress mode, row) pairs
// form one GEMM
//   D[n][(k, p)] = sum_s q_b^n[s] dH^k[p][s]      (M = 128 steps, K = s)
// on tcgen05 (kind::tf32, split TF32 as in the grouped plate kernel: both
// operands split into a round-to-nearest TF32 part and the FP32 remainder,
// three products, error about 2^-21 of |dH||q|).  The epilogue reads D from
// tensor memory, one step per lane: each thread forms q_a^n . U and
// w_a^n . U for its step over the chunk's 16 rows p and accumulates
// xi_k^n (.) + eta_k^n (.) per stress mode.  Columns of D are k-major
// (column = 16 k + p), so a 16-column tensor-memory load holds one stress
// mode's 16 rows.  One CTA per (plate, stress class c, row class a); the
// stages run in order (operand staging by all threads, the MMAs by one
// thread, then the epilogue by all eight warps, two per lane quarter).
namespace {

constexpr int kTcThreads = 256;
constexpr int kTcM = 128;          // steps per tile (MMA M, tensor-memory lanes)
constexpr int kTcP = 16;           // rows p per chunk
constexpr int kTcQ = 16;           // stress modes per chunk
constexpr int kTcRs = kTcM + 1;    // row stride of the q_a / w_a tiles
constexpr int kTcXs = kTcQ + 1;    // row stride of the xi / eta tiles
constexpr int kTcCtrl = 1024;      // control block at the start of shared memory
constexpr long long kTcWait = 1LL << 22;
constexpr int kTcBatch = 8;        // global loads in flight per thread in the staging loops

struct DirTcCtrl {
    uint64_t mma_bar;
    uint32_t tmem;
    int fail;
    long long boff[kTcQ];   // float offset of each stress mode's class-a row 0
    int rstride[kTcQ];      // floats between its rows
    int kk[kTcQ];           // global stress index
    float red[kTcThreads / 32][kTcQ / 2];
};
static_assert(sizeof(DirTcCtrl) <= kTcCtrl, "control block");

__host__ __device__ inline size_t tc_align(size_t x) { return (x + 127) & ~(size_t)127; }

struct TcLayout {
    size_t ahi, alo, bhi, blo, qa, wa, xi, et, cols, end;
};

__host__ __device__ inline TcLayout tc_layout(int kc, int nmax) {
    TcLayout L;
    size_t o = kTcCtrl;
    L.ahi = o; o = tc_align(o + (size_t)kTcM * kc * 4);
    L.alo = o; o = tc_align(o + (size_t)kTcM * kc * 4);
    L.bhi = o; o = tc_align(o + (size_t)nmax * kc * 4);
    L.blo = o; o = tc_align(o + (size_t)nmax * kc * 4);
    L.qa = o; o = tc_align(o + (size_t)kTcP * kTcRs * 4);
    L.wa = o; o = tc_align(o + (size_t)kTcP * kTcRs * 4);
    L.xi = o; o = tc_align(o + (size_t)kTcM * kTcXs * 4);
    L.et = o; o = tc_align(o + (size_t)kTcM * kTcXs * 4);
    L.cols = o; o = tc_align(o + (size_t)(kc + kTcP) * 4);
    L.end = o;
    return L;
}

__global__ void __launch_bounds__(kTcThreads, 1) dir_tc_kernel(const DirParams P) {
    using namespace tc;
    extern __shared__ __align__(1024) unsigned char smem[];
    DirTcCtrl &C = *reinterpret_cast<DirTcCtrl *>(smem);
    const int KC = P.tc_kc;
    const TcLayout L = tc_layout(KC, P.tc_nmax);
    float *Ahi = reinterpret_cast<float *>(smem + L.ahi);
    float *Alo = reinterpret_cast<float *>(smem + L.alo);
    float *Bhi = reinterpret_cast<float *>(smem + L.bhi);
    float *Blo = reinterpret_cast<float *>(smem + L.blo);
    float *Qa = reinterpret_cast<float *>(smem + L.qa);
    float *Wa = reinterpret_cast<float *>(smem + L.wa);
    float *XI = reinterpret_cast<float *>(smem + L.xi);
    float *ET = reinterpret_cast<float *>(smem + L.et);
    int *colm = reinterpret_cast<int *>(smem + L.cols);   // [KC] column modes, then [16] row modes
    int *rowm = colm + KC;

    const DirGroup Gp = P.groups[blockIdx.x];
    const InstDesc d = P.inst[Gp.inst];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long TM = P.total_modes;
    const int bcl = Gp.a ^ Gp.c;
    const int nr = pick4d(d.ncls, Gp.a), nc = pick4d(d.ncls, bcl);
    const int orow = pick4d(d.ocls, Gp.a), ocol = pick4d(d.ocls, bcl);
    const int nb4 = (nc + 3) & ~3;
    const int Kp = (nc + 7) & ~7;
    const int nkch = (Kp + KC - 1) / KC;
    const int steps = P.steps;
    const int quarter = warp & 3, half = warp >> 2;
    const int nloc = quarter * 32 + lane;                  // this thread's step in a tile
    const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;
    const uint32_t sbo = (uint32_t)(KC / 4) * 128u;

    if (tid == 0) {
        bar_init(&C.mma_bar, 1);
        C.fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(
                         su32(&C.tmem))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = C.tmem;
    uint32_t phase = 0;
    bool issued = false;
    bool failed = false;

    for (int kb = 0; kb < Gp.nk && !failed; kb += kTcQ) {
        const int nq = min(kTcQ, Gp.nk - kb);
        const int nrow = nq * kTcP;                          // B rows (a multiple of 16)
        if (tid < nq) {
            const DirUnit u = P.units[Gp.unit0 + kb + tid];
            long long sb = 0;
            for (int a2 = 0; a2 < Gp.a; ++a2) {
                const int nb2 = (pick4d(d.ncls, a2 ^ Gp.c) + 3) & ~3;
                sb += (long long)pick4d(d.ncls, a2) * u.mc * nb2;
            }
            C.boff[tid] = u.off + sb + (long long)u.kpos * nb4;
            C.rstride[tid] = u.mc * nb4;
            C.kk[tid] = (int)(d.k_off + u.kl);
        }
        float tot[kTcQ / 2];
#pragma unroll
        for (int j = 0; j < kTcQ / 2; ++j) tot[j] = 0.f;
        __syncthreads();
        for (int p0 = 0; p0 < nr && !failed; p0 += kTcP) {
            const int np = min(kTcP, nr - p0);
            if (tid < kTcP) rowm[tid] = tid < np ? P.perm[d.perm_off + orow + p0 + tid] : 0;
            for (int t0 = 0; t0 < steps && !failed; t0 += kTcM) {
                __syncthreads();   // rowm visible; the previous epilogue is done with Qa / XI
                // q_a, w_a of the chunk's rows and xi, eta of its stress modes for the
                // tile.  Every staging loop issues its global loads in batches of
                // kTcBatch before the shared-memory stores, so they overlap.
                for (int e0 = tid; e0 < kTcM * kTcP; e0 += kTcThreads * kTcBatch) {
                    float qv[kTcBatch], wv[kTcBatch];
#pragma unroll
                    for (int j = 0; j < kTcBatch; ++j) {
                        const int e = e0 + j * kTcThreads;
                        const int n = e / kTcP, pp = e % kTcP;
                        qv[j] = 0.f;
                        wv[j] = 0.f;
                        if (e < kTcM * kTcP && pp < np && t0 + n < steps) {
                            const long long g = (long long)(t0 + n) * TM + d.mode_off + rowm[pp];
                            qv[j] = __ldg(P.seg_q + g);
                            wv[j] = __ldg(P.seg_w + g);
                        }
                    }
#pragma unroll
                    for (int j = 0; j < kTcBatch; ++j) {
                        const int e = e0 + j * kTcThreads;
                        if (e >= kTcM * kTcP) break;
                        const int n = e / kTcP, pp = e % kTcP;
                        Qa[pp * kTcRs + n] = qv[j];
                        Wa[pp * kTcRs + n] = wv[j];
                    }
                }
                for (int e0 = tid; e0 < kTcM * kTcQ; e0 += kTcThreads * kTcBatch) {
                    float xv[kTcBatch], ev[kTcBatch];
#pragma unroll
                    for (int j = 0; j < kTcBatch; ++j) {
                        const int e = e0 + j * kTcThreads;
                        const int n = e / kTcQ, q = e % kTcQ;
                        xv[j] = 0.f;
                        ev[j] = 0.f;
                        if (e < kTcM * kTcQ && q < nq && t0 + n < steps) {
                            const long long base = (long long)(t0 + n) * 2 * P.total_k + C.kk[q];
                            xv[j] = __ldg(P.xe + base);
                            ev[j] = __ldg(P.xe + base + P.total_k);
                        }
                    }
#pragma unroll
                    for (int j = 0; j < kTcBatch; ++j) {
                        const int e = e0 + j * kTcThreads;
                        if (e >= kTcM * kTcQ) break;
                        const int n = e / kTcQ, q = e % kTcQ;
                        XI[n * kTcXs + q] = xv[j];
                        ET[n * kTcXs + q] = ev[j];
                    }
                }
                for (int kc = 0; kc < nkch && !failed; ++kc) {
                    const int k0 = kc * KC;
                    const int kw = min(KC, Kp - k0);            // multiple of 8
                    if (tid < KC) colm[tid] = (k0 + tid < nc) ? P.perm[d.perm_off + ocol + k0 + tid] : 0;
                    __syncthreads();
                    // A = q_b^T of the tile: element e of the core-matrix image is
                    // (row n, column s) with e = cm_index(n, s, KC)
                    for (int e0 = tid; e0 < kTcM * KC; e0 += kTcThreads * kTcBatch) {
                        float v[kTcBatch];
#pragma unroll
                        for (int j = 0; j < kTcBatch; ++j) {
                            const int e = e0 + j * kTcThreads;
                            const int cmi = e >> 5, r = (e >> 2) & 7, cc = e & 3;
                            const int n = (cmi / (KC >> 2)) * 8 + r;
                            const int sl = (cmi % (KC >> 2)) * 4 + cc;
                            v[j] = 0.f;
                            if (e < kTcM * KC && t0 + n < steps && k0 + sl < nc)
                                v[j] = __ldg(P.seg_q + (long long)(t0 + n) * TM + d.mode_off + colm[sl]);
                        }
#pragma unroll
                        for (int j = 0; j < kTcBatch; ++j) {
                            const int e = e0 + j * kTcThreads;
                            if (e >= kTcM * KC) break;
                            const float h = tf32_hi(v[j]);
                            Ahi[e] = h;
                            Alo[e] = v[j] - h;
                        }
                    }
                    // B = dH rows (k, p) of the chunk, 16-byte pieces
                    const bool stage_b = (nkch > 1) || (t0 == 0);
                    if (stage_b) {
                        const int n4 = nrow * (KC >> 2);
                        for (int e0 = tid; e0 < n4; e0 += kTcThreads * (kTcBatch / 2)) {
                            float4 v[kTcBatch / 2];
#pragma unroll
                            for (int j = 0; j < kTcBatch / 2; ++j) {
                                const int e4 = e0 + j * kTcThreads;
                                const int cmi = e4 >> 3, r = e4 & 7;
                                const int row = (cmi / (KC >> 2)) * 8 + r;
                                const int s4 = (cmi % (KC >> 2)) * 4;
                                const int q = row / kTcP, pp = row % kTcP;
                                v[j] = make_float4(0.f, 0.f, 0.f, 0.f);
                                if (e4 < n4 && pp < np && k0 + s4 < nb4) {
                                    v[j] = __ldg(reinterpret_cast<const float4 *>(
                                        P.dH + C.boff[q] + (long long)(p0 + pp) * C.rstride[q] + k0 + s4));
                                    if (k0 + s4 + 1 >= nc) v[j].y = 0.f;
                                    if (k0 + s4 + 2 >= nc) v[j].z = 0.f;
                                    if (k0 + s4 + 3 >= nc) v[j].w = 0.f;
                                }
                            }
#pragma unroll
                            for (int j = 0; j < kTcBatch / 2; ++j) {
                                const int e4 = e0 + j * kTcThreads;
                                if (e4 >= n4) break;
                                float4 h, l;
                                h.x = tf32_hi(v[j].x);
                                h.y = tf32_hi(v[j].y);
                                h.z = tf32_hi(v[j].z);
                                h.w = tf32_hi(v[j].w);
                                l.x = v[j].x - h.x;
                                l.y = v[j].y - h.y;
                                l.z = v[j].z - h.z;
                                l.w = v[j].w - h.w;
                                reinterpret_cast<float4 *>(Bhi)[e4] = h;
                                reinterpret_cast<float4 *>(Blo)[e4] = l;
                            }
                        }
                    }
                    fence_async_smem();
                    tc_fence_before();
                    __syncthreads();
                    if (tid == 0) {
                        tc_fence_after();
                        const uint32_t idesc = idesc_tf32(kTcM, nrow);
                        const uint32_t ah = su32(Ahi), al = su32(Alo), bh = su32(Bhi), bl = su32(Blo);
                        for (int ks = 0; ks < kw / 8; ++ks) {
                            const uint32_t o = (uint32_t)ks * 256u;
                            const uint64_t ad = smem_desc(ah + o, 128u, sbo);
                            const uint64_t ald = smem_desc(al + o, 128u, sbo);
                            const uint64_t bd = smem_desc(bh + o, 128u, sbo);
                            const uint64_t bld = smem_desc(bl + o, 128u, sbo);
                            mma_tf32(tmem, ad, bd, idesc, (kc | ks) ? 1u : 0u);
                            mma_tf32(tmem, ad, bld, idesc, 1u);
                            mma_tf32(tmem, ald, bd, idesc, 1u);
                        }
                        mma_commit(&C.mma_bar);
                        issued = true;
                        long long i = 0;
                        while (!bar_try(&C.mma_bar, phase) && ++i < kTcWait) {
                        }
                        if (i >= kTcWait) C.fail = 1;
                    }
                    phase ^= 1u;
                    __syncthreads();
                    tc_fence_after();
                    failed = C.fail != 0;
                }
                if (failed) break;
                // epilogue: this thread's step, stress modes q = 2 j + half
                float qa[kTcP], wa[kTcP];
#pragma unroll
                for (int pp = 0; pp < kTcP; ++pp) {
                    qa[pp] = Qa[pp * kTcRs + nloc];
                    wa[pp] = Wa[pp * kTcRs + nloc];
                }
#pragma unroll
                for (int j = 0; j < kTcQ / 2; ++j) {
                    const int q = 2 * j + half;
                    if (q >= nq) break;
                    float v[16];
                    tmem_ld16(tmem + lane_base + (uint32_t)(q * kTcP), v);
                    float al = 0.f, be = 0.f;
#pragma unroll
                    for (int pp = 0; pp < kTcP; ++pp) {
                        al = fmaf(v[pp], qa[pp], al);
                        be = fmaf(v[pp], wa[pp], be);
                    }
                    tot[j] = fmaf(XI[nloc * kTcXs + q], al, fmaf(ET[nloc * kTcXs + q], be, tot[j]));
                }
                tc_fence_before();
            }
        }
        // per stress mode: sum over the 128 steps of a tile (lanes, then the
        // four warps of a half), then -kappa_k times it into the accumulator
#pragma unroll
        for (int j = 0; j < kTcQ / 2; ++j) {
            const float v = warp_sum(tot[j]);
            if (lane == 0) C.red[warp][j] = v;
        }
        __syncthreads();
        if (!failed && tid < nq) {
            const int hh = tid & 1, j = tid >> 1;
            float t = 0.f;
            for (int w = 0; w < 4; ++w) t += C.red[hh * 4 + w][j];
            const int kk = C.kk[tid];
            P.dir_acc[(long long)kk * 4 + Gp.a] += -(double)P.kappa[kk] * (double)t;
        }
        __syncthreads();
    }
    if (failed) {
        set_status(P.status, Gp.inst, MDX_ERR_TIMEOUT);
        // the MMAs still in flight finish before the tensor memory is released
        if (tid == 0 && issued) {
            long long i = 0;
            while (!bar_try(&C.mma_bar, phase ^ 1u) && ++i < kTcWait) {
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
}

}  // namespace

size_t dir_tc_smem_bytes(int kc, int nmax) { return tc_layout(kc, nmax).end; }

cudaError_t dir_tc_configure(size_t smem) {
    return cudaFuncSetAttribute(dir_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
}

cudaError_t launch_dir_contract(const DirParams &p, int n_units, cudaStream_t s) {
    if (p.groups && p.n_groups > 0 && p.tc_kc > 0) {
        dir_tc_kernel<<<p.n_groups, kTcThreads, p.tc_smem, s>>>(p);
        return cudaGetLastError();
    }
    if (p.groups && p.n_groups > 0) {
        dir_class_kernel<false><<<p.n_groups, kDirThreads, 0, s>>>(p);
        return cudaGetLastError();
    }
    if (n_units <= 0) return cudaSuccess;
    dir_contract_kernel<false><<<n_units, kDirThreads, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_dH_accumulate(const DirParams &p, int n_units, cudaStream_t s) {
    if (p.groups && p.n_groups > 0) {
        dir_class_kernel<true><<<p.n_groups, kDirThreads, 0, s>>>(p);
        return cudaGetLastError();
    }
    if (n_units <= 0) return cudaSuccess;
    dir_contract_kernel<true><<<n_units, kDirThreads, 0, s>>>(p);
    return cudaGetLastError();
}

namespace {

__global__ void dh_symmetrize_kernel(double *dH, const long long *dh_off, const InstDesc *inst,
                                     const int *plates) {
    const InstDesc d = inst[plates[blockIdx.y]];
    double *base = dH + dh_off[plates[blockIdx.y]];
    const long long N = d.N, total = (long long)d.M * N * N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long k = e / (N * N), r = e - k * N * N;
        const long long i = r / N, j = r - i * N;
        if (i >= j) continue;
        double *a = base + k * N * N + i * N + j;
        double *b = base + k * N * N + j * N + i;
        const double m = 0.5 * (*a + *b);
        *a = m;
        *b = m;
    }
}

}  // namespace

cudaError_t launch_dH_symmetrize(double *dH, const long long *dh_off, const InstDesc *inst,
                                 const int *plates, int n_plates, cudaStream_t s) {
    if (n_plates <= 0) return cudaSuccess;
    dh_symmetrize_kernel<<<dim3(64, n_plates), 256, 0, s>>>(dH, dh_off, inst, plates);
    return cudaGetLastError();
}

}  // namespace mdx
