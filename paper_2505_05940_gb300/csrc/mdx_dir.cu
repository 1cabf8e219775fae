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

#include "mdx_common.cuh"

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

cudaError_t launch_dir_contract(const DirParams &p, int n_units, cudaStream_t s) {
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
