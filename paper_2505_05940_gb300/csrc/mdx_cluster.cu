// Cluster-resident von Karman plates: the forward pass of a few plates at
// the lowest latency per step.
//
// Per step and plate (Sec. 3.1, Eq. 9; Sec. 3.2, Eq. 20), as in the streaming
// plate kernel: u^k = H^k q, eta_k = q . u^k, f = sum_k kappa_k eta_k u^k,
// then the difference-form Stormer-Verlet update and the pickup.  When the
// plate's coupling rows fit the register files of one thread-block cluster,
// nothing of H is read from memory after the launch starts:
//   * one cluster of cs CTAs per plate; CTA r owns the stress modes
//     k = r nkc .. r nkc + nkc - 1 (one slot each) and, per slot, one thread
//     per row of H^k, in class order (row i = class-ordered mode; rows of
//     class a hold the columns of class b = a ^ class(k), the only nonzero
//     block of that row: the symmetry-class layout);
//   * each thread keeps its row (up to RL floats) in registers and forms
//     u_i = H^k_i q_b from the class-ordered q in shared memory;
//   * eta_k: warp sums of q_i u_i, then the slot's warps through shared memory;
//   * the thread's force term kappa_k eta_k u_i goes to a per-slot shared
//     array (double-buffered by step parity); after one cluster barrier,
//     thread m of every CTA gathers f_m from all CTAs' slots over distributed
//     shared memory in a fixed order, so every CTA forms the identical f and
//     applies the identical update to all modes (state in registers of thread
//     m); no second exchange is needed.
// Per step: two CTA barriers and one cluster barrier.  The hardware cluster
// barrier needs no spin loop: every CTA of a cluster is resident, and all run
// the same number of steps.
#include <cuda_runtime.h>

#include "../../include/mdx.h"
#include "mdx_common.cuh"

namespace mdx {

namespace {

constexpr int kEChunk = 256;   // excitation samples staged per shared-memory block

__device__ __forceinline__ uint32_t cta_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Load a float from the shared memory of CTA `rank` of this cluster at the
// address that `local` has in this CTA.
__device__ __forceinline__ float ld_peer(const float *local, uint32_t rank) {
    const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(local));
    uint32_t ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(ra) : "memory");
    return v;
}

__device__ __forceinline__ int pick4c(const int (&v)[4], int a) {
    return a == 0 ? v[0] : (a == 1 ? v[1] : (a == 2 ? v[2] : v[3]));
}

__device__ __forceinline__ int class_of(const InstDesc &d, int i) {
    return (i >= d.ocls[1]) + (i >= d.ocls[2]) + (i >= d.ocls[3]);
}

}  // namespace

template <int RL>
__global__ void __launch_bounds__(512, 1) cluster_kernel(const ClusterParams P) {
    extern __shared__ __align__(16) float sm[];
    const int cs = P.cs, nkc = P.nkc, wk = P.wk;
    const int rowsp = wk * 32;                    // row slots per stress mode
    const int nthreads = blockDim.x;
    const int nwarps = nthreads >> 5;
    float *qc = sm;                               // [4][RL] class blocks of q (padded)
    float *fslot = qc + 4 * RL;                   // [2][nkc][rowsp] force terms
    float *red = fslot + 2 * nkc * rowsp;         // [nwarps] eta partials
    float *redy = red + nwarps;                   // [2][2][32] pickup partials
    float *ebuf = redy + 4 * 32;                  // [2][kEChunk] excitation

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t rank = cta_rank();
    const int plate = P.plates[blockIdx.x / cs];
    const InstDesc d = P.inst[plate];
    const int N = d.N;
    const long long TM = P.total_modes;

    // ---- this thread's coupling row: stress slot, class-ordered row i
    const int kslot = warp / wk;
    const int i = (warp % wk) * 32 + lane;
    const int kl = (int)rank * nkc + kslot;        // internal stress index
    float h[RL];
#pragma unroll
    for (int j = 0; j < RL; ++j) h[j] = 0.f;
    int qoff = 0;                                  // class block of the row's columns
    float kap = 0.f;
    int ia = 0, ip = 0;                            // row class and position in it
    if (kslot < nkc && kl < d.M && i < N) {
        const ClusterK K = P.kinfo[d.k_off + kl];
        ia = class_of(d, i);
        ip = i - pick4c(d.ocls, ia);
        const int b = ia ^ K.c;
        const int nbc = pick4c(d.ncls, b);
        long long sb = 0;
        for (int a2 = 0; a2 < ia; ++a2)
            sb += (long long)pick4c(d.ncls, a2) * K.mc * ((pick4c(d.ncls, a2 ^ K.c) + 3) & ~3);
        const float *row = P.H + K.off + sb + ((long long)ip * K.mc + K.kpos) * ((nbc + 3) & ~3);
#pragma unroll
        for (int j = 0; j < RL; ++j) h[j] = (j < nbc) ? row[j] : 0.f;
        qoff = b * RL;
        kap = P.kappa[d.k_off + kl];
    } else if (i < N) {
        ia = class_of(d, i);
        ip = i - pick4c(d.ocls, ia);
    }
    const bool row_live = (kslot < nkc) && (i < N);

    // ---- per-mode state and coefficients: thread m < N owns class-ordered mode m
    float qhi = 0.f, qlo = 0.f, vhi = 0.f, vlo = 0.f;
    float eps = 0.f, rw2 = 0.f, rw2l = 0.f, r = 0.f, bw = 0.f, cw = 0.f, clo = 0.f;
    int ma = 0, mpos = 0;
    if (tid < N) {
        const long long m = d.mode_off + P.perm[d.perm_off + tid];
        qhi = P.state_io[m];
        qlo = P.state_io[TM + m];
        vhi = P.state_io[2 * TM + m];
        vlo = P.state_io[3 * TM + m];
        eps = P.coef.eps[m];
        rw2 = P.coef.rw2[m];
        rw2l = P.coef.rw2lo[m];
        r = P.coef.r[m];
        bw = P.coef.b[m];
        cw = P.coef.c[m];
        clo = P.coef.clo[m];
        ma = class_of(d, tid);
        mpos = tid - pick4c(d.ocls, ma);
    }
    for (int e = tid; e < 4 * RL; e += nthreads) qc[e] = 0.f;
    __syncthreads();
    if (tid < N) qc[ma * RL + mpos] = qhi;
    const float *exc = P.exc ? P.exc + (long long)plate * P.total_steps : nullptr;
    // every CTA of the cluster is running before any peer access
    cluster_sync_all();

    for (int it = 0; it < P.steps; ++it) {
        const int n = P.n_begin + it;
        const int buf = it & 1;
        if ((it % kEChunk) == 0) {
            float *eb = ebuf + ((it / kEChunk) & 1) * kEChunk;
            for (int e = tid; e < kEChunk; e += nthreads)
                eb[e] = (exc && it + e < P.steps) ? exc[n + e] : 0.f;
        }
        // pickup of the previous step (rank 0 writes the audio sample)
        if (it > 0 && rank == 0 && tid == 0) {
            const float *ry = redy + (buf ^ 1) * 64;
            float y = 0.f, yc = 0.f;
            for (int w = 0; w < (N + 31) / 32; ++w) pickup_merge(y, yc, ry[w], ry[32 + w]);
            y += yc;
            if (P.audio) P.audio[(long long)plate * P.total_steps + n - 1] = y;
            if (!isfinite(y)) set_status(P.status, plate, MDX_ERR_NONFINITE);
        }
        // u_i = H^k_i q_b, from registers and the class-blocked q
        float u = 0.f;
        {
            const float4 *q4 = reinterpret_cast<const float4 *>(qc + qoff);
            float u1 = 0.f;
#pragma unroll
            for (int j = 0; j < RL / 4; j += 2) {
                const float4 a = q4[j];
                u = fmaf(h[4 * j], a.x, u);
                u = fmaf(h[4 * j + 1], a.y, u);
                u = fmaf(h[4 * j + 2], a.z, u);
                u = fmaf(h[4 * j + 3], a.w, u);
                const float4 c = q4[j + 1];
                u1 = fmaf(h[4 * j + 4], c.x, u1);
                u1 = fmaf(h[4 * j + 5], c.y, u1);
                u1 = fmaf(h[4 * j + 6], c.z, u1);
                u1 = fmaf(h[4 * j + 7], c.w, u1);
            }
            u += u1;
        }
        const float qi = (i < N) ? qc[ia * RL + ip] : 0.f;
        const float part = warp_sum(row_live ? qi * u : 0.f);
        if (lane == 0) red[warp] = part;
        __syncthreads();
        if (kslot < nkc) {
            float eta = 0.f;
            for (int w = 0; w < wk; ++w) eta += red[kslot * wk + w];
            fslot[(buf * nkc + kslot) * rowsp + i] = row_live ? kap * eta * u : 0.f;
        }
        cluster_sync_all();
        // f_m from every CTA's slots (same order in every CTA), then the update
        float ys = 0.f, ye = 0.f;
        if (tid < N) {
            float f = 0.f;
            for (int rr = 0; rr < cs; ++rr)
                for (int q = 0; q < nkc; ++q)
                    f += ld_peer(fslot + (buf * nkc + q) * rowsp + tid, (uint32_t)rr);
            const float e = ebuf[((it / kEChunk) & 1) * kEChunk + (it % kEChunk)];
            sv_step(qhi, qlo, vhi, vlo, eps, rw2, rw2l, r, fmaf(bw, e, -f));
            pickup_add(ys, ye, cw, clo, qhi, qlo);
            qc[ma * RL + mpos] = qhi;
        }
        if (warp * 32 < N) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float s2 = __shfl_xor_sync(0xffffffffu, ys, o);
                const float e2 = __shfl_xor_sync(0xffffffffu, ye, o);
                pickup_merge(ys, ye, s2, e2);
            }
            if (lane == 0) {
                redy[buf * 64 + warp] = ys;
                redy[buf * 64 + 32 + warp] = ye;
            }
        }
        __syncthreads();
    }
    if (P.steps > 0 && rank == 0 && tid == 0) {
        const float *ry = redy + ((P.steps - 1) & 1) * 64;
        float y = 0.f, yc = 0.f;
        for (int w = 0; w < (N + 31) / 32; ++w) pickup_merge(y, yc, ry[w], ry[32 + w]);
        y += yc;
        if (P.audio) P.audio[(long long)plate * P.total_steps + P.n_begin + P.steps - 1] = y;
        if (!isfinite(y)) set_status(P.status, plate, MDX_ERR_NONFINITE);
    }
    if (rank == 0 && tid < N) {
        const long long m = d.mode_off + P.perm[d.perm_off + tid];
        P.state_io[m] = qhi;
        P.state_io[TM + m] = qlo;
        P.state_io[2 * TM + m] = vhi;
        P.state_io[3 * TM + m] = vlo;
    }
    // no CTA leaves while a peer may still read its shared memory
    cluster_sync_all();
}

int cluster_row_len(int max_class) {
    if (max_class <= 32) return 32;
    if (max_class <= 64) return 64;
    return 0;
}

int cluster_max_threads(int) { return 512; }

static size_t cluster_smem(int nkc, int wk, int threads, int RL) {
    return sizeof(float) * ((size_t)4 * RL + 2 * (size_t)nkc * wk * 32 + threads / 32 + 128 +
                            2 * kEChunk);
}

template <int RL>
static cudaError_t launch_rl(const ClusterParams &P, int n_plates, cudaStream_t s) {
    const int threads = P.nkc * P.wk * 32;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(n_plates * P.cs));
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = cluster_smem(P.nkc, P.wk, threads, RL);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)P.cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, cluster_kernel<RL>, P);
}

cudaError_t launch_cluster(const ClusterParams &P, int n_plates, int row_len, cudaStream_t s) {
    if (P.steps <= 0 || n_plates <= 0) return cudaSuccess;
    return row_len == 32 ? launch_rl<32>(P, n_plates, s) : launch_rl<64>(P, n_plates, s);
}

// Allows clusters above the portable size where needed and reports how many
// clusters of this shape the device can hold at once (0: not launchable).
cudaError_t cluster_check(int cs, int threads, int row_len, int *max_clusters) {
    *max_clusters = 0;
    const void *fn = row_len == 32 ? reinterpret_cast<const void *>(cluster_kernel<32>)
                                   : reinterpret_cast<const void *>(cluster_kernel<64>);
    // the attribute belongs to the kernel, not to a plan: it is only ever
    // raised, so a plan with a portable cluster never withdraws it from
    // another plan's larger one
    if (cs > 8) {
        const cudaError_t e =
            cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)cs);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = 16384;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(max_clusters, fn, &cfg);
}

}  // namespace mdx
