// Von Karman plates: persistent coupling-pass kernel.
//
// Per step and plate (Sec. 3.1, Eq. 9 with C^s_pn = H^n_ps, Sec. 4.3.3):
//   u^k   = H^k q                  (one pass over H, shared by eta and f)
//   eta_k = q . u^k
//   fnl   = sum_k kappa_k eta_k u^k
// followed by the difference-form Stormer-Verlet update (Sec. 3.2, Eq. 20)
// and the pickup.  The reverse sweep evaluates, per step, H^k [q^n, w] with
// w = r a^{n+1} in the same single pass and forms
//   J w = sum_k kappa_k (2 u^k (u^k . w) + eta_k H^k w)  (J symmetric: fnl = grad V).
//
// Execution model (one CTA per SM, cooperative launch so that all CTAs are
// resident):
//   * every CTA owns a list of work items (plate, contiguous stress-mode
//     range); the host splits the (plate, stress mode) units over the CTAs by
//     a min-max partition of their cost (bytes plus a fixed cost per class
//     chunk and per item);
//   * one producer warp streams the CTA's coupling data through a ring of
//     shared-memory stages with TMA bulk copies (cp.async.bulk + mbarrier
//     transaction counts, an L2 evict_last policy on a fraction of the
//     stream).  H does not depend on the state, so the producer runs ahead
//     across step boundaries while the consumers wait for q;
//   * 8 consumer warps.  Class layout (PAR): H^k_ij is nonzero only when
//     class(i) ^ class(j) == class(k), and only those blocks are stored; a
//     chunk of stress modes of one class is four super-blocks [p][k][s], and
//     thread (k, column quad) accumulates the R right-hand sides over the
//     rows.  Dense layout: float4 column strips x row groups over [p][s];
//   * R = 1: forward / recompute; R = 2: reverse sweep ([q^n, w]); R = 3: the
//     fused sweep, the reverse of segment s and the recompute of segment s-1
//     ([q^n, w, q']) in the same pass over H;
//   * plates split over several CTAs exchange partial forces through global
//     memory, with a per-plate monotonic arrival counter (release / acquire,
//     bounded spin); every contributor then applies the identical update so
//     no second exchange is needed.
#include <cuda_runtime.h>

#include "../../include/mdx.h"
#include "mdx_common.cuh"

namespace mdx {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false if the limit was reached or the launch is aborting.
__device__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit,
                          volatile int *abort_flag) {
    for (long long i = 0; i < limit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 1023) == 1023 && *abort_flag) return false;
    }
    return false;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Same copy with an L2 eviction-priority hint (a policy from createpolicy).
__device__ __forceinline__ void bulk_g2s_hint(void *dst, const void *src, uint32_t bytes,
                                              uint64_t *bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
        "[%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

// L2 policy: a `fraction` of the addresses (chosen by the hardware's address
// hash) is kept with evict_last priority, the rest is marked evict_first.
__device__ __forceinline__ uint64_t l2_keep_policy(float fraction) {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.L2::evict_first.b64 %0, %1;"
                 : "=l"(pol)
                 : "f"(fraction));
    return pol;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ float ld_cg(const float *p) {
    float v;
    asm volatile("ld.global.cg.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

// Named barrier of the 256 consumer threads.  Lanes of a warp can arrive here
// after lane-divergent code (one lane spinning on a counter), so the warp is
// reconverged first and the non-aligned barrier form is used.
__device__ __forceinline__ void consumer_bar() {
    __syncwarp();
    asm volatile("barrier.sync 1, %0;" ::"n"(kPlateThreads) : "memory");
}

struct Smem {
    uint64_t *full, *empty;
    float *ring;
    float *U;      // [kChunkK][u_slots][G x Npad <= kUPartFloats] row-group partial sums
    float *red;    // [2][kChunkK][4][kPlateWarps]
    float *red2;   // [2][2][kPlateWarps]
    float *state;  // item state blocks
    int *misc;     // [1] consumer failure flag, [4..5] stages issued, [8..9] stages consumed
};

}  // namespace

// Threads per stress mode in the class layout: the largest power of two
// <= 32 with mc * tpk <= 256.
__host__ __device__ __forceinline__ int par_tpk(int mc) {
    int t = 32;
    while (t > 1 && t * mc > kPlateThreads) t >>= 1;
    return t;
}

// Element of a 4-array by a run-time index without forcing the array into
// local memory (selects only).
__device__ __forceinline__ int pick4(const int (&v)[4], int a) {
    return a == 0 ? v[0] : (a == 1 ? v[1] : (a == 2 ? v[2] : v[3]));
}
__device__ __forceinline__ float comp4(const float4 &v, int e) {
    return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}
__device__ __forceinline__ void fma4(float4 &acc, const float4 &h, float x) {
    acc.x = fmaf(h.x, x, acc.x);
    acc.y = fmaf(h.y, x, acc.y);
    acc.z = fmaf(h.z, x, acc.z);
    acc.w = fmaf(h.w, x, acc.w);
}

// Per-item shared-memory block: the state arrays, then for the item's stress
// modes [k0, k1): (d kappa sum, compensation) pairs and kappa, then the
// per-mode coefficients [ITEM_NCOEF][Npad] and the class permutation [Npad],
// then (owner items of a reverse launch) the gradient sums [GA_N][2][Npad].
template <bool PAR>
__device__ __forceinline__ float *item_kacc(float *st, int Np) {
    return st + (PAR ? ST_NARR_FUSED : ST_NARR) * Np;
}
__device__ __forceinline__ int item_kr4(const PlateItem &it) { return ((it.k1 - it.k0) + 3) & ~3; }
enum ItemCoef : int { IC_EPS = 0, IC_RW2, IC_RW2LO, IC_R, IC_B, IC_C, IC_CLO, ITEM_NCOEF };
template <bool PAR>
__device__ __forceinline__ float *item_coef(float *st, int Np, const PlateItem &it) {
    return item_kacc<PAR>(st, Np) + 3 * item_kr4(it);
}
template <bool PAR>
__device__ __forceinline__ int *item_perm(float *st, int Np, const PlateItem &it) {
    return reinterpret_cast<int *>(item_coef<PAR>(st, Np, it) + ITEM_NCOEF * Np);
}
template <bool PAR>
__device__ __forceinline__ float *item_gacc(float *st, int Np, const PlateItem &it) {
    return item_coef<PAR>(st, Np, it) + (ITEM_NCOEF + 1) * Np;
}

// R: right-hand sides of the H pass (1: forward / recompute; 2: reverse;
// 3: fused reverse + recompute of the previous segment, class layout only).
// PAR: coupling stored in symmetry-class chunks (see ParityChunk).
template <int R, bool PAR>
__global__ void __launch_bounds__(kPlateBlock, 1) plate_kernel(const PlateParams P) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int tid = threadIdx.x;
    const int RING = P.ring_stages;
    const int stage_floats = P.stage_bytes / 4;
    const int it0 = P.cta_item_off[blockIdx.x];
    const int it1 = P.cta_item_off[blockIdx.x + 1];

    // ---- shared memory carve-up (must match plate_smem_bytes on the host)
    Smem S;
    unsigned char *p = smem_raw;
    S.full = reinterpret_cast<uint64_t *>(p);
    S.empty = S.full + RING;
    p += 2 * RING * sizeof(uint64_t);
    S.misc = reinterpret_cast<int *>(p);
    p += 16 * sizeof(int);
    p = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(p) + 127) & ~uintptr_t(127));
    S.ring = reinterpret_cast<float *>(p);
    p += (size_t)RING * P.stage_bytes;
    S.U = reinterpret_cast<float *>(p);
    p += (size_t)P.u_floats * sizeof(float);
    S.red = reinterpret_cast<float *>(p);
    p += (size_t)2 * kChunkK * 4 * kPlateWarps * sizeof(float);
    S.red2 = reinterpret_cast<float *>(p);
    p += (size_t)2 * 2 * kPlateWarps * sizeof(float);
    S.state = reinterpret_cast<float *>(p);

    volatile int *gabort = P.abort_flag;
    constexpr bool FUSED = (R == 3);
    static_assert(!FUSED || PAR, "the fused sweep exists for the class layout only");
    const bool reverse = FUSED || (P.mode == MODE_REVERSE);
    // reverse steps of this launch (the fused sweep may run more recompute steps)
    const int rsteps = FUSED ? P.rev_steps : P.steps;

    if (tid == 0) {
        for (int s = 0; s < RING; ++s) {
            mbar_init(&S.full[s], 1);
            mbar_init(&S.empty[s], kPlateWarps);
        }
        S.misc[0] = 0;
        S.misc[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // ======================================================= producer warp
    if (tid >= kPlateThreads) {
        if (tid == kPlateThreads) {
            long long seq = 0;
            int slot = 0;              // seq % RING and the parity of seq / RING, kept
            uint32_t ring_ph = 0;      // incrementally (no 64-bit division per stage)
            bool ok = true;
            // The coupling data is re-read every step: when it (nearly) fits in
            // L2, keeping a fraction of it resident saves that share of the
            // HBM traffic of every later step.
            const bool hint = P.l2_keep > 0.f;
            const uint64_t pol = hint ? l2_keep_policy(fminf(P.l2_keep, 1.f)) : 0ull;
            auto copy = [&](void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
                if (hint)
                    bulk_g2s_hint(dst, src, bytes, bar, pol);
                else
                    bulk_g2s(dst, src, bytes, bar);
            };
            for (int it = 0; it < P.steps && ok; ++it) {
                for (int ii = it0; ii < it1 && ok; ++ii) {
                    const PlateItem item = P.items[ii];
                    const InstDesc d = P.inst[item.inst];
                    const int rows_per_stage = max(1, stage_floats / d.Npad);
                    const int nmat = 1;   // the direction tensor is contracted per segment (mdx_dir.cu)
                    if constexpr (PAR) {
                        // class chunks: super-blocks a = 0..3, rows of mc * nb4 floats
                        for (int ci = item.chunk0; ci < item.chunk1 && ok; ++ci) {
                            const ParityChunk ch = P.chunks[ci];
                            for (int mat = 0; mat < nmat && ok; ++mat) {
                                const float *base = P.H + (mat == 0 ? ch.off : ch.doff);
                                long long cur = 0;
                                for (int a = 0; a < 4 && ok; ++a) {
                                    const int na = pick4(d.ncls, a), nbc = pick4(d.ncls, a ^ ch.c);
                                    if (na == 0 || nbc == 0) continue;
                                    const int L = ch.mc * ((nbc + 3) & ~3);
                                    const int rps = max(1, stage_floats / L);
                                    for (int p0 = 0; p0 < na; p0 += rps) {
                                        const int nr = min(rps, na - p0);
                                        const int s = slot;
                                        const uint32_t ph = ring_ph;
                                        if (!mbar_wait(&S.empty[s], ph ^ 1u, P.wait_limit, gabort)) {
                                            ok = false;
                                            break;
                                        }
                                        const uint32_t bytes = (uint32_t)nr * L * 4u;
                                        mbar_arrive_expect_tx(&S.full[s], bytes);
                                        copy(S.ring + (size_t)s * stage_floats, base + cur, bytes,
                                             &S.full[s]);
                                        cur += (long long)nr * L;
                                        ++seq;
                                        if (++slot == RING) {
                                            slot = 0;
                                            ring_ph ^= 1u;
                                        }
                                    }
                                }
                            }
                        }
                    } else {
                    for (int k = item.k0; k < item.k1 && ok; ++k) {
                        for (int mat = 0; mat < nmat && ok; ++mat) {
                            const float *base = (mat == 0 ? P.H + d.H_off : P.dH + d.dH_off) +
                                                (long long)k * d.N * d.Npad;
                            for (int p0 = 0; p0 < d.N; p0 += rows_per_stage) {
                                const int nr = min(rows_per_stage, d.N - p0);
                                const int s = slot;
                                const uint32_t ph = ring_ph;
                                if (!mbar_wait(&S.empty[s], ph ^ 1u, P.wait_limit, gabort)) {
                                    ok = false;
                                    break;
                                }
                                const uint32_t bytes = (uint32_t)nr * d.Npad * 4u;
                                mbar_arrive_expect_tx(&S.full[s], bytes);
                                copy(S.ring + (size_t)s * stage_floats,
                                     base + (long long)p0 * d.Npad, bytes, &S.full[s]);
                                ++seq;
                                if (++slot == RING) {
                                    slot = 0;
                                    ring_ph ^= 1u;
                                }
                            }
                        }
                    }
                    }
                }
            }
            if (!ok) atomicExch((int *)gabort, 1);
            *reinterpret_cast<volatile long long *>(&S.misc[4]) = seq;
        }
        __syncwarp();
        __syncthreads();
        return;
    }

    // ======================================================= consumer warps
    const int warp = tid >> 5, lane = tid & 31;
    const long long TM = P.total_modes;
    int slot = 0;              // ring slot of the next stage to consume
    uint32_t ring_ph = 0;      // its mbarrier phase parity
    int chunk_parity = 0;
    int red2_parity = 0;
    // A failed wait is recorded in fail / S.misc[1] but the thread keeps the
    // common control flow (same barriers) until the end of the step, where all
    // consumer threads read S.misc[1] after a barrier and leave together.
    bool fail = false;
    bool ok = true;

    // ---- load per-item state
    for (int ii = it0; ii < it1; ++ii) {
        const PlateItem item = P.items[ii];
        const InstDesc d = P.inst[item.inst];
        float *st = S.state + item.smem_state;
        const float *src;
        long long stride;
        if (!reverse) {
            src = (P.mode == MODE_RECOMPUTE)
                      ? P.ckpt + (long long)(P.n_begin / P.ckpt_K) * kStateArrays * TM
                      : P.state_io;
            stride = TM;
        } else {
            src = P.adj;
            stride = TM;
        }
        for (int s = tid; s < d.Npad; s += kPlateThreads) {
            const bool in = s < d.N;
            st[ST_QHI * d.Npad + s] = in ? src[d.mode_off + s] : 0.f;
            st[ST_QLO * d.Npad + s] = in ? src[stride + d.mode_off + s] : 0.f;
            st[ST_V * d.Npad + s] = in ? src[2 * stride + d.mode_off + s] : 0.f;
            st[ST_VLO * d.Npad + s] = (in && !reverse) ? src[3 * stride + d.mode_off + s] : 0.f;
            if constexpr (FUSED) {
                const float *ck = P.ckpt + (long long)(P.rec_begin / P.ckpt_K) * kStateArrays * TM;
                st[ST_RQHI * d.Npad + s] = in ? ck[d.mode_off + s] : 0.f;
                st[ST_RQLO * d.Npad + s] = in ? ck[TM + d.mode_off + s] : 0.f;
                st[ST_RV * d.Npad + s] = in ? ck[2 * TM + d.mode_off + s] : 0.f;
                st[ST_RVLO * d.Npad + s] = in ? ck[3 * TM + d.mode_off + s] : 0.f;
            }
        }
        // kappa and the d kappa sums of the item's stress modes; the owner's
        // gradient sums (reverse): kept in shared memory for the whole launch
        float *kac = item_kacc<PAR>(st, d.Npad);
        const int kr4 = item_kr4(item), nk = item.k1 - item.k0;
        for (int q = tid; q < kr4; q += kPlateThreads) {
            const bool in = q < nk;
            kac[2 * kr4 + q] = in ? P.kappa[d.k_off + item.k0 + q] : 0.f;
            kac[2 * q] = (in && reverse) ? P.kacc[2 * (d.k_off + item.k0 + q)] : 0.f;
            kac[2 * q + 1] = (in && reverse) ? P.kacc[2 * (d.k_off + item.k0 + q) + 1] : 0.f;
        }
        if (item.cache) {
            float *cf = item_coef<PAR>(st, d.Npad, item);
            int *pm = item_perm<PAR>(st, d.Npad, item);
            for (int s = tid; s < d.Npad; s += kPlateThreads) {
                const bool in = s < d.N;
                const long long m = d.mode_off + s;
                cf[IC_EPS * d.Npad + s] = in ? P.coef.eps[m] : 0.f;
                cf[IC_RW2 * d.Npad + s] = in ? P.coef.rw2[m] : 0.f;
                cf[IC_RW2LO * d.Npad + s] = in ? P.coef.rw2lo[m] : 0.f;
                cf[IC_R * d.Npad + s] = in ? P.coef.r[m] : 0.f;
                cf[IC_B * d.Npad + s] = in ? P.coef.b[m] : 0.f;
                cf[IC_C * d.Npad + s] = in ? P.coef.c[m] : 0.f;
                cf[IC_CLO * d.Npad + s] = in ? P.coef.clo[m] : 0.f;
                pm[s] = (PAR && in) ? P.perm[d.perm_off + s] : s;
            }
        }
        if (reverse && item.owner && item.cache) {
            float *gac = item_gacc<PAR>(st, d.Npad, item);
            for (int e = tid; e < 2 * GA_N * d.Npad; e += kPlateThreads) {
                const int row = e / d.Npad, s = e - row * d.Npad;
                gac[e] = (s < d.N) ? P.gacc[(long long)row * TM + d.mode_off + s] : 0.f;
            }
        }
    }
    consumer_bar();

    for (int it = 0; it < P.steps; ++it) {
        // global step index: forward counts up, reverse counts down
        const int t_loc = reverse ? (rsteps - 1 - it) : it;
        const int n = P.n_begin + t_loc;
        const bool rev_on = it < rsteps;   // false only in the tail of a fused launch

        // -------- pre-pass: right-hand sides, checkpoints, stored states
        for (int ii = it0; ii < it1; ++ii) {
            const PlateItem item = P.items[ii];
            const InstDesc d = P.inst[item.inst];
            float *st = S.state + item.smem_state;
            const int Np = d.Npad;
            for (int s = tid; s < Np; s += kPlateThreads) {
                const bool in = s < d.N;
                const long long m = d.mode_off + s;
                if (!reverse) {
                    if (in && item.owner) {
                        if (P.mode == MODE_FORWARD && P.ckpt && (n % P.ckpt_K) == 0) {
                            float *ck = P.ckpt + (long long)(n / P.ckpt_K) * kStateArrays * TM;
                            ck[m] = st[ST_QHI * Np + s];
                            ck[TM + m] = st[ST_QLO * Np + s];
                            ck[2 * TM + m] = st[ST_V * Np + s];
                            ck[3 * TM + m] = st[ST_VLO * Np + s];
                        }
                        if (P.mode == MODE_RECOMPUTE) {
                            P.seg_q[(long long)t_loc * TM + m] = st[ST_QHI * Np + s];
                            P.seg_v[(long long)t_loc * TM + m] = st[ST_V * Np + s];
                        }
                    }
                    st[ST_FLOC * Np + s] = 0.f;
                } else {
                    const bool live = in && rev_on;
                    const float qn = live ? P.seg_q[(long long)t_loc * TM + m] : 0.f;
                    const float rr = item.cache ? item_coef<PAR>(st, Np, item)[IC_R * Np + s]
                                                : (live ? P.coef.r[m] : 0.f);
                    const float wv = live ? rr * st[ST_QHI * Np + s] : 0.f;
                    st[ST_SRC0 * Np + s] = qn;
                    st[ST_SRC1 * Np + s] = wv;
                    if (live && item.owner && P.seg_w) P.seg_w[(long long)t_loc * TM + m] = wv;
                    st[ST_FLOC * Np + s] = 0.f;
                    st[ST_FLOC2 * Np + s] = 0.f;
                    if constexpr (FUSED) {
                        if (in && item.owner) {
                            P.rseg_q[(long long)it * TM + m] = st[ST_RQHI * Np + s];
                            P.rseg_v[(long long)it * TM + m] = st[ST_RV * Np + s];
                        }
                        st[ST_RFLOC * Np + s] = 0.f;
                    }
                }
            }
        }
        consumer_bar();
        if constexpr (PAR) {
            // right-hand sides in class order
            for (int ii = it0; ii < it1; ++ii) {
                const PlateItem item = P.items[ii];
                const InstDesc d = P.inst[item.inst];
                float *st = S.state + item.smem_state;
                const int Np = d.Npad;
                const float *q = reverse ? st + ST_SRC0 * Np : st + ST_QHI * Np;
                for (int mp = tid; mp < d.N; mp += kPlateThreads) {
                    const int su = item.cache ? item_perm<PAR>(st, Np, item)[mp] : P.perm[d.perm_off + mp];
                    st[ST_QP * Np + mp] = q[su];
                    if (reverse) st[ST_WP * Np + mp] = st[ST_SRC1 * Np + su];
                    if constexpr (FUSED) st[ST_RQP * Np + mp] = st[ST_RQHI * Np + su];
                }
            }
            consumer_bar();
        }

        // -------- phase A: coupling pass over this CTA's items
        // Thread layout over a stage of rows (p) x columns (s) of H^k: thread
        // (g, c) owns the float4 column strip c and the g-th contiguous block
        // of the stage's rows.  Partial sums of the G row groups are combined
        // through shared memory once per chunk of kChunkK stress modes.
        for (int ii = it0; ii < it1; ++ii) {
            const PlateItem item = P.items[ii];
            const InstDesc d = P.inst[item.inst];
            float *st = S.state + item.smem_state;
            const int Np = d.Npad;
            const int ncol4 = Np >> 2;
            const int G = max(1, min(kPlateThreads / ncol4, 32));
            const int g = tid / ncol4, c4 = tid - (tid / ncol4) * ncol4;
            const bool active = g < G;
            const int rows_per_stage = max(1, stage_floats / Np);
            const int nmat = 1;   // the direction tensor is contracted per segment (mdx_dir.cu)
            const float *src0 = reverse ? st + ST_SRC0 * Np : st + ST_QHI * Np;
            const float *src1 = st + ST_SRC1 * Np;
            const int spt = (Np + kPlateThreads - 1) / kPlateThreads;
            if constexpr (PAR) {
                // u slots per stress mode: H q, H w (reverse), H q' (fused recompute)
                constexpr int US = FUSED ? 3 : 2;
                const float *qp = st + ST_QP * Np;
                const float *wp = st + ST_WP * Np;
                const float *rp = st + (FUSED ? ST_RQP : ST_QP) * Np;
                float *red = S.red;
                for (int ci = item.chunk0; ci < item.chunk1; ++ci) {
                    const ParityChunk ch = P.chunks[ci];
                    const int mc = ch.mc;
                    const int tpk = par_tpk(mc);
                    const int kl = tid / tpk, c4 = tid - (tid / tpk) * tpk;
                    const bool kact = kl < mc;
                    float dsum[3] = {0.f, 0.f, 0.f};
                    for (int a = 0; a < 4; ++a) {
                        const int bcl = a ^ ch.c;
                        const int na = pick4(d.ncls, a), nbc = pick4(d.ncls, bcl);
                        if (na == 0 || nbc == 0) continue;
                        const int oa = pick4(d.ocls, a), ob = pick4(d.ocls, bcl);
                        const int nb4 = (nbc + 3) & ~3, nq = nb4 >> 2;
                        const int L = mc * nb4;
                        const int rps = max(1, stage_floats / L);
                        // each thread owns column quads qi0 = c4 and qi1 = c4 + tpk
                        const int qi0 = c4, qi1 = c4 + tpk;
                        const bool h0 = kact && qi0 < nq, h1 = kact && qi1 < nq;
                        constexpr bool two = R > 1;
                        float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0, b0 = a0, b1 = a0;
                        float4 c0 = a0, c1 = a0;
                        for (int p0 = 0; p0 < na; p0 += rps) {
                            const int nr = min(rps, na - p0);
                            const int s = slot;
                            const uint32_t ph = ring_ph;
                            if (!fail && !mbar_wait(&S.full[s], ph, P.wait_limit, gabort)) {
                                fail = true;
                                *reinterpret_cast<volatile int *>(&S.misc[1]) = 1;
                                atomicExch((int *)gabort, 1);
                            }
                            if (h0) {
                                const float *row = S.ring + (size_t)s * stage_floats + kl * nb4 + 4 * qi0;
                                const float *xs = qp + oa + p0;
                                const float *ys = wp + oa + p0;
                                const float *zs = rp + oa + p0;
                                if (h1) {
#pragma unroll 2
                                    for (int r = 0; r < nr; ++r) {
                                        const float4 hA = *reinterpret_cast<const float4 *>(row + (size_t)r * L);
                                        const float4 hB = *reinterpret_cast<const float4 *>(row + (size_t)r * L + 4 * tpk);
                                        const float x = xs[r];
                                        fma4(a0, hA, x);
                                        fma4(b0, hB, x);
                                        if (two) {
                                            const float y = ys[r];
                                            fma4(a1, hA, y);
                                            fma4(b1, hB, y);
                                        }
                                        if constexpr (FUSED) {
                                            const float z = zs[r];
                                            fma4(c0, hA, z);
                                            fma4(c1, hB, z);
                                        }
                                    }
                                } else {
                                    // one column quad: two independent chains over
                                    // alternate rows (odd rows accumulate in the
                                    // second quad's registers, folded in below)
                                    int r = 0;
#pragma unroll 2
                                    for (; r + 1 < nr; r += 2) {
                                        const float4 hA = *reinterpret_cast<const float4 *>(row + (size_t)r * L);
                                        const float4 hB = *reinterpret_cast<const float4 *>(row + (size_t)(r + 1) * L);
                                        fma4(a0, hA, xs[r]);
                                        fma4(b0, hB, xs[r + 1]);
                                        if (two) {
                                            fma4(a1, hA, ys[r]);
                                            fma4(b1, hB, ys[r + 1]);
                                        }
                                        if constexpr (FUSED) {
                                            fma4(c0, hA, zs[r]);
                                            fma4(c1, hB, zs[r + 1]);
                                        }
                                    }
                                    if (r < nr) {
                                        const float4 hA = *reinterpret_cast<const float4 *>(row + (size_t)r * L);
                                        fma4(a0, hA, xs[r]);
                                        if (two) fma4(a1, hA, ys[r]);
                                        if constexpr (FUSED) fma4(c0, hA, zs[r]);
                                    }
                                }
                            }
                            __syncwarp();
                            if (lane == 0) mbar_arrive(&S.empty[s]);
                            if (++slot == RING) {
                                slot = 0;
                                ring_ph ^= 1u;
                            }
                        }
                        if (h0 && !h1) {
                            a0 = make_float4(a0.x + b0.x, a0.y + b0.y, a0.z + b0.z, a0.w + b0.w);
                            a1 = make_float4(a1.x + b1.x, a1.y + b1.y, a1.z + b1.z, a1.w + b1.w);
                            c0 = make_float4(c0.x + c1.x, c0.y + c1.y, c0.z + c1.z, c0.w + c1.w);
                        }
                        // this super-block completes u^k (and z^k, u'^k) on the columns of class b
#pragma unroll
                        for (int half = 0; half < 2; ++half) {
                            const bool has = half == 0 ? h0 : h1;
                            if (!has) continue;
                            const int qi = half == 0 ? qi0 : qi1;
                            const float4 va = half == 0 ? a0 : b0;
                            const float4 vb = half == 0 ? a1 : b1;
                            const float4 vc = half == 0 ? c0 : c1;
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const int cs = 4 * qi + e;
                                if (cs >= nbc) break;
                                const int mp = ob + cs;
                                const float v0 = comp4(va, e);
                                S.U[((size_t)kl * US + 0) * P.npad_max + mp] = v0;
                                dsum[0] = fmaf(qp[mp], v0, dsum[0]);
                                if (R > 1) {
                                    S.U[((size_t)kl * US + 1) * P.npad_max + mp] = comp4(vb, e);
                                    dsum[1] = fmaf(wp[mp], v0, dsum[1]);
                                }
                                if constexpr (FUSED) {
                                    const float v2 = comp4(vc, e);
                                    S.U[((size_t)kl * US + 2) * P.npad_max + mp] = v2;
                                    dsum[2] = fmaf(rp[mp], v2, dsum[2]);
                                }
                            }
                        }
                    }
                    // dot products of each stress mode: reduce over its tpk lanes
                    constexpr int ND = FUSED ? 3 : (R > 1 ? 2 : 1);
#pragma unroll
                    for (int dd = 0; dd < ND; ++dd) {
                        float v = dsum[dd];
                        for (int o = tpk >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                        if (kact && c4 == 0) red[kl * 4 + dd] = v;
                    }
                    // slot 3: kappa of the stress mode, so the force loop reads shared memory only
                    float *kac = item_kacc<PAR>(st, Np);
                    const int kr4 = item_kr4(item);
                    if (kact && c4 == 0) red[kl * 4 + 3] = kac[2 * kr4 + ch.kl0 + kl - item.k0];
                    consumer_bar();
                    // forces, per mode in class order (each thread owns distinct modes)
                    const int *pmc = item.cache ? item_perm<PAR>(st, Np, item) : P.perm + d.perm_off;
                    for (int mp = tid; mp < d.N; mp += kPlateThreads) {
                        const int su = pmc[mp];
                        float fa = 0.f, fb = 0.f, fr = 0.f;
#pragma unroll 4
                        for (int q = 0; q < mc; ++q) {
                            const float kap = red[q * 4 + 3];
                            const float eta = red[q * 4 + 0];
                            const float u = S.U[((size_t)q * US + 0) * P.npad_max + mp];
                            if (!reverse) {
                                fa = fmaf(kap * eta, u, fa);
                            } else {
                                const float z = S.U[((size_t)q * US + 1) * P.npad_max + mp];
                                fb = fmaf(kap * eta, u, fb);
                                fa = fmaf(kap, fmaf(2.f * red[q * 4 + 1], u, eta * z), fa);
                            }
                            if constexpr (FUSED) {
                                const float u2 = S.U[((size_t)q * US + 2) * P.npad_max + mp];
                                fr = fmaf(kap * red[q * 4 + 2], u2, fr);
                            }
                        }
                        st[ST_FLOC * Np + su] += fa;
                        if (reverse) st[ST_FLOC2 * Np + su] += fb;
                        if constexpr (FUSED) st[ST_RFLOC * Np + su] += fr;
                    }
                    if (reverse && rev_on && tid < mc) {
                        // one thread per stress mode of the chunk; the sums stay in
                        // shared memory until the end of the launch
                        const int q = tid;
                        const long long kk = d.k_off + ch.kl0 + q;
                        const float eta = red[q * 4 + 0], xi = red[q * 4 + 1];
                        float *ka = kac + 2 * (ch.kl0 + q - item.k0);
                        float s0 = ka[0], c0 = ka[1];
                        kahan_add(s0, c0, -eta * xi);
                        ka[0] = s0;
                        ka[1] = c0;
                        if ((d.has_dir || P.xe_all) && P.xe) {
                            P.xe[((long long)t_loc * 2 + 0) * P.total_k + kk] = xi;
                            P.xe[((long long)t_loc * 2 + 1) * P.total_k + kk] = eta;
                        }
                    }
                    consumer_bar();
                }
            } else {
            for (int kc = item.k0; kc < item.k1; kc += kChunkK) {
                const int nk = min(kChunkK, item.k1 - kc);
                float *red = S.red + chunk_parity * (kChunkK * 4 * kPlateWarps);
                for (int kk = 0; kk < nk; ++kk) {
                    for (int mat = 0; mat < nmat; ++mat) {
                        float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f);
                        float4 a1 = make_float4(0.f, 0.f, 0.f, 0.f);
                        for (int p0 = 0; p0 < d.N; p0 += rows_per_stage) {
                            const int nr = min(rows_per_stage, d.N - p0);
                            const int s = slot;
                            const uint32_t ph = ring_ph;
                            if (!fail && !mbar_wait(&S.full[s], ph, P.wait_limit, gabort)) {
                                fail = true;
                                *reinterpret_cast<volatile int *>(&S.misc[1]) = 1;
                                atomicExch((int *)gabort, 1);
                            }
                            if (active) {
                                const int rpg = (nr + G - 1) / G;
                                const int r0 = g * rpg;
                                const int r1 = min(nr, r0 + rpg);
                                const float *stg = S.ring + (size_t)s * stage_floats + 4 * c4;
                                if (mat == 0 && R > 1) {
#pragma unroll 4
                                    for (int r = r0; r < r1; ++r) {
                                        const float4 h = *reinterpret_cast<const float4 *>(stg + (size_t)r * Np);
                                        const float x = src0[p0 + r], y = src1[p0 + r];
                                        a0.x = fmaf(h.x, x, a0.x); a0.y = fmaf(h.y, x, a0.y);
                                        a0.z = fmaf(h.z, x, a0.z); a0.w = fmaf(h.w, x, a0.w);
                                        a1.x = fmaf(h.x, y, a1.x); a1.y = fmaf(h.y, y, a1.y);
                                        a1.z = fmaf(h.z, y, a1.z); a1.w = fmaf(h.w, y, a1.w);
                                    }
                                } else {
                                    // two independent chains over alternate rows
#pragma unroll 4
                                    for (int r = r0; r < r1; r += 2) {
                                        const float4 h = *reinterpret_cast<const float4 *>(stg + (size_t)r * Np);
                                        const float x = src0[p0 + r];
                                        a0.x = fmaf(h.x, x, a0.x); a0.y = fmaf(h.y, x, a0.y);
                                        a0.z = fmaf(h.z, x, a0.z); a0.w = fmaf(h.w, x, a0.w);
                                        if (r + 1 < r1) {
                                            const float4 h2 = *reinterpret_cast<const float4 *>(stg + (size_t)(r + 1) * Np);
                                            const float x2 = src0[p0 + r + 1];
                                            a1.x = fmaf(h2.x, x2, a1.x); a1.y = fmaf(h2.y, x2, a1.y);
                                            a1.z = fmaf(h2.z, x2, a1.z); a1.w = fmaf(h2.w, x2, a1.w);
                                        }
                                    }
                                }
                            }
                            __syncwarp();
                            if (lane == 0) mbar_arrive(&S.empty[s]);
                            if (++slot == RING) {
                                slot = 0;
                                ring_ph ^= 1u;
                            }
                        }
                        if (active) {
                            // slot 0: H q, slot 1: H w (reverse)
                            if (mat == 0 && R > 1) {
                                float *u0 = S.U + ((size_t)(kk * P.u_slots + 0) * G + g) * Np + 4 * c4;
                                float *u1 = S.U + ((size_t)(kk * P.u_slots + 1) * G + g) * Np + 4 * c4;
                                *reinterpret_cast<float4 *>(u0) = a0;
                                *reinterpret_cast<float4 *>(u1) = a1;
                            } else {
                                const float4 sum = make_float4(a0.x + a1.x, a0.y + a1.y,
                                                               a0.z + a1.z, a0.w + a1.w);
                                float *u0 = S.U + ((size_t)(kk * P.u_slots + (mat == 0 ? 0 : 2)) * G + g) * Np + 4 * c4;
                                *reinterpret_cast<float4 *>(u0) = sum;
                            }
                        }
                    }
                }
                consumer_bar();
                // combine the row groups: u (H q), z (H w) for own modes
                float uu[kChunkK][kMaxSpt], zz[kChunkK][kMaxSpt];
#pragma unroll
                for (int kk = 0; kk < kChunkK; ++kk) {
                    float dsum[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int j = 0; j < kMaxSpt; ++j) {
                        uu[kk][j] = 0.f;
                        zz[kk][j] = 0.f;
                        const int sj = tid + j * kPlateThreads;
                        if (kk < nk && j < spt && sj < Np) {
                            float u = 0.f, z = 0.f, t = 0.f;
                            for (int gg = 0; gg < G; ++gg) {
                                u += S.U[((size_t)(kk * P.u_slots + 0) * G + gg) * Np + sj];
                                if (R > 1) z += S.U[((size_t)(kk * P.u_slots + 1) * G + gg) * Np + sj];
                                if (nmat > 1) t += S.U[((size_t)(kk * P.u_slots + 2) * G + gg) * Np + sj];
                            }
                            uu[kk][j] = u;
                            zz[kk][j] = z;
                            const float qs = src0[sj];
                            dsum[0] = fmaf(qs, u, dsum[0]);
                            if (R > 1) {
                                const float ws = src1[sj];
                                dsum[1] = fmaf(ws, u, dsum[1]);
                                dsum[2] = fmaf(qs, t, dsum[2]);
                                dsum[3] = fmaf(ws, t, dsum[3]);
                            }
                        }
                    }
                    if (kk < nk) {
#pragma unroll
                        for (int dd = 0; dd < 4; ++dd) {
                            const float v = warp_sum(dsum[dd]);
                            if (lane == 0) red[(kk * 4 + dd) * kPlateWarps + warp] = v;
                        }
                    }
                }
                consumer_bar();
                // chunk epilogue: reduce the dot products, accumulate the forces
#pragma unroll
                for (int kk = 0; kk < kChunkK; ++kk) {
                    if (kk >= nk) break;
                    const int k = kc + kk;
                    float dv[4];
#pragma unroll
                    for (int dd = 0; dd < 4; ++dd) {
                        float a = 0.f;
#pragma unroll
                        for (int w = 0; w < kPlateWarps; ++w) a += red[(kk * 4 + dd) * kPlateWarps + w];
                        dv[dd] = a;
                    }
                    float *kac = item_kacc<PAR>(st, Np);
                    const int kr4 = item_kr4(item);
                    const float kap = kac[2 * kr4 + k - item.k0];
#pragma unroll
                    for (int j = 0; j < kMaxSpt; ++j) {
                        const int sj = tid + j * kPlateThreads;
                        if (j < spt && sj < Np) {
                            const float u = uu[kk][j];
                            if (!reverse) {
                                st[ST_FLOC * Np + sj] = fmaf(kap * dv[0], u, st[ST_FLOC * Np + sj]);
                            } else {
                                const float z = zz[kk][j];
                                // f = sum kappa eta u ; J w = sum kappa (2 xi u + eta z)
                                st[ST_FLOC2 * Np + sj] = fmaf(kap * dv[0], u, st[ST_FLOC2 * Np + sj]);
                                st[ST_FLOC * Np + sj] =
                                    fmaf(kap, fmaf(2.f * dv[1], u, dv[0] * z), st[ST_FLOC * Np + sj]);
                            }
                        }
                    }
                    if (reverse && tid == 0) {
                        // d kappa_k -= eta xi ; directional derivative
                        float *ka = kac + 2 * (k - item.k0);
                        float s0 = ka[0], c0 = ka[1];
                        kahan_add(s0, c0, -dv[0] * dv[1]);
                        ka[0] = s0;
                        ka[1] = c0;
                        if ((d.has_dir || P.xe_all) && P.xe) {
                            P.xe[((long long)t_loc * 2 + 0) * P.total_k + d.k_off + k] = dv[1];
                            P.xe[((long long)t_loc * 2 + 1) * P.total_k + d.k_off + k] = dv[0];
                        }
                    }
                }
                chunk_parity ^= 1;
            }
            }
            // publish partial forces of a shared plate
            if (d.n_contrib > 1) {
                const long long slot_base = (long long)(it & 1) * P.part_stride +
                                            d.part_off + (long long)item.slot * 3 * Np;
                for (int s = tid; s < Np; s += kPlateThreads) {
                    P.part[slot_base + s] = st[ST_FLOC * Np + s];
                    if (reverse) P.part[slot_base + Np + s] = st[ST_FLOC2 * Np + s];
                    if constexpr (FUSED) P.part[slot_base + 2 * Np + s] = st[ST_RFLOC * Np + s];
                }
                consumer_bar();
                if (tid == 0 && !((P.debug_flags & 1) && item.slot == 1)) {
                    __threadfence();
                    atomicAdd(P.counters + item.inst, 1u);
                }
            }
        }

        // -------- phase B: gather forces and update every item's state
        for (int ii = it0; ii < it1; ++ii) {
            const PlateItem item = P.items[ii];
            const InstDesc d = P.inst[item.inst];
            float *st = S.state + item.smem_state;
            const int Np = d.Npad;
            if (d.n_contrib > 1) {
                if (tid == 0 && !fail) {
                    const unsigned target = (unsigned)(it + 1) * (unsigned)d.n_contrib;
                    long long spins = 0;
                    while (ld_acquire_u32(P.counters + item.inst) < target) {
                        if (++spins > P.wait_limit || ((spins & 255) == 0 && *gabort)) {
                            atomicExch((int *)gabort, 1);
                            set_status(P.status, item.inst, MDX_ERR_TIMEOUT);
                            fail = true;
                            *reinterpret_cast<volatile int *>(&S.misc[1]) = 1;
                            break;
                        }
                        __nanosleep(64);
                    }
                }
                consumer_bar();
            }
            const float e = (P.exc && rev_on) ? P.exc[(long long)item.inst * P.total_steps + n] : 0.f;
            const float e_rec =
                (FUSED && P.exc) ? P.exc[(long long)item.inst * P.total_steps + P.rec_begin + it] : 0.f;
            float ys = 0.f, ye = 0.f;   // compensated pickup (owner)
            for (int s = tid; s < d.N; s += kPlateThreads) {
                const long long m = d.mode_off + s;
                // every global load of the mode's update is issued before the first
                // result is used, so their latencies overlap: the stored states and
                // targets of the reverse sweep, then the partial forces of the other
                // contributors in batches (summed in contributor order)
                float vn = 0.f, qn1 = 0.f, ybn = 0.f, ybm = 0.f;
                if (reverse && rev_on) {
                    if (item.owner) {
                        vn = P.seg_v[(long long)t_loc * TM + m];
                        qn1 = P.seg_q[(long long)(t_loc + 1) * TM + m];
                        ybn = P.ybar[(long long)item.inst * P.total_steps + n];
                    }
                    ybm = (n >= 1) ? P.ybar[(long long)item.inst * P.total_steps + n - 1] : 0.f;
                }
                float fA, fB = 0.f, fR = 0.f;
                if (d.n_contrib > 1) {
                    const float *pb = P.part + (long long)(it & 1) * P.part_stride + d.part_off + s;
                    fA = 0.f;
                    constexpr int kXB = 4;
                    for (int c0 = 0; c0 < d.n_contrib; c0 += kXB) {
                        float xa[kXB], xb[kXB], xr[kXB];
#pragma unroll
                        for (int j = 0; j < kXB; ++j) {
                            xa[j] = xb[j] = xr[j] = 0.f;
                            if (c0 + j < d.n_contrib) {
                                const float *q = pb + (long long)(c0 + j) * 3 * Np;
                                xa[j] = ld_cg(q);
                                if (reverse) xb[j] = ld_cg(q + Np);
                                if constexpr (FUSED) xr[j] = ld_cg(q + 2 * Np);
                            }
                        }
#pragma unroll
                        for (int j = 0; j < kXB; ++j) {
                            if (c0 + j >= d.n_contrib) break;
                            fA += xa[j];
                            if (reverse) fB += xb[j];
                            if constexpr (FUSED) fR += xr[j];
                        }
                    }
                } else {
                    fA = st[ST_FLOC * Np + s];
                    if (reverse) fB = st[ST_FLOC2 * Np + s];
                    if constexpr (FUSED) fR = st[ST_RFLOC * Np + s];
                }
                // cached: [coef][Np] in shared memory; else the plan's global arrays
                const float *cf = item.cache ? item_coef<PAR>(st, Np, item) : nullptr;
                const float eps = cf ? cf[IC_EPS * Np + s] : P.coef.eps[m];
                const float rw2 = cf ? cf[IC_RW2 * Np + s] : P.coef.rw2[m];
                const float r = cf ? cf[IC_R * Np + s] : P.coef.r[m];
                const float rw2l = cf ? cf[IC_RW2LO * Np + s] : P.coef.rw2lo[m];
                const float b = cf ? cf[IC_B * Np + s] : P.coef.b[m];
                const float c = cf ? cf[IC_C * Np + s] : P.coef.c[m];
                const float clo = cf ? cf[IC_CLO * Np + s] : P.coef.clo[m];
                float x0 = st[ST_QHI * Np + s], x1 = st[ST_QLO * Np + s], x2 = st[ST_V * Np + s];
                float x3 = st[ST_VLO * Np + s];
                if (!reverse) {
                    sv_step(x0, x1, x2, x3, eps, rw2, rw2l, r, fmaf(b, e, -fA));
                    pickup_add(ys, ye, c, clo, x0, x1);
                } else if (rev_on) {
                    // fA = J w (summed), fB = fnl(q^n)
                    if (item.owner) {
                        const float a = x0;
                        const float qn = st[ST_SRC0 * Np + s];
                        // the owner's gradient sums: shared memory when cached
                        float *g = item.cache ? item_gacc<PAR>(st, Np, item) + s : P.gacc + m;
                        const long long gst = item.cache ? (long long)Np : TM;
                        float gsum, gcmp;
#define MDX_ACC(IDX, X)                                                    \
    gsum = g[(2 * (IDX)) * gst];                                           \
    gcmp = g[(2 * (IDX) + 1) * gst];                                       \
    kahan_add(gsum, gcmp, (X));                                            \
    g[(2 * (IDX)) * gst] = gsum;                                           \
    g[(2 * (IDX) + 1) * gst] = gcmp;
                        MDX_ACC(GA_A, a * qn)
                        MDX_ACC(GA_V, a * vn)
                        MDX_ACC(GA_F, a * fmaf(b, e, -fB))
                        MDX_ACC(GA_E, a * e)
                        MDX_ACC(GA_C, ybn * qn1)
#undef MDX_ACC
                    }
                    adj_step(x0, x1, x2, eps, rw2, fA, c * ybm);
                }
                st[ST_QHI * Np + s] = x0;
                st[ST_QLO * Np + s] = x1;
                st[ST_V * Np + s] = x2;
                st[ST_VLO * Np + s] = x3;
                if constexpr (FUSED) {
                    // recompute of the previous segment: the forward update at q'
                    float y0 = st[ST_RQHI * Np + s], y1 = st[ST_RQLO * Np + s];
                    float y2 = st[ST_RV * Np + s], y3 = st[ST_RVLO * Np + s];
                    sv_step(y0, y1, y2, y3, eps, rw2, rw2l, r, fmaf(b, e_rec, -fR));
                    st[ST_RQHI * Np + s] = y0;
                    st[ST_RQLO * Np + s] = y1;
                    st[ST_RV * Np + s] = y2;
                    st[ST_RVLO * Np + s] = y3;
                }
            }
            if (!reverse) {
                // pickup y^n (owner) ; reduction buffer alternates so one barrier suffices
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float s2 = __shfl_xor_sync(0xffffffffu, ys, o);
                    const float e2 = __shfl_xor_sync(0xffffffffu, ye, o);
                    pickup_merge(ys, ye, s2, e2);
                }
                float *r2 = S.red2 + red2_parity * 2 * kPlateWarps;
                if (lane == 0) {
                    r2[warp] = ys;
                    r2[kPlateWarps + warp] = ye;
                }
                consumer_bar();
                if (tid == 0 && item.owner) {
                    float y = 0.f, ycomp = 0.f;
#pragma unroll
                    for (int w = 0; w < kPlateWarps; ++w) pickup_merge(y, ycomp, r2[w], r2[kPlateWarps + w]);
                    y += ycomp;
                    if (P.mode == MODE_FORWARD && P.audio)
                        P.audio[(long long)item.inst * P.total_steps + n] = y;
                    if (!isfinite(y)) set_status(P.status, item.inst, MDX_ERR_NONFINITE);
                }
                red2_parity ^= 1;
            }
        }
        // uniform exit decision for all consumer threads
        consumer_bar();
        if (*reinterpret_cast<volatile int *>(&S.misc[1])) {
            ok = false;
            break;
        }
    }

    // ---- write back per-item state (owner)
    if (ok) {
        consumer_bar();
        for (int ii = it0; ii < it1; ++ii) {
            const PlateItem item = P.items[ii];
            if (!item.owner) continue;
            const InstDesc d = P.inst[item.inst];
            float *st = S.state + item.smem_state;
            const int Np = d.Npad;
            for (int s = tid; s < d.N; s += kPlateThreads) {
                const long long m = d.mode_off + s;
                if (!reverse) {
                    if (P.mode == MODE_RECOMPUTE) {
                        P.seg_q[(long long)P.steps * TM + m] = st[ST_QHI * Np + s];
                        P.seg_v[(long long)P.steps * TM + m] = st[ST_V * Np + s];
                    } else {
                        P.state_io[m] = st[ST_QHI * Np + s];
                        P.state_io[TM + m] = st[ST_QLO * Np + s];
                        P.state_io[2 * TM + m] = st[ST_V * Np + s];
                        P.state_io[3 * TM + m] = st[ST_VLO * Np + s];
                    }
                } else {
                    P.adj[m] = st[ST_QHI * Np + s];
                    P.adj[TM + m] = st[ST_QLO * Np + s];
                    P.adj[2 * TM + m] = st[ST_V * Np + s];
                    if (item.cache) {
                        const float *g = item_gacc<PAR>(st, Np, item);
#pragma unroll
                        for (int row = 0; row < 2 * GA_N; ++row)
                            P.gacc[(long long)row * TM + m] = g[row * Np + s];
                    }
                    if constexpr (FUSED) {
                        P.rseg_q[(long long)P.steps * TM + m] = st[ST_RQHI * Np + s];
                        P.rseg_v[(long long)P.steps * TM + m] = st[ST_RV * Np + s];
                    }
                }
            }
        }
        // every item's d kappa sums (its own stress-mode range)
        if (reverse) {
            for (int ii = it0; ii < it1; ++ii) {
                const PlateItem item = P.items[ii];
                const InstDesc d = P.inst[item.inst];
                const float *kac = item_kacc<PAR>(S.state + item.smem_state, d.Npad);
                for (int q = tid; q < item.k1 - item.k0; q += kPlateThreads) {
                    P.kacc[2 * (d.k_off + item.k0 + q)] = kac[2 * q];
                    P.kacc[2 * (d.k_off + item.k0 + q) + 1] = kac[2 * q + 1];
                }
            }
        }
    } else if (tid == 0) {
        atomicExch((int *)gabort, 1);
        for (int ii = it0; ii < it1; ++ii) set_status(P.status, P.items[ii].inst, MDX_ERR_TIMEOUT);
    }
    __syncwarp();
    __syncthreads();
    // Drain: no bulk copy may still be writing shared memory when the CTA
    // exits.  Phases of one slot complete in order, so waiting for the last
    // issued phase of every slot covers all copies.  Copies from valid global
    // addresses always complete, so this wait is generous.
    if (tid == 0) {
        const long long issued = *reinterpret_cast<volatile long long *>(&S.misc[4]);
        for (int s = 0; s < RING; ++s) {
            if (issued <= s) continue;
            const long long last = s + ((issued - 1 - s) / RING) * RING;
            const uint32_t ph = (uint32_t)((last / RING) & 1);
            long long i = 0;
            while (!mbar_try_wait(&S.full[s], ph) && ++i < (1LL << 26)) {
            }
        }
    }
}

size_t plate_smem_bytes(int ring_stages, int stage_bytes, int u_floats, int state_floats) {
    size_t b = 2 * ring_stages * sizeof(uint64_t) + 16 * sizeof(int);
    b = (b + 127) & ~size_t(127);
    b += (size_t)ring_stages * stage_bytes;
    b += (size_t)u_floats * sizeof(float);
    b += (size_t)2 * kChunkK * 4 * kPlateWarps * sizeof(float);
    b += (size_t)2 * 2 * kPlateWarps * sizeof(float);
    b += (size_t)state_floats * sizeof(float);
    return b;
}

cudaError_t plate_set_smem_limit(size_t smem) {
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(plate_kernel<1, false>, A, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(plate_kernel<2, false>, A, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(plate_kernel<1, true>, A, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(plate_kernel<2, true>, A, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(plate_kernel<3, true>, A, (int)smem);
    return e;
}

// Cooperative launch (all CTAs resident: the per-plate exchange waits on
// other CTAs) through cudaLaunchKernelEx, which is also valid inside stream
// capture.
cudaError_t launch_plate(const PlateParams &p, int grid, size_t smem, cudaStream_t s) {
    if (grid <= 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kPlateBlock);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (p.parity) {
        if (p.mode == MODE_FUSED) return cudaLaunchKernelEx(&cfg, plate_kernel<3, true>, p);
        if (p.mode == MODE_REVERSE) return cudaLaunchKernelEx(&cfg, plate_kernel<2, true>, p);
        return cudaLaunchKernelEx(&cfg, plate_kernel<1, true>, p);
    }
    if (p.mode == MODE_FUSED) return cudaErrorInvalidValue;   // class layout only
    if (p.mode == MODE_REVERSE) return cudaLaunchKernelEx(&cfg, plate_kernel<2, false>, p);
    return cudaLaunchKernelEx(&cfg, plate_kernel<1, false>, p);
}

}  // namespace mdx
