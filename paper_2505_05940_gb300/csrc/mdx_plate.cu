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
//     range); the host balances the H bytes of the items over the CTAs;
//   * one producer warp streams the H rows of the CTA's items through a ring
//     of shared-memory stages with TMA bulk copies (cp.async.bulk + mbarrier
//     transaction counts).  H does not depend on the state, so the producer
//     runs ahead across step boundaries while the consumers wait for q;
//   * 8 consumer warps: thread t accumulates u_s for s = t, t+256, ...
//     (rows of H^k are contiguous in s, so the reads are conflict free);
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

// R: right-hand sides of the H pass (1: forward / recompute; 2: reverse).
template <int R>
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
    p += (size_t)kChunkK * P.u_slots * kUPartFloats * sizeof(float);
    S.red = reinterpret_cast<float *>(p);
    p += (size_t)2 * kChunkK * 4 * kPlateWarps * sizeof(float);
    S.red2 = reinterpret_cast<float *>(p);
    p += (size_t)2 * 2 * kPlateWarps * sizeof(float);
    S.state = reinterpret_cast<float *>(p);

    volatile int *gabort = P.abort_flag;
    const bool reverse = (P.mode == MODE_REVERSE);

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
            bool ok = true;
            for (int it = 0; it < P.steps && ok; ++it) {
                for (int ii = it0; ii < it1 && ok; ++ii) {
                    const PlateItem item = P.items[ii];
                    const InstDesc d = P.inst[item.inst];
                    const int rows_per_stage = max(1, stage_floats / d.Npad);
                    const int nmat = (reverse && d.has_dir) ? 2 : 1;
                    for (int k = item.k0; k < item.k1 && ok; ++k) {
                        for (int mat = 0; mat < nmat && ok; ++mat) {
                            const float *base = (mat == 0 ? P.H + d.H_off : P.dH + d.dH_off) +
                                                (long long)k * d.N * d.Npad;
                            for (int p0 = 0; p0 < d.N; p0 += rows_per_stage) {
                                const int nr = min(rows_per_stage, d.N - p0);
                                const int s = (int)(seq % RING);
                                const uint32_t ph = (uint32_t)((seq / RING) & 1);
                                if (!mbar_wait(&S.empty[s], ph ^ 1u, P.wait_limit, gabort)) {
                                    ok = false;
                                    break;
                                }
                                const uint32_t bytes = (uint32_t)nr * d.Npad * 4u;
                                mbar_arrive_expect_tx(&S.full[s], bytes);
                                bulk_g2s(S.ring + (size_t)s * stage_floats,
                                         base + (long long)p0 * d.Npad, bytes, &S.full[s]);
                                ++seq;
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
    long long seq = 0;         // stages consumed
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
        }
    }
    consumer_bar();

    for (int it = 0; it < P.steps; ++it) {
        // global step index: forward counts up, reverse counts down
        const int t_loc = reverse ? (P.steps - 1 - it) : it;
        const int n = P.n_begin + t_loc;

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
                    const float qn = in ? P.seg_q[(long long)t_loc * TM + m] : 0.f;
                    st[ST_SRC0 * Np + s] = qn;
                    st[ST_SRC1 * Np + s] = in ? P.coef.r[m] * st[ST_QHI * Np + s] : 0.f;
                    st[ST_FLOC * Np + s] = 0.f;
                    st[ST_FLOC2 * Np + s] = 0.f;
                }
            }
        }
        consumer_bar();

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
            const int nmat = (reverse && d.has_dir) ? 2 : 1;
            const float *src0 = reverse ? st + ST_SRC0 * Np : st + ST_QHI * Np;
            const float *src1 = st + ST_SRC1 * Np;
            const int spt = (Np + kPlateThreads - 1) / kPlateThreads;
            for (int kc = item.k0; kc < item.k1; kc += kChunkK) {
                const int nk = min(kChunkK, item.k1 - kc);
                float *red = S.red + chunk_parity * (kChunkK * 4 * kPlateWarps);
                for (int kk = 0; kk < nk; ++kk) {
                    for (int mat = 0; mat < nmat; ++mat) {
                        float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f);
                        float4 a1 = make_float4(0.f, 0.f, 0.f, 0.f);
                        for (int p0 = 0; p0 < d.N; p0 += rows_per_stage) {
                            const int nr = min(rows_per_stage, d.N - p0);
                            const int s = (int)(seq % RING);
                            const uint32_t ph = (uint32_t)((seq / RING) & 1);
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
                            ++seq;
                        }
                        if (active) {
                            // slot 0: H q, slot 1: H w (reverse), slot 2: dH q (direction)
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
                // combine the row groups: u (H q), z (H w), t (dH q) for own modes
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
                    const float kap = P.kappa[d.k_off + k];
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
                        float *ka = P.kacc + 2 * (d.k_off + k);
                        float s0 = ka[0], c0 = ka[1];
                        kahan_add(s0, c0, -dv[0] * dv[1]);
                        ka[0] = s0;
                        ka[1] = c0;
                        if (d.has_dir) {
                            float *da = P.diracc + 2 * (d.k_off + k);
                            float s1 = da[0], c1 = da[1];
                            kahan_add(s1, c1, -kap * fmaf(dv[1], dv[2], dv[0] * dv[3]));
                            da[0] = s1;
                            da[1] = c1;
                        }
                    }
                }
                chunk_parity ^= 1;
            }
            // publish partial forces of a shared plate
            if (d.n_contrib > 1) {
                const long long slot_base = (long long)(it & 1) * P.part_stride +
                                            d.part_off + (long long)item.slot * 3 * Np;
                for (int s = tid; s < Np; s += kPlateThreads) {
                    P.part[slot_base + s] = st[ST_FLOC * Np + s];
                    if (reverse) P.part[slot_base + Np + s] = st[ST_FLOC2 * Np + s];
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
            const float e = P.exc ? P.exc[(long long)item.inst * P.total_steps + n] : 0.f;
            float yp = 0.f;
            for (int s = tid; s < d.N; s += kPlateThreads) {
                const long long m = d.mode_off + s;
                float fA, fB = 0.f;
                if (d.n_contrib > 1) {
                    const long long base = (long long)(it & 1) * P.part_stride + d.part_off;
                    fA = 0.f;
                    for (int c = 0; c < d.n_contrib; ++c) {
                        fA += ld_cg(P.part + base + (long long)c * 3 * Np + s);
                        if (reverse) fB += ld_cg(P.part + base + (long long)c * 3 * Np + Np + s);
                    }
                } else {
                    fA = st[ST_FLOC * Np + s];
                    if (reverse) fB = st[ST_FLOC2 * Np + s];
                }
                const float eps = P.coef.eps[m], rw2 = P.coef.rw2[m], r = P.coef.r[m];
                const float rw2l = P.coef.rw2lo[m];
                const float b = P.coef.b[m], c = P.coef.c[m];
                float x0 = st[ST_QHI * Np + s], x1 = st[ST_QLO * Np + s], x2 = st[ST_V * Np + s];
                float x3 = st[ST_VLO * Np + s];
                if (!reverse) {
                    sv_step(x0, x1, x2, x3, eps, rw2, rw2l, r, fmaf(b, e, -fA));
                    yp = fmaf(c, x0, yp);
                } else {
                    // fA = J w (summed), fB = fnl(q^n)
                    if (item.owner) {
                        const float a = x0;
                        const float qn = st[ST_SRC0 * Np + s];
                        const float vn = P.seg_v[(long long)t_loc * TM + m];
                        const float qn1 = P.seg_q[(long long)(t_loc + 1) * TM + m];
                        const float ybn = P.ybar[(long long)item.inst * P.total_steps + n];
                        float *g = P.gacc;
                        float gsum, gcmp;
#define MDX_ACC(IDX, X)                                                    \
    gsum = g[(long long)(2 * (IDX)) * TM + m];                             \
    gcmp = g[(long long)(2 * (IDX) + 1) * TM + m];                         \
    kahan_add(gsum, gcmp, (X));                                            \
    g[(long long)(2 * (IDX)) * TM + m] = gsum;                             \
    g[(long long)(2 * (IDX) + 1) * TM + m] = gcmp;
                        MDX_ACC(GA_A, a * qn)
                        MDX_ACC(GA_V, a * vn)
                        MDX_ACC(GA_F, a * fmaf(b, e, -fB))
                        MDX_ACC(GA_E, a * e)
                        MDX_ACC(GA_C, ybn * qn1)
#undef MDX_ACC
                    }
                    const float ybm =
                        (n >= 1) ? P.ybar[(long long)item.inst * P.total_steps + n - 1] : 0.f;
                    adj_step(x0, x1, x2, eps, rw2, fA, c * ybm);
                }
                st[ST_QHI * Np + s] = x0;
                st[ST_QLO * Np + s] = x1;
                st[ST_V * Np + s] = x2;
                st[ST_VLO * Np + s] = x3;
            }
            if (!reverse) {
                // pickup y^n (owner) ; reduction buffer alternates so one barrier suffices
                yp = warp_sum(yp);
                float *r2 = S.red2 + red2_parity * 2 * kPlateWarps;
                if (lane == 0) r2[warp] = yp;
                consumer_bar();
                if (tid == 0 && item.owner) {
                    float y = 0.f;
#pragma unroll
                    for (int w = 0; w < kPlateWarps; ++w) y += r2[w];
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

size_t plate_smem_bytes(int ring_stages, int stage_bytes, int u_slots, int state_floats) {
    size_t b = 2 * ring_stages * sizeof(uint64_t) + 16 * sizeof(int);
    b = (b + 127) & ~size_t(127);
    b += (size_t)ring_stages * stage_bytes;
    b += (size_t)kChunkK * u_slots * kUPartFloats * sizeof(float);
    b += (size_t)2 * kChunkK * 4 * kPlateWarps * sizeof(float);
    b += (size_t)2 * 2 * kPlateWarps * sizeof(float);
    b += (size_t)state_floats * sizeof(float);
    return b;
}

cudaError_t plate_set_smem_limit(size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(plate_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(plate_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
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
    if (p.mode == MODE_REVERSE) return cudaLaunchKernelEx(&cfg, plate_kernel<2>, p);
    return cudaLaunchKernelEx(&cfg, plate_kernel<1>, p);
}

}  // namespace mdx
