// Grouped von Karman plates: plates that share one coupling tensor, stepped
// together with the coupling contraction on the tensor cores.
//
// Plates of one geometry (for a simply supported rectangle of fixed area, one
// aspect ratio) share their modes: a smaller plate's transverse and stress
// modes are prefixes of the largest member's (Sec. 3, Eq. 2; Eq. 10).  With
// Q = [q_1 ... q_B] the plates' states, zero-padded to the largest mode set,
//   U^k = H^k Q                      (one GEMM per stress mode k and step)
//   eta_{k,b} = q_b . U^k_{:,b},   f_b = sum_k kappa_{k,b} eta_{k,b} U^k_{:,b}
// (Sec. 3.1, Eq. 9 with C^s_pn = H^n_ps, Sec. 4.3.3), followed by the
// difference-form Stormer-Verlet update (Sec. 3.2, Eq. 20) and the pickup.
// A plate that lacks stress mode k gets kappa_{k,b} = 0; its padded modes
// carry q = 0, so every plate sees exactly its own coupling tensor.
//
// Symmetry classes: H^k_ij vanishes unless class(i) ^ class(j) == class(k),
// so with rows s of class sb the GEMM of H^k only needs the columns p of class
// c ^ sb (c = class(k)): per stress mode, four dense blocks (rows of one class
// against columns of another), cut into 128-row tiles.
//
// Precision: split TF32 on tcgen05 (kind::tf32, FP32 accumulation in tensor
// memory).  Both operands are split into a TF32 high part (round to nearest)
// and the FP32 remainder, x = hi + lo exactly, and each tile accumulates
//   H_hi Q_hi + H_hi Q_lo + H_lo Q_hi,
// whose error is about 2^-21 of |H||Q| (the dropped H_lo Q_lo and the TF32
// rounding of the remainders), the accuracy of the FP32 path.
//
// Execution (one 256-thread CTA per SM, cooperative launch, all steps in one
// launch).  Each CTA holds a contiguous range of one group's stress modes:
//   warp 0  producer: streams the CTA's coupling tiles from global memory in
//           16-column chunks (cp.async.bulk into a ring of 8 KB stages,
//           mbarrier transaction counts); the tiles were laid out at plan time
//           as the MMA's shared-memory image (8-row x 16-byte core matrices,
//           K-major, no swizzle), so one bulk copy moves one chunk;
//   warps 2-3 convert each chunk in place into its TF32 high part plus a
//           remainder stage;
//   warp 1  issues the MMAs (one thread) into tensor memory: per tile a
//           [128 rows x Bp plates] FP32 accumulator;
//   warps 4-7 (epilogue, one tensor-memory lane quarter each): eta from the
//           accumulators, then f accumulated in a second tensor-memory region;
//           at the end of the step the partial forces go to global slots.
// The CTAs of a group then meet at a group barrier (monotonic counter,
// release / acquire, bounded spin); the owner CTA of each plate sums the
// partial forces, steps the plate, writes its audio sample and its new q, and
// the group meets again before the next step's Q images are built.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "../../include/mdx.h"
#include "mdx_common.cuh"
#include "mdx_tc.cuh"

namespace mdx {

namespace {

using namespace tc;

// Named barrier of the four epilogue warps.
__device__ __forceinline__ void epi_bar() {
    __syncwarp();
    asm volatile("barrier.sync 1, 128;" ::: "memory");
}

__device__ __forceinline__ unsigned ld_acq(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ float ldcg(const float *p) {
    float v;
    asm volatile("ld.global.cg.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

// Writes q of plate b at class-order position pos into a Q image (global or
// shared): TF32 high part in class a's image, the FP32 remainder in the image
// that follows it.
__device__ __forceinline__ void q_image_put(float *img, const GrpDesc &G, int b, int pos, float q) {
    int a = 0;
    if (pos >= G.ocls[1]) a = 1;
    if (pos >= G.ocls[2]) a = 2;
    if (pos >= G.ocls[3]) a = 3;
    const int kp = G.kpad[a];
    const int e = G.qoff[a] + cm_index(b, pos - G.ocls[a], kp);
    const float h = tf32_hi(q);
    img[e] = h;
    img[e + G.Bp * kp] = q - h;
}

// In-warp reduction of 16 values per lane: on return, lane l (l even) holds
// the warp's sum of value ((l >> 4) & 1) * 8 + ((l >> 3) & 1) * 4 +
// ((l >> 2) & 1) * 2 + ((l >> 1) & 1), after 16 shuffles instead of 80.
__device__ __forceinline__ float warp_reduce16(float (&t)[16], int lane) {
#pragma unroll
    for (int half = 8, o = 16; half >= 1; half >>= 1, o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (i < half) {
                const float keep = up ? t[i + half] : t[i];
                const float send = up ? t[i] : t[i + half];
                t[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
    }
    return t[0] + __shfl_xor_sync(0xffffffffu, t[0], 1);
}

__device__ __forceinline__ int reduce16_index(int lane) {
    return ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
}

struct Ctrl {
    uint64_t full[8], empty[8], conv[8];
    uint64_t qready, mma_done[2], epi_free[2], drain;
    uint32_t tmem_base;
    int fail;            // set by any role that gave up; read by the epilogue warps
    int pad[2];
    float eta_red[4][kGrpMaxB];
    float ke[kGrpMaxB];
    float pick[2][8];
};

}  // namespace

__global__ void __launch_bounds__(kGrpThreads, 1) group_kernel(const GroupParams P) {
    extern __shared__ __align__(1024) unsigned char smem[];
    Ctrl &C = *reinterpret_cast<Ctrl *>(smem);
    __shared__ GrpDesc G;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int cta = blockIdx.x;
    const int gi = P.cta_group[cta];
    const int u0 = P.cta_units[2 * cta], u1 = P.cta_units[2 * cta + 1];
    const int R = P.ring_stages;
    float *ring = reinterpret_cast<float *>(smem + P.ring_off);
    float *lo = reinterpret_cast<float *>(smem + P.lo_off);
    float *qimg = reinterpret_cast<float *>(smem + P.q_off);
    // this CTA's work units, cached in shared memory (every role walks them
    // once per chunk)
    GrpUnit *units = reinterpret_cast<GrpUnit *>(smem + P.scratch_off);
    volatile int *gabort = P.abort_flag;

    if (tid == 0) {
        G = P.groups[gi];
        for (int s = 0; s < R; ++s) {
            bar_init(&C.full[s], 1);
            bar_init(&C.empty[s], 1);
            bar_init(&C.conv[s], 2);
        }
        bar_init(&C.qready, 1);
        for (int b = 0; b < 2; ++b) {
            bar_init(&C.mma_done[b], 1);
            bar_init(&C.epi_free[b], 4);
        }
        bar_init(&C.drain, 1);
        C.fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int x = tid; x < (u1 - u0) * (int)(sizeof(GrpUnit) / 4); x += kGrpThreads)
        reinterpret_cast<int *>(units)[x] = reinterpret_cast<const int *>(P.units + u0)[x];
    if (warp == 1) {
        // the whole tensor memory of the SM (one CTA per SM)
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                         su32(&C.tmem_base))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = C.tmem_base;
    const int Bp = G.Bp;
    const int nt = G.n_tiles;
    const int steps = P.steps;
    long long issued = 0;   // producer: bulk copies issued (for the drain at exit)
    bool mma_issued = false;

    if (warp == 0) {
        // ============================================================ producer
        if (lane == 0) {
            const bool hint = P.l2_keep > 0.f;
            const uint64_t pol = hint ? keep_policy(fminf(P.l2_keep, 1.f)) : 0ull;
            int slot = 0;
            uint32_t ph = 0;
            bool ok = true;
            for (int it = 0; it < steps && ok; ++it)
                for (int u = u0; u < u1 && ok; ++u) {
                    const GrpUnit &U = units[u - u0];
                    for (int t = 0; t < nt && ok; ++t) {
                        const long long off = U.off[t];
                        if (off < 0) continue;
                        const int a = U.c ^ G.tile_sb[t];
                        const int r8 = (G.tile_rows[t] + 7) & ~7;
                        const uint32_t bytes = (uint32_t)r8 * kGrpChunk * 4u;
                        for (int j = 0; j < G.kpad[a] / kGrpChunk; ++j) {
                            if (!bar_spin(&C.empty[slot], ph ^ 1u, P.wait_limit, gabort)) {
                                ok = false;
                                break;
                            }
                            bar_expect_tx(&C.full[slot], bytes);
                            bulk_load(ring + (size_t)slot * (kGrpStageBytes / 4),
                                      P.img + off + (long long)j * r8 * kGrpChunk, bytes,
                                      &C.full[slot], hint, pol);
                            ++issued;
                            if (++slot == R) {
                                slot = 0;
                                ph ^= 1u;
                            }
                        }
                    }
                }
            if (!ok) {
                C.fail = 1;
                atomicExch((int *)gabort, 1);
            }
        }
    } else if (warp == 1) {
        // ============================================================ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_tf32(128, Bp);
            int slot = 0;
            uint32_t ph = 0;
            long long ucount = 0;
            bool ok = true;
            for (int it = 0; it < steps && ok; ++it) {
                if (!bar_wait(&C.qready, (uint32_t)(it & 1), P.wait_limit, gabort)) {
                    ok = false;
                    break;
                }
                for (int u = u0; u < u1 && ok; ++u, ++ucount) {
                    const GrpUnit &U = units[u - u0];
                    // two accumulator sets: the epilogue of the unit two back has read this one
                    const int buf = (int)(ucount & 1);
                    if (!bar_wait(&C.epi_free[buf], (uint32_t)(((ucount >> 1) & 1) ^ 1),
                                  P.wait_limit, gabort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    for (int t = 0; t < nt && ok; ++t) {
                        if (U.off[t] < 0) continue;
                        const int a = U.c ^ G.tile_sb[t];
                        const int kp = G.kpad[a];
                        const uint32_t sbo_q = (uint32_t)(kp / 4) * 128u;
                        const uint32_t qa = su32(qimg + G.qoff[a]);
                        const uint32_t qla = su32(qimg + G.qoff[a] + Bp * kp);
                        const uint32_t d = tmem + (uint32_t)((buf * nt + t) * Bp);
                        for (int j = 0; j < kp / kGrpChunk; ++j) {
                            if (!bar_spin(&C.conv[slot], ph, P.wait_limit, gabort)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const uint32_t as = su32(ring + (size_t)slot * (kGrpStageBytes / 4));
                            const uint32_t als = su32(lo + (size_t)slot * (kGrpStageBytes / 4));
                            // K-steps of 8 columns (two core matrices) within the chunk;
                            // 8-row groups are kGrpChunk / 4 core matrices apart
                            constexpr uint32_t sbo_a = (kGrpChunk / 4) * 128u;
#pragma unroll
                            for (int kk = 0; kk < kGrpChunk / 8; ++kk) {
                                const uint64_t ad = smem_desc(as + kk * 256u, 128u, sbo_a);
                                const uint64_t ald = smem_desc(als + kk * 256u, 128u, sbo_a);
                                const uint32_t qo = (uint32_t)(j * (kGrpChunk / 4) + kk * 2) * 128u;
                                const uint64_t qd = smem_desc(qa + qo, 128u, sbo_q);
                                const uint64_t qld = smem_desc(qla + qo, 128u, sbo_q);
                                mma_tf32(d, ad, qd, idesc, (j | kk) ? 1u : 0u);
                                mma_tf32(d, ad, qld, idesc, 1u);
                                mma_tf32(d, ald, qd, idesc, 1u);
                            }
                            mma_issued = true;
                            mma_commit(&C.empty[slot]);
                            if (++slot == R) {
                                slot = 0;
                                ph ^= 1u;
                            }
                        }
                    }
                    if (ok) mma_commit(&C.mma_done[buf]);
                }
            }
            if (!ok) {
                C.fail = 1;
                atomicExch((int *)gabort, 1);
            }
            // every MMA issued has finished before the tensor memory is released
            if (mma_issued) {
                mma_commit(&C.drain);
                long long i = 0;
                while (!bar_try(&C.drain, 0) && ++i < (1LL << 24)) {
                }
            }
        }
    } else if (warp < 4) {
        // ============================================================ converters
        const int ct = tid - 64;   // 0..63
        int slot = 0;
        uint32_t ph = 0;
        bool ok = true;
        for (int it = 0; it < steps && ok; ++it)
            for (int u = u0; u < u1 && ok; ++u) {
                const GrpUnit &U = units[u - u0];
                for (int t = 0; t < nt && ok; ++t) {
                    if (U.off[t] < 0) continue;
                    const int a = U.c ^ G.tile_sb[t];
                    const int r8 = (G.tile_rows[t] + 7) & ~7;
                    const int n4 = r8 * kGrpChunk / 4;
                    for (int j = 0; j < G.kpad[a] / kGrpChunk; ++j) {
                        if (!bar_spin(&C.full[slot], ph, P.wait_limit, gabort)) {
                            ok = false;
                            break;
                        }
                        float4 *x = reinterpret_cast<float4 *>(ring + (size_t)slot * (kGrpStageBytes / 4));
                        float4 *y = reinterpret_cast<float4 *>(lo + (size_t)slot * (kGrpStageBytes / 4));
                        for (int i = ct; i < n4; i += 64) {
                            const float4 v = x[i];
                            float4 h, l;
                            h.x = tf32_hi(v.x);
                            h.y = tf32_hi(v.y);
                            h.z = tf32_hi(v.z);
                            h.w = tf32_hi(v.w);
                            l.x = v.x - h.x;
                            l.y = v.y - h.y;
                            l.z = v.z - h.z;
                            l.w = v.w - h.w;
                            x[i] = h;
                            y[i] = l;
                        }
                        fence_async_smem();
                        __syncwarp();
                        if (lane == 0) bar_arrive(&C.conv[slot]);
                        if (++slot == R) {
                            slot = 0;
                            ph ^= 1u;
                        }
                    }
                }
            }
        if (!ok) {
            C.fail = 1;
            atomicExch((int *)gabort, 1);
        }
    } else {
        // ============================================================ epilogue / owners
        const int et = tid - 128;              // 0..127
        const int quarter = warp - 4;          // tensor-memory lane quarter
        const int r = 32 * quarter + lane;     // accumulator row of this thread
        const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;
        const unsigned nct = (unsigned)G.n_ctas;
        const int fcol = 2 * nt * Bp;          // first column of the force accumulators
        const int slot_in_group = cta - G.cta0;
        unsigned *cnt = P.counters + gi;
        const long long TM = P.total_modes;
        long long ucount = 0;
        bool ok = true;
        bool owner = false;
        for (int b = 0; b < G.B; ++b) owner = owner || (P.plates[G.plate0 + b].owner == cta);
        // owners: initial q (class order) of the plates this CTA steps
        for (int b = 0; b < G.B; ++b) {
            const GrpPlate pl = P.plates[G.plate0 + b];
            if (pl.owner != cta) continue;
            const InstDesc d = P.inst[pl.inst];
            for (int j = et; j < d.N; j += 128)
                q_image_put(P.qbuf + G.qbuf_off, G, b, P.gpos[G.gpos_off + j],
                            P.state_io[d.mode_off + j]);
        }
        epi_bar();
        if (et == 0) {
            __threadfence();
            atomicAdd(cnt, 1u);
        }
        auto group_wait = [&](unsigned target) {
            if (et == 0) {
                long long spins = 0;
                while (ld_acq(cnt) < target) {
                    if (++spins > P.wait_limit || ((spins & 255) == 0 && *gabort)) {
                        C.fail = 1;
                        atomicExch((int *)gabort, 1);
                        break;
                    }
                    __nanosleep(64);
                }
                if (C.fail) atomicExch((int *)gabort, 1);
            }
            epi_bar();
            return *reinterpret_cast<volatile int *>(&C.fail) == 0;
        };
        for (int it = 0; it < steps && ok; ++it) {
            const int n = P.n_begin + it;
            // ---- wait for every owner's q of this step, build the Q images
            if (!group_wait(nct * (unsigned)(1 + 2 * it))) {
                ok = false;
                break;
            }
            // the group's Q image (TF32 high parts and remainders, as the MMAs read
            // them) comes in with bulk copies; the MMA issuer and this warp group
            // wait on the same barrier
            if (et == 0) {
                fence_async_global();
                const uint32_t total = (uint32_t)G.q_floats * 4u;
                bar_expect_tx(&C.qready, total);
                for (uint32_t o = 0; o < total; o += 32768u)
                    bulk_load(reinterpret_cast<unsigned char *>(qimg) + o,
                              reinterpret_cast<const unsigned char *>(P.qbuf + G.qbuf_off) + o,
                              min(32768u, total - o), &C.qready, false, 0ull);
            }
            if (!bar_wait(&C.qready, (uint32_t)(it & 1), P.wait_limit, gabort)) C.fail = 1;
            // ---- zero the force accumulators
            {
                float z[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) z[i] = 0.f;
                for (int t = 0; t < nt; ++t)
                    for (int cb = 0; cb < Bp; cb += 16)
                        tmem_st16(tmem + lane_base + (uint32_t)(fcol + t * Bp + cb), z);
                tmem_wait_st();
            }
            // ---- stress modes of this CTA
            for (int u = u0; u < u1; ++u, ++ucount) {
                const GrpUnit &U = units[u - u0];
                const int buf = (int)(ucount & 1);
                const uint32_t dcol = (uint32_t)(buf * nt * Bp);
                bool got = bar_wait(&C.mma_done[buf], (uint32_t)((ucount >> 1) & 1), P.wait_limit,
                                    gabort);
                if (!got) C.fail = 1;
                epi_bar();
                if (*reinterpret_cast<volatile int *>(&C.fail)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                // eta_{k,b} = sum over rows s of q_b[s] U[s][b]
                for (int cb = 0; cb < Bp; cb += 16) {
                    float acc[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) acc[i] = 0.f;
                    for (int t = 0; t < nt; ++t) {
                        if (U.off[t] < 0) continue;
                        float v[16];
                        tmem_ld16(tmem + lane_base + dcol + (uint32_t)(t * Bp + cb), v);
                        const int sb = G.tile_sb[t];
                        if (r < G.tile_rows[t]) {
                            const int kp = G.kpad[sb];
                            const float *qh = qimg + G.qoff[sb];
                            const float *ql = qh + Bp * kp;
                            const int p = G.tile_r0[t] + r;
#pragma unroll
                            for (int i = 0; i < 16; ++i) {
                                const int e = cm_index(cb + i, p, kp);
                                acc[i] = fmaf(qh[e] + ql[e], v[i], acc[i]);
                            }
                        }
                    }
                    const float sum = warp_reduce16(acc, lane);
                    if ((lane & 1) == 0) C.eta_red[quarter][cb + reduce16_index(lane)] = sum;
                }
                epi_bar();
                if (et < Bp) {
                    const float eta = (C.eta_red[0][et] + C.eta_red[1][et]) +
                                      (C.eta_red[2][et] + C.eta_red[3][et]);
                    C.ke[et] = P.kap[G.kap_off + (long long)U.row * Bp + et] * eta;
                }
                epi_bar();
                // f[s][b] += kappa_{k,b} eta_{k,b} U[s][b]
                for (int t = 0; t < nt; ++t) {
                    if (U.off[t] < 0) continue;
                    for (int cb = 0; cb < Bp; cb += 16) {
                        float v[16], f[16];
                        tmem_ld16(tmem + lane_base + dcol + (uint32_t)(t * Bp + cb), v);
                        tmem_ld16(tmem + lane_base + (uint32_t)(fcol + t * Bp + cb), f);
#pragma unroll
                        for (int i = 0; i < 16; ++i) f[i] = fmaf(C.ke[cb + i], v[i], f[i]);
                        tmem_st16(tmem + lane_base + (uint32_t)(fcol + t * Bp + cb), f);
                    }
                }
                tmem_wait_st();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) bar_arrive(&C.epi_free[buf]);
            }
            if (!ok) break;
            // ---- partial forces of this CTA -> global slot (class order)
            for (int t = 0; t < nt; ++t) {
                const int sb = G.tile_sb[t];
                for (int cb = 0; cb < Bp; cb += 16) {
                    float f[16];
                    tmem_ld16(tmem + lane_base + (uint32_t)(fcol + t * Bp + cb), f);
                    if (r < G.tile_rows[t]) {
                        const long long pos = G.ocls[sb] + G.tile_r0[t] + r;
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const int b = cb + i;
                            if (b < G.B)
                                P.part[G.part_off + ((long long)slot_in_group * Bp + b) * G.Np + pos] = f[i];
                        }
                    }
                }
            }
            epi_bar();
            if (et == 0) {
                __threadfence();
                atomicAdd(cnt, 1u);
            }
            // ---- owners: gather the forces, step the plates, pickup, new q
            if (owner) {
                if (!group_wait(nct * (unsigned)(2 + 2 * it))) {
                    ok = false;
                    break;
                }
                for (int b = 0; b < G.B; ++b) {
                    const GrpPlate pl = P.plates[G.plate0 + b];
                    if (pl.owner != cta) continue;
                    const InstDesc d = P.inst[pl.inst];
                    const float e = P.exc ? P.exc[(long long)pl.inst * P.total_steps + n] : 0.f;
                    float ys = 0.f, ye = 0.f;
                    for (int j = et; j < d.N; j += 128) {
                        const int pos = P.gpos[G.gpos_off + j];
                        float f = 0.f;
                        for (int s = 0; s < G.n_ctas; ++s)
                            f += ldcg(P.part + G.part_off + ((long long)s * Bp + b) * G.Np + pos);
                        const long long m = d.mode_off + j;
                        float x0 = P.state_io[m], x1 = P.state_io[TM + m];
                        float x2 = P.state_io[2 * TM + m], x3 = P.state_io[3 * TM + m];
                        sv_step(x0, x1, x2, x3, P.coef.eps[m], P.coef.rw2[m], P.coef.rw2lo[m],
                                P.coef.r[m], fmaf(P.coef.b[m], e, -f));
                        pickup_add(ys, ye, P.coef.c[m], P.coef.clo[m], x0, x1);
                        P.state_io[m] = x0;
                        P.state_io[TM + m] = x1;
                        P.state_io[2 * TM + m] = x2;
                        P.state_io[3 * TM + m] = x3;
                        q_image_put(P.qbuf + G.qbuf_off, G, b, pos, x0);
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const float s2 = __shfl_xor_sync(0xffffffffu, ys, o);
                        const float e2 = __shfl_xor_sync(0xffffffffu, ye, o);
                        pickup_merge(ys, ye, s2, e2);
                    }
                    if (lane == 0) {
                        C.pick[0][quarter] = ys;
                        C.pick[1][quarter] = ye;
                    }
                    epi_bar();
                    if (et == 0) {
                        float y = 0.f, yc = 0.f;
                        for (int w = 0; w < 4; ++w) pickup_merge(y, yc, C.pick[0][w], C.pick[1][w]);
                        y += yc;
                        if (P.audio) P.audio[(long long)pl.inst * P.total_steps + n] = y;
                        if (!isfinite(y)) set_status(P.status, pl.inst, MDX_ERR_NONFINITE);
                    }
                    epi_bar();
                }
            }
            epi_bar();
            if (et == 0) {
                __threadfence();
                atomicAdd(cnt, 1u);
            }
        }
        if (!ok && et == 0) {
            atomicExch((int *)gabort, 1);
            for (int b = 0; b < G.B; ++b)
                set_status(P.status, P.plates[G.plate0 + b].inst, MDX_ERR_TIMEOUT);
        }
    }

    __syncwarp();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // release the tensor memory (every MMA has finished: see the MMA issuer)
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    // no bulk copy may still be writing shared memory when the CTA exits:
    // wait for the last issued phase of every stage
    if (tid == 0) {
        for (int s = 0; s < R; ++s) {
            if (issued <= s) continue;
            const long long last = s + ((issued - 1 - s) / R) * R;
            const uint32_t ph = (uint32_t)((last / R) & 1);
            long long i = 0;
            while (!bar_try(&C.full[s], ph) && ++i < (1LL << 26)) {
            }
        }
    }
}

// ====================================================================== host

struct GroupPlan {
    int device = 0;
    int n_ctas = 0;
    int ring_stages = 3;
    size_t smem = 0;
    int ring_off = 0, lo_off = 0, q_off = 0, scratch_off = 0;
    std::vector<GrpDesc> groups;
    std::vector<GrpUnit> units;
    std::vector<int> cta_group, cta_units;
    std::vector<GrpPlate> plates;
    std::vector<int> gpos;
    std::vector<std::vector<int>> unit_user_k;   // per kernel group: user stress index of each unit
    std::vector<std::vector<int>> plate_kcount;  // per kernel group: stress modes of each plate
    std::vector<std::vector<int>> plate_inst;    // per kernel group: instance of each plate
    long long part_floats = 0, qbuf_floats = 0, kap_floats = 0;
    double bytes_per_step = 0.0, flops_per_step = 0.0;
    // device memory
    GrpDesc *d_groups = nullptr;
    GrpUnit *d_units = nullptr;
    int *d_cta_group = nullptr, *d_cta_units = nullptr, *d_gpos = nullptr;
    GrpPlate *d_plates = nullptr;
    float *d_kap = nullptr, *d_img = nullptr, *d_part = nullptr, *d_qbuf = nullptr;
    unsigned *d_counters = nullptr;
    long long wait_limit = 1 << 22;
};

namespace {

int gfail(int code, const char *msg) { return set_last_error(code, msg); }

template <class T>
cudaError_t gupload(T **dst, const std::vector<T> &src) {
    const size_t n = std::max<size_t>(src.size(), 1);
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(dst), n * sizeof(T));
    if (e != cudaSuccess) return e;
    if (!src.empty()) e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

}  // namespace

void group_plan_free(GroupPlan *g) {
    if (!g) return;
    cudaSetDevice(g->device);
    void *ptrs[] = {g->d_groups, g->d_units, g->d_cta_group, g->d_cta_units, g->d_gpos,
                    g->d_plates, g->d_kap, g->d_img, g->d_part, g->d_qbuf, g->d_counters};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete g;
}

int group_plan_ctas(const GroupPlan *g) { return g ? g->n_ctas : 0; }
double group_plan_bytes_per_step(const GroupPlan *g) { return g ? g->bytes_per_step : 0.0; }
double group_plan_flops_per_step(const GroupPlan *g) { return g ? g->flops_per_step : 0.0; }

int group_plan_build(GroupPlan **out, const mdx_instance *I, const std::vector<InstDesc> &inst,
                     const std::vector<int> &grouped, int device, int n_sms, int smem_optin,
                     long long wait_limit) {
    *out = nullptr;
    GroupPlan *gp = new GroupPlan();
    gp->device = device;
    gp->wait_limit = wait_limit;
    auto bail = [&](int rc) {
        group_plan_free(gp);
        return rc;
    };
    // ---- members of every geometry group (ascending id, plan order)
    std::map<int, std::vector<int>> members;
    for (size_t i = 0; i < inst.size(); ++i)
        if (grouped[i]) members[I[i].geom_group].push_back((int)i);
    struct Image {
        int master, N, M;
        int ncls[4], ocls[4], kpad[4];
        std::vector<int> gperm, gpos, kord, kcls;
        std::vector<int> tile_sb, tile_r0, tile_rows;
        long long off0 = 0;                 // float offset of the image
        std::vector<std::vector<long long>> tile_off;   // [internal k][tile]
        double floats = 0.0;                // image floats (one pass per step)
    };
    std::vector<Image> images;
    std::vector<std::vector<int>> image_members;
    std::vector<float> img;
    for (auto &kv : members) {
        const std::vector<int> &mem = kv.second;
        Image im;
        im.master = mem[0];
        for (int i : mem)
            if (inst[i].N > inst[im.master].N ||
                (inst[i].N == inst[im.master].N && I[i].n_psi > I[im.master].n_psi))
                im.master = i;
        const mdx_instance &Mi = I[im.master];
        im.N = Mi.n_phi;
        im.M = Mi.n_psi;
        if (!Mi.phi_class || !Mi.psi_class)
            return bail(gfail(MDX_ERR_ARG, "grouped plates need phi_class and psi_class"));
        for (int i : mem) {
            const mdx_instance &S = I[i];
            if (S.n_psi > im.M)
                return bail(gfail(MDX_ERR_ARG,
                                  "geom_group: the member with the most modes must also have the "
                                  "most stress modes"));
            if (!S.phi_class || !S.psi_class)
                return bail(gfail(MDX_ERR_ARG, "grouped plates need phi_class and psi_class"));
            for (int m = 0; m < S.n_phi; ++m)
                if (S.phi_class[m] != Mi.phi_class[m])
                    return bail(gfail(MDX_ERR_ARG, "geom_group: mode classes differ from the group's"));
            for (int k = 0; k < S.n_psi; ++k)
                if (S.psi_class[k] != Mi.psi_class[k])
                    return bail(gfail(MDX_ERR_ARG, "geom_group: stress classes differ from the group's"));
            // a member's coupling tensor is the leading block of the master's
            for (int k = 0; k < S.n_psi; ++k)
                for (int x = 0; x < S.n_phi; ++x) {
                    const float *a = S.H + ((size_t)k * S.n_phi + x) * S.n_phi;
                    const float *b = Mi.H + ((size_t)k * im.N + x) * im.N;
                    if (std::memcmp(a, b, (size_t)S.n_phi * sizeof(float)) != 0)
                        return bail(gfail(MDX_ERR_ARG,
                                          "geom_group: a member's H is not the leading block of "
                                          "the group's largest member"));
                }
        }
        for (int a = 0; a < 4; ++a) im.ncls[a] = 0;
        for (int m = 0; m < im.N; ++m) {
            const int c = Mi.phi_class[m];
            if (c < 0 || c > 3) return bail(gfail(MDX_ERR_ARG, "phi_class outside 0..3"));
            im.ncls[c]++;
        }
        im.ocls[0] = 0;
        for (int a = 1; a < 4; ++a) im.ocls[a] = im.ocls[a - 1] + im.ncls[a - 1];
        for (int a = 0; a < 4; ++a) im.kpad[a] = (im.ncls[a] + kGrpChunk - 1) / kGrpChunk * kGrpChunk;
        im.gperm.resize(im.N);
        im.gpos.resize(im.N);
        int fill[4] = {im.ocls[0], im.ocls[1], im.ocls[2], im.ocls[3]};
        for (int m = 0; m < im.N; ++m) {
            const int pos = fill[Mi.phi_class[m]]++;
            im.gperm[pos] = m;
            im.gpos[m] = pos;
        }
        im.kord.resize(im.M);
        for (int k = 0; k < im.M; ++k) {
            const int c = Mi.psi_class[k];
            if (c < 0 || c > 3) return bail(gfail(MDX_ERR_ARG, "psi_class outside 0..3"));
            im.kord[k] = k;
        }
        std::stable_sort(im.kord.begin(), im.kord.end(),
                         [&](int x, int y) { return Mi.psi_class[x] < Mi.psi_class[y]; });
        im.kcls.resize(im.M);
        for (int k = 0; k < im.M; ++k) im.kcls[k] = Mi.psi_class[im.kord[k]];
        // the class pattern of H (entries outside it at most 1e-6 of max |H^k|)
        for (int k = 0; k < im.M; ++k) {
            const float *Hk = Mi.H + (size_t)k * im.N * im.N;
            float amax = 0.f;
            for (size_t t = 0; t < (size_t)im.N * im.N; ++t) amax = std::max(amax, std::fabs(Hk[t]));
            for (int x = 0; x < im.N; ++x)
                for (int y = 0; y < im.N; ++y)
                    if ((Mi.phi_class[x] ^ Mi.phi_class[y]) != Mi.psi_class[k] &&
                        std::fabs(Hk[(size_t)x * im.N + y]) > 1e-6f * amax)
                        return bail(gfail(MDX_ERR_ARG,
                                          "grouped plate: H lies outside the declared symmetry classes"));
        }
        // tiles: rows of class sb in blocks of 128
        for (int sb = 0; sb < 4; ++sb)
            for (int r0 = 0; r0 < im.ncls[sb]; r0 += 128) {
                im.tile_sb.push_back(sb);
                im.tile_r0.push_back(r0);
                im.tile_rows.push_back(std::min(128, im.ncls[sb] - r0));
            }
        if ((int)im.tile_sb.size() > kGrpMaxTiles)
            return bail(gfail(MDX_ERR_UNSUPPORTED, "grouped plate: too many modes per symmetry class"));
        // the image: per internal stress mode, per tile, chunks of [r8][16] in core-matrix order
        im.off0 = (long long)img.size();
        im.tile_off.assign(im.M, std::vector<long long>(im.tile_sb.size(), -1));
        for (int kk = 0; kk < im.M; ++kk) {
            const int ku = im.kord[kk], c = im.kcls[kk];
            const float *Hk = Mi.H + (size_t)ku * im.N * im.N;
            for (size_t t = 0; t < im.tile_sb.size(); ++t) {
                const int sb = im.tile_sb[t], a = c ^ sb;
                const int rows = im.tile_rows[t], r8 = (rows + 7) & ~7;
                if (rows == 0 || im.ncls[a] == 0) continue;
                const int kp = im.kpad[a];
                const long long base = (long long)img.size();
                im.tile_off[kk][t] = base;
                img.resize(img.size() + (size_t)r8 * kp, 0.f);
                for (int rr = 0; rr < rows; ++rr) {
                    const int srow = im.gperm[im.ocls[sb] + im.tile_r0[t] + rr];
                    for (int pc = 0; pc < im.ncls[a]; ++pc) {
                        const int scol = im.gperm[im.ocls[a] + pc];
                        const int j = pc / kGrpChunk, w = pc % kGrpChunk;
                        const long long e = base + (long long)j * r8 * kGrpChunk +
                                            (((rr >> 3) * (kGrpChunk / 4) + (w >> 2)) << 5) +
                                            ((rr & 7) << 2) + (w & 3);
                        img[e] = Hk[(size_t)srow * im.N + scol];
                    }
                }
                im.floats += (double)r8 * kp;
            }
        }
        images.push_back(std::move(im));
        image_members.push_back(mem);
    }
    // ---- kernel groups: members of an image in batches of at most Bsub plates
    const int ctrl_bytes = (int)((sizeof(Ctrl) + 1023) & ~size_t(1023));
    const int min_ring = 4;   // at least this many stages beside the Q images
    const int fixed = ctrl_bytes + 2 * min_ring * kGrpStageBytes;
    struct KG {
        int image;
        std::vector<int> plates;
    };
    std::vector<KG> kgs;
    for (size_t ii = 0; ii < images.size(); ++ii) {
        const Image &im = images[ii];
        int sumk = 0;
        for (int a = 0; a < 4; ++a) sumk += im.kpad[a];
        const int nt = (int)im.tile_sb.size();
        // two accumulator sets and the forces in tensor memory; the Q images and
        // at least min_ring stages in shared memory
        int bsub = 32;
        while (bsub > 16 && (3 * nt * bsub > 512 || fixed + 8LL * bsub * sumk > smem_optin)) bsub -= 16;
        if (3 * nt * bsub > 512 || fixed + 8LL * bsub * sumk > smem_optin)
            return bail(gfail(MDX_ERR_UNSUPPORTED, "grouped plate: modes exceed the shared-memory budget"));
        const std::vector<int> &mem = image_members[ii];
        const int nb = (int)((mem.size() + bsub - 1) / bsub);
        for (int q = 0; q < nb; ++q) {
            KG kg;
            kg.image = (int)ii;
            for (size_t x = q; x < mem.size(); x += nb) kg.plates.push_back(mem[x]);
            kgs.push_back(kg);
        }
    }
    const int ng = (int)kgs.size();
    if (ng > n_sms) return bail(gfail(MDX_ERR_UNSUPPORTED, "more plate groups than SMs"));
    // ---- CTAs per kernel group, proportional to the bytes streamed per step
    std::vector<double> work(ng);
    std::vector<int> units_of(ng);
    double total = 0.0;
    for (int g = 0; g < ng; ++g) {
        const Image &im = images[kgs[g].image];
        int mmax = 0;
        for (int i : kgs[g].plates) mmax = std::max(mmax, I[i].n_psi);
        int nu = 0;
        for (int kk = 0; kk < im.M; ++kk)
            if (im.kord[kk] < mmax) ++nu;
        units_of[g] = nu;
        work[g] = im.floats * nu / std::max(im.M, 1);
        total += work[g];
    }
    std::vector<int> ctas(ng, 1);
    int used = ng;
    while (used < n_sms) {
        int best = -1;
        double best_load = -1.0;
        for (int g = 0; g < ng; ++g) {
            if (ctas[g] >= units_of[g]) continue;
            const double load = work[g] / ctas[g];
            if (load > best_load) {
                best_load = load;
                best = g;
            }
        }
        if (best < 0) break;
        ctas[best]++;
        used++;
    }
    // ---- descriptors, units, plates, kappa tables, buffers
    int q_floats_max = 0;
    long long kap_off = 0, part_off = 0, qbuf_off = 0, gpos_base = 0;
    std::vector<long long> gpos_off(images.size());
    for (size_t ii = 0; ii < images.size(); ++ii) {
        gpos_off[ii] = gpos_base;
        gp->gpos.insert(gp->gpos.end(), images[ii].gpos.begin(), images[ii].gpos.end());
        gpos_base += images[ii].N;
    }
    int cta = 0;
    for (int g = 0; g < ng; ++g) {
        const Image &im = images[kgs[g].image];
        GrpDesc d{};
        d.B = (int)kgs[g].plates.size();
        d.Bp = (d.B + 15) / 16 * 16;
        d.N = im.N;
        d.M = im.M;
        d.Np = (im.N + 3) & ~3;
        for (int a = 0; a < 4; ++a) {
            d.ncls[a] = im.ncls[a];
            d.ocls[a] = im.ocls[a];
            d.kpad[a] = im.kpad[a];
        }
        d.n_tiles = (int)im.tile_sb.size();
        for (int t = 0; t < d.n_tiles; ++t) {
            d.tile_sb[t] = im.tile_sb[t];
            d.tile_r0[t] = im.tile_r0[t];
            d.tile_rows[t] = im.tile_rows[t];
        }
        int qf = 0;
        for (int a = 0; a < 4; ++a) {
            d.qoff[a] = qf;
            qf += 2 * d.Bp * d.kpad[a];
        }
        q_floats_max = std::max(q_floats_max, qf);
        d.q_floats = qf;
        d.cta0 = cta;
        d.n_ctas = ctas[g];
        d.plate0 = (int)gp->plates.size();
        d.gpos_off = gpos_off[kgs[g].image];
        d.kap_off = kap_off;
        d.part_off = part_off;
        d.qbuf_off = qbuf_off;
        // units of this group (internal stress order; only modes some plate has)
        int mmax = 0;
        for (int i : kgs[g].plates) mmax = std::max(mmax, I[i].n_psi);
        std::vector<int> ulist;
        for (int kk = 0; kk < im.M; ++kk)
            if (im.kord[kk] < mmax) ulist.push_back(kk);
        const int nu = (int)ulist.size();
        const int unit0 = (int)gp->units.size();
        std::vector<int> ukey;
        for (int x = 0; x < nu; ++x) {
            const int kk = ulist[x];
            GrpUnit U{};
            U.g = g;
            U.row = x;
            U.c = im.kcls[kk];
            for (int t = 0; t < kGrpMaxTiles; ++t) U.off[t] = -1;
            for (int t = 0; t < d.n_tiles; ++t) U.off[t] = im.tile_off[kk][t];
            gp->units.push_back(U);
            ukey.push_back(im.kord[kk]);
            // algorithmic work: the nonzero class block of H^k (rows x columns of class
            // c ^ sb), once per step, applied to the group's B plates
            for (int t = 0; t < d.n_tiles; ++t)
                if (U.off[t] >= 0) {
                    const double nz = (double)d.tile_rows[t] * d.ncls[U.c ^ d.tile_sb[t]];
                    gp->bytes_per_step += 4.0 * nz;
                    gp->flops_per_step += 2.0 * nz * d.B;
                }
        }
        gp->unit_user_k.push_back(ukey);
        // contiguous unit ranges over the group's CTAs
        for (int c = 0; c < d.n_ctas; ++c) {
            gp->cta_group.push_back(g);
            gp->cta_units.push_back(unit0 + (int)((long long)nu * c / d.n_ctas));
            gp->cta_units.push_back(unit0 + (int)((long long)nu * (c + 1) / d.n_ctas));
        }
        // owners: each plate's update costs about its mode count; largest first
        // onto the least-loaded CTA of the group
        std::vector<int> owner_of(d.B), order(d.B);
        std::vector<long long> load(d.n_ctas, 0);
        for (int b = 0; b < d.B; ++b) order[b] = b;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
            return inst[kgs[g].plates[x]].N > inst[kgs[g].plates[y]].N;
        });
        for (int b : order) {
            const int c = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            owner_of[b] = d.cta0 + c;
            load[c] += inst[kgs[g].plates[b]].N;
        }
        std::vector<int> kc, pi;
        for (int b = 0; b < d.B; ++b) {
            GrpPlate pl{};
            pl.inst = kgs[g].plates[b];
            pl.owner = owner_of[b];
            gp->plates.push_back(pl);
            kc.push_back(I[pl.inst].n_psi);   // (the per-instance planner zeroes M)
            pi.push_back(pl.inst);
        }
        gp->plate_kcount.push_back(kc);
        gp->plate_inst.push_back(pi);
        kap_off += (long long)nu * d.Bp;
        part_off += (long long)d.n_ctas * d.Bp * d.Np;
        qbuf_off += (qf + 63) / 64 * 64;   // 256-byte aligned images
        cta += d.n_ctas;
        gp->groups.push_back(d);
    }
    gp->n_ctas = cta;
    gp->kap_floats = kap_off;
    gp->part_floats = part_off;
    gp->qbuf_floats = qbuf_off;
    // shared memory: control block, ring, remainder ring, Q images, the CTA's
    // work units; as many stages as fit (at most 8)
    int max_units = 1;
    for (size_t c = 0; c + 1 < gp->cta_units.size(); c += 2)
        max_units = std::max(max_units, gp->cta_units[c + 1] - gp->cta_units[c]);
    const int unit_bytes = (int)((max_units * sizeof(GrpUnit) + 127) & ~size_t(127));
    const int ring = std::max(min_ring, std::min(8, (smem_optin - ctrl_bytes - q_floats_max * 4 -
                                                     unit_bytes) / (2 * kGrpStageBytes)));
    gp->ring_stages = ring;
    gp->ring_off = ctrl_bytes;
    gp->lo_off = gp->ring_off + ring * kGrpStageBytes;
    gp->q_off = gp->lo_off + ring * kGrpStageBytes;
    gp->scratch_off = gp->q_off + q_floats_max * 4;
    gp->smem = (size_t)gp->scratch_off + unit_bytes;
    if ((int)gp->smem > smem_optin)
        return bail(gfail(MDX_ERR_UNSUPPORTED, "grouped plates exceed the shared-memory budget"));
    // kappa tables stay zero until group_plan_set_kappa
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = gupload(&gp->d_groups, gp->groups);
    if (e == cudaSuccess) e = gupload(&gp->d_units, gp->units);
    if (e == cudaSuccess) e = gupload(&gp->d_cta_group, gp->cta_group);
    if (e == cudaSuccess) e = gupload(&gp->d_cta_units, gp->cta_units);
    if (e == cudaSuccess) e = gupload(&gp->d_plates, gp->plates);
    if (e == cudaSuccess) e = gupload(&gp->d_gpos, gp->gpos);
    if (e == cudaSuccess) e = gupload(&gp->d_img, img);
    if (e == cudaSuccess) e = gupload(&gp->d_kap, std::vector<float>(std::max<long long>(kap_off, 1), 0.f));
    if (e == cudaSuccess) e = cudaMalloc(&gp->d_part, std::max<long long>(part_off, 1) * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&gp->d_qbuf, std::max<long long>(qbuf_off, 1) * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&gp->d_counters, std::max(ng, 1) * sizeof(unsigned));
    // every plan sets the same (largest) limit, so plans of different sizes can
    // launch in any order
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(group_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem_optin);
    if (e != cudaSuccess) {
        const int code = (e == cudaErrorMemoryAllocation) ? MDX_ERR_OOM : MDX_ERR_CUDA;
        return bail(gfail(code, cudaGetErrorString(e)));
    }
    *out = gp;
    return MDX_OK;
}

int group_plan_set_kappa(GroupPlan *g, const std::vector<InstDesc> &inst,
                         const std::vector<double> &kappa_user) {
    std::vector<float> tab(std::max<long long>(g->kap_floats, 1), 0.f);
    for (size_t q = 0; q < g->groups.size(); ++q) {
        const GrpDesc &d = g->groups[q];
        const std::vector<int> &uk = g->unit_user_k[q];
        for (int b = 0; b < d.B; ++b) {
            const InstDesc &id = inst[g->plate_inst[q][b]];
            const int Mb = g->plate_kcount[q][b];
            for (size_t x = 0; x < uk.size(); ++x)
                if (uk[x] < Mb)
                    tab[d.kap_off + (long long)x * d.Bp + b] = (float)kappa_user[id.k_off + uk[x]];
        }
    }
    cudaError_t e = cudaSetDevice(g->device);
    if (e == cudaSuccess)
        e = cudaMemcpy(g->d_kap, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return gfail(MDX_ERR_CUDA, cudaGetErrorString(e));
    return MDX_OK;
}

cudaError_t group_plan_launch(GroupPlan *g, const InstDesc *d_inst, const ModeCoef &coef,
                              int steps, int total_steps, const float *exc, float *audio,
                              float *state_io, long long total_modes, int *status, int *abort_flag,
                              float l2_keep, cudaStream_t s) {
    if (!g || g->n_ctas == 0 || steps <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(g->d_counters, 0, g->groups.size() * sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->d_qbuf, 0, g->qbuf_floats * sizeof(float), s);
    if (e != cudaSuccess) return e;
    GroupParams P{};
    P.inst = d_inst;
    P.groups = g->d_groups;
    P.units = g->d_units;
    P.cta_group = g->d_cta_group;
    P.cta_units = g->d_cta_units;
    P.plates = g->d_plates;
    P.gpos = g->d_gpos;
    P.kap = g->d_kap;
    P.img = g->d_img;
    P.part = g->d_part;
    P.qbuf = g->d_qbuf;
    P.coef = coef;
    P.steps = steps;
    P.n_begin = 0;
    P.total_steps = total_steps;
    P.exc = exc;
    P.audio = audio;
    P.state_io = state_io;
    P.total_modes = total_modes;
    P.counters = g->d_counters;
    P.status = status;
    P.abort_flag = abort_flag;
    P.wait_limit = g->wait_limit;
    P.ring_stages = g->ring_stages;
    P.ring_off = g->ring_off;
    P.lo_off = g->lo_off;
    P.q_off = g->q_off;
    P.scratch_off = g->scratch_off;
    P.l2_keep = l2_keep;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(g->n_ctas);
    cfg.blockDim = dim3(kGrpThreads);
    cfg.dynamicSmemBytes = g->smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, group_kernel, P);
}

}  // namespace mdx
