// Internal layout of an mdx plan, shared by the host planner and the kernels.
//
// Modal state on the device uses the difference form of the Stormer-Verlet
// update (Sec. 3.2, Eq. 20-23 rewritten exactly):
//     v^{n+1} = v^n - eps v^n - (r omega^2) q^n + r (b e^n - fnl(q^n)),
//     q^{n+1} = q^n + v^{n+1},
// with v^n = q^n - q^{n-1}, eps = 2 gamma T / (1 + gamma T),
// r = T^2 / (1 + gamma T).  q and v are carried as unevaluated FP32 pairs
// (hi + lo, compensated addition) and r omega^2 as an FP32 pair: the per-step
// increments are small against the values, and plain FP32 would accumulate
// a phase drift of order 1e-5 over 1e4-1e5 steps.  The nonlinear force is
// evaluated at q_hi.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/mdx.h"

namespace mdx {

constexpr int kPlateThreads = 256;     // consumer threads of the plate kernel
constexpr int kPlateWarps = kPlateThreads / 32;
constexpr int kProducerWarps = 1;      // one warp issues the TMA bulk copies
constexpr int kPlateBlock = kPlateThreads + 32 * kProducerWarps;
constexpr int kStateArrays = 4;      // q_hi, q_lo, v_hi, v_lo
constexpr int kMaxSpt = 4;             // modes per consumer thread (N_pad <= 1024)
constexpr int kChunkK = 4;             // stress modes reduced together
constexpr int kUPartFloats = 1024;     // row groups x N_pad <= 256 threads x 4 columns
constexpr int kParQmax = 2;            // parity layout: column quads per thread
constexpr int kParMcMax = 16;          // parity layout: stress modes per chunk
constexpr int kTensionWarpsPerBlock = 4;
constexpr int kTensionMaxJ = 32;       // modes per lane (N <= 1024)

enum KernelMode : int {
    MODE_FORWARD = 0,   // simulate: writes audio / checkpoints / final state
    MODE_RECOMPUTE = 1, // re-run one segment from a checkpoint, storing every state
    MODE_REVERSE = 2,   // adjoint sweep over one stored segment
    MODE_FUSED = 4,     // adjoint sweep over segment s and recompute of segment s-1 in
                        // one pass over the coupling tensor per step (class layout)
};

// Per-mode FP32 coefficients, concatenated over instances (struct of arrays).
struct ModeCoef {
    const float *eps;   // 2 gamma T / (1 + gamma T)
    const float *rw2;   // r omega^2 (high part)
    const float *rw2lo; // r omega^2 - rw2 (low part)
    const float *r;     // T^2 / (1 + gamma T)
    const float *b;     // input weight
    const float *c;     // pickup weight
    const float *lam;   // Laplacian eigenvalue (tension kind)
    const float *clo;   // c - (float)c (low part of the pickup weight)
};

struct InstDesc {
    int kind;           // MDX_KIND_TENSION / MDX_KIND_PLATE
    int N;              // transverse modes
    int M;              // stress modes (0 for tension / linear)
    int Npad;           // row stride of H (multiple of 4 floats)
    long long mode_off; // offset into per-mode arrays
    long long H_off;    // float offset of H^0 (layout [M][N][Npad])
    long long k_off;    // offset into per-stress-mode arrays (kappa, d_kappa)
    float taup;         // tension coefficient / density
    int n_contrib;      // plate: number of CTAs holding a part of the k range
    long long part_off; // plate: first exchange slot (slots are [n_contrib][3][Npad])
    int has_dir;        // plate: a direction tensor dH is present
    int grouped;        // plate: simulated by the grouped kernel (shared coupling tensor)
    long long dH_off;   // float offset of dH^0 (same layout as H)
    // symmetry-class layout (parity != 0): transverse modes in class order
    int parity;
    int ncls[4];        // transverse modes per class
    int ocls[4];        // first class-ordered position of each class
    long long perm_off; // perm[perm_off + class position] = mode index within the instance
};

// One class chunk of a plate item (parity layout): mc consecutive internal
// stress modes, all of class c, starting at internal index kl0.  Its coupling
// data is four super-blocks a = 0..3 (rows p of class a, columns s of class
// b = a ^ c), each stored as [p][k in chunk][s padded to 4] at float offset
// off (H) and doff (dH).
struct ParityChunk {
    int c, kl0, mc, pad;
    long long off, doff;
};

// One contiguous range of stress modes of one plate, processed by one CTA.
struct PlateItem {
    int inst;
    int k0, k1;         // stress modes [k0, k1)
    int slot;           // this CTA's index among the instance's contributors
    int owner;          // 1: this CTA writes audio / state / gradients of the instance
    int smem_state;     // float offset of this item's state block in shared memory
    int chunk0, chunk1; // parity layout: the item's class chunks
    int cache;          // 1: per-mode coefficients, class permutation and (owner)
                        // gradient sums are kept in the item's shared-memory block
    int pad;
};

// Shared-memory state block of one item (floats, each of length Npad).
enum StateArr : int {
    ST_QHI = 0, ST_QLO, ST_V, ST_VLO,  // forward / recompute state (reverse: a_hi, a_lo, mu)
    ST_FLOC,                        // local partial force (forward) / J w (reverse)
    ST_SRC0, ST_SRC1,               // right-hand sides of the H pass (reverse: q^n, w)
    ST_FLOC2,                       // reverse: local partial force at q^n
    ST_QP, ST_WP,                   // parity layout: right-hand sides in class order
    ST_NARR,
    // fused sweep only: the recompute state of the previous segment
    ST_RQHI = ST_NARR, ST_RQLO, ST_RV, ST_RVLO,
    ST_RFLOC,                       // local partial force at the recompute state
    ST_RQP,                         // recompute state in class order
    ST_NARR_FUSED
};

// Accumulators of the reverse sweep, per mode (compensated FP32 pairs).
enum GradAcc : int {
    GA_A = 0,   // sum a^{n+1} q^n
    GA_V,       // sum a^{n+1} v^n
    GA_F,       // sum a^{n+1} (b e^n - fnl^n)
    GA_E,       // sum a^{n+1} e^n
    GA_C,       // sum ybar^n q^{n+1}
    GA_N
};

// Persistent adjoint state between segment launches (per mode):
// a_hi, a_lo (adjoint a^{n+1}), mu = a^{n+1} - a^{n+2}.
enum AdjArr : int { AD_HI = 0, AD_LO, AD_MU, AD_N };

struct PlateParams {
    const InstDesc *inst;
    const PlateItem *items;
    const int *cta_item_off;      // [gridDim+1]
    ModeCoef coef;
    const float *H;
    const float *dH;
    const float *kappa;           // [total stress modes]
    int n_inst;
    int steps;                    // steps of this launch
    int n_begin;                  // global step index of the first step
    int total_steps;              // steps of the whole simulate call (exc / audio row length)
    int mode;                     // KernelMode
    int stage_bytes;
    int ring_stages;
    int u_slots;                  // row-group partial-sum slots: 1 forward, 2-3 reverse
    int u_floats;                 // floats of the partial-sum region
    int parity;                   // 1: coupling in symmetry-class chunks
    int npad_max;                 // parity layout: row stride of the per-chunk u buffer
    const ParityChunk *chunks;
    const int *perm;
    int max_spt;
    int smem_state_floats;
    // forward I/O
    const float *exc;             // [n_inst][total_steps]
    float *audio;                 // [n_inst][total_steps]
    float *state_io;              // [4][total_modes] q_hi, q_lo, v_hi, v_lo in / out
    int ckpt_K;
    float *ckpt;                  // [n_ckpt][4][total_modes]
    float *seg_q;                 // recompute/reverse: [(steps+1)][total_modes] q_hi^n
    float *seg_v;                 // recompute/reverse: [(steps+1)][total_modes] v^n
    // fused sweep: the reverse covers rev_steps (<= steps) steps from n_begin and
    // reads seg_q / seg_v; the recompute runs steps steps from rec_begin (a
    // checkpoint) and writes rseg_q / rseg_v
    int rev_steps;
    int rec_begin;
    float *rseg_q;
    float *rseg_v;
    long long total_modes;
    // reverse I/O
    const float *ybar;            // [n_inst][total_steps]
    float *adj;                   // [AD_N][total_modes]
    float *gacc;                  // [GA_N][2][total_modes]
    float *kacc;                  // [total stress modes][2] d kappa (Kahan pair)
    float *seg_w;                 // reverse: [steps][total_modes] w^n = r a^{n+1} (owners)
    float *xe;                    // reverse: [steps][2][total_k] xi_k^n, eta_k^n
    int xe_all;                   // 1: store xi, eta for every plate (full dL/dH), else
                                  // only for plates with a direction tensor
    long long total_k;
    // synchronisation
    float *part;                  // exchange slots, two parities of part_stride floats
    long long part_stride;
    unsigned *counters;           // [n_inst]
    int *status;                  // [n_inst] or nullptr
    int *abort_flag;
    long long wait_limit;
    int debug_flags;
    float l2_keep;                // fraction of the coupling stream kept in L2 (0: no hint)
};

// One (plate, stress mode) of the directional-derivative contraction.
struct DirUnit {
    int inst;
    int kl;            // internal stress index within the plate
    int c, mc, kpos;   // class layout: class, chunk size, position in the chunk
    int pad;
    long long off;     // class layout: float offset of the chunk's dH super-blocks
};

// Class layout: all stress modes of class c of one plate against row class a.
struct DirGroup {
    int inst, c, a;
    int unit0, nk;     // the class-c stress modes: units[unit0 .. unit0 + nk)
    int pad;
};

struct DirParams {
    const InstDesc *inst;
    const DirUnit *units;
    const DirGroup *groups;
    int n_groups;
    const float *dH;
    const int *perm;
    const float *kappa;
    const float *seg_q;           // [(steps+1)][total_modes]
    const float *seg_w;           // [steps][total_modes]
    const float *xe;              // [steps][2][total_k]
    double *dir_acc;              // [total_k][4] (class layout: one slot per row class)
    int steps;
    long long total_modes, total_k;
    // full dL/dH: -kappa_k G_k accumulated into the user-layout output
    double *dH_out;               // [per plate: M][N][N]
    const long long *dh_off;      // [n_inst] double offset of each plate's block
    const int *kperm;             // internal stress index -> user index (at k_off)
    // tensor-core contraction (class layout): K columns staged per chunk
    // (multiple of 8; 0 = CUDA-core kernels), B-operand row capacity, status
    int tc_kc, tc_nmax;
    size_t tc_smem;
    int *status;
};

// Cluster-resident plates: one thread-block cluster per plate, the plate's
// coupling rows held in registers for the whole launch (forward pass).
struct ClusterK {
    long long off;     // float offset of the stress mode's class chunk (H)
    int mc, kpos, c;   // chunk size, position in the chunk, class
    int pad;
};

struct ClusterParams {
    const InstDesc *inst;
    const int *plates;            // plate instance indices (one cluster each)
    const ClusterK *kinfo;        // [total_k]
    const float *H;
    const float *kappa;
    const int *perm;
    ModeCoef coef;
    int cs;                       // CTAs per cluster
    int nkc;                      // stress-mode slots per CTA
    int wk;                       // warps per slot (rows: class-ordered modes)
    int steps, n_begin, total_steps;
    const float *exc;
    float *audio;
    float *state_io;              // [4][total_modes]: q_hi, q_lo, v_hi, v_lo
    long long total_modes;
    int *status;
};

// Row length (floats) of the register-resident coupling rows: 32 or 64; 0
// when a plate does not fit.  cluster_plan picks the cluster shape.
int cluster_row_len(int max_class);
int cluster_max_threads(int row_len);
cudaError_t launch_cluster(const ClusterParams &P, int n_plates, int row_len, cudaStream_t s);
cudaError_t cluster_check(int cs, int threads, int row_len, int *max_clusters);

struct TensionParams {
    const InstDesc *inst;
    const int *list;              // tension instance indices
    int n_list;
    ModeCoef coef;
    int steps, n_begin, total_steps, mode;
    const float *exc;
    float *audio;
    float *state_io;
    int ckpt_K;
    float *ckpt;
    float *seg_q, *seg_v;
    long long total_modes;
    const float *ybar;
    float *adj;
    float *gacc;
    float *tacc;                  // [n_inst][2] d tau' (Kahan sum, compensation)
    int *status;
};

// ---------------------------------------------------------------- grouped plates
// Plates that share one coupling tensor (same geometry: their modes are
// prefixes of the largest member's, Sec. 3, Eq. 2 and Eq. 10) are stepped
// together: per step and stress mode k, U^k = H^k [q_1 ... q_B] is one
// tensor-core GEMM over the plates of the group (split TF32 on tcgen05, FP32
// accumulation in tensor memory), see mdx_group.cu.
constexpr int kGrpThreads = 256;      // 8 warps: producer, MMA, 2 converters, 4 epilogue
constexpr int kGrpChunk = 16;         // K elements (columns of H^k) per ring stage
constexpr int kGrpStageBytes = 128 * kGrpChunk * 4;   // one 128-row stage (8 KB)
constexpr int kGrpMaxTiles = 16;      // (row class, 128-row tile) blocks per stress mode
constexpr int kGrpMaxB = 64;          // plates per kernel group

// One kernel group: up to kGrpMaxB plates stepped together on one coupling image.
struct GrpDesc {
    int B, Bp;              // plates, padded to a multiple of 16 (the MMA's N)
    int N, M;               // transverse / stress modes of the image (largest member)
    int Np;                 // row stride of the class-ordered buffers (N rounded up to 4)
    int ncls[4], ocls[4];   // transverse modes per class, class-order offset of each class
    int kpad[4];            // class sizes rounded up to kGrpChunk (K of the MMAs)
    int n_tiles;
    int tile_sb[kGrpMaxTiles];    // row class of each tile
    int tile_r0[kGrpMaxTiles];    // first row within the class
    int tile_rows[kGrpMaxTiles];  // rows (<= 128)
    int cta0, n_ctas;       // CTAs [cta0, cta0 + n_ctas) hold this group's stress modes
    int plate0;             // plates: GroupParams::plates[plate0 .. plate0 + B)
    int qoff[4];            // shared-memory float offset of class a's Q image [Bp][kpad[a]]
                            // (its low part follows at qoff[a] + Bp * kpad[a])
    long long gpos_off;     // gpos[gpos_off + j] = class position of mode j
    long long kap_off;      // kappa table [units of the group][Bp], 0 where a plate lacks the mode
    long long part_off;     // partial forces [n_ctas][Bp][Np] (class order)
    long long qbuf_off;     // the group's Q image in global memory (the layout of the
                            // shared-memory Q region), written by the owners
    int q_floats;           // floats of the Q region (all classes, high and low parts)
    int pad2;
};

// One stress mode of a kernel group (the MMA and epilogue work unit).
struct GrpUnit {
    int g;                  // kernel group
    int row;                // row of the group's kappa table
    int c;                  // symmetry class of the stress mode
    int pad;
    long long off[kGrpMaxTiles];   // float offset of each tile's image (-1: empty block)
};

struct GrpPlate {
    int inst;               // instance index
    int owner;              // CTA that steps this plate's state
};

struct GroupParams {
    const InstDesc *inst;
    const GrpDesc *groups;
    const GrpUnit *units;
    const int *cta_group;         // [grid] kernel group of each CTA
    const int *cta_units;         // [grid][2] unit range of each CTA
    const GrpPlate *plates;
    const int *gpos;
    const float *kap;
    const float *img;             // coupling images (tile chunks, see mdx_group.cu)
    float *part, *qbuf;
    ModeCoef coef;
    int steps, n_begin, total_steps;
    const float *exc;
    float *audio;
    float *state_io;              // [4][total_modes]
    long long total_modes;
    unsigned *counters;           // [kernel groups]
    int *status;
    int *abort_flag;
    long long wait_limit;
    int ring_stages;
    int ring_off, lo_off, q_off, scratch_off;   // shared-memory byte offsets
    float l2_keep;
};

// Linear response parallel in time (mdx_linear.cu): chunks of kLinChunk steps.
constexpr int kLinChunk = 256;
struct LinearParams {
    const InstDesc *inst;
    int n_inst;
    const int *mode_inst;           // [total_modes] instance of each mode
    const double *omega2, *gamma, *dt, *b, *c;   // per mode FP64
    int scheme;
    int steps, total_steps, L, n_chunks;
    const float *exc;               // [n_inst][total_steps] or nullptr
    const double *q0, *qm1;         // [total_modes] or nullptr
    float *audio;                   // [n_inst][total_steps] or nullptr
    double *q_end, *qm1_end;        // [total_modes] or nullptr
    double *E, *S;                  // [n_chunks][total_modes][2] each
    long long total_modes;
    int *status;
};
cudaError_t launch_linear(const LinearParams &P, cudaStream_t s);

struct GroupPlan;   // host side of the grouped path (mdx_group.cu)
// Builds the grouped path for the plates with grouped[i] != 0 (host FP32 H,
// classes and kappa from the instance descriptions); fails with an MDX_ERR_*.
int group_plan_build(GroupPlan **out, const mdx_instance *I, const std::vector<InstDesc> &inst,
                     const std::vector<int> &grouped, int device, int n_sms, int smem_optin,
                     long long wait_limit);
void group_plan_free(GroupPlan *g);
int group_plan_ctas(const GroupPlan *g);
double group_plan_bytes_per_step(const GroupPlan *g);
double group_plan_flops_per_step(const GroupPlan *g);
// kappa of every plate (user order, concatenated over all instances' stress modes)
int group_plan_set_kappa(GroupPlan *g, const std::vector<InstDesc> &inst,
                         const std::vector<double> &kappa_user);
cudaError_t group_plan_launch(GroupPlan *g, const InstDesc *d_inst, const ModeCoef &coef,
                              int steps, int total_steps, const float *exc, float *audio,
                              float *state_io, long long total_modes, int *status, int *abort_flag,
                              float l2_keep, cudaStream_t s);

// Sets the thread-local message returned by mdx_last_error; returns code.
int set_last_error(int code, const char *msg);

// Launchers (defined in the kernel translation units).
size_t plate_smem_bytes(int ring_stages, int stage_bytes, int u_floats, int state_floats);
cudaError_t launch_plate(const PlateParams &p, int grid, size_t smem, cudaStream_t s);
cudaError_t plate_set_smem_limit(size_t smem);
cudaError_t launch_tension(const TensionParams &p, int max_n, cudaStream_t s);

struct AuxInit {
    const double *q0, *qm1;      // [total_modes] or nullptr
    float *state;                // [4][total_modes]
    long long total_modes;
};
cudaError_t launch_init_state(const AuxInit &a, cudaStream_t s);
cudaError_t launch_finalize_state(const float *state, long long total_modes, double *q_end,
                                  double *qm1_end, cudaStream_t s);
// a^{steps} = c ybar^{steps-1}, mu^{steps} = a^{steps}; every mode of every instance.
cudaError_t launch_init_adjoint(const InstDesc *inst, int n_inst, const float *c,
                                const float *ybar, int steps, float *adj, long long total_modes,
                                int max_n, cudaStream_t s);

struct GradEpilogue {
    const InstDesc *inst;
    int n_inst;
    long long total_modes, total_k;
    const double *omega2, *gamma, *dt;  // per mode FP64
    const float *adj, *gacc, *kacc, *tacc;
    const double *dir_acc;
    const int *kperm;                   // internal stress index -> user index (per plate)
    int scheme;                         // MDX_SCHEME_SV / MDX_SCHEME_TF
    double *d_omega2, *d_gamma, *d_b, *d_c, *d_q0, *d_qm1, *d_tau, *d_kappa, *d_dir;
};
cudaError_t launch_grad_epilogue(const GradEpilogue &g, int max_n, cudaStream_t s);
cudaError_t launch_dir_contract(const DirParams &p, int n_units, cudaStream_t s);
// Shared memory of the tensor-core contraction for a K chunk of kc columns and
// nmax B-operand rows; dir_tc_configure sets the kernel's opt-in limit (the
// planner passes the device maximum, since every plan shares the kernel).
size_t dir_tc_smem_bytes(int kc, int nmax);
cudaError_t dir_tc_configure(size_t smem);
// Adds -kappa_k G_k of one segment into p.dH_out (units / groups over every plate).
cudaError_t launch_dH_accumulate(const DirParams &p, int n_units, cudaStream_t s);
// dH_out[k][i][j] = dH_out[k][j][i] = their mean, for every plate.
cudaError_t launch_dH_symmetrize(double *dH, const long long *dh_off, const InstDesc *inst,
                                 const int *plates, int n_plates, cudaStream_t s);

}  // namespace mdx
