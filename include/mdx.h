/*
 * mdx.h - C ABI of the GB300 modal-synthesis library (libmdx.so).
 *
 * The library runs the per-time-step modal update of nonlinear strings,
 * membranes and plates (Diaz & Sandler, "Fast Differentiable Modal
 * Simulation of Non-linear Strings, Membranes, and Plates", DAFx25):
 *
 *   modal oscillators              Sec. 3.2, Eq. 12-14
 *   Stormer-Verlet update          Sec. 3.2, Eq. 20-23
 *     q^{n+1} = g q^n + p q^{n-1} + r (fext^n - fnl^n)
 *   tension modulation (strings, membranes)        Sec. 3.1, Eq. 8
 *     fnl_mu = tau' lambda_mu q_mu sum_nu lambda_nu q_nu^2
 *   von Karman coupling (plates)   Sec. 3.1, Eq. 9, with C^s_pn = H^n_ps (Sec. 4.3.3)
 *     eta_n = sum_pq H^n_pq q_p q_q,  fnl_s = sum_n kappa_n eta_n sum_p H^n_ps q_p
 *   pickup                         y^n = sum_mu c_mu q^{n+1}_mu
 *
 * and its reverse-mode derivative (adjoint time loop with checkpoints).
 *
 * Conventions shared by every entry point
 *   - Every call returns an int status: MDX_OK (0) or one of MDX_ERR_*.
 *     mdx_last_error() returns a thread-local message for the last failure.
 *   - "device" pointers are CUDA global-memory addresses on the plan's
 *     device; "host" pointers are ordinary CPU memory.  The caller owns every
 *     buffer it passes; the library never frees caller memory and keeps no
 *     reference to host arrays after a call returns.
 *   - Work is enqueued asynchronously on the given cudaStream_t (passed as
 *     void*, NULL = legacy default stream).  Device-side failures (non-finite
 *     state, a synchronisation wait that gave up) are reported per instance in
 *     the optional `status` array once the stream has reached that point.
 *   - Modes of all instances are concatenated in plan order: instance i owns
 *     modes [mode_offset(i), mode_offset(i) + n_phi(i)).
 *   - Calls that share a plan share its scratch memory: do not run two calls
 *     on the same plan concurrently on different streams.
 */
#ifndef MDX_H
#define MDX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MDX_OK 0
#define MDX_ERR_ARG 1          /* invalid argument (message names the instance / mode) */
#define MDX_ERR_UNSTABLE 2     /* coefficients outside the scheme's stability region */
#define MDX_ERR_NONFINITE 3    /* non-finite input or state */
#define MDX_ERR_TIMEOUT 4      /* a bounded device-side wait gave up */
#define MDX_ERR_CUDA 5         /* a CUDA runtime call failed */
#define MDX_ERR_OOM 6          /* device allocation failed */
#define MDX_ERR_UNSUPPORTED 7  /* size or feature outside the library's limits */

#define MDX_KIND_TENSION 0     /* string (Kirchhoff-Carrier) or membrane (Berger) */
#define MDX_KIND_PLATE 1       /* von Karman plate */

/* Time discretisation of the modal oscillators (Sec. 3.2). */
#define MDX_SCHEME_SV 0        /* Stormer-Verlet, Eq. 20-23 (default) */
#define MDX_SCHEME_TF 1        /* impulse invariance, Eq. 15-19: the recursion takes the
                                  denominator's roots (-a1, -a2) and b1 carries the factor T
                                  of a sampled force; oscillatory modes only (omega > gamma) */

#define MDX_MAX_PHI 1024       /* transverse modes per instance */
#define MDX_MAX_PSI 1024       /* stress modes per instance */

/*
 * One simulated object, described by its modal coefficients (Sec. 3.2, Eq. 12).
 * All arrays are host memory, read during mdx_plan_create only.
 *   kind     MDX_KIND_TENSION or MDX_KIND_PLATE
 *   n_phi    N, number of transverse modes, 1..MDX_MAX_PHI
 *   n_psi    M, number of in-plane stress modes (plate; 0 = linear plate)
 *   dt       sampling period T > 0 (s)
 *   omega2   [N] squared angular frequencies omega_mu^2 > 0 (Eq. 13)
 *   gamma    [N] damping rates gamma_mu >= 0 (Eq. 14)
 *   b        [N] input weights: fext^n_mu = b_mu e^n
 *   c        [N] pickup weights: y^n = sum c_mu q^{n+1}_mu
 *   lambda   [N] Laplacian eigenvalues (tension kind; may be NULL for plates)
 *   tau      tau' = tension-modulation coefficient / mass density (tension kind)
 *   H        [M][N][N] coupling tensor H^k_ij (Eq. 10), FP32, symmetric in i, j
 *   kappa    [M] kappa_k = E / (2 rho zeta_k^4) (Eq. 9)
 *   dH       optional [M][N][N] FP32 direction tensor (e.g. dH/d aspect) for
 *            mdx_grad's directional derivative <dL/dH, dH>; NULL if unused
 *   phi_class, psi_class  optional [N] and [M] symmetry classes in 0..3 (plate).
 *            For a simply supported rectangle, L(Phi_i, Phi_j) (Eq. 7) is odd
 *            about a mid-line when exactly one of Phi_i, Phi_j is, so H^k_ij
 *            (Eq. 10) vanishes unless phi_class[i] ^ phi_class[j] == psi_class[k]
 *            (bit 1: odd about x = Lx/2, bit 0: odd about y = Ly/2).  When
 *            every plate of a plan gives classes, the plan stores and streams
 *            only the nonzero class blocks (a quarter of H).  The plan checks
 *            the pattern: an entry outside it larger than 1e-6 max|H^k| fails
 *            with MDX_ERR_ARG; smaller ones are treated as zero.
 *   geom_group  plates of one geometry (> 0; 0 = none).  Plates with the same
 *            id share their modes: for a simply supported rectangle of fixed
 *            area and aspect ratio, a plate with fewer modes has a prefix of
 *            the largest member's transverse and stress modes (Sec. 3, Eq. 2),
 *            so its H (Eq. 10) is the leading block of the largest member's.
 *            The plan checks that (bit for bit), and that the member with the
 *            most transverse modes also has the most stress modes; classes are
 *            required.  Unless mdx_options.group_engine is MDX_GROUP_OFF, such
 *            plates are stepped together: per step and stress mode, H^k times
 *            the group's states is one GEMM on the tensor cores (split TF32,
 *            FP32 accumulation; error about 2^-21 of |H||q|, like FP32).
 *            Plans with grouped plates simulate only: checkpoints and mdx_grad
 *            fail with MDX_ERR_UNSUPPORTED (plan with MDX_GROUP_OFF to
 *            differentiate them).
 * Stability: every mode needs omega_mu * dt < 2 (Eq. 20 is explicit);
 * otherwise mdx_plan_create fails with MDX_ERR_UNSTABLE naming the mode.
 */
typedef struct mdx_instance {
    int kind;
    int n_phi;
    int n_psi;
    double dt;
    const double *omega2;
    const double *gamma;
    const double *b;
    const double *c;
    const double *lambda;
    double tau;
    const float *H;
    const double *kappa;
    const float *dH;
    const int *phi_class;
    const int *psi_class;
    int geom_group;
} mdx_instance;

/* Plan options; zero-initialise for defaults. */
typedef struct mdx_options {
    int device;        /* CUDA device ordinal of the plan (default 0) */
    int max_ctas;      /* cap on persistent CTAs for the plate kernel (0 = one per SM) */
    int ring_stages;   /* TMA ring depth of the plate kernel (0 = default) */
    int stage_bytes;   /* bytes per ring stage (0 = default; multiple of 16) */
    int force_split;   /* >0: split every plate over at least this many CTAs (tests) */
    int wait_limit;    /* >0: spin-iteration cap of device waits (tests); 0 = default */
    int debug_flags;   /* bit 0: the second contributor of every shared plate withholds its
                          arrival, so the other contributors' bounded waits run out and the
                          call reports MDX_ERR_TIMEOUT (fault-path tests);
                          bit 1: run the gradient as separate recompute and reverse launches
                          instead of the fused sweep (equivalence tests);
                          bit 2: keep no per-plate coefficients or gradient sums in the plate
                          kernel's shared memory (the path of plates too large for it;
                          equivalence tests);
                          bit 3: run the direction contraction on the CUDA-core kernel instead
                          of the tensor cores (equivalence tests);
                          bit 4: run forward passes on the streaming plate kernel even where
                          the plates fit cluster-resident (equivalence tests); 0 in normal use */
    int scheme;        /* MDX_SCHEME_SV (default) or MDX_SCHEME_TF */
    int group_engine;  /* plates with geom_group > 0: MDX_GROUP_TF32X3 (default) steps each
                          group with one shared coupling tensor on the tensor cores;
                          MDX_GROUP_OFF gives every plate its own copy (FP32 CUDA-core path) */
} mdx_options;

#define MDX_GROUP_TF32X3 0
#define MDX_GROUP_OFF 1

typedef struct mdx_plan mdx_plan;

/* Thread-local description of the last error of this thread (never NULL). */
const char *mdx_last_error(void);

/* Library version string. */
const char *mdx_version(void);

/*
 * Build a plan: validates every instance, computes the FP32 difference-form
 * coefficients (eps = 2 gamma T / (1 + gamma T), r omega^2, r = T^2/(1+gamma T),
 * algebraically equal to Eq. 21-23), copies H into the device layout and
 * builds the work assignment.  The plan owns all device memory it allocates.
 *   out      receives the plan (set to NULL on failure)
 *   inst     [n_inst] instance descriptions (host)
 *   opts     options or NULL
 * Errors: MDX_ERR_ARG, MDX_ERR_UNSTABLE, MDX_ERR_NONFINITE, MDX_ERR_UNSUPPORTED,
 *         MDX_ERR_OOM, MDX_ERR_CUDA.
 */
int mdx_plan_create(mdx_plan **out, const mdx_instance *inst, int n_inst,
                    const mdx_options *opts);

/*
 * Replace the per-mode coefficients of a plan without rebuilding it (the
 * coupling tensors and the work assignment stay): host FP64 arrays over all
 * modes in plan order (omega2 and gamma of Eq. 13-14, b, c; NULL keeps the
 * current values), tau [n_inst] (tension instances; NULL keeps) and kappa of
 * Eq. 9 over all stress modes in plan order (NULL keeps).  The FP32
 * difference-form coefficients of Eq. 20-23 are recomputed from them.  Used
 * by every iteration of an inverse fit (Sec. 4.3).  Validated like
 * mdx_plan_create; on error the plan is unchanged.  Synchronises the plan's
 * device.  Errors: MDX_ERR_ARG, MDX_ERR_UNSTABLE, MDX_ERR_NONFINITE,
 * MDX_ERR_CUDA.
 */
int mdx_plan_set_coefficients(mdx_plan *plan, const double *omega2, const double *gamma,
                              const double *b, const double *c, const double *tau,
                              const double *kappa);

/*
 * Linear response of every instance of the plan, parallel in time (Sec.
 * 4.3.2: the linear modes evolve by repeated multiplication with their
 * discrete poles, evaluated as a prefix scan over time).  The nonlinear terms
 * are dropped (tau' and kappa ignored); every mode follows the plan scheme's
 * recursion q^{n+1} = g q^n + p q^{n-1} + r b e^n exactly (Eq. 20-23, or Eq.
 * 15-19), written as X^{n+1} = A X^n + (r b e^n, 0) with the companion matrix
 * A of the mode's poles.  Time is cut into chunks of 256 steps: each chunk's
 * response to its own input from rest, then the chunk boundary states
 * S_j = A^256 S_{j-1} + E_j, then every chunk again from its true state with
 * the pickup.  FP64 arithmetic, FP32 audio.  Arguments as in mdx_simulate;
 * work is caller-owned device scratch of mdx_linear_workspace_bytes(plan,
 * steps).  Asynchronous on `stream`.  Errors: MDX_ERR_ARG (workspace, steps),
 * MDX_ERR_CUDA.
 */
size_t mdx_linear_workspace_bytes(const mdx_plan *plan, int steps);
int mdx_simulate_linear(mdx_plan *plan, const float *exc, const double *q0, const double *qm1,
                        int steps, float *audio, double *q_end, double *qm1_end, void *work,
                        size_t work_bytes, int *status, void *stream);

/*
 * Replace the coupling tensor H (Eq. 10) of plate `inst` in a plan, and its
 * direction tensor dH if the plate was planned with one (dH NULL keeps it):
 * host FP32 [M][N][N], symmetric in the last two indices, read during the call
 * only.  Used when H itself is fitted (Sec. 4.3.3: the coupling coefficients of
 * the von Karman plate are optimised from a random initialisation).  A plan in
 * the symmetry-class layout stores only the class pattern, so the new H must
 * follow it (entries outside it at most 1e-6 of max |H^k|); plan without
 * classes (dense layout) to fit an unstructured H.  Synchronises the plan's
 * device.  Errors: MDX_ERR_ARG (index, symmetry, class pattern),
 * MDX_ERR_NONFINITE, MDX_ERR_UNSUPPORTED (a grouped plate), MDX_ERR_CUDA.
 */
int mdx_plan_set_coupling(mdx_plan *plan, int inst, const float *H, const float *dH);

/*
 * Host FP64 coefficients of the difference form the kernels step (Sec. 3.2):
 *   v^{n+1} = v^n - eps v^n - rho q^n + r F^n,  q^{n+1} = q^n + v^{n+1},
 * i.e. the recursion q^{n+1} = g q^n + p q^{n-1} + r F^n of Eq. 20 (scheme
 * MDX_SCHEME_SV, Eq. 21-23) or of Eq. 19 (MDX_SCHEME_TF, Eq. 16-18) with
 * eps = 1 + p and rho = 1 - g - p, for n modes of period T.  Arrays are host
 * memory of n doubles.  Errors: MDX_ERR_ARG (null array, unknown scheme, T <= 0),
 * MDX_ERR_UNSTABLE (SV: omega T >= 2; TF: omega <= gamma; either: gamma < 0).
 */
int mdx_difference_coefficients(int scheme, int n, const double *omega2, const double *gamma,
                                double T, double *eps, double *rho, double *r);

/*
 * Host FP64 chain rule from the adjoint sums of the reverse sweep,
 * A = sum a^{n+1} q^n, V = sum a^{n+1} v^n, F = sum a^{n+1} F^n (so that
 * dL/d rho = -A, dL/d eps = -V, dL/d r = F), to dL/d omega^2 and dL/d gamma
 * for the scheme's coefficients (Sec. 3.2: Eq. 21-23 for MDX_SCHEME_SV,
 * Eq. 16-18 for MDX_SCHEME_TF); the gradient epilogue of mdx_grad runs the
 * same function on the device.  Arrays of n doubles, host memory.
 * Errors: as mdx_difference_coefficients.
 */
int mdx_coefficient_grads(int scheme, int n, const double *omega2, const double *gamma,
                          double T, const double *A, const double *V, const double *F,
                          double *d_omega2, double *d_gamma);

/* Release every resource of the plan (synchronises its device first).
 * Bookkeeping of this library (the paper has no plan object).  NULL is a
 * no-op returning MDX_OK. */
int mdx_plan_destroy(mdx_plan *plan);

/* Plan geometry: number of instances, total modes, per-instance mode offset
 * (the concatenation order of every per-mode array; bookkeeping, no
 * counterpart in the paper).  Output pointers may be NULL.  Errors:
 * MDX_ERR_ARG for a NULL plan. */
int mdx_plan_info(const mdx_plan *plan, int *n_inst, long *total_modes,
                  long *mode_offset /* [n_inst] or NULL */);

/* Bytes of the checkpoint buffer mdx_simulate writes for `steps` steps with
 * checkpoint interval K (state before steps 0, K, 2K, ...; the checkpointed
 * adjoint of this library, the paper differentiates through its whole loop).
 * Returns 0 for a NULL plan or steps, K <= 0. */
size_t mdx_checkpoint_bytes(const mdx_plan *plan, int steps, int K);

/*
 * Run `steps` steps of Eq. 20 for every instance.
 *   exc      device [n_inst][steps] FP32 excitation e^n (NULL = zero)
 *   q0, qm1  device [total_modes] FP64 initial states q^0, q^{-1} (NULL = zero)
 *   audio    device [n_inst][steps] FP32 output y^n (NULL = not written)
 *   q_end, qm1_end  device [total_modes] FP64 final q^steps, q^{steps-1} (NULL = skip);
 *            feeding them back as q0, qm1 continues the run (resume)
 *   K, ckpt  checkpoint interval and device buffer of mdx_checkpoint_bytes
 *            (ckpt NULL = none)
 *   status   device [n_inst] int, written MDX_OK / MDX_ERR_NONFINITE /
 *            MDX_ERR_TIMEOUT per instance (NULL = not written)
 *   stream   cudaStream_t
 */
int mdx_simulate(mdx_plan *plan, const float *exc, const double *q0, const double *qm1,
                 int steps, float *audio, double *q_end, double *qm1_end, int K,
                 void *ckpt, int *status, void *stream);

/* Gradient outputs of mdx_grad: device FP64 arrays, each optional (NULL). */
typedef struct mdx_grads {
    double *d_omega2;   /* [total_modes] dL/d omega^2 */
    double *d_gamma;    /* [total_modes] dL/d gamma */
    double *d_b;        /* [total_modes] dL/d b */
    double *d_c;        /* [total_modes] dL/d c */
    double *d_q0;       /* [total_modes] dL/d q^0 */
    double *d_qm1;      /* [total_modes] dL/d q^{-1} */
    double *d_tau;      /* [n_inst] dL/d tau' (tension instances; 0 for plates) */
    double *d_kappa;    /* [total stress modes] dL/d kappa, plates in plan order */
    double *d_dir;      /* [n_inst] <dL/dH, dH> for plates planned with dH (else 0) */
    double *d_H;        /* dL/dH^k_ij (Eq. 10; symmetrised over i, j, as H is symmetric):
                           for each plate with n_psi > 0 in plan order, [n_psi][N][N] in the
                           instance's own mode order; with the symmetry-class layout the
                           entries outside the class pattern (structurally zero in H) are
                           0, i.e. the gradient within class-structured tensors.  Used to fit
                           the coupling tensor itself (Sec. 4.3.3). */
} mdx_grads;

/* Bytes of the caller-owned device workspace mdx_grad needs for (steps, K):
 * two K-step segment buffers, the adjoint state and the gradient
 * accumulators.  Returns 0 for a NULL plan or K <= 0. */
size_t mdx_grad_workspace_bytes(const mdx_plan *plan, int steps, int K);

/*
 * Reverse-mode derivative of a scalar loss L(y) through the whole time loop of
 * Eq. 20 with the forces of Eq. 8-9 (the gradients the paper obtains by
 * automatic differentiation for its inverse problems, Sec. 4.3), written as a
 * hand-derived adjoint recursion.
 * Given dL/dy it runs the adjoint recursion backwards, segment by segment:
 * each K-step segment is recomputed from the checkpoint mdx_simulate wrote
 * (same arguments, same K), then swept in reverse.  With the class layout the
 * recompute of segment s-1 runs in the same launch, and the same pass over
 * the coupling tensor per step, as the reverse sweep of segment s; the
 * results are bitwise those of separate launches.
 *   exc, q0, qm1, steps  as passed to mdx_simulate
 *   d_audio  device [n_inst][steps] FP32 dL/dy^n
 *   K, ckpt  the checkpoint interval and buffer filled by mdx_simulate
 *   work     device workspace of mdx_grad_workspace_bytes (caller-owned scratch)
 *   out      gradient outputs (fields may be NULL)
 *   status   as in mdx_simulate
 */
int mdx_grad(mdx_plan *plan, const float *exc, const double *q0, const double *qm1,
             int steps, const float *d_audio, int K, const void *ckpt, void *work,
             size_t work_bytes, const mdx_grads *out, int *status, void *stream);

/*
 * Tile configuration of the plate kernel (used by the autotuner; a
 * performance control with no counterpart in the paper): TMA stage
 * size in bytes (multiple of 16, 0 = default 64 KB) and ring depth (0 = as
 * many stages as shared memory allows).  Takes effect for later launches;
 * fails with MDX_ERR_UNSUPPORTED if the stages do not fit in shared memory.
 * mdx_plan_tiles reports the current stage size, ring depths of the forward
 * and reverse launches, and the number of persistent CTAs.
 */
int mdx_plan_configure(mdx_plan *plan, int stage_bytes, int ring_stages);
int mdx_plan_tiles(const mdx_plan *plan, int *stage_bytes, int *ring_fwd, int *ring_rev,
                   int *ctas);

/*
 * L2 residency of the coupling stream.  Every step re-reads the whole
 * coupling tensor; the plate kernel's bulk copies carry an L2 policy that
 * gives a fraction of those addresses evict_last priority (the rest
 * evict_first), so that when the tensors of the plan are about as large as
 * the L2 (129 MB on GB300) that fraction stays resident across steps.
 * fraction in [0, 1] (0 = no hint), or negative for the default: all of the
 * stream when it fits in 70 % of the L2, else the share that does.  Results
 * do not depend on it (a cache hint; the paper has no counterpart).
 * mdx_plan_l2_keep returns the fraction in use (0 for a NULL plan).
 */
int mdx_plan_set_l2_keep(mdx_plan *plan, double fraction);
double mdx_plan_l2_keep(const mdx_plan *plan);

/*
 * Kernel timing (tracing; no counterpart in the paper, whose timings are
 * wall-clock, Sec. 4.2).  When enabled, every plate-kernel launch of the
 * plan is bracketed by CUDA events on its launch stream.  mdx_plan_kernel_stats
 * synchronises those events and returns, for one launch class
 * (0 = forward, 1 = checkpoint recompute, 2 = reverse sweep, 3 = per-segment
 * contraction of the direction tensor, 4 = fused sweep: the adjoint of one
 * segment and the recompute of the previous one in the same launch,
 * 5 = grouped plates on the tensor cores: bytes are the nonzero class blocks
 * of each group's shared coupling tensor, one pass per step, 6 = forward pass
 * of a few plates with their coupling rows resident in the registers of one
 * thread-block cluster per plate: bytes count one pass over H per step as for
 * class 0, although H is read from memory once per launch), the
 * number of launches, their summed device time in ms and their summed
 * algorithmic bytes (coupling-tensor bytes each launch must stream: one pass
 * over H per step; the direction tensor is counted by class 3).
 * mdx_plan_reset_stats clears the counters.  Off by default.
 */
int mdx_plan_set_profiling(mdx_plan *plan, int enable);
/* Work of the grouped-plate launch per simulated step (bookkeeping for
 * rooflines; the paper has no counterpart): bytes of the shared coupling
 * tensors' nonzero class blocks (one pass per step) and the contraction's
 * algorithmic flops, 2 x (nonzero entries) x (plates of the group), summed
 * over groups (the split-TF32 form executes three MMAs per product).  Zero for
 * a plan without grouped plates.  Errors: MDX_ERR_ARG for a NULL plan. */
int mdx_plan_group_work(const mdx_plan *plan, double *bytes_per_step, double *flops_per_step);
int mdx_plan_kernel_stats(mdx_plan *plan, int which, long *launches, double *ms, double *bytes);
int mdx_plan_reset_stats(mdx_plan *plan);

/*
 * Host FP64 map from physical parameters to modal coefficients for one
 * mode set (Sec. 3.2, Eq. 13-14):
 *   omega2_mu = (D lambda_mu^2 + T0 lambda_mu) / rho,  gamma_mu = s0 + s1 omega2_mu
 * and its vector-Jacobian product: given dL/domega2 and dL/dgamma, returns
 * dL/dD, dL/dT0, dL/ds0, dL/ds1 and dL/dlambda (per mode, for geometry).
 * lambda, omega2, gamma, d_omega2, d_gamma, d_lambda: host [n] arrays.
 */
int mdx_coeffs_from_physics(int n, const double *lambda, double D, double T0, double rho,
                            double s0, double s1, double *omega2, double *gamma);
int mdx_coeffs_vjp(int n, const double *lambda, double D, double T0, double rho, double s0,
                   double s1, const double *d_omega2, const double *d_gamma, double *dD,
                   double *dT0, double *ds0, double *ds1, double *d_lambda);

/*
 * Physical description of one object -> the modal coefficients of an
 * mdx_instance (host FP64, plan preparation):
 *   Laplacian eigenpairs, Sec. 3, Eq. 2:
 *     string (length L)            lambda_mu = (mu pi / L)^2,  mu = 1..N
 *     rectangle (simply supported)  lambda_mn = (m pi / Lx)^2 + (n pi / Ly)^2,
 *       the first N by ascending lambda, ties by (m, n), with Lx = sqrt(A / a),
 *       Ly = sqrt(A a) for area A and aspect a = Ly / Lx;
 *     unit-norm shapes sqrt(2/L) sin(mu pi x/L), 2/sqrt(Lx Ly) sin(m pi x/Lx) sin(n pi y/Ly)
 *   omega^2 = (D lambda^2 + T0 lambda) / rho (Eq. 13), gamma = sigma0 + sigma1 omega^2 (Eq. 14)
 *   b = Phi(x_strike) / rho, c = Phi(x_pickup)   (point force, displacement pickup)
 *   tau' = EA / (2 L) / rho (string) or E h / (2 Lx Ly (1 - nu^2)) / rho (membrane), Eq. 4
 *   kappa_k = E / (2 rho_vol zeta_k^4) (plate, Eq. 9)
 *   stability cut: the modes from the first with omega T >= omega_dt_max on are
 *   dropped (Stormer-Verlet needs omega T < 2, Eq. 20); a shortened plate keeps
 *   floor(n_psi N_kept / N) stress modes (at least 1).
 * The Airy eigenvalues zeta^4 and the coupling tensor H of Eq. 10 come from an
 * offline FP64 quadrature (the library takes H as an input of mdx_plan_create).
 */
#define MDX_SHAPE_STRING 0     /* fixed string of length L */
#define MDX_SHAPE_RECTANGLE 1  /* simply supported rectangle of area A and aspect a = Ly / Lx */

typedef struct mdx_physics {
    int kind;              /* MDX_KIND_TENSION (string, membrane) or MDX_KIND_PLATE */
    int shape;             /* MDX_SHAPE_STRING or MDX_SHAPE_RECTANGLE (plates: rectangle) */
    int n_phi;             /* transverse modes requested, 1..MDX_MAX_PHI */
    int n_psi;             /* stress modes requested (plate), 0..MDX_MAX_PSI */
    double dt;             /* sampling period T > 0 (s) */
    double omega_dt_max;   /* stability cut on omega T (e.g. 1.9); <= 0 keeps every mode */
    double length;         /* string length L (m) */
    double area, aspect;   /* rectangle area A (m^2) and aspect a = Ly / Lx */
    double D, T0, rho;     /* stiffness, tension, mass per unit length / area (Eq. 13) */
    double sigma0, sigma1; /* damping gamma = sigma0 + sigma1 omega^2 */
    double strike[2];      /* strike point relative to L, or to (Lx, Ly) */
    double pickup[2];      /* pickup point, same convention */
    double tension_stiffness; /* Eq. 4 numerator: EA (string) or E h / (1 - nu^2) (membrane);
                                 0 = linear */
    double vk_scale;       /* E / (2 rho_vol) of Eq. 9 (plate); 0 = linear */
    const double *zeta4;   /* host [n_psi] Airy eigenvalues zeta^4 (1/m^4), ascending
                              (nonlinear plate); NULL: kappa is not written, n_psi of
                              mdx_modal still gives the kept count (the count the
                              coupling tensor is then computed for) */
} mdx_physics;

/* Outputs of mdx_modal_from_physics: caller-owned host arrays sized for the
 * requested counts (n_phi of mdx_physics for the per-mode arrays, n_psi for
 * kappa); the call writes the kept counts. */
typedef struct mdx_modal {
    int n_phi;             /* out: modes kept by the stability cut */
    int n_psi;             /* out: stress modes kept (0 unless a nonlinear plate) */
    int *labels;           /* [n_phi][2] (mu, 0) or (m, n); may be NULL */
    double *lambda, *omega2, *gamma, *b, *c;   /* [n_phi] */
    double tau;            /* out: tau' (tension kind), else 0 */
    double *kappa;         /* [n_psi] (nonlinear plate with zeta4), else may be NULL */
} mdx_modal;

/* Gradients of a scalar loss with respect to the physical parameters. */
typedef struct mdx_physics_grads {
    double d_T0, d_D, d_aspect, d_sigma0, d_sigma1;
    double d_tension_stiffness;   /* through tau' (tension kind) */
    double d_vk_scale;            /* through kappa (plate) */
} mdx_physics_grads;

/* Fill `out` from the physical description (see above).  Errors: MDX_ERR_ARG,
 * MDX_ERR_NONFINITE, MDX_ERR_UNSUPPORTED, MDX_ERR_UNSTABLE (no mode below the
 * cut). */
int mdx_modal_from_physics(const mdx_physics *ph, mdx_modal *out);

/*
 * Vector-Jacobian product of mdx_modal_from_physics (Sec. 4.3: the inverse
 * problems fit these parameters by gradient descent): maps the per-mode
 * gradients of mdx_grad back to (T0, D, aspect, sigma0, sigma1) and to the
 * nonlinear scales (tension_stiffness, vk_scale).
 *   n_phi, n_psi  the kept counts mdx_modal_from_physics returned
 *   d_omega2, d_gamma  [n_phi] dL/d omega^2, dL/d gamma
 *   d_tau    dL/d tau' (tension kind)
 *   d_kappa  [n_psi] dL/d kappa (plate; may be NULL when n_psi = 0)
 *   d_dir    <dL/dH, dH/da> of mdx_grad for a plate planned with dH = dH/da
 *   dzeta4   [n_psi] d zeta^4 / da (plate; NULL = treat zeta^4 as fixed)
 * With A and the relative strike and pickup points fixed, b, c and a
 * membrane's tau' do not depend on the aspect; lambda does,
 *   d lambda_mn / da = (m pi)^2 / A - (n pi)^2 / (A a^2),
 * and so do kappa (through zeta^4) and H (d_dir).  d_aspect is 0 for strings.
 * Errors: MDX_ERR_ARG, MDX_ERR_NONFINITE, MDX_ERR_UNSUPPORTED.
 */
int mdx_physics_vjp(const mdx_physics *ph, int n_phi, int n_psi, const double *d_omega2,
                    const double *d_gamma, double d_tau, const double *d_kappa, double d_dir,
                    const double *dzeta4, mdx_physics_grads *out);

/*
 * Learned proposal network (initial parameter estimates for inverse fitting).
 * A multilayer perceptron d0 -> d1 -> ... -> dL with ReLU after every hidden
 * layer and a linear output.  Weights BF16 (raw bit patterns, row-major
 * [d_{l+1}][d_l]), biases FP32; every product accumulates in FP32 on the
 * tensor cores; hidden activations are stored in BF16.  The paper has no
 * network; this serves the learned initialisation of the inverse fits
 * (Sec. 4.3.3 notes the fits' sensitivity to initialisation).  All pointers
 * are device memory owned by the caller.
 */
#define MDX_MLP_MAX_LAYERS 8
typedef struct mdx_mlp {
    int n_layers;
    int dims[MDX_MLP_MAX_LAYERS + 1];
    const uint16_t *W[MDX_MLP_MAX_LAYERS];
    const float *b[MDX_MLP_MAX_LAYERS];
} mdx_mlp;

/* Elements (uint16) of the hidden-activation buffer, and of the backward
 * work buffer, for a batch (learned proposal, see above).  0 for invalid
 * arguments. */
size_t mdx_mlp_act_elems(const mdx_mlp *net, int batch);
size_t mdx_mlp_work_elems(const mdx_mlp *net, int batch);

/* y [batch][dL] (FP32) = net(x), x BF16 [batch][d0]; acts receives the hidden
 * activations (needed by the backward pass).  Learned proposal, see above.
 * Errors: MDX_ERR_ARG (layer count, widths, missing weights or buffers),
 * MDX_ERR_CUDA (launch). */
int mdx_mlp_forward(const mdx_mlp *net, int batch, const uint16_t *x, uint16_t *acts, float *y,
                    void *stream);

/* Learned proposal (see above).
 * Gradients of sum(dy . y) for the same x and acts: dW[l] FP32 [d_{l+1}][d_l],
 * db[l] FP32 [d_{l+1}] (overwritten).  dy is rounded to BF16 once; the
 * back-propagated signals are BF16 like the activations. */
int mdx_mlp_backward(const mdx_mlp *net, int batch, const uint16_t *x, const uint16_t *acts,
                     const float *dy, float *const *dW, float *const *db, uint16_t *work,
                     void *stream);

/* Learned proposal training (see above; Adam as in the paper's fits, Sec. 4.3).
 * One Adam step on n FP32 master weights w (moments m, v; step number t >= 1),
 * refreshing the BF16 copy w_bf16 (may be NULL). */
int mdx_adam_step(long long n, float *w, uint16_t *w_bf16, const float *g, float *m, float *v,
                  float lr, float beta1, float beta2, float eps, int t, void *stream);

/* Round-to-nearest-even FP32 -> BF16 of n elements (learned proposal inputs
 * and weights).  Errors: MDX_ERR_ARG, MDX_ERR_CUDA. */
int mdx_f32_to_bf16(long long n, const float *x, uint16_t *y, void *stream);

/*
 * Log-mel features of a batch of signals: the input of the learned proposal
 * network (the paper has no network or feature front end; its fits start
 * from random draws, Sec. 4.3).  For each signal x (length T) and segment s:
 * the power spectra of centred frames (the signal extended by reflection by
 * n_fft / 2 on both sides, hop `hop`, periodic Hann window), projected on
 * n_mels triangular filters equally spaced on the HTK mel scale
 * mel(f) = 2595 log10(1 + f / 700) between fmin and fmax, log(. + 1e-6),
 * averaged over the frames floor(s F / S) .. floor((s + 1) F / S) - 1 (at least
 * one), F = 1 + T / hop frames, S = segments.
 *   audio  device [batch][T] FP32
 *   out    device [batch][n_mels][segments] FP32 (overwritten)
 * Deterministic (fixed summation order).  Allocates nothing.
 * Errors: MDX_ERR_ARG (n_fft not a power of two in [16, 2048], T <= n_fft / 2,
 * fewer frames than segments, n_mels outside [1, 512], frequencies outside
 * 0 <= fmin < fmax <= fs / 2, NULL buffers), MDX_ERR_CUDA (launch).
 */
int mdx_logmel(const float *audio, int batch, int T, double fs, int n_fft, int hop, int n_mels,
               double fmin, double fmax, int segments, float *out, void *stream);

/*
 * Forward run of strings and membranes that allocates no device memory.
 * The paper has no counterpart: this entry point exists for callers that must
 * not call cudaMalloc, such as a real-time audio callback (cudaMalloc can
 * block for milliseconds and synchronises the device) or a plug-in whose host
 * application owns every device buffer.  For MDX_KIND_TENSION instances it
 * computes, bit for bit, the forward pass of mdx_plan_create (scheme
 * MDX_SCHEME_SV, the only scheme it offers) + mdx_simulate, without a plan.
 *   inst     [n_inst] host descriptions, all MDX_KIND_TENSION (H, kappa, dH unused)
 *   exc      device [n_inst][steps] FP32 excitation (NULL = zero)
 *   q0, qm1  device [total_modes] FP64 initial state (NULL = zero)
 *   audio    device [n_inst][steps] FP32 output (NULL = not written)
 *   q_end, qm1_end  device [total_modes] FP64 final state (NULL = skip)
 *   status   device [n_inst] int, as in mdx_simulate (NULL = not written)
 * Scratch: one fixed 1 MiB block of device memory per GPU, owned by the
 * library (a file-scope __device__ array held until the process exits).  It
 * bounds the problem: for n instances, total modes must not exceed
 *   (1048576 - align16(120 n) - align16(4 n) - 192) / 48   (rounded down,
 *   align16(x) = x rounded up to a multiple of 16; 21 838 modes for n = 1);
 * larger requests fail with MDX_ERR_UNSUPPORTED.  No call allocates or frees
 * device memory.  The first call on a device looks up the block's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  The coefficient table computed on the host
 * reaches the block inside the parameters of small copy kernels enqueued on
 * `stream`, so no host buffer is read after the call returns.  Every call
 * reuses the same block: calls that overlap on the GPU (e.g. on two streams)
 * race and must be serialised.  Errors: MDX_ERR_ARG, MDX_ERR_UNSTABLE,
 * MDX_ERR_NONFINITE, MDX_ERR_UNSUPPORTED, MDX_ERR_CUDA (message in
 * mdx_last_error).
 */
int mdx_simulate_strings_noalloc(const mdx_instance *inst, int n_inst, const float *exc,
                                 const double *q0, const double *qm1, int steps, float *audio,
                                 double *q_end, double *qm1_end, int *status, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MDX_H */
