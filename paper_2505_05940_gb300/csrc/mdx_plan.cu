// Host side of libmdx: validation, FP64 -> FP32 coefficient preparation, the
// plate work assignment, device memory of the plan, and the simulate / grad
// drivers that enqueue the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/mdx.h"
#include "mdx_internal.h"
#include "mdx_scheme.cuh"

using namespace mdx;

namespace {

thread_local std::string g_err = "no error";

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation)
        return fail(MDX_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(MDX_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define MDX_CUDA(call, what)                         \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace

int mdx::set_last_error(int code, const char *msg) { return fail(code, "%s", msg); }

struct mdx_plan {
    int device = 0;
    int n_inst = 0;
    long long total_modes = 0;
    long long total_k = 0;
    std::vector<InstDesc> inst;
    std::vector<double> dt;          // per instance
    // device memory owned by the plan
    std::vector<void *> allocs;
    InstDesc *d_inst = nullptr;
    ModeCoef coef{};
    double *d_omega2 = nullptr, *d_gamma = nullptr, *d_dt = nullptr;
    double *d_b64 = nullptr, *d_c64 = nullptr;   // FP64 b, c (linear solver)
    int *d_mode_inst = nullptr;                  // instance of each mode
    float *d_H = nullptr, *d_dH = nullptr, *d_kappa = nullptr;
    // plate work assignment
    int n_cta = 0;
    PlateItem *d_items = nullptr;
    int *d_cta_off = nullptr;
    int npad_max = 4;
    int state_floats = 0;
    int ring_fwd = 0, ring_rev = 0, stage_bytes = 0, u_slots_fwd = 1, u_slots_rev = 2;
    int u_floats_fwd = 0, u_floats_rev = 0;
    size_t smem_fwd = 0, smem_rev = 0;
    // fused adjoint sweep (reverse of segment s + recompute of segment s-1)
    bool fuse = false;
    int ring_fused = 0, u_floats_fused = 0;
    size_t smem_fused = 0;
    long long part_stride = 0;
    float *d_part = nullptr;
    unsigned *d_counters = nullptr;
    int *d_abort = nullptr;
    // tension instances (strings, membranes, linear plates)
    std::vector<int> tension;
    int *d_tension = nullptr;
    int tension_max_n = 1;
    bool any_plate = false;
    // scratch for simulate
    float *d_state = nullptr;        // [4][total_modes]
    long long wait_limit = 1 << 22;
    int debug_flags = 0;
    int scheme = MDX_SCHEME_SV;      // time discretisation (mdx_options.scheme)
    // optional per-launch timing of the plate kernel
    bool profiling = false;
    struct Rec {
        int which;
        double bytes;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    long stat_launch[7] = {0, 0, 0, 0, 0, 0, 0};
    double stat_ms[7] = {0, 0, 0, 0, 0, 0, 0}, stat_bytes[7] = {0, 0, 0, 0, 0, 0, 0};
    double H_bytes_per_step = 0, dH_bytes_per_step = 0;
    int smem_optin = 0;
    // L2 residency of the coupling stream: requested fraction (< 0: automatic)
    double l2_keep_req = -1.0;
    float l2_keep = 0.f;
    long long l2_bytes = 0;
    // symmetry-class layout
    bool parity = false;
    int mc_max = kParMcMax;
    int min_stage_floats = 4;
    ParityChunk *d_chunks = nullptr;
    int *d_perm = nullptr, *d_kperm = nullptr;
    // directional-derivative contraction units (plates planned with dH)
    DirUnit *d_dir_units = nullptr;
    int n_dir_units = 0;
    DirGroup *d_dir_groups = nullptr;
    int n_dir_groups = 0;
    // tensor-core contraction: K chunk (0 = CUDA-core kernel), B rows, shared memory
    int dir_tc_kc = 0, dir_tc_nmax = 0;
    size_t dir_tc_smem = 0;
    // the same units over every plate, for the full dL/dH output
    DirUnit *d_all_units = nullptr;
    int n_all_units = 0;
    DirGroup *d_all_groups = nullptr;
    int n_all_groups = 0;
    long long *d_dh_off = nullptr;   // [n_inst] offset (doubles) of each plate's dL/dH block
    int *d_dh_plates = nullptr;      // plates with stress modes (per-instance path)
    int n_dh_plates = 0;
    long long dh_total = 0;          // doubles of the dL/dH output
    // host copies of the layout, for mdx_plan_set_coupling
    std::vector<PlateItem> h_items;
    std::vector<ParityChunk> h_chunks;
    std::vector<std::vector<int>> h_perm;
    // host copies for coefficient updates
    std::vector<double> h_omega2, h_gamma, h_b, h_c, h_tau, h_kappa;
    std::vector<int> h_kperm;      // internal stress index -> user index, at each k_off
    float *d_coef_all = nullptr;   // the 8 FP32 coefficient arrays
    // plates sharing a coupling tensor, stepped by the grouped tensor-core kernel
    GroupPlan *grp = nullptr;
    std::vector<int> grouped;      // per instance
    bool any_grouped = false;
    // cluster-resident forward pass (few plates, class layout): one cluster per plate
    bool cluster_ok = false;
    int cl_cs = 0, cl_nkc = 0, cl_wk = 0, cl_rl = 0, n_cplates = 0;
    ClusterK *d_kinfo = nullptr;
    int *d_cplates = nullptr;
};

namespace {

int dalloc(mdx_plan *p, void **out, size_t bytes) {
    *out = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(out, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    p->allocs.push_back(*out);
    return MDX_OK;
}

template <class T>
int upload(mdx_plan *p, T **out, const T *host, size_t n) {
    int rc = dalloc(p, reinterpret_cast<void **>(out), n * sizeof(T));
    if (rc) return rc;
    if (n) MDX_CUDA(cudaMemcpy(*out, host, n * sizeof(T), cudaMemcpyHostToDevice), "upload");
    return MDX_OK;
}

bool finite(double x) { return std::isfinite(x); }

// Stability and domain of one mode under the plan's scheme.
int check_mode(int scheme, double w2, double gm, double T, int i, int m) {
    if (!(w2 > 0.0)) return fail(MDX_ERR_ARG, "instance %d mode %d: omega2 must be > 0", i, m);
    if (gm < 0.0)
        return fail(MDX_ERR_UNSTABLE, "instance %d mode %d: gamma < 0 puts a pole in the right half-plane", i, m);
    if (scheme == MDX_SCHEME_TF) {
        if (!(w2 > gm * gm))
            return fail(MDX_ERR_UNSTABLE,
                        "instance %d mode %d: the impulse-invariant scheme needs omega > gamma", i, m);
    } else if (std::sqrt(w2) * T >= 2.0) {
        return fail(MDX_ERR_UNSTABLE,
                    "instance %d mode %d: omega*dt = %.4f >= 2 (Stormer-Verlet stability bound)",
                    i, m, std::sqrt(w2) * T);
    }
    return MDX_OK;
}

int validate(const mdx_instance &I, int i, int scheme) {
    if (I.kind != MDX_KIND_TENSION && I.kind != MDX_KIND_PLATE)
        return fail(MDX_ERR_ARG, "instance %d: unknown kind %d", i, I.kind);
    if (I.n_phi < 1 || I.n_phi > MDX_MAX_PHI)
        return fail(MDX_ERR_UNSUPPORTED, "instance %d: n_phi=%d outside [1, %d]", i, I.n_phi,
                    MDX_MAX_PHI);
    if (!(I.dt > 0.0) || !finite(I.dt)) return fail(MDX_ERR_ARG, "instance %d: dt must be > 0", i);
    if (!I.omega2 || !I.gamma || !I.b || !I.c)
        return fail(MDX_ERR_ARG, "instance %d: omega2, gamma, b and c are required", i);
    for (int m = 0; m < I.n_phi; ++m) {
        if (!finite(I.omega2[m]) || !finite(I.gamma[m]) || !finite(I.b[m]) || !finite(I.c[m]))
            return fail(MDX_ERR_NONFINITE, "instance %d mode %d: non-finite coefficient", i, m);
        const int rc = check_mode(scheme, I.omega2[m], I.gamma[m], I.dt, i, m);
        if (rc) return rc;
    }
    if (I.kind == MDX_KIND_TENSION) {
        if (!I.lambda) return fail(MDX_ERR_ARG, "instance %d: lambda is required for the tension kind", i);
        if (!finite(I.tau) || I.tau < 0.0) return fail(MDX_ERR_ARG, "instance %d: tau must be finite and >= 0", i);
        for (int m = 0; m < I.n_phi; ++m)
            if (!finite(I.lambda[m]) || I.lambda[m] < 0.0)
                return fail(MDX_ERR_ARG, "instance %d mode %d: lambda must be finite and >= 0", i, m);
    } else {
        if (I.n_psi < 0 || I.n_psi > MDX_MAX_PSI)
            return fail(MDX_ERR_UNSUPPORTED, "instance %d: n_psi=%d outside [0, %d]", i, I.n_psi, MDX_MAX_PSI);
        if (I.n_psi > 0) {
            if (!I.H || !I.kappa) return fail(MDX_ERR_ARG, "instance %d: H and kappa are required when n_psi > 0", i);
            const int N = I.n_phi;
            for (int k = 0; k < I.n_psi; ++k) {
                if (!finite(I.kappa[k])) return fail(MDX_ERR_NONFINITE, "instance %d: kappa[%d] is not finite", i, k);
                const float *Hk = I.H + (size_t)k * N * N;
                float amax = 0.f;
                for (size_t t = 0; t < (size_t)N * N; ++t) {
                    if (!std::isfinite(Hk[t]))
                        return fail(MDX_ERR_NONFINITE, "instance %d: H[%d] has a non-finite entry", i, k);
                    amax = std::max(amax, std::fabs(Hk[t]));
                }
                for (int a = 0; a < N; ++a)
                    for (int b = a + 1; b < N; ++b)
                        if (std::fabs(Hk[(size_t)a * N + b] - Hk[(size_t)b * N + a]) > 1e-5f * amax + 1e-30f)
                            return fail(MDX_ERR_ARG, "instance %d: H[%d] is not symmetric at (%d, %d)", i, k, a, b);
                if (I.dH) {
                    const float *Dk = I.dH + (size_t)k * N * N;
                    for (size_t t = 0; t < (size_t)N * N; ++t)
                        if (!std::isfinite(Dk[t]))
                            return fail(MDX_ERR_NONFINITE, "instance %d: dH[%d] has a non-finite entry", i, k);
                }
            }
        }
    }
    return MDX_OK;
}

// Balance the H bytes of all plate items over at most `max_cta` CTAs.
struct Piece {
    int inst, k0, k1;
    double cost;
};

int configure_tiles(mdx_plan *p, int stage_req, int ring_req);
void update_l2_keep(mdx_plan *p);

// Packs the coupling tensor H (and the direction tensor dH, if the plate has
// one and dH is not NULL) of plate i into the plan's device layout: dense rows
// [M][N][N_pad], or the symmetry-class chunks of the plate's work items.
int upload_coupling(mdx_plan *p, int i, const float *H, const float *dH) {
    const InstDesc &d = p->inst[i];
    auto nb4 = [](int n) { return (n + 3) & ~3; };
    std::vector<float> tmp;
    if (p->parity) {
        const std::vector<int> &perm = p->h_perm[i];
        for (const auto &it : p->h_items) {
            if (it.inst != i) continue;
            for (int ci = it.chunk0; ci < it.chunk1; ++ci) {
                const ParityChunk &ch = p->h_chunks[ci];
                for (int which = 0; which < (d.has_dir ? 2 : 1); ++which) {
                    const float *src = which == 0 ? H : dH;
                    if (!src) continue;
                    tmp.clear();
                    for (int a = 0; a < 4; ++a) {
                        const int bcl = a ^ ch.c, na = d.ncls[a], nbc = d.ncls[bcl];
                        const int w = nb4(nbc);
                        for (int pp = 0; pp < na; ++pp) {
                            const int row = perm[d.ocls[a] + pp];
                            for (int kl = 0; kl < ch.mc; ++kl) {
                                const int ku = p->h_kperm[d.k_off + ch.kl0 + kl];
                                const float *Hr = src + ((size_t)ku * d.N + row) * d.N;
                                for (int cs = 0; cs < w; ++cs)
                                    tmp.push_back(cs < nbc ? Hr[perm[d.ocls[bcl] + cs]] : 0.f);
                            }
                        }
                    }
                    float *dst = p->d_H + (which == 0 ? ch.off : ch.doff);
                    if (!tmp.empty())
                        MDX_CUDA(cudaMemcpy(dst, tmp.data(), tmp.size() * sizeof(float),
                                            cudaMemcpyHostToDevice), "upload H");
                }
            }
        }
    } else {
        const size_t blk = (size_t)d.M * d.N * d.Npad;
        for (int which = 0; which < (d.has_dir ? 2 : 1); ++which) {
            const float *src = which == 0 ? H : dH;
            if (!src) continue;
            tmp.assign(blk, 0.f);
            for (int k = 0; k < d.M; ++k)
                for (int a2 = 0; a2 < d.N; ++a2)
                    std::memcpy(&tmp[((size_t)k * d.N + a2) * d.Npad], src + ((size_t)k * d.N + a2) * d.N,
                                d.N * sizeof(float));
            float *dst = p->d_H + (which == 0 ? d.H_off : d.dH_off);
            MDX_CUDA(cudaMemcpy(dst, tmp.data(), blk * sizeof(float), cudaMemcpyHostToDevice),
                     "upload H");
        }
    }
    return MDX_OK;
}

}  // namespace

extern "C" {

const char *mdx_last_error(void) { return g_err.c_str(); }

const char *mdx_version(void) { return "mdx 0.1 (sm_103a)"; }

int mdx_plan_destroy(mdx_plan *p) {
    if (!p) return MDX_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    for (auto &r : p->recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (void *a : p->allocs) cudaFree(a);
    group_plan_free(p->grp);
    if (prev >= 0) cudaSetDevice(prev);
    delete p;
    return MDX_OK;
}

int mdx_plan_info(const mdx_plan *p, int *n_inst, long *total_modes, long *mode_offset) {
    if (!p) return fail(MDX_ERR_ARG, "plan is NULL");
    if (n_inst) *n_inst = p->n_inst;
    if (total_modes) *total_modes = (long)p->total_modes;
    if (mode_offset)
        for (int i = 0; i < p->n_inst; ++i) mode_offset[i] = (long)p->inst[i].mode_off;
    return MDX_OK;
}

int mdx_plan_create(mdx_plan **out, const mdx_instance *I, int n_inst, const mdx_options *opts) {
    if (!out) return fail(MDX_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n_inst < 1 || !I) return fail(MDX_ERR_ARG, "need at least one instance");
    mdx_options o{};
    if (opts) o = *opts;
    if (o.scheme != MDX_SCHEME_SV && o.scheme != MDX_SCHEME_TF)
        return fail(MDX_ERR_ARG, "unknown scheme %d", o.scheme);
    for (int i = 0; i < n_inst; ++i) {
        int rc = validate(I[i], i, o.scheme);
        if (rc) return rc;
    }
    MDX_CUDA(cudaSetDevice(o.device), "cudaSetDevice");
    mdx_plan *p = new mdx_plan();
    p->device = o.device;
    p->n_inst = n_inst;
    p->scheme = o.scheme;
    if (o.wait_limit > 0) p->wait_limit = o.wait_limit;
    p->debug_flags = o.debug_flags;
    auto bail = [&](int rc) {
        mdx_plan_destroy(p);
        return rc;
    };

    // ---- per-instance layout and FP64 -> FP32 coefficients (difference form)
    std::vector<float> eps, rw2, rw2lo, r, b, c, lam, clo;
    std::vector<double> w2d, gmd, dtd;
    p->inst.resize(n_inst);
    p->dt.resize(n_inst);
    for (int i = 0; i < n_inst; ++i) {
        const mdx_instance &S = I[i];
        InstDesc d{};
        d.kind = S.kind;
        d.N = S.n_phi;
        d.M = (S.kind == MDX_KIND_PLATE) ? S.n_psi : 0;
        d.Npad = (S.n_phi + 3) & ~3;
        d.mode_off = p->total_modes;
        d.k_off = p->total_k;
        d.taup = (S.kind == MDX_KIND_TENSION) ? (float)S.tau : 0.f;
        d.has_dir = (d.M > 0 && S.dH) ? 1 : 0;
        p->total_modes += d.N;
        p->total_k += d.M;
        p->dt[i] = S.dt;
        const double T = S.dt;
        for (int m = 0; m < S.n_phi; ++m) {
            const ModeF32 k = mode_f32(p->scheme, S.omega2[m], S.gamma[m], T);
            eps.push_back(k.eps);
            rw2.push_back(k.rho_hi);
            rw2lo.push_back(k.rho_lo);
            r.push_back(k.r);
            b.push_back((float)S.b[m]);
            c.push_back((float)S.c[m]);
            clo.push_back((float)(S.c[m] - (double)(float)S.c[m]));
            lam.push_back(S.kind == MDX_KIND_TENSION ? (float)S.lambda[m] : 0.f);
            w2d.push_back(S.omega2[m]);
            gmd.push_back(S.gamma[m]);
            dtd.push_back(T);
        }
        p->inst[i] = d;
    }
    const size_t TM = (size_t)p->total_modes;
    // Plates of one geometry group (geom_group > 0) are stepped by the grouped
    // tensor-core kernel unless the options ask for per-instance copies; the
    // per-instance machinery below sees them as plates without stress modes.
    p->grouped.assign(n_inst, 0);
    if (o.group_engine != MDX_GROUP_OFF) {
        for (int i = 0; i < n_inst; ++i) {
            InstDesc &d = p->inst[i];
            if (d.kind == MDX_KIND_PLATE && d.M > 0 && I[i].geom_group > 0) {
                p->grouped[i] = 1;
                p->any_grouped = true;
                d.grouped = 1;
                d.M = 0;
                d.has_dir = 0;
            }
        }
    }
    for (int i = 0; i < n_inst; ++i) {
        const mdx_instance &S = I[i];
        for (int m = 0; m < S.n_phi; ++m) {
            p->h_b.push_back(S.b[m]);
            p->h_c.push_back(S.c[m]);
        }
        p->h_tau.push_back(S.kind == MDX_KIND_TENSION ? S.tau : 0.0);
        const int M = (S.kind == MDX_KIND_PLATE) ? S.n_psi : 0;
        for (int k = 0; k < M; ++k) p->h_kappa.push_back(S.kappa[k]);
    }
    p->h_omega2 = w2d;
    p->h_gamma = gmd;
    {
        std::vector<float> all;
        all.reserve(8 * TM);
        for (auto *v : {&eps, &rw2, &r, &b, &c, &lam, &rw2lo, &clo})
            all.insert(all.end(), v->begin(), v->end());
        float *dc = nullptr;
        int rc = upload(p, &dc, all.data(), all.size());
        if (rc) return bail(rc);
        p->d_coef_all = dc;
        p->coef.eps = dc;
        p->coef.rw2 = dc + TM;
        p->coef.r = dc + 2 * TM;
        p->coef.b = dc + 3 * TM;
        p->coef.c = dc + 4 * TM;
        p->coef.lam = dc + 5 * TM;
        p->coef.rw2lo = dc + 6 * TM;
        p->coef.clo = dc + 7 * TM;
        if ((rc = upload(p, &p->d_omega2, w2d.data(), TM))) return bail(rc);
        if ((rc = upload(p, &p->d_gamma, gmd.data(), TM))) return bail(rc);
        if ((rc = upload(p, &p->d_dt, dtd.data(), TM))) return bail(rc);
        if ((rc = upload(p, &p->d_b64, p->h_b.data(), TM))) return bail(rc);
        if ((rc = upload(p, &p->d_c64, p->h_c.data(), TM))) return bail(rc);
        std::vector<int> mi;
        for (int i = 0; i < n_inst; ++i) mi.insert(mi.end(), (size_t)p->inst[i].N, i);
        if ((rc = upload(p, &p->d_mode_inst, mi.data(), mi.size()))) return bail(rc);
    }
    // ---- tension list (strings, membranes and plates without coupling)
    for (int i = 0; i < n_inst; ++i) {
        const InstDesc &d = p->inst[i];
        if (d.grouped) continue;
        if (d.kind == MDX_KIND_TENSION || d.M == 0) {
            p->tension.push_back(i);
            p->tension_max_n = std::max(p->tension_max_n, d.N);
        } else {
            p->any_plate = true;
        }
    }

    // ---- plate work assignment
    std::vector<PlateItem> items;
    std::vector<int> cta_off{0};
    if (p->any_plate) {
        int dev_sms = 0, smem_optin = 0;
        MDX_CUDA(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, p->device), "attr");
        MDX_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device), "attr");
        int l2 = 0;
        MDX_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, p->device), "attr");
        p->l2_bytes = l2;
        int max_cta = dev_sms;
        if (o.max_ctas > 0) max_cta = std::min(max_cta, o.max_ctas);
        // Symmetry-class layout: used when every coupled plate gives classes
        // that match its coupling tensor (entries outside the class pattern at
        // most 1e-6 of the largest of their H^k; those are dropped).
        bool parity = true;
        for (int i = 0; i < n_inst; ++i) {
            const InstDesc &d = p->inst[i];
            if (d.kind == MDX_KIND_PLATE && d.M > 0 && (!I[i].phi_class || !I[i].psi_class))
                parity = false;
        }
        std::vector<std::vector<int>> perm(n_inst), kperm(n_inst);
        std::vector<std::vector<int>> kcls(n_inst);
        for (int i = 0; i < n_inst; ++i) {
            InstDesc &d = p->inst[i];
            if (d.M == 0) continue;
            kperm[i].resize(d.M);
            std::iota(kperm[i].begin(), kperm[i].end(), 0);
            if (!parity) continue;
            const int *fc = I[i].phi_class, *kc = I[i].psi_class;
            for (int m = 0; m < d.N; ++m)
                if (fc[m] < 0 || fc[m] > 3)
                    return bail(fail(MDX_ERR_ARG, "instance %d: phi_class[%d] outside 0..3", i, m));
            for (int k = 0; k < d.M; ++k)
                if (kc[k] < 0 || kc[k] > 3)
                    return bail(fail(MDX_ERR_ARG, "instance %d: psi_class[%d] outside 0..3", i, k));
            for (int which = 0; which < (d.has_dir ? 2 : 1); ++which) {
                const float *src = which == 0 ? I[i].H : I[i].dH;
                for (int k = 0; k < d.M; ++k) {
                    const float *Hk = src + (size_t)k * d.N * d.N;
                    float amax = 0.f;
                    for (size_t t = 0; t < (size_t)d.N * d.N; ++t) amax = std::max(amax, std::fabs(Hk[t]));
                    for (int x = 0; x < d.N; ++x)
                        for (int y = 0; y < d.N; ++y)
                            if ((fc[x] ^ fc[y]) != kc[k] &&
                                std::fabs(Hk[(size_t)x * d.N + y]) > 1e-6f * amax)
                                return bail(fail(MDX_ERR_ARG,
                                    "instance %d: %s[%d][%d][%d] lies outside the declared symmetry classes",
                                    i, which == 0 ? "H" : "dH", k, x, y));
                }
            }
            d.parity = 1;
            for (int a = 0; a < 4; ++a) d.ncls[a] = 0;
            for (int m = 0; m < d.N; ++m) d.ncls[fc[m]]++;
            d.ocls[0] = 0;
            for (int a = 1; a < 4; ++a) d.ocls[a] = d.ocls[a - 1] + d.ncls[a - 1];
            perm[i].resize(d.N);
            int fill[4] = {d.ocls[0], d.ocls[1], d.ocls[2], d.ocls[3]};
            for (int m = 0; m < d.N; ++m) perm[i][fill[fc[m]]++] = m;
            std::stable_sort(kperm[i].begin(), kperm[i].end(),
                             [&](int x, int y) { return kc[x] < kc[y]; });
            kcls[i].resize(d.M);
            for (int kk = 0; kk < d.M; ++kk) kcls[i][kk] = kc[kperm[i][kk]];
        }
        auto nb4 = [](int n) { return (n + 3) & ~3; };
        // a class wider than 32 threads x kParQmax quads keeps the dense layout
        for (int i = 0; i < n_inst && parity; ++i)
            for (int a = 0; a < 4; ++a)
                if (p->inst[i].M > 0 && nb4(p->inst[i].ncls[a]) / 4 > 32 * kParQmax) parity = false;
        if (!parity)
            for (int i = 0; i < n_inst; ++i) {
                p->inst[i].parity = 0;
                if (p->inst[i].M > 0) std::iota(kperm[i].begin(), kperm[i].end(), 0);
            }
        p->parity = parity;
        // the fused adjoint sweep needs the class layout (disabled by debug flag bit 1)
        p->fuse = parity && !(p->debug_flags & 2);
        const int narr = parity ? ST_NARR_FUSED : ST_NARR;   // state arrays per item
        // bytes (floats) one internal stress mode streams per pass
        auto unit_cost = [&](int i, int kk) -> double {
            const InstDesc &d = p->inst[i];
            if (!parity) return (double)d.N * d.Npad;
            const int c = kcls[i][kk];
            double t = 0.0;
            for (int a = 0; a < 4; ++a) t += (double)d.ncls[a] * nb4(d.ncls[a ^ c]);
            return t;
        };
        // Contiguous split: walk all (plate, stress mode) units in plan order
        // and cut them into G ranges (dense layout: equal H bytes; class
        // layout: the min-max partition below); each CTA then holds at most
        // one contiguous k range per plate.  A forced split (tests) or an
        // overfull shared-memory state falls back to longest-processing-time
        // assignment of explicit pieces.
        const int state_cap = 24 * 1024;   // 96 KB of item state per CTA at most
        // shared-memory block of one item: its state arrays, then its stress
        // modes' d kappa pairs and kappa (+ the per-mode coefficients and the
        // class permutation, 8 arrays, and the owner's gradient sums, when the
        // item caches them: plates up to 512 modes, while the CTA's state fits).
        // The work split is sized without the caches; each CTA then turns them
        // on item by item within the state budget.
        auto item_cachable = [&](const InstDesc &d) { return d.Npad <= 512; };
        auto item_floats = [&](const InstDesc &d, int nk, bool owner, bool cached) {
            return narr * d.Npad + 3 * ((nk + 3) & ~3) +
                   (cached ? 8 * d.Npad + (owner ? 2 * GA_N * d.Npad : 0) : 0);
        };
        double total = 0.0;
        long long total_kk = 0;
        for (int i = 0; i < n_inst; ++i) {
            const InstDesc &d = p->inst[i];
            if (d.M == 0) continue;
            for (int kk = 0; kk < d.M; ++kk) total += unit_cost(i, kk);
            total_kk += d.M;
        }
        const int G = (int)std::min<long long>(max_cta, total_kk);
        const double target = total / G;
        std::vector<std::vector<Piece>> per(G);
        bool contiguous_ok = (o.force_split <= 0);
        // chunk size of the class layout (also used by the split's cost model)
        int npad_plates = 4;
        for (int i = 0; i < n_inst; ++i)
            if (p->inst[i].M > 0) npad_plates = std::max(npad_plates, p->inst[i].Npad);
        int mc_glob = kParMcMax;
        if (parity) {
            for (int i = 0; i < n_inst; ++i) {
                const InstDesc &d = p->inst[i];
                if (d.M == 0) continue;
                int nq = 1;
                for (int a = 0; a < 4; ++a) nq = std::max(nq, nb4(d.ncls[a]) / 4);
                const int cap = std::max(1, std::min(kParMcMax, 8192 / (2 * npad_plates)));
                int mc = cap;
                auto tpk = [](int m) { int t = 32; while (t > 1 && t * m > 256) t >>= 1; return t; };
                while (mc > 1 && tpk(mc) * kParQmax < nq) --mc;
                mc_glob = std::min(mc_glob, mc);
            }
        }
        if (contiguous_ok && !parity) {
            double cum = 0.0;
            for (int i = 0; i < n_inst; ++i) {
                const InstDesc &d = p->inst[i];
                if (d.M == 0) continue;
                for (int k = 0; k < d.M; ++k) {
                    const double c = unit_cost(i, k);
                    int g = (int)((cum + 0.5 * c) / target);
                    g = std::max(0, std::min(G - 1, g));
                    cum += c;
                    auto &v = per[g];
                    if (!v.empty() && v.back().inst == i && v.back().k1 == k) {
                        v.back().k1 = k + 1;
                        v.back().cost += c;
                    } else {
                        v.push_back({i, k, k + 1, c});
                    }
                }
            }
        }
        if (contiguous_ok && parity) {
            // Class layout: a CTA's time is its bytes plus a fixed cost per class
            // chunk (every super-block of a chunk is a full pass over its rows,
            // whatever the chunk's size) and per plate item.  Cut the unit
            // sequence greedily under a time bound and bisect the bound until
            // the cuts fit in G CTAs (min-max contiguous partition).
            const double beta = 65536.0, gamma = 16384.0;   // floats-equivalent
            std::vector<std::pair<int, int>> units;
            for (int i = 0; i < n_inst; ++i)
                for (int k = 0; k < p->inst[i].M; ++k) units.push_back({i, k});
            std::vector<int> cut(units.size(), 0);
            auto greedy = [&](double T, bool record) {
                int g = 0, prev_i = -1, prev_c = -1, run = 0;
                double cur = 0.0;
                bool empty = true;
                for (size_t u = 0; u < units.size(); ++u) {
                    const int i = units[u].first, k = units[u].second;
                    const double c = unit_cost(i, k);
                    bool new_item = empty || prev_i != i;
                    bool new_chunk = new_item || kcls[i][k] != prev_c || run >= mc_glob;
                    double delta = c + (new_chunk ? beta : 0.0) + (new_item ? gamma : 0.0);
                    if (!empty && cur + delta > T) {
                        ++g;
                        cur = 0.0;
                        new_item = new_chunk = true;
                        delta = c + beta + gamma;
                    }
                    cur += delta;
                    empty = false;
                    run = new_chunk ? 1 : run + 1;
                    prev_i = i;
                    prev_c = kcls[i][k];
                    if (record) cut[u] = g;
                }
                return g + 1;
            };
            double lo = 0.0, hi = 0.0;
            for (const auto &u : units) {
                const double c = unit_cost(u.first, u.second) + beta + gamma;
                lo = std::max(lo, c);
                hi += c;
            }
            if (greedy(lo, false) > G) {
                for (int it = 0; it < 60 && hi - lo > 1e-6 * hi; ++it) {
                    const double mid = 0.5 * (lo + hi);
                    if (greedy(mid, false) <= G) hi = mid; else lo = mid;
                }
            } else {
                hi = lo;
            }
            greedy(hi, true);
            for (size_t u = 0; u < units.size(); ++u) {
                const int i = units[u].first, k = units[u].second;
                const double c = unit_cost(i, k);
                auto &v = per[cut[u]];
                if (!v.empty() && v.back().inst == i && v.back().k1 == k) {
                    v.back().k1 = k + 1;
                    v.back().cost += c;
                } else {
                    v.push_back({i, k, k + 1, c});
                }
            }
        }
        if (contiguous_ok) {
            for (int g = 0; g < G && contiguous_ok; ++g) {
                int need = 0;
                for (const Piece &q : per[g])
                    need += item_floats(p->inst[q.inst], q.k1 - q.k0, true, false);
                if (need > state_cap) contiguous_ok = false;
            }
        }
        if (!contiguous_ok) {
            for (auto &v : per) v.clear();
            std::vector<Piece> pieces;
            for (int i = 0; i < n_inst; ++i) {
                const InstDesc &d = p->inst[i];
                if (d.M == 0) continue;
                double cost = 0.0;
                for (int kk = 0; kk < d.M; ++kk) cost += unit_cost(i, kk);
                int np = (int)std::ceil(cost / target - 1e-9);
                np = std::max(1, std::min(np, std::min(d.M, G)));
                if (o.force_split > 0) np = std::max(np, std::min(o.force_split, std::min(d.M, G)));
                for (int j = 0; j < np; ++j) {
                    const int k0 = (int)((long long)d.M * j / np);
                    const int k1 = (int)((long long)d.M * (j + 1) / np);
                    double pc = 0.0;
                    for (int kk = k0; kk < k1; ++kk) pc += unit_cost(i, kk);
                    pieces.push_back({i, k0, k1, pc});
                }
            }
            std::stable_sort(pieces.begin(), pieces.end(),
                             [](const Piece &a, const Piece &b) { return a.cost > b.cost; });
            std::vector<double> load(G, 0.0);
            std::vector<int> sfl(G, 0);
            for (const Piece &pc : pieces) {
                const InstDesc &d = p->inst[pc.inst];
                const int need = item_floats(d, pc.k1 - pc.k0, true, false);
                int best = -1;
                for (int g = 0; g < G; ++g) {
                    bool has = false;
                    for (const Piece &q : per[g]) has = has || (q.inst == pc.inst);
                    if (has || sfl[g] + need > state_cap) continue;
                    if (best < 0 || load[g] < load[best]) best = g;
                }
                if (best < 0)
                    return bail(fail(MDX_ERR_UNSUPPORTED,
                                     "plate work does not fit: too many plate modes for %d CTAs", G));
                per[best].push_back(pc);
                load[best] += pc.cost;
                sfl[best] += need;
            }
        }
        // contributors per instance, in CTA order
        std::vector<std::vector<int>> contrib(n_inst);
        for (int g = 0; g < G; ++g)
            for (const Piece &q : per[g]) contrib[q.inst].push_back(g);
        long long part_off = 0;
        for (int i = 0; i < n_inst; ++i) {
            InstDesc &d = p->inst[i];
            d.n_contrib = (int)contrib[i].size();
            d.part_off = part_off;
            if (d.n_contrib > 1) part_off += (long long)d.n_contrib * 3 * d.Npad;
        }
        p->part_stride = std::max<long long>(part_off, 4);
        int max_state = 0;
        for (int g = 0; g < G; ++g) {
            if (per[g].empty()) continue;
            int soff = 0;
            std::sort(per[g].begin(), per[g].end(),
                      [](const Piece &a, const Piece &b) { return a.inst < b.inst; });
            int spare = state_cap;
            for (const Piece &q : per[g]) spare -= item_floats(p->inst[q.inst], q.k1 - q.k0, true, false);
            for (const Piece &q : per[g]) {
                const InstDesc &d = p->inst[q.inst];
                PlateItem it{};
                it.inst = q.inst;
                it.k0 = q.k0;
                it.k1 = q.k1;
                const auto &cl = contrib[q.inst];
                it.slot = (int)(std::find(cl.begin(), cl.end(), g) - cl.begin());
                it.owner = (it.slot == 0) ? 1 : 0;
                it.smem_state = soff;
                const int base = item_floats(d, it.k1 - it.k0, it.owner != 0, false);
                const int extra = item_floats(d, it.k1 - it.k0, it.owner != 0, true) - base;
                it.cache = (!(p->debug_flags & 4) && item_cachable(d) && extra <= spare) ? 1 : 0;
                if (it.cache) spare -= extra;
                soff += base + (it.cache ? extra : 0);
                items.push_back(it);
                p->npad_max = std::max(p->npad_max, d.Npad);
            }
            max_state = std::max(max_state, soff);
            cta_off.push_back((int)items.size());
        }
        p->n_cta = (int)cta_off.size() - 1;
        p->state_floats = max_state;
        // ---- coupling data in HBM
        // dense layout: per plate [M][N][N_pad] rows (zero padded);
        // class layout: per item, per class chunk, super-blocks in stream order.
        std::vector<ParityChunk> chunks;
        long long H_total = 0;
        if (parity) {
            for (auto &it : items) {
                const InstDesc &d = p->inst[it.inst];
                it.chunk0 = (int)chunks.size();
                int kk = it.k0;
                while (kk < it.k1) {
                    const int c = kcls[it.inst][kk];
                    int e = kk;
                    while (e < it.k1 && kcls[it.inst][e] == c && e - kk < mc_glob) ++e;
                    ParityChunk ch{};
                    ch.c = c;
                    ch.kl0 = kk;
                    ch.mc = e - kk;
                    long long sz = 0;
                    for (int a = 0; a < 4; ++a) sz += (long long)d.ncls[a] * ch.mc * nb4(d.ncls[a ^ c]);
                    ch.off = H_total;
                    H_total += sz;
                    ch.doff = d.has_dir ? H_total : 0;
                    if (d.has_dir) H_total += sz;
                    chunks.push_back(ch);
                    kk = e;
                }
                it.chunk1 = (int)chunks.size();
            }
        } else {
            for (int i = 0; i < n_inst; ++i) {
                InstDesc &d = p->inst[i];
                d.H_off = H_total;
                if (d.M > 0) H_total += (long long)d.M * d.N * d.Npad;
            }
            for (int i = 0; i < n_inst; ++i) {
                InstDesc &d = p->inst[i];
                d.dH_off = H_total;
                if (d.has_dir) H_total += (long long)d.M * d.N * d.Npad;
            }
        }
        p->mc_max = mc_glob;
        {
            int rc2 = dalloc(p, reinterpret_cast<void **>(&p->d_H), std::max<long long>(H_total, 4) * sizeof(float));
            if (rc2) return bail(rc2);
            p->d_dH = p->d_H;
            p->h_items = items;
            p->h_chunks = chunks;
            p->h_perm = perm;
            // internal -> user stress index at each plate's k_off (the packing reads it)
            p->h_kperm.assign(std::max<long long>(p->total_k, 1), 0);
            for (int i = 0; i < n_inst; ++i)
                for (int kk = 0; kk < p->inst[i].M; ++kk) p->h_kperm[p->inst[i].k_off + kk] = kperm[i][kk];
            for (int i = 0; i < n_inst; ++i) {
                if (p->inst[i].M == 0) continue;
                const int rcu = upload_coupling(p, i, I[i].H, I[i].dH);
                if (rcu) return bail(rcu);
            }
            // algorithmic bytes of one pass (the stored, structurally nonzero part of H)
            for (int i = 0; i < n_inst; ++i) {
                const InstDesc &d = p->inst[i];
                if (d.M == 0) continue;
                double per_step = 0.0;
                if (parity) {
                    for (int kk = 0; kk < d.M; ++kk) {
                        const int c = kcls[i][kk];
                        for (int a = 0; a < 4; ++a) per_step += 4.0 * d.ncls[a] * d.ncls[a ^ c];
                    }
                } else {
                    per_step = 4.0 * d.M * d.N * d.N;
                }
                p->H_bytes_per_step += per_step;
                if (d.has_dir) p->dH_bytes_per_step += per_step;
            }
            // kappa in internal (class-sorted) order, class permutations
            // indexed by each plate's k_off (grouped plates keep their range, unused here)
            std::vector<float> kap2(std::max<long long>(p->total_k, 1), 0.f);
            std::vector<int> perm_all, kperm_all(std::max<long long>(p->total_k, 1), 0);
            for (int i = 0; i < n_inst; ++i) {
                InstDesc &d = p->inst[i];
                for (int kk = 0; kk < d.M; ++kk) {
                    kap2[d.k_off + kk] = (float)I[i].kappa[kperm[i][kk]];
                    kperm_all[d.k_off + kk] = kperm[i][kk];
                }
                d.perm_off = (long long)perm_all.size();
                for (int v : perm[i]) perm_all.push_back(v);
            }
            if ((rc2 = upload(p, &p->d_kappa, kap2.data(), kap2.size()))) return bail(rc2);
            if ((rc2 = upload(p, &p->d_perm, perm_all.data(), perm_all.size()))) return bail(rc2);
            if ((rc2 = upload(p, &p->d_kperm, kperm_all.data(), kperm_all.size()))) return bail(rc2);
            if ((rc2 = upload(p, &p->d_chunks, chunks.data(), chunks.size()))) return bail(rc2);
            // cluster-resident forward pass: every plate's rows in the registers of
            // one cluster (class layout, class blocks of at most 64 modes, at most
            // 512 threads a CTA), and all clusters resident at once; not for plans
            // whose options shape the streaming kernel's work split (tests of it)
            if (parity && o.force_split <= 0 && o.max_ctas <= 0 && !(p->debug_flags & 1)) {
                std::vector<int> cplates;
                int maxN = 0, maxM = 0, maxcls = 0;
                for (int i = 0; i < n_inst; ++i) {
                    const InstDesc &d = p->inst[i];
                    if (d.kind != MDX_KIND_PLATE || d.M == 0 || d.grouped) continue;
                    cplates.push_back(i);
                    maxN = std::max(maxN, d.N);
                    maxM = std::max(maxM, d.M);
                    for (int a = 0; a < 4; ++a) maxcls = std::max(maxcls, d.ncls[a]);
                }
                const int rl = cluster_row_len(maxcls);
                const int wk = (maxN + 31) / 32;
                if (!cplates.empty() && rl > 0 && !(p->debug_flags & 16)) {
                    for (int cs : {std::min(maxM, 8), 16}) {
                        if (cs > maxM && cs != std::min(maxM, 8)) break;
                        const int nkc = (maxM + cs - 1) / cs;
                        const int threads = nkc * wk * 32;
                        if (threads > cluster_max_threads(rl)) continue;
                        int fit = 0;
                        if (cluster_check(cs, threads, rl, &fit) != cudaSuccess) {
                            cudaGetLastError();
                            continue;
                        }
                        if (fit < (int)cplates.size()) continue;
                        std::vector<ClusterK> kinfo(std::max<long long>(p->total_k, 1));
                        for (const auto &it : items)
                            for (int ci = it.chunk0; ci < it.chunk1; ++ci)
                                for (int q = 0; q < chunks[ci].mc; ++q) {
                                    ClusterK &K = kinfo[p->inst[it.inst].k_off + chunks[ci].kl0 + q];
                                    K.off = chunks[ci].off;
                                    K.mc = chunks[ci].mc;
                                    K.kpos = q;
                                    K.c = chunks[ci].c;
                                }
                        if ((rc2 = upload(p, &p->d_kinfo, kinfo.data(), kinfo.size()))) return bail(rc2);
                        if ((rc2 = upload(p, &p->d_cplates, cplates.data(), cplates.size())))
                            return bail(rc2);
                        p->cluster_ok = true;
                        p->cl_cs = cs;
                        p->cl_nkc = nkc;
                        p->cl_wk = wk;
                        p->cl_rl = rl;
                        p->n_cplates = (int)cplates.size();
                        break;
                    }
                }
            }
            // contraction units: plates with a direction tensor (direction
            // derivative), and every plate (full dL/dH output)
            auto build_units = [&](bool all, std::vector<DirUnit> &units,
                                   std::vector<DirGroup> &groups) {
                if (parity) {
                    for (const auto &it : items) {
                        if (!all && !p->inst[it.inst].has_dir) continue;
                        for (int ci = it.chunk0; ci < it.chunk1; ++ci)
                            for (int q = 0; q < chunks[ci].mc; ++q) {
                                DirUnit u{};
                                u.inst = it.inst;
                                u.kl = chunks[ci].kl0 + q;
                                u.c = chunks[ci].c;
                                u.mc = chunks[ci].mc;
                                u.kpos = q;
                                u.off = chunks[ci].doff;
                                units.push_back(u);
                            }
                    }
                } else {
                    for (int i = 0; i < n_inst; ++i) {
                        const InstDesc &d = p->inst[i];
                        if (d.M == 0 || (!all && !d.has_dir)) continue;
                        for (int k = 0; k < d.M; ++k) {
                            DirUnit u{};
                            u.inst = i;
                            u.kl = k;
                            u.mc = 1;
                            units.push_back(u);
                        }
                    }
                }
                std::stable_sort(units.begin(), units.end(), [](const DirUnit &x, const DirUnit &y) {
                    return x.inst != y.inst ? x.inst < y.inst : x.kl < y.kl;
                });
                if (parity) {
                    // class-c stress modes of a plate are contiguous in internal order
                    size_t u0 = 0;
                    while (u0 < units.size()) {
                        size_t u1 = u0;
                        while (u1 < units.size() && units[u1].inst == units[u0].inst &&
                               units[u1].c == units[u0].c)
                            ++u1;
                        for (int a = 0; a < 4; ++a) {
                            DirGroup gr{};
                            gr.inst = units[u0].inst;
                            gr.c = units[u0].c;
                            gr.a = a;
                            gr.unit0 = (int)u0;
                            gr.nk = (int)(u1 - u0);
                            const InstDesc &d = p->inst[gr.inst];
                            if (d.ncls[a] > 0 && d.ncls[a ^ gr.c] > 0) groups.push_back(gr);
                        }
                        u0 = u1;
                    }
                }
            };
            std::vector<DirUnit> units, all_units;
            std::vector<DirGroup> groups, all_groups;
            build_units(false, units, groups);
            build_units(true, all_units, all_groups);
            p->n_dir_units = (int)units.size();
            p->n_dir_groups = (int)groups.size();
            if (!groups.empty() && !(p->debug_flags & 8)) {
                // tensor-core contraction: B rows for up to 16 stress modes x 16 rows;
                // the K chunk covers a whole class block when shared memory allows
                int nk_max = 1, kp_max = 8;
                for (const auto &g : groups) {
                    const InstDesc &d = p->inst[g.inst];
                    nk_max = std::max(nk_max, g.nk);
                    kp_max = std::max(kp_max, (d.ncls[g.a ^ g.c] + 7) & ~7);
                }
                const int nmax = 16 * std::min(16, nk_max);
                int kc = std::min(kp_max, 128);
                while (kc > 8 && dir_tc_smem_bytes(kc, nmax) + 1024 > (size_t)smem_optin) kc -= 8;
                const size_t need = dir_tc_smem_bytes(kc, nmax);
                if (need + 1024 <= (size_t)smem_optin) {
                    // at least 80 KB, so that at most two CTAs (256 tensor-memory
                    // columns each) share an SM
                    p->dir_tc_smem = std::min<size_t>(std::max<size_t>(need, 80 * 1024),
                                                      (size_t)smem_optin - 1024);
                    // the kernel's opt-in limit is shared by every plan: raise it
                    // to the device maximum rather than to this plan's need
                    MDX_CUDA(dir_tc_configure((size_t)smem_optin), "direction contraction attribute");
                    p->dir_tc_kc = kc;
                    p->dir_tc_nmax = nmax;
                }
            }
            if ((rc2 = upload(p, &p->d_dir_units, units.data(), units.size()))) return bail(rc2);
            if ((rc2 = upload(p, &p->d_dir_groups, groups.data(), groups.size()))) return bail(rc2);
            p->n_all_units = (int)all_units.size();
            p->n_all_groups = (int)all_groups.size();
            if ((rc2 = upload(p, &p->d_all_units, all_units.data(), all_units.size()))) return bail(rc2);
            if ((rc2 = upload(p, &p->d_all_groups, all_groups.data(), all_groups.size()))) return bail(rc2);
            std::vector<long long> dh_off(n_inst, 0);
            std::vector<int> dh_plates;
            for (int i = 0; i < n_inst; ++i) {
                const InstDesc &d = p->inst[i];
                dh_off[i] = p->dh_total;
                if (d.M > 0) {
                    p->dh_total += (long long)d.M * d.N * d.N;
                    dh_plates.push_back(i);
                }
            }
            p->n_dh_plates = (int)dh_plates.size();
            if ((rc2 = upload(p, &p->d_dh_off, dh_off.data(), dh_off.size()))) return bail(rc2);
            if ((rc2 = upload(p, &p->d_dh_plates, dh_plates.data(), dh_plates.size()))) return bail(rc2);
        }
        p->min_stage_floats = p->npad_max;
        if (parity) {
            for (const auto &it : items) {
                const InstDesc &d = p->inst[it.inst];
                for (int ci = it.chunk0; ci < it.chunk1; ++ci)
                    for (int a = 0; a < 4; ++a)
                        p->min_stage_floats = std::max(p->min_stage_floats, chunks[ci].mc * nb4(d.ncls[a]));
            }
        }
        // ring: stages of >= one padded row, filling the remaining shared memory
        p->smem_optin = smem_optin;
        {
            const int rcc = configure_tiles(p, o.stage_bytes, o.ring_stages);
            if (rcc) return bail(rcc);
        }
        update_l2_keep(p);
        int rc;
        if ((rc = upload(p, &p->d_items, items.data(), items.size()))) return bail(rc);
        if ((rc = upload(p, &p->d_cta_off, cta_off.data(), cta_off.size()))) return bail(rc);
        if ((rc = dalloc(p, reinterpret_cast<void **>(&p->d_part), 2 * p->part_stride * sizeof(float)))) return bail(rc);
    }
    int rc;
    if (p->any_grouped) {
        int dev_sms = 0, smem_optin = 0;
        MDX_CUDA(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, p->device), "attr");
        MDX_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device), "attr");
        if (o.max_ctas > 0) dev_sms = std::min(dev_sms, o.max_ctas);
        if ((rc = group_plan_build(&p->grp, I, p->inst, p->grouped, p->device, dev_sms,
                                   smem_optin - 2048, p->wait_limit)))
            return bail(rc);
        if ((rc = group_plan_set_kappa(p->grp, p->inst, p->h_kappa))) return bail(rc);
        if (!p->d_abort && (rc = dalloc(p, reinterpret_cast<void **>(&p->d_abort), 16))) return bail(rc);
    }
    if ((rc = upload(p, &p->d_inst, p->inst.data(), p->inst.size()))) return bail(rc);
    if ((rc = upload(p, &p->d_tension, p->tension.data(), p->tension.size()))) return bail(rc);
    if ((rc = dalloc(p, reinterpret_cast<void **>(&p->d_counters), n_inst * sizeof(unsigned)))) return bail(rc);
    if ((rc = dalloc(p, reinterpret_cast<void **>(&p->d_abort), 16))) return bail(rc);
    if ((rc = dalloc(p, reinterpret_cast<void **>(&p->d_state), kStateArrays * TM * sizeof(float)))) return bail(rc);
    *out = p;
    return MDX_OK;
}

size_t mdx_checkpoint_bytes(const mdx_plan *p, int steps, int K) {
    if (!p || steps <= 0 || K <= 0) return 0;
    const size_t nck = (size_t)((steps + K - 1) / K);
    return nck * kStateArrays * (size_t)p->total_modes * sizeof(float);
}

}  // extern "C"

namespace {

// Ring geometry: stage size (default 64 KB, halved while two stages do not fit
// beside the reverse sweep's buffers) and as many stages as shared memory
// allows, separately for the forward and the reverse launch.
int configure_tiles(mdx_plan *p, int stage_req, int ring_req) {
    const int smem_optin = p->smem_optin;
    const int min_stage = std::max(p->min_stage_floats, p->npad_max) * 4;
    int stage = stage_req > 0 ? stage_req : 64 * 1024;
    stage = std::max(stage, min_stage);
    stage = (stage + 15) & ~15;
    bool dir = false;
    for (const auto &d : p->inst) dir = dir || d.has_dir;
    const int us_fwd = 1, us_rev = 2, us_fused = 3;
    (void)dir;
    auto ufl = [&](int us) {
        // partial sums: dense row groups [kChunkK][slots][1024]; class chunks
        // [mc][u, z, u'][N_pad] (the direction pass needs no stored vector)
        if (p->parity) return p->mc_max * (us == us_fwd ? 2 : us) * p->npad_max;
        return kChunkK * us * kUPartFloats;
    };
    const int us_big = p->fuse ? us_fused : us_rev;
    if (stage_req <= 0) {
        while (stage > 16 * 1024 && stage / 2 >= min_stage &&
               plate_smem_bytes(2, stage, ufl(us_big), p->state_floats) + 1024 > (size_t)smem_optin)
            stage = ((stage / 2) + 15) & ~15;
    }
    int rings[3] = {0, 0, 0};
    size_t smems[3] = {0, 0, 0};
    const int n_cfg = p->fuse ? 3 : 2;
    for (int which = 0; which < n_cfg; ++which) {
        const int us = which == 0 ? us_fwd : (which == 1 ? us_rev : us_fused);
        const size_t fixed = plate_smem_bytes(0, stage, ufl(us), p->state_floats);
        if (fixed + 2 * (size_t)stage + 1024 > (size_t)smem_optin)
            return fail(MDX_ERR_UNSUPPORTED, "plate kernel needs %zu B of shared memory (> %d)",
                        fixed + 2 * (size_t)stage, smem_optin);
        int ring = ring_req > 0 ? ring_req : (int)((size_t)(smem_optin - 1024 - fixed) / stage);
        ring = std::max(2, std::min(ring, 16));
        const size_t need = plate_smem_bytes(ring, stage, ufl(us), p->state_floats);
        if (need > (size_t)smem_optin)
            return fail(MDX_ERR_UNSUPPORTED, "plate kernel needs %zu B of shared memory (> %d)",
                        need, smem_optin);
        rings[which] = ring;
        smems[which] = need;
    }
    // the device's limit, the same for every plan, so that plans of different
    // tile shapes can launch in any order
    MDX_CUDA(plate_set_smem_limit((size_t)smem_optin), "cudaFuncSetAttribute");
    p->stage_bytes = stage;
    p->u_slots_fwd = us_fwd;
    p->u_slots_rev = us_rev;
    p->u_floats_fwd = ufl(us_fwd);
    p->u_floats_rev = ufl(us_rev);
    p->u_floats_fused = p->fuse ? ufl(us_fused) : 0;
    p->ring_fwd = rings[0];
    p->ring_rev = rings[1];
    p->ring_fused = rings[2];
    p->smem_fwd = smems[0];
    p->smem_rev = smems[1];
    p->smem_fused = smems[2];
    return MDX_OK;
}

// Fraction of the per-step coupling stream marked evict_last in L2.  The
// automatic choice keeps about 70 % of the L2 for it (the rest serves the
// state, checkpoint and segment traffic): all of it when it fits, else the
// share that fits.
void update_l2_keep(mdx_plan *p) {
    if (p->l2_keep_req >= 0.0) {
        p->l2_keep = (float)std::min(1.0, p->l2_keep_req);
        return;
    }
    const double budget = 0.7 * (double)p->l2_bytes;
    p->l2_keep = (p->H_bytes_per_step > 0.0)
                     ? (float)std::min(1.0, budget / p->H_bytes_per_step) : 0.f;
}

PlateParams base_plate(mdx_plan *p, int mode, int steps, int n_begin, int total_steps) {
    PlateParams P{};
    P.inst = p->d_inst;
    P.items = p->d_items;
    P.cta_item_off = p->d_cta_off;
    P.coef = p->coef;
    P.H = p->d_H;
    P.dH = p->d_dH;
    P.kappa = p->d_kappa;
    P.n_inst = p->n_inst;
    P.steps = steps;
    P.n_begin = n_begin;
    P.total_steps = total_steps;
    P.mode = mode;
    P.stage_bytes = p->stage_bytes;
    P.ring_stages = (mode == MODE_FUSED) ? p->ring_fused
                    : (mode == MODE_REVERSE) ? p->ring_rev : p->ring_fwd;
    P.u_slots = (mode == MODE_FUSED) ? 3 : (mode == MODE_REVERSE) ? p->u_slots_rev : p->u_slots_fwd;
    P.u_floats = (mode == MODE_FUSED) ? p->u_floats_fused
                 : (mode == MODE_REVERSE) ? p->u_floats_rev : p->u_floats_fwd;
    P.parity = p->parity ? 1 : 0;
    P.npad_max = p->npad_max;
    P.chunks = p->d_chunks;
    P.perm = p->d_perm;
    P.max_spt = (p->npad_max + kPlateThreads - 1) / kPlateThreads;
    P.smem_state_floats = p->state_floats;
    P.total_modes = p->total_modes;
    P.part = p->d_part;
    P.part_stride = p->part_stride;
    P.counters = p->d_counters;
    P.abort_flag = p->d_abort;
    P.wait_limit = p->wait_limit;
    P.debug_flags = p->debug_flags;
    P.l2_keep = p->l2_keep;
    return P;
}

TensionParams base_tension(mdx_plan *p, int mode, int steps, int n_begin, int total_steps) {
    TensionParams T{};
    T.inst = p->d_inst;
    T.list = p->d_tension;
    T.n_list = (int)p->tension.size();
    T.coef = p->coef;
    T.steps = steps;
    T.n_begin = n_begin;
    T.total_steps = total_steps;
    T.mode = mode;
    T.total_modes = p->total_modes;
    return T;
}

int run_cluster(mdx_plan *p, const PlateParams &P, cudaStream_t s) {
    ClusterParams C{};
    C.inst = p->d_inst;
    C.plates = p->d_cplates;
    C.kinfo = p->d_kinfo;
    C.H = p->d_H;
    C.kappa = p->d_kappa;
    C.perm = p->d_perm;
    C.coef = p->coef;
    C.cs = p->cl_cs;
    C.nkc = p->cl_nkc;
    C.wk = p->cl_wk;
    C.steps = P.steps;
    C.n_begin = P.n_begin;
    C.total_steps = P.total_steps;
    C.exc = P.exc;
    C.audio = P.audio;
    C.state_io = P.state_io;
    C.total_modes = p->total_modes;
    C.status = P.status;
    mdx_plan::Rec rec{};
    if (p->profiling) {
        rec.which = 6;
        rec.bytes = (double)P.steps * p->H_bytes_per_step;
        MDX_CUDA(cudaEventCreate(&rec.a), "event");
        MDX_CUDA(cudaEventCreate(&rec.b), "event");
        MDX_CUDA(cudaEventRecord(rec.a, s), "event");
    }
    MDX_CUDA(launch_cluster(C, p->n_cplates, p->cl_rl, s), "cluster plate kernel");
    if (p->profiling) {
        MDX_CUDA(cudaEventRecord(rec.b, s), "event");
        p->recs.push_back(rec);
    }
    return MDX_OK;
}

int run_plate(mdx_plan *p, PlateParams &P, cudaStream_t s) {
    if (!p->any_plate) return MDX_OK;
    // a forward pass without checkpoints of a few small plates: cluster-resident
    if (p->cluster_ok && P.mode == MODE_FORWARD && !P.ckpt) return run_cluster(p, P, s);
    MDX_CUDA(cudaMemsetAsync(p->d_counters, 0, p->n_inst * sizeof(unsigned), s), "memset");
    MDX_CUDA(cudaMemsetAsync(p->d_abort, 0, sizeof(int), s), "memset");
    const size_t smem = (P.mode == MODE_FUSED) ? p->smem_fused
                        : (P.mode == MODE_REVERSE) ? p->smem_rev : p->smem_fwd;
    mdx_plan::Rec rec{};
    if (p->profiling) {
        rec.which = P.mode;
        rec.bytes = (double)P.steps * p->H_bytes_per_step;
        MDX_CUDA(cudaEventCreate(&rec.a), "event");
        MDX_CUDA(cudaEventCreate(&rec.b), "event");
        MDX_CUDA(cudaEventRecord(rec.a, s), "event");
    }
    MDX_CUDA(launch_plate(P, p->n_cta, smem, s), "plate kernel");
    if (p->profiling) {
        MDX_CUDA(cudaEventRecord(rec.b, s), "event");
        p->recs.push_back(rec);
    }
    return MDX_OK;
}

int run_grouped(mdx_plan *p, const PlateParams &P, cudaStream_t s) {
    if (!p->grp) return MDX_OK;
    MDX_CUDA(cudaMemsetAsync(p->d_abort, 0, sizeof(int), s), "memset");
    mdx_plan::Rec rec{};
    if (p->profiling) {
        rec.which = 5;
        rec.bytes = (double)P.steps * group_plan_bytes_per_step(p->grp);
        MDX_CUDA(cudaEventCreate(&rec.a), "event");
        MDX_CUDA(cudaEventCreate(&rec.b), "event");
        MDX_CUDA(cudaEventRecord(rec.a, s), "event");
    }
    MDX_CUDA(group_plan_launch(p->grp, p->d_inst, p->coef, P.steps, P.total_steps, P.exc, P.audio,
                               P.state_io, p->total_modes, P.status, p->d_abort, p->l2_keep, s),
             "grouped plate kernel");
    if (p->profiling) {
        MDX_CUDA(cudaEventRecord(rec.b, s), "event");
        p->recs.push_back(rec);
    }
    return MDX_OK;
}

int run_segment(mdx_plan *p, PlateParams &P, TensionParams &T, cudaStream_t s) {
    if (!p->tension.empty()) MDX_CUDA(launch_tension(T, p->tension_max_n, s), "tension kernel");
    const int rc = run_plate(p, P, s);
    if (rc) return rc;
    return run_grouped(p, P, s);
}

}  // namespace

extern "C" int mdx_simulate(mdx_plan *p, const float *exc, const double *q0, const double *qm1,
                            int steps, float *audio, double *q_end, double *qm1_end, int K,
                            void *ckpt, int *status, void *stream) {
    if (!p) return fail(MDX_ERR_ARG, "plan is NULL");
    if (steps < 0) return fail(MDX_ERR_ARG, "steps must be >= 0");
    if (ckpt && K <= 0) return fail(MDX_ERR_ARG, "checkpoint interval K must be > 0");
    if (ckpt && p->any_grouped)
        return fail(MDX_ERR_UNSUPPORTED,
                    "checkpoints (and mdx_grad) need per-instance coupling tensors: plan grouped "
                    "plates with group_engine = MDX_GROUP_OFF");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MDX_CUDA(cudaSetDevice(p->device), "cudaSetDevice");
    if (status) MDX_CUDA(cudaMemsetAsync(status, 0, p->n_inst * sizeof(int), s), "memset status");
    AuxInit a{q0, qm1, p->d_state, p->total_modes};
    MDX_CUDA(launch_init_state(a, s), "init state");
    if (steps > 0) {
        PlateParams P = base_plate(p, MODE_FORWARD, steps, 0, steps);
        TensionParams T = base_tension(p, MODE_FORWARD, steps, 0, steps);
        P.exc = T.exc = exc;
        P.audio = T.audio = audio;
        P.state_io = T.state_io = p->d_state;
        P.ckpt_K = T.ckpt_K = ckpt ? K : 1 << 30;
        P.ckpt = T.ckpt = static_cast<float *>(ckpt);
        P.status = T.status = status;
        int rc = run_segment(p, P, T, s);
        if (rc) return rc;
    }
    MDX_CUDA(launch_finalize_state(p->d_state, p->total_modes, q_end, qm1_end, s), "finalize");
    return MDX_OK;
}

namespace {

struct GradWork {
    float *seg_q, *seg_v, *adj, *gacc, *kacc, *tacc, *seg_w, *xe;
    float *seg_q2, *seg_v2;   // second segment buffer of the fused sweep (or null)
    double *dir_acc;
    size_t bytes;
};

GradWork grad_layout(const mdx_plan *p, int K, void *base) {
    const size_t TM = (size_t)p->total_modes, TK = (size_t)std::max<long long>(p->total_k, 1);
    auto al = [](size_t x) { return (x + 63) & ~size_t(63); };
    size_t off = 0;
    GradWork w{};
    char *b = static_cast<char *>(base);
    auto take = [&](size_t floats) {
        float *ptr = b ? reinterpret_cast<float *>(b + off) : nullptr;
        off += al(floats * sizeof(float));
        return ptr;
    };
    w.seg_q = take((size_t)(K + 1) * TM);
    w.seg_v = take((size_t)(K + 1) * TM);
    w.seg_q2 = p->fuse ? take((size_t)(K + 1) * TM) : nullptr;
    w.seg_v2 = p->fuse ? take((size_t)(K + 1) * TM) : nullptr;
    w.adj = take(AD_N * TM);
    w.gacc = take(2 * GA_N * TM);
    w.kacc = take(2 * TK);
    w.tacc = take(2 * (size_t)p->n_inst);
    // w^n and (xi, eta) per step: for the direction contraction and the full dL/dH
    const bool dir = p->n_all_units > 0;
    w.seg_w = dir ? take((size_t)K * TM) : nullptr;
    w.xe = dir ? take((size_t)K * 2 * TK) : nullptr;
    w.dir_acc = reinterpret_cast<double *>(take(8 * TK));
    w.bytes = off;
    return w;
}

}  // namespace

extern "C" size_t mdx_grad_workspace_bytes(const mdx_plan *p, int steps, int K) {
    if (!p || K <= 0) return 0;
    (void)steps;
    return grad_layout(p, K, nullptr).bytes;
}

extern "C" int mdx_grad(mdx_plan *p, const float *exc, const double *q0, const double *qm1,
                        int steps, const float *d_audio, int K, const void *ckpt, void *work,
                        size_t work_bytes, const mdx_grads *out, int *status, void *stream) {
    if (!p) return fail(MDX_ERR_ARG, "plan is NULL");
    if (p->any_grouped)
        return fail(MDX_ERR_UNSUPPORTED,
                    "mdx_grad needs per-instance coupling tensors: plan grouped plates with "
                    "group_engine = MDX_GROUP_OFF");
    if (steps <= 0) return fail(MDX_ERR_ARG, "steps must be > 0");
    if (K <= 0 || !ckpt) return fail(MDX_ERR_ARG, "mdx_grad needs the checkpoints of mdx_simulate (K > 0)");
    if (!d_audio) return fail(MDX_ERR_ARG, "d_audio is required");
    GradWork w = grad_layout(p, K, work);
    if (!work || work_bytes < w.bytes)
        return fail(MDX_ERR_ARG, "workspace of %zu bytes is smaller than the %zu bytes required",
                    work_bytes, w.bytes);
    (void)q0;
    (void)qm1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MDX_CUDA(cudaSetDevice(p->device), "cudaSetDevice");
    if (status) MDX_CUDA(cudaMemsetAsync(status, 0, p->n_inst * sizeof(int), s), "memset status");
    const size_t TM = (size_t)p->total_modes, TK = (size_t)std::max<long long>(p->total_k, 1);
    MDX_CUDA(cudaMemsetAsync(w.gacc, 0, 2 * GA_N * TM * sizeof(float), s), "memset");
    MDX_CUDA(cudaMemsetAsync(w.kacc, 0, 2 * TK * sizeof(float), s), "memset");
    MDX_CUDA(cudaMemsetAsync(w.dir_acc, 0, 4 * TK * sizeof(double), s), "memset");
    MDX_CUDA(cudaMemsetAsync(w.tacc, 0, 2 * p->n_inst * sizeof(float), s), "memset");
    double *dH_out = (out && out->d_H && p->dh_total > 0) ? out->d_H : nullptr;
    if (dH_out) MDX_CUDA(cudaMemsetAsync(dH_out, 0, p->dh_total * sizeof(double), s), "memset dH");
    MDX_CUDA(launch_init_adjoint(p->d_inst, p->n_inst, p->coef.c, d_audio, steps, w.adj,
                                 p->total_modes, 0, s),
             "init adjoint");
    const int nseg = (steps + K - 1) / K;
    float *const ckf = const_cast<float *>(static_cast<const float *>(ckpt));
    auto seg_len = [&](int sg) { return std::min(K, steps - sg * K); };
    // recompute segment sg from its checkpoint into (sq, sv), every state stored
    auto recompute = [&](int sg, float *sq, float *sv, bool plates, bool tension) -> int {
        PlateParams P = base_plate(p, MODE_RECOMPUTE, seg_len(sg), sg * K, steps);
        TensionParams T = base_tension(p, MODE_RECOMPUTE, seg_len(sg), sg * K, steps);
        P.exc = T.exc = exc;
        P.ckpt_K = T.ckpt_K = K;
        P.ckpt = T.ckpt = ckf;
        P.seg_q = T.seg_q = sq;
        P.seg_v = T.seg_v = sv;
        P.status = T.status = status;
        if (tension && !p->tension.empty())
            MDX_CUDA(launch_tension(T, p->tension_max_n, s), "tension kernel");
        return plates ? run_plate(p, P, s) : MDX_OK;
    };
    auto reverse_params = [&](int sg, int mode, float *sq, float *sv, PlateParams &P,
                              TensionParams &T) {
        P = base_plate(p, mode, seg_len(sg), sg * K, steps);
        T = base_tension(p, MODE_REVERSE, seg_len(sg), sg * K, steps);
        P.exc = T.exc = exc;
        P.ckpt_K = T.ckpt_K = K;
        P.ckpt = T.ckpt = ckf;
        P.seg_q = T.seg_q = sq;
        P.seg_v = T.seg_v = sv;
        P.status = T.status = status;
        P.ybar = T.ybar = d_audio;
        P.adj = T.adj = w.adj;
        P.gacc = T.gacc = w.gacc;
        P.kacc = w.kacc;
        P.seg_w = w.seg_w;
        P.xe = w.xe;
        P.xe_all = dH_out ? 1 : 0;
        P.total_k = p->total_k;
        T.tacc = w.tacc;
    };
    // direction contraction of segment sg (reads its stored states), and its
    // share of the full dL/dH
    auto direction = [&](int sg, const float *sq) -> int {
        if (dH_out) {
            DirParams D{};
            D.inst = p->d_inst;
            D.units = p->d_all_units;
            D.groups = p->parity ? p->d_all_groups : nullptr;
            D.n_groups = p->parity ? p->n_all_groups : 0;
            D.perm = p->d_perm;
            D.kappa = p->d_kappa;
            D.seg_q = sq;
            D.seg_w = w.seg_w;
            D.xe = w.xe;
            D.steps = seg_len(sg);
            D.total_modes = p->total_modes;
            D.total_k = p->total_k;
            D.dH_out = dH_out;
            D.dh_off = p->d_dh_off;
            D.kperm = p->d_kperm;
            MDX_CUDA(launch_dH_accumulate(D, p->n_all_units, s), "dL/dH accumulation");
        }
        if (p->n_dir_units <= 0) return MDX_OK;
        DirParams D{};
        D.inst = p->d_inst;
        D.units = p->d_dir_units;
        D.groups = p->parity ? p->d_dir_groups : nullptr;
        D.n_groups = p->parity ? p->n_dir_groups : 0;
        D.dH = p->d_dH;
        D.perm = p->d_perm;
        D.kappa = p->d_kappa;
        D.seg_q = sq;
        D.seg_w = w.seg_w;
        D.xe = w.xe;
        D.dir_acc = w.dir_acc;
        D.steps = seg_len(sg);
        D.total_modes = p->total_modes;
        D.total_k = p->total_k;
        D.tc_kc = p->parity ? p->dir_tc_kc : 0;
        D.tc_nmax = p->dir_tc_nmax;
        D.tc_smem = p->dir_tc_smem;
        D.status = status;
        mdx_plan::Rec rec{};
        if (p->profiling) {
            rec.which = 3;
            MDX_CUDA(cudaEventCreate(&rec.a), "event");
            MDX_CUDA(cudaEventCreate(&rec.b), "event");
            MDX_CUDA(cudaEventRecord(rec.a, s), "event");
        }
        MDX_CUDA(launch_dir_contract(D, p->n_dir_units, s), "direction contraction");
        if (p->profiling) {
            MDX_CUDA(cudaEventRecord(rec.b, s), "event");
            p->recs.push_back(rec);
        }
        return MDX_OK;
    };
    int rc;
    if (!p->fuse || !p->any_plate) {
        for (int sg = nseg - 1; sg >= 0; --sg) {
            if ((rc = recompute(sg, w.seg_q, w.seg_v, true, true))) return rc;
            PlateParams P;
            TensionParams T;
            reverse_params(sg, MODE_REVERSE, w.seg_q, w.seg_v, P, T);
            if ((rc = run_segment(p, P, T, s))) return rc;
            if ((rc = direction(sg, w.seg_q))) return rc;
        }
    } else {
        // Fused sweep: the launch for segment sg runs its adjoint (reading
        // buffer sg & 1) and, in the same pass over H per step, recomputes
        // segment sg - 1 from its checkpoint into the other buffer.  H is
        // streamed nseg + 1 times per gradient instead of 2 nseg times.
        float *bq[2] = {w.seg_q, w.seg_q2}, *bv[2] = {w.seg_v, w.seg_v2};
        if ((rc = recompute(nseg - 1, bq[(nseg - 1) & 1], bv[(nseg - 1) & 1], true, true))) return rc;
        for (int sg = nseg - 1; sg >= 1; --sg) {
            const int cur = sg & 1, prv = (sg - 1) & 1;
            PlateParams P;
            TensionParams T;
            reverse_params(sg, MODE_FUSED, bq[cur], bv[cur], P, T);
            P.steps = K;                      // segment sg - 1 is a full segment
            P.rev_steps = seg_len(sg);
            P.rec_begin = (sg - 1) * K;
            P.rseg_q = bq[prv];
            P.rseg_v = bv[prv];
            if ((rc = recompute(sg - 1, bq[prv], bv[prv], false, true))) return rc;
            if (!p->tension.empty()) MDX_CUDA(launch_tension(T, p->tension_max_n, s), "tension kernel");
            if ((rc = run_plate(p, P, s))) return rc;
            if ((rc = direction(sg, bq[cur]))) return rc;
        }
        PlateParams P;
        TensionParams T;
        reverse_params(0, MODE_REVERSE, bq[0], bv[0], P, T);
        if ((rc = run_segment(p, P, T, s))) return rc;
        if ((rc = direction(0, bq[0]))) return rc;
    }
    if (dH_out)
        MDX_CUDA(launch_dH_symmetrize(dH_out, p->d_dh_off, p->d_inst, p->d_dh_plates,
                                      p->n_dh_plates, s),
                 "dL/dH symmetrisation");
    GradEpilogue g{};
    g.inst = p->d_inst;
    g.n_inst = p->n_inst;
    g.total_modes = p->total_modes;
    g.total_k = p->total_k;
    g.omega2 = p->d_omega2;
    g.gamma = p->d_gamma;
    g.dt = p->d_dt;
    g.adj = w.adj;
    g.gacc = w.gacc;
    g.kacc = w.kacc;
    g.dir_acc = w.dir_acc;
    g.tacc = w.tacc;
    g.kperm = p->d_kperm;
    g.scheme = p->scheme;
    if (out) {
        g.d_omega2 = out->d_omega2;
        g.d_gamma = out->d_gamma;
        g.d_b = out->d_b;
        g.d_c = out->d_c;
        g.d_q0 = out->d_q0;
        g.d_qm1 = out->d_qm1;
        g.d_tau = out->d_tau;
        g.d_kappa = out->d_kappa;
        g.d_dir = out->d_dir;
    }
    MDX_CUDA(launch_grad_epilogue(g, 0, s), "grad epilogue");
    return MDX_OK;
}

extern "C" int mdx_coeffs_from_physics(int n, const double *lambda, double D, double T0, double rho,
                                       double s0, double s1, double *omega2, double *gamma) {
    if (n < 0 || !lambda || !omega2 || !gamma) return fail(MDX_ERR_ARG, "null argument");
    if (!(rho > 0.0)) return fail(MDX_ERR_ARG, "rho must be > 0");
    for (int m = 0; m < n; ++m) {
        const double l = lambda[m];
        omega2[m] = (D * l * l + T0 * l) / rho;   // Sec. 3.2, Eq. 13
        gamma[m] = s0 + s1 * omega2[m];           // damping family of Eq. 14
    }
    return MDX_OK;
}

extern "C" int mdx_difference_coefficients(int scheme, int n, const double *omega2,
                                           const double *gamma, double T, double *eps,
                                           double *rho, double *r) {
    if (scheme != MDX_SCHEME_SV && scheme != MDX_SCHEME_TF) return fail(MDX_ERR_ARG, "unknown scheme %d", scheme);
    if (n < 0 || (n > 0 && (!omega2 || !gamma || !eps || !rho || !r))) return fail(MDX_ERR_ARG, "null argument");
    if (!(T > 0.0) || !std::isfinite(T)) return fail(MDX_ERR_ARG, "T must be > 0");
    for (int m = 0; m < n; ++m) {
        const int rc = check_mode(scheme, omega2[m], gamma[m], T, 0, m);
        if (rc) return rc;
        const SchemeCoef k = scheme_coef(scheme, omega2[m], gamma[m], T);
        eps[m] = k.eps;
        rho[m] = k.rho;
        r[m] = k.r;
    }
    return MDX_OK;
}

extern "C" int mdx_coefficient_grads(int scheme, int n, const double *omega2, const double *gamma,
                                     double T, const double *A, const double *V, const double *F,
                                     double *d_omega2, double *d_gamma) {
    if (scheme != MDX_SCHEME_SV && scheme != MDX_SCHEME_TF) return fail(MDX_ERR_ARG, "unknown scheme %d", scheme);
    if (n < 0 || (n > 0 && (!omega2 || !gamma || !A || !V || !F || !d_omega2 || !d_gamma)))
        return fail(MDX_ERR_ARG, "null argument");
    if (!(T > 0.0) || !std::isfinite(T)) return fail(MDX_ERR_ARG, "T must be > 0");
    for (int m = 0; m < n; ++m) {
        const int rc = check_mode(scheme, omega2[m], gamma[m], T, 0, m);
        if (rc) return rc;
        scheme_grads(scheme, omega2[m], gamma[m], T, A[m], V[m], F[m], d_omega2 + m, d_gamma + m);
    }
    return MDX_OK;
}

extern "C" int mdx_coeffs_vjp(int n, const double *lambda, double D, double T0, double rho,
                              double s0, double s1, const double *d_omega2, const double *d_gamma,
                              double *dD, double *dT0, double *ds0, double *ds1, double *d_lambda) {
    if (n < 0 || !lambda || !d_omega2 || !d_gamma) return fail(MDX_ERR_ARG, "null argument");
    (void)s0;
    double aD = 0, aT = 0, a0 = 0, a1 = 0;
    for (int m = 0; m < n; ++m) {
        const double l = lambda[m];
        const double w2 = (D * l * l + T0 * l) / rho;
        const double gw = d_omega2[m] + s1 * d_gamma[m];   // total derivative through gamma(omega2)
        aD += gw * l * l / rho;
        aT += gw * l / rho;
        a0 += d_gamma[m];
        a1 += d_gamma[m] * w2;
        if (d_lambda) d_lambda[m] = gw * (2.0 * D * l + T0) / rho;
    }
    if (dD) *dD = aD;
    if (dT0) *dT0 = aT;
    if (ds0) *ds0 = a0;
    if (ds1) *ds1 = a1;
    return MDX_OK;
}

extern "C" int mdx_plan_set_coupling(mdx_plan *p, int i, const float *H, const float *dH) {
    if (!p) return fail(MDX_ERR_ARG, "plan is NULL");
    if (i < 0 || i >= p->n_inst) return fail(MDX_ERR_ARG, "instance %d outside the plan", i);
    const InstDesc &d = p->inst[i];
    if (d.grouped)
        return fail(MDX_ERR_UNSUPPORTED, "instance %d shares a grouped coupling tensor", i);
    if (d.kind != MDX_KIND_PLATE || d.M == 0)
        return fail(MDX_ERR_ARG, "instance %d is not a plate with stress modes", i);
    if (!H) return fail(MDX_ERR_ARG, "H is required");
    const int N = d.N;
    for (int which = 0; which < 2; ++which) {
        const float *src = which == 0 ? H : dH;
        if (!src) continue;
        for (int k = 0; k < d.M; ++k) {
            const float *Hk = src + (size_t)k * N * N;
            float amax = 0.f;
            for (size_t t = 0; t < (size_t)N * N; ++t) {
                if (!std::isfinite(Hk[t]))
                    return fail(MDX_ERR_NONFINITE, "instance %d: non-finite coupling entry", i);
                amax = std::max(amax, std::fabs(Hk[t]));
            }
            for (int a = 0; a < N; ++a)
                for (int b = a + 1; b < N; ++b)
                    if (std::fabs(Hk[(size_t)a * N + b] - Hk[(size_t)b * N + a]) > 1e-5f * amax + 1e-30f)
                        return fail(MDX_ERR_ARG, "instance %d: H[%d] is not symmetric", i, k);
        }
    }
    if (p->parity) {
        // the class layout stores only the class pattern: the new tensor must follow it
        std::vector<int> cls(N);
        for (int a = 0; a < 4; ++a)
            for (int q = 0; q < d.ncls[a]; ++q) cls[p->h_perm[i][d.ocls[a] + q]] = a;
        std::vector<int> kc(d.M);
        for (const auto &it : p->h_items) {
            if (it.inst != i) continue;
            for (int ci = it.chunk0; ci < it.chunk1; ++ci) {
                const ParityChunk &ch = p->h_chunks[ci];
                for (int q = 0; q < ch.mc; ++q) kc[p->h_kperm[d.k_off + ch.kl0 + q]] = ch.c;
            }
        }
        for (int k = 0; k < d.M; ++k) {
            const float *Hk = H + (size_t)k * N * N;
            float amax = 0.f;
            for (size_t t = 0; t < (size_t)N * N; ++t) amax = std::max(amax, std::fabs(Hk[t]));
            for (int x = 0; x < N; ++x)
                for (int y = 0; y < N; ++y)
                    if ((cls[x] ^ cls[y]) != kc[k] && std::fabs(Hk[(size_t)x * N + y]) > 1e-6f * amax)
                        return fail(MDX_ERR_ARG,
                                    "instance %d: H lies outside the plan's symmetry classes", i);
        }
    }
    MDX_CUDA(cudaSetDevice(p->device), "cudaSetDevice");
    MDX_CUDA(cudaDeviceSynchronize(), "synchronise");
    return upload_coupling(p, i, H, d.has_dir ? dH : nullptr);
}

extern "C" size_t mdx_linear_workspace_bytes(const mdx_plan *p, int steps) {
    if (!p || steps <= 0) return 0;
    const size_t nch = (size_t)((steps + kLinChunk - 1) / kLinChunk);
    return 2 * nch * (size_t)p->total_modes * 2 * sizeof(double);
}

extern "C" int mdx_simulate_linear(mdx_plan *p, const float *exc, const double *q0,
                                   const double *qm1, int steps, float *audio, double *q_end,
                                   double *qm1_end, void *work, size_t work_bytes, int *status,
                                   void *stream) {
    if (!p) return fail(MDX_ERR_ARG, "plan is NULL");
    if (steps < 0) return fail(MDX_ERR_ARG, "steps must be >= 0");
    const size_t need = mdx_linear_workspace_bytes(p, steps);
    if (steps > 0 && (!work || work_bytes < need))
        return fail(MDX_ERR_ARG, "workspace of %zu bytes is smaller than the %zu bytes required",
                    work_bytes, need);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MDX_CUDA(cudaSetDevice(p->device), "cudaSetDevice");
    if (status) MDX_CUDA(cudaMemsetAsync(status, 0, p->n_inst * sizeof(int), s), "memset status");
    if (steps == 0) {
        AuxInit a{q0, qm1, p->d_state, p->total_modes};
        MDX_CUDA(launch_init_state(a, s), "init state");
        MDX_CUDA(launch_finalize_state(p->d_state, p->total_modes, q_end, qm1_end, s), "finalize");
        return MDX_OK;
    }
    LinearParams L{};
    L.inst = p->d_inst;
    L.n_inst = p->n_inst;
    L.mode_inst = p->d_mode_inst;
    L.omega2 = p->d_omega2;
    L.gamma = p->d_gamma;
    L.dt = p->d_dt;
    L.b = p->d_b64;
    L.c = p->d_c64;
    L.scheme = p->scheme;
    L.steps = steps;
    L.total_steps = steps;
    L.L = kLinChunk;
    L.n_chunks = (steps + kLinChunk - 1) / kLinChunk;
    L.exc = exc;
    L.q0 = q0;
    L.qm1 = qm1;
    L.audio = audio;
    L.q_end = q_end;
    L.qm1_end = qm1_end;
    L.E = static_cast<double *>(work);
    L.S = L.E + (size_t)L.n_chunks * p->total_modes * 2;
    L.total_modes = p->total_modes;
    L.status = status;
    MDX_CUDA(launch_linear(L, s), "linear solver");
    return MDX_OK;
}

extern "C" int mdx_plan_group_work(const mdx_plan *p, double *bytes_per_step,
                                   double *flops_per_step) {
    if (!p) return fail(MDX_ERR_ARG, "plan is NULL");
    if (bytes_per_step) *bytes_per_step = group_plan_bytes_per_step(p->grp);
    if (flops_per_step) *flops_per_step = group_plan_flops_per_step(p->grp);
    return MDX_OK;
}

extern "C" int mdx_plan_set_profiling(mdx_plan *p, int enable) {
    if (!p) return fail(MDX_ERR_ARG, "plan is NULL");
    p->profiling = enable != 0;
    return MDX_OK;
}

extern "C" int mdx_plan_reset_stats(mdx_plan *p) {
    if (!p) return fail(MDX_ERR_ARG, "plan is NULL");
    for (auto &r : p->recs) {
        cudaEventSynchronize(r.b);
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    p->recs.clear();
    for (int i = 0; i < 7; ++i) p->stat_launch[i] = 0, p->stat_ms[i] = 0, p->stat_bytes[i] = 0;
    return MDX_OK;
}

extern "C" int mdx_plan_kernel_stats(mdx_plan *p, int which, long *launches, double *ms,
                                     double *bytes) {
    if (!p) return fail(MDX_ERR_ARG, "plan is NULL");
    if (which < 0 || which > 6) return fail(MDX_ERR_ARG, "which must be 0..6");
    for (auto &r : p->recs) {
        MDX_CUDA(cudaEventSynchronize(r.b), "event sync");
        float t = 0.f;
        MDX_CUDA(cudaEventElapsedTime(&t, r.a, r.b), "elapsed");
        p->stat_launch[r.which] += 1;
        p->stat_ms[r.which] += t;
        p->stat_bytes[r.which] += r.bytes;
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    p->recs.clear();
    if (launches) *launches = p->stat_launch[which];
    if (ms) *ms = p->stat_ms[which];
    if (bytes) *bytes = p->stat_bytes[which];
    return MDX_OK;
}

extern "C" int mdx_plan_configure(mdx_plan *p, int stage_bytes, int ring_stages) {
    if (!p) return fail(MDX_ERR_ARG, "plan is NULL");
    if (stage_bytes < 0 || ring_stages < 0 || (stage_bytes % 16) != 0)
        return fail(MDX_ERR_ARG, "stage_bytes must be a non-negative multiple of 16");
    if (!p->any_plate) return MDX_OK;
    MDX_CUDA(cudaSetDevice(p->device), "cudaSetDevice");
    return configure_tiles(p, stage_bytes, ring_stages);
}

extern "C" int mdx_plan_set_l2_keep(mdx_plan *p, double fraction) {
    if (!p) return fail(MDX_ERR_ARG, "plan is NULL");
    if (!(fraction <= 1.0) && !(fraction < 0.0)) return fail(MDX_ERR_ARG, "fraction must be <= 1");
    p->l2_keep_req = fraction < 0.0 ? -1.0 : fraction;
    update_l2_keep(p);
    return MDX_OK;
}

extern "C" double mdx_plan_l2_keep(const mdx_plan *p) { return p ? (double)p->l2_keep : 0.0; }

extern "C" int mdx_plan_tiles(const mdx_plan *p, int *stage_bytes, int *ring_fwd, int *ring_rev,
                              int *ctas) {
    if (!p) return fail(MDX_ERR_ARG, "plan is NULL");
    if (stage_bytes) *stage_bytes = p->stage_bytes;
    if (ring_fwd) *ring_fwd = p->ring_fwd;
    if (ring_rev) *ring_rev = p->ring_rev;
    if (ctas) *ctas = p->n_cta;
    return MDX_OK;
}

extern "C" int mdx_plan_set_coefficients(mdx_plan *p, const double *omega2, const double *gamma,
                                         const double *b, const double *c, const double *tau,
                                         const double *kappa) {
    if (!p) return fail(MDX_ERR_ARG, "plan is NULL");
    const size_t TM = (size_t)p->total_modes;
    std::vector<double> w2 = omega2 ? std::vector<double>(omega2, omega2 + TM) : p->h_omega2;
    std::vector<double> gm = gamma ? std::vector<double>(gamma, gamma + TM) : p->h_gamma;
    std::vector<double> bb = b ? std::vector<double>(b, b + TM) : p->h_b;
    std::vector<double> cc = c ? std::vector<double>(c, c + TM) : p->h_c;
    std::vector<double> tt = tau ? std::vector<double>(tau, tau + p->n_inst) : p->h_tau;
    std::vector<double> kp = kappa ? std::vector<double>(kappa, kappa + p->total_k) : p->h_kappa;
    for (int i = 0; i < p->n_inst; ++i) {
        const InstDesc &d = p->inst[i];
        const double T = p->dt[i];
        for (int m = 0; m < d.N; ++m) {
            const size_t g = d.mode_off + m;
            if (!std::isfinite(w2[g]) || !std::isfinite(gm[g]) || !std::isfinite(bb[g]) || !std::isfinite(cc[g]))
                return fail(MDX_ERR_NONFINITE, "instance %d mode %d: non-finite coefficient", i, m);
            const int rc = check_mode(p->scheme, w2[g], gm[g], T, i, m);
            if (rc) return rc;
        }
        if (!std::isfinite(tt[i]) || tt[i] < 0.0) return fail(MDX_ERR_ARG, "instance %d: tau must be finite and >= 0", i);
    }
    for (double v : kp)
        if (!std::isfinite(v)) return fail(MDX_ERR_NONFINITE, "non-finite kappa");
    std::vector<float> eps(TM), rw2(TM), rr(TM), bf(TM), cf(TM), rwl(TM), cl(TM);
    for (int i = 0; i < p->n_inst; ++i) {
        const InstDesc &d = p->inst[i];
        const double T = p->dt[i];
        for (int m = 0; m < d.N; ++m) {
            const size_t g = d.mode_off + m;
            const ModeF32 k = mode_f32(p->scheme, w2[g], gm[g], T);
            eps[g] = k.eps;
            rw2[g] = k.rho_hi;
            rwl[g] = k.rho_lo;
            rr[g] = k.r;
            bf[g] = (float)bb[g];
            cf[g] = (float)cc[g];
            cl[g] = (float)(cc[g] - (double)cf[g]);
        }
    }
    MDX_CUDA(cudaSetDevice(p->device), "cudaSetDevice");
    MDX_CUDA(cudaDeviceSynchronize(), "synchronise");
    float *dc = p->d_coef_all;
    MDX_CUDA(cudaMemcpy(dc, eps.data(), TM * 4, cudaMemcpyHostToDevice), "upload");
    MDX_CUDA(cudaMemcpy(dc + TM, rw2.data(), TM * 4, cudaMemcpyHostToDevice), "upload");
    MDX_CUDA(cudaMemcpy(dc + 2 * TM, rr.data(), TM * 4, cudaMemcpyHostToDevice), "upload");
    MDX_CUDA(cudaMemcpy(dc + 3 * TM, bf.data(), TM * 4, cudaMemcpyHostToDevice), "upload");
    MDX_CUDA(cudaMemcpy(dc + 4 * TM, cf.data(), TM * 4, cudaMemcpyHostToDevice), "upload");
    MDX_CUDA(cudaMemcpy(dc + 6 * TM, rwl.data(), TM * 4, cudaMemcpyHostToDevice), "upload");
    MDX_CUDA(cudaMemcpy(dc + 7 * TM, cl.data(), TM * 4, cudaMemcpyHostToDevice), "upload");
    MDX_CUDA(cudaMemcpy(p->d_omega2, w2.data(), TM * 8, cudaMemcpyHostToDevice), "upload");
    MDX_CUDA(cudaMemcpy(p->d_gamma, gm.data(), TM * 8, cudaMemcpyHostToDevice), "upload");
    MDX_CUDA(cudaMemcpy(p->d_b64, bb.data(), TM * 8, cudaMemcpyHostToDevice), "upload");
    MDX_CUDA(cudaMemcpy(p->d_c64, cc.data(), TM * 8, cudaMemcpyHostToDevice), "upload");
    // tau lives in the instance table; kappa in internal (class-sorted) order
    for (int i = 0; i < p->n_inst; ++i) p->inst[i].taup = (p->inst[i].kind == MDX_KIND_TENSION) ? (float)tt[i] : 0.f;
    MDX_CUDA(cudaMemcpy(p->d_inst, p->inst.data(), p->inst.size() * sizeof(InstDesc), cudaMemcpyHostToDevice), "upload");
    if (p->total_k > 0 && p->d_kappa) {
        std::vector<float> k2(p->total_k);
        for (int i = 0; i < p->n_inst; ++i) {
            const InstDesc &d = p->inst[i];
            for (int kk = 0; kk < d.M; ++kk) {
                const int ku = p->h_kperm.empty() ? kk : p->h_kperm[d.k_off + kk];
                k2[d.k_off + kk] = (float)kp[d.k_off + ku];
            }
        }
        MDX_CUDA(cudaMemcpy(p->d_kappa, k2.data(), p->total_k * 4, cudaMemcpyHostToDevice), "upload");
    }
    if (p->grp) {
        const int rc = group_plan_set_kappa(p->grp, p->inst, kp);
        if (rc) return rc;
    }
    p->h_omega2 = w2;
    p->h_gamma = gm;
    p->h_b = bb;
    p->h_c = cc;
    p->h_tau = tt;
    p->h_kappa = kp;
    return MDX_OK;
}
