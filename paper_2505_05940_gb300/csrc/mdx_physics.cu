// Host FP64 map from the physical description of a string, membrane or plate
// to the modal coefficients a plan takes, and the vector-Jacobian product
// that carries the plan's per-mode gradients back to the physical
// parameters (tension, stiffness, aspect ratio, damping).
//
//   Laplacian eigenpairs, Sec. 3, Eq. 2: fixed string lambda = (mu pi / L)^2,
//     simply supported rectangle lambda = (m pi / Lx)^2 + (n pi / Ly)^2, the
//     first N modes by ascending lambda (ties by (m, n)); unit-norm shapes
//     sqrt(2/L) sin(mu pi x/L) and 2/sqrt(Lx Ly) sin(m pi x/Lx) sin(n pi y/Ly).
//   Oscillator coefficients, Sec. 3.2, Eq. 13-14:
//     omega^2 = (D lambda^2 + T0 lambda) / rho,  gamma = sigma0 + sigma1 omega^2.
//   Point force and pickup: b = Phi(x_s) / rho, c = Phi(x_o).
//   Tension modulation, Sec. 3.1, Eq. 4 (divided by rho for the modal form):
//     string tau = EA / (2 L), membrane tau = E h / (2 Lx Ly (1 - nu^2)).
//   Von Karman scale, Sec. 3.1, Eq. 9: kappa_k = E / (2 rho_vol zeta_k^4).
//   Stability cut: the modes from the first one with omega T >= omega_dt_max
//     on are dropped (Stormer-Verlet, Eq. 20, needs omega T < 2); a
//     shortened plate keeps the same fraction of its stress modes.
//
// With the area Lx Ly fixed and the strike and pickup points given relative
// to the sides, b, c, the mode-shape scale and the membrane's tau do not
// depend on the aspect a = Ly / Lx; lambda does, through
//     lambda_mn(a) = (m pi)^2 a / A + (n pi)^2 / (A a),
// kappa does through zeta^4(a), and H does (its contribution <dL/dH, dH/da>
// comes from mdx_grad).
#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/mdx.h"
#include "mdx_internal.h"

using namespace mdx;

namespace {

constexpr double kPi = 3.14159265358979323846;

int phys_fail(int code, const char *msg) { return set_last_error(code, msg); }

struct Mode {
    double lam;
    int m, n;
};

// First n modes of the shape in ascending lambda, ties by (m, n).  The
// rectangle's candidates are (m, n) in [1, K]^2, with K doubled until the
// n-th eigenvalue lies below every excluded one.
std::vector<Mode> laplacian_modes(const mdx_physics &ph, int n) {
    std::vector<Mode> out;
    if (ph.shape == MDX_SHAPE_STRING) {
        for (int mu = 1; mu <= n; ++mu) {
            const double k = kPi * mu / ph.length;
            out.push_back({k * k, mu, 0});
        }
        return out;
    }
    const double Lx = std::sqrt(ph.area / ph.aspect), Ly = std::sqrt(ph.area * ph.aspect);
    int K = (int)std::sqrt(4.0 * n / kPi * std::max(Lx / Ly, Ly / Lx)) + 6;
    for (;;) {
        std::vector<Mode> cand;
        cand.reserve((size_t)K * K);
        for (int m = 1; m <= K; ++m)
            for (int k = 1; k <= K; ++k) {
                const double a = kPi * m / Lx, b = kPi * k / Ly;
                cand.push_back({a * a + b * b, m, k});
            }
        std::sort(cand.begin(), cand.end(), [](const Mode &x, const Mode &y) {
            if (x.lam != y.lam) return x.lam < y.lam;
            if (x.m != y.m) return x.m < y.m;
            return x.n < y.n;
        });
        const double ex = kPi * (K + 1) / Lx, ey = kPi * (K + 1) / Ly;
        const double bound = std::min(ex * ex, ey * ey);
        if (cand[n - 1].lam < bound) {
            cand.resize(n);
            return cand;
        }
        K *= 2;
    }
}

double shape_at(const mdx_physics &ph, const Mode &md, const double *x) {
    if (ph.shape == MDX_SHAPE_STRING)
        return std::sqrt(2.0 / ph.length) * std::sin(md.m * kPi * x[0]);
    const double Lx = std::sqrt(ph.area / ph.aspect), Ly = std::sqrt(ph.area * ph.aspect);
    return 2.0 / std::sqrt(Lx * Ly) * std::sin(md.m * kPi * x[0]) * std::sin(md.n * kPi * x[1]);
}

int check_physics(const mdx_physics *ph) {
    if (!ph) return phys_fail(MDX_ERR_ARG, "physics description is NULL");
    if (ph->kind != MDX_KIND_TENSION && ph->kind != MDX_KIND_PLATE)
        return phys_fail(MDX_ERR_ARG, "kind must be MDX_KIND_TENSION or MDX_KIND_PLATE");
    if (ph->shape != MDX_SHAPE_STRING && ph->shape != MDX_SHAPE_RECTANGLE)
        return phys_fail(MDX_ERR_ARG, "shape must be MDX_SHAPE_STRING or MDX_SHAPE_RECTANGLE");
    if (ph->kind == MDX_KIND_PLATE && ph->shape != MDX_SHAPE_RECTANGLE)
        return phys_fail(MDX_ERR_ARG, "a plate is a rectangle");
    if (ph->n_phi < 1 || ph->n_phi > MDX_MAX_PHI)
        return phys_fail(MDX_ERR_UNSUPPORTED, "n_phi outside [1, MDX_MAX_PHI]");
    if (ph->n_psi < 0 || ph->n_psi > MDX_MAX_PSI)
        return phys_fail(MDX_ERR_UNSUPPORTED, "n_psi outside [0, MDX_MAX_PSI]");
    if (!(ph->dt > 0.0) || !std::isfinite(ph->dt)) return phys_fail(MDX_ERR_ARG, "dt must be > 0");
    if (ph->shape == MDX_SHAPE_STRING && !(ph->length > 0.0))
        return phys_fail(MDX_ERR_ARG, "string length must be > 0");
    if (ph->shape == MDX_SHAPE_RECTANGLE && !(ph->area > 0.0 && ph->aspect > 0.0))
        return phys_fail(MDX_ERR_ARG, "rectangle area and aspect must be > 0");
    if (!(ph->rho > 0.0)) return phys_fail(MDX_ERR_ARG, "rho must be > 0");
    const double v[] = {ph->D, ph->T0, ph->sigma0, ph->sigma1, ph->strike[0], ph->strike[1],
                        ph->pickup[0], ph->pickup[1], ph->tension_stiffness, ph->vk_scale,
                        ph->omega_dt_max};
    for (double x : v)
        if (!std::isfinite(x)) return phys_fail(MDX_ERR_NONFINITE, "non-finite physical parameter");
    if (ph->kind == MDX_KIND_PLATE && ph->n_psi > 0 && ph->vk_scale != 0.0 && ph->zeta4) {
        for (int k = 0; k < ph->n_psi; ++k)
            if (!(ph->zeta4[k] > 0.0) || !std::isfinite(ph->zeta4[k]))
                return phys_fail(MDX_ERR_ARG, "zeta4 must be finite and > 0");
    }
    return MDX_OK;
}

// Modes kept by the stability cut and the stress modes kept with them.
void kept_counts(const mdx_physics &ph, const std::vector<Mode> &modes, int *n_eff, int *m_eff) {
    int n = (int)modes.size();
    if (ph.omega_dt_max > 0.0) {
        for (int i = 0; i < (int)modes.size(); ++i) {
            const double l = modes[i].lam;
            const double w2 = (ph.D * l * l + ph.T0 * l) / ph.rho;
            if (!(std::sqrt(w2) * ph.dt < ph.omega_dt_max)) {
                n = i;
                break;
            }
        }
    }
    *n_eff = n;
    int M = (ph.kind == MDX_KIND_PLATE) ? ph.n_psi : 0;
    if (n < ph.n_phi && M > 0) M = std::min(M, std::max(1, (M * n) / ph.n_phi));
    *m_eff = M;
}

}  // namespace

extern "C" int mdx_modal_from_physics(const mdx_physics *ph, mdx_modal *out) {
    int rc = check_physics(ph);
    if (rc) return rc;
    if (!out) return phys_fail(MDX_ERR_ARG, "output is NULL");
    if (!out->lambda || !out->omega2 || !out->gamma || !out->b || !out->c)
        return phys_fail(MDX_ERR_ARG, "lambda, omega2, gamma, b and c are required");
    const std::vector<Mode> modes = laplacian_modes(*ph, ph->n_phi);
    int n_eff = 0, m_eff = 0;
    kept_counts(*ph, modes, &n_eff, &m_eff);
    if (n_eff < 1) return phys_fail(MDX_ERR_UNSTABLE, "every mode is beyond the stability cut");
    for (int i = 0; i < n_eff; ++i) {
        const Mode &md = modes[i];
        const double l = md.lam;
        const double w2 = (ph->D * l * l + ph->T0 * l) / ph->rho;   // Eq. 13
        if (out->labels) {
            out->labels[2 * i] = md.m;
            out->labels[2 * i + 1] = md.n;
        }
        out->lambda[i] = l;
        out->omega2[i] = w2;
        out->gamma[i] = ph->sigma0 + ph->sigma1 * w2;                // Eq. 14 family
        out->b[i] = shape_at(*ph, md, ph->strike) / ph->rho;
        out->c[i] = shape_at(*ph, md, ph->pickup);
    }
    out->tau = 0.0;
    if (ph->kind == MDX_KIND_TENSION && ph->tension_stiffness != 0.0) {
        // Eq. 4: tau = EA / (2 L) (string) or E h / (2 Lx Ly (1 - nu^2)) (membrane)
        const double span = (ph->shape == MDX_SHAPE_STRING) ? ph->length : ph->area;
        out->tau = ph->tension_stiffness / (2.0 * span) / ph->rho;
    }
    if (ph->kind == MDX_KIND_PLATE && ph->vk_scale != 0.0 && m_eff > 0 && ph->zeta4) {
        if (!out->kappa) return phys_fail(MDX_ERR_ARG, "kappa output is required when zeta4 is given");
        for (int k = 0; k < m_eff; ++k) out->kappa[k] = ph->vk_scale / ph->zeta4[k];  // Eq. 9
    }
    out->n_phi = n_eff;
    out->n_psi = (ph->kind == MDX_KIND_PLATE && ph->vk_scale != 0.0) ? m_eff : 0;
    return MDX_OK;
}

extern "C" int mdx_physics_vjp(const mdx_physics *ph, int n_phi, int n_psi,
                               const double *d_omega2, const double *d_gamma, double d_tau,
                               const double *d_kappa, double d_dir, const double *dzeta4,
                               mdx_physics_grads *out) {
    int rc = check_physics(ph);
    if (rc) return rc;
    if (!out || !d_omega2 || !d_gamma) return phys_fail(MDX_ERR_ARG, "null argument");
    if (n_phi < 1 || n_phi > ph->n_phi) return phys_fail(MDX_ERR_ARG, "n_phi outside [1, requested]");
    if (n_psi < 0 || n_psi > ph->n_psi) return phys_fail(MDX_ERR_ARG, "n_psi outside [0, requested]");
    if (n_psi > 0 && (!d_kappa || !ph->zeta4))
        return phys_fail(MDX_ERR_ARG, "d_kappa and zeta4 are required when n_psi > 0");
    const std::vector<Mode> modes = laplacian_modes(*ph, n_phi);
    const bool rect = ph->shape == MDX_SHAPE_RECTANGLE;
    const double A = ph->area, a = ph->aspect;
    double gD = 0, gT = 0, gs0 = 0, gs1 = 0, ga = 0;
    for (int i = 0; i < n_phi; ++i) {
        const double l = modes[i].lam;
        const double w2 = (ph->D * l * l + ph->T0 * l) / ph->rho;
        // total derivative through omega^2, gamma = sigma0 + sigma1 omega^2
        const double gw = d_omega2[i] + ph->sigma1 * d_gamma[i];
        gD += gw * l * l / ph->rho;
        gT += gw * l / ph->rho;
        gs0 += d_gamma[i];
        gs1 += d_gamma[i] * w2;
        if (rect) {
            const double pm = kPi * modes[i].m, pn = kPi * modes[i].n;
            const double dl_da = pm * pm / A - pn * pn / (A * a * a);
            ga += gw * (2.0 * ph->D * l + ph->T0) / ph->rho * dl_da;
        }
    }
    if (rect && ph->kind == MDX_KIND_PLATE && n_psi > 0 && dzeta4) {
        // kappa_k = s / zeta_k^4  =>  d kappa_k / da = -kappa_k dzeta_k^4/da / zeta_k^4
        for (int k = 0; k < n_psi; ++k) {
            const double z = ph->zeta4[k];
            ga += d_kappa[k] * (-ph->vk_scale / (z * z)) * dzeta4[k];
        }
    }
    if (rect) ga += d_dir;
    // nonlinear scales: tau' = s_t / (2 span rho) (Eq. 4), kappa_k = s_vk / zeta_k^4 (Eq. 9)
    double gst = 0.0, gvk = 0.0;
    if (ph->kind == MDX_KIND_TENSION) {
        const double span = (ph->shape == MDX_SHAPE_STRING) ? ph->length : ph->area;
        gst = d_tau / (2.0 * span * ph->rho);
    } else {
        for (int k = 0; k < n_psi; ++k) gvk += d_kappa[k] / ph->zeta4[k];
    }
    out->d_tension_stiffness = gst;
    out->d_vk_scale = gvk;
    out->d_T0 = gT;
    out->d_D = gD;
    out->d_aspect = rect ? ga : 0.0;
    out->d_sigma0 = gs0;
    out->d_sigma1 = gs1;
    return MDX_OK;
}
