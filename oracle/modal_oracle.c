/*
 * FP64 CPU oracle for the per-time-step modal update.
 *
 * TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's
 * CPU-baseline leg use this file.  It shares no code with the CUDA library.
 *
 * What it computes (all in double precision, plain loops, no blocking):
 *   - Stormer-Verlet update, Sec. 3.2, Eq. 20:
 *       q^{n+1} = g*q^n + p*q^{n-1} + r*(fext^n - fnl(q^n))
 *     with g, p, r supplied by the caller (Eqs. 21-23 are evaluated in
 *     physics_oracle.py) and fext^n_mu = b_mu * e^n.
 *   - Tension-modulated force (Kirchhoff-Carrier string / Berger membrane),
 *     Sec. 3.1, Eq. 8 read with unit-norm modes:
 *       fnl_mu = tau' * lambda_mu * q_mu * sum_nu lambda_nu q_nu^2
 *   - Von Karman force, Sec. 3.1, Eq. 9, with C^s_{pn} = H^n_{ps} (Sec. 4.3.3):
 *       eta_n  = sum_{q,r} H^n_{qr} q_q q_r
 *       fnl_s  = sum_n kappa_n * eta_n * sum_p H^n_{ps} q_p,
 *     kappa_n = E / (2 rho zeta_n^4) supplied by the caller.
 *   - Pickup y^n = sum_mu c_mu q^{n+1}_mu (displacement at one point).
 *   - Reverse-mode derivative of a loss L(y) through the whole recursion,
 *     given dL/dy (hand-written adjoint recursion; pinned against central
 *     finite differences in the tests).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TENSION 0
#define ORC_PLATE 1

typedef struct {
    int kind;            /* ORC_TENSION or ORC_PLATE */
    int N;               /* transverse modes */
    int M;               /* stress modes (plate) */
    const double *g, *p, *r, *b, *c;
    const double *lam;   /* [N] eigenvalues (tension kind) */
    double taup;         /* tau / rho_lin (tension kind) */
    const double *H;     /* [M][N][N] (plate) */
    const double *kappa; /* [M] (plate) */
} orc_model;

/* u: [M][N] scratch, eta: [M] scratch (plate); returns S = sum lam q^2 (tension) */
static double nl_force(const orc_model *m, const double *q, double *f, double *u, double *eta)
{
    int N = m->N;
    if (m->kind == ORC_TENSION) {
        double S = 0.0;
        for (int nu = 0; nu < N; ++nu) S += m->lam[nu] * q[nu] * q[nu];
        for (int mu = 0; mu < N; ++mu) f[mu] = m->taup * m->lam[mu] * q[mu] * S;
        return S;
    }
    int M = m->M;
    for (int k = 0; k < M; ++k) {
        const double *Hk = m->H + (size_t)k * N * N;
        double e = 0.0;
        /* u_s = sum_p H_ps q_p, each sum taken over p = 0, 1, ... in order;
           H^k is walked row by row (memory order only, same arithmetic) */
        double *uk = u + (size_t)k * N;
        for (int s = 0; s < N; ++s) uk[s] = 0.0;
        for (int pp = 0; pp < N; ++pp)
            for (int s = 0; s < N; ++s) uk[s] += Hk[(size_t)pp * N + s] * q[pp];
        for (int a = 0; a < N; ++a)
            for (int bb = 0; bb < N; ++bb) e += Hk[(size_t)a * N + bb] * q[a] * q[bb];
        eta[k] = e;
    }
    for (int s = 0; s < N; ++s) {
        double acc = 0.0;
        for (int k = 0; k < M; ++k) acc += m->kappa[k] * eta[k] * u[(size_t)k * N + s];
        f[s] = acc;
    }
    return 0.0;
}

static void *xcalloc(size_t n, size_t sz) { return calloc(n ? n : 1, sz); }

/*
 * Forward run.  e: [steps]; q0, qm1: [N]; y: [steps];
 * traj (optional, may be NULL): [(steps+2)][N] holding q^{-1}, q^0, ..., q^{steps}.
 * qN, qNm1 (optional): final q^{steps}, q^{steps-1}.
 * Returns 0, or 1 if a non-finite value appeared.
 */
int orc_forward(int kind, int N, int M, const double *g, const double *p, const double *r,
                const double *b, const double *c, const double *lam, double taup,
                const double *H, const double *kappa, int steps, const double *e,
                const double *q0, const double *qm1, double *y, double *traj,
                double *qN, double *qNm1)
{
    orc_model m = {kind, N, M, g, p, r, b, c, lam, taup, H, kappa};
    double *qprev = xcalloc(N, sizeof(double)), *qcur = xcalloc(N, sizeof(double));
    double *qnext = xcalloc(N, sizeof(double)), *f = xcalloc(N, sizeof(double));
    double *u = xcalloc((size_t)(M > 0 ? M : 1) * N, sizeof(double));
    double *eta = xcalloc(M > 0 ? M : 1, sizeof(double));
    int bad = 0;
    memcpy(qprev, qm1, N * sizeof(double));
    memcpy(qcur, q0, N * sizeof(double));
    if (traj) {
        memcpy(traj, qprev, N * sizeof(double));
        memcpy(traj + N, qcur, N * sizeof(double));
    }
    for (int n = 0; n < steps; ++n) {
        nl_force(&m, qcur, f, u, eta);
        double yn = 0.0;
        for (int mu = 0; mu < N; ++mu) {
            double F = b[mu] * e[n] - f[mu];
            qnext[mu] = g[mu] * qcur[mu] + p[mu] * qprev[mu] + r[mu] * F;
            yn += c[mu] * qnext[mu];
        }
        y[n] = yn;
        if (!isfinite(yn)) bad = 1;
        double *t = qprev; qprev = qcur; qcur = qnext; qnext = t;
        if (traj) memcpy(traj + (size_t)(n + 2) * N, qcur, N * sizeof(double));
    }
    if (qN) memcpy(qN, qcur, N * sizeof(double));
    if (qNm1) memcpy(qNm1, qprev, N * sizeof(double));
    free(qprev); free(qcur); free(qnext); free(f); free(u); free(eta);
    return bad;
}

/* out = J(q) w, the Jacobian of the nonlinear force (symmetric: fnl = grad V). */
static void jac_vec(const orc_model *m, const double *q, const double *w, double *out,
                    double *u, double *eta, double *z)
{
    int N = m->N;
    if (m->kind == ORC_TENSION) {
        double S = 0.0, P = 0.0;
        for (int nu = 0; nu < N; ++nu) {
            S += m->lam[nu] * q[nu] * q[nu];
            P += m->lam[nu] * q[nu] * w[nu];
        }
        /* d/dq_nu [tau' lam_mu q_mu S] = tau' lam_mu (delta S + 2 q_mu lam_nu q_nu) */
        for (int mu = 0; mu < N; ++mu)
            out[mu] = m->taup * m->lam[mu] * (S * w[mu] + 2.0 * q[mu] * P);
        return;
    }
    int M = m->M;
    for (int s = 0; s < N; ++s) out[s] = 0.0;
    for (int k = 0; k < M; ++k) {
        const double *Hk = m->H + (size_t)k * N * N;
        double uq = 0.0, uw = 0.0;
        /* u = H^k q, z = H^k w, each sum over p in order (row-by-row walk) */
        for (int s = 0; s < N; ++s) { u[s] = 0.0; z[s] = 0.0; }
        for (int pp = 0; pp < N; ++pp)
            for (int s = 0; s < N; ++s) {
                u[s] += Hk[(size_t)pp * N + s] * q[pp];
                z[s] += Hk[(size_t)pp * N + s] * w[pp];
            }
        for (int s = 0; s < N; ++s) {
            uq += u[s] * q[s];
            uw += u[s] * w[s];
        }
        eta[k] = uq;
        /* d/dq [kappa eta u] w = kappa (2 u (u.w) + eta H w) */
        for (int s = 0; s < N; ++s) out[s] += m->kappa[k] * (2.0 * u[s] * uw + uq * z[s]);
    }
}

/*
 * Reverse run.  traj: [(steps+2)][N] from orc_forward; ybar: [steps] = dL/dy.
 * Outputs (all accumulated from zero, any may be NULL except the arrays the
 * recursion itself needs):
 *   dq0, dqm1 [N]: dL/dq^0, dL/dq^{-1}
 *   dg, dp, dr, db, dc [N]: dL/d(coefficient)
 *   dtau [1] (tension) : dL/dtau'
 *   dkappa [M] (plate): dL/dkappa_n
 *   dH [M][N][N] (plate): dL/dH, symmetrised over the last two indices
 * Adjoint variables a^n = dL/dq^n obey, for n = steps..1,
 *   a^n = c*ybar^{n-1} + g*a^{n+1} + p*a^{n+2} - J(q^n) (r*a^{n+1}).
 */
int orc_adjoint(int kind, int N, int M, const double *g, const double *p, const double *r,
                const double *b, const double *c, const double *lam, double taup,
                const double *H, const double *kappa, int steps, const double *e,
                const double *traj, const double *ybar,
                double *dq0, double *dqm1, double *dg, double *dp, double *dr, double *db,
                double *dc, double *dtau, double *dkappa, double *dH)
{
    orc_model m = {kind, N, M, g, p, r, b, c, lam, taup, H, kappa};
    double *a1 = xcalloc(N, sizeof(double)), *a2 = xcalloc(N, sizeof(double));
    double *an = xcalloc(N, sizeof(double)), *w = xcalloc(N, sizeof(double));
    double *Jw = xcalloc(N, sizeof(double)), *f = xcalloc(N, sizeof(double));
    double *u = xcalloc((size_t)(M > 0 ? M : 1) * N, sizeof(double));
    double *eta = xcalloc(M > 0 ? M : 1, sizeof(double));
    double *z = xcalloc(N, sizeof(double)), *uk = xcalloc(N, sizeof(double));
    double *zk = xcalloc(N, sizeof(double));
    double sdtau = 0;
    if (dg) memset(dg, 0, N * sizeof(double));
    if (dp) memset(dp, 0, N * sizeof(double));
    if (dr) memset(dr, 0, N * sizeof(double));
    if (db) memset(db, 0, N * sizeof(double));
    if (dc) memset(dc, 0, N * sizeof(double));
    if (dkappa && M > 0) memset(dkappa, 0, M * sizeof(double));
    if (dH && M > 0) memset(dH, 0, (size_t)M * N * N * sizeof(double));
#define Q(n) (traj + (size_t)((n) + 1) * N) /* q^n for n = -1..steps */
    /* a1 holds a^{n+1}, a2 holds a^{n+2}.  q^{steps} only feeds y^{steps-1},
       so a^{steps} = c ybar^{steps-1} and a^{steps+1} = 0. */
    if (steps > 0)
        for (int mu = 0; mu < N; ++mu) a1[mu] = c[mu] * ybar[steps - 1];
    for (int n = steps - 1; n >= 0; --n) {
        /* a^{n+1} is complete in a1: q^{n+1} -> y^n, q^{n+2}, q^{n+3} already folded in.
           Now accumulate parameter gradients of step n (q^{n+1} = g q^n + p q^{n-1} + r F^n). */
        const double *qn = Q(n), *qnm1 = Q(n - 1), *qn1 = Q(n + 1);
        double S = nl_force(&m, qn, f, u, eta);
        for (int mu = 0; mu < N; ++mu) {
            double F = b[mu] * e[n] - f[mu];
            if (dg) dg[mu] += a1[mu] * qn[mu];
            if (dp) dp[mu] += a1[mu] * qnm1[mu];
            if (dr) dr[mu] += a1[mu] * F;
            if (db) db[mu] += a1[mu] * r[mu] * e[n];
            if (dc) dc[mu] += ybar[n] * qn1[mu];
            w[mu] = r[mu] * a1[mu];
        }
        if (kind == ORC_TENSION) {
            double P = 0.0;
            for (int mu = 0; mu < N; ++mu) P += w[mu] * lam[mu] * qn[mu];
            sdtau -= S * P;
        } else {
            for (int k = 0; k < M; ++k) {
                double xi = 0.0;
                for (int s = 0; s < N; ++s) xi += u[(size_t)k * N + s] * w[s];
                if (dkappa) dkappa[k] -= eta[k] * xi;
                if (dH) {
                    /* dL/dH^k_ij (symmetrised) = -kappa_k [xi q_i q_j + eta_k (w_i q_j + w_j q_i)/2] */
                    double *G = dH + (size_t)k * N * N;
                    for (int i = 0; i < N; ++i)
                        for (int j = 0; j < N; ++j)
                            G[(size_t)i * N + j] -= kappa[k] * (xi * qn[i] * qn[j] +
                                0.5 * eta[k] * (w[i] * qn[j] + w[j] * qn[i]));
                }
            }
        }
        /* a^n = c ybar^{n-1} + g a^{n+1} + p a^{n+2} - J(q^n) w   (for n >= 1);
           for n = 0 the same expression without the pickup term is dL/dq^0. */
        jac_vec(&m, qn, w, Jw, uk, eta, zk);
        for (int mu = 0; mu < N; ++mu) {
            double v = g[mu] * a1[mu] + p[mu] * a2[mu] - Jw[mu];
            if (n >= 1) v += c[mu] * ybar[n - 1];
            an[mu] = v;
        }
        if (n == 0) {
            if (dq0) memcpy(dq0, an, N * sizeof(double));
            if (dqm1) for (int mu = 0; mu < N; ++mu) dqm1[mu] = p[mu] * a1[mu];
        }
        double *t = a2; a2 = a1; a1 = an; an = t;
    }
#undef Q
    if (dtau) *dtau = sdtau;
    free(a1); free(a2); free(an); free(w); free(Jw); free(f); free(u); free(eta);
    free(z); free(uk); free(zk);
    return 0;
}

/* Many independent instances (used for CPU timing); one thread per instance
 * when compiled with OpenMP. Arrays are concatenated per instance with the
 * given offsets. */
int orc_forward_batch(int n_inst, const int *kind, const int *N, const int *M,
                      const long *off_mode, const long *off_H, const long *off_M,
                      const double *g, const double *p, const double *r, const double *b,
                      const double *c, const double *lam, const double *taup,
                      const double *H, const double *kappa, int steps, const double *e,
                      const double *q0, const double *qm1, double *y)
{
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int i = 0; i < n_inst; ++i) {
        long o = off_mode[i];
        bad |= orc_forward(kind[i], N[i], M[i], g + o, p + o, r + o, b + o, c + o, lam + o,
                           taup[i], H + off_H[i], kappa + off_M[i], steps,
                           e + (size_t)i * steps, q0 + o, qm1 + o, y + (size_t)i * steps,
                           NULL, NULL, NULL);
    }
    return bad;
}

/* fnl(q) alone (Eq. 8 or Eq. 9), for the brute-force tests. f: [N]. */
int orc_force(int kind, int N, int M, const double *lam, double taup, const double *H,
              const double *kappa, const double *q, double *f)
{
    orc_model m = {kind, N, M, NULL, NULL, NULL, NULL, NULL, lam, taup, H, kappa};
    double *u = xcalloc((size_t)(M > 0 ? M : 1) * N, sizeof(double));
    double *eta = xcalloc(M > 0 ? M : 1, sizeof(double));
    nl_force(&m, q, f, u, eta);
    free(u); free(eta);
    return 0;
}
