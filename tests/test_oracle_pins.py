"""Pins of the FP64 oracle against facts fixed outside the oracle itself:
closed forms, library routines for special cases, brute-force quadrature,
invariants, published tabulated values and finite differences."""
import math
import os

import numpy as np
import pytest
import scipy.integrate
import scipy.signal

import oracle
from oracle import coupling_oracle as CO
from oracle import physics_oracle as PO
from paper_2505_05940_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([float(t) for t in line.split()])
    return np.array(rows)


def _tiny(kind, n_phi, n_psi=0, seed=0, steps=200, coupling=True, fs=44100.0, **override):
    wl = W.tiny_random(seed, kind, n_phi, n_psi, steps=steps, fs=fs)
    inst = wl.instances[0]
    for k, v in override.items():
        setattr(inst, k, v)
    cp = CO.oracle_coupling if (kind == "plate" and coupling) else None
    return PO.build_instance(inst, wl.fs, wl.steps, coupling=cp), wl


# ---------------------------------------------------------------- coefficients

def test_sv_coefficients_closed_form():
    """Eq. 21-23 simplify to r = T^2/(1+gT), g = (2 - w^2 T^2)/(1+gT),
    p = -(1 - gT)/(1 + gT); with gamma = 0 they are 2 - w^2 T^2, -1, T^2."""
    rng = np.random.default_rng(1)
    T = 1.0 / 44100.0
    w2 = rng.uniform(1.0, (1.9 / T) ** 2, 100)
    gm = rng.uniform(0.0, 1e4, 100)
    g, p, r = PO.sv_coefficients(w2, gm, T)
    den = 1.0 + gm * T
    np.testing.assert_allclose(r, T ** 2 / den, rtol=1e-14)
    np.testing.assert_allclose(g, (2.0 - w2 * T ** 2) / den, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(p, -(1.0 - gm * T) / den, rtol=1e-13)
    g0, p0, r0 = PO.sv_coefficients(w2, 0.0 * gm, T)
    np.testing.assert_allclose(g0, 2.0 - w2 * T ** 2, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(p0, -1.0, rtol=0, atol=1e-15)
    np.testing.assert_allclose(r0, T ** 2, rtol=1e-15)


def test_stiff_string_dispersion_golden():
    """omega^2 of Eq. 13 with lambda of Eq. 2 reproduces the textbook stiff
    string frequencies."""
    wl = W.string_40()
    oi = PO.build_instance(wl.instances[0], wl.fs, wl.steps)
    gold = _read_golden("string40_frequencies.txt")
    f = np.sqrt(oi.omega2) / (2.0 * math.pi)
    for mu, fref in gold:
        assert abs(f[int(mu) - 1] - fref) < 1e-4 * 1.0001, (mu, f[int(mu) - 1], fref)
    assert oi.N == 40


def test_rect_mode_ordering_bruteforce():
    """First N rectangle modes are the N smallest lambda over a large (m, n)
    grid, ties broken by (m, n)."""
    inst = W.plate_100x30().instances[0]
    labels, lam = PO.rect_modes(inst, 100)
    Lx, Ly = PO.rect_sides(inst)
    allm = [((m * math.pi / Lx) ** 2 + (k * math.pi / Ly) ** 2, m, k)
            for m in range(1, 60) for k in range(1, 60)]
    allm.sort()
    assert [tuple(x) for x in labels] == [(m, k) for _, m, k in allm[:100]]
    assert np.all(np.diff(lam) >= 0)


def test_stability_truncation_rule():
    wl = W.batched_ragged(seed=0, n_inst=512, steps=10)
    T = 1.0 / wl.fs
    dropped = 0
    for inst in wl.instances:
        oi = PO.build_instance(inst, wl.fs, wl.steps, coupling=None)
        assert np.all(np.sqrt(oi.omega2) * T < PO.SV_OMEGA_T_MAX)
        if oi.N < inst.n_phi:
            dropped += 1
            # the first dropped mode really is beyond the bound
            labels, lam = (PO.rect_modes(inst, oi.N + 1))
            w2 = PO.omega2_of(lam[-1], inst.D, inst.T0, inst.rho_lin)
            assert math.sqrt(w2) * T >= PO.SV_OMEGA_T_MAX
    assert dropped > 0


def test_pluck_projection_closed_form():
    """<w0, Phi_mu> for the raised-cosine pluck equals
    sqrt(2/L) A sin(k x0) sin(k W/2) a^2 / (k (a^2 - k^2)), k = mu pi / L, a = 2 pi / W."""
    inst = W.string_40().instances[0]
    labels, _ = PO.string_modes(inst, 40)
    q0 = PO.pluck_projection(inst, labels)
    L, A = inst.length, inst.pluck_amp
    x0, Wd = inst.pluck_x0 * L, inst.pluck_width * L
    k = labels[:, 0] * math.pi / L
    a = 2.0 * math.pi / Wd
    sing = np.isclose(k, a)
    ks = np.where(sing, 1.0, k)
    ref = math.sqrt(2.0 / L) * A * np.sin(k * x0) * np.sin(k * Wd / 2) * a ** 2 / (ks * (a ** 2 - ks ** 2))
    # removable singularity at k = a: the bracket 1/k + k/(a^2 - k^2) times sin(kW/2) tends to W/4
    ref = np.where(sing, math.sqrt(2.0 / L) * A * np.sin(k * x0) * Wd / 4.0, ref)
    assert sing.sum() == 1
    np.testing.assert_allclose(q0, ref, rtol=1e-10, atol=1e-16)


# ---------------------------------------------------------------- linear scheme

def _linear(kind="string", n=5, gamma0=True):
    oi, wl = _tiny(kind, n, 0, seed=3, steps=4000)
    oi.taup = 0.0
    if gamma0:
        oi.gamma = 0.0 * oi.gamma
        oi.g, oi.p, oi.r = PO.sv_coefficients(oi.omega2, oi.gamma, 1.0 / wl.fs)
    return oi, wl


def test_linear_free_response_closed_form():
    """With fnl = 0 and e = 0 each mode obeys q^{n+1} = g q^n + p q^{n-1}:
    q^n = A z+^n + B z-^n with z^2 - g z - p = 0 (damped, complex roots)."""
    oi, wl = _linear("string", 6, gamma0=False)
    steps = 3000
    out = oracle.forward(oi, steps=steps, want_traj=True)
    n = np.arange(-1, steps + 1)
    for mu in range(oi.N):
        zp, zm = np.roots([1.0, -oi.g[mu], -oi.p[mu]])
        # fit A, B from q^{-1}, q^0
        Mx = np.array([[zp ** -1, zm ** -1], [1.0, 1.0]])
        AB = np.linalg.solve(Mx, np.array([oi.qm1[mu], oi.q0[mu]], dtype=complex))
        ref = (AB[0] * zp ** n + AB[1] * zm ** n).real
        np.testing.assert_allclose(out["traj"][:, mu], ref, rtol=0,
                                   atol=1e-11 * np.abs(ref).max())


def test_linear_undamped_exact_dispersion():
    """gamma = 0: the free response is exactly cos(theta n) (times amplitude)
    with cos(theta) = 1 - omega^2 T^2 / 2, the Stormer-Verlet dispersion; the
    continuous solution cos(omega t) is missed only by the phase n(theta - omega T)."""
    oi, wl = _linear("string", 4, gamma0=True)
    T = 1.0 / wl.fs
    oi.qm1 = oi.q0.copy()
    steps = 2000
    out = oracle.forward(oi, steps=steps, want_traj=True)
    n = np.arange(-1, steps + 1)
    for mu in range(oi.N):
        th = math.acos(1.0 - oi.omega2[mu] * T * T / 2.0)
        # q^{-1} = q^0 starts at the midpoint of a symmetric oscillation: q^n = Q cos(theta (n + 1/2))
        Q = oi.q0[mu] / math.cos(th / 2.0)
        ref = Q * np.cos(th * (n + 0.5))
        # FP64 rounding of g shifts theta by ~1e-16 / sin(theta); over 2000 steps
        # that is a phase (hence amplitude-relative) error below 1e-10
        np.testing.assert_allclose(out["traj"][:, mu], ref, rtol=0, atol=1e-10 * abs(Q))
        # distance to the continuous oscillator is the dispersion phase error
        w = math.sqrt(oi.omega2[mu])
        cont = Q * np.cos(w * T * (n + 0.5))
        err = np.abs(out["traj"][:, mu] - cont).max() / abs(Q)
        bound = abs(th - w * T) * (steps + 1) + 1e-12
        assert err <= bound * 1.01


def test_linear_forced_matches_lfilter():
    """fnl = 0: the forced response of each mode is the IIR filter
    r b / (1 - g z^-1 - p z^-2) applied to e (scipy.signal.lfilter)."""
    oi, wl = _tiny("plate", 7, 0, seed=5, steps=600, coupling=False)
    out = oracle.forward(oi, want_traj=True)
    for mu in range(oi.N):
        x = scipy.signal.lfilter([oi.r[mu] * oi.b[mu]], [1.0, -oi.g[mu], -oi.p[mu]], oi.e)
        # x[n] is q^{n+1}
        np.testing.assert_allclose(out["traj"][2:, mu], x, rtol=0, atol=1e-12 * np.abs(x).max())
    y_ref = out["traj"][2:] @ oi.c
    np.testing.assert_allclose(out["y"], y_ref, rtol=1e-13, atol=1e-20)


def test_linear_energy_exact():
    """Undamped, unforced linear scheme conserves
    E = 1/2 |(q^{n+1}-q^n)/T|^2 + 1/2 sum omega^2 q^{n+1} q^n exactly."""
    oi, wl = _linear("string", 8, gamma0=True)
    T = 1.0 / wl.fs
    tr = oracle.forward(oi, steps=3000, want_traj=True)["traj"]
    E = 0.5 * (((tr[1:] - tr[:-1]) / T) ** 2).sum(1) + 0.5 * (oi.omega2 * tr[1:] * tr[:-1]).sum(1)
    assert np.abs(E - E[0]).max() <= 1e-11 * abs(E[0])


# ---------------------------------------------------------------- nonlinear forces

def test_string_tension_force_bruteforce():
    """Eq. 8 (unit-norm modes) equals tau' * int(w_x^2) * <-w_xx, Phi_mu> by
    quadrature of the physical displacement w(x) = sum q Phi(x)."""
    oi, _ = _tiny("string", 9, seed=7)
    rng = np.random.default_rng(2)
    q = rng.normal(size=oi.N) * 1e-4
    L = oi.src.length
    xg, wg = np.polynomial.legendre.leggauss(200)
    x = (xg + 1) * L / 2
    wq = wg * L / 2
    mu = oi.labels[:, 0]
    k = mu * math.pi / L
    phi = math.sqrt(2 / L) * np.sin(np.outer(x, k))
    dphi = math.sqrt(2 / L) * np.cos(np.outer(x, k)) * k
    w_x = dphi @ q
    w_xx = -(phi * k ** 2) @ q
    S = np.sum(wq * w_x ** 2)
    f_ref = oi.taup * S * (phi.T @ (wq * (-w_xx)))
    np.testing.assert_allclose(oracle.force(oi, q), f_ref, rtol=1e-11, atol=1e-14 * np.abs(f_ref).max())


def test_membrane_tension_force_bruteforce():
    """Berger membrane: sum lambda q^2 = int |grad w|^2 over the rectangle."""
    oi, _ = _tiny("membrane", 7, seed=8)
    rng = np.random.default_rng(3)
    q = rng.normal(size=oi.N) * 1e-4
    Lx, Ly = PO.rect_sides(oi.src)
    xg, wg = np.polynomial.legendre.leggauss(80)
    x = (xg + 1) * Lx / 2
    y = (xg + 1) * Ly / 2
    X, Y = np.meshgrid(x, y, indexing="ij")
    Wt = np.outer(wg, wg) * Lx * Ly / 4
    A = 2 / math.sqrt(Lx * Ly)
    gx = np.zeros_like(X)
    gy = np.zeros_like(X)
    for (m, n), qq in zip(oi.labels, q):
        a, b = m * math.pi / Lx, n * math.pi / Ly
        gx += qq * A * a * np.cos(a * X) * np.sin(b * Y)
        gy += qq * A * b * np.sin(a * X) * np.cos(b * Y)
    S_ref = np.sum(Wt * (gx ** 2 + gy ** 2))
    f = oracle.force(oi, q)
    f_ref = oi.taup * oi.lam * q * S_ref
    np.testing.assert_allclose(f, f_ref, rtol=1e-11)


def _plate_bruteforce_force(oi, q, n_quad=72):
    """fnl through the PDE operators: Airy stress from Delta Delta phi = -(Eh/2) L(w,w)
    projected on the Airy modes, then -int Phi_s L(w, phi) dS / (rho h)."""
    inst = oi.src
    Lx, Ly = PO.rect_sides(inst)
    zeta4, psi_eval = CO.airy_modes(Lx, Ly, oi.M, n_basis=CO.default_basis(oi.M),
                                    n_quad=max(64, CO.default_basis(oi.M) + 8))
    xg, wg = np.polynomial.legendre.leggauss(n_quad)
    x = (xg + 1) * Lx / 2
    y = (xg + 1) * Ly / 2
    X, Y = np.meshgrid(x, y, indexing="ij")
    X, Y = X.reshape(-1), Y.reshape(-1)
    Wt = (np.outer(wg, wg) * Lx * Ly / 4).reshape(-1)
    A = 2 / math.sqrt(Lx * Ly)
    w = np.zeros_like(X)
    wxx = np.zeros_like(X)
    wyy = np.zeros_like(X)
    wxy = np.zeros_like(X)
    Phi = []
    for (m, n), qq in zip(oi.labels, q):
        a, b = m * math.pi / Lx, n * math.pi / Ly
        s = A * np.sin(a * X) * np.sin(b * Y)
        Phi.append(s)
        w += qq * s
        wxx += -qq * a * a * s
        wyy += -qq * b * b * s
        wxy += qq * A * a * b * np.cos(a * X) * np.cos(b * Y)
    Lww = wxx * wyy + wyy * wxx - 2 * wxy * wxy
    Psi, Pxx, Pyy, Pxy = psi_eval(X, Y)
    chi = Psi.T @ (Wt * Lww)
    h = inst.thickness
    phik = -(inst.E * h / 2.0) * chi / zeta4
    fxx, fyy, fxy = Pxx @ phik, Pyy @ phik, Pxy @ phik
    Lwf = wxx * fyy + wyy * fxx - 2 * wxy * fxy
    f = np.array([-(np.sum(Wt * s * Lwf)) / inst.rho_lin for s in Phi])
    return f


@pytest.mark.parametrize("seed", [0, 1])
def test_plate_force_bruteforce(seed):
    """Eq. 9 with C^s_pn = H^n_ps equals the force obtained directly from the
    von Karman operators (Eq. 5-7) on a tiny mode set."""
    oi, _ = _tiny("plate", 6, 4, seed=seed)
    rng = np.random.default_rng(10 + seed)
    q = rng.normal(size=oi.N) * 1e-5
    f = oracle.force(oi, q)
    f_ref = _plate_bruteforce_force(oi, q)
    np.testing.assert_allclose(f, f_ref, rtol=1e-8, atol=1e-10 * np.abs(f_ref).max())


def test_plate_force_sign_invariance():
    """The sign of each Airy mode is arbitrary: flipping H^k leaves fnl unchanged."""
    oi, _ = _tiny("plate", 10, 5, seed=4)
    q = np.random.default_rng(5).normal(size=oi.N) * 1e-5
    f0 = oracle.force(oi, q)
    oi.H = oi.H.copy()
    oi.H[[1, 3]] *= -1.0
    np.testing.assert_allclose(oracle.force(oi, q), f0, rtol=1e-14, atol=0)


# ---------------------------------------------------------------- coupling tensors

def test_airy_modes_leissa_clamped_square():
    gold = _read_golden("clamped_square_plate.txt")[:, 0]
    z4, _ = CO.airy_modes(1.0, 1.0, len(gold), n_basis=20)
    np.testing.assert_allclose(np.sqrt(z4), gold, rtol=1e-3)


def test_H_symmetry_and_C_identity():
    """H^k_ij = H^k_ji (symmetry of L, Eq. 7) and H^k_ij = C^j_ik
    (simply supported identity, Sec. 4.3.3) with C from its own quadrature (Eq. 11)."""
    oi, _ = _tiny("plate", 12, 6, seed=2)
    H = oi.H
    assert np.abs(H - H.transpose(0, 2, 1)).max() <= 1e-13 * np.abs(H).max()
    C = CO.coupling_C(oi.src, oi.labels, oi.M)           # C[s][i][j]
    # H^k_ij = C^j_ik  ->  H[k, i, j] == C[j, i, k]
    np.testing.assert_allclose(H, C.transpose(2, 1, 0), rtol=0, atol=1e-9 * np.abs(H).max())


def test_H_quadrature_and_ritz_converged():
    oi, _ = _tiny("plate", 20, 6, seed=6)
    nb = CO.default_basis(6)
    nq = CO.default_quadrature(oi.labels, nb)
    H1, z1 = CO.coupling_H(oi.src, oi.labels, 6, n_basis=nb, n_quad=nq)
    H2, z2 = CO.coupling_H(oi.src, oi.labels, 6, n_basis=nb, n_quad=nq + 24)
    assert np.abs(H1 - H2).max() <= 1e-11 * np.abs(H1).max()
    H3, z3 = CO.coupling_H(oi.src, oi.labels, 6, n_basis=nb + 6, n_quad=nq + 6)
    np.testing.assert_allclose(z3, z1, rtol=1e-7)   # Ritz error well below FP32 rounding
    assert np.abs(np.abs(H3) - np.abs(H1)).max() <= 1e-6 * np.abs(H1).max()


# ---------------------------------------------------------------- nonlinear scheme

def _energy(oi, tr, T):
    q1, q0 = tr[1:], tr[:-1]
    kin = 0.5 * (((q1 - q0) / T) ** 2).sum(1)
    pot = 0.5 * (oi.omega2 * q1 * q0).sum(1)
    if oi.kind == "plate":
        V = lambda q: 0.25 * np.sum(oi.kappa * np.einsum("kij,ni,nj->nk", oi.H, q, q) ** 2, 1)
    else:
        V = lambda q: 0.25 * oi.taup * ((q ** 2) @ oi.lam) ** 2
    return kin + pot + 0.5 * (V(q1) + V(q0))


def test_nonlinear_string_energy_bounded():
    """Lossless, unforced Kirchhoff-Carrier string: the discrete energy shows
    no secular drift (Stormer-Verlet is symplectic); its bounded oscillation
    is small."""
    wl = W.string_40()
    inst = wl.instances[0]
    inst.sigma0 = inst.sigma1 = 0.0
    oi = PO.build_instance(inst, wl.fs, wl.steps)
    T = 1.0 / wl.fs
    tr = oracle.forward(oi, steps=48000, want_traj=True)["traj"]
    E = _energy(oi, tr, T)[1:]       # E[0] straddles the start q^{-1} = q^0
    V = 0.25 * oi.taup * ((tr ** 2) @ oi.lam) ** 2
    assert V.max() > 0.02 * E[0]      # the nonlinearity is active (about 5 % of the energy)
    # bounded oscillation (a fraction of the nonlinear energy share) ...
    assert np.ptp(E) <= 1e-2 * E[0]
    # ... and no secular drift over 48 000 steps
    head, tail = E[:4800].mean(), E[-4800:].mean()
    assert abs(tail - head) <= 2e-5 * E[0]


def test_nonlinear_plate_energy_bounded():
    """Lossless von Karman plate after the strike: bounded energy, no drift."""
    inst = W.plate_100x30().instances[0]
    inst.n_phi, inst.n_psi = 30, 10
    inst.sigma0 = inst.sigma1 = 0.0
    inst.F0 = 400.0                      # strongly nonlinear
    oi = PO.build_instance(inst, 44100.0, 20000, coupling=CO.oracle_coupling)
    T = 1.0 / 44100.0
    tr = oracle.forward(oi, steps=20000, want_traj=True)["traj"]
    E = _energy(oi, tr, T)[100:]          # after the 1 ms pulse (45 samples)
    V = 0.25 * np.sum(oi.kappa * np.einsum("kij,ni,nj->nk", oi.H, tr[100:], tr[100:]) ** 2, 1)
    assert V.max() > 1e-2 * E[0]          # the nonlinearity is active
    # bounded: the band over the second half is no wider than over the first half
    half = len(E) // 2
    assert np.ptp(E) <= 1e-3 * E[0]
    assert np.abs(E[half:] - E[0]).max() <= 1.5 * np.abs(E[:half] - E[0]).max() + 1e-6 * E[0]


def test_nonlinear_reduces_to_linear():
    """tau' = 0 (string) or kappa = 0 (plate) gives the linear lfilter response."""
    oi, _ = _tiny("plate", 8, 3, seed=9, steps=400)
    oi.kappa = 0.0 * oi.kappa
    out = oracle.forward(oi, want_traj=True)
    for mu in range(oi.N):
        x = scipy.signal.lfilter([oi.r[mu] * oi.b[mu]], [1.0, -oi.g[mu], -oi.p[mu]], oi.e)
        np.testing.assert_allclose(out["traj"][2:, mu], x, rtol=0, atol=1e-12 * np.abs(x).max())


@pytest.mark.parametrize("scheme", ["sv", "tf"])
def test_scheme_second_order_vs_dop853(scheme):
    """Fig. 1's claim: the Stormer-Verlet and the impulse-invariant solutions
    of the tension-modulated string converge to the DOP853 solution of Eq. 12
    at second order in T."""
    base = W.string_40().instances[0]
    base.n_phi = 12
    dur = 0.004
    errs = []
    for fs in (96000.0, 192000.0):
        oi = PO.build_instance(base, fs, int(dur * fs), scheme=scheme)
        # ODE: qdd + 2 gamma qd + w2 q = -fnl(q), q(0) = q0, qd(0) = 0
        def rhs(t, z):
            q, v = z[:oi.N], z[oi.N:]
            return np.concatenate([v, -2 * oi.gamma * v - oi.omega2 * q - oracle.force(oi, q)])
        steps = int(dur * fs)
        tt = np.arange(1, steps + 1) / fs
        sol = scipy.integrate.solve_ivp(rhs, (0, tt[-1]), np.concatenate([oi.q0, 0 * oi.q0]),
                                        method="DOP853", t_eval=tt, rtol=1e-12, atol=1e-16)
        y_ref = oi.c @ sol.y[:oi.N]
        # second-order start: q^{-1} = q(-T) = q0 + T^2/2 qdd(0) for zero initial velocity
        # (the plain start q^{-1} = q^0 is only first order in the velocity)
        T = 1.0 / fs
        qm1 = oi.q0 + 0.5 * T * T * (-oi.omega2 * oi.q0 - oracle.force(oi, oi.q0))
        y = oracle.forward(oi, steps=steps, qm1=qm1)["y"]
        errs.append(np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref))
    ratio = errs[0] / errs[1]
    assert 3.0 < ratio < 5.0, (errs, ratio)


# ---------------------------------------------------------------- adjoint

def _loss(oi, ybar, **kw):
    return float(ybar @ oracle.forward(oi, **kw)["y"])


def _fd(oi, ybar, setter, h):
    a = setter(oi, +h)
    lp = _loss(a, ybar)
    a = setter(oi, -h)
    lm = _loss(a, ybar)
    return (lp - lm) / (2 * h)


def _clone(oi):
    import copy
    return copy.deepcopy(oi)


def _coef_setter(idx, which, T):
    def s(oi, h):
        o = _clone(oi)
        w2, gm = o.omega2.copy(), o.gamma.copy()
        if which == "omega2":
            w2[idx] += h
        else:
            gm[idx] += h
        o.omega2, o.gamma = w2, gm
        o.g, o.p, o.r = PO.sv_coefficients(w2, gm, T)
        return o
    return s


@pytest.mark.parametrize("kind", ["string", "plate"])
def test_adjoint_matches_central_fd(kind):
    # relative FD steps ~1e-4: truncation O(h^2) ~ 1e-8, while the summed loss
    # still resolves the difference well above FP64 cancellation
    n_psi = 3 if kind == "plate" else 0
    oi, wl = _tiny(kind, 6, n_psi, seed=11, steps=300)
    if kind == "plate":
        oi.kappa = oi.kappa * 50.0         # make the nonlinearity matter over 300 steps
        oi.e = oi.e * 5.0
    T = 1.0 / wl.fs
    rng = np.random.default_rng(0)
    ybar = rng.normal(size=300)
    adj = oracle.adjoint(oi, ybar, want_dH=True)
    d_w2, d_gm = oracle.coefficient_grads(oi, adj, T)
    checks = []
    for mu in (0, 3, 5):
        checks.append((d_w2[mu], _fd(oi, ybar, _coef_setter(mu, "omega2", T), 1e-4 * oi.omega2[mu])))
        checks.append((d_gm[mu], _fd(oi, ybar, _coef_setter(mu, "gamma", T), 1e-3 * (oi.gamma[mu] + 1))))

        def sb(o, h, mu=mu):
            o = _clone(o); o.b = o.b.copy(); o.b[mu] += h; return o
        checks.append((adj["db"][mu], _fd(oi, ybar, sb, 1e-4 * abs(oi.b[mu]))))

        def sc(o, h, mu=mu):
            o = _clone(o); o.c = o.c.copy(); o.c[mu] += h; return o
        checks.append((adj["dc"][mu], _fd(oi, ybar, sc, 1e-4 * abs(oi.c[mu]))))

        def sq(o, h, mu=mu):
            o = _clone(o); o.q0 = o.q0.copy(); o.q0[mu] += h; return o
        checks.append((adj["dq0"][mu], _fd(oi, ybar, sq, 1e-10)))

        def sqm(o, h, mu=mu):
            o = _clone(o); o.qm1 = o.qm1.copy(); o.qm1[mu] += h; return o
        checks.append((adj["dqm1"][mu], _fd(oi, ybar, sqm, 1e-10)))
    if kind == "string":
        def st(o, h):
            o = _clone(o); o.taup = o.taup + h; return o
        checks.append((adj["dtau"], _fd(oi, ybar, st, 1e-4 * oi.taup)))
    else:
        for k in range(oi.M):
            def sk(o, h, k=k):
                o = _clone(o); o.kappa = o.kappa.copy(); o.kappa[k] += h; return o
            checks.append((adj["dkappa"][k], _fd(oi, ybar, sk, 1e-4 * oi.kappa[k])))
        for (k, i, j) in ((0, 1, 2), (2, 0, 0), (1, 5, 3)):
            def sh(o, h, k=k, i=i, j=j):
                o = _clone(o); o.H = o.H.copy()
                o.H[k, i, j] += h
                if i != j:
                    o.H[k, j, i] += h
                return o
            g = adj["dH"][k, i, j] * (2.0 if i != j else 1.0)
            checks.append((g, _fd(oi, ybar, sh, 1e-4 * np.abs(oi.H[k]).max())))
    for got, ref in checks:
        assert abs(got - ref) <= 1e-6 * abs(ref) + 1e-9 * max(abs(c[1]) for c in checks), (got, ref)


# ---------------------------------------------------------------- proposal MLP oracle

def _mlp(rng, dims):
    Ws = [rng.normal(size=(dims[l + 1], dims[l])) / np.sqrt(dims[l]) for l in range(len(dims) - 1)]
    bs = [rng.normal(size=dims[l + 1]) * 0.1 for l in range(len(dims) - 1)]
    return Ws, bs


def test_mlp_oracle_backward_matches_fd():
    from oracle import mlp_oracle as MO
    rng = np.random.default_rng(3)
    dims = [12, 9, 7, 5]
    Ws, bs = _mlp(rng, dims)
    x = rng.normal(size=(6, 12))
    dy = rng.normal(size=(6, 5))
    y, hs = MO.forward(Ws, bs, x, bf16=False)
    dWs, dbs = MO.backward(Ws, bs, hs, dy, bf16=False)
    L = lambda W2, b2: float(np.sum(dy * MO.forward(W2, b2, x, bf16=False)[0]))
    h = 1e-6
    for l in range(3):
        for (i, j) in ((0, 0), (2, 3), (4, 1)):
            if i >= dims[l + 1] or j >= dims[l]:
                continue
            Wp = [w.copy() for w in Ws]; Wp[l][i, j] += h
            Wm = [w.copy() for w in Ws]; Wm[l][i, j] -= h
            fd = (L(Wp, bs) - L(Wm, bs)) / (2 * h)
            assert abs(dWs[l][i, j] - fd) <= 1e-6 * max(1.0, abs(fd))
        bp = [b.copy() for b in bs]; bp[l][1] += h
        bm = [b.copy() for b in bs]; bm[l][1] -= h
        fd = (L(Ws, bp) - L(Ws, bm)) / (2 * h)
        assert abs(dbs[l][1] - fd) <= 1e-6 * max(1.0, abs(fd))


def test_bf16_rounding_is_round_to_nearest_even():
    from oracle import mlp_oracle as MO
    # 1 + 2^-8 is exactly halfway between 1 and 1 + 2^-7 in BF16: ties to even -> 1
    assert MO.bf16_round(1.0 + 2.0 ** -8) == 1.0
    assert MO.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert MO.bf16_round(-3.0) == -3.0
    v = np.array([0.1, 1 / 3, 1e-3, 123.456])
    r = MO.bf16_round(v)
    assert np.all(np.abs(r - v) <= np.abs(v) * 2.0 ** -8)


def test_mlp_oracle_exact_on_small_integers():
    """With small integer weights and inputs every BF16 rounding is exact, so
    the BF16-emulating oracle equals plain integer arithmetic."""
    from oracle import mlp_oracle as MO
    rng = np.random.default_rng(5)
    dims = [8, 6, 4]
    Ws = [rng.integers(-3, 4, size=(dims[l + 1], dims[l])).astype(float) for l in range(2)]
    bs = [rng.integers(-2, 3, size=dims[l + 1]).astype(float) for l in range(2)]
    x = rng.integers(-2, 3, size=(5, 8)).astype(float)
    y, _ = MO.forward(Ws, bs, x, bf16=True)
    h = np.maximum(x @ Ws[0].T + bs[0], 0)
    np.testing.assert_array_equal(y, h @ Ws[1].T + bs[1])


@pytest.mark.parametrize("n,m,f0", [(48, 12, 200.0), (100, 30, 50.0)])
def test_parity_cases_are_well_conditioned(n, m, f0):
    """A 1e-12 relative change of the excitation moves the FP64 output by far
    less than the 1e-5 parity tolerance, so agreement to 1e-5 measures the
    arithmetic and not the sensitivity of the system."""
    from paper_2505_05940_gb300 import workloads as W
    steps = 4410
    wl = W.plate_100x30() if n == 100 else W.tiny_random(n + 3, "plate", n, m, steps=steps)
    inst = wl.instances[0]
    inst.F0 = f0
    oi = PO.build_instance(inst, wl.fs, steps, coupling=CO.oracle_coupling)
    a = oracle.forward(oi, steps=steps)["y"]
    b = oracle.forward(oi, steps=steps, e=oi.e[:steps] * (1.0 + 1e-12))["y"]
    d = np.linalg.norm(a - b) / np.linalg.norm(a)
    assert d < 1e-9, d


# ----------------------------------------------------------------- spectral losses

def test_stft_oracle_tone_at_bin_centre():
    """A unit cosine at an exact bin frequency gives |STFT| = n_fft / 4 at that
    bin for every interior frame (sum of the periodic Hann window / 2)."""
    from oracle import stft_oracle as SO
    n_fft, k = 256, 17
    t = np.arange(4096)
    x = np.cos(2 * np.pi * k * t / n_fft + 0.3)
    Y = SO.stft_mag(x, n_fft)
    interior = Y[:, 4:-4]
    np.testing.assert_allclose(interior[k], n_fft / 4, rtol=1e-12)
    assert np.all(interior[k + 2:] < 1e-9 * n_fft)


def test_spectral_losses_closed_forms():
    from oracle import stft_oracle as SO
    rng = np.random.default_rng(3)
    x = rng.standard_normal(3000)
    # spectral convergence of a scaled copy is |a - 1|
    assert SO.spectral_convergence(0.7 * x, x) == pytest.approx(0.3, rel=1e-12)
    # log-STFT distance of a scaled copy is |log a| where eps is negligible
    big = 1e6 * x
    assert SO.log_stft_l1(2.0 * big, big, 256) == pytest.approx(math.log(2.0), rel=1e-6)
    # optimal transport between two pure tones: spectra concentrate on their
    # bins, W1 approaches the bin distance
    t = np.arange(8192)
    a = np.cos(2 * np.pi * 40 * t / 1024)
    b = np.cos(2 * np.pi * 52 * t / 1024)
    assert SO.spectral_ot(a, b, 1024) == pytest.approx(12.0, rel=0.02)


def test_library_losses_match_oracle():
    """losses.py (torch, CPU, FP64) equals the numpy oracle."""
    torch = pytest.importorskip("torch")
    from oracle import stft_oracle as SO
    from paper_2505_05940_gb300 import losses
    rng = np.random.default_rng(9)
    y = rng.standard_normal((2, 5000)) * 1e-3
    t = rng.standard_normal((2, 5000)) * 1e-3
    Y, T = torch.tensor(y), torch.tensor(t)
    got = losses.multires_log_stft(Y, T).numpy()
    ref = [SO.multires_log_stft(y[i], t[i]) for i in range(2)]
    np.testing.assert_allclose(got, ref, rtol=1e-10)
    np.testing.assert_allclose(losses.spectral_convergence(Y, T).numpy(),
                               [SO.spectral_convergence(y[i], t[i]) for i in range(2)], rtol=1e-10)
    np.testing.assert_allclose(losses.spectral_ot(Y, T).numpy(),
                               [SO.spectral_ot(y[i], t[i]) for i in range(2)], rtol=1e-9)


# ----------------------------------------------------------------- impulse-invariant scheme

def _single_modes(omega2, gamma, T, steps, q0, qm1, e=None):
    n = len(omega2)
    g, p, r = PO.tf_coefficients(omega2, gamma, T)
    return PO.OracleInstance(kind="string", N=n, M=0, labels=np.arange(1, n + 1).reshape(-1, 1),
                             lam=np.ones(n), omega2=np.asarray(omega2, float),
                             gamma=np.asarray(gamma, float), g=g, p=p, r=r, b=np.ones(n),
                             c=np.ones(n), taup=0.0,
                             e=np.zeros(steps) if e is None else e,
                             q0=np.asarray(q0, float), qm1=np.asarray(qm1, float))


def _free_continuous(w2, gm, t):
    """q(t) with q(0) = 1, q'(0) = 0 for q'' + 2 gm q' + w2 q = 0."""
    d = w2 - gm ** 2
    if d > 0:
        w = math.sqrt(d)
        return np.exp(-gm * t) * (np.cos(w * t) + gm / w * np.sin(w * t))
    if d < 0:
        k = math.sqrt(-d)
        return np.exp(-gm * t) * (np.cosh(k * t) + gm / k * np.sinh(k * t))
    return np.exp(-gm * t) * (1.0 + gm * t)


def test_tf_free_response_is_exact_at_the_samples():
    """Impulse invariance puts the discrete poles at exp(s T): the free
    response equals the continuous solution at every sample, for any omega T
    (including omega T > 2, where Stormer-Verlet is unstable), and for
    under-, critically and over-damped modes."""
    T = 1.0 / 44100.0
    w2 = np.array([(0.3 / T) ** 2, (1.7 / T) ** 2, (2.9 / T) ** 2, 400.0 ** 2, 900.0 ** 2, 300.0 ** 2])
    gm = np.array([5.0, 40.0, 1e3, 400.0, 1.2e3, 100.0])
    gm[3] = math.sqrt(w2[3])                     # critically damped
    steps = 4000
    q0 = np.ones(len(w2))
    qm1 = np.array([_free_continuous(w2[i], gm[i], -T) for i in range(len(w2))])
    oi = _single_modes(w2, gm, T, steps, q0, qm1)
    traj = oracle.forward(oi, steps=steps, want_traj=True)["traj"]
    t = np.arange(-1, steps + 1) * T
    for i in range(len(w2)):
        ref = _free_continuous(w2[i], gm[i], t)
        np.testing.assert_allclose(traj[:, i], ref, rtol=0, atol=1e-11 * np.abs(ref).max())


def test_tf_impulse_response_is_the_sampled_continuous_one():
    """A unit force sample at n = 0 from rest gives q^n = T h(nT), with
    h(t) = exp(-gamma t) sin(w~ t) / w~ the continuous impulse response."""
    T = 1.0 / 48000.0
    w2 = np.array([(2 * math.pi * 440.0) ** 2, (2 * math.pi * 9000.0) ** 2])
    gm = np.array([3.0, 250.0])
    steps = 3000
    e = np.zeros(steps)
    e[0] = 1.0
    oi = _single_modes(w2, gm, T, steps, np.zeros(2), np.zeros(2), e=e)
    traj = oracle.forward(oi, steps=steps, want_traj=True)["traj"]
    n = np.arange(-1, steps + 1)
    for i in range(2):
        wt = math.sqrt(w2[i] - gm[i] ** 2)
        h = np.where(n > 0, np.exp(-gm[i] * n * T) * np.sin(wt * n * T) / wt, 0.0)
        # FP64 rounding of the recursion stays below 1e-9 of the peak T / w~
        np.testing.assert_allclose(traj[:, i], T * h, rtol=0, atol=1e-9 * T / wt)


def test_tf_coefficient_grads_match_central_fd():
    """d L / d omega^2 and d L / d gamma through the impulse-invariant
    coefficients (oracle adjoint + chain rule) against central differences
    of the FP64 forward, on a nonlinear string."""
    wl = W.tiny_random(5, "string", 8, steps=600, fs=48000.0)
    T = 1.0 / wl.fs
    oi = PO.build_instance(wl.instances[0], wl.fs, wl.steps, scheme="tf")
    rng = np.random.default_rng(2)
    ybar = rng.standard_normal(wl.steps)

    def loss(w2, gm):
        o = PO.OracleInstance(**{**oi.__dict__})
        o.omega2, o.gamma = w2, gm
        o.g, o.p, o.r = PO.tf_coefficients(w2, gm, T)
        return float(ybar @ oracle.forward(o, steps=wl.steps)["y"])

    adj = oracle.adjoint(oi, ybar)
    dw2, dgm = oracle.coefficient_grads_tf(oi, adj, T)
    for mu in (0, 3, 7):
        h = 1e-6 * oi.omega2[mu]
        e = np.zeros(oi.N)
        e[mu] = h
        fd = (loss(oi.omega2 + e, oi.gamma) - loss(oi.omega2 - e, oi.gamma)) / (2 * h)
        assert dw2[mu] == pytest.approx(fd, rel=1e-5, abs=1e-12 * abs(fd) + 1e-30)
        hg = 1e-5 * max(oi.gamma[mu], 1e-3)
        e = np.zeros(oi.N)
        e[mu] = hg
        fdg = (loss(oi.omega2, oi.gamma + e) - loss(oi.omega2, oi.gamma - e)) / (2 * hg)
        assert dgm[mu] == pytest.approx(fdg, rel=1e-5, abs=1e-9 * abs(fdg) + 1e-30)
