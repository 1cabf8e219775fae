"""FP64 oracle: modes, oscillator coefficients, excitation, modal projections.

TEST INFRASTRUCTURE: imported only by the tests, the smoke check and the
benchmark's CPU-baseline leg.  Shares no code with the CUDA library.

Everything here follows the paper's statement of the problem:
  * eigenvalues of the Laplacian, Sec. 3, Eq. 2 (fixed string: lambda = (mu pi / L)^2;
    simply supported rectangle: lambda = (m pi / Lx)^2 + (n pi / Ly)^2),
    with unit-norm modes (string sqrt(2/L) sin, rectangle 2/sqrt(Lx Ly) sin sin);
  * oscillator coefficients, Sec. 3.2, Eq. 13 (omega^2 = (D lambda^2 + T0 lambda)/rho)
    and the damping family of Eq. 14 written gamma = sigma0 + sigma1 omega^2;
  * Stormer-Verlet coefficients r, g, p, Sec. 3.2, Eqs. 21-23, evaluated exactly
    as printed;
  * impulse-invariant (transfer-function) coefficients, Sec. 3.2, Eq. 15-19,
    as the same three-term recursion (see tf_coefficients for the readings);
  * tension-modulation coefficients, Sec. 3.1, Eq. 4 (tau_string = EA / 2L,
    tau_membrane = E h / (2 Lx Ly (1 - nu^2))), divided by rho for the modal form;
  * von Karman scale E / (2 rho zeta^4) of Sec. 3.1, Eq. 9 (volumetric rho);
  * point force projected on unit-norm modes, f_ext = Phi(x_s) F(t) / rho;
  * pluck: q^0 = <w0, Phi> by Gauss-Legendre quadrature, q^{-1} = q^0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Optional

import numpy as np

SV_OMEGA_T_MAX = 1.9   # modes with omega*T >= 1.9 are dropped (Stormer-Verlet needs omega*T < 2)


def rect_sides(inst):
    """Lx, Ly from the fixed area and the aspect a = Ly / Lx."""
    Lx = math.sqrt(inst.area / inst.aspect)
    Ly = math.sqrt(inst.area * inst.aspect)
    return Lx, Ly


def string_modes(inst, n):
    mu = np.arange(1, n + 1)
    lam = (mu * math.pi / inst.length) ** 2
    return mu.reshape(-1, 1), lam


def rect_modes(inst, n):
    """First n simply supported rectangle modes by ascending eigenvalue; ties
    broken by (m, n) lexicographically."""
    Lx, Ly = rect_sides(inst)
    cand = []
    K = int(math.ceil(math.sqrt(n))) + 4
    while True:
        cand = []
        for m in range(1, K + 1):
            for k in range(1, K + 1):
                cand.append(((m * math.pi / Lx) ** 2 + (k * math.pi / Ly) ** 2, m, k))
        cand.sort()
        lam_n = cand[n - 1][0]
        # enough candidates if the n-th eigenvalue is below the smallest excluded one
        edge = min((K + 1) * math.pi / Lx, (K + 1) * math.pi / Ly) ** 2
        if lam_n < edge:
            break
        K *= 2
    sel = cand[:n]
    labels = np.array([[m, k] for _, m, k in sel], dtype=np.int64)
    lam = np.array([l for l, _, _ in sel])
    return labels, lam


def mode_shape_string(inst, labels, x):
    """Unit-norm string modes at relative positions x (fraction of L)."""
    L = inst.length
    mu = labels[:, 0]
    return math.sqrt(2.0 / L) * np.sin(mu * math.pi * np.asarray(x))


def mode_shape_rect(inst, labels, xi, eta):
    """Unit-norm simply supported rectangle modes at relative point (xi, eta)."""
    Lx, Ly = rect_sides(inst)
    m, k = labels[:, 0], labels[:, 1]
    return 2.0 / math.sqrt(Lx * Ly) * np.sin(m * math.pi * xi) * np.sin(k * math.pi * eta)


def omega2_of(lam, D, T0, rho_lin):
    return (D * lam ** 2 + T0 * lam) / rho_lin


def sv_coefficients(omega2, gamma, T):
    """Eqs. 21-23 exactly as printed."""
    r = 2.0 * T ** 2 / (2.0 + 2.0 * gamma * T)
    g = r * (2.0 / T ** 2 - omega2)
    p = r * (-1.0 / T ** 2 + 2.0 * gamma / (2.0 * T))
    return g, p, r


def tau_prime(inst):
    """Tension-modulation coefficient divided by the mass density (Eq. 4)."""
    if inst.kind == "string":
        return inst.EA / (2.0 * inst.length) / inst.rho_lin
    if inst.kind == "membrane":
        Lx, Ly = rect_sides(inst)
        tau = inst.E * inst.thickness / (2.0 * Lx * Ly * (1.0 - inst.nu ** 2))
        return tau / inst.rho_lin
    return 0.0


def tf_coefficients(omega2, gamma, T):
    """Impulse-invariant discretisation of each modal oscillator (Sec. 3.2,
    Eq. 15-19), returned as (g, p, r) of the same three-term recursion
    q^{n+1} = g q^n + p q^{n-1} + r F^n that Eq. 20 uses.

    The roots of z^2 + a1 z + a2 are exp((-gamma +- i w~) T), so
    g = -a1 = 2 exp(-gamma T) cos(w~ T) and p = -a2 = -exp(-2 gamma T).  Two
    readings of the printed Eq. 19: the recursion takes -a1, -a2 (the
    denominator's roots, not the printed signs), and b1 carries the factor T
    that impulse invariance gives a sampled force (the printed 1/rho is part
    of the modal force here): r = T exp(-gamma T) sin(w~ T) / w~, with
    w~ = sqrt(omega^2 - gamma^2).  Over-damped modes (gamma > omega) use the
    hyperbolic forms, the critically damped limit sin(w~ T)/w~ -> T."""
    w2 = np.asarray(omega2, np.float64)
    gm = np.asarray(gamma, np.float64)
    d = w2 - gm ** 2
    e1 = np.exp(-gm * T)
    g = np.empty_like(d)
    s = np.empty_like(d)          # sin(w~ T) / w~ (or its hyperbolic / limit form)
    osc, over = d > 0, d < 0
    wt = np.sqrt(np.abs(d))
    g[osc] = 2.0 * e1[osc] * np.cos(wt[osc] * T)
    s[osc] = np.sin(wt[osc] * T) / wt[osc]
    g[over] = 2.0 * e1[over] * np.cosh(wt[over] * T)
    s[over] = np.sinh(wt[over] * T) / wt[over]
    crit = ~(osc | over)
    g[crit] = 2.0 * e1[crit]
    s[crit] = T
    p = -np.exp(-2.0 * gm * T)
    r = T * e1 * s
    return g, p, r


def strike_signal(inst, fs, steps):
    """Raised-cosine force pulse F(t) = F0/2 (1 - cos(2 pi t / tw)), 0 <= t <= tw,
    sampled at t = n T."""
    t = np.arange(steps) / fs
    e = 0.5 * inst.F0 * (1.0 - np.cos(2.0 * math.pi * t / inst.t_width))
    e[t > inst.t_width] = 0.0
    return e


def pluck_shape(inst, x_rel):
    """Raised-cosine displacement w0 at relative positions x_rel."""
    d = (np.asarray(x_rel) - inst.pluck_x0) / inst.pluck_width
    w = 0.5 * inst.pluck_amp * (1.0 + np.cos(2.0 * math.pi * d))
    return np.where(np.abs(d) <= 0.5, w, 0.0)


def pluck_projection(inst, labels, n_quad=64):
    """q^0_mu = integral_0^L w0(x) Phi_mu(x) dx, by Gauss-Legendre quadrature over
    the support of the pluck (the integrand is smooth there)."""
    L = inst.length
    xg, wg = np.polynomial.legendre.leggauss(n_quad)
    a = (inst.pluck_x0 - 0.5 * inst.pluck_width)
    b = (inst.pluck_x0 + 0.5 * inst.pluck_width)
    xr = a + (xg + 1.0) * 0.5 * (b - a)               # relative positions
    w0 = pluck_shape(inst, xr)
    phi = math.sqrt(2.0 / L) * np.sin(np.outer(labels[:, 0], xr) * math.pi)
    return phi @ (w0 * wg) * 0.5 * (b - a) * L


@dataclass
class OracleInstance:
    kind: str
    N: int
    M: int
    labels: np.ndarray
    lam: np.ndarray
    omega2: np.ndarray
    gamma: np.ndarray
    g: np.ndarray
    p: np.ndarray
    r: np.ndarray
    b: np.ndarray
    c: np.ndarray
    taup: float
    e: np.ndarray
    q0: np.ndarray
    qm1: np.ndarray
    kappa: Optional[np.ndarray] = None   # [M]
    H: Optional[np.ndarray] = None       # [M][N][N]
    zeta4: Optional[np.ndarray] = None
    src: object = None


def n_psi_after_truncation(n_psi, n_phi, n_phi_eff):
    """Stress modes kept when stability truncation shortens the transverse set."""
    if n_phi_eff >= n_phi:
        return n_psi
    return min(n_psi, max(1, (n_psi * n_phi_eff) // n_phi))


def build_instance(inst, fs, steps, coupling=None, scheme="sv"):
    """All FP64 inputs of one instance.

    `coupling`, for plates, is a callable (inst, labels, n_psi) -> (H, zeta4)
    returning the coupling tensor of Sec. 3.1, Eq. 10 for the given transverse
    mode labels, and the Airy eigenvalues zeta^4.  `scheme` selects the
    time discretisation: "sv" (Stormer-Verlet, Eq. 20-23) or "tf" (impulse
    invariance, Eq. 15-19; the same mode truncation is applied so the two
    schemes see the same modes).
    """
    T = 1.0 / fs
    if inst.kind == "string":
        labels, lam = string_modes(inst, inst.n_phi)
    else:
        labels, lam = rect_modes(inst, inst.n_phi)
    omega2 = omega2_of(lam, inst.D, inst.T0, inst.rho_lin)
    keep = np.sqrt(omega2) * T < SV_OMEGA_T_MAX
    # modes are sorted by lambda and omega^2 grows with lambda: keep a prefix
    n_eff = int(np.argmin(keep)) if not keep.all() else len(keep)
    labels, lam, omega2 = labels[:n_eff], lam[:n_eff], omega2[:n_eff]
    gamma = inst.sigma0 + inst.sigma1 * omega2
    if scheme == "tf":
        g, p, r = tf_coefficients(omega2, gamma, T)
    else:
        g, p, r = sv_coefficients(omega2, gamma, T)
    if inst.kind == "string":
        c = mode_shape_string(inst, labels, inst.pickup[0])
        bshape = mode_shape_string(inst, labels, inst.strike[0])
    else:
        c = mode_shape_rect(inst, labels, *inst.pickup)
        bshape = mode_shape_rect(inst, labels, *inst.strike)
    if inst.excitation == "pluck":
        e = np.zeros(steps)
        q0 = pluck_projection(inst, labels)
        b = bshape / inst.rho_lin
    else:
        e = strike_signal(inst, fs, steps)
        q0 = np.zeros(n_eff)
        b = bshape / inst.rho_lin
    qm1 = q0.copy()
    taup = tau_prime(inst) if inst.nonlinear else 0.0
    M = 0
    H = kappa = zeta4 = None
    if inst.kind == "plate":
        M = n_psi_after_truncation(inst.n_psi, inst.n_phi, n_eff)
        if inst.nonlinear and coupling is not None and M > 0:
            H, zeta4 = coupling(inst, labels, M)
            kappa = inst.E / (2.0 * inst.rho_vol * zeta4)
        else:
            M = 0
    return OracleInstance(kind=inst.kind, N=n_eff, M=M, labels=labels, lam=lam,
                          omega2=omega2, gamma=gamma, g=g, p=p, r=r, b=b, c=c, taup=taup,
                          e=e, q0=q0, qm1=qm1, kappa=kappa, H=H, zeta4=zeta4, src=inst)
