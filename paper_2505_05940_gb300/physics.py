"""Host FP64 preparation of plan inputs from physical parameters.

  * Laplacian eigenpairs (Sec. 3, Eq. 2): fixed string lambda = (mu pi/L)^2,
    simply supported rectangle lambda = (m pi/Lx)^2 + (n pi/Ly)^2, modes in
    ascending lambda with ties ordered by (m, n); unit-norm mode shapes.
  * omega^2, gamma (Sec. 3.2, Eq. 13-14) through the library's
    mdx_coeffs_from_physics.
  * stability truncation: modes with omega T >= 1.9 are dropped (the
    Stormer-Verlet update of Eq. 20 needs omega T < 2); a shortened plate keeps
    the same fraction of stress modes.
  * tension-modulation coefficient tau / rho (Eq. 4), von Karman scale
    kappa = E / (2 rho zeta^4) (Eq. 9).
  * excitation: point force projected on the modes (b = Phi(x_s) / rho_lin,
    raised-cosine force pulse e^n), or a raised-cosine pluck projected in
    closed form (q^0 = <w0, Phi>, q^{-1} = q^0).
"""
from __future__ import annotations

import math
from typing import List

import numpy as np

from . import _native
from . import coupling as _coupling

OMEGA_T_LIMIT = 1.9


def rectangle_sides(inst):
    return _coupling.sides(inst.area, inst.aspect)


def string_eigen(length, n):
    mu = np.arange(1, n + 1, dtype=np.int64)
    return mu[:, None], (math.pi * mu / length) ** 2


def rectangle_eigen(Lx, Ly, n):
    """First n (m, n) labels by ascending eigenvalue, ties by (m, n)."""
    # Weyl: N(lambda) ~ Lx Ly lambda / (4 pi); enlarge the window until it is safe
    span = int(math.sqrt(4.0 * n / math.pi * max(Lx / Ly, Ly / Lx))) + 6
    while True:
        mm, nn = np.meshgrid(np.arange(1, span + 1), np.arange(1, span + 1), indexing="ij")
        mm, nn = mm.ravel(), nn.ravel()
        lam = (math.pi * mm / Lx) ** 2 + (math.pi * nn / Ly) ** 2
        order = np.lexsort((nn, mm, lam))[:n]
        bound = min((math.pi * (span + 1) / Lx) ** 2, (math.pi * (span + 1) / Ly) ** 2)
        if lam[order[-1]] < bound:
            return np.stack([mm[order], nn[order]], axis=1), lam[order]
        span *= 2


def shape_string(length, labels, xrel):
    return math.sqrt(2.0 / length) * np.sin(math.pi * labels[:, 0] * xrel)


def shape_rectangle(Lx, Ly, labels, xrel, yrel):
    return (2.0 / math.sqrt(Lx * Ly)) * np.sin(math.pi * labels[:, 0] * xrel) * \
        np.sin(math.pi * labels[:, 1] * yrel)


def raised_cosine_force(F0, width, fs, steps):
    t = np.arange(steps) / fs
    return np.where(t <= width, 0.5 * F0 * (1.0 - np.cos(2.0 * math.pi * t / width)), 0.0)


def pluck_modal(length, labels, amp, x0_rel, width_rel):
    """<w0, Phi_mu> of w0 = amp/2 (1 + cos(2 pi (x - x0)/W)) on |x - x0| <= W/2,
    in closed form (removable singularity at mu pi / L = 2 pi / W)."""
    k = math.pi * labels[:, 0].astype(np.float64) / length
    x0 = x0_rel * length
    W = width_rel * length
    a = 2.0 * math.pi / W
    num = amp * np.sin(k * x0) * np.sin(0.5 * k * W) * a * a
    den = k * (a * a - k * k)
    near = np.abs(a - k) < 1e-9 * a
    safe = np.where(near, 1.0, den)
    val = np.where(near, amp * np.sin(k * x0) * W / 4.0, num / safe)
    return math.sqrt(2.0 / length) * val


class PreparedInstance(dict):
    """Plan-ready description of one instance (plus its inputs)."""


def prepare(inst, fs, steps, coupling="auto", want_aspect_derivative=False):
    """Physical parameters -> dict with the mdx_instance fields, the excitation
    e [steps], the initial state q0, qm1 and bookkeeping (labels, lambda)."""
    T = 1.0 / fs
    if inst.kind == "string":
        labels, lam = string_eigen(inst.length, inst.n_phi)
    else:
        Lx, Ly = rectangle_sides(inst)
        labels, lam = rectangle_eigen(Lx, Ly, inst.n_phi)
    omega2, gamma = _native.coeffs_from_physics(lam, inst.D, inst.T0, inst.rho_lin,
                                                inst.sigma0, inst.sigma1)
    ok = np.sqrt(omega2) * T < OMEGA_T_LIMIT
    n_eff = len(ok) if ok.all() else int(np.argmin(ok))
    labels, lam, omega2, gamma = labels[:n_eff], lam[:n_eff], omega2[:n_eff], gamma[:n_eff]
    if inst.kind == "string":
        b = shape_string(inst.length, labels, inst.strike[0]) / inst.rho_lin
        c = shape_string(inst.length, labels, inst.pickup[0])
    else:
        b = shape_rectangle(Lx, Ly, labels, *inst.strike) / inst.rho_lin
        c = shape_rectangle(Lx, Ly, labels, *inst.pickup)
    if inst.excitation == "pluck":
        e = np.zeros(steps)
        q0 = pluck_modal(inst.length, labels, inst.pluck_amp, inst.pluck_x0, inst.pluck_width)
    else:
        e = raised_cosine_force(inst.F0, inst.t_width, fs, steps)
        q0 = np.zeros(n_eff)
    out = PreparedInstance(kind="tension" if inst.kind != "plate" else "plate",
                           omega2=omega2, gamma=gamma, b=b, c=c, dt=T, lam=lam,
                           labels=labels, e=e, q0=q0, qm1=q0.copy(), src=inst)
    if inst.kind == "string":
        out["tau"] = (inst.EA / (2.0 * inst.length)) / inst.rho_lin if inst.nonlinear else 0.0
    elif inst.kind == "membrane":
        tau = inst.E * inst.thickness / (2.0 * Lx * Ly * (1.0 - inst.nu ** 2))
        out["tau"] = tau / inst.rho_lin if inst.nonlinear else 0.0
    else:
        M = inst.n_psi if n_eff >= inst.n_phi else min(inst.n_psi, max(1, inst.n_psi * n_eff // inst.n_phi))
        out["tau"] = 0.0
        if inst.nonlinear and M > 0 and coupling is not None:
            psi_cls = None
            if callable(coupling):
                res = coupling(inst, labels, M)
                H, zeta4 = res[0], res[1]
                if len(res) > 2:
                    psi_cls = res[2]
                dH = dz = None
            elif want_aspect_derivative:
                H, zeta4, dH, dz, psi_cls = _coupling.coupling_with_aspect_derivative(
                    inst.area, inst.aspect, labels, M)
            else:
                airy = _coupling.airy_modes(Lx, Ly, M)
                H, zeta4 = _coupling.coupling_tensor(Lx, Ly, labels, M, airy=airy)
                psi_cls = _coupling.airy_classes(airy[1])
                dH = dz = None
            if psi_cls is not None:
                # symmetry classes: H^k_ij vanishes unless class(i) ^ class(j) == class(k)
                out["phi_class"] = _coupling.transverse_classes(labels)
                out["psi_class"] = psi_cls
            out["H"] = H.astype(np.float32)
            out["zeta4"] = zeta4
            out["kappa"] = inst.E / (2.0 * inst.rho_vol * zeta4)
            if dH is not None:
                out["dH"] = dH.astype(np.float32)
                out["dzeta4"] = dz
    return out


def prepare_workload(wl, coupling="auto", want_aspect_derivative=False) -> List[PreparedInstance]:
    return [prepare(inst, wl.fs, wl.steps, coupling, want_aspect_derivative)
            for inst in wl.instances]
