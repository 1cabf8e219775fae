"""Host FP64 entry points from physical parameters to modal coefficients
(mdx_modal_from_physics) and back (mdx_physics_vjp), on the CPU.

  * The map matches the oracle's own derivation (Sec. 3, Eq. 2; Sec. 3.2,
    Eq. 13-14; Eq. 4; Eq. 9; projections; stability cut) for strings,
    membranes and plates, including a plate the stability cut shortens.
  * The vector-Jacobian product, fed with the FP64 oracle adjoint of a small
    plate (and with the oracle's own finite-difference derivative of its
    coupling tensor and Airy eigenvalues with respect to the aspect ratio),
    matches central finite differences of the oracle's whole map
    theta -> modal coefficients -> H -> audio -> loss, for tension, stiffness,
    aspect ratio, both damping parameters and the von Karman scale.
"""
import copy
import math

import numpy as np
import pytest

import oracle
from oracle import coupling_oracle as CO
from oracle import physics_oracle as PO
from paper_2505_05940_gb300 import _native as N
from paper_2505_05940_gb300 import physics as PH
from paper_2505_05940_gb300 import workloads as W


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("case", ["string", "membrane", "plate", "plate-cut", "string-cut"])
def test_modal_from_physics_matches_oracle(case):
    fs = 44100.0
    if case.startswith("string"):
        inst = W.tiny_random(3, "string", 60 if case == "string" else 400).instances[0]
    elif case == "membrane":
        inst = W.tiny_random(4, "membrane", 150).instances[0]
    else:
        inst = W.tiny_random(5, "plate", 90, 22).instances[0]
        if case == "plate-cut":
            inst.n_phi, inst.n_psi, inst.D = 400, 100, inst.D * 40.0
    zeta4 = None
    if inst.kind == "plate":
        zeta4 = np.sort(np.random.default_rng(1).uniform(1e3, 1e6, inst.n_psi))
    cp = (lambda i, lab, m: (np.zeros((m, len(lab), len(lab))), zeta4[:m])) \
        if inst.kind == "plate" else None
    oi = PO.build_instance(inst, fs, 10, coupling=cp)
    got = N.modal_from_physics(PH.physics_of(inst, fs, zeta4=zeta4))
    if case.endswith("cut"):
        assert oi.N < inst.n_phi              # the stability cut shortened it
    assert len(got["lam"]) == oi.N
    assert np.array_equal(got["labels"][:, :oi.labels.shape[1]], oi.labels)
    for k, ref in (("lam", oi.lam), ("omega2", oi.omega2), ("gamma", oi.gamma), ("b", oi.b),
                   ("c", oi.c)):
        assert _rel(got[k], ref) <= 1e-14, k
    assert abs(got["tau"] - oi.taup) <= 1e-14 * max(abs(oi.taup), 1e-300)
    if inst.kind == "plate":
        assert got["n_psi"] == oi.M
        assert _rel(got["kappa"], oi.kappa) <= 1e-14


def _loss(inst, fs, steps, ybar):
    """The oracle's whole map theta -> L = sum_n ybar^n y^n."""
    oi = PO.build_instance(inst, fs, steps, coupling=CO.oracle_coupling)
    return float(ybar @ oracle.forward(oi, steps=steps)["y"]), oi


def _aligned(Ha, Hb):
    """Airy modes carry an arbitrary sign: flip the modes of Ha whose
    coupling tensor points away from Hb's."""
    s = np.sign(np.einsum("kij,kij->k", Ha, Hb))
    return Ha * s[:, None, None]


def test_physics_vjp_matches_oracle_finite_differences():
    fs, steps = 44100.0, 600
    inst = W.tiny_random(8, "plate", 14, 5, steps=steps).instances[0]
    inst.F0 = 400.0
    inst.T0 = 60.0
    rng = np.random.default_rng(2)
    ybar = rng.normal(size=steps)
    L0, oi = _loss(inst, fs, steps, ybar)
    assert oi.N == inst.n_phi and oi.M == inst.n_psi
    adj = oracle.adjoint(oi, ybar, want_dH=True)
    dw2, dgm = oracle.coefficient_grads(oi, adj, 1.0 / fs)
    # the oracle's own aspect derivative of H and zeta^4 (central differences)
    ha = 1e-5 * inst.aspect
    Hs, zs = [], []
    for a in (inst.aspect + ha, inst.aspect - ha):
        i2 = copy.deepcopy(inst)
        i2.aspect = a
        lab, _ = PO.rect_modes(i2, i2.n_phi)
        assert np.array_equal(lab, oi.labels)
        H, z = CO.coupling_H(i2, lab, oi.M)
        Hs.append(_aligned(H, oi.H))
        zs.append(z)
    dHda = (Hs[0] - Hs[1]) / (2 * ha)
    dzda = (zs[0] - zs[1]) / (2 * ha)
    d_dir = float(np.sum(adj["dH"] * dHda))
    ph = PH.physics_of(inst, fs, zeta4=oi.zeta4)
    got = N.physics_vjp(ph, oi.N, oi.M, dw2, dgm, 0.0, adj["dkappa"], d_dir, dzda)

    def fd(attr, rel_h):
        x0 = getattr(inst, attr)
        h = rel_h * abs(x0)
        vals = []
        for x in (x0 + h, x0 - h):
            i2 = copy.deepcopy(inst)
            setattr(i2, attr, x)
            vals.append(_loss(i2, fs, steps, ybar)[0])
        return (vals[0] - vals[1]) / (2 * h)

    # relative steps: large enough that the loss's rounding noise (about 1e-13
    # after 600 nonlinear steps) stays far below the difference, small enough
    # that the O(h^2) truncation does too (aspect 0.99 sits near degenerate
    # mode pairs, so its step is the smallest)
    checks = {"d_T0": fd("T0", 1e-3), "d_D": fd("D", 1e-4), "d_aspect": fd("aspect", 1e-5),
              "d_sigma0": fd("sigma0", 1e-3), "d_sigma1": fd("sigma1", 1e-3)}
    # von Karman scale E / (2 rho_vol): through E at fixed rho_vol
    i2 = copy.deepcopy(inst)
    hE = 1e-3 * inst.E
    vals = []
    for E in (inst.E + hE, inst.E - hE):
        i2.E = E
        vals.append(_loss(i2, fs, steps, ybar)[0])
    checks["d_vk_scale"] = (vals[0] - vals[1]) / (2 * hE) * (2.0 * inst.rho_vol)
    for k, ref in checks.items():
        assert abs(got[k] - ref) <= 2e-6 * abs(ref), (k, got[k], ref)


def test_physics_vjp_string_tension_scale():
    """A string's d_tension_stiffness is dL/dtau' / (2 L rho) and its aspect
    gradient is zero; checked against finite differences of the oracle map in
    EA."""
    fs, steps = 48000.0, 800
    inst = W.tiny_random(9, "string", 12, steps=steps, fs=fs).instances[0]
    rng = np.random.default_rng(4)
    ybar = rng.normal(size=steps)
    oi = PO.build_instance(inst, fs, steps)
    adj = oracle.adjoint(oi, ybar)
    dw2, dgm = oracle.coefficient_grads(oi, adj, 1.0 / fs)
    got = N.physics_vjp(PH.physics_of(inst, fs), oi.N, 0, dw2, dgm, adj["dtau"])
    assert got["d_aspect"] == 0.0 and got["d_vk_scale"] == 0.0
    h = 1e-3 * inst.EA
    vals = []
    for ea in (inst.EA + h, inst.EA - h):
        i2 = copy.deepcopy(inst)
        i2.EA = ea
        o2 = PO.build_instance(i2, fs, steps)
        vals.append(float(ybar @ oracle.forward(o2, steps=steps)["y"]))
    ref = (vals[0] - vals[1]) / (2 * h)
    assert abs(got["d_tension_stiffness"] - ref) <= 1e-6 * abs(ref)


def test_modal_from_physics_rejects_bad_input():
    inst = W.tiny_random(5, "plate", 20, 5).instances[0]
    with pytest.raises(N.MdxError):
        N.modal_from_physics(PH.physics_of(inst, 44100.0, rho=0.0))
    with pytest.raises(N.MdxError):
        N.modal_from_physics(PH.physics_of(inst, 44100.0, n_phi=0))
    with pytest.raises(N.MdxError):
        N.modal_from_physics(PH.physics_of(inst, 44100.0, shape=N.SHAPE_STRING))
