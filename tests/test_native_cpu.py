"""CPU-side checks of the library surface: the shared library loads, exports
every entry point declared in include/mdx.h, its host-only functions are
right, and plan validation rejects bad instances before touching the GPU.
No compute kernel is launched here."""
import math
import os
import re

import numpy as np
import pytest

from paper_2505_05940_gb300 import _native as N
from paper_2505_05940_gb300 import coupling as PC
from paper_2505_05940_gb300 import physics as PH
from paper_2505_05940_gb300 import workloads as W
from oracle import coupling_oracle as CO
from oracle import physics_oracle as PO

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(mdx_\w+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol():
    L = N.load()
    declared = _declared()
    assert "mdx_simulate" in declared and "mdx_grad" in declared
    for name in declared:
        assert hasattr(L, name), name
    assert L.mdx_version().startswith(b"mdx")


def test_coeffs_from_physics_and_vjp():
    rng = np.random.default_rng(0)
    lam = rng.uniform(10, 1e4, 17)
    D, T0, rho, s0, s1 = 18.3, 100.0, 7.8, 1.0, 3e-6
    w2, gm = N.coeffs_from_physics(lam, D, T0, rho, s0, s1)
    np.testing.assert_allclose(w2, (D * lam ** 2 + T0 * lam) / rho, rtol=1e-15)
    np.testing.assert_allclose(gm, s0 + s1 * w2, rtol=1e-15)
    dw, dg = rng.normal(size=17), rng.normal(size=17)
    v = N.coeffs_vjp(lam, D, T0, rho, s0, s1, dw, dg)
    L = lambda D_, T_, a, b_: float(dw @ ((D_ * lam ** 2 + T_ * lam) / rho) +
                                   dg @ (a + b_ * (D_ * lam ** 2 + T_ * lam) / rho))
    # L is affine in each parameter separately: a wide central difference is exact
    for key, i, h in (("D", 0, 1.0), ("T0", 1, 10.0), ("s0", 2, 0.1), ("s1", 3, 1e-6)):
        x = [D, T0, s0, s1]
        xp = list(x); xp[i] += h
        xm = list(x); xm[i] -= h
        fd = (L(*xp) - L(*xm)) / (2 * h)
        assert abs(v[key] - fd) <= 1e-7 * abs(fd), (key, v[key], fd)


def _inst(**kw):
    d = dict(kind="tension", omega2=np.array([100.0, 400.0]), gamma=np.array([1.0, 1.0]),
             b=np.ones(2), c=np.ones(2), lam=np.array([1.0, 4.0]), tau=0.0, dt=1e-4)
    d.update(kw)
    return d


@pytest.mark.parametrize("bad, code", [
    (dict(gamma=np.array([1.0, -1.0])), 2),                   # pole in the right half-plane
    (dict(omega2=np.array([100.0, (2.0 / 1e-4) ** 2])), 2),   # omega T = 2: unstable
    (dict(omega2=np.array([100.0, np.nan])), 3),
    (dict(omega2=np.array([100.0, -1.0])), 1),
    (dict(dt=0.0), 1),
    (dict(tau=-1.0), 1),
])
def test_plan_validation_rejects(bad, code):
    with pytest.raises(N.MdxError) as ei:
        N.Plan([_inst(**bad)])
    assert ei.value.code == code


def test_plan_rejects_asymmetric_H():
    H = np.ones((1, 2, 2), np.float32)
    H[0, 0, 1] = 2.0
    d = _inst(kind="plate", H=H, kappa=np.ones(1))
    with pytest.raises(N.MdxError) as ei:
        N.Plan([d])
    assert ei.value.code == 1 and "symmetric" in str(ei.value)


def test_product_physics_matches_oracle():
    """The library's host-side plan inputs (modes, omega^2, gamma, b, c, q0,
    truncation) equal the oracle's independent derivation."""
    wls = [W.string_40(), W.plate_100x30(), W.tiny_random(3, "membrane", 50),
           W.batched_ragged(seed=0, n_inst=40, steps=64)]
    for wl in wls:
        for inst in wl.instances:
            a = PH.prepare(inst, wl.fs, wl.steps, coupling=None)
            o = PO.build_instance(inst, wl.fs, wl.steps)
            assert len(a["omega2"]) == o.N
            np.testing.assert_array_equal(a["labels"], o.labels)
            for k_a, k_o in (("omega2", "omega2"), ("gamma", "gamma"), ("b", "b"), ("c", "c"),
                             ("lam", "lam"), ("e", "e")):
                np.testing.assert_allclose(a[k_a], getattr(o, k_o), rtol=1e-12, atol=1e-300)
            np.testing.assert_allclose(a["q0"], o.q0, rtol=1e-9, atol=1e-15)
            assert math.isclose(a["tau"], o.taup, rel_tol=1e-14, abs_tol=0)


def test_product_coupling_matches_oracle():
    """Separable 1D-integral generator == 2D-quadrature oracle (Eq. 10)."""
    inst = W.tiny_random(5, "plate", 40, 10).instances[0]
    labels, _ = PO.rect_modes(inst, 40)
    Lx, Ly = PO.rect_sides(inst)
    H1, z1 = PC.coupling_tensor(Lx, Ly, labels, 10)
    H2, z2 = CO.coupling_H(inst, labels, 10)
    np.testing.assert_allclose(z1, z2, rtol=1e-10)
    assert np.abs(H1 - H2).max() <= 1e-9 * np.abs(H2).max()


def test_aspect_derivative_matches_secant():
    inst = W.tiny_random(6, "plate", 20, 5).instances[0]
    labels, _ = PO.rect_modes(inst, 20)
    H, z, dH, dz, _ = PC.coupling_with_aspect_derivative(inst.area, inst.aspect, labels, 5)
    h = 1e-3 * inst.aspect
    Hp, zp = PC.coupling_tensor(*PC.sides(inst.area, inst.aspect + h), labels, 5)
    Hm, zm = PC.coupling_tensor(*PC.sides(inst.area, inst.aspect - h), labels, 5)
    # align Airy signs by the sign of the overlap with H
    sp = np.sign(np.einsum("kij,kij->k", Hp, H))[:, None, None]
    sm = np.sign(np.einsum("kij,kij->k", Hm, H))[:, None, None]
    sec = (sp * Hp - sm * Hm) / (2 * h)
    assert np.abs(dH - sec).max() <= 1e-4 * np.abs(sec).max()
    np.testing.assert_allclose(dz, (zp - zm) / (2 * h), rtol=1e-5)


def test_coupling_symmetry_classes():
    """H^k_ij vanishes (to rounding) unless class(i) ^ class(j) == class(k);
    a quarter of the tensor is structurally nonzero."""
    inst = W.tiny_random(7, "plate", 120, 30).instances[0]
    labels, _ = PO.rect_modes(inst, 120)
    Lx, Ly = PO.rect_sides(inst)
    airy = PC.airy_modes(Lx, Ly, 30)
    H, _ = PC.coupling_tensor(Lx, Ly, labels, 30, airy=airy)
    fc = PC.transverse_classes(labels)
    kc = PC.airy_classes(airy[1])
    mask = (fc[:, None] ^ fc[None, :])[None] == kc[:, None, None]
    assert np.abs(H[~mask]).max() <= 1e-12 * np.abs(H).max()
    assert 0.2 < mask.mean() < 0.3
    # the same classes describe the oracle's independently generated tensor (its
    # full-basis eigensolver mixes the parity blocks at solver rounding, ~1e-10)
    Ho, _ = CO.coupling_H(inst, labels, 30)
    assert np.abs(Ho[~mask]).max() <= 1e-9 * np.abs(Ho).max()


# ----------------------------------------------------------------- time schemes

def _modes(seed, n=200):
    rng = np.random.default_rng(seed)
    T = 1.0 / 44100.0
    w2 = (rng.uniform(0.001, 1.85, n) / T) ** 2
    gm = rng.uniform(0.0, 1.0, n) * np.minimum(np.sqrt(w2) * 0.5, 2e3)
    return w2, gm, T


@pytest.mark.parametrize("scheme", ["sv", "tf"])
def test_difference_coefficients_match_oracle(scheme):
    """eps = 1 + p and rho = 1 - g - p of the oracle's three-term recursion
    (Eq. 21-23 for Stormer-Verlet, Eq. 16-19 for impulse invariance)."""
    w2, gm, T = _modes(1)
    eps, rho, r = N.difference_coefficients(scheme, w2, gm, T)
    f = PO.sv_coefficients if scheme == "sv" else PO.tf_coefficients
    g, p, rr = f(w2, gm, T)
    np.testing.assert_allclose(r, rr, rtol=1e-13)
    np.testing.assert_allclose(eps, 1.0 + p, rtol=1e-9, atol=1e-15)
    # 1 - g - p cancels in the oracle's form: compare at its rounding level
    np.testing.assert_allclose(rho, 1.0 - g - p, rtol=1e-8, atol=4e-16)


def test_sv_difference_coefficients_are_the_planned_ones():
    """The Stormer-Verlet branch is the closed form the plan always used,
    bit for bit (eps = 2 gamma T/(1+gamma T), r = T^2/(1+gamma T), rho = r omega^2)."""
    w2, gm, T = _modes(2)
    eps, rho, r = N.difference_coefficients("sv", w2, gm, T)
    den = 1.0 + gm * T
    rr = T * T / den
    assert np.array_equal(eps, 2.0 * gm * T / den)
    assert np.array_equal(r, rr)
    assert np.array_equal(rho, rr * w2)


@pytest.mark.parametrize("scheme", ["sv", "tf"])
def test_coefficient_grads_match_oracle_chain_rule(scheme):
    """The chain rule the gradient epilogue runs equals the oracle's (which
    is pinned against finite differences), with the adjoint sums mapped
    through eps = 1 + p, rho = 1 - g - p: A = dL/dg, V = dL/dg - dL/dp,
    F = dL/dr."""
    import oracle
    w2, gm, T = _modes(3)
    rng = np.random.default_rng(4)
    dg, dp, dr = (rng.standard_normal(len(w2)) for _ in range(3))
    f = PO.sv_coefficients if scheme == "sv" else PO.tf_coefficients
    g, p, r = f(w2, gm, T)
    oi = PO.OracleInstance(kind="string", N=len(w2), M=0, labels=None, lam=None, omega2=w2,
                           gamma=gm, g=g, p=p, r=r, b=None, c=None, taup=0.0, e=None, q0=None,
                           qm1=None)
    adj = dict(dg=dg, dp=dp, dr=dr)
    ref = (oracle.coefficient_grads if scheme == "sv" else oracle.coefficient_grads_tf)(oi, adj, T)
    got = N.coefficient_grads(scheme, w2, gm, T, dg, dg - dp, dr)
    for a, b in zip(got, ref):
        np.testing.assert_allclose(a, b, rtol=1e-7, atol=1e-12 * np.abs(b).max())


def test_scheme_domains():
    T = 1.0 / 44100.0
    with pytest.raises(N.MdxError):       # Stormer-Verlet: omega T >= 2
        N.difference_coefficients("sv", [(2.5 / T) ** 2], [1.0], T)
    eps, rho, r = N.difference_coefficients("tf", [(2.5 / T) ** 2], [1.0], T)
    assert np.isfinite(rho).all()         # impulse invariance has no such bound
    with pytest.raises(N.MdxError):       # ... but needs an oscillatory mode
        N.difference_coefficients("tf", [100.0], [20.0], T)
