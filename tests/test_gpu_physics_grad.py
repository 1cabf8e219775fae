"""Gradients with respect to the physical parameters through the GPU path
(Sec. 4.3: the inverse problems fit tension, stiffness, geometry and damping
by gradient descent through the simulation).

A 48 x 12 steel plate is prepared by the library (mdx_modal_from_physics,
the coupling tensor and its aspect derivative from the FP64 generator),
simulated and differentiated on the GPU (mdx_simulate + mdx_grad, fused
adjoint sweep), and its per-mode gradients are mapped to
(T0, D, aspect, sigma0, sigma1, E / (2 rho_vol)) by mdx_physics_vjp.  Each is
compared with a central finite difference of the independent FP64 oracle's
whole map theta -> modes -> H -> audio -> L, L = sum_n ybar^n y^n.
Tolerance 1e-4 relative (the gradient tolerance of the other GPU tests; the
finite differences are accurate to about 1e-6 with the steps below)."""
import copy

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle
from oracle import coupling_oracle as CO
from oracle import physics_oracle as PO
from paper_2505_05940_gb300 import _native as N
from paper_2505_05940_gb300 import modal, physics, workloads as W

GTOL = 1e-4


def _oracle_loss(inst, fs, steps, ybar):
    oi = PO.build_instance(inst, fs, steps, coupling=CO.oracle_coupling)
    return float(ybar @ oracle.forward(oi, steps=steps)["y"])


def test_physical_gradients_match_oracle_finite_differences():
    fs, steps, K = 44100.0, 800, 128
    inst = W.tiny_random(8, "plate", 48, 12, steps=steps).instances[0]
    inst.F0, inst.T0, inst.aspect = 400.0, 60.0, 1.37
    rng = np.random.default_rng(2)
    ybar = rng.normal(size=steps).astype(np.float32).astype(np.float64)
    p = physics.prepare(inst, fs, steps, want_aspect_derivative=True)
    assert len(p["omega2"]) == 48 and len(p["kappa"]) == 12 and p.get("dH") is not None
    sim = modal.Simulator([p], force_split=3)
    r = sim.simulate(steps, K=K)
    g = sim.grad(steps, torch.tensor(ybar[None], dtype=torch.float32, device="cuda"), K,
                 r["ckpt"], want_status=True)
    torch.cuda.synchronize()
    assert int(g["status"][0]) == 0
    got = N.physics_vjp(physics.physics_struct(p), 48, 12, g["d_omega2"].cpu().numpy(),
                        g["d_gamma"].cpu().numpy(), 0.0, g["d_kappa"].cpu().numpy(),
                        float(g["d_dir"][0]), p["dzeta4"])

    def fd(attr, rel_h, scale=1.0):
        x0 = getattr(inst, attr)
        h = rel_h * abs(x0)
        vals = []
        for x in (x0 + h, x0 - h):
            i2 = copy.deepcopy(inst)
            setattr(i2, attr, x)
            vals.append(_oracle_loss(i2, fs, steps, ybar))
        return (vals[0] - vals[1]) / (2 * h) * scale

    refs = {"d_T0": fd("T0", 1e-3), "d_D": fd("D", 1e-4), "d_aspect": fd("aspect", 1e-5),
            "d_sigma0": fd("sigma0", 1e-3), "d_sigma1": fd("sigma1", 1e-3),
            "d_vk_scale": fd("E", 1e-3, scale=2.0 * inst.rho_vol)}
    for k, ref in refs.items():
        e = abs(got[k] - ref) / abs(ref)
        assert e <= GTOL, (k, got[k], ref, e)
