"""Parity at the benchmark's full size: the 64-plate adjoint batch (200 x 50
modes, 22 050 steps, K = 1024) in the launch configuration bench.py times.
One plate, built by the oracle, is checked against the FP64 oracle over the
whole run; the gradient is checked through properties that hold at any size
(the fused sweep equals separate launches bit for bit, and the result does
not depend on the checkpoint interval)."""
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle
from paper_2505_05940_gb300 import modal, physics, workloads as W

from test_gpu_parity import TOL, oracle_instance, rel, to_plan

SAMPLE = 5      # the plate the oracle checks


@pytest.fixture(scope="module")
def batch():
    _, inits = W.adjoint_plates(seed=0, n_inst=64, steps=22050)
    prep = [physics.prepare(i, inits.fs, inits.steps) for i in inits.instances]
    oi = oracle_instance(inits.instances[SAMPLE], inits.fs, inits.steps)
    prep[SAMPLE] = to_plan(oi, inits.fs)
    return prep, oi, inits


def test_full_size_forward_sampled_plate(batch):
    prep, oi, inits = batch
    sim = modal.Simulator(prep)
    r = sim.simulate(inits.steps, K=1024, want_state=True, want_status=True)
    torch.cuda.synchronize()
    assert (r["status"].cpu().numpy() == 0).all()
    ref = oracle.forward(oi, steps=inits.steps)
    assert rel(r["audio"][SAMPLE].cpu().numpy(), ref["y"]) <= TOL
    off = sim.plan.mode_offset[SAMPLE]
    q = r["q_end"].cpu().numpy()[off:off + oi.N]
    assert rel(q, ref["qN"]) <= TOL


def test_full_size_gradient_properties(batch):
    prep, _, inits = batch
    steps = inits.steps
    yb = torch.randn(len(prep), steps, dtype=torch.float32, device="cuda") * 1e-3
    outs = []
    for flags, K in ((0, 1024), (2, 1024), (0, 256)):
        sim = modal.Simulator(prep, debug_flags=flags)
        r = sim.simulate(steps, K=K)
        g = sim.grad(steps, yb, K, r["ckpt"], want_status=True)
        torch.cuda.synchronize()
        assert (g["status"] == 0).all()
        outs.append(g)
        del sim
    for k in ("d_omega2", "d_gamma", "d_b", "d_c", "d_q0", "d_qm1", "d_kappa"):
        assert torch.equal(outs[0][k], outs[1][k]), ("fused vs separate", k)
        assert torch.equal(outs[0][k], outs[2][k]), ("K = 1024 vs 256", k)
