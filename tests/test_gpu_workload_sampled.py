"""Parity at the benchmark's full size: the 64-plate adjoint batch (200 x 50
modes, 22 050 steps, K = 1024) in the launch configuration bench.py times.
Plates built by the oracle sit at sampled positions of the batch:
  * one plate is checked against the FP64 oracle over the whole run;
  * two plates' gradients (d omega^2, d gamma, d b, d c, d kappa and the
    contraction <dL/dH, dH> with a direction tensor) are checked against the
    oracle adjoint over a few hundred steps with K = 64, i.e. several fused
    segments, while every plate is split over several CTAs;
  * at the full length the gradient is checked through properties that hold
    at any size (the fused sweep equals separate launches bit for bit, and
    the result does not depend on the checkpoint interval)."""
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import numpy as np

import oracle
from paper_2505_05940_gb300 import modal, physics, workloads as W

from test_gpu_parity import GTOL, TOL, classes_of, oracle_instance, rel, to_plan

SAMPLE = 5          # the plate the oracle checks over the whole run
GRAD_SAMPLES = (5, 50)   # plates whose gradients the oracle adjoint checks


@pytest.fixture(scope="module")
def batch():
    _, inits = W.adjoint_plates(seed=0, n_inst=64, steps=22050)
    prep = [physics.prepare(i, inits.fs, inits.steps) for i in inits.instances]
    ois = {}
    rng = np.random.default_rng(11)
    for j in GRAD_SAMPLES:
        oi = oracle_instance(inits.instances[j], inits.fs, inits.steps)
        d = to_plan(oi, inits.fs)
        # direction tensor for <dL/dH, dH>: symmetric, on the class pattern
        fc, kc = classes_of(oi)
        R = rng.normal(size=oi.H.shape)
        d["dH"] = ((R + R.transpose(0, 2, 1)) *
                   ((fc[:, None] ^ fc[None, :])[None] == kc[:, None, None])).astype(np.float32)
        prep[j] = d
        ois[j] = oi
    return prep, ois[SAMPLE], inits, ois


def test_full_size_forward_sampled_plate(batch):
    prep, oi, inits, _ = batch
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
    prep, _, inits, _ = batch
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


def test_batch_gradients_against_oracle_adjoint(batch):
    """The benchmark batch, 400 steps with K = 64 (fused sweep over six
    segments and a partial one), plates split over several CTAs: the sampled
    plates' gradients against the FP64 oracle adjoint."""
    import concurrent.futures as cf

    prep, _, inits, ois = batch
    steps, K = 400, 64
    sim = modal.Simulator(prep)
    assert sim.plan.tiles()["ctas"] >= 3 * len(prep) // 2   # plates shared by CTAs
    rng = np.random.default_rng(3)
    ybar = rng.normal(size=(len(prep), steps))
    r = sim.simulate(steps, K=K)
    g = sim.grad(steps, torch.tensor(ybar, dtype=torch.float32, device="cuda"), K, r["ckpt"],
                 want_status=True)
    torch.cuda.synchronize()
    assert (g["status"].cpu().numpy() == 0).all()
    got = {k: v.cpu().numpy() for k, v in g.items()}
    off = sim.plan.mode_offset
    koff = np.concatenate([[0], np.cumsum(sim.plan.n_stress)])
    T = 1.0 / inits.fs
    yb64 = ybar.astype(np.float32).astype(np.float64)
    with cf.ThreadPoolExecutor(max_workers=len(ois)) as ex:
        adjs = dict(zip(ois, ex.map(lambda j: oracle.adjoint(ois[j], yb64[j], steps=steps,
                                                            want_dH=True), ois)))
    for j, oi in ois.items():
        adj = adjs[j]
        dw2, dgm = oracle.coefficient_grads(oi, adj, T)
        sl = slice(off[j], off[j] + oi.N)
        dH = prep[j]["dH"].astype(np.float64)
        checks = [("d_omega2", got["d_omega2"][sl], dw2), ("d_gamma", got["d_gamma"][sl], dgm),
                  ("d_b", got["d_b"][sl], adj["db"]), ("d_c", got["d_c"][sl], adj["dc"]),
                  ("d_kappa", got["d_kappa"][koff[j]:koff[j + 1]], adj["dkappa"]),
                  ("d_dir", got["d_dir"][j:j + 1], np.array([np.sum(adj["dH"] * dH)]))]
        for name, a, ref in checks:
            e = rel(a, ref)
            assert e <= GTOL, (j, name, e)
