"""GPU parity at the edges of the batched workload: the largest mode count on
the tension kernel, and a ragged batch split over two plans."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2505_05940_gb300 import workloads as W

from test_gpu_parity import check_parity, oracle_instance, rel, run_gpu


def test_membrane_400_modes():
    """The largest mode count of the batched workload on the tension kernel
    (up to 16 modes per lane, 13 used)."""
    wl = W.tiny_random(400, "membrane", 400, steps=3000)
    oi = oracle_instance(wl.instances[0], wl.fs, wl.steps)
    assert oi.N == 400
    check_parity([oi], wl.fs, wl.steps)


def test_batch_split_and_concatenate():
    """Instances are independent: a ragged batch run whole and as two separate
    plans gives each instance's audio to FP32 summation order (the work
    split over CTAs differs between the plans)."""
    fs, steps = 44100.0, 1200
    insts = [W.tiny_random(60, "plate", 48, 12, steps=steps).instances[0],
             W.tiny_random(61, "string", 35, steps=steps).instances[0],
             W.tiny_random(62, "plate", 30, 7, steps=steps).instances[0],
             W.tiny_random(63, "membrane", 50, steps=steps).instances[0],
             W.tiny_random(64, "plate", 64, 16, steps=steps).instances[0],
             W.tiny_random(65, "string", 20, steps=steps).instances[0]]
    for i in (0, 2, 4):
        insts[i].F0 = 200.0
    ois = [oracle_instance(i, fs, steps) for i in insts]
    whole, _, st, _ = run_gpu(ois, fs, steps)
    first, _, st1, _ = run_gpu(ois[:3], fs, steps)
    second, _, st2, _ = run_gpu(ois[3:], fs, steps)
    assert (st == 0).all() and (st1 == 0).all() and (st2 == 0).all()
    halves = np.concatenate([first, second], 0)
    for i in range(len(ois)):
        assert rel(halves[i], whole[i]) <= 1e-6, (i, rel(halves[i], whole[i]))


def test_batched_workload_seeded_subset():
    """The batched workload's own draws (first 24 instances with N_phi <= 120:
    plates and membranes of uneven sizes, aspects on the shared grid, varied
    thickness) in one plan, 2 205 steps, each against the oracle."""
    wl = W.batched_ragged(seed=0, n_inst=512, steps=2205)
    sel = [i for i, inst in enumerate(wl.instances) if inst.n_phi <= 120][:24]
    ois = [oracle_instance(wl.instances[i], wl.fs, wl.steps) for i in sel]
    assert {o.kind for o in ois} == {"plate", "membrane"}
    check_parity(ois, wl.fs, wl.steps)
