"""Grouped plates on the tensor cores against the FP64 oracle.

Plates of one geometry (simply supported rectangles of the same area and
aspect ratio) share their modes: a plate with fewer modes has a prefix of the
largest member's (Sec. 3, Eq. 2), so its coupling tensor (Eq. 10) is the
leading block of the largest member's.  The grouped path steps them together,
with H^k [q_1 ... q_B] as one split-TF32 tcgen05 GEMM per stress mode and
step.  Each plate is compared with the oracle (the same tolerance as the FP32
path: 1e-5 relative L2 on audio and final state) and with the per-instance
FP32 CUDA-core path."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import copy

import oracle
from oracle import coupling_oracle as CO
from oracle import physics_oracle as PO
from paper_2505_05940_gb300 import modal, workloads as W

from test_gpu_parity import TOL, classes_of, rel, to_plan


def _group(insts, fs, steps):
    """Oracle instances of plates sharing one aspect: the oracle's H at the
    largest member's modes, sliced for every member (prefix checked)."""
    big = max(insts, key=lambda i: (i.n_phi, i.n_psi))
    labels, _ = PO.rect_modes(big, big.n_phi)
    H, zeta4 = CO.coupling_H(big, labels, big.n_psi)

    def cp(inst, lab, m):
        assert np.array_equal(labels[:len(lab)], lab)
        return H[:m, :len(lab), :len(lab)], zeta4[:m]

    ois = []
    for inst in insts:
        oi = PO.build_instance(inst, fs, steps, coupling=cp)
        oi.H = oi.H.astype(np.float32).astype(np.float64)
        ois.append(oi)
    return ois


def _plans(ois, fs, group_id):
    plans = []
    for oi in ois:
        d = to_plan(oi, fs)
        d["geom_group"] = group_id
        plans.append(d)
    return plans


def _run(plans, steps, **opts):
    sim = modal.Simulator(plans, **opts)
    sim.plan.set_profiling(True)
    r = sim.simulate(steps, want_state=True, want_status=True)
    torch.cuda.synchronize()
    off = sim.plan.mode_offset
    q = r["q_end"].cpu().numpy()
    return (r["audio"].cpu().numpy(), [q[off[i]:off[i] + len(p["omega2"])]
                                       for i, p in enumerate(plans)],
            r["status"].cpu().numpy(), sim)


def test_grouped_small_group_against_oracle():
    """Three plates of one aspect (48 x 12, 40 x 10, 30 x 6 modes) with
    different stiffness, tension and strike points, one kernel group of
    three (padded to 16 columns)."""
    fs, steps = 44100.0, 1500
    base = W.tiny_random(71, "plate", 48, 12, steps=steps).instances[0]
    base.F0 = 300.0
    insts = [base]
    rng = np.random.default_rng(5)
    for n, m in ((40, 10), (30, 6)):
        x = copy.deepcopy(base)
        x.n_phi, x.n_psi = n, m
        x.D *= float(rng.uniform(0.7, 1.4))
        x.T0 *= float(rng.uniform(0.5, 2.0))
        x.strike = (float(rng.uniform(0.1, 0.9)), float(rng.uniform(0.1, 0.9)))
        insts.append(x)
    ois = _group(insts, fs, steps)
    plans = _plans(ois, fs, 1)
    audio, qend, status, sim = _run(plans, steps)
    assert (status == 0).all(), status
    # the grouped kernel ran, over the nonzero class blocks of the shared tensor
    assert sim.plan.kernel_stats(5)[0] == 1 and sim.plan.kernel_stats(0)[0] == 0
    fc, kc = classes_of(ois[0])
    blocks = int(np.sum((fc[:, None] ^ fc[None, :])[None] == kc[:, None, None]))
    assert sim.plan.group_work()[0] == 4 * blocks
    ref_cc, qref_cc, _, csim = _run(plans, steps, group_engine="off")
    # per-instance copies: the streaming kernel or, for a few small plates,
    # the cluster-resident one
    assert csim.plan.kernel_stats(5)[0] == 0
    assert csim.plan.kernel_stats(0)[0] + csim.plan.kernel_stats(6)[0] == 1
    for i, oi in enumerate(ois):
        ref = oracle.forward(oi, steps=steps)
        ea, eq = rel(audio[i], ref["y"]), rel(qend[i], ref["qN"])
        assert ea <= TOL and eq <= TOL, (i, ea, eq)
        # the FP32 CUDA-core path on per-instance copies agrees to about 1e-7
        assert rel(audio[i], ref_cc[i]) <= 1e-6, (i, rel(audio[i], ref_cc[i]))


def test_grouped_plans_reject_gradients_and_checkpoints():
    fs, steps = 44100.0, 64
    inst = W.tiny_random(72, "plate", 24, 6, steps=steps).instances[0]
    ois = _group([inst], fs, steps)
    sim = modal.Simulator(_plans(ois, fs, 3))
    from paper_2505_05940_gb300 import _native
    with pytest.raises(_native.MdxError):
        sim.simulate(steps, K=16)
