"""GPU parity at the edges of the batched workload: the largest mode count on
the tension kernel, a ragged batch split over two plans, and the whole
512-instance batched workload against the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle
from oracle import coupling_oracle as CO
from oracle import physics_oracle as PO
from paper_2505_05940_gb300 import modal, workloads as W

from test_gpu_parity import TOL, check_parity, oracle_instance, rel, run_gpu


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


def _group_coupling(wl):
    """Oracle coupling for the batched workload: one oracle H per aspect group,
    computed at the group's largest mode counts.  Plates of one aspect share
    Lx and Ly (the area is fixed), so a plate's modes (ascending eigenvalue)
    and its lowest Airy modes are prefixes of the group's, and its H is the
    leading block of the group's H; the prefix property of the labels is
    asserted for every plate."""
    groups = {}
    for inst in wl.instances:
        if inst.kind == "plate":
            key = float(inst.aspect)
            n, m = groups.get(key, (0, 0))
            groups[key] = (max(n, inst.n_phi), max(m, inst.n_psi))
    cache = {}

    def coupling(inst, labels, n_psi):
        key = float(inst.aspect)
        if key not in cache:
            n, m = groups[key]
            glabels, _ = PO.rect_modes(inst, n)
            H, zeta4 = CO.coupling_H(inst, glabels, m)
            cache[key] = (glabels, H, zeta4)
        glabels, H, zeta4 = cache[key]
        N = len(labels)
        assert np.array_equal(glabels[:N], labels)
        return H[:n_psi, :N, :N], zeta4[:n_psi]

    return coupling


@pytest.fixture(scope="module")
def batched512():
    """The whole batched workload (512 seeded plates and membranes, N_phi
    log-uniform in [20, 400], aspects on the shared grid, varied thickness) at
    2 205 steps, with the FP64 oracle's audio and final state of every
    instance (thread pool, one instance per task)."""
    import concurrent.futures as cf
    import os

    wl = W.batched_ragged(seed=0, n_inst=512, steps=2205)
    cp = _group_coupling(wl)
    ois = []
    for inst in wl.instances:
        oi = PO.build_instance(inst, wl.fs, wl.steps, coupling=cp if inst.kind == "plate" else None)
        if oi.H is not None:
            oi.H = oi.H.astype(np.float32).astype(np.float64)
        ois.append(oi)
    assert len(ois) == 512 and {o.kind for o in ois} == {"plate", "membrane"}
    assert max(o.N for o in ois) >= 390
    order = sorted(range(len(ois)), key=lambda i: -(ois[i].M * ois[i].N ** 2 + ois[i].N))
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        refs = dict(zip(order, ex.map(lambda i: oracle.forward(ois[i], steps=wl.steps), order)))
    return wl, ois, refs


def _check_all(ois, refs, audio, qend, label):
    errs = [(rel(audio[i], refs[i]["y"]), rel(qend[i], refs[i]["qN"]), i) for i in range(len(ois))]
    for ea, eq, i in sorted(errs, reverse=True)[:5]:
        print(f"{label}: instance {i} ({ois[i].kind} {ois[i].N}x{ois[i].M}): "
              f"audio {ea:.2e} state {eq:.2e}")
    for ea, eq, i in errs:
        assert ea <= TOL and eq <= TOL, (label, i, ois[i].kind, ois[i].N, ois[i].M, ea, eq)


def test_batched_workload_all_512(batched512):
    """Every instance of the batched workload in one plan (per-instance
    coupling copies, FP32 CUDA-core contraction) against the oracle."""
    wl, ois, refs = batched512
    audio, qend, status, sim = run_gpu(ois, wl.fs, wl.steps)
    assert (status == 0).all(), status
    assert sim.plan.tiles()["ctas"] >= 100
    _check_all(ois, refs, audio, qend, "per-instance")


def test_batched_workload_all_512_grouped(batched512):
    """The same 512 instances with the plates of each aspect stepped as one
    group on the tensor cores (split-TF32 tcgen05 GEMM per stress mode and
    step) against the oracle."""
    wl, ois, refs = batched512
    from test_gpu_parity import to_plan
    aspects = sorted({float(i.aspect) for i in wl.instances if i.kind == "plate"})
    plans = []
    for inst, oi in zip(wl.instances, ois):
        d = to_plan(oi, wl.fs)
        if oi.kind == "plate":
            d["geom_group"] = 1 + aspects.index(float(inst.aspect))
        plans.append(d)
    sim = modal.Simulator(plans)
    r = sim.simulate(wl.steps, want_state=True, want_status=True)
    torch.cuda.synchronize()
    assert (r["status"].cpu().numpy() == 0).all()
    off = sim.plan.mode_offset
    q = r["q_end"].cpu().numpy()
    qend = [q[off[i]:off[i] + o.N] for i, o in enumerate(ois)]
    _check_all(ois, refs, r["audio"].cpu().numpy(), qend, "grouped")
