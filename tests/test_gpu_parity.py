"""GPU parity: the CUDA kernels (through the C ABI) against the FP64 oracle.

Tolerance (from the FP32 error analysis of the difference-form update with a
compensated state): relative L2 error <= 1e-5 on output audio and final
state; gradients <= 1e-4 relative (normwise per gradient vector) against the
oracle adjoint.  Inputs are the oracle's own FP64 coefficients with the
coupling tensor rounded to FP32, the precision the library takes it in."""

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

TOL = 1e-5
GTOL = 1e-4


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def oracle_instance(inst, fs, steps, coupling=True):
    cp = CO.oracle_coupling if (inst.kind == "plate" and coupling) else None
    oi = PO.build_instance(inst, fs, steps, coupling=cp)
    if oi.H is not None:
        oi.H = oi.H.astype(np.float32).astype(np.float64)   # the FP32 input both sides see
    return oi


def classes_of(oi):
    """Symmetry classes of the oracle's modes: transverse from (m, n), Airy
    from the position of the largest entry of each H^k."""
    m, n = oi.labels[:, 0], oi.labels[:, 1]
    fc = (2 * ((m + 1) % 2) + ((n + 1) % 2)).astype(np.int32)
    kc = []
    for Hk in oi.H:
        i, j = np.unravel_index(np.argmax(np.abs(Hk)), Hk.shape)
        kc.append(fc[i] ^ fc[j])
    return fc, np.array(kc, dtype=np.int32)


def to_plan(oi, fs, layout="classes"):
    d = dict(kind="plate" if oi.kind == "plate" else "tension", omega2=oi.omega2,
             gamma=oi.gamma, b=oi.b, c=oi.c, dt=1.0 / fs, lam=oi.lam, tau=oi.taup,
             e=oi.e, q0=oi.q0, qm1=oi.qm1)
    if oi.kind == "plate" and oi.H is not None:
        d["H"] = oi.H.astype(np.float32)
        d["kappa"] = oi.kappa
        if layout == "classes":
            d["phi_class"], d["psi_class"] = classes_of(oi)
    return d


def run_gpu(ois, fs, steps, layout="classes", force_profile=False, **opts):
    sim = modal.Simulator([to_plan(o, fs, layout) for o in ois], **opts)
    if force_profile:
        sim.plan.set_profiling(True)
    r = sim.simulate(steps, want_state=True, want_status=True)
    torch.cuda.synchronize()
    off = sim.plan.mode_offset
    q_end = r["q_end"].cpu().numpy()
    return (r["audio"].cpu().numpy(), [q_end[off[i]:off[i] + o.N] for i, o in enumerate(ois)],
            r["status"].cpu().numpy(), sim)


def check_parity(ois, fs, steps, tol=TOL, layout="classes", **opts):
    audio, qend, status, _ = run_gpu(ois, fs, steps, layout, **opts)
    assert (status == 0).all(), status
    for i, oi in enumerate(ois):
        ref = oracle.forward(oi, steps=steps)
        assert rel(audio[i], ref["y"]) <= tol, (i, rel(audio[i], ref["y"]))
        assert rel(qend[i], ref["qN"]) <= tol, (i, rel(qend[i], ref["qN"]))
    return audio


def test_string40_full_length():
    wl = W.string_40()
    oi = oracle_instance(wl.instances[0], wl.fs, wl.steps)
    check_parity([oi], wl.fs, wl.steps)


def test_plate100x30_full_length():
    wl = W.plate_100x30()
    oi = oracle_instance(wl.instances[0], wl.fs, wl.steps)
    check_parity([oi], wl.fs, wl.steps)


@pytest.mark.parametrize("n", [1, 31, 32, 33, 100])
def test_string_sizes(n):
    wl = W.tiny_random(n, "string", n, steps=1500, fs=48000.0)
    check_parity([oracle_instance(wl.instances[0], wl.fs, wl.steps)], wl.fs, wl.steps)


@pytest.mark.parametrize("layout", ["dense", "classes"])
@pytest.mark.parametrize("n,m", [(4, 1), (31, 3), (33, 8), (64, 16), (257, 9)])
def test_plate_sizes(n, m, layout):
    wl = W.tiny_random(7 + n, "plate", n, m, steps=1200)
    wl.instances[0].F0 = 200.0
    check_parity([oracle_instance(wl.instances[0], wl.fs, wl.steps)], wl.fs, wl.steps,
                 layout=layout)


def test_class_layout_equals_dense_layout():
    """Streaming only the nonzero symmetry-class blocks gives the dense
    layout's results up to FP32 summation order."""
    wl = W.tiny_random(77, "plate", 120, 30, steps=2000)
    wl.instances[0].F0 = 300.0
    oi = oracle_instance(wl.instances[0], wl.fs, wl.steps)
    a, qa, _, _ = run_gpu([oi], wl.fs, wl.steps, layout="dense")
    b, qb, _, sim = run_gpu([oi], wl.fs, wl.steps, layout="classes", force_split=3)
    assert sim.plan.tiles()["ctas"] >= 3
    assert rel(b, a) <= 1e-6 and rel(qb[0], qa[0]) <= 1e-6


def test_plate_split_over_ctas_matches_single_and_oracle():
    wl = W.tiny_random(21, "plate", 64, 16, steps=1500)
    wl.instances[0].F0 = 300.0
    oi = oracle_instance(wl.instances[0], wl.fs, wl.steps)
    a1 = check_parity([oi], wl.fs, wl.steps)
    a4 = check_parity([oi], wl.fs, wl.steps, force_split=4)
    assert rel(a4, a1) <= 1e-6


def test_mixed_ragged_batch():
    """Strings, membranes, nonlinear and linear plates of uneven sizes in one plan."""
    fs, steps = 44100.0, 1000
    insts = [W.tiny_random(1, "string", 40, steps=steps).instances[0],
             W.tiny_random(2, "membrane", 77, steps=steps).instances[0],
             W.tiny_random(3, "plate", 50, 12, steps=steps).instances[0],
             W.tiny_random(4, "plate", 23, 5, steps=steps).instances[0],
             W.tiny_random(5, "membrane", 3, steps=steps).instances[0]]
    lin = W.tiny_random(6, "plate", 30, 0, steps=steps).instances[0]
    lin.nonlinear = False
    insts.append(lin)
    ois = [oracle_instance(i, fs, steps) for i in insts]
    check_parity(ois, fs, steps, force_split=2)


def test_resume_equals_single_run():
    wl = W.tiny_random(9, "plate", 40, 10, steps=2000)
    oi = oracle_instance(wl.instances[0], wl.fs, wl.steps)
    sim = modal.Simulator([to_plan(oi, wl.fs)])
    full = sim.simulate(2000, want_state=True)
    a = sim.simulate(1000, want_state=True)
    exc2 = sim.exc[:, 1000:2000].contiguous()
    b = sim.simulate(1000, q0=a["q_end"], qm1=a["qm1_end"], want_state=True, exc=exc2)
    joined = torch.cat([a["audio"], b["audio"]], 1).cpu().numpy()
    assert rel(joined, full["audio"].cpu().numpy()) <= 1e-6
    assert rel(b["q_end"].cpu().numpy(), full["q_end"].cpu().numpy()) <= 1e-6


def _grad_case(kind, seed, steps):
    if kind == "string":
        wl = W.tiny_random(seed, "string", 12, steps=steps, fs=48000.0)
    else:
        wl = W.tiny_random(seed, "plate", 24, 6, steps=steps)
        wl.instances[0].F0 = 300.0
    oi = oracle_instance(wl.instances[0], wl.fs, wl.steps)
    return oi, wl.fs


@pytest.mark.parametrize("kind", ["string", "plate-dense", "plate-classes"])
def test_gradients_match_oracle_adjoint(kind):
    steps = 1500
    layout = kind.split("-")[1] if "-" in kind else "dense"
    kind = kind.split("-")[0]
    oi, fs = _grad_case(kind, 31, steps)
    rng = np.random.default_rng(1)
    ybar = rng.normal(size=steps)
    # direction tensor for <dL/dH, dH>: a fixed symmetric random tensor
    # (restricted to the symmetry-class pattern for the class layout)
    dH = None
    d = to_plan(oi, fs, layout)
    if kind == "plate":
        R = rng.normal(size=oi.H.shape)
        dH = (R + R.transpose(0, 2, 1))
        if layout == "classes":
            fc, kc = classes_of(oi)
            dH = dH * ((fc[:, None] ^ fc[None, :])[None] == kc[:, None, None])
        dH = dH.astype(np.float32)
        d["dH"] = dH
    sim = modal.Simulator([d])
    K = 256
    r = sim.simulate(steps, K=K)
    g = sim.grad(steps, torch.tensor(ybar[None, :], dtype=torch.float32, device="cuda"), K,
                 r["ckpt"], want_status=True, want_dH=(kind == "plate"))
    torch.cuda.synchronize()
    assert int(g["status"][0]) == 0
    adj = oracle.adjoint(oi, ybar, want_dH=(kind == "plate"))
    T = 1.0 / fs
    dw2, dgm = oracle.coefficient_grads(oi, adj, T)
    got = {k: v.cpu().numpy() for k, v in g.items()}
    checks = [("d_omega2", dw2), ("d_gamma", dgm), ("d_b", adj["db"]), ("d_c", adj["dc"]),
              ("d_q0", adj["dq0"]), ("d_qm1", adj["dqm1"])]
    if kind == "string":
        checks.append(("d_tau", np.array([adj["dtau"]])))
    else:
        checks.append(("d_kappa", adj["dkappa"]))
        checks.append(("d_dir", np.array([np.sum(adj["dH"] * dH.astype(np.float64))])))
    for name, ref in checks:
        if kind == "plate" and name in ("d_q0", "d_qm1"):
            pass   # a struck plate starts at rest: still a valid comparison
        e = rel(got[name][:len(ref)], ref)
        assert e <= GTOL, (name, e)
    if kind == "plate":
        # full dL/dH (symmetrised); the class layout gives it on the class pattern
        dHg = got["d_H"][:oi.M * oi.N * oi.N].reshape(oi.M, oi.N, oi.N)
        ref = adj["dH"]
        if layout == "classes":
            fc, kc = classes_of(oi)
            mask = (fc[:, None] ^ fc[None, :])[None] == kc[:, None, None]
            assert np.all(dHg[~mask] == 0.0)
            ref = np.where(mask, ref, 0.0)
        assert rel(dHg, ref) <= GTOL, rel(dHg, ref)


def test_direction_contraction_on_tensor_cores():
    """The aspect-direction contraction <dL/dH, dH> on the tensor cores
    (split-TF32 GEMM over each segment's states) against the oracle adjoint,
    and against the CUDA-core kernel (debug flag 8), on a 90 x 70 plate whose
    stress classes hold 14-20 modes and row classes 19-25 modes (several
    16 x 16 chunks of the GEMM's columns) over segments of 256 steps and a
    ragged last one.  The other gradients do not depend on the contraction
    and stay bitwise equal."""
    steps, K = 700, 256
    wl = W.tiny_random(41, "plate", 90, 70, steps=steps)
    wl.instances[0].F0 = 300.0
    oi = oracle_instance(wl.instances[0], wl.fs, wl.steps)
    rng = np.random.default_rng(1)
    ybar = rng.normal(size=steps)
    fc, kc = classes_of(oi)
    R = rng.normal(size=oi.H.shape)
    dH = ((R + R.transpose(0, 2, 1)) * ((fc[:, None] ^ fc[None, :])[None] == kc[:, None, None]))
    dH = dH.astype(np.float32)
    d = to_plan(oi, wl.fs)
    d["dH"] = dH
    yb = torch.tensor(ybar[None, :], dtype=torch.float32, device="cuda")
    outs = []
    for flags in (0, 8):
        sim = modal.Simulator([d], debug_flags=flags)
        r = sim.simulate(steps, K=K)
        g = sim.grad(steps, yb, K, r["ckpt"], want_status=True)
        torch.cuda.synchronize()
        assert int(g["status"][0]) == 0
        outs.append(g)
    adj = oracle.adjoint(oi, ybar, want_dH=True)
    ref = float(np.sum(adj["dH"] * dH.astype(np.float64)))
    tc, cc = float(outs[0]["d_dir"][0]), float(outs[1]["d_dir"][0])
    assert abs(tc - ref) <= GTOL * abs(ref), (tc, ref)
    assert abs(tc - cc) <= 1e-5 * abs(cc), (tc, cc)
    for k in ("d_omega2", "d_gamma", "d_b", "d_c", "d_kappa"):
        assert torch.equal(outs[0][k], outs[1][k]), k


def test_cluster_resident_forward_matches_oracle_and_streaming_kernel():
    """A checkpoint-free forward pass of a few small plates runs with each
    plate's coupling rows in the registers of one thread-block cluster (stats
    class 6).  A 100 x 30 plate, a 48 x 12 and a 20 x 4 plate (one shape for
    all: clusters of 8 CTAs with 4 stress-mode slots each, so the small plates
    leave slots and CTAs empty) and a string in one plan, against the oracle
    and against the streaming kernel (debug flag 16), over 3 000 steps
    (excitation staged in blocks of 256 steps)."""
    fs, steps = 44100.0, 3000
    insts = [W.tiny_random(60, "plate", 100, 30, steps=steps).instances[0],
             W.tiny_random(61, "plate", 48, 12, steps=steps).instances[0],
             W.tiny_random(62, "plate", 20, 4, steps=steps).instances[0],
             W.tiny_random(63, "string", 30, steps=steps).instances[0]]
    for x in insts[:3]:
        x.F0 = 300.0
    ois = [oracle_instance(i, fs, steps) for i in insts]
    outs = []
    for flags in (0, 16):
        audio, qend, status, sim = run_gpu(ois, fs, steps, debug_flags=flags, force_profile=True)
        assert (status == 0).all(), status
        outs.append((audio, qend))
        if flags == 0:
            assert sim.plan.kernel_stats(6)[0] == 1 and sim.plan.kernel_stats(0)[0] == 0
        else:
            assert sim.plan.kernel_stats(6)[0] == 0 and sim.plan.kernel_stats(0)[0] == 1
    for i, oi in enumerate(ois):
        ref = oracle.forward(oi, steps=steps)
        for audio, qend in outs:
            assert rel(audio[i], ref["y"]) <= TOL, (i, rel(audio[i], ref["y"]))
            assert rel(qend[i], ref["qN"]) <= TOL, (i, rel(qend[i], ref["qN"]))
        assert rel(outs[0][0][i], outs[1][0][i]) <= 5e-6


def test_direction_contraction_with_split_k():
    """Class blocks wider than the contraction's shared-memory K chunk (a
    260 x 64 plate: 61-71 columns per class against a 56-column chunk) are
    contracted in two K chunks with the dH operand restaged per tile; d_dir
    against the oracle adjoint and the CUDA-core kernel."""
    steps, K = 300, 256
    wl = W.tiny_random(71, "plate", 260, 64, steps=steps)
    wl.instances[0].F0 = 300.0
    oi = oracle_instance(wl.instances[0], wl.fs, wl.steps)
    rng = np.random.default_rng(1)
    ybar = rng.normal(size=steps)
    fc, kc = classes_of(oi)
    assert np.bincount(fc).max() > 64
    R = rng.normal(size=oi.H.shape)
    dH = ((R + R.transpose(0, 2, 1)) * ((fc[:, None] ^ fc[None, :])[None] == kc[:, None, None]))
    d = to_plan(oi, wl.fs)
    d["dH"] = dH.astype(np.float32)
    yb = torch.tensor(ybar[None, :], dtype=torch.float32, device="cuda")
    got = []
    for flags in (0, 8):
        sim = modal.Simulator([d], debug_flags=flags)
        r = sim.simulate(steps, K=K)
        g = sim.grad(steps, yb, K, r["ckpt"], want_status=True)
        torch.cuda.synchronize()
        assert int(g["status"][0]) == 0
        got.append(float(g["d_dir"][0]))
    adj = oracle.adjoint(oi, ybar, want_dH=True)
    ref = float(np.sum(adj["dH"] * d["dH"].astype(np.float64)))
    assert abs(got[0] - ref) <= GTOL * abs(ref), (got[0], ref)
    assert abs(got[0] - got[1]) <= 1e-5 * abs(got[1]), got


def test_cluster_resident_forward_with_64_wide_rows():
    """Plates whose symmetry-class blocks hold 33-64 modes keep 64-float rows in
    registers (a 180 x 24 plate: 16-CTA clusters of 2 stress-mode slots x 6
    warps); forward pass against the oracle."""
    fs, steps = 44100.0, 1500
    wl = W.tiny_random(64, "plate", 180, 24, steps=steps)
    wl.instances[0].F0 = 300.0
    oi = oracle_instance(wl.instances[0], fs, steps)
    fc, _ = classes_of(oi)
    assert 32 < np.bincount(fc).max() <= 64
    audio, qend, status, sim = run_gpu([oi], fs, steps, force_profile=True)
    assert (status == 0).all()
    assert sim.plan.kernel_stats(6)[0] == 1
    ref = oracle.forward(oi, steps=steps)
    assert rel(audio[0], ref["y"]) <= TOL, rel(audio[0], ref["y"])
    assert rel(qend[0], ref["qN"]) <= TOL


def test_two_live_plans_share_kernel_attributes():
    """Kernel attributes belong to the kernels, not to plans: a small plan
    created after a large one leaves the large one's launches intact (its
    16-CTA clusters and its larger direction-contraction shared memory), and
    the large plan's results are unchanged bit for bit."""
    fs, steps, K = 44100.0, 600, 256
    plans = []
    for seed, n, m in ((41, 90, 70), (8, 48, 12)):
        wl = W.tiny_random(seed, "plate", n, m, steps=steps)
        wl.instances[0].F0 = 300.0
        oi = oracle_instance(wl.instances[0], fs, steps)
        fc, kc = classes_of(oi)
        R = np.random.default_rng(seed).normal(size=oi.H.shape)
        d = to_plan(oi, fs)
        d["dH"] = ((R + R.transpose(0, 2, 1)) *
                   ((fc[:, None] ^ fc[None, :])[None] == kc[:, None, None])).astype(np.float32)
        plans.append(d)
    yb = torch.randn(1, steps, dtype=torch.float32, device="cuda")

    def run(sim):
        a = sim.simulate(steps)["audio"].clone()
        r = sim.simulate(steps, K=K)
        g = sim.grad(steps, yb, K, r["ckpt"], want_status=True)
        torch.cuda.synchronize()
        assert int(g["status"][0]) == 0
        return a, g["d_dir"].clone(), g["d_omega2"].clone()

    big = modal.Simulator([plans[0]])
    ref = run(big)
    small = modal.Simulator([plans[1]])
    run(small)
    again = run(big)
    for x, y in zip(ref, again):
        assert torch.equal(x, y)


def test_gradients_independent_of_checkpoint_interval():
    steps = 1000
    oi, fs = _grad_case("plate", 33, steps)
    sim = modal.Simulator([to_plan(oi, fs)])
    yb = torch.randn(1, steps, dtype=torch.float32, device="cuda")
    outs = []
    for K in (64, 1000, 333):
        r = sim.simulate(steps, K=K)
        outs.append(sim.grad(steps, yb, K, r["ckpt"]))
    for k in ("d_omega2", "d_gamma", "d_kappa", "d_q0"):
        for o in outs[1:]:
            assert torch.equal(outs[0][k], o[k]), k


@pytest.mark.parametrize("flags", [2, 4])
@pytest.mark.parametrize("force_split", [0, 3])
def test_fused_sweep_equals_separate_launches(force_split, flags):
    """The fused adjoint sweep (reverse of segment s and recompute of segment
    s-1 in one launch) gives bitwise the gradients of separate recompute and
    reverse launches (flags 2), and the plate kernel gives bitwise the same
    audio and gradients without its per-plate shared-memory caches of
    coefficients and gradient sums (flags 4, the path of plates too large for
    them), on a ragged batch with a partial last segment, a direction tensor,
    and plates shared by several CTAs."""
    fs, steps, K = 44100.0, 1100, 256
    insts = [W.tiny_random(50, "plate", 48, 12, steps=steps).instances[0],
             W.tiny_random(51, "string", 30, steps=steps).instances[0],
             W.tiny_random(52, "plate", 30, 7, steps=steps).instances[0],
             W.tiny_random(53, "membrane", 40, steps=steps).instances[0]]
    for i in (0, 2):
        insts[i].F0 = 300.0
    ois = [oracle_instance(i, fs, steps) for i in insts]
    rng = np.random.default_rng(7)
    plans = []
    for o in ois:
        d = to_plan(o, fs)
        if o.kind == "plate":
            R = rng.normal(size=o.H.shape)
            fc, kc = classes_of(o)
            dH = (R + R.transpose(0, 2, 1)) * ((fc[:, None] ^ fc[None, :])[None] == kc[:, None, None])
            d["dH"] = dH.astype(np.float32)
        plans.append(d)
    yb = torch.randn(len(ois), steps, dtype=torch.float32, device="cuda")
    outs = []
    for f in (0, flags):
        sim = modal.Simulator(plans, force_split=force_split, debug_flags=f)
        r = sim.simulate(steps, K=K)
        g = sim.grad(steps, yb, K, r["ckpt"], want_status=True)
        torch.cuda.synchronize()
        assert (g["status"] == 0).all()
        g["audio"] = r["audio"]
        outs.append(g)
    for k in ("audio", "d_omega2", "d_gamma", "d_b", "d_c", "d_q0", "d_qm1", "d_tau", "d_kappa",
              "d_dir"):
        assert torch.equal(outs[0][k], outs[1][k]), k


def test_nonfinite_state_is_reported():
    wl = W.tiny_random(12, "plate", 20, 4, steps=400)
    oi = oracle_instance(wl.instances[0], wl.fs, wl.steps)
    oi.e = oi.e * 1e30
    _, _, status, _ = run_gpu([oi], wl.fs, wl.steps)
    assert status[0] == 3


def test_bounded_wait_reports_timeout_and_context_survives():
    """A contributor withholds its arrival (debug flag): the others' bounded
    waits run out, the call reports MDX_ERR_TIMEOUT, nothing hangs, and the
    next plan on the same device still gives oracle-exact results."""
    wl = W.tiny_random(13, "plate", 32, 8, steps=300)
    oi = oracle_instance(wl.instances[0], wl.fs, wl.steps)
    _, _, status, _ = run_gpu([oi], wl.fs, wl.steps, force_split=2, wait_limit=20000,
                              debug_flags=1)
    assert status[0] == 4
    check_parity([oi], wl.fs, wl.steps, force_split=2)


def test_cuda_graph_replay_matches_direct_calls():
    """A ragged batch captured once in a CUDA graph (forward + adjoint) and
    replayed gives bit-identical audio and gradients to direct calls."""
    fs, steps = 44100.0, 600
    insts = [W.tiny_random(40, "plate", 48, 12, steps=steps).instances[0],
             W.tiny_random(41, "membrane", 60, steps=steps).instances[0],
             W.tiny_random(42, "plate", 30, 7, steps=steps).instances[0]]
    ois = [oracle_instance(i, fs, steps) for i in insts]
    sim = modal.Simulator([to_plan(o, fs) for o in ois])
    K = 128
    run = sim.capture(steps, K=K, with_grad=True)
    yb = torch.randn(len(ois), steps, device="cuda")
    run.d_audio.copy_(yb)
    for _ in range(2):
        audio = run.replay().clone()
    torch.cuda.synchronize()
    direct = sim.simulate(steps, K=K)
    g = sim.grad(steps, yb, K, direct["ckpt"])
    torch.cuda.synchronize()
    assert torch.equal(audio, direct["audio"])
    for k in ("d_omega2", "d_gamma", "d_kappa"):
        assert torch.equal(run.grads[k][:g[k].numel()], g[k]), k


def test_autotuner_picks_a_fitting_stage_and_keeps_parity(tmp_path):
    from paper_2505_05940_gb300 import autotune
    wl = W.tiny_random(50, "plate", 96, 24, steps=500)
    wl.instances[0].F0 = 300.0
    oi = oracle_instance(wl.instances[0], wl.fs, wl.steps)
    sim = modal.Simulator([to_plan(oi, wl.fs)])
    res = autotune.tune(sim, steps=64, cache_path=str(tmp_path / "tune.json"))
    assert res["stage_bytes"] in autotune.STAGE_CANDIDATES and not res["cached"]
    assert sim.plan.tiles()["stage_bytes"] == res["stage_bytes"]
    again = autotune.tune(sim, steps=64, cache_path=str(tmp_path / "tune.json"))
    assert again["cached"] and again["stage_bytes"] == res["stage_bytes"]
    r = sim.simulate(wl.steps)
    torch.cuda.synchronize()
    ref = oracle.forward(oi)["y"]
    assert rel(r["audio"].cpu().numpy()[0], ref) <= TOL


def test_set_coupling_equals_a_fresh_plan():
    """mdx_plan_set_coupling repacks a new H into a live plan (dense and class
    layouts): the next run equals a plan created with that H."""
    fs, steps = 44100.0, 600
    oi, _ = _grad_case("plate", 41, steps)
    rng = np.random.default_rng(9)
    for layout in ("dense", "classes"):
        d = to_plan(oi, fs, layout)
        sim = modal.Simulator([d])
        H2 = oi.H * (1.0 + 0.05 * rng.standard_normal(oi.H.shape))
        H2 = 0.5 * (H2 + H2.transpose(0, 2, 1))
        if layout == "classes":
            fc, kc = classes_of(oi)
            H2 = H2 * ((fc[:, None] ^ fc[None, :])[None] == kc[:, None, None])
        sim.plan.set_coupling(0, H2.astype(np.float32))
        a = sim.simulate(steps)["audio"].cpu().numpy()
        d2 = dict(d)
        d2["H"] = H2.astype(np.float32)
        b = modal.Simulator([d2]).simulate(steps)["audio"].cpu().numpy()
        assert np.array_equal(a, b), layout
