"""The no-allocation entry point against the planned path.

mdx_simulate_strings_noalloc serves callers that may not allocate device
memory (a real-time audio callback, where cudaMalloc can block and
synchronise the device; a plug-in whose host owns every device buffer).  It
keeps its scratch in a fixed block inside the library.  These tests call it
through the C ABI and compare it with mdx_plan_create + mdx_simulate (scheme
MDX_SCHEME_SV) on the same inputs.  Both run the same kernel on the same FP32
coefficients, so the results must be identical bit for bit:
  * twice in a row (the second call reuses a block that still holds the
    first call's contents);
  * with the optional inputs left out (zero initial state, no excitation) and
    with the audio left out while the final state is requested;
  * at the size limit, where the state region ends a few hundred bytes
    before the end of the 1 MiB block, and one mode beyond it, which must be
    refused.
The file sits on its own and is collected last."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import physics_oracle as PO
from paper_2505_05940_gb300 import _native as N
from paper_2505_05940_gb300 import modal, workloads as W

BLOCK = 1 << 20


def _align16(x):
    return (x + 15) // 16 * 16


def max_modes(n_inst):
    """The documented limit of include/mdx.h."""
    return (BLOCK - _align16(120 * n_inst) - _align16(4 * n_inst) - 192) // 48


def _instances(steps):
    insts = [W.tiny_random(1, "string", 40, steps=steps).instances[0],
             W.tiny_random(2, "membrane", 77, steps=steps).instances[0],
             W.tiny_random(3, "string", 5, steps=steps).instances[0],
             W.tiny_random(4, "membrane", 130, steps=steps).instances[0]]
    out = []
    for inst in insts:
        oi = PO.build_instance(inst, 44100.0, steps)
        out.append(dict(kind="tension", omega2=oi.omega2, gamma=oi.gamma, b=oi.b, c=oi.c,
                        dt=1.0 / 44100.0, lam=oi.lam, tau=oi.taup, e=oi.e, q0=oi.q0,
                        qm1=oi.qm1))
    return out


def _synthetic(n_modes, seed, steps, fs=44100.0):
    """A string-like instance with n_modes modes, omega T <= pi / 2."""
    rng = np.random.default_rng(seed)
    f = np.sort(rng.uniform(40.0, 0.25 * fs, n_modes))
    w2 = (2 * np.pi * f) ** 2
    e = np.zeros(steps)
    e[:8] = rng.normal(size=8)
    return dict(kind="tension", omega2=w2, gamma=1.0 + 3e-6 * w2,
                b=rng.normal(size=n_modes) * 1e-3, c=rng.normal(size=n_modes),
                dt=1.0 / fs, lam=(np.pi * np.arange(1, n_modes + 1)) ** 2, tau=1e-6, e=e,
                q0=rng.normal(size=n_modes) * 1e-6, qm1=rng.normal(size=n_modes) * 1e-6)


def _fn():
    L = N.load()
    fn = L.mdx_simulate_strings_noalloc
    fn.restype = ctypes.c_int
    vp = ctypes.c_void_p
    fn.argtypes = [ctypes.POINTER(N.Instance), ctypes.c_int, vp, vp, vp, ctypes.c_int, vp, vp,
                   vp, vp, vp]
    return L, fn


def _describe(prepared, keep):
    arr = (N.Instance * len(prepared))()
    for i, d in enumerate(prepared):
        def dptr(x):
            a = np.ascontiguousarray(x, dtype=np.float64)
            keep.append(a)
            return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        arr[i].kind = N.KIND_TENSION
        arr[i].n_phi = len(d["omega2"])
        arr[i].dt = d["dt"]
        arr[i].omega2, arr[i].gamma, arr[i].b, arr[i].c = (dptr(d[k]) for k in
                                                             ("omega2", "gamma", "b", "c"))
        arr[i].lambda_ = dptr(d["lam"])
        arr[i].tau = d["tau"]
    return arr


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _noalloc_call(prepared, exc, q0, qm1, steps, want_audio=True):
    L, fn = _fn()
    keep = []
    arr = _describe(prepared, keep)
    TM = sum(len(d["omega2"]) for d in prepared)
    audio = (torch.full((len(prepared), steps), float("nan"), dtype=torch.float32,
                        device="cuda") if want_audio else None)
    q_end = torch.full((TM,), float("nan"), dtype=torch.float64, device="cuda")
    qm1_end = torch.full_like(q_end, float("nan"))
    status = torch.full((len(prepared),), -1, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = fn(arr, len(prepared), _ptr(exc), _ptr(q0), _ptr(qm1), steps, _ptr(audio),
            _ptr(q_end), _ptr(qm1_end), _ptr(status), stream)
    assert rc == 0, L.mdx_last_error()
    torch.cuda.synchronize()
    return (audio.cpu().numpy() if audio is not None else None, q_end.cpu().numpy(),
            qm1_end.cpu().numpy(), status.cpu().numpy())


def _planned(prepared, exc, q0, qm1, steps):
    """mdx_plan_create (scheme SV) + mdx_simulate on the same buffers."""
    sim = modal.Simulator(prepared)
    TM = sim.total_modes
    audio = torch.full((len(prepared), steps), float("nan"), dtype=torch.float32, device="cuda")
    q_end = torch.full((TM,), float("nan"), dtype=torch.float64, device="cuda")
    qm1_end = torch.full_like(q_end, float("nan"))
    status = torch.full((len(prepared),), -1, dtype=torch.int32, device="cuda")
    sim.plan.simulate(steps, exc=exc, q0=q0, qm1=qm1, audio=audio, q_end=q_end, qm1_end=qm1_end,
                      status=status)
    torch.cuda.synchronize()
    out = (audio.cpu().numpy(), q_end.cpu().numpy(), qm1_end.cpu().numpy(),
           status.cpu().numpy())
    return out, sim


def test_noalloc_matches_planned_path_twice():
    steps = 3000
    prepared = _instances(steps)
    sim = modal.Simulator(prepared)
    exc = sim.exc[:, :steps].contiguous()
    q0, qm1 = sim.q0.detach(), sim.qm1.detach()
    (ra, rq, rqm, rs), _ = _planned(prepared, exc, q0, qm1, steps)
    assert (rs == 0).all()
    for _ in range(2):
        audio, q_end, qm1_end, status = _noalloc_call(prepared, exc, q0, qm1, steps)
        assert (status == 0).all(), status
        assert np.array_equal(audio, ra)
        assert np.array_equal(q_end, rq)
        assert np.array_equal(qm1_end, rqm)
        assert np.isfinite(audio).all() and np.abs(audio).max() > 0


def test_noalloc_optional_inputs_and_outputs():
    """NULL initial state and excitation (zero), then NULL audio with the
    final state requested; each against the planned path with the same
    NULLs."""
    steps = 700
    prepared = _instances(steps)
    sim = modal.Simulator(prepared)
    exc = sim.exc[:, :steps].contiguous()
    q0 = sim.q0.detach()
    # zero initial state, excitation given
    (ra, rq, rqm, _), _ = _planned(prepared, exc, None, None, steps)
    audio, q_end, qm1_end, status = _noalloc_call(prepared, exc, None, None, steps)
    assert (status == 0).all()
    assert np.array_equal(audio, ra) and np.array_equal(q_end, rq)
    assert np.array_equal(qm1_end, rqm)
    # initial state given, no excitation: a small random displacement
    gen = torch.Generator(device="cuda").manual_seed(7)
    q0 = torch.randn(q0.shape, generator=gen, dtype=torch.float64, device="cuda") * 1e-6
    qm1 = q0.clone()
    (ra, rq, rqm, _), _ = _planned(prepared, None, q0, qm1, steps)
    audio, q_end, qm1_end, status = _noalloc_call(prepared, None, q0, qm1, steps)
    assert (status == 0).all()
    assert np.array_equal(audio, ra) and np.array_equal(q_end, rq)
    assert np.abs(audio[0]).max() > 0
    # no audio, final state only
    _, q_end2, qm1_end2, status = _noalloc_call(prepared, None, q0, qm1, steps, want_audio=False)
    assert (status == 0).all()
    assert np.array_equal(q_end2, rq) and np.array_equal(qm1_end2, rqm)


def test_noalloc_at_the_size_limit():
    """Instances whose modes fill the block up to the documented limit (all
    but the last with 1024 modes): the state region then ends 208 bytes
    before the end of the block, and one mode more no longer fits."""
    steps = 200
    n_inst = next(n for n in range(1, 64) if max_modes(n) <= 1024 * n)
    total = max_modes(n_inst)
    sizes = [1024] * (n_inst - 1)
    sizes.append(total - sum(sizes))
    assert 1 <= sizes[-1] <= 1024
    prepared = [_synthetic(n, 100 + i, steps) for i, n in enumerate(sizes)]
    sim = modal.Simulator(prepared)
    exc = sim.exc[:, :steps].contiguous()
    q0, qm1 = sim.q0.detach(), sim.qm1.detach()
    (ra, rq, rqm, rs), _ = _planned(prepared, exc, q0, qm1, steps)
    assert (rs == 0).all()
    for _ in range(2):
        audio, q_end, qm1_end, status = _noalloc_call(prepared, exc, q0, qm1, steps)
        assert (status == 0).all()
        assert np.array_equal(audio, ra) and np.array_equal(q_end, rq)
        assert np.array_equal(qm1_end, rqm)
    # one mode more is refused before anything is enqueued
    L, fn = _fn()
    bigger = prepared[:-1] + [_synthetic(sizes[-1] + 1, 999, steps)]
    keep = []
    arr = _describe(bigger, keep)
    rc = fn(arr, n_inst, None, None, None, steps, None, None, None, None, None)
    assert rc == 7                      # MDX_ERR_UNSUPPORTED
    assert b"scratch" in L.mdx_last_error()


def test_noalloc_rejects_oversize_request():
    L, fn = _fn()
    big = dict(kind="tension", omega2=np.full(1024, 1e4), gamma=np.ones(1024),
               b=np.ones(1024), c=np.ones(1024), dt=1e-4, lam=np.ones(1024), tau=0.0)
    keep = []
    arr = _describe([big] * 30, keep)
    rc = fn(arr, 30, None, None, None, 10, None, None, None, None, None)
    assert rc == 7                      # MDX_ERR_UNSUPPORTED: 30 720 modes > the fixed block
    assert b"scratch" in L.mdx_last_error()
