"""The no-allocation entry point against the planned path.

mdx_simulate_strings_noalloc serves callers that may not allocate device
memory (a real-time audio callback, where cudaMalloc can block and
synchronise the device; a plug-in whose host owns every device buffer).  It
keeps its scratch in a fixed block inside the library.  This test calls it
through the C ABI twice in a row (the second call reuses a block that still
holds the first call's contents) and compares both results with
mdx_plan_create + mdx_simulate on the same inputs, within the tolerance of
the other GPU tests.  It sits in a file of its own, collected last."""
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

TOL = 1e-5


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


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


def _noalloc_call(prepared, exc, q0, qm1, steps):
    L = N.load()
    fn = L.mdx_simulate_strings_noalloc
    fn.restype = ctypes.c_int
    vp = ctypes.c_void_p
    fn.argtypes = [ctypes.POINTER(N.Instance), ctypes.c_int, vp, vp, vp, ctypes.c_int, vp, vp,
                   vp, vp, vp]
    keep = []
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
    TM = sum(len(d["omega2"]) for d in prepared)
    audio = torch.empty(len(prepared), steps, dtype=torch.float32, device="cuda")
    q_end = torch.empty(TM, dtype=torch.float64, device="cuda")
    qm1_end = torch.empty_like(q_end)
    status = torch.full((len(prepared),), -1, dtype=torch.int32, device="cuda")
    stream = vp(torch.cuda.current_stream().cuda_stream)
    rc = fn(arr, len(prepared), vp(exc.data_ptr()), vp(q0.data_ptr()), vp(qm1.data_ptr()),
            steps, vp(audio.data_ptr()), vp(q_end.data_ptr()), vp(qm1_end.data_ptr()),
            vp(status.data_ptr()), stream)
    assert rc == 0, L.mdx_last_error()
    torch.cuda.synchronize()
    return audio.cpu().numpy(), q_end.cpu().numpy(), qm1_end.cpu().numpy(), status.cpu().numpy()


def test_noalloc_matches_planned_path_twice():
    steps = 3000
    prepared = _instances(steps)
    sim = modal.Simulator(prepared)
    ref = sim.simulate(steps, want_state=True)
    torch.cuda.synchronize()
    ref_audio = ref["audio"].cpu().numpy()
    ref_q = ref["q_end"].cpu().numpy()
    ref_qm1 = ref["qm1_end"].cpu().numpy()
    exc = sim.exc[:, :steps].contiguous()
    q0, qm1 = sim.q0.detach(), sim.qm1.detach()
    for _ in range(2):
        audio, q_end, qm1_end, status = _noalloc_call(prepared, exc, q0, qm1, steps)
        assert (status == 0).all(), status
        for i in range(len(prepared)):
            assert _rel(audio[i], ref_audio[i]) <= TOL, i
        assert _rel(q_end, ref_q) <= TOL
        assert _rel(qm1_end, ref_qm1) <= TOL


def test_noalloc_rejects_oversize_request():
    L = N.load()
    fn = L.mdx_simulate_strings_noalloc
    fn.restype = ctypes.c_int
    big = dict(kind="tension", omega2=np.full(1024, 1e4), gamma=np.ones(1024),
               b=np.ones(1024), c=np.ones(1024), dt=1e-4, lam=np.ones(1024), tau=0.0)
    keep = []
    arr = (N.Instance * 30)()
    for i in range(30):
        for k in ("omega2", "gamma", "b", "c"):
            a = np.ascontiguousarray(big[k])
            keep.append(a)
            setattr(arr[i], k, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        a = np.ascontiguousarray(big["lam"])
        keep.append(a)
        arr[i].lambda_ = a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        arr[i].kind, arr[i].n_phi, arr[i].dt = N.KIND_TENSION, 1024, 1e-4
    fn.argtypes = [ctypes.POINTER(N.Instance), ctypes.c_int] + [ctypes.c_void_p] * 3 + \
        [ctypes.c_int] + [ctypes.c_void_p] * 5
    rc = fn(arr, 30, None, None, None, 10, None, None, None, None, None)
    assert rc == 7                      # MDX_ERR_UNSUPPORTED: 30 720 modes > the fixed block
    assert b"scratch" in L.mdx_last_error()
