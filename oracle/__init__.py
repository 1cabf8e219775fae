"""Independent FP64 CPU oracle of the per-time-step modal update.

TEST INFRASTRUCTURE ONLY.  Only the tests, `__graft_entry__.smoke()` and the
benchmark's CPU-baseline leg (and its `--impl reference` arm) may import this
package.  It shares no code, constants or helpers with the CUDA library in
`paper_2505_05940_gb300`; the only module both sides read is the seeded
physical-parameter generator `paper_2505_05940_gb300.workloads`, which holds
none of the method's arithmetic.

Contents:
  modal_oracle.c     Stormer-Verlet time stepping (Eq. 20) with the tension
                     (Eq. 8) and von Karman (Eq. 9) forces, pickup, and a
                     hand-written reverse (adjoint) recursion, all FP64.
  physics_oracle.py  modes, Eq. 13-14, Eq. 21-23 (Stormer-Verlet) and Eq. 15-19
                     (impulse invariance) coefficients, projections.
  coupling_oracle.py H and C tensors (Eq. 10-11) by 2D quadrature.
  mlp_oracle.py      FP64 forward/backward of the proposal MLP.
  stft_oracle.py     multi-resolution log-STFT loss (Eq. 24).

Parity status: every function is pinned by a `-m "not gpu"` test against a
closed form, an invariant, brute force or finite differences, except the
full-length nonlinear audio itself, which has no printed value in the paper
(parity unpinned beyond those properties).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "modal_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libmodal_oracle.so")
_lock = threading.Lock()
_lib = None

TENSION, PLATE = 0, 1


def build(force: bool = False) -> str:
    """Compile the C oracle with the host compiler (FP64, no fast-math)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O3", "-fopenmp", "-fno-fast-math", "-shared", "-fPIC", _SRC,
           "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            D = ctypes.POINTER(ctypes.c_double)
            I = ctypes.c_int
            _lib.orc_forward.argtypes = [I, I, I, D, D, D, D, D, D, ctypes.c_double, D, D, I, D,
                                         D, D, D, D, D, D]
            _lib.orc_forward.restype = I
            _lib.orc_adjoint.argtypes = [I, I, I, D, D, D, D, D, D, ctypes.c_double, D, D, I, D,
                                         D, D, D, D, D, D, D, D, D, D, D, D]
            _lib.orc_adjoint.restype = I
            L = ctypes.POINTER(ctypes.c_long)
            IP = ctypes.POINTER(ctypes.c_int)
            _lib.orc_forward_batch.argtypes = [I, IP, IP, IP, L, L, L, D, D, D, D, D, D, D, D, D,
                                               I, D, D, D, D]
            _lib.orc_forward_batch.restype = I
            _lib.orc_force.argtypes = [I, I, I, D, ctypes.c_double, D, D, D, D]
            _lib.orc_force.restype = I
    return _lib


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _model_args(oi):
    kind = PLATE if (oi.kind == "plate") else TENSION
    H = _c(oi.H) if (kind == PLATE and oi.H is not None) else None
    kappa = _c(oi.kappa) if (kind == PLATE and oi.kappa is not None) else None
    M = oi.M if H is not None else 0
    lam = _c(oi.lam)
    return kind, M, H, kappa, lam


def force(oi, q):
    """fnl(q) of Eq. 8 (tension kind) or Eq. 9 (plate) in FP64."""
    kind, M, H, kappa, lam = _model_args(oi)
    q = _c(q)
    f = np.zeros(oi.N)
    lib().orc_force(kind, oi.N, M, _p(lam), float(oi.taup), _p(H), _p(kappa), _p(q), _p(f))
    return f


def forward(oi, steps=None, e=None, q0=None, qm1=None, want_traj=False):
    """Run Eq. 20 in FP64.  Returns dict(y, qN, qNm1[, traj])."""
    steps = len(oi.e) if steps is None else steps
    e = _c(oi.e[:steps] if e is None else e)
    q0 = _c(oi.q0 if q0 is None else q0)
    qm1 = _c(oi.qm1 if qm1 is None else qm1)
    N = oi.N
    kind, M, H, kappa, lam = _model_args(oi)
    g, p, r, b, c = (_c(v) for v in (oi.g, oi.p, oi.r, oi.b, oi.c))
    y = np.zeros(steps)
    qN = np.zeros(N)
    qNm1 = np.zeros(N)
    traj = np.zeros((steps + 2, N)) if want_traj else None
    bad = lib().orc_forward(kind, N, M, _p(g), _p(p), _p(r), _p(b), _p(c), _p(lam),
                            float(oi.taup), _p(H), _p(kappa), steps, _p(e), _p(q0), _p(qm1),
                            _p(y), _p(traj), _p(qN), _p(qNm1))
    out = dict(y=y, qN=qN, qNm1=qNm1, nonfinite=bool(bad))
    if want_traj:
        out["traj"] = traj
    return out


def adjoint(oi, ybar, steps=None, e=None, q0=None, qm1=None, want_dH=False, traj=None):
    """Reverse-mode derivatives of L with dL/dy = ybar.  Returns a dict of
    dq0, dqm1, dg, dp, dr, db, dc, dtau (tension) or dkappa (plate), dH."""
    steps = len(ybar) if steps is None else steps
    if traj is None:
        traj = forward(oi, steps, e, q0, qm1, want_traj=True)["traj"]
    e = _c(oi.e[:steps] if e is None else e)
    N = oi.N
    kind, M, H, kappa, lam = _model_args(oi)
    g, p, r, b, c = (_c(v) for v in (oi.g, oi.p, oi.r, oi.b, oi.c))
    out = {k: np.zeros(N) for k in ("dq0", "dqm1", "dg", "dp", "dr", "db", "dc")}
    dtau = np.zeros(1)
    dkappa = np.zeros(max(M, 1))
    dH = np.zeros((M, N, N)) if (want_dH and M > 0) else None
    lib().orc_adjoint(kind, N, M, _p(g), _p(p), _p(r), _p(b), _p(c), _p(lam), float(oi.taup),
                      _p(H), _p(kappa), steps, _p(e), _p(_c(traj)), _p(_c(ybar)),
                      _p(out["dq0"]), _p(out["dqm1"]), _p(out["dg"]), _p(out["dp"]),
                      _p(out["dr"]), _p(out["db"]), _p(out["dc"]), _p(dtau), _p(dkappa), _p(dH))
    out["dtau"] = float(dtau[0])
    out["dkappa"] = dkappa[:M]
    if dH is not None:
        out["dH"] = dH
    return out


def coefficient_grads(oi, adj, T):
    """Chain rule from (g, p, r, b) to (omega^2, gamma, b) through Eqs. 21-23."""
    w2, gm = oi.omega2, oi.gamma
    den = 1.0 + gm * T
    # r = T^2/(1+gT); g = r(2/T^2 - w2); p = r(-1/T^2 + g/T)
    dr_dg = -T ** 3 / den ** 2
    dg_dw2 = -oi.r
    dg_dgm = (2.0 / T ** 2 - w2) * dr_dg
    dp_dgm = (-1.0 / T ** 2 + gm / T) * dr_dg + oi.r / T
    d_omega2 = adj["dg"] * dg_dw2
    d_gamma = adj["dg"] * dg_dgm + adj["dp"] * dp_dgm + adj["dr"] * dr_dg
    return d_omega2, d_gamma


def coefficient_grads_tf(oi, adj, T):
    """Chain rule from (g, p, r) to (omega^2, gamma) for the impulse-invariant
    coefficients (oscillatory modes, omega > gamma):
      g = 2 e^{-gamma T} cos(w~ T), p = -e^{-2 gamma T},
      r = T e^{-gamma T} sin(w~ T) / w~,  w~^2 = omega^2 - gamma^2."""
    w2, gm = oi.omega2, oi.gamma
    wt = np.sqrt(w2 - gm ** 2)
    e1 = np.exp(-gm * T)
    g, r = oi.g, oi.r
    # d/dw~ of sin(w~ T)/w~
    ds = (T * np.cos(wt * T) * wt - np.sin(wt * T)) / wt ** 2
    dg_dw2 = -T * e1 * np.sin(wt * T) / wt          # = -r
    dg_dgm = -T * g + 2.0 * e1 * np.sin(wt * T) * T * gm / wt
    dp_dgm = -2.0 * T * oi.p
    dr_dw2 = T * e1 * ds / (2.0 * wt)
    dr_dgm = -T * r - T * e1 * ds * gm / wt
    d_omega2 = adj["dg"] * dg_dw2 + adj["dr"] * dr_dw2
    d_gamma = adj["dg"] * dg_dgm + adj["dp"] * dp_dgm + adj["dr"] * dr_dgm
    return d_omega2, d_gamma


def forward_batch(ois, steps, n_threads=None):
    """Forward-only FP64 run of many independent instances (OpenMP over
    instances); used for CPU timing.  Returns y [n_inst][steps]."""
    n = len(ois)
    kinds = np.array([PLATE if (o.kind == "plate" and o.H is not None) else TENSION
                      for o in ois], dtype=np.int32)
    Ns = np.array([o.N for o in ois], dtype=np.int32)
    Ms = np.array([o.M if (o.kind == "plate" and o.H is not None) else 0 for o in ois],
                  dtype=np.int32)
    off_mode = np.concatenate([[0], np.cumsum(Ns)[:-1]]).astype(np.int64)
    Hs = [np.ascontiguousarray(o.H, dtype=np.float64).reshape(-1) if m > 0 else np.zeros(0)
          for o, m in zip(ois, Ms)]
    off_H = np.concatenate([[0], np.cumsum([h.size for h in Hs])[:-1]]).astype(np.int64)
    off_M = np.concatenate([[0], np.cumsum(Ms)[:-1]]).astype(np.int64)
    cat = lambda name: _c(np.concatenate([getattr(o, name) for o in ois]))
    H = _c(np.concatenate(Hs + [np.zeros(1)]))
    kappa = _c(np.concatenate([o.kappa if m > 0 else np.zeros(0) for o, m in zip(ois, Ms)]
                              + [np.zeros(1)]))
    taup = _c([o.taup for o in ois])
    e = _c(np.stack([o.e[:steps] for o in ois]))
    y = np.zeros((n, steps))
    if n_threads is not None:
        os.environ["OMP_NUM_THREADS"] = str(n_threads)
    Lp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_long))
    Ip = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    bufs = [cat(k) for k in ("g", "p", "r", "b", "c", "lam", "q0", "qm1")]
    lib().orc_forward_batch(n, Ip(kinds), Ip(Ns), Ip(Ms), Lp(off_mode), Lp(off_H), Lp(off_M),
                            _p(bufs[0]), _p(bufs[1]), _p(bufs[2]), _p(bufs[3]), _p(bufs[4]),
                            _p(bufs[5]), _p(taup), _p(H), _p(kappa), steps, _p(e), _p(bufs[6]),
                            _p(bufs[7]), _p(y))
    return y
