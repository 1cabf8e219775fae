"""ctypes binding of libmdx.so (include/mdx.h).

Argument marshalling only: every step of the time loop runs in the library's
CUDA kernels.  PyTorch supplies device memory and the current stream.  There
is no fallback: if the compiled library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

KIND_TENSION = 0
KIND_PLATE = 1

_ERRORS = {
    0: "MDX_OK", 1: "MDX_ERR_ARG", 2: "MDX_ERR_UNSTABLE", 3: "MDX_ERR_NONFINITE",
    4: "MDX_ERR_TIMEOUT", 5: "MDX_ERR_CUDA", 6: "MDX_ERR_OOM", 7: "MDX_ERR_UNSUPPORTED",
}

EXPORTED = ("mdx_last_error", "mdx_version", "mdx_plan_create", "mdx_plan_destroy",
            "mdx_plan_info", "mdx_checkpoint_bytes", "mdx_simulate", "mdx_grad_workspace_bytes",
            "mdx_grad", "mdx_coeffs_from_physics", "mdx_coeffs_vjp", "mdx_plan_set_profiling",
            "mdx_plan_kernel_stats", "mdx_plan_reset_stats", "mdx_plan_configure",
            "mdx_plan_tiles", "mdx_simulate_strings_noalloc", "mdx_plan_set_coefficients",
            "mdx_mlp_act_elems", "mdx_mlp_work_elems", "mdx_mlp_forward", "mdx_mlp_backward",
            "mdx_adam_step", "mdx_f32_to_bf16", "mdx_plan_set_l2_keep", "mdx_plan_l2_keep",
            "mdx_difference_coefficients", "mdx_coefficient_grads", "mdx_modal_from_physics",
            "mdx_physics_vjp", "mdx_plan_group_work", "mdx_plan_set_coupling",
            "mdx_linear_workspace_bytes", "mdx_simulate_linear", "mdx_logmel")


class MdxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRORS.get(code, code)}: {msg}")
        self.code = code


_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)


class Instance(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n_phi", ctypes.c_int), ("n_psi", ctypes.c_int),
                ("dt", ctypes.c_double), ("omega2", _D), ("gamma", _D), ("b", _D), ("c", _D),
                ("lambda_", _D), ("tau", ctypes.c_double), ("H", _F), ("kappa", _D), ("dH", _F),
                ("phi_class", ctypes.POINTER(ctypes.c_int)),
                ("psi_class", ctypes.POINTER(ctypes.c_int)), ("geom_group", ctypes.c_int)]


class Options(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("max_ctas", ctypes.c_int),
                ("ring_stages", ctypes.c_int), ("stage_bytes", ctypes.c_int),
                ("force_split", ctypes.c_int), ("wait_limit", ctypes.c_int),
                ("debug_flags", ctypes.c_int), ("scheme", ctypes.c_int),
                ("group_engine", ctypes.c_int)]


SHAPE_STRING = 0
SHAPE_RECTANGLE = 1


class Physics(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("shape", ctypes.c_int), ("n_phi", ctypes.c_int),
                ("n_psi", ctypes.c_int), ("dt", ctypes.c_double),
                ("omega_dt_max", ctypes.c_double), ("length", ctypes.c_double),
                ("area", ctypes.c_double), ("aspect", ctypes.c_double), ("D", ctypes.c_double),
                ("T0", ctypes.c_double), ("rho", ctypes.c_double), ("sigma0", ctypes.c_double),
                ("sigma1", ctypes.c_double), ("strike", ctypes.c_double * 2),
                ("pickup", ctypes.c_double * 2), ("tension_stiffness", ctypes.c_double),
                ("vk_scale", ctypes.c_double), ("zeta4", _D)]


class Modal(ctypes.Structure):
    _fields_ = [("n_phi", ctypes.c_int), ("n_psi", ctypes.c_int),
                ("labels", ctypes.POINTER(ctypes.c_int)), ("lambda_", _D), ("omega2", _D),
                ("gamma", _D), ("b", _D), ("c", _D), ("tau", ctypes.c_double), ("kappa", _D)]


class PhysicsGrads(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("d_T0", "d_D", "d_aspect", "d_sigma0",
                                                "d_sigma1", "d_tension_stiffness",
                                                "d_vk_scale")]


MLP_MAX_LAYERS = 8


class MLPDesc(ctypes.Structure):
    _fields_ = [("n_layers", ctypes.c_int), ("dims", ctypes.c_int * (MLP_MAX_LAYERS + 1)),
                ("W", ctypes.c_void_p * MLP_MAX_LAYERS), ("b", ctypes.c_void_p * MLP_MAX_LAYERS)]


class Grads(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("d_omega2", "d_gamma", "d_b", "d_c", "d_q0",
                                                "d_qm1", "d_tau", "d_kappa", "d_dir", "d_H")]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libmdx.so (building it first when nvcc is available)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise OSError(f"libmdx.so not found at {path}; run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        vp, i32, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        L.mdx_last_error.restype = ctypes.c_char_p
        L.mdx_version.restype = ctypes.c_char_p
        L.mdx_plan_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Instance), i32,
                                      ctypes.POINTER(Options)]
        L.mdx_plan_destroy.argtypes = [vp]
        L.mdx_plan_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_long),
                                    ctypes.POINTER(ctypes.c_long)]
        L.mdx_checkpoint_bytes.argtypes = [vp, i32, i32]
        L.mdx_checkpoint_bytes.restype = sz
        L.mdx_simulate.argtypes = [vp, vp, vp, vp, i32, vp, vp, vp, i32, vp, vp, vp]
        L.mdx_grad_workspace_bytes.argtypes = [vp, i32, i32]
        L.mdx_grad_workspace_bytes.restype = sz
        L.mdx_grad.argtypes = [vp, vp, vp, vp, i32, vp, i32, vp, vp, sz, ctypes.POINTER(Grads),
                               vp, vp]
        L.mdx_coeffs_from_physics.argtypes = [i32, _D, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                              _D, _D]
        L.mdx_coeffs_vjp.argtypes = [i32, _D, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, _D, _D, _D, _D, _D, _D, _D]
        L.mdx_plan_set_coefficients.argtypes = [vp, _D, _D, _D, _D, _D, _D]
        L.mdx_plan_set_coupling.argtypes = [vp, i32, _F, _F]
        L.mdx_linear_workspace_bytes.argtypes = [vp, i32]
        L.mdx_linear_workspace_bytes.restype = sz
        L.mdx_simulate_linear.argtypes = [vp, vp, vp, vp, i32, vp, vp, vp, vp, sz, vp, vp]
        L.mdx_modal_from_physics.argtypes = [ctypes.POINTER(Physics), ctypes.POINTER(Modal)]
        L.mdx_physics_vjp.argtypes = [ctypes.POINTER(Physics), i32, i32, _D, _D,
                                      ctypes.c_double, _D, ctypes.c_double, _D,
                                      ctypes.POINTER(PhysicsGrads)]
        L.mdx_difference_coefficients.argtypes = [i32, i32, _D, _D, ctypes.c_double, _D, _D, _D]
        L.mdx_coefficient_grads.argtypes = [i32, i32, _D, _D, ctypes.c_double, _D, _D, _D, _D, _D]
        L.mdx_mlp_act_elems.argtypes = [ctypes.POINTER(MLPDesc), i32]
        L.mdx_mlp_act_elems.restype = sz
        L.mdx_mlp_work_elems.argtypes = [ctypes.POINTER(MLPDesc), i32]
        L.mdx_mlp_work_elems.restype = sz
        L.mdx_mlp_forward.argtypes = [ctypes.POINTER(MLPDesc), i32, vp, vp, vp, vp]
        L.mdx_mlp_backward.argtypes = [ctypes.POINTER(MLPDesc), i32, vp, vp, vp,
                                       ctypes.POINTER(vp), ctypes.POINTER(vp), vp, vp]
        L.mdx_adam_step.argtypes = [ctypes.c_longlong, vp, vp, vp, vp, vp, ctypes.c_float,
                                    ctypes.c_float, ctypes.c_float, ctypes.c_float, i32, vp]
        L.mdx_f32_to_bf16.argtypes = [ctypes.c_longlong, vp, vp, vp]
        L.mdx_logmel.argtypes = [vp, i32, i32, ctypes.c_double, i32, i32, i32, ctypes.c_double,
                                 ctypes.c_double, i32, vp, vp]
        L.mdx_plan_configure.argtypes = [vp, i32, i32]
        L.mdx_plan_set_l2_keep.argtypes = [vp, ctypes.c_double]
        L.mdx_plan_l2_keep.argtypes = [vp]
        L.mdx_plan_l2_keep.restype = ctypes.c_double
        L.mdx_plan_tiles.argtypes = [vp] + [ctypes.POINTER(i32)] * 4
        L.mdx_plan_set_profiling.argtypes = [vp, i32]
        L.mdx_plan_group_work.argtypes = [vp, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double)]
        L.mdx_plan_reset_stats.argtypes = [vp]
        L.mdx_plan_kernel_stats.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_long),
                                            ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_double)]
        for name in EXPORTED[2:]:
            fn = getattr(L, name)
            if fn.restype is None or fn.restype is ctypes.c_int:
                fn.restype = ctypes.c_int
        _lib = L
        return L


def check(rc):
    if rc != 0:
        raise MdxError(rc, load().mdx_last_error().decode())


def _ptr(t):
    """Device (or host) address of a torch tensor or numpy array, or None."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return ctypes.c_void_p(t.data_ptr())
    return ctypes.c_void_p(t.ctypes.data)


def _stream(stream=None):
    """cudaStream_t of a torch stream (default: torch's current stream)."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """A compiled set of instances on one device (owns the library plan).

    `instances` is a list of dicts with keys kind ('tension' | 'plate'),
    omega2, gamma, b, c (float64 arrays [N]), dt, and either lam, tau
    (tension) or H [M][N][N] float32, kappa [M] (plate), optional dH.
    """

    def __init__(self, instances, device=0, max_ctas=0, ring_stages=0, stage_bytes=0,
                 force_split=0, wait_limit=0, debug_flags=0, use_classes=True, scheme="sv",
                 group_engine="tf32x3"):
        L = load()
        self._keep = []
        arr = (Instance * len(instances))()
        for i, d in enumerate(instances):
            kind = KIND_PLATE if d["kind"] == "plate" else KIND_TENSION
            N = int(len(d["omega2"]))
            s = arr[i]
            s.kind = kind
            s.n_phi = N
            s.dt = float(d["dt"])

            def dptr(x):
                a = np.ascontiguousarray(x, dtype=np.float64)
                self._keep.append(a)
                return a.ctypes.data_as(_D)

            def fptr(x):
                a = np.ascontiguousarray(x, dtype=np.float32)
                self._keep.append(a)
                return a.ctypes.data_as(_F)

            def iptr(x):
                a = np.ascontiguousarray(x, dtype=np.int32)
                self._keep.append(a)
                return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))

            s.omega2, s.gamma, s.b, s.c = (dptr(d[k]) for k in ("omega2", "gamma", "b", "c"))
            if kind == KIND_TENSION:
                s.lambda_ = dptr(d["lam"])
                s.tau = float(d.get("tau", 0.0))
                s.n_psi = 0
            else:
                H = d.get("H")
                if H is not None and len(H) > 0:
                    s.n_psi = int(H.shape[0])
                    s.H = fptr(H)
                    s.kappa = dptr(d["kappa"])
                    if d.get("dH") is not None:
                        s.dH = fptr(d["dH"])
                    if (d.get("phi_class") is not None and d.get("psi_class") is not None
                            and use_classes):
                        s.phi_class = iptr(d["phi_class"])
                        s.psi_class = iptr(d["psi_class"])
                    s.geom_group = int(d.get("geom_group", 0))
                else:
                    s.n_psi = 0
        opts = Options(device, max_ctas, ring_stages, stage_bytes, force_split, wait_limit,
                       debug_flags, SCHEMES[scheme] if isinstance(scheme, str) else int(scheme),
                       GROUP_ENGINES[group_engine])
        h = ctypes.c_void_p()
        check(L.mdx_plan_create(ctypes.byref(h), arr, len(instances), ctypes.byref(opts)))
        self._h = h
        self._keep = []
        n = ctypes.c_int()
        tm = ctypes.c_long()
        check(L.mdx_plan_info(h, ctypes.byref(n), ctypes.byref(tm), None))
        self.n_inst = n.value
        self.total_modes = tm.value
        offs = (ctypes.c_long * self.n_inst)()
        check(L.mdx_plan_info(h, None, None, offs))
        self.mode_offset = np.array(offs[:], dtype=np.int64)
        self.n_modes = np.array([len(d["omega2"]) for d in instances], dtype=np.int64)
        self.n_stress = np.array([0 if d["kind"] != "plate" or d.get("H") is None
                                  else len(d["H"]) for d in instances], dtype=np.int64)
        self.device = device

    def close(self):
        if getattr(self, "_h", None):
            load().mdx_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ coefficients
    def set_coefficients(self, omega2=None, gamma=None, b=None, c=None, tau=None, kappa=None):
        """Host FP64 arrays in plan order (None keeps the current values)."""
        def dp(x):
            if x is None:
                return None
            a = np.ascontiguousarray(x, dtype=np.float64)
            keep.append(a)
            return a.ctypes.data_as(_D)
        keep = []
        check(load().mdx_plan_set_coefficients(self._h, dp(omega2), dp(gamma), dp(b), dp(c),
                                               dp(tau), dp(kappa)))

    def set_coupling(self, inst, H, dH=None):
        """New coupling tensor [M][N][N] (host FP32) for plate `inst`."""
        h = np.ascontiguousarray(H, dtype=np.float32)
        d = None if dH is None else np.ascontiguousarray(dH, dtype=np.float32)
        check(load().mdx_plan_set_coupling(self._h, int(inst), h.ctypes.data_as(_F),
                                           d.ctypes.data_as(_F) if d is not None else None))

    # ------------------------------------------------------------------ tiles
    def configure(self, stage_bytes=0, ring_stages=0):
        check(load().mdx_plan_configure(self._h, int(stage_bytes), int(ring_stages)))

    def set_l2_keep(self, fraction=-1.0):
        """Fraction of the coupling stream kept in L2 (negative: automatic)."""
        check(load().mdx_plan_set_l2_keep(self._h, float(fraction)))

    def l2_keep(self):
        return float(load().mdx_plan_l2_keep(self._h))

    def tiles(self):
        v = [ctypes.c_int() for _ in range(4)]
        check(load().mdx_plan_tiles(self._h, *[ctypes.byref(x) for x in v]))
        return dict(stage_bytes=v[0].value, ring_fwd=v[1].value, ring_rev=v[2].value,
                    ctas=v[3].value)

    # ------------------------------------------------------------------ tracing
    def group_work(self):
        """(bytes, flops) per step of the grouped-plate launch (0, 0 if none)."""
        b, f = ctypes.c_double(), ctypes.c_double()
        check(load().mdx_plan_group_work(self._h, ctypes.byref(b), ctypes.byref(f)))
        return b.value, f.value

    def set_profiling(self, enable=True):
        check(load().mdx_plan_set_profiling(self._h, 1 if enable else 0))

    def reset_stats(self):
        check(load().mdx_plan_reset_stats(self._h))

    def kernel_stats(self, which):
        """which: 0 forward, 1 recompute, 2 reverse, 3 direction contraction,
        4 fused sweep, 5 grouped plates, 6 cluster-resident forward
        -> (launches, ms, bytes)."""
        n = ctypes.c_long()
        ms = ctypes.c_double()
        by = ctypes.c_double()
        check(load().mdx_plan_kernel_stats(self._h, which, ctypes.byref(n), ctypes.byref(ms),
                                           ctypes.byref(by)))
        return n.value, ms.value, by.value

    # ------------------------------------------------------------------ calls
    def checkpoint_bytes(self, steps, K):
        return int(load().mdx_checkpoint_bytes(self._h, steps, K))

    def workspace_bytes(self, steps, K):
        return int(load().mdx_grad_workspace_bytes(self._h, steps, K))

    def simulate(self, steps, exc=None, q0=None, qm1=None, K=0, ckpt=None, audio=None,
                 q_end=None, qm1_end=None, status=None, stream=None):
        """Raw call: every tensor argument is a CUDA tensor already allocated
        by the caller (see include/mdx.h for shapes)."""
        check(load().mdx_simulate(self._h, _ptr(exc), _ptr(q0), _ptr(qm1), int(steps),
                                  _ptr(audio), _ptr(q_end), _ptr(qm1_end), int(K), _ptr(ckpt),
                                  _ptr(status), _stream(stream)))

    def simulate_linear(self, steps, work, exc=None, q0=None, qm1=None, audio=None, q_end=None,
                        qm1_end=None, status=None, stream=None):
        """Raw call of mdx_simulate_linear (device tensors allocated by the caller)."""
        wb = work.numel() * work.element_size()
        check(load().mdx_simulate_linear(self._h, _ptr(exc), _ptr(q0), _ptr(qm1), int(steps),
                                         _ptr(audio), _ptr(q_end), _ptr(qm1_end), _ptr(work), wb,
                                         _ptr(status), _stream(stream)))

    def linear_workspace_bytes(self, steps):
        return int(load().mdx_linear_workspace_bytes(self._h, steps))

    def grad(self, steps, d_audio, K, ckpt, work, exc=None, q0=None, qm1=None, out=None,
             status=None, stream=None):
        g = Grads()
        if out:
            for k, v in out.items():
                setattr(g, k, _ptr(v).value if v is not None else None)
        wb = work.numel() * work.element_size()
        check(load().mdx_grad(self._h, _ptr(exc), _ptr(q0), _ptr(qm1), int(steps),
                              _ptr(d_audio), int(K), _ptr(ckpt), _ptr(work), wb,
                              ctypes.byref(g), _ptr(status), _stream(stream)))


SCHEMES = {"sv": 0, "tf": 1}
GROUP_ENGINES = {"tf32x3": 0, "off": 1}


def difference_coefficients(scheme, omega2, gamma, T):
    """(eps, rho, r) of the difference form for the given scheme ('sv' | 'tf')."""
    w2 = np.ascontiguousarray(omega2, dtype=np.float64)
    gm = np.ascontiguousarray(gamma, dtype=np.float64)
    eps, rho, r = (np.zeros_like(w2) for _ in range(3))
    check(load().mdx_difference_coefficients(SCHEMES[scheme], len(w2), w2.ctypes.data_as(_D),
                                             gm.ctypes.data_as(_D), float(T),
                                             eps.ctypes.data_as(_D), rho.ctypes.data_as(_D),
                                             r.ctypes.data_as(_D)))
    return eps, rho, r


def coefficient_grads(scheme, omega2, gamma, T, A, V, F):
    """dL/d omega^2, dL/d gamma from the adjoint sums A, V, F (see include/mdx.h)."""
    arr = [np.ascontiguousarray(x, dtype=np.float64) for x in (omega2, gamma, A, V, F)]
    dw2, dgm = np.zeros_like(arr[0]), np.zeros_like(arr[0])
    check(load().mdx_coefficient_grads(SCHEMES[scheme], len(arr[0]),
                                       *[a.ctypes.data_as(_D) for a in arr[:2]], float(T),
                                       *[a.ctypes.data_as(_D) for a in arr[2:]],
                                       dw2.ctypes.data_as(_D), dgm.ctypes.data_as(_D)))
    return dw2, dgm


def coeffs_from_physics(lam, D, T0, rho, s0, s1):
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    w2 = np.zeros_like(lam)
    gm = np.zeros_like(lam)
    check(load().mdx_coeffs_from_physics(len(lam), lam.ctypes.data_as(_D), D, T0, rho, s0, s1,
                                         w2.ctypes.data_as(_D), gm.ctypes.data_as(_D)))
    return w2, gm


def coeffs_vjp(lam, D, T0, rho, s0, s1, d_omega2, d_gamma):
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    dw = np.ascontiguousarray(d_omega2, dtype=np.float64)
    dg = np.ascontiguousarray(d_gamma, dtype=np.float64)
    out = [ctypes.c_double() for _ in range(4)]
    dl = np.zeros_like(lam)
    check(load().mdx_coeffs_vjp(len(lam), lam.ctypes.data_as(_D), D, T0, rho, s0, s1,
                                dw.ctypes.data_as(_D), dg.ctypes.data_as(_D),
                                *[ctypes.byref(o) for o in out], dl.ctypes.data_as(_D)))
    return dict(D=out[0].value, T0=out[1].value, s0=out[2].value, s1=out[3].value, lam=dl)


def physics_struct(kind, shape, n_phi, n_psi, dt, omega_dt_max, length=0.0, area=0.0,
                   aspect=1.0, D=0.0, T0=0.0, rho=1.0, sigma0=0.0, sigma1=0.0,
                   strike=(0.5, 0.5), pickup=(0.5, 0.5), tension_stiffness=0.0, vk_scale=0.0,
                   zeta4=None):
    """mdx_physics of include/mdx.h (zeta4 is kept alive on the returned struct)."""
    ph = Physics()
    ph.kind, ph.shape, ph.n_phi, ph.n_psi = int(kind), int(shape), int(n_phi), int(n_psi)
    ph.dt, ph.omega_dt_max = float(dt), float(omega_dt_max)
    ph.length, ph.area, ph.aspect = float(length), float(area), float(aspect)
    ph.D, ph.T0, ph.rho = float(D), float(T0), float(rho)
    ph.sigma0, ph.sigma1 = float(sigma0), float(sigma1)
    st = list(strike) + [0.0] * (2 - len(strike))
    pk = list(pickup) + [0.0] * (2 - len(pickup))
    ph.strike[0], ph.strike[1] = float(st[0]), float(st[1])
    ph.pickup[0], ph.pickup[1] = float(pk[0]), float(pk[1])
    ph.tension_stiffness, ph.vk_scale = float(tension_stiffness), float(vk_scale)
    if zeta4 is not None:
        z = np.ascontiguousarray(zeta4, dtype=np.float64)
        ph._zeta4 = z
        ph.zeta4 = z.ctypes.data_as(_D)
    return ph


def modal_from_physics(ph):
    """mdx_modal_from_physics: dict of labels, lam, omega2, gamma, b, c, tau,
    kappa (kept modes only)."""
    n, m = ph.n_phi, max(ph.n_psi, 1)
    labels = np.zeros((n, 2), np.int32)
    arrs = {k: np.zeros(n) for k in ("lam", "omega2", "gamma", "b", "c")}
    kappa = np.zeros(m)
    out = Modal()
    out.labels = labels.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    out.lambda_, out.omega2, out.gamma, out.b, out.c = (
        arrs[k].ctypes.data_as(_D) for k in ("lam", "omega2", "gamma", "b", "c"))
    out.kappa = kappa.ctypes.data_as(_D)
    check(load().mdx_modal_from_physics(ctypes.byref(ph), ctypes.byref(out)))
    ne, me = out.n_phi, out.n_psi
    res = {k: v[:ne].copy() for k, v in arrs.items()}
    res["labels"] = labels[:ne].astype(np.int64)
    res["tau"] = out.tau
    res["kappa"] = kappa[:me].copy()
    res["n_psi"] = me
    return res


def physics_vjp(ph, n_phi, n_psi, d_omega2, d_gamma, d_tau=0.0, d_kappa=None, d_dir=0.0,
                dzeta4=None):
    """mdx_physics_vjp: dict of d_T0, d_D, d_aspect, d_sigma0, d_sigma1,
    d_tension_stiffness, d_vk_scale."""
    dw = np.ascontiguousarray(d_omega2, dtype=np.float64)
    dg = np.ascontiguousarray(d_gamma, dtype=np.float64)
    dk = None if d_kappa is None else np.ascontiguousarray(d_kappa, dtype=np.float64)
    dz = None if dzeta4 is None else np.ascontiguousarray(dzeta4, dtype=np.float64)
    out = PhysicsGrads()
    check(load().mdx_physics_vjp(ctypes.byref(ph), int(n_phi), int(n_psi), dw.ctypes.data_as(_D),
                                 dg.ctypes.data_as(_D), float(d_tau),
                                 dk.ctypes.data_as(_D) if dk is not None else None,
                                 float(d_dir),
                                 dz.ctypes.data_as(_D) if dz is not None else None,
                                 ctypes.byref(out)))
    return {k: getattr(out, k) for k, _ in PhysicsGrads._fields_}


def logmel(audio, fs=44100.0, n_fft=1024, hop=256, n_mels=128, fmin=20.0, fmax=None,
           segments=8, stream=None):
    """mdx_logmel: [B, T] FP32 CUDA tensor -> [B, n_mels * segments] log-mel
    features (mel-major, segments innermost)."""
    import torch
    if not (audio.is_cuda and audio.dtype == torch.float32 and audio.dim() == 2):
        raise ValueError("audio must be a [batch, T] float32 CUDA tensor")
    x = audio.contiguous()
    B, T = x.shape
    out = torch.empty(B, n_mels * segments, dtype=torch.float32, device=x.device)
    check(load().mdx_logmel(_ptr(x), B, T, float(fs), n_fft, hop, n_mels, float(fmin),
                            float(fs / 2.0 if fmax is None else fmax), segments, _ptr(out),
                            _stream(stream)))
    return out
