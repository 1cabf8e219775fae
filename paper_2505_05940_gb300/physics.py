"""Plan inputs from physical parameters (argument marshalling around the C ABI).

  * Laplacian eigenpairs (Sec. 3, Eq. 2), omega^2 and gamma (Sec. 3.2,
    Eq. 13-14), the strike and pickup projections, the tension-modulation
    coefficient tau' (Eq. 4), the von Karman scale kappa (Eq. 9) and the
    stability cut (omega T < 1.9, a shortened plate keeps the same fraction
    of its stress modes) all come from the library's mdx_modal_from_physics.
  * The Airy modes and the coupling tensor H (Eq. 10) come from the offline
    FP64 generator in coupling.py (an input of mdx_plan_create).
  * The excitation signal (raised-cosine force pulse e^n, or a raised-cosine
    pluck projected in closed form, q^0 = <w0, Phi>, q^{-1} = q^0) is the
    user-side input of the simulation.
"""
from __future__ import annotations

import math
from typing import List

import numpy as np

from . import _native
from . import coupling as _coupling

OMEGA_T_LIMIT = 1.9


def rectangle_sides(inst):
    return _coupling.sides(inst.area, inst.aspect)


def physics_args(inst, fs, zeta4=None, omega_dt_max=OMEGA_T_LIMIT, **override):
    """Fields of the mdx_physics of one workload instance (a plain dict that
    pickles; override replaces fields)."""
    plate = inst.kind == "plate"
    ts = 0.0
    if inst.nonlinear and inst.kind == "string":
        ts = inst.EA
    elif inst.nonlinear and inst.kind == "membrane":
        ts = inst.E * inst.thickness / (1.0 - inst.nu ** 2)
    args = dict(kind=_native.KIND_PLATE if plate else _native.KIND_TENSION,
                shape=_native.SHAPE_STRING if inst.kind == "string" else _native.SHAPE_RECTANGLE,
                n_phi=inst.n_phi, n_psi=inst.n_psi if plate else 0, dt=1.0 / fs,
                omega_dt_max=omega_dt_max, length=inst.length, area=inst.area,
                aspect=inst.aspect, D=inst.D, T0=inst.T0, rho=inst.rho_lin, sigma0=inst.sigma0,
                sigma1=inst.sigma1, strike=inst.strike, pickup=inst.pickup,
                tension_stiffness=ts,
                vk_scale=inst.E / (2.0 * inst.rho_vol) if (plate and inst.nonlinear) else 0.0,
                zeta4=None if zeta4 is None else np.asarray(zeta4, np.float64))
    args.update(override)
    return args


def physics_of(inst, fs, zeta4=None, omega_dt_max=OMEGA_T_LIMIT, **override):
    """mdx_physics of one workload instance (override replaces fields)."""
    return _native.physics_struct(**physics_args(inst, fs, zeta4, omega_dt_max, **override))


def physics_struct(prepared):
    """mdx_physics of a prepared instance (for mdx_physics_vjp)."""
    return _native.physics_struct(**prepared["physics_args"])


def mode_labels(inst, n, fs=44100.0):
    """The first n mode labels of the instance's shape (no stability cut)."""
    return _native.modal_from_physics(physics_of(inst, fs, omega_dt_max=0.0, n_phi=n,
                                                 n_psi=0))["labels"]


def raised_cosine_force(F0, width, fs, steps):
    t = np.arange(steps) / fs
    return np.where(t <= width, 0.5 * F0 * (1.0 - np.cos(2.0 * math.pi * t / width)), 0.0)


def pluck_modal(length, labels, amp, x0_rel, width_rel):
    """<w0, Phi_mu> of w0 = amp/2 (1 + cos(2 pi (x - x0)/W)) on |x - x0| <= W/2,
    in closed form (removable singularity at mu pi / L = 2 pi / W)."""
    k = math.pi * labels[:, 0].astype(np.float64) / length
    x0 = x0_rel * length
    W = width_rel * length
    a = 2.0 * math.pi / W
    num = amp * np.sin(k * x0) * np.sin(0.5 * k * W) * a * a
    den = k * (a * a - k * k)
    near = np.abs(a - k) < 1e-9 * a
    safe = np.where(near, 1.0, den)
    val = np.where(near, amp * np.sin(k * x0) * W / 4.0, num / safe)
    return math.sqrt(2.0 / length) * val


class PreparedInstance(dict):
    """Plan-ready description of one instance (plus its inputs)."""


def prepare(inst, fs, steps, coupling="auto", want_aspect_derivative=False):
    """Physical parameters -> dict with the mdx_instance fields, the excitation
    e [steps], the initial state q0, qm1 and bookkeeping (labels, lambda, for
    plates zeta4, and `physics_args`, the fields of the mdx_physics
    description, see physics_struct)."""
    T = 1.0 / fs
    pargs = physics_args(inst, fs)
    mod = _native.modal_from_physics(_native.physics_struct(**pargs))
    labels, lam = mod["labels"], mod["lam"]
    n_eff = len(lam)
    if inst.kind == "string":
        labels = labels[:, :1]
    if inst.excitation == "pluck":
        e = np.zeros(steps)
        q0 = pluck_modal(inst.length, labels, inst.pluck_amp, inst.pluck_x0, inst.pluck_width)
    else:
        e = raised_cosine_force(inst.F0, inst.t_width, fs, steps)
        q0 = np.zeros(n_eff)
    out = PreparedInstance(kind="tension" if inst.kind != "plate" else "plate",
                           omega2=mod["omega2"], gamma=mod["gamma"], b=mod["b"], c=mod["c"],
                           dt=T, lam=lam, labels=labels, e=e, q0=q0, qm1=q0.copy(), src=inst,
                           tau=mod["tau"])
    M = mod["n_psi"]
    if inst.kind == "plate" and inst.nonlinear and M > 0 and coupling is not None:
        Lx, Ly = rectangle_sides(inst)
        psi_cls = None
        if callable(coupling):
            res = coupling(inst, labels, M)
            H, zeta4 = res[0], res[1]
            if len(res) > 2:
                psi_cls = res[2]
            dH = dz = None
        elif want_aspect_derivative:
            H, zeta4, dH, dz, psi_cls = _coupling.coupling_with_aspect_derivative(
                inst.area, inst.aspect, labels, M)
        else:
            airy = _coupling.airy_modes(Lx, Ly, M)
            H, zeta4 = _coupling.coupling_tensor(Lx, Ly, labels, M, airy=airy)
            psi_cls = _coupling.airy_classes(airy[1])
            dH = dz = None
        if psi_cls is not None:
            # symmetry classes: H^k_ij vanishes unless class(i) ^ class(j) == class(k)
            out["phi_class"] = _coupling.transverse_classes(labels)
            out["psi_class"] = psi_cls
        zeta4 = np.asarray(zeta4, np.float64)
        # kappa of Eq. 9 for the kept stress modes (second call, with zeta^4)
        pargs = physics_args(inst, fs, zeta4=np.concatenate([zeta4, np.full(inst.n_psi - M, 1.0)]))
        out["kappa"] = _native.modal_from_physics(_native.physics_struct(**pargs))["kappa"]
        out["H"] = H.astype(np.float32)
        out["zeta4"] = zeta4
        if dH is not None:
            out["dH"] = dH.astype(np.float32)
            out["dzeta4"] = dz
    out["physics_args"] = pargs
    return out


def prepare_workload(wl, coupling="auto", want_aspect_derivative=False) -> List[PreparedInstance]:
    return [prepare(inst, wl.fs, wl.steps, coupling, want_aspect_derivative)
            for inst in wl.instances]
