"""Seeded synthetic workloads: the physical parameters of every instance.

This module is shared by the CUDA path, the benchmarks and the tests.  It only
draws and lists *physical* inputs (geometry, material, tension, stiffness,
damping law, excitation shape, strike/pickup positions, mode counts, sample
rate).  It computes no part of the modal method itself: no eigenvalues, no
frequencies, no scheme coefficients, no coupling tensors, no modal projections.
Each side (the library and the independent FP64 oracle) derives those from
these parameters on its own.

Workloads follow the problem statement of the paper: strings, membranes and
plates obeying Sec. 3, Eq. 1, with tension modulation (Eq. 3-4) or von Karman
coupling (Eq. 5-7), damping gamma = sigma0 + sigma1 * omega^2 (the d1 + d3*lambda
family of Eq. 14), a raised-cosine pluck or a raised-cosine strike, and a
displacement pickup at one point (Sec. 4.3.3).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

STEEL_E = 2.0e11       # Young's modulus (Pa)
STEEL_RHO = 7800.0     # volumetric density (kg/m^3)
STEEL_NU = 0.3         # Poisson ratio
PLATE_AREA = 0.24      # m^2: every rectangle has the area of the 0.4 x 0.6 m plate


@dataclasses.dataclass
class Instance:
    """Physical description of one simulated object.

    Lengths in metres, forces in newtons, times in seconds.  Relative positions
    are fractions of the side lengths (string: x/L; rectangle: (x/Lx, y/Ly)).
    """
    kind: str                 # 'string' | 'membrane' | 'plate'
    n_phi: int                # requested transverse modes (before stability truncation)
    n_psi: int = 0            # requested in-plane (Airy stress) modes, plates only
    # geometry
    length: float = 1.0       # string length L
    aspect: float = 1.0       # rectangle aspect a = Ly / Lx (area fixed at PLATE_AREA)
    area: float = PLATE_AREA
    thickness: float = 1e-3   # h (membranes and plates)
    # linear physics (Eq. 1): mass per unit length/area, tension, bending stiffness
    rho_lin: float = 1.0      # rho*A (string) or rho*h (membrane/plate)
    T0: float = 0.0           # tension: N (string) or N/m (membrane/plate)
    D: float = 0.0            # bending stiffness: EI (N m^2, string) or D (N m, plate)
    sigma0: float = 0.0       # gamma = sigma0 + sigma1 * omega^2
    sigma1: float = 0.0
    # nonlinearity inputs
    E: float = STEEL_E
    rho_vol: float = STEEL_RHO
    nu: float = STEEL_NU
    EA: float = 0.0           # string axial stiffness (tension modulation, Eq. 4)
    nonlinear: bool = True
    # excitation
    excitation: str = "strike"  # 'strike' | 'pluck'
    F0: float = 50.0            # strike: peak force of the raised-cosine pulse
    t_width: float = 1e-3       # strike: pulse duration
    strike: tuple = (0.31, 0.43)  # strike point (relative)
    pluck_amp: float = 5e-3     # pluck: raised-cosine displacement amplitude
    pluck_x0: float = 0.3       # pluck: centre (relative)
    pluck_width: float = 0.1    # pluck: width (relative)
    pickup: tuple = (0.73, 0.62)  # pickup point (relative)


@dataclasses.dataclass
class Workload:
    name: str
    instances: List[Instance]
    fs: float
    steps: int
    note: str = ""


def _steel_plate(n_phi: int, n_psi: int, aspect: float = 1.5, h: float = 1e-3,
                 D: Optional[float] = None, T0: float = 0.0,
                 sigma0: float = 1.0, sigma1: float = 3e-6, **kw) -> Instance:
    if D is None:
        D = STEEL_E * h ** 3 / (12.0 * (1.0 - STEEL_NU ** 2))
    return Instance(kind="plate", n_phi=n_phi, n_psi=n_psi, aspect=aspect,
                    thickness=h, rho_lin=STEEL_RHO * h, T0=T0, D=D,
                    sigma0=sigma0, sigma1=sigma1, **kw)


def string_40() -> Workload:
    """Tension-modulated stiff string: L = 1 m, T = 100 N, rhoA = 1e-3 kg/m,
    EI = 1e-4 N m^2, 40 modes, sigma = 0.5 + 1e-5 omega^2, raised-cosine pluck
    (width 0.1 L at 0.3 L, 5 mm), pickup at 0.7 L, 48 kHz x 1 s.

    EA is not given with the string; a solid circular steel section is assumed
    (I = A^2 / (4 pi), hence EA = sqrt(4 pi E EI))."""
    EI = 1e-4
    EA = math.sqrt(4.0 * math.pi * STEEL_E * EI)
    inst = Instance(kind="string", n_phi=40, length=1.0, rho_lin=1e-3, T0=100.0,
                    D=EI, sigma0=0.5, sigma1=1e-5, EA=EA, excitation="pluck",
                    pluck_amp=5e-3, pluck_x0=0.3, pluck_width=0.1, pickup=(0.7,))
    return Workload("string40_48k_1s", [inst], fs=48000.0, steps=48000)


def plate_100x30() -> Workload:
    """Von Karman plate, simply supported 0.4 x 0.6 m, h = 1 mm, steel,
    N_phi = 100, N_psi = 30, 1 ms raised-cosine strike of 50 N, 44.1 kHz x 1 s,
    sigma = 1 + 3e-6 omega^2."""
    inst = _steel_plate(100, 30, aspect=1.5)
    return Workload("plate100x30_44k_1s", [inst], fs=44100.0, steps=44100)


def _loguniform(rng, centre, decades, size=None):
    return centre * 10.0 ** rng.uniform(-decades, decades, size)


def batched_ragged(seed: int = 0, n_inst: int = 512, steps: int = 22050,
                   n_groups: Optional[int] = 8) -> Workload:
    """512 instances, half plates and half membranes, N_phi log-uniform in
    [20, 400], N_psi = N_phi // 4, aspect U[0.5, 2] (quantised to `n_groups`
    shared values when n_groups is not None), h U[0.5, 2] mm, tension and
    stiffness log-uniform over +-1 decade of 100 N/m and 18.3 N m."""
    rng = np.random.default_rng(seed)
    insts = []
    group_aspects = None
    if n_groups:
        group_aspects = np.linspace(0.5, 2.0, n_groups)
    for i in range(n_inst):
        kind = "plate" if rng.uniform() < 0.5 else "membrane"
        n_phi = int(math.floor(math.exp(rng.uniform(math.log(20.0), math.log(400.0)))))
        n_phi = max(1, min(400, n_phi))
        aspect = float(rng.uniform(0.5, 2.0))
        if group_aspects is not None:
            aspect = float(group_aspects[int(np.argmin(np.abs(group_aspects - aspect)))])
        h = float(rng.uniform(0.5e-3, 2e-3))
        strike = (float(rng.uniform(0.1, 0.9)), float(rng.uniform(0.1, 0.9)))
        pickup = (float(rng.uniform(0.1, 0.9)), float(rng.uniform(0.1, 0.9)))
        if kind == "plate":
            D = float(_loguniform(rng, 18.315, 1.0))
            insts.append(_steel_plate(n_phi, max(1, n_phi // 4), aspect=aspect, h=h, D=D,
                                      strike=strike, pickup=pickup))
        else:
            T0 = float(_loguniform(rng, 100.0, 1.0))
            insts.append(Instance(kind="membrane", n_phi=n_phi, aspect=aspect, thickness=h,
                                  rho_lin=STEEL_RHO * h, T0=T0, D=0.0, sigma0=1.0,
                                  sigma1=3e-6, strike=strike, pickup=pickup, F0=1.0))
    return Workload(f"batched{n_inst}_seed{seed}", insts, fs=44100.0, steps=steps,
                    note="membrane strike 1 N, plate strike 50 N")


ADJOINT_TARGET = dict(T0=100.0, D=18.315, aspect=1.5, sigma0=1.0, sigma1=3e-6)


def adjoint_plates(seed: int = 0, n_inst: int = 64, n_phi: int = 200, n_psi: int = 50,
                   steps: int = 22050, spread_decades: float = 0.3):
    """Target von Karman plate with tension (T0 = 100 N/m, D = 18.315 N m,
    aspect 1.5, sigma0 = 1, sigma1 = 3e-6) and `n_inst` initial guesses drawn
    log-uniform within +-`spread_decades` of each target parameter."""
    rng = np.random.default_rng(seed)
    tgt = _steel_plate(n_phi, n_psi, **ADJOINT_TARGET)
    inits = []
    for _ in range(n_inst):
        p = {k: float(_loguniform(rng, v, spread_decades)) for k, v in ADJOINT_TARGET.items()}
        p["aspect"] = float(min(2.0, max(0.5, p["aspect"])))
        inits.append(_steel_plate(n_phi, n_psi, **p))
    return (Workload(f"adjoint_target_{n_phi}x{n_psi}", [tgt], fs=44100.0, steps=steps),
            Workload(f"adjoint{n_inst}_{n_phi}x{n_psi}_seed{seed}", inits, fs=44100.0,
                     steps=steps))


# The six quantities a learned proposal predicts (log scale); see proposal draws.
PROPOSAL_PARAMS = ("T0_hat", "D_hat", "aspect", "sigma0", "sigma1", "nl_scale")


def proposal_draws(seed: int, n: int, steps: int = 11025):
    """Instances for the learned-proposal data set: half strings (40-100 modes),
    half plates (N_phi 50-200, N_psi = N_phi // 4), parameters log-uniform as in
    the batched workload, 0.25 s at 44.1 kHz.  Strings are struck like plates so
    every sample has the same excitation family."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        if rng.uniform() < 0.5:
            n_phi = int(rng.integers(40, 101))
            T0 = float(_loguniform(rng, 100.0, 1.0))
            EI = float(_loguniform(rng, 1e-4, 1.0))
            s0 = float(_loguniform(rng, 0.5, 0.5))
            s1 = float(_loguniform(rng, 1e-5, 0.5))
            EA = float(_loguniform(rng, math.sqrt(4 * math.pi * STEEL_E * 1e-4), 1.0))
            out.append(Instance(kind="string", n_phi=n_phi, length=1.0, rho_lin=1e-3, T0=T0,
                                D=EI, sigma0=s0, sigma1=s1, EA=EA, excitation="strike",
                                F0=1.0, strike=(float(rng.uniform(0.1, 0.9)),),
                                pickup=(float(rng.uniform(0.1, 0.9)),)))
        else:
            n_phi = int(rng.integers(50, 201))
            out.append(_steel_plate(
                n_phi, max(1, n_phi // 4), aspect=float(rng.uniform(0.5, 2.0)),
                D=float(_loguniform(rng, 18.315, 1.0)), T0=float(_loguniform(rng, 100.0, 1.0)),
                sigma0=float(_loguniform(rng, 1.0, 0.5)),
                sigma1=float(_loguniform(rng, 3e-6, 0.5)),
                E=float(_loguniform(rng, STEEL_E, 0.5)),
                strike=(float(rng.uniform(0.1, 0.9)), float(rng.uniform(0.1, 0.9))),
                pickup=(float(rng.uniform(0.1, 0.9)), float(rng.uniform(0.1, 0.9)))))
    return Workload(f"proposal{n}_seed{seed}", out, fs=44100.0, steps=steps)


def tiny_random(seed: int, kind: str, n_phi: int, n_psi: int = 0, steps: int = 256,
                fs: float = 44100.0) -> Workload:
    """Small seeded instance for parity sweeps over mode counts and edge sizes."""
    rng = np.random.default_rng(seed)
    if kind == "string":
        inst = Instance(kind="string", n_phi=n_phi, length=1.0, rho_lin=1e-3,
                        T0=float(_loguniform(rng, 100.0, 0.5)),
                        D=float(_loguniform(rng, 1e-4, 0.5)), sigma0=0.5, sigma1=1e-5,
                        EA=float(_loguniform(rng, 1.6e4, 0.5)), excitation="pluck",
                        pluck_x0=float(rng.uniform(0.2, 0.8)), pickup=(float(rng.uniform(0.1, 0.9)),))
    elif kind == "membrane":
        inst = Instance(kind="membrane", n_phi=n_phi, aspect=float(rng.uniform(0.5, 2.0)),
                        thickness=1e-3, rho_lin=STEEL_RHO * 1e-3,
                        T0=float(_loguniform(rng, 100.0, 1.0)), sigma0=1.0, sigma1=3e-6,
                        F0=1.0, strike=(float(rng.uniform(0.1, 0.9)), float(rng.uniform(0.1, 0.9))),
                        pickup=(float(rng.uniform(0.1, 0.9)), float(rng.uniform(0.1, 0.9))))
    else:
        inst = _steel_plate(n_phi, n_psi, aspect=float(rng.uniform(0.5, 2.0)),
                            D=float(_loguniform(rng, 18.315, 0.5)),
                            T0=float(_loguniform(rng, 30.0, 1.0)),
                            strike=(float(rng.uniform(0.1, 0.9)), float(rng.uniform(0.1, 0.9))),
                            pickup=(float(rng.uniform(0.1, 0.9)), float(rng.uniform(0.1, 0.9))))
    return Workload(f"tiny_{kind}{n_phi}x{n_psi}_seed{seed}", [inst], fs=fs, steps=steps)
