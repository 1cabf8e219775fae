"""The parallel-in-time linear solver (Sec. 4.3.2) against the FP64 oracle.

mdx_simulate_linear evaluates every mode's linear recursion (the plan's
scheme, nonlinear terms dropped) as a blocked prefix scan over time in FP64.
Linear instances (strings, membranes and plates with the nonlinearity off)
are compared with the oracle's time stepping, which is itself pinned to
scipy.signal.lfilter and to the closed form of the recursion.  The scan
carries no FP32 state; its only FP32 quantities are the excitation it reads
and the audio it writes, so audio and final state must agree to 1e-6.
Chunk boundaries (256 steps), a ragged last chunk, a start from rest and from
a given state, both schemes, and a batch of uneven instances are covered."""
import copy

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle
from oracle import physics_oracle as PO
from paper_2505_05940_gb300 import modal, workloads as W

from test_gpu_parity import rel, to_plan


def _linear(inst):
    x = copy.deepcopy(inst)
    x.nonlinear = False
    return x


@pytest.mark.parametrize("scheme", ["sv", "tf"])
@pytest.mark.parametrize("steps", [1, 255, 256, 257, 3001])
def test_linear_solver_matches_oracle(scheme, steps):
    fs = 44100.0
    insts = [_linear(W.tiny_random(1, "string", 40, steps=steps).instances[0]),
             _linear(W.tiny_random(2, "membrane", 77, steps=steps).instances[0]),
             _linear(W.tiny_random(3, "plate", 130, 0, steps=steps).instances[0]),
             _linear(W.tiny_random(4, "string", 3, steps=steps).instances[0])]
    ois = [PO.build_instance(i, fs, steps, scheme=scheme) for i in insts]
    sim = modal.Simulator([to_plan(o, fs) for o in ois], scheme=scheme)
    r = sim.simulate_linear(steps, want_state=True, want_status=True)
    torch.cuda.synchronize()
    assert (r["status"].cpu().numpy() == 0).all()
    audio = r["audio"].cpu().numpy()
    q = r["q_end"].cpu().numpy()
    qm = r["qm1_end"].cpu().numpy()
    off = sim.plan.mode_offset
    for i, oi in enumerate(ois):
        ref = oracle.forward(oi, steps=steps)
        assert rel(audio[i], ref["y"]) <= 1e-6, (i, rel(audio[i], ref["y"]))
        assert rel(q[off[i]:off[i] + oi.N], ref["qN"]) <= 1e-6
        assert rel(qm[off[i]:off[i] + oi.N], ref["qNm1"]) <= 1e-6


def test_linear_solver_from_a_given_state_equals_time_stepping():
    """A plucked string (initial state, no excitation) against mdx_simulate on
    the same linear plan: the FP32 time stepping with a compensated state
    agrees with the FP64 scan to its own accuracy."""
    fs, steps = 48000.0, 48000
    inst = _linear(W.string_40().instances[0])
    oi = PO.build_instance(inst, fs, steps)
    sim = modal.Simulator([to_plan(oi, fs)])
    lin = sim.simulate_linear(steps)["audio"].cpu().numpy()[0]
    ts = sim.simulate(steps)["audio"].cpu().numpy()[0]
    ref = oracle.forward(oi, steps=steps)["y"]
    assert rel(lin, ref) <= 1e-6
    assert rel(ts, lin) <= 1e-5
