"""High-level API: simulate many instances on the GPU and differentiate.

    sim = Simulator(physics.prepare_workload(workload))
    audio = sim.simulate(steps)                          # [n_inst, steps] FP32 on the GPU
    audio = simulate_autograd(sim, steps, K=256)         # with a torch.autograd graph
    loss(audio).backward()                               # runs the adjoint kernels
    sim.omega2.grad, sim.gamma.grad, ...                 # FP64 gradients per mode

PyTorch provides device memory, the stream and the autograd graph; every
step of the time loop (forward, checkpoint recompute, adjoint) runs in the
libmdx CUDA kernels through the C ABI.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _native


class Simulator:
    def __init__(self, prepared, device="cuda:0", **plan_options):
        if not torch.cuda.is_available():
            raise RuntimeError("libmdx needs a CUDA device; no CPU fallback exists")
        self.device = torch.device(device)
        idx = self.device.index if self.device.index is not None else torch.cuda.current_device()
        self.prepared = list(prepared)
        self.plan = _native.Plan(self.prepared, device=idx, **plan_options)
        dev = self.device
        f64 = dict(dtype=torch.float64, device=dev)
        cat = lambda k: torch.tensor(np.concatenate([np.asarray(p[k], np.float64)
                                                     for p in self.prepared]), **f64)
        # coefficient tensors (leaves of the autograd graph; values are baked into the plan)
        self.omega2 = cat("omega2").requires_grad_()
        self.gamma = cat("gamma").requires_grad_()
        self.b = cat("b").requires_grad_()
        self.c = cat("c").requires_grad_()
        self.tau = torch.tensor([float(p.get("tau", 0.0)) for p in self.prepared], **f64).requires_grad_()
        kap = [np.asarray(p["kappa"], np.float64) for p in self.prepared
               if p["kind"] == "plate" and p.get("H") is not None]
        self.kappa = torch.tensor(np.concatenate(kap) if kap else np.zeros(0), **f64).requires_grad_()
        self.q0 = cat("q0").requires_grad_()
        self.qm1 = cat("qm1").requires_grad_()
        self.direction = torch.zeros(len(self.prepared), **f64).requires_grad_()
        steps = max(len(p["e"]) for p in self.prepared)
        exc = np.zeros((len(self.prepared), steps), np.float32)
        for i, p in enumerate(self.prepared):
            exc[i, :len(p["e"])] = p["e"]
        self.exc = torch.tensor(exc, device=dev)
        self.n_inst = len(self.prepared)
        self.total_modes = self.plan.total_modes

    # ------------------------------------------------------------------ raw calls
    def _exc_for(self, steps):
        if steps <= self.exc.shape[1]:
            return self.exc[:, :steps].contiguous()
        pad = torch.zeros(self.n_inst, steps, dtype=torch.float32, device=self.device)
        pad[:, :self.exc.shape[1]] = self.exc
        return pad

    def simulate(self, steps, K=0, q0=None, qm1=None, want_state=False, exc=None,
                 want_status=False):
        dev = self.device
        exc = self._exc_for(steps) if exc is None else exc
        audio = torch.empty(self.n_inst, steps, dtype=torch.float32, device=dev)
        ckpt = None
        if K > 0:
            nb = self.plan.checkpoint_bytes(steps, K)
            ckpt = torch.empty(nb // 4, dtype=torch.float32, device=dev)
        q_end = qm1_end = None
        if want_state:
            q_end = torch.empty(self.total_modes, dtype=torch.float64, device=dev)
            qm1_end = torch.empty_like(q_end)
        status = torch.empty(self.n_inst, dtype=torch.int32, device=dev) if want_status else None
        q0 = self.q0.detach() if q0 is None else q0
        qm1 = self.qm1.detach() if qm1 is None else qm1
        self.plan.simulate(steps, exc=exc, q0=q0, qm1=qm1, K=K, ckpt=ckpt, audio=audio,
                           q_end=q_end, qm1_end=qm1_end, status=status)
        out = dict(audio=audio, ckpt=ckpt, exc=exc)
        if want_state:
            out["q_end"], out["qm1_end"] = q_end, qm1_end
        if want_status:
            out["status"] = status
        return out

    def simulate_linear(self, steps, q0=None, qm1=None, exc=None, want_state=False,
                        want_status=False):
        """Linear response (nonlinear terms dropped), parallel in time."""
        dev = self.device
        exc = self._exc_for(steps) if exc is None else exc
        audio = torch.empty(self.n_inst, steps, dtype=torch.float32, device=dev)
        work = torch.empty(max(1, self.plan.linear_workspace_bytes(steps) // 8),
                           dtype=torch.float64, device=dev)
        out = dict(audio=audio)
        q_end = qm1_end = status = None
        if want_state:
            q_end = torch.empty(self.total_modes, dtype=torch.float64, device=dev)
            qm1_end = torch.empty_like(q_end)
            out["q_end"], out["qm1_end"] = q_end, qm1_end
        if want_status:
            status = torch.empty(self.n_inst, dtype=torch.int32, device=dev)
            out["status"] = status
        q0 = self.q0.detach() if q0 is None else q0
        qm1 = self.qm1.detach() if qm1 is None else qm1
        self.plan.simulate_linear(steps, work, exc=exc, q0=q0, qm1=qm1, audio=audio,
                                  q_end=q_end, qm1_end=qm1_end, status=status)
        return out

    def dH_layout(self):
        """Offsets of each plate's [M][N][N] block in the d_H output (plan
        order, plates with stress modes only) and the total length."""
        offs, tot = {}, 0
        for i, (n, m) in enumerate(zip(self.plan.n_modes, self.plan.n_stress)):
            if m > 0:
                offs[i] = tot
                tot += int(m) * int(n) * int(n)
        return offs, tot

    def grad(self, steps, d_audio, K, ckpt, exc=None, want_status=False, want_dH=False):
        dev = self.device
        exc = self._exc_for(steps) if exc is None else exc
        work = torch.empty(self.plan.workspace_bytes(steps, K) // 4 + 1, dtype=torch.float32,
                           device=dev)
        f64 = dict(dtype=torch.float64, device=dev)
        TM = self.total_modes
        out = dict(d_omega2=torch.empty(TM, **f64), d_gamma=torch.empty(TM, **f64),
                   d_b=torch.empty(TM, **f64), d_c=torch.empty(TM, **f64),
                   d_q0=torch.empty(TM, **f64), d_qm1=torch.empty(TM, **f64),
                   d_tau=torch.empty(self.n_inst, **f64),
                   d_kappa=torch.empty(max(1, self.kappa.numel()), **f64),
                   d_dir=torch.empty(self.n_inst, **f64))
        if want_dH:
            out["d_H"] = torch.empty(max(1, self.dH_layout()[1]), **f64)
        status = torch.empty(self.n_inst, dtype=torch.int32, device=dev) if want_status else None
        self.plan.grad(steps, d_audio.contiguous(), K, ckpt, work, exc=exc, out=out,
                       status=status)
        out["d_kappa"] = out["d_kappa"][:self.kappa.numel()]
        if want_status:
            out["status"] = status
        return out


    # ------------------------------------------------------------------ CUDA graphs
    def capture(self, steps, K=0, with_grad=False):
        """Capture one forward call (and, with with_grad, the adjoint with a
        fixed dL/dy buffer) into a CUDA graph.  Returns a GraphRun whose
        replay() re-executes the whole captured sequence with one launch from
        the host; inputs are read from, and outputs written to, the static
        buffers of the GraphRun (copy new inputs into them before replay)."""
        return GraphRun(self, steps, K, with_grad)


class GraphRun:
    def __init__(self, sim, steps, K, with_grad):
        dev = sim.device
        self.sim, self.steps, self.K = sim, steps, K
        self.exc = sim._exc_for(steps).clone()
        self.q0 = sim.q0.detach().clone()
        self.qm1 = sim.qm1.detach().clone()
        self.audio = torch.empty(sim.n_inst, steps, dtype=torch.float32, device=dev)
        self.ckpt = None
        if K > 0:
            self.ckpt = torch.empty(sim.plan.checkpoint_bytes(steps, K) // 4, dtype=torch.float32,
                                    device=dev)
        self.d_audio = self.grads = self.work = None
        if with_grad:
            assert K > 0, "the adjoint needs checkpoints (K > 0)"
            self.d_audio = torch.zeros(sim.n_inst, steps, dtype=torch.float32, device=dev)
            self.work = torch.empty(sim.plan.workspace_bytes(steps, K) // 4 + 1,
                                    dtype=torch.float32, device=dev)
            f64 = dict(dtype=torch.float64, device=dev)
            TM = sim.total_modes
            self.grads = dict(d_omega2=torch.empty(TM, **f64), d_gamma=torch.empty(TM, **f64),
                              d_b=torch.empty(TM, **f64), d_c=torch.empty(TM, **f64),
                              d_q0=torch.empty(TM, **f64), d_qm1=torch.empty(TM, **f64),
                              d_tau=torch.empty(sim.n_inst, **f64),
                              d_kappa=torch.empty(max(1, sim.kappa.numel()), **f64),
                              d_dir=torch.empty(sim.n_inst, **f64))
        self._body()                       # warm-up outside capture
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._body()

    def _body(self):
        sim = self.sim
        sim.plan.simulate(self.steps, exc=self.exc, q0=self.q0, qm1=self.qm1, K=self.K,
                          ckpt=self.ckpt, audio=self.audio)
        if self.grads is not None:
            sim.plan.grad(self.steps, self.d_audio, self.K, self.ckpt, self.work, exc=self.exc,
                          out=self.grads)

    def replay(self):
        self.graph.replay()
        return self.audio


class _SimulateFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sim, steps, K, omega2, gamma, b, c, tau, kappa, q0, qm1, direction):
        r = sim.simulate(steps, K=K)
        ctx.sim, ctx.steps, ctx.K = sim, steps, K
        ctx.ckpt, ctx.exc = r["ckpt"], r["exc"]
        return r["audio"]

    @staticmethod
    def backward(ctx, d_audio):
        g = ctx.sim.grad(ctx.steps, d_audio.float(), ctx.K, ctx.ckpt, exc=ctx.exc)
        return (None, None, None, g["d_omega2"], g["d_gamma"], g["d_b"], g["d_c"], g["d_tau"],
                g["d_kappa"], g["d_q0"], g["d_qm1"], g["d_dir"])


def simulate_autograd(sim: Simulator, steps: int, K: int = 256):
    """Audio [n_inst, steps] whose backward runs the checkpointed adjoint with
    interval K; gradients land on sim.omega2, sim.gamma, sim.b, sim.c,
    sim.tau, sim.kappa, sim.q0, sim.qm1 and sim.direction (<dL/dH, dH>)."""
    return _SimulateFn.apply(sim, steps, K, sim.omega2, sim.gamma, sim.b, sim.c, sim.tau,
                             sim.kappa, sim.q0, sim.qm1, sim.direction)
