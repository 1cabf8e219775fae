"""Profiling driver: the benchmark's plate batch through the C ABI alone.

Runs mdx_simulate (with checkpoints) and, with --grad, mdx_grad on the
64-plate adjoint batch (200 x 50 modes, aspect direction tensor included),
allocating device memory with the CUDA runtime directly.  PyTorch is not
imported, so a profiler attached to this process sees only libmdx's kernels
and does not pay for loading PyTorch's device code.

    python -m paper_2505_05940_gb300.profile_case --steps 200 --K 64 --grad
    python -m paper_2505_05940_gb300.profile_case --steps 22050 --K 1024 --grad

--cache FILE keeps the prepared instances (host FP64 work) between runs.
"""
from __future__ import annotations

import argparse
import ctypes
import os
import pickle
import time

import numpy as np

from . import _native, physics, workloads as W


def _prep(args):
    inst, fs, steps = args
    return physics.prepare(inst, fs, steps, want_aspect_derivative=True)


def prepared(n_inst, steps, cache, workers):
    if cache and os.path.exists(cache):
        with open(cache, "rb") as f:
            P = pickle.load(f)
        if len(P) == n_inst and len(P[0]["e"]) >= steps:
            return P
    import concurrent.futures as cf
    import multiprocessing as mp
    _, inits = W.adjoint_plates(seed=0, n_inst=n_inst, steps=steps)
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        P = list(ex.map(_prep, [(i, inits.fs, steps) for i in inits.instances]))
    if cache:
        with open(cache, "wb") as f:
            pickle.dump(P, f)
    return P


class _Cuda:
    def __init__(self):
        path = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64", "libcudart.so")
        self.rt = ctypes.CDLL(path)
        self.ptrs = []

    def check(self, rc, what):
        if rc != 0:
            raise RuntimeError(f"{what}: CUDA error {rc}")

    def alloc(self, nbytes):
        p = ctypes.c_void_p()
        self.check(self.rt.cudaMalloc(ctypes.byref(p), ctypes.c_size_t(max(16, nbytes))), "cudaMalloc")
        self.ptrs.append(p)
        return p

    def upload(self, arr):
        a = np.ascontiguousarray(arr)
        p = self.alloc(a.nbytes)
        self.check(self.rt.cudaMemcpy(p, a.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(a.nbytes), 1),
                   "cudaMemcpy")
        return p

    def sync(self):
        self.check(self.rt.cudaDeviceSynchronize(), "cudaDeviceSynchronize")

    def free(self):
        for p in self.ptrs:
            self.rt.cudaFree(p)
        self.ptrs = []


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-inst", type=int, default=64)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--K", type=int, default=64)
    ap.add_argument("--grad", action="store_true")
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--cache", default="")
    ap.add_argument("--prep-steps", type=int, default=22050)
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    P = prepared(a.n_inst, max(a.steps, a.prep_steps), a.cache, a.workers)
    L = _native.load()
    cu = _Cuda()
    plan = _native.Plan(P)
    n, steps, TM = len(P), a.steps, plan.total_modes
    exc = np.zeros((n, steps), np.float32)
    for i, p in enumerate(P):
        exc[i] = p["e"][:steps]
    d_exc = cu.upload(exc)
    q0 = cu.upload(np.concatenate([p["q0"] for p in P]).astype(np.float64))
    qm1 = cu.upload(np.concatenate([p["qm1"] for p in P]).astype(np.float64))
    audio = cu.alloc(n * steps * 4)
    ckpt = cu.alloc(plan.checkpoint_bytes(steps, a.K))
    status = cu.alloc(n * 4)
    work_bytes = plan.workspace_bytes(steps, a.K)
    work = cu.alloc(work_bytes) if a.grad else None
    ybar = cu.upload(np.random.default_rng(0).standard_normal((n, steps)).astype(np.float32))
    g = _native.Grads()
    if a.grad:
        for name, count in (("d_omega2", TM), ("d_gamma", TM), ("d_b", TM), ("d_c", TM),
                            ("d_q0", TM), ("d_qm1", TM), ("d_tau", n),
                            ("d_kappa", max(1, int(plan.n_stress.sum()))), ("d_dir", n)):
            setattr(g, name, cu.alloc(count * 8).value)
    t = []
    for _ in range(a.reps):
        cu.sync()
        t0 = time.perf_counter()
        _native.check(L.mdx_simulate(plan._h, d_exc, q0, qm1, steps, audio, None, None, a.K, ckpt,
                                     status, None))
        if a.grad:
            _native.check(L.mdx_grad(plan._h, d_exc, q0, qm1, steps, ybar, a.K, ckpt, work,
                                     work_bytes, ctypes.byref(g), status, None))
        cu.sync()
        t.append(time.perf_counter() - t0)
    st = np.zeros(n, np.int32)
    cu.check(cu.rt.cudaMemcpy(st.ctypes.data_as(ctypes.c_void_p), status, ctypes.c_size_t(n * 4), 2),
             "cudaMemcpy")
    print(f"plates {n}, modes {TM}, steps {steps}, K {a.K}, grad {a.grad}: "
          f"{min(t) * 1e3:.1f} ms per call (wall, synchronised); status max {int(st.max())}")
    plan.close()
    cu.free()
    if st.max() != 0:
        raise SystemExit(1)


if __name__ == "__main__":
    main()
