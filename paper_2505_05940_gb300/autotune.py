"""Tile autotuner for the plate kernel.

For a given set of instances the tuner times a short checkpointed forward
run (the streaming plate kernel, which also serves every gradient pass) for
each candidate TMA stage size (the ring depth follows from the shared memory
left over) and keeps the fastest.  Checkpoint-free forward passes of a few
small plates run cluster-resident instead and have no stages to tune.  Results are cached in a JSON file keyed by the
GPU name and a signature of the plate shapes, so a workload is tuned once per
device type.  Timing uses the library's own per-launch CUDA events
(mdx_plan_kernel_stats).
"""
from __future__ import annotations

import hashlib
import json
import os
import threading

STAGE_CANDIDATES = (32 * 1024, 48 * 1024, 64 * 1024, 80 * 1024, 96 * 1024)
_lock = threading.Lock()


def default_cache_path():
    base = os.environ.get("MDX_AUTOTUNE_CACHE")
    if base:
        return base
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def signature(prepared):
    shapes = sorted((len(p["omega2"]), 0 if p.get("H") is None else len(p["H"]),
                     p["kind"]) for p in prepared)
    h = hashlib.sha1(json.dumps(shapes).encode()).hexdigest()[:16]
    return f"{len(prepared)}x{h}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune(sim, steps=128, repeats=2, cache_path=None, candidates=STAGE_CANDIDATES, force=False):
    """Pick the stage size for sim.plan (a modal.Simulator); applies it and
    returns {'stage_bytes', 'us_per_step', 'cached', 'trials'}."""
    import torch
    if not any(p["kind"] == "plate" and p.get("H") is not None for p in sim.prepared):
        return {"stage_bytes": 0, "us_per_step": None, "cached": False, "trials": []}
    path = cache_path or default_cache_path()
    key = f"{torch.cuda.get_device_name(sim.device)}|{signature(sim.prepared)}"
    with _lock:
        cache = _load(path)
    if not force and key in cache:
        sim.plan.configure(stage_bytes=cache[key]["stage_bytes"])
        return dict(cache[key], cached=True)
    trials = []
    for stage in candidates:
        try:
            sim.plan.configure(stage_bytes=stage)
        except Exception as e:  # does not fit in shared memory
            trials.append({"stage_bytes": stage, "error": str(e)})
            continue
        sim.simulate(steps, K=steps)
        torch.cuda.synchronize()
        sim.plan.set_profiling(True)
        sim.plan.reset_stats()
        for _ in range(repeats):
            sim.simulate(steps, K=steps)
        n, ms, _ = sim.plan.kernel_stats(0)
        sim.plan.set_profiling(False)
        trials.append({"stage_bytes": stage, "us_per_step": 1e3 * ms / max(n, 1) / steps,
                       "tiles": sim.plan.tiles()})
    ok = [t for t in trials if "us_per_step" in t]
    best = min(ok, key=lambda t: t["us_per_step"])
    sim.plan.configure(stage_bytes=best["stage_bytes"])
    entry = {"stage_bytes": best["stage_bytes"], "us_per_step": best["us_per_step"],
             "trials": trials}
    with _lock:
        cache = _load(path)
        cache[key] = entry
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, path)
    return dict(entry, cached=False)
