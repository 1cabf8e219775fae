"""bench.py's host-side contract (no GPU): the reference arm's JSON line, the
defaults, and the traffic figure read from the committed ncu summary."""
import importlib.util
import json
import os
import subprocess
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_defaults_finish_within_minutes():
    b = _bench()
    sys_argv = sys.argv
    try:
        sys.argv = ["bench.py"]
        a = b.parse()
    finally:
        sys.argv = sys_argv
    assert a.gpus == 1 and a.steps >= 1 and a.warmup >= 3 and a.impl == "ours"
    assert (a.n_inst, a.n_phi, a.n_psi, a.sim_steps, a.K) == (64, 200, 50, 22050, 1024)


def test_profiled_traffic_follows_the_kernel_source():
    b = _bench()
    a = types.SimpleNamespace(n_inst=64, n_phi=200, n_psi=50)
    t = b.profiled_traffic(a, 1024)
    # the committed summary matches the current plate kernel source
    assert t is not None and 5e10 < t < 1.4e11
    # another workload has no captured traffic
    assert b.profiled_traffic(types.SimpleNamespace(n_inst=32, n_phi=200, n_psi=50), 1024) is None


def test_reference_arm_prints_one_contract_line():
    pytest.importorskip("torch")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["metric"] == b_metric()


def b_metric():
    return _bench().METRIC
