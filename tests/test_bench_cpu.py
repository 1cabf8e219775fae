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


def test_profiled_traffic_follows_the_kernel_source(tmp_path, monkeypatch):
    """The traffic figure is read from the committed ncu summary only while the
    kernel source still has the hash recorded there; after a kernel edit it
    is null until the kernel is profiled again."""
    import hashlib
    b = _bench()
    a = types.SimpleNamespace(n_inst=64, n_phi=200, n_psi=50)
    src = os.path.join(ROOT, "paper_2505_05940_gb300", "csrc", "mdx_plate.cu")
    digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    root = tmp_path / "r"
    (root / "profiles").mkdir(parents=True)
    (root / "paper_2505_05940_gb300" / "csrc").mkdir(parents=True)
    (root / "paper_2505_05940_gb300" / "csrc" / "mdx_plate.cu").write_bytes(open(src, "rb").read())
    summary = root / "profiles" / "plate_kernel_fused_64plates_200x50.md"
    summary.write_text("kernel-source: paper_2505_05940_gb300/csrc/mdx_plate.cu sha256 "
                       f"{digest}\ntraffic_bytes_per_step: 75827031\n")
    monkeypatch.setattr(b, "ROOT", str(root))
    assert b.profiled_traffic(a, 1024) == 75827031 * 1024
    summary.write_text("kernel-source: paper_2505_05940_gb300/csrc/mdx_plate.cu sha256 "
                       "0123456789abcdef\ntraffic_bytes_per_step: 75827031\n")
    assert b.profiled_traffic(a, 1024) is None
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


def test_single_instance_oracle_sample():
    """The single-thread oracle baseline of the single-instance workloads
    times the oracle's forward pass on a bounded sample."""
    import bench
    from paper_2505_05940_gb300 import workloads as W
    v, desc = bench.oracle_forward_sample(W.string_40(), 2000, runs=1)
    assert v > 0 and "one host thread" in desc and "2000 steps" in desc
