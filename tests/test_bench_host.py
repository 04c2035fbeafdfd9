"""Host-side logic of the benchmark (no GPU): the reference arm's JSON line,
the issue-bound roofline arithmetic, the tier-weighted operation counts, the
asymptotic-pair fraction and the rule that drops stale DRAM-traffic figures."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
from paper_2505_22797_gb300 import synthetic as syn  # noqa: E402


def test_reference_arm_prints_one_contract_line():
    """`--impl reference` times the FP64 oracle on the host cores and prints
    one JSON line with the keys of the benchmark contract."""
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "3", "--ref-samples", "2048"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 3
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["higher_is_better"] is True
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert "workload" in d["config"] and "model" not in d["config"]
    # both arms describe the workload with the same config
    from paper_2505_22797_gb300 import synthetic as syn
    assert d["config"] == json.loads(json.dumps(bench._config_desc(syn.config(bench.WORKLOAD))))


def test_issue_bound_arithmetic():
    # 152 SMs at 2070 MHz issue 128 thread instructions per clock each
    assert bench.issue_bound_gpair(152, 2070.0, 12.0, 1.0) == pytest.approx(
        152 * 2070e6 * 128 / 13 / 1e9)
    # an XU-heavy pair is held by the 32-lane XU pipe, not by issue
    assert bench.issue_bound_gpair(1, 1000.0, 1.0, 10.0) == pytest.approx(1000e6 * 32 / 10 / 1e9)
    # the scalar-issue bound of the forward operator's tier mix on the spiral workload
    f32, xu = bench.mixed_ops("k_forward", 0.9772)
    assert bench.issue_bound_gpair(152, 2070.0, f32, xu) == pytest.approx(3055.1, rel=1e-4)


def test_mixed_ops_interpolates_the_two_regimes():
    for k, ops in bench.ALG_OPS.items():
        assert bench.mixed_ops(k, 0.0) == pytest.approx(ops["far"])
        assert bench.mixed_ops(k, 1.0) == pytest.approx(ops["vfar"])
        lo, hi = bench.mixed_ops(k, 0.25), bench.mixed_ops(k, 0.75)
        mid = bench.mixed_ops(k, 0.5)
        assert mid[0] == pytest.approx((lo[0] + hi[0]) / 2)
        assert mid[1] == pytest.approx((lo[1] + hi[1]) / 2)


def test_vfar_fraction_limits():
    """All pairs asymptotic for a trajectory far outside the grid; none for a
    trajectory on the voxel centres with a PSF wider than the grid."""
    g = syn.square_grid(8, 4.0)
    m = syn.default_model()
    far = np.tile(np.array([[1e3, 1e3]]), (64, 1))
    assert bench.vfar_fraction(m, g, far, stride=1) == 1.0
    xs, ys = syn.voxel_centres(g)
    on = np.stack([xs[:8], ys[:8]], 1)
    wide = dict(m, beta=m["beta"] * 1e-3)
    assert bench.vfar_fraction(wide, g, on, stride=1) == 0.0
    f = bench.vfar_fraction(m, g, on, stride=1)
    assert 0.0 < f < 1.0


def test_traffic_is_dropped_for_other_sources(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.json").write_text(json.dumps(
        {"k_forward": {"dram_bytes_per_launch": 123, "source_digest": "aaaa"},
         "k_adjoint": {"dram_bytes_per_launch": 456, "source_digest": "bbbb"}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_digest", lambda: "aaaa")
    assert bench._traffic("k_forward") == 123
    assert bench._traffic("k_adjoint") is None      # captured on other sources
    assert bench._traffic("k_missing") is None
    (prof / "traffic.json").write_text("not json")
    assert bench._traffic("k_forward") is None


def test_kernel_digest_sees_code_not_comments():
    src = {f: "int a = 1;  // one\n/* block\n comment */\nint b = a + 2;\n" for f in bench.KERNEL_SOURCES}
    base = bench.kernel_digest(lambda f: src[f])
    edited = {f: "// a new comment\nint a = 1;\n\n\nint b = a + 2;   /* sum */\n" for f in bench.KERNEL_SOURCES}
    assert bench.kernel_digest(lambda f: edited[f]) == base
    changed = dict(src)
    changed[bench.KERNEL_SOURCES[0]] = "int a = 1;\nint b = a + 3;\n"
    assert bench.kernel_digest(lambda f: changed[f]) != base
    assert bench.code_only("x = 1; // c\n/* d */ y = 2;") == "x = 1;\n y = 2;"


def test_reference_arm_under_torchrun_prints_once():
    """Launched as the benchmark contract launches N > 1 ranks, the reference
    arm runs on rank 0 alone (one JSON line, n_gpus = N); the other rank
    exits 0 without work."""
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    res = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                          "--master-addr", "127.0.0.1", "--master-port", str(port),
                          os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                          "--steps", "1", "--warmup", "3", "--ref-samples", "2048"],
                         capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert res.returncode == 0, res.stderr[-3000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, res.stdout[-3000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    # rank 0 uses the host's cores although torchrun sets one thread per rank
    assert d["cpu_baseline"]["cores"] == (os.cpu_count() or 1)


def test_roofline_bases():
    """Three bases of the pair kernels' roofline: the tier-weighted
    algorithmic count with measured pipe rates, the plain closed-form count
    (25 FP32 + 3 XU at 128 / 16 per SM per clock) and the executed
    instruction count at the issue rate."""
    rates = {"fma": 128.0, "rsqrt": 16.0, "ex2": 16.0, "rcp": 16.0}
    b = bench.roofline_bases("k_adjoint", 1.0, 152, 2070.0, rates, 2000.0, executed=12.5)
    # all pairs asymptotic: 9 FP32 + 1 XU, issued as 4.5 packed + 1 -> the
    # FP32 lanes bind: 128 / 9 pairs per SM per clock
    assert b["tier_weighted"]["peak"] == pytest.approx(152 * 2070e6 * 128 / 9 / 1e9)
    assert bench.packed_issue("k_adjoint", 1.0) == pytest.approx(5.5)
    assert bench.packed_issue("k_adjoint", 0.0) == pytest.approx(20.0)
    # a faster packed-FMA rate raises the lane bound
    b2 = bench.roofline_bases("k_adjoint", 1.0, 152, 2070.0, dict(rates, fma=120.0, fma2=126.0), None)
    assert b2["tier_weighted"]["peak"] == pytest.approx(152 * 2070e6 * 126 / 9 / 1e9)
    assert b["plain_closed_form"]["peak"] == pytest.approx(152 * 2070e6 * 5.12 / 1e9)
    assert b["executed"]["peak"] == pytest.approx(152 * 2070e6 * 128 / 12.5 / 1e9)
    assert b["tier_weighted"]["frac"] == pytest.approx(2000.0 / b["tier_weighted"]["peak"])
    # all pairs in the closed form: 3 XU at 16 per clock bind before issue (20 / 128)
    far = bench.roofline_bases("k_adjoint", 0.0, 1, 1000.0, rates, None)
    assert far["tier_weighted"]["peak"] == pytest.approx(1000e6 / (3 / 16) / 1e9)
    assert far["tier_weighted"]["frac"] is None and "executed" not in far
    assert bench.xu_cycles_mixed(0.5, rates) == pytest.approx(0.5 * 3 / 16 + 0.5 / 16)
