"""Host logic of the benchmark (CPU): the roofline's algorithmic bytes, the
clock-record parsing that decides whether a run is kept, the committed DRAM
traffic keyed to the kernel sources, and the warm-start records the JSON line
carries."""
import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_algorithmic_bytes_are_nineteen_reads_and_writes():
    # 19 populations read and 19 written per update: 152 B in FP32, 76 B in 16-bit
    assert bench.algorithmic_bytes(512, "fp32") == 20_401_094_656
    assert bench.algorithmic_bytes(512, "fp32") == 152 * 512 ** 3
    assert bench.algorithmic_bytes(256, "bf16") == 76 * 256 ** 3
    assert bench.algorithmic_bytes(128, "fp64") == 304 * 128 ** 3


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.lines = lines
    return s


def test_clock_summary_median_and_reasons():
    idle = "Not Active"
    rows = [f"0, {mhz}, 2070, 900.0, 0x0, {idle}, {idle}, {idle}, {cap}"
            for mhz, cap in ((2070, idle), (2055, "Active"), (2070, idle))]
    s = _sampler(rows).summary()
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    hot = _sampler([f"0, 1400, 2070, 1400.0, 0x0, {idle}, Active, {idle}, {idle}"]).summary()
    assert hot["reasons"] == ["hw_thermal_slowdown"]


def test_clock_summary_without_samples_says_so():
    assert _sampler([]).summary()["reasons"] == ["unsampled"]
    # malformed or short lines are skipped, not guessed
    assert _sampler(["0, [N/A], 2070", "garbage"]).summary()["reasons"] == ["unsampled"]


def test_committed_traffic_follows_the_source_hash():
    from paper_2010_01628_gb300 import build
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        stored = json.load(fh)["fluid_step_direct_fp32_512"]
    got = bench.committed_traffic("fluid_step_direct_fp32_512")
    if stored["source_sha"] == build.source_hash("fluid"):
        assert got == stored["dram_bytes_per_launch"]
        # the counters cover the algorithmic bytes to within a few per cent
        assert abs(got / bench.algorithmic_bytes(512, "fp32") - 1) < 0.05
    else:
        assert got is None
    assert bench.committed_traffic("no_such_kernel") is None


def test_warm_start_record_is_the_study_summary():
    rec = bench.warm_start_record()
    assert rec is not None and "cases" not in rec and "loss_history" not in rec
    assert rec["provenance"].startswith("recorded")
    assert rec["grid"] == 128 and rec["heldout"] == 32 and rec["train_states"] == 512
    assert 0 < rec["mean_time_reduction"] < 1 and rec["warm_mean_s"] < rec["cold_mean_s"]


def test_committed_weights_match_the_network():
    pytest.importorskip("torch")
    from paper_2010_01628_gb300 import binding as L
    from paper_2010_01628_gb300 import surrogate as S
    w, meta = S.load_weights(bench.WARM_WEIGHTS)
    assert w.dtype == np.float32 and w.size == L.lbm_cnn_param_count()
    assert np.all(np.isfinite(w))
    assert meta["grid"] == 128 and meta["train_count"] == 512 and meta["heldout_count"] == 32
    assert meta["tol"] == 1e-6 and meta["reynolds_seed"] == 4


def test_solver_judges_the_network():
    """surrogate.judge: the prediction against the cold run's converged fields
    (u against ||u_cold||, rho against ||rho_cold - 1||) and the warm run's
    final fields against the cold run's."""
    torch = pytest.importorskip("torch")
    from paper_2010_01628_gb300 import surrogate as S
    g = torch.Generator().manual_seed(0)
    rc = 1.0 + 1e-3 * torch.randn(6, 5, 4, generator=g, dtype=torch.float64)
    uc = 0.05 * torch.randn(3, 6, 5, 4, generator=g, dtype=torch.float64)
    same = S.judge((rc, uc), (rc, uc), (rc, uc))
    assert all(v == 0.0 for v in same.values())
    # the rest state as a prediction: u error 1, rho error 1 (rho - 1 = 0 everywhere)
    rest = S.judge((torch.ones_like(rc), torch.zeros_like(uc)), (rc, uc), (rc, uc))
    assert abs(rest["net_err_u"] - 1.0) < 1e-15 and abs(rest["net_err_rho"] - 1.0) < 1e-15
    # a warm run ending 1% off in u and 2% off in rho - 1
    r = S.judge((rc, uc), (rc, uc), (1.0 + 1.02 * (rc - 1.0), 1.01 * uc))
    assert abs(r["warm_vs_cold_u"] - 0.01) < 1e-12 and abs(r["warm_vs_cold_rho"] - 0.02) < 1e-9
