"""Host-side helpers of bench.py: the default start of the implicit solves,
the configuration the measured DRAM traffic belongs to, and the algorithmic
flop count behind the roofline figure."""
import argparse
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _args(**kw):
    base = dict(workload="nai", guess=None, precision="fp64", solver="lanczos")
    base.update(kw)
    return argparse.Namespace(**base)


def test_default_start_is_euler():
    assert bench._guess(_args()) == 0 and bench._guess_name(_args()) == "euler"
    assert bench._guess(_args(workload="2d")) == 0
    assert bench._guess(_args(workload="batched")) == 0
    assert bench._guess(_args(guess="zero")) == 1 and bench._guess_name(_args(guess="zero")) == "zero"


def test_traffic_only_for_the_measured_configuration_and_sources(tmp_path, monkeypatch):
    import json
    rec = tmp_path / "traffic.json"
    monkeypatch.setattr(bench, "TRAFFIC_RECORD", str(rec))
    assert bench._traffic(_args(), 152) is None                      # no record
    rec.write_text(json.dumps({"sources_sha16": bench.kernel_sources_sha16(), "dram_bytes_per_launch": 1.5e10,
                               "surfaces_per_fft": 1}))
    assert bench._traffic(_args(), 152) == 1.5e10
    assert bench._traffic(_args(), 152, {"surfaces_per_fft": 1}) == 1.5e10
    assert bench._traffic(_args(), 152, {"surfaces_per_fft": 0}) is None   # another launch shape
    assert bench._traffic(_args(precision="mixed"), 152) is None
    assert bench._traffic(_args(solver="gmres"), 152) is None
    assert bench._traffic(_args(guess="zero"), 152) is None
    assert bench._traffic(_args(), 64) is None
    rec.write_text(json.dumps({"sources_sha16": "0" * 16, "dram_bytes_per_launch": 1.5e10}))
    assert bench._traffic(_args(), 152) is None                      # kernel changed since the capture


def test_flop_count_by_hand():
    N, S = 1024, 2
    st = dict(n_hpsi=3, n_ortho=5, n_krylov=2, n_update=4, n_outer=1)
    hpsi = 4 * S * 5 * N * 10 + (4 * S * S + 10 * S) * N
    want = 3 * hpsi + 5 * 2 * 16 * S * N + 2 * 6 * S * N + 4 * 8 * S * N
    assert math.isclose(bench._flops_per_launch([st], N, S), want, rel_tol=1e-15)
    want_mixed = 3 * hpsi + 1 * 8 * S * N
    assert math.isclose(bench._flops_per_launch([st], N, S, mixed=True), want_mixed, rel_tol=1e-15)
    assert math.isclose(bench._flops_per_launch([st, st], N, S), 2 * want, rel_tol=1e-15)
