"""Host-side arithmetic of the benchmark (no GPU): the means behind the reported
GTEPS, the open-loop arrival trace of the serving run and its latency summary,
and the workload descriptions."""
import math

import numpy as np
import pytest

import bench


def test_means_match_scipy():
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(7)
    xs = list(rng.uniform(50.0, 900.0, 64))
    assert bench.hmean(xs) == pytest.approx(float(stats.hmean(xs)), rel=1e-12)
    assert bench.gmean(xs) == pytest.approx(float(stats.gmean(xs)), rel=1e-12)
    # non-positive entries (a run that traversed nothing) are left out
    assert bench.hmean(xs + [0.0]) == pytest.approx(bench.hmean(xs), rel=1e-12)
    assert bench.hmean([]) == 0.0 and bench.gmean([]) == 0.0
    # the harmonic mean of rates is total work over total time for equal work per run
    t = rng.uniform(0.1, 2.0, 16)
    assert bench.hmean(list(1.0 / t)) == pytest.approx(len(t) / t.sum(), rel=1e-12)


def test_serve_trace_is_seeded_poisson():
    rate, count = 4000, 20000
    a = bench.serve_trace(rate, count, n_graphs=5, n_sources=1024, seed=4000)
    b = bench.serve_trace(rate, count, n_graphs=5, n_sources=1024, seed=4000)
    assert a == b
    assert a != bench.serve_trace(rate, count, n_graphs=5, n_sources=1024, seed=4001)
    offs = np.array([x[0] for x in a], dtype=np.int64)
    gids = np.array([x[1] for x in a])
    idx = np.array([x[2] for x in a])
    assert len(a) == count
    assert np.all(np.diff(offs) >= 0)
    assert gids.min() >= 0 and gids.max() <= 4 and idx.min() >= 0 and idx.max() <= 1023
    # mean gap 1/rate (exponential gaps: relative standard error 1/sqrt(count))
    assert offs[-1] / count == pytest.approx(1e9 / rate, rel=5 / math.sqrt(count))
    # graphs drawn uniformly
    counts = np.bincount(gids, minlength=5)
    assert np.all(np.abs(counts - count / 5) < 5 * math.sqrt(count / 5))


def test_latency_summary():
    rng = np.random.default_rng(11)
    lat_ns = rng.integers(100_000, 5_000_000, 1000)
    s = bench.latency_summary(lat_ns, t_first=1_000_000_000, t_last=1_500_000_000, count=1000)
    assert s["queries"] == 1000
    assert s["qps"] == pytest.approx(2000.0)
    assert s["p50_ms"] == pytest.approx(np.percentile(lat_ns / 1e6, 50))
    assert s["p99_ms"] == pytest.approx(np.percentile(lat_ns / 1e6, 99))
    assert s["mean_ms"] == pytest.approx(lat_ns.mean() / 1e6)
    assert bench.latency_summary([1], 5, 5, 1)["qps"] is None


def test_workload_descriptions():
    for name, w in bench.WORKLOADS.items():
        c = bench.config_of(name, w)
        assert c["workload"] == name and c["n"] == 1 << w["scale"]
        assert c["sources"] == bench.N_SOURCES and c["alpha"] == 10 and c["schedule"] == "beamer_stay" and c["beta"] == 18
        if w["kind"] == "rmat":
            assert c["edge_factor"] == 16 and c["abcd"] == [0.57, 0.19, 0.19, 0.05]
        else:
            assert c["avg_degree"] == w["avgdeg"]
    assert bench.WORKLOADS["rmat22"]["scale"] == 22 and bench.WORKLOADS["rmat22"]["th"] == 64
