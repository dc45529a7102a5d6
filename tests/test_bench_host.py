"""Host logic of bench.py (no GPU): the PPR seeds and segment bounds, the
traffic summary's gating, the measured-ceiling helper and the source hash."""
import json
import os

import numpy as np

import graphgen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_ppr_seeds_distinct_with_out_edges_and_deterministic():
    import bench
    g = graphgen.rmat(12, 16, seed=1)
    s1, s2 = bench.ppr_seeds(g), bench.ppr_seeds(g)
    assert np.array_equal(s1, s2) and s1.dtype == np.int32
    assert len(s1) == 64 and len(set(s1.tolist())) == 64
    outdeg = np.bincount(g.src, minlength=g.V)
    assert np.all(outdeg[s1] > 0)
    assert not np.array_equal(s1, bench.ppr_seeds(g, seed=2))


def test_ppr_bounds_cover_the_vertex_range():
    import bench
    for nd, V, k in ((1000, 1500, 8), (1000, 1000, 3), (7, 10, 16), (5, 5, 1)):
        b = bench._ppr_bounds(nd, V, k)
        assert b[0] == 0 and b[-1] == V and np.all(np.diff(b) > 0)
        assert nd in b  # the edgeless tail [nd, V) is a segment of its own
        assert len(b) - 1 <= k + 1


def test_traffic_summary_is_gated_by_workload_and_sources(monkeypatch):
    import bench
    with open(os.path.join(ROOT, "profiles", "pagerank_iteration_rmat25_traffic.json")) as f:
        t = json.load(f)
    E = 1000
    assert bench._traffic_per_iteration(E, scale=20) is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: t["kernel_source_sha"])
    assert bench._traffic_per_iteration(E) == float(t["dram_bytes_per_edge"]) * E
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench._traffic_per_iteration(E) is None


def test_kernel_source_hash_is_stable():
    import bench
    h = bench.kernel_source_hash()
    assert h == bench.kernel_source_hash() and len(h) == 16
    int(h, 16)


def test_gather_peaks_keys_and_units():
    import bench

    class FakeC:
        def measure_row_gather(self, rb, tb):
            return 1e9 * rb

        def measure_smem_lookups(self):
            return 3e12

    p = bench.gather_peaks(FakeC(), [(4, 64), (128, 1 << 20)], smem=True)
    assert p[(4, 64)] == 4.0 and p[(128, 1 << 20)] == 128.0 and p["smem"] == 3000.0
    assert "smem" not in bench.gather_peaks(FakeC(), [(4, 64)])
