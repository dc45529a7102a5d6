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
    seg = int(t["plan"]["segments"])
    assert bench._traffic_per_iteration(E, 25, seg) == float(t["dram_bytes_per_edge"]) * E
    assert bench._traffic_per_iteration(E, 25, seg + 1) is None  # another plan than profiled
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


def test_parity_report_flags_a_planted_error():
    import bench
    import oracle as O
    g = graphgen.rmat(10, 16, seed=2)
    want, bound = O.pagerank_bound(g.offsets, g.src, iters=20)
    ok = bench.parity_report(want.astype(np.float32), want, bound)
    assert ok["ok"] and ok["vertices_outside_bound"] == 0 and ok["rel_l1"] < 1e-6
    bad = want.astype(np.float32)
    bad[17] *= np.float32(1.001)  # one vertex 0.1% off: inside any global L1 budget
    rep = bench.parity_report(bad, want, bound)
    assert rep["rel_l1"] <= 1e-5 and rep["vertices_outside_bound"] == 1 and not rep["ok"]


def test_reference_arm_times_iterations_net_of_setup(capsys):
    """--impl reference reports one oracle iteration per step, timed inside the
    oracle, on the same routine as the cpu_baseline leg."""
    import bench

    class A:
        scale, steps, warmup, gpus = 12, 3, 1, 1
    bench.run_reference(A())
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "GTEPS"
    assert line["cpu_baseline"]["value"] == line["value"] and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0
