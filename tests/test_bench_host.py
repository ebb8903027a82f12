"""Host logic of bench.py that needs no GPU: the CPU baseline over all host
cores for a batch of replicas (one oracle chain per core, spawned workers)."""
import bench
from paper_2506_21290_gb300 import workloads as W


def test_all_core_cpu_baseline_runs_one_replica_per_core():
    wl = bench.make_workload("batched-256")
    # keep the test short: the first two replicas only
    k = 2
    n3 = 3 * wl["n_mol"][:k]
    wl = dict(wl, replicas=k, n_mol=wl["n_mol"][:k], L=wl["L"][:k], T=wl["T"][:k], seeds=wl["seeds"][:k],
              xyz=wl["xyz"][:n3.sum()], types=wl["types"][:n3.sum()])
    out = bench.cpu_baseline(wl, "batched-256", 0.2, None, W.PAPER_MIX)
    assert out["kind"] == "oracle" and out["unit"] == bench.UNIT
    assert 1 <= out["cores"] <= k
    assert out["value"] > 0
    assert "one per core" in out["sample"]


def test_cells_per_axis_matches_the_library_rule():
    # n_c = 2, 4, 8, 10, 16, 34 at M = 64, 256, 1000, 2000, 8000, 64000 (rho = 1.2)
    for M, nc in ((64, 2), (256, 4), (1000, 8), (2000, 10), (8000, 16), (64000, 34)):
        assert bench._cells_per_axis(W.box_length(M)) == nc
