"""The N-GPU host logic of bench.py on two CPU ranks (gloo, 127.0.0.1).

An N-GPU run gives each rank an independent replica set (the same start,
Monte Carlo seeds offset by rank) and combines the ranks' numbers without any
data-path collective: the whole-job time is the slowest rank's, the work is
the sum.  These tests run that logic on two gloo ranks, and run the oracle
chain on each rank to check that the rank offset gives independent chains.
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle
        from paper_2506_21290_gb300 import workloads as W

        wl = bench.make_workload("tiny-64", rank)
        # each rank runs its own chain: one oracle sweep with the rank's seed
        oracle.build()
        ch = oracle.Chain(wl["L"], wl["xyz"], wl["types"], W.PAPER_POT, nc=2)
        ch.run(1, wl["T"], W.PAPER_MIX, seed=int(wl["seeds"]))
        # rank r took 10 + r ms for 100 (r + 1) attempts and 7 (r + 1) pair evaluations
        ms, att, pairs = bench.combine_ranks(10.0 + rank, 100 * (rank + 1), 7 * (rank + 1), dist, "cpu")
        np.savez(os.path.join(out_dir, "rank%d.npz" % rank), seed=int(wl["seeds"]), q=ch.q,
                 combined=np.array([ms, att, pairs]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_and_run_independent_replicas(tmp_path):
    import oracle
    oracle.build()              # once, before the ranks start
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r0 = np.load(tmp_path / "rank0.npz")
    r1 = np.load(tmp_path / "rank1.npz")
    # whole-job numbers: max time, summed work, the same on every rank
    for r in (r0, r1):
        assert r["combined"].tolist() == [11.0, 300.0, 21.0]
    # independent replica sets: different seeds, different chains from the same start
    assert int(r0["seed"]) != int(r1["seed"])
    assert not np.array_equal(r0["q"], r1["q"])


def test_single_rank_combine_is_the_identity():
    import bench
    assert bench.combine_ranks(12.5, 40, 9) == (12.5, 40.0, 9.0)


def _ensemble_rank(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import correlation as OC
        from paper_2506_21290_gb300 import ensemble as E
        rng = np.random.default_rng(100 + rank)
        M = 20
        ss = [(rng.uniform(-0.3, 1, 3 * M), rng.uniform(-0.2, 1, M), rng.uniform(-0.5, 1, M)) for _ in range(3)]
        res = E.ensemble_results(OC.sums_of_samples(ss), 3 * M, dist)
        np.savez(os.path.join(out_dir, "ens%d.npz" % rank), res=res)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_ensemble_over_two_gloo_ranks_equals_the_pooled_samples(tmp_path):
    """Each rank holds its own samples; the all-reduced sums give the
    statistics of all samples together (the oracle's, on the pooled list)."""
    from oracle import correlation as OC
    from paper_2506_21290_gb300 import build as B
    B.build()
    port = _free_port()
    mp.start_processes(_ensemble_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r0 = np.load(tmp_path / "ens0.npz")["res"]
    r1 = np.load(tmp_path / "ens1.npz")["res"]
    assert np.array_equal(r0, r1)
    pooled = []
    for rank in range(2):
        rng = np.random.default_rng(100 + rank)
        pooled += [(rng.uniform(-0.3, 1, 60), rng.uniform(-0.2, 1, 20), rng.uniform(-0.5, 1, 20)) for _ in range(3)]
    want = OC.stats_of_samples(pooled)
    assert r0[0] == 6
    assert np.allclose(r0[1:], want[1:], rtol=0, atol=1e-10)
