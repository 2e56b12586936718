"""The multi-rank host logic of bench.py on CPU: two `gloo` ranks shard an
ensemble of configurations (each configuration on exactly one rank, no
data-path collective) and combine their timings into one whole-job
throughput (entries summed over ranks, time = the slowest rank)."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, outdir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        mine = bench.shard_configs(16, rank, world)
        entries = 2016.0 * len(mine)            # C entries per step of this rank's configurations
        ms = 100.0 + 50.0 * rank                # this rank's timed region
        value, all_entries, ms_max = bench.job_throughput(entries, ms, 3, dist)
        # each rank's configurations' C (here filled with the configuration
        # number) reach rank 0 in configuration order
        import torch
        local = {c: torch.full((2, 3, 3, 4), complex(c, -c), dtype=torch.complex128) for c in mine}
        got = bench.gather_C(local, 16, dist)
        gathered = None if got is None else [float(x.real.flat[0]) for x in got]
        with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
            json.dump({"mine": mine, "value": value, "all": all_entries, "ms": ms_max, "gathered": gathered}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_combine(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    shards = [set(r["mine"]) for r in res]
    assert shards[0].isdisjoint(shards[1]) and shards[0] | shards[1] == set(range(16))
    total = 2016.0 * 16
    for r in res:   # every rank agrees on the whole-job numbers
        assert r["all"] == total and r["ms"] == 150.0
        assert r["value"] == pytest.approx(total * 3 / 0.150)
    assert res[0]["gathered"] == [float(c) for c in range(16)] and res[1]["gathered"] is None


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.shard_configs(5, 0, 1) == [0, 1, 2, 3, 4]
    assert bench.shard_configs(5, 2, 4) == [2]
    value, all_entries, ms = bench.job_throughput(100.0, 200.0, 4)
    assert (all_entries, ms) == (100.0, 200.0) and value == pytest.approx(100 * 4 / 0.2)
    import torch
    local = {c: torch.full((1,), float(c)) for c in (2, 0, 1)}
    assert [float(t[0]) for t in bench.gather_C(local, 3)] == [0.0, 1.0, 2.0]


def _rank_timeslices(rank, world, port, outdir):
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        nt = 10
        mine = bench.shard_timeslices(nt, rank, world, 7)        # 5 distinct timeslices, two repeated
        C = np.zeros((2, 3, 3, nt), dtype=np.complex128)
        for t in mine:                                          # this rank fills only its columns
            C[..., t] = complex(t, rank)
        got = bench.gather_columns(C, [0] + mine, dist)         # every rank also computed t = 0 itself
        value, all_entries, ms_max = bench.job_throughput(2 * 9.0, 100.0 + 10 * rank, 7, dist)
        res = {"mine": mine, "all": all_entries, "ms": ms_max,
               "cols": None if got is None else {str(t): [c.real.flat[0], c.imag.flat[0]] for t, c in got.items()}}
        with open(os.path.join(outdir, f"ts{rank}.json"), "w") as f:
            json.dump(res, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_one_configuration_by_timeslice(tmp_path):
    """One configuration split over ranks by timeslice: rank r takes t = r
    mod N, the columns of C reach rank 0 after the run (each from the rank
    that computed it), and the job throughput sums the ranks' entries over
    the slowest rank's time."""
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_timeslices, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"ts{r}.json")) for r in range(world)]
    assert res[0]["mine"] == [0, 2, 4, 6, 8, 0, 2] and res[1]["mine"] == [1, 3, 5, 7, 9, 1, 3]
    cols = res[0]["cols"]
    assert sorted(int(t) for t in cols) == list(range(10))
    for t, (re, im) in cols.items():
        t = int(t)
        if t == 0:
            continue                      # every rank has a t = 0 column; the last gathered wins
        assert re == t and im == t % 2
    assert res[1]["cols"] is None
    assert res[0]["all"] == res[1]["all"] == 36.0 and res[0]["ms"] == 110.0
