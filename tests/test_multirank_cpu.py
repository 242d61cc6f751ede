"""Sharding across ranks on the CPU (gloo, world size 2): each rank traces
its share of the tracks with the oracle and the per-pixel counts are summed
with an all-reduce; the result equals one process tracing every track (the
keyed random numbers make photons independent of the sharding)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, result_path):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2309_12496_gb300 import workloads as W
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = W.batched(32, seed=2)
    sc = oracle.Scene(wl.scene)
    prm = oracle.params(wl, n_threads=1)
    _, _, off = oracle.track_yield(wl.tracks, prm)
    # shard by event: rank r takes events r, r + world, ...
    ev_of_track = wl.tracks.event
    mine = np.zeros(32 * sc.pixels_per_event, np.int64)
    sums = np.zeros((32, sc.n_planes, 4))
    for e in range(rank, 32, world):
        idx = np.nonzero(ev_of_track == e)[0]
        if len(idx) == 0:
            continue
        r = sc.trace(wl.tracks, prm, offsets=off, track_range=(int(idx[0]), int(idx[-1]) + 1),
                     n_hist_events=32)
        mine += r["pixel_counts"].reshape(-1).astype(np.int64)
        sums += r["event_sums"]
    t = torch.from_numpy(mine)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    s = torch.from_numpy(sums)
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    if rank == 0:
        np.savez(result_path, counts=t.numpy(), sums=s.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_equals_single_process(tmp_path, oracle_lib):
    from paper_2309_12496_gb300 import workloads as W
    path = str(tmp_path / "res.npz")
    mp.start_processes(_rank_main, args=(2, _free_port(), path), nprocs=2, join=True,
                       start_method="spawn")
    res = np.load(path)
    wl = W.batched(32, seed=2)
    sc = oracle_lib.Scene(wl.scene)
    ref = sc.trace(wl.tracks, oracle_lib.params(wl), n_hist_events=32)
    np.testing.assert_array_equal(res["counts"], ref["pixel_counts"].reshape(-1).astype(np.int64))
    np.testing.assert_allclose(res["sums"], ref["event_sums"], rtol=1e-12)
    assert res["counts"].sum() > 100
