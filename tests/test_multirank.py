"""The N > 1 bench path on CPU: two gloo ranks.  Each rank draws its own
queries against an identical library (weak scaling over query batches, no
data-path collective), and the whole-job figures are the slowest rank's time
and the sum of the ranks' work."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        refs, queries, spec = bench.workload(0.002, rank)
        # this rank's step: pretend it took (rank + 1) * 10 ms for (rank + 1) * 1000 comparisons
        sec, units = bench.reduce_over_ranks(0.01 * (rank + 1), 1000 * (rank + 1))
        out[rank] = {"refs_mz": refs.precursor_mz.copy(), "q_mz": queries.precursor_mz.copy(),
                     "sec": sec, "units": units}
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        r = dict(out)
    assert np.array_equal(r[0]["refs_mz"], r[1]["refs_mz"])          # replicated library
    assert not np.array_equal(r[0]["q_mz"], r[1]["q_mz"])             # each rank its own queries
    for k in range(world):
        assert r[k]["sec"] == pytest.approx(0.02)                     # slowest rank
        assert r[k]["units"] == 3000                                  # all ranks' work


def test_single_process_passthrough():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(0.5, 7) == (0.5, 7)
