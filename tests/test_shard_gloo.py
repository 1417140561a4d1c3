"""Multi-rank batch sharding on CPU: world_size 2 over gloo.

Each rank takes its cost-balanced contiguous slice of a ragged batch,
computes its objects' peaks (here with the CPU oracle, as no GPU is assumed),
and the peaks are gathered on rank 0.  The gathered result must equal the
single-process result object for object.  No collective touches the data
path; the gather carries only the peak records.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import synth
from paper_2105_04006_gb300 import shard

GRID = synth.Grid(0.24, 12.0, 1500)


def _batch():
    return synth.ragged_survey(37, seed=12, grid=GRID)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _peaks_of(t, y, off):
    import oracle
    from paper_2105_04006_gb300 import PEAK_DTYPE
    res = oracle.lsp_batch(t, y, off, GRID.f_min, GRID.f_max, GRID.n_f)
    pk = np.zeros(off.size - 1, dtype=PEAK_DTYPE)
    pk["idx"] = res["arg_idx"]
    pk["power"] = res["arg_pow"]
    pk["flags"] = res["flags"]
    return pk


def _worker(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = _batch()
    ranges = shard.shard_ranges(b.offsets, world)
    a, e = ranges[rank]
    t, y, off = shard.local_slice(b.t, b.y, b.offsets, a, e)
    local = _peaks_of(t, y, off)
    full = shard.gather_peaks(local, ranges, rank)
    if rank == 0:
        np.save(out_path, full)
    dist.barrier()
    dist.destroy_process_group()


def test_shard_ranges_balance_and_cover():
    b = _batch()
    for world in (1, 2, 3, 8, 50):
        rs = shard.shard_ranges(b.offsets, world)
        assert len(rs) == world and rs[0][0] == 0 and rs[-1][1] == b.n_obj
        assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
        if world <= 3:
            cost = [int(b.offsets[e] - b.offsets[a]) for a, e in rs]
            # each cut lies within one object of its ideal position
            assert max(cost) - min(cost) <= 2 * int(b.n_t.max())


def test_two_rank_gather_equals_single_process(tmp_path):
    import oracle
    oracle.build()
    out = str(tmp_path / "peaks.npy")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    got = np.load(out)
    b = _batch()
    ref = _peaks_of(b.t, b.y, b.offsets)
    np.testing.assert_array_equal(got["idx"], ref["idx"])
    np.testing.assert_array_equal(got["power"], ref["power"])
