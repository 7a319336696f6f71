"""Splitting a batch across ranks (cells are independent, no exchange): the
longest-processing-time split covers every cell once, is the same on every
rank, and keeps the ranks' loads within one cell of each other's greedy bound;
two gloo ranks agree on it without communicating it."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1810_12742_gb300 import inputs as I
from paper_1810_12742_gb300 import shard as S


def _check_cover(ncomp, parts):
    allc = np.concatenate(parts)
    assert np.array_equal(np.sort(allc), np.arange(len(ncomp)))
    for p in parts:
        assert np.all(np.diff(p) > 0)


@pytest.mark.parametrize("n_parts", [1, 2, 3, 8])
def test_lpt_covers_and_balances(n_parts):
    rng = np.random.default_rng(4)
    ncomp = np.concatenate([rng.integers(200, 3000, 700), rng.integers(30000, 200000, 300)])
    parts = S.lpt_partition(ncomp, n_parts)
    _check_cover(ncomp, parts)
    loads = S.shard_loads(ncomp, parts)
    assert loads.sum() == ncomp.sum()
    # greedy rule: the last cell placed on the fullest part went to the least loaded
    # part at that time, so max - min <= the largest cell
    assert loads.max() - loads.min() <= ncomp.max()
    assert loads.max() <= ncomp.sum() / n_parts + ncomp.max()


def test_lpt_small_cases():
    assert [p.tolist() for p in S.lpt_partition([5, 3, 3, 2], 2)] == [[0, 3], [1, 2]]
    assert [p.tolist() for p in S.lpt_partition([], 3)] == [[], [], []]
    assert [p.tolist() for p in S.lpt_partition([1, 1], 4)] == [[0], [1], [], []]
    # ties by index, then by rank
    assert [p.tolist() for p in S.lpt_partition([4, 4, 4, 4], 2)] == [[0, 2], [1, 3]]
    with pytest.raises(ValueError):
        S.lpt_partition([1], 0)


def test_uneven_population_split():
    w = I.WORKLOADS["uneven_mixed"]
    ncomp, _ = I.population_trees(w, np.arange(400))
    parts = S.lpt_partition(ncomp, 4)
    _check_cover(ncomp, parts)
    loads = S.shard_loads(ncomp, parts)
    assert loads.max() / loads.mean() < 1.02


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ncomp = np.random.default_rng(9).integers(10, 5000, 301)
        mine = S.lpt_partition(ncomp, world)[rank]
        sizes = [None] * world
        dist.all_gather_object(sizes, mine.tolist())  # test only: check the ranks' splits fit together
        out[rank] = sizes
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_split_without_exchange():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    assert out[0] == out[1]
    _check_cover(np.zeros(301), [np.array(p) for p in out[0]])
