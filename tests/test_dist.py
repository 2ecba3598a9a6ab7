"""Row-partitioned sketch (the multi-GPU form of Algorithm 2's sketch step): the partition logic and
the single sum all-reduce, run as two gloo ranks on the CPU.  The ranks' partial sketches come
from the oracle, standing in for the device kernel (which the GPU tests check against the
same oracle)."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as tdist
import torch.multiprocessing as mp

from oracle import sketch
from paper_2104_05877_gb300 import dist


@pytest.mark.parametrize("m,world,align", [(1000, 2, 32), (8192, 8, 32), (37, 3, 32), (100, 4, 4), (5, 1, 4)])
def test_row_partition(m, world, align):
    parts = dist.row_partition(m, world, align)
    assert len(parts) == world
    r = 0
    for row0, rows in parts:
        assert row0 == r and rows >= 0
        if rows:
            assert row0 % align == 0
        r += rows
    assert r == m
    sizes = [rows for _, rows in parts if rows]
    assert max(sizes) - min(sizes) <= align


def test_partial_sketches_sum_to_the_sketch():
    """Gamma's columns depend only on their global index: the partial sketches of any row
    partition sum to the sketch of the whole matrix (Gaussian and sparse sign)."""
    rng = np.random.default_rng(3)
    A = rng.standard_normal((300, 40))
    l = 24
    for parts in (dist.row_partition(300, 3, 32), [(0, 4), (4, 196), (200, 100)]):
        g = sum(sketch.gaussian_sketch_rows(A[r0:r0 + mr], l, 7, r0) for r0, mr in parts)
        assert np.allclose(g, sketch.gaussian_sketch(A, l, 7), rtol=0, atol=1e-12 * np.abs(A).sum())
        s = sum(sketch.sparse_sign_sketch_rows(A[r0:r0 + mr], l, 6, 7, r0) for r0, mr in parts)
        assert np.allclose(s, sketch.sparse_sign_sketch(A, l, 6, 7), rtol=0, atol=1e-12 * np.abs(A).sum())


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, A, l, seed, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        row0, rows = dist.row_partition(A.shape[0], world, 32)[rank]
        part = sketch.gaussian_sketch_rows(A[row0:row0 + rows], l, seed, row0)
        X = dist.allreduce_partial(torch.from_numpy(part))
        out[rank] = X.numpy().copy()
    finally:
        tdist.destroy_process_group()


def test_gloo_two_ranks_allreduce():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((500, 30))
    l, seed, world = 20, 11, 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, _free_port(), A, l, seed, out), nprocs=world,
                           start_method="spawn")
        want = sketch.gaussian_sketch(A, l, seed)
        for r in range(world):
            assert np.allclose(out[r], want, rtol=0, atol=1e-12 * np.abs(A).sum())
