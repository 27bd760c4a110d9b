"""The N > 1 path of bench.py on CPU (world size 2, gloo): replicas only, no
collective on the data path, so the host logic is the rank roles, the max over
ranks of the timed region and the whole-job time per registration."""

import argparse
import contextlib
import io
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.dist_setup()
        t_max = bench.reduce_max(10.0 + 5.0 * rank)          # rank 1 is the slowest replica
        out[rank] = (w, r, local, t_max, bench.per_registration(t_max, 4, w))
        # the reference arm: rank 0 alone does the work, the others return at once
        args = argparse.Namespace(size=32, warmup=0, steps=0, gpus=world)
        if rank != 0:
            buf = io.StringIO()
            with contextlib.redirect_stdout(buf):
                bench.run_reference(args, w, r)
            assert buf.getvalue() == ""
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_timed_region():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        w, r, local, t_max, per_reg = res[rank]
        assert (w, r, local) == (world, rank, rank)
        assert t_max == 15.0
        assert per_reg == pytest.approx(15.0 / (4 * world))


def test_single_process_needs_no_process_group():
    assert not dist.is_initialized()
    assert bench.reduce_max(3.5) == 3.5
    assert bench.per_registration(12.0, 3, 1) == pytest.approx(4.0)
