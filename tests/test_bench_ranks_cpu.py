"""The N > 1 host logic of bench.py on CPU ranks (gloo, world size 2): every
GPU runs an independent replica, so the only cross-rank step is the timing
reduction (the slowest rank's time, max over ranks) and the whole-job rate
(all ranks' units over that time); the reference arm runs on rank 0 alone."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # rank r took r + 1 seconds for 1000 units
        rate, slowest = bench.job_rate(1000, rank + 1.0, world, "cpu")
        out[rank] = (rate, slowest)
        torch.distributed.barrier()
    finally:
        torch.distributed.destroy_process_group()


def test_job_rate_is_all_units_over_the_slowest_rank():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        rate, slowest = res[r]
        assert slowest == 2.0                       # max over ranks, seen by every rank
        assert rate == pytest.approx(2000 / 2.0)    # units of both ranks over the slowest time


def test_job_rate_single_rank_needs_no_process_group():
    import bench
    rate, slowest = bench.job_rate(300, 1.5, 1, "cpu")
    assert slowest == 1.5 and rate == pytest.approx(200.0)


def test_reference_arm_prints_on_rank_zero_only():
    """Under torchrun the reference arm's other ranks exit without work or output."""
    import bench
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.reference_arm(None, rank=1, world=2)  # returns before reading its arguments
    assert buf.getvalue() == ""
