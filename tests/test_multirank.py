"""The multi-rank host logic of bench.py on CPU (gloo, world size 2): the
timed region is the maximum over the ranks, and the whole-job value counts
every rank's field.  Each rank refactors its own field (weak scaling), so
no data-path collective exists to test beyond this reduction."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(3.0 + 2.0 * rank, world, torch.device("cpu"))
    out[rank] = (ms, bench.whole_job_gbs(512 << 20, world, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 5.0            # the slower rank's time
    want = 2 * 2 * (512 << 20) / 5e-3 / 1e9          # both ranks' fields in that time
    assert abs(res[0][1] - want) < 1e-9 and res[0][1] == res[1][1]


def test_single_rank_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(4.25, 1, None) == 4.25
    assert bench.whole_job_gbs(100, 1, 1.0) == 2 * 100 / 1e-3 / 1e9
