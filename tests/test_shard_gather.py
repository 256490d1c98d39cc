"""Host side of the distributed block-sharding path on CPU (gloo, world
size 2): every rank contributes the planning states of the slabs it holds;
gather_states returns all of them, sorted by slab id, identically on every
rank; a slab numbered twice is refused."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q, dup):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2609_04573_b300.shard import gather_states
        # rank 0 holds slabs 0 and 3, rank 1 slabs 1 and 2 (or slab 0 again)
        ids = [0, 3] if rank == 0 else ([1, 2] if not dup else [1, 0])
        items = [(i, bytes([i]) * (i + 1), (i + 2, 5, 6)) for i in ids]
        try:
            q.put((rank, gather_states(items)))
        except ValueError as e:
            q.put((rank, "refused: " + str(e)))
    finally:
        dist.destroy_process_group()


def _run(dup):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q, dup)) for r in range(2)]
    for p in ps:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    return got


def test_states_gathered_in_slab_order_on_every_rank():
    pytest.importorskip("paper_2609_04573_b300")
    got = _run(dup=False)
    want = [(i, bytes([i]) * (i + 1), (i + 2, 5, 6)) for i in range(4)]
    assert got[0] == want and got[1] == want


def test_a_slab_numbered_twice_is_refused():
    pytest.importorskip("paper_2609_04573_b300")
    got = _run(dup=True)
    assert all(isinstance(v, str) and v.startswith("refused") for v in got.values())
