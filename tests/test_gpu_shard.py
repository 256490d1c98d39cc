"""Block sharding of one field against the oracle (axis-0 slabs refactored
independently, planned together for whole-field targets).

* ShardedField on this GPU: the slabs' streams equal the oracle's slab
  refactors; the global plans (relative error bound, PSNR) equal
  oracle.shard.plan_global's plan for plan; the assembled retrieval equals
  the oracle's bit for bit and meets the whole-field target; one slab gives
  the plain plan.
* Planning states: handles imported from export_plan_state plan exactly as
  the live handles; an imported handle refuses retrieval.
* Two processes (gloo over the host, both on this GPU -- their kernels
  never wait on each other), each holding some slabs, plan through
  distributed_plans and get the single-process plans.
"""
import math
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SCH = dict(interp="level", degree="cubic", decomp_axis=2)
SHAPE = (30, 34, 44)
TARGETS = [("rel", 1e-3), ("rel", 1e-5), ("psnr", 60.0), ("psnr", 90.0)]


def _field():
    from synth import grf
    return grf(SHAPE, 501, np.float32)


@pytest.mark.parametrize("k", [1, 3])
def test_sharded_field_matches_the_oracle(k):
    import oracle
    from oracle import shard as oshard
    import paper_2609_04573_b300 as pcr
    from paper_2609_04573_b300.shard import ShardedField
    from _compare import oracle_scheme, compare_streams
    X = _field()
    sch = pcr.Scheme(**SCH)
    sf = ShardedField(torch.from_numpy(X).cuda(), k, sch)
    hs_or, sl = oshard.refactor_blocks(X, oracle_scheme(sch, 3), k)
    assert [tuple(s) for s in sf.slabs] == [tuple(s) for s in sl]
    for h, ho in zip(sf.handles, hs_or):
        compare_streams(h, ho)
    R = float(X.max()) - float(X.min())
    for kind, v in TARGETS:
        pls, bound, ok = sf.plan(pcr.Target(kind, v))
        pls_or, bound_or, ok_or = oshard.plan_global(hs_or, oracle.Target(kind, v))
        assert ok == ok_or and [p.planes for p in pls] == [p["b"] for p in pls_or], (kind, v)
        if k == 1:
            assert pls[0].planes == sf.handles[0].plan(pcr.Target(kind, v), allow_unsat=True).planes
        out = sf.retrieve(pls).cpu().numpy()
        Y = oshard.retrieve_blocks(hs_or, sl, pls_or, X.shape, X.dtype)
        assert np.array_equal(out, Y), (kind, v)
        d = out.astype(np.float64) - X.astype(np.float64)
        if ok and kind == "rel":
            assert float(np.abs(d).max()) <= v * R
        elif ok:
            mse = float(np.mean(d * d))
            assert mse == 0 or 20 * math.log10(R / math.sqrt(mse)) >= v


def test_imported_plan_states_plan_like_live_handles():
    import paper_2609_04573_b300 as pcr
    from paper_2609_04573_b300.shard import ShardedField
    sf = ShardedField(torch.from_numpy(_field()).cuda(), 3, pcr.Scheme(**SCH))
    imp = [pcr.import_plan_state(h.export_plan_state(), h.shape) for h in sf.handles]
    for kind, v in TARGETS:
        a, ba, oa = sf.plan(pcr.Target(kind, v))
        b, bb, ob = pcr.plan_global(imp, pcr.Target(kind, v))
        assert [p.planes for p in a] == [p.planes for p in b] and ba == bb and oa == ob
        assert imp[0].plan(pcr.Target(kind, v), allow_unsat=True).planes == \
            sf.handles[0].plan(pcr.Target(kind, v), allow_unsat=True).planes
    with pytest.raises(pcr.PcrError) as ei:
        imp[0].retrieve(imp[0].plan(pcr.Target("rel", 1e-3)), out=torch.empty(imp[0].shape, device="cuda"))
    assert ei.value.status == pcr.ERR_UNSUPPORTED


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import paper_2609_04573_b300 as pcr
        from paper_2609_04573_b300.shard import slabs, distributed_plans
        X = _field()
        sl = slabs(X.shape[0], 3)
        mine = [0, 2] if rank == 0 else [1]
        local = [(i, pcr.refactor(torch.from_numpy(np.ascontiguousarray(X[sl[i][0]:sl[i][1]])).cuda(),
                                  pcr.Scheme(**SCH))) for i in mine]
        res = {}
        for kind, v in TARGETS:
            plans, bound, ok = distributed_plans(local, pcr.Target(kind, v))
            res[(kind, v)] = ({i: p.planes for i, p in plans.items()}, bound, ok)
        q.put((rank, res))
    finally:
        dist.destroy_process_group()


def test_two_ranks_plan_like_one_process():
    import torch.multiprocessing as mp
    import paper_2609_04573_b300 as pcr
    from paper_2609_04573_b300.shard import ShardedField
    sf = ShardedField(torch.from_numpy(_field()).cuda(), 3, pcr.Scheme(**SCH))
    want = {}
    for kind, v in TARGETS:
        pls, bound, ok = sf.plan(pcr.Target(kind, v))
        want[(kind, v)] = ([p.planes for p in pls], bound, ok)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = dict(q.get(timeout=300) for _ in range(2))
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    for key, (planes, bound, ok) in want.items():
        for rank in (0, 1):
            gp, gb, gok = got[rank][key]
            assert gb == bound and gok == ok
            for i, pl in gp.items():
                assert pl == planes[i], (rank, key, i)
