"""Block sharding of one field (Sec. VII: fixed blocks of a field refactored
independently, one per core) and its retrieval for whole-field targets.

ShardedField: a field split along axis 0 into contiguous slabs (the first
n0 mod k slabs one plane thicker), the slabs refactored together on this
GPU (pcr_refactor_batch), planned together for a whole-field target
(pcr_plan_global: error bounds relative to the whole field's range, PSNR
with one squared-error budget for the whole field) and retrieved into one
output (pcr_retrieve_batch_plan, each slab into its rows).

distributed_plans: slabs held by different ranks (one process per GPU).
Each rank exports the planning state of its slabs (statistics and tables,
no planes), the states are all-gathered over a torch.distributed group
(host bytes: any backend), every rank imports all of them and plans the
whole field with pcr_plan_global in slab order -- the same plans on every
rank -- and keeps the plans of its own slabs.  No field data crosses ranks.
"""
import torch
import torch.distributed as dist

from . import Scheme, import_plan_state, plan_global, refactor_batch, retrieve_batch


def slabs(n0, k):
    """Axis-0 slabs (start, stop) of n0 planes into k blocks."""
    if not 1 <= k <= n0:
        raise ValueError("need 1 <= k <= n0")
    out, a = [], 0
    for i in range(k):
        t = n0 // k + (1 if i < n0 % k else 0)
        out.append((a, a + t))
        a += t
    return out


class ShardedField:
    """A field refactored as k independent axis-0 slabs on this GPU."""

    def __init__(self, x, k, scheme=None, stream=None):
        if not (x.is_cuda and x.is_contiguous() and x.dim() in (2, 3)):
            raise ValueError("ShardedField expects a contiguous 2-D/3-D CUDA tensor")
        self.shape = tuple(x.shape)
        self.dtype = x.dtype
        self.device = x.device
        self.slabs = slabs(x.shape[0], k)
        self.handles = refactor_batch([x[a:b] for a, b in self.slabs], scheme or Scheme(), stream=stream)

    def plan(self, target):
        """(plans per slab, bound, satisfied) for a whole-field target."""
        return plan_global(self.handles, target)

    def retrieve(self, plans, out=None, stream=None):
        if out is None:
            out = torch.empty(self.shape, dtype=self.dtype, device=self.device)
        retrieve_batch(self.handles, plans, [out[a:b] for a, b in self.slabs], stream=stream)
        return out


def gather_states(items, group=None):
    """All-gather (slab id, state bytes, slab shape) tuples from every rank;
    returns them from all ranks sorted by slab id (the same list on every
    rank)."""
    world = dist.get_world_size(group)
    got = [None] * world
    dist.all_gather_object(got, list(items), group=group)
    allitems = [it for part in got for it in part]
    allitems.sort(key=lambda it: it[0])
    ids = [it[0] for it in allitems]
    if ids != list(range(len(ids))):
        raise ValueError(f"slab ids are not 0..{len(ids) - 1} exactly once: {ids}")
    return allitems


def distributed_plans(local, target, group=None):
    """Plans of this rank's slabs for a whole-field target.  `local`: list of
    (slab id, Handle) this rank holds; slab ids number all slabs of the
    field 0..n-1 along axis 0 across the ranks."""
    items = [(i, h.export_plan_state(), h.shape) for i, h in local]
    allitems = gather_states(items, group)
    hs = [import_plan_state(st, shape) for _, st, shape in allitems]
    plans, bound, ok = plan_global(hs, target)
    mine = {i for i, _ in local}
    out = {}
    for (i, _, _), p in zip(allitems, plans):
        if i in mine:
            out[i] = p
    return out, bound, ok
