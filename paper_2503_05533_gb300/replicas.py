"""Several GPUs: replicas, and the one exchange a sharded estimate needs.

Samples of a level are independent (Sec. 4.1), so the data path needs no
collective.  ``bench.py --gpus N`` runs one independent estimate per rank (one
process per GPU) and reports the maximum time over ranks.  An estimate sharded
across ranks would give each rank a disjoint range of sample indices per level
(the random inputs are counter-based, so ranges never overlap) and merge the
ranks' per-level accumulators once per round of Alg. 4.1; the merge is
``mlmc_acc_merge`` (Chan's pairwise update with compensated sums) applied in
rank order, so every rank obtains the same bits.  These helpers use only
``torch.distributed`` object and tensor collectives and run on gloo (CPU) as
well as NCCL.
"""
from . import capi

_ACC_FIELDS = [name for name, _ in capi.mlmc_acc._fields_]


def acc_to_tuple(acc):
    """Plain-Python copy of an mlmc_acc (picklable)."""
    return tuple(getattr(acc, f) for f in _ACC_FIELDS)


def tuple_to_acc(values):
    acc = capi.mlmc_acc()
    for f, v in zip(_ACC_FIELDS, values):
        setattr(acc, f, v)
    return acc


def merge_over_ranks(dist, accs):
    """Per-level accumulators of every rank merged in rank order; the same result on every rank.

    accs: this rank's list of mlmc_acc, one per level (all ranks pass the same number of levels).
    """
    world = dist.get_world_size()
    gathered = [None] * world
    dist.all_gather_object(gathered, [acc_to_tuple(a) for a in accs])
    merged = []
    for level in range(len(accs)):
        total = capi.mlmc_acc()
        for r in range(world):
            capi.mlmc_acc_merge(total, tuple_to_acc(gathered[r][level]))
        merged.append(total)
    return merged


def max_over_ranks(dist, value, device="cpu"):
    """The largest of the ranks' values (the whole-job time of a replicated run)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
