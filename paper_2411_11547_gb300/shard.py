"""Sharding one batch over ranks (one process per GPU).

Pairs are independent (Sec. II-B, inter-task parallelism), so the forward needs no exchange.
The adjoint's per-read gradient sums all pairs that share a read, so every read's pairs are
kept on one rank: ranks take contiguous read ranges, balanced by their cells (sum of m * n over
the pairs).  The only cross-rank sum is d/d(gap-continuation quality), one number, which
`allreduce_scalar` adds over the process group.  Host-side index arithmetic only.
"""
from __future__ import annotations

import numpy as np


def partition_by_read(batch, world: int):
    """[(read_lo, read_hi)] per rank: contiguous read ranges with balanced cells."""
    if world < 1:
        raise ValueError("world must be >= 1")
    ro = np.asarray(batch["read_off"], dtype=np.int64)
    ho = np.asarray(batch["hap_off"], dtype=np.int64)
    pr = np.asarray(batch["pair_read"], dtype=np.int64)
    ph = np.asarray(batch["pair_hap"], dtype=np.int64)
    R = len(ro) - 1
    cells = np.zeros(R, dtype=np.float64)
    np.add.at(cells, pr, (ro[pr + 1] - ro[pr]) * (ho[ph + 1] - ho[ph]))
    cum = np.concatenate([[0.0], np.cumsum(cells)])
    total = cum[-1]
    bounds = [0]
    for k in range(1, world):
        cut = int(np.searchsorted(cum, total * k / world, side="left"))
        bounds.append(min(max(cut, bounds[-1]), R))
    bounds.append(R)
    return [(bounds[k], bounds[k + 1]) for k in range(world)]


def shard(batch, rank: int, world: int):
    """(sub-batch, global pair ids, (read_lo, read_hi)) of `rank`.

    The sub-batch holds the rank's reads (renumbered from 0, bases and qualities copied),
    the haplotypes its pairs use (renumbered) and its pairs, in global pair order.  Its
    per-base gradients belong at read_off[read_lo]:read_off[read_hi] of the global arrays.
    """
    lo, hi = partition_by_read(batch, world)[rank]
    ro = np.asarray(batch["read_off"], dtype=np.int64)
    ho = np.asarray(batch["hap_off"], dtype=np.int64)
    pr = np.asarray(batch["pair_read"], dtype=np.int64)
    ph = np.asarray(batch["pair_hap"], dtype=np.int64)
    pairs = np.nonzero((pr >= lo) & (pr < hi))[0]
    haps = np.unique(ph[pairs])
    hmap = np.full(len(ho) - 1, -1, dtype=np.int64)
    hmap[haps] = np.arange(len(haps))
    b0, b1 = ro[lo], ro[hi]
    hl = ho[haps + 1] - ho[haps]
    hbase = [batch["hap_bases"][ho[h]:ho[h + 1]] for h in haps]
    sub = {
        "name": f"{batch.get('name', 'batch')}[{rank}/{world}]",
        "read_bases": np.ascontiguousarray(batch["read_bases"][b0:b1]),
        "base_q": np.ascontiguousarray(batch["base_q"][b0:b1]),
        "ins_q": np.ascontiguousarray(batch["ins_q"][b0:b1]),
        "del_q": np.ascontiguousarray(batch["del_q"][b0:b1]),
        "read_off": (ro[lo:hi + 1] - b0).astype(np.int64),
        "hap_bases": (np.concatenate(hbase) if len(hbase) else
                      np.zeros(0, dtype=np.uint8)).astype(np.uint8),
        "hap_off": np.concatenate([[0], np.cumsum(hl)]).astype(np.int64),
        "pair_read": (pr[pairs] - lo).astype(np.int32),
        "pair_hap": hmap[ph[pairs]].astype(np.int32),
        "gcp": float(batch["gcp"]),
    }
    if "alpha_mode" in batch:
        sub["alpha_mode"] = batch["alpha_mode"]
    if batch.get("gcp_q") is not None:
        sub["gcp_q"] = np.ascontiguousarray(batch["gcp_q"][b0:b1])
    return sub, pairs, (lo, hi)


def sharded_step(batch, dL, rank: int, world: int, compute, group=None):
    """One training step of `batch` sharded over `world` ranks, from this rank's side.

    The rank takes its shard (contiguous reads, every pair of those reads), runs
    compute(sub_batch, dL of the shard's pairs) -> (log10 L [shard pairs], d_base_q, d_ins_q,
    d_del_q [shard read bases], d_gcp), and adds d_gcp over the ranks (the one exchange).
    Returns a dict: "pairs" (global pair ids of the shard), "bases" (the global read-base
    range (b0, b1) its gradients cover), "log10", "d_base_q", "d_ins_q", "d_del_q" (the
    shard's values) and "d_gcp" (the sum over every rank).  Each global array is the
    concatenation of the ranks' slices: no rank's slice overlaps another's.
    """
    sub, pairs, (lo, hi) = shard(batch, rank, world)
    y, gb, gi, gd, gg = compute(sub, np.asarray(dL)[pairs])
    ro = np.asarray(batch["read_off"], dtype=np.int64)
    return {"pairs": pairs, "bases": (int(ro[lo]), int(ro[hi])), "log10": y, "d_base_q": gb,
            "d_ins_q": gi, "d_del_q": gd, "d_gcp": allreduce_scalar(gg, group)}


def allreduce_tensor_(t, group=None):
    """Sum a tensor in place over the default (or given) process group (no host wait with
    NCCL); identity without one."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def allreduce_scalar(x, group=None):
    """Sum a float over the default (or given) process group; identity without one."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return float(t.item())
