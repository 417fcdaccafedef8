"""Weak scaling over independent proofs: one process per GPU, each tracing a
workload of its own (seeded by its rank), with no collective on the data path.
The job's throughput is the units all ranks processed divided by the slowest
rank's time, so the only collective is this reduction of four numbers."""
from __future__ import annotations


def reduce_timing(ms, units, e2e_s, e2e_units, world, device):
    """(max ms, sum units, max e2e seconds, sum e2e units) over the ranks of
    the default process group (world == 1: the local values)."""
    if world <= 1:
        return float(ms), float(units), float(e2e_s), float(e2e_units)
    import torch
    import torch.distributed as dist
    agg = torch.tensor([ms, float(units), e2e_s, float(e2e_units)], dtype=torch.float64,
                       device=device)
    mx = agg.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = agg.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return mx[0].item(), sm[1].item(), mx[2].item(), sm[3].item()
