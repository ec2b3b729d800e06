"""Host-side multi-GPU helpers: one process per GPU, no collective on the data path.

The propagations of different total angular momenta J are independent (they share no
state), so a list of J values is split across ranks and each rank propagates its own
J values on its own GPU; the per-J results are gathered once at the end. The bench
workload (one J) runs as independent replicas. torch.distributed carries only the
final gather and the timing reduction (barrier, maximum over ranks); with the gloo
backend the same code runs on CPU processes.
"""
from __future__ import annotations


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def rank_world():
    d = _dist()
    return (d.get_rank(), d.get_world_size()) if d else (0, 1)


def shard(items, rank: int, world: int):
    """Contiguous block of `items` for `rank` (sizes differ by at most one)."""
    items = list(items)
    n = len(items)
    lo = rank * n // world
    hi = (rank + 1) * n // world
    return items[lo:hi]


def barrier():
    d = _dist()
    if d:
        d.barrier()


def max_over_ranks(x: float) -> float:
    """The largest value of `x` over all ranks (every rank gets it)."""
    d = _dist()
    if not d:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64)
    if d.get_backend() == "nccl":
        t = t.cuda()
    d.all_reduce(t, op=d.ReduceOp.MAX)
    return float(t.item())


def gather_by_key(local: dict) -> dict:
    """Union of every rank's {key: value} dictionary (keys are disjoint across ranks)."""
    d = _dist()
    if not d:
        return dict(local)
    parts = [None] * d.get_world_size()
    d.all_gather_object(parts, local)
    out = {}
    for p in parts:
        out.update(p)
    return out


def propagate_J_sharded(cfg: dict, steps: int, precision: str = "mixed", device: int = 0):
    """Propagate this rank's share of cfg["J"] (one batched context) and gather the
    probabilities of every J: returns (E, {J: P_total[nE]}, {J: P_inel[nelec, v, j, nE]})."""
    import copy

    from . import mw3
    rank, world = rank_world()
    mine = shard(cfg["J"], rank, world)
    local_tot, local_in = {}, {}
    E = None
    if mine:
        c = copy.deepcopy(cfg)
        c["J"] = mine
        pr = mw3.Propagator(c, device=device, precision=precision)
        pr.propagate(steps)
        E, P, Pin = pr.probabilities()
        pr.close()
        for i, J in enumerate(mine):
            local_tot[J] = P[i]
            local_in[J] = None if Pin is None else Pin[i]
    tot = gather_by_key(local_tot)
    inel = gather_by_key(local_in)
    Es = gather_by_key({rank: E})
    E = next((Es[r] for r in sorted(Es) if Es[r] is not None), None)
    return E, tot, inel
