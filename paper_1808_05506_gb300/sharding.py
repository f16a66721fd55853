"""Independent systems of a batched solve spread over ranks (one GPU each).

The systems D(m_i) x_i = b_i of a batch share nothing but the gauge field,
so each rank solves its own subset with dirac_solve_batched and no data ever
crosses ranks; only the per-system statistics are gathered afterwards (a
host-side collective outside the solve).  The assignment balances the total
number of right-hand sides per rank: systems are taken in decreasing Nv (ties
by index) and each goes to the rank with the least work so far (ties to the
lower rank), which is deterministic, so every rank computes the same plan
without communicating.
"""
from __future__ import annotations


def assign_systems(nvs, world: int):
    """Rank -> sorted list of system indices, balancing sum(Nv) per rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    plan = [[] for _ in range(world)]
    for i in sorted(range(len(nvs)), key=lambda i: (-int(nvs[i]), i)):
        r = min(range(world), key=lambda k: (load[k], k))
        plan[r].append(i)
        load[r] += int(nvs[i])
    return [sorted(p) for p in plan]


def solve_batched_sharded(solve, nvs, masses, make_b, rank: int, world: int, gather=None, **kw):
    """Solve this rank's share of the systems.

    solve(bs, masses, **kw) -> (xs, residuals, sys_stats, totals, status) is
    `Dirac.solve_batched` of this rank's handle; make_b(i) builds b_i on this
    rank's device (only the local systems are ever built).  gather(obj) returns
    the list of every rank's obj (torch.distributed.all_gather_object by
    default when a process group is up, else [obj]).  Returns (local indices,
    local solutions, status, stats of all systems in system order, this rank's
    solver totals)."""
    local = assign_systems(nvs, world)[rank]
    xs, stats, status, totals = [], [], 0, {}
    if local:
        bs = [make_b(i) for i in local]
        xs, res, sys_stats, totals, status = solve(bs, [masses[i] for i in local], **kw)
        stats = [dict(system=i, nv=int(nvs[i]), rank=rank, **s) for i, s in zip(local, sys_stats)]
    if gather is None:
        import torch.distributed as dist
        if dist.is_available() and dist.is_initialized():
            def gather(obj):
                out = [None] * dist.get_world_size()
                dist.all_gather_object(out, obj)
                return out
        else:
            def gather(obj):
                return [obj]
    everyone = [s for part in gather(stats) for s in part]
    everyone.sort(key=lambda s: s["system"])
    return local, xs, status, everyone, totals
