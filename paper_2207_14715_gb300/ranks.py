"""Walkers over several ranks (one process per GPU; arXiv:2207.14715, Sec. 1: walkers are
independent, so a VMC run shards them with no data-path exchange).  The exchange steps of a
multi-rank DMC run live here: the estimator sums and the population that set the trial energy
are global (Sec. 2.3.2, Eq. E0DMCweights), and walkers move between ranks to keep the per-rank
populations even.  Everything goes through torch.distributed: NCCL with CUDA tensors on GPUs,
gloo with host tensors (the tests).  Single-rank calls (no process group) return their input.
"""
from __future__ import annotations

import math


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def world():
    """(rank, world size) of the default process group, (0, 1) without one."""
    d = _dist()
    return (d.get_rank(), d.get_world_size()) if d else (0, 1)


def walker_offset(rank: int, walkers_per_rank: int) -> int:
    """First global walker index of a rank: the Philox counters of its walkers (the
    walker_offset argument of vbqmc_vmc_steps) then never coincide with another rank's."""
    return rank * walkers_per_rank


def max_over_ranks(x: float, device=None) -> float:
    """The largest x over the ranks (the timing rule: a step takes as long as its slowest rank)."""
    d = _dist()
    if d is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    d.all_reduce(t, op=d.ReduceOp.MAX)
    return float(t.item())


def dmc_global_sums(sum_wE: float, sum_w: float, population: int, device=None):
    """Sums over the ranks of one DMC step's weighted local energies, weights and populations."""
    d = _dist()
    if d is None:
        return float(sum_wE), float(sum_w), int(population)
    import torch
    t = torch.tensor([float(sum_wE), float(sum_w), float(population)], dtype=torch.float64, device=device)
    d.all_reduce(t, op=d.ReduceOp.SUM)
    return float(t[0]), float(t[1]), int(round(float(t[2])))


def trial_energy(sum_wE: float, sum_w: float, population: int, target: int, tau: float) -> float:
    """The trial-energy update of the DMC step (the one vbqmc_dmc_steps applies to its own
    population), from global sums: E_T = sum w E_L / sum w - (0.1 / tau) ln(population / target)."""
    return sum_wE / sum_w - (0.1 / tau) * math.log(population / target)


def balance_plan(pops):
    """Transfers (source rank, destination rank, count) that leave every rank with
    total // ranks walkers, the first total % ranks ranks with one more; ranks above their share
    give their last walkers, in rank order, to ranks below theirs, in rank order."""
    n = len(pops)
    total = sum(pops)
    want = [total // n + (1 if r < total % n else 0) for r in range(n)]
    give = [(r, pops[r] - want[r]) for r in range(n) if pops[r] > want[r]]
    take = [(r, want[r] - pops[r]) for r in range(n) if pops[r] < want[r]]
    plan = []
    gi = ti = 0
    while gi < len(give) and ti < len(take):
        (src, g), (dst, t) = give[gi], take[ti]
        k = min(g, t)
        plan.append((src, dst, k))
        give[gi], take[ti] = (src, g - k), (dst, t - k)
        if give[gi][1] == 0:
            gi += 1
        if take[ti][1] == 0:
            ti += 1
    return plan


def balance_walkers(R, W: int) -> int:
    """Moves walkers between ranks by balance_plan.  R [cap, ...] holds this rank's population
    in rows [0, W) (as vbqmc_dmc_steps leaves it; weights are 1 after branching, so positions
    are all a walker carries); returns the new population, in rows [0, W').  Raises if a rank's
    share exceeds its capacity."""
    d = _dist()
    if d is None:
        return W
    import torch
    rank, n = d.get_rank(), d.get_world_size()
    mine = torch.tensor([W], dtype=torch.int64, device=R.device)
    allp = [torch.zeros_like(mine) for _ in range(n)]
    d.all_gather(allp, mine)
    pops = [int(p.item()) for p in allp]
    plan = balance_plan(pops)
    total = sum(pops)
    share = total // n + (1 if rank < total % n else 0)
    if share > R.shape[0]:
        raise ValueError("rank %d: %d walkers exceed the capacity %d" % (rank, share, R.shape[0]))
    reqs = []
    top = W
    for src, dst, k in plan:  # the sources give rows from the end of their population
        if src == rank:
            top -= k
            reqs.append(d.isend(R[top:top + k].contiguous(), dst))
    recv = []
    fill = top
    for src, dst, k in plan:
        if dst == rank:
            buf = torch.empty((k,) + tuple(R.shape[1:]), dtype=R.dtype, device=R.device)
            reqs.append(d.irecv(buf, src))
            recv.append((fill, buf))
            fill += k
    for q in reqs:
        q.wait()
    for at, buf in recv:
        R[at:at + buf.shape[0]] = buf
    return share


def dmc_run(dmc_step, R, W: int, nsteps: int, tau: float, E_T: float, target_per_rank: int,
            balance_every: int = 1, device=None):
    """nsteps DMC steps of this rank's population under one global trial energy.  dmc_step(W, E_T)
    advances the population in R by one step at trial energy E_T and returns (W', sum of
    pre-branching w E_L, sum of w), e.g. Context.dmc_steps with nsteps = 1 reading back its sums.
    After each step the sums and populations of all ranks set E_T (trial_energy with the target
    target_per_rank x ranks), and every balance_every steps the walkers are evened out over the
    ranks.  Returns (W, E_T, [(global sum w E_L, global sum w, global population) per step]);
    the DMC energy estimate is the ratio of the summed sums."""
    n = world()[1]
    target = target_per_rank * n
    hist = []
    for k in range(nsteps):
        W, swE, sw = dmc_step(W, E_T)
        gwE, gw, gpop = dmc_global_sums(swE, sw, W, device)
        hist.append((gwE, gw, gpop))
        if gpop == 0:
            break
        E_T = trial_energy(gwE, gw, gpop, target, tau)
        if balance_every and (k + 1) % balance_every == 0:
            W = balance_walkers(R, W)
    return W, E_T, hist
