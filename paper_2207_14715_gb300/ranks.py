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


def dmc_global_sums(sum_wE: float, sum_w: float, population: int, device=None, failed=None, sum_wEb=None):
    """Sums over the ranks of one DMC step's weighted local energies, weights and populations
    (and, if given, of the weighted branching energies, appended to the result).  With failed
    given (this rank's step raised, True/False), the count of failed ranks travels in the same
    reduction and is returned last."""
    d = _dist()
    nf = 1 if failed else 0
    vals = [float(sum_wE), float(sum_w), float(population)]
    if sum_wEb is not None:
        vals.append(float(sum_wEb))
    if failed is not None:
        vals.append(float(nf))
    if d is not None:
        import torch
        t = torch.tensor(vals, dtype=torch.float64, device=device)
        d.all_reduce(t, op=d.ReduceOp.SUM)
        vals = [float(x) for x in t]
    out = (vals[0], vals[1], int(round(vals[2])))
    k = 3
    if sum_wEb is not None:
        out += (vals[k],)
        k += 1
    if failed is not None:
        out += (int(round(vals[k])),)
    return out


def trial_energy(sum_wEb: float, sum_w: float, population: int, target: int, tau: float) -> float:
    """The trial-energy update of the DMC step (the one vbqmc_dmc_steps applies to its own
    population), from global sums of the weights and of the weights times the limited branching
    energies: E_T = sum w E_b / sum w - (0.1 / tau) ln(population / target)."""
    return sum_wEb / sum_w - (0.1 / tau) * math.log(population / target)


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
    in rows [0, W) (as vbqmc_dmc_steps leaves it; weights are 1 after branching, and
    vbqmc_dmc_steps re-evaluates its walkers at the start of every call, so positions are all a
    walker carries); returns the new population, in rows [0, W').  Populations and capacities
    are gathered first, so that every rank sees an overflow on any rank and all of them raise
    before any walker moves (no rank is left waiting in a send or receive)."""
    d = _dist()
    if d is None:
        return W
    import torch
    rank, n = d.get_rank(), d.get_world_size()
    mine = torch.tensor([W, R.shape[0]], dtype=torch.int64, device=R.device)
    allp = [torch.zeros_like(mine) for _ in range(n)]
    d.all_gather(allp, mine)
    pops = [int(p[0].item()) for p in allp]
    caps = [int(p[1].item()) for p in allp]
    total = sum(pops)
    shares = [total // n + (1 if r < total % n else 0) for r in range(n)]
    over = [r for r in range(n) if shares[r] > caps[r]]
    if over:
        r = over[0]
        raise ValueError("rank %d: a share of %d walkers exceeds its capacity %d" % (r, shares[r], caps[r]))
    plan = balance_plan(pops)
    reqs, sends = [], []
    top = W
    for src, dst, k in plan:  # the sources give rows from the end of their population
        if src == rank:
            top -= k
            buf = R[top:top + k].clone()  # a copy: R may be written before the send completes
            sends.append(buf)
            reqs.append(d.isend(buf, dst))
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
    return shares[rank]


class RankFailure(RuntimeError):
    """Raised on every rank of a group when a step failed on one of them."""


def dmc_run(dmc_step, R, W: int, nsteps: int, tau: float, E_T: float, target_per_rank: int,
            balance_every: int = 1, device=None, step0: int = 0):
    """nsteps DMC steps of this rank's population under one global trial energy.
    dmc_step(W, E_T, step, walker_offset) advances the population in R by one step at trial
    energy E_T and returns (W', sum of pre-branching w E_L, sum of w, sum of w E_b), e.g.
        lambda W, E_T, step, off: Context.dmc_steps(sys, prec, R, W, 1, tau, E_T, target, seed,
                                                    step0=step, walker_offset=off) (+ its sums);
    'step' is the global step number step0 + k and 'walker_offset' = rank x capacity, so the
    Philox streams differ between steps and between ranks.  dmc_step must keep no walker state
    between calls (the walkers move between ranks).  After each step the sums and populations of
    all ranks set E_T (trial_energy with the target target_per_rank x ranks), and every
    balance_every steps the walkers are evened out over the ranks.  A step that raises on one
    rank stops all ranks together: an error flag travels with the sums, the failing rank re-raises
    its error and the others raise RankFailure.  Returns (W, E_T, [(global sum w E_L,
    global sum w, global population) per step]); the DMC estimate is the ratio of the summed sums."""
    rank, n = world()
    target = target_per_rank * n
    offset = rank * R.shape[0]
    hist = []
    for k in range(nsteps):
        err = None
        try:
            W, swE, sw, swEb = dmc_step(W, E_T, step0 + k, offset)
        except Exception as e:  # decided as a group below
            err, swE, sw, swEb = e, 0.0, 0.0, 0.0
        gwE, gw, gpop, gwEb, nfail = dmc_global_sums(swE, sw, W, device, failed=err is not None, sum_wEb=swEb)
        if nfail:
            if err is not None:
                raise err
            raise RankFailure("DMC step %d failed on %d other rank(s)" % (step0 + k, nfail))
        hist.append((gwE, gw, gpop))
        if gpop == 0:
            break
        E_T = trial_energy(gwEb, gw, gpop, target, tau)
        if balance_every and (k + 1) % balance_every == 0:
            W = balance_walkers(R, W)
    return W, E_T, hist


def vmc_energy_moments(sum_w: float, sum_wE: float, sum_wE2: float, device=None):
    """Sums over the ranks of a VMC block's weights, w E_L and w E_L^2 (Sec. 2.3.1, Eq. Elav):
    the global mean energy is sum_wE / sum_w and its variance sum_wE2 / sum_w - mean^2."""
    d = _dist()
    if d is None:
        return float(sum_w), float(sum_wE), float(sum_wE2)
    import torch
    t = torch.tensor([float(sum_w), float(sum_wE), float(sum_wE2)], dtype=torch.float64, device=device)
    d.all_reduce(t, op=d.ReduceOp.SUM)
    return float(t[0]), float(t[1]), float(t[2])


def merge_lin_parts(part, device=None):
    """The linear-method estimators of the samples of all ranks (Sec. 2.3.1, Eqs. Hi0..Sij) from
    each rank's own: part = dict(wsum, mean [P], E0, gL [P], gR [P], S [P, P], H [P, P]) as this
    rank's accumulation gives them (e.g. Context.lin_part).  The parts are all-gathered (one
    flat float64 vector of 2 + 3P + 2P^2 entries per rank) and merged by vbqmc_lin_merge, the
    same on every rank.  Single-rank calls merge one part (the identity)."""
    import numpy as np
    from . import vbqmc
    P = len(np.asarray(part["gL"]))
    flat = np.concatenate([[float(part["wsum"]), float(np.asarray(part["E0"]).ravel()[0])],
                           np.asarray(part["mean"], np.float64).ravel(), np.asarray(part["gL"], np.float64).ravel(),
                           np.asarray(part["gR"], np.float64).ravel(), np.asarray(part["S"], np.float64).ravel(),
                           np.asarray(part["H"], np.float64).ravel()])
    d = _dist()
    if d is None:
        rows = [flat]
    else:
        import torch
        t = torch.tensor(flat, dtype=torch.float64, device=device)
        allt = [torch.zeros_like(t) for _ in range(d.get_world_size())]
        d.all_gather(allt, t)
        rows = [a.cpu().numpy() for a in allt]
    parts = []
    for r in rows:
        o = 2
        mean, o = r[o:o + P], o + P
        gL, o = r[o:o + P], o + P
        gR, o = r[o:o + P], o + P
        S, o = r[o:o + P * P].reshape(P, P), o + P * P
        H = r[o:o + P * P].reshape(P, P)
        parts.append({"wsum": r[0], "E0": r[1], "mean": mean, "gL": gL, "gR": gR, "S": S, "H": H})
    return vbqmc.lin_merge(parts)
