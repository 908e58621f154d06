"""Multi-rank host logic (paper_2207_14715_gb300/ranks.py) on CPU: the walker-exchange plan,
and two gloo ranks running the reductions and the walker exchange of a multi-rank DMC step
(the same calls run over NCCL with CUDA tensors on GPUs)."""
import math
import socket

import pytest

from paper_2207_14715_gb300 import ranks

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("pops", [[7, 1], [0, 9], [5, 5], [3, 0, 0, 9], [1, 2, 3, 4, 5], [0, 0, 1]])
def test_balance_plan_evens_the_populations(pops):
    plan = ranks.balance_plan(pops)
    after = list(pops)
    for src, dst, k in plan:
        assert k > 0 and src != dst
        after[src] -= k
        after[dst] += k
    total, n = sum(pops), len(pops)
    assert after == [total // n + (1 if r < total % n else 0) for r in range(n)]
    assert all(a >= 0 for a in after)
    # a rank either gives or takes
    assert not ({s for s, _, _ in plan} & {d for _, d, _ in plan})


def test_single_rank_calls_return_their_input():
    assert ranks.world() == (0, 1)
    assert ranks.max_over_ranks(2.5) == 2.5
    assert ranks.dmc_global_sums(1.0, 2.0, 3) == (1.0, 2.0, 3)
    assert ranks.dmc_global_sums(1.0, 2.0, 3, sum_wEb=4.0, failed=False) == (1.0, 2.0, 3, 4.0, 0)
    assert ranks.walker_offset(3, 1024) == 3072
    R = torch.zeros((4, 2, 3))
    assert ranks.balance_walkers(R, 3) == 3


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _two_rank_worker(rank, world, port):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        assert ranks.world() == (rank, world)
        assert ranks.max_over_ranks(rank + 0.5) == world - 0.5
        # one DMC step's sums: the trial energy follows the global population
        swE, sw, pop = ranks.dmc_global_sums(-2.0 * (rank + 1), 2.0 + rank, 10 + 5 * rank)
        assert (swE, sw, pop) == (-6.0, 5.0, 25)
        e_t = ranks.trial_energy(swE, sw, pop, target=20, tau=0.01)
        assert abs(e_t - (-6.0 / 5.0 - 10.0 * math.log(25 / 20))) < 1e-12
        # walker exchange: 7 walkers on rank 0, 1 on rank 1, capacity 8 each; every row marked
        W = 7 if rank == 0 else 1
        R = torch.full((8, 2, 3), -1.0, dtype=torch.float64)
        for i in range(W):
            R[i] = 100.0 * rank + i
        W2 = ranks.balance_walkers(R, W)
        assert W2 == 4
        rows = torch.full((8,), -1.0, dtype=torch.float64)
        rows[:W2] = R[:W2, 0, 0]
        everything = [torch.zeros_like(rows) for _ in range(world)]
        dist.all_gather(everything, rows)
        got = sorted(float(v) for t in everything for v in t if v >= 0)
        assert got == sorted([float(i) for i in range(7)] + [100.0])
        assert torch.all(R[:W2] == R[:W2, :1, :1])  # whole rows moved
        # walker offsets of the ranks never overlap
        assert ranks.walker_offset(rank, 4096) == 4096 * rank
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    torch.multiprocessing.spawn(_two_rank_worker, args=(2, _free_port()), nprocs=2, join=True)


def _dmc_run_worker(rank, world, port):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        R = torch.zeros((16, 1, 3), dtype=torch.float64)
        seen = []

        keys, last_ret = [], []

        def step(W, E_T, k, off):  # a stand-in step: rank 0 grows by 3, rank 1 shrinks by 1; E_L = -1 - rank
            seen.append(E_T)
            keys.append((k, off))
            W2 = W + 3 if rank == 0 else max(W - 1, 0)
            R[:W2, 0, 0] = float(rank)
            last_ret.append((W2, (-1.0 - rank) * W2, float(W2), (-1.5 - rank) * W2))
            return last_ret[-1]
        W, E_T, hist = ranks.dmc_run(step, R, 4, 3, tau=0.01, E_T=-1.0, target_per_rank=4, step0=100)
        # every rank sees the same global sums and trial energies
        assert [h[2] for h in hist] == [10, 12, 14]
        gwE, gw, gpop = hist[-1]
        # E_T follows the global sum of w E_b of the last step (the fourth value each rank returned)
        last = torch.tensor([last_ret[-1][3]], dtype=torch.float64)
        dist.all_reduce(last)
        assert abs(E_T - (float(last) / gw - 10.0 * math.log(gpop / 8))) < 1e-12
        assert W == 7 and seen[0] == -1.0 and len(set(seen)) == 3
        # the random-number keys: global step numbers, and walker ranges [off, off + cap) that
        # differ between the ranks (the streams of vbqmc_dmc_steps never coincide)
        assert [k for k, _ in keys] == [100, 101, 102]
        offs = [torch.tensor([keys[0][1]]) for _ in range(world)]
        dist.all_gather(offs, torch.tensor([keys[0][1]]))
        lo = sorted(int(o) for o in offs)
        assert lo == [0, 16] and lo[1] - lo[0] >= R.shape[0]
    finally:
        dist.destroy_process_group()


def test_dmc_run_two_gloo_ranks():
    torch.multiprocessing.spawn(_dmc_run_worker, args=(2, _free_port()), nprocs=2, join=True)


def _failure_worker(rank, world, port, mode):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        if mode == "step":
            R = torch.zeros((8, 1, 3), dtype=torch.float64)

            def step(W, E_T, k, off):  # rank 1 fails at its second step
                if rank == 1 and k == 1:
                    raise ValueError("capacity exceeded on rank 1")
                return W, -1.0 * W, float(W), -1.0 * W
            try:
                ranks.dmc_run(step, R, 4, 5, tau=0.01, E_T=-1.0, target_per_rank=4)
            except ValueError as e:
                assert rank == 1 and "rank 1" in str(e)
            except ranks.RankFailure as e:
                assert rank == 0 and "1 other rank" in str(e)
            else:
                raise AssertionError("no rank may continue after a failed step")
        else:  # a share above one rank's capacity: every rank raises before any transfer
            R = torch.zeros((12 if rank == 0 else 3, 1, 3), dtype=torch.float64)
            try:
                ranks.balance_walkers(R, 12 if rank == 0 else 0)
            except ValueError as e:
                assert "rank 1" in str(e)
            else:
                raise AssertionError("the overflow must be seen on every rank")
        # the group is still usable: a collective after the failure completes
        t = torch.ones(1)
        dist.all_reduce(t)
        assert float(t) == world
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["step", "capacity"])
def test_failures_stop_every_rank(mode):
    torch.multiprocessing.spawn(_failure_worker, args=(2, _free_port(), mode), nprocs=2, join=True)


def _lin_worker(rank, world, port):
    import numpy as np
    import torch.distributed as dist
    from oracle import oracle as orc
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(42)
        M, P = 700, 9
        O = rng.normal(size=(M, P)) + 2.0 * rng.normal(size=P)
        dE = rng.normal(size=(M, P))
        E = -7.0 + rng.normal(size=M) + 0.3 * O[:, 1]
        w = rng.uniform(0.3, 1.7, M)
        cut = 250  # uneven parts
        sl = slice(0, cut) if rank == 0 else slice(cut, M)
        m = orc.lin_matrices(O[sl], dE[sl], E[sl], w[sl])
        part = dict(m, wsum=w[sl].sum(), mean=(w[sl, None] * O[sl]).sum(0) / w[sl].sum())
        got = ranks.merge_lin_parts(part)
        ref = orc.lin_matrices(O, dE, E, w)
        for k in ("S", "H", "gL", "gR"):
            assert np.abs(got[k] - ref[k]).max() <= 1e-12 * np.abs(ref[k]).max(), k
        assert abs(got["E0"][0] - ref["E0"]) <= 1e-12 * abs(ref["E0"])
        sw, swe, swe2 = ranks.vmc_energy_moments(w[sl].sum(), (w[sl] * E[sl]).sum(), (w[sl] * E[sl] ** 2).sum())
        assert abs(swe / sw - (w * E).sum() / w.sum()) < 1e-12
        assert abs(swe2 / sw - (w * E * E).sum() / w.sum()) < 1e-10
    finally:
        dist.destroy_process_group()


def test_linear_method_parts_merge_to_the_union():
    """Two ranks each accumulate the estimators of their own samples; the all-gathered merge
    equals one accumulation over the union of the samples (S, H, g to 1e-12 of scale)."""
    torch.multiprocessing.spawn(_lin_worker, args=(2, _free_port()), nprocs=2, join=True)
