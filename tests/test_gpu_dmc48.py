"""The 48-electron DMC system (12 nuclei, 24 electrons per spin, 256 determinants, 70 unique
determinants per spin), whose determinants go through the reference-determinant tables.

Against the oracle, element by element: FP64 form ln|Psi| and E_L within 1e-10 of max(1, |x|)
and grad ln|Psi| within 1e-9; mixed form |d ln|Psi|| <= 1e-5 and |d E_L| <= 1e-4 max(1,|E_L|)
(worst walker printed).  DMC: the FP64 form step by step against the oracle's DMC on the same
Philox streams; at the full population (65536 walkers) the mixed form evaluates every walker
finitely, its extreme and sampled walkers match the oracle, and one step keeps a nonempty
population within the capacity (1.5x) whose sampled walkers match the oracle."""
import numpy as np
import pytest

from paper_2207_14715_gb300 import systems as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def vb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_14715_gb300 import build, vbqmc
    build.build()
    ctx = vbqmc.create(0)
    yield vbqmc, ctx
    ctx.close()


@pytest.fixture(scope="module")
def spec():
    return S.dmc48()


def gpu_eval(vb, spec, R, precision):
    mod, ctx = vb
    ctx.set_system(0, spec)
    W = R.shape[0]
    Rt = torch.tensor(R, device="cuda")
    lp, sg, el = (torch.zeros(W, dtype=torch.float64, device="cuda") for _ in range(3))
    g = torch.zeros_like(Rt)
    ctx.eval_walkers(0, precision, Rt, lp, sg, el, g)
    torch.cuda.synchronize()
    return {"logpsi": lp.cpu().numpy(), "sign": sg.cpu().numpy(), "eloc": el.cpu().numpy(), "grad": g.cpu().numpy()}


def _rel(a, b):
    return np.abs(a - b) / np.maximum(1.0, np.abs(b))


def test_table_mode_limits(vb, spec):
    """The tables carry no per-determinant inverses: a walker state is refused (evaluation and
    sweeps), sweeps without one run (test_gpu_tables.py checks them against the oracle), and
    the system cannot be switched to per-determinant inverses (they do not fit)."""
    mod, ctx = vb
    ctx.set_system(0, spec)
    assert ctx.launch_info(0, 0)["eval_walkers_per_block"] >= 1
    R = torch.tensor(S.initial_walkers(spec, 2, 1), device="cuda")
    z = torch.zeros(2, dtype=torch.float64, device="cuda")
    st = torch.zeros((2, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(mod.VbqmcError, match="reference"):
        ctx.eval_walkers(0, 0, R, z, z, z, state_out=st)
    with pytest.raises(mod.VbqmcError, match="state"):
        ctx.vmc_steps(0, 0, R, 1, 0.3, 1, state=st)
    ctx.vmc_steps(0, 0, R, 1, 0.3, 1)
    with pytest.raises(mod.VbqmcError, match="shared memory"):
        ctx.use_tables(0, False)


@pytest.mark.parametrize("precision", [0, 1])
def test_dmc48_eval_matches_oracle(vb, orc, spec, precision):
    R = S.initial_walkers(spec, 6, 48)
    ref = orc.evaluate(spec, R, grad=True)
    got = gpu_eval(vb, spec, R, precision)
    np.testing.assert_array_equal(got["sign"], ref["sign"])
    dl = np.abs(got["logpsi"] - ref["logpsi"])
    de = _rel(got["eloc"], ref["eloc"])
    print("dmc48 %s: worst |d ln Psi| %.2e, worst rel d E_L %.2e" % ("mixed" if precision else "fp64", dl.max(),
                                                                      de.max()))
    if precision == 0:
        assert _rel(got["logpsi"], ref["logpsi"]).max() < 1e-10
        assert de.max() < 1e-10
        assert _rel(got["grad"], ref["grad"]).max() < 1e-9
    else:
        assert dl.max() <= 1e-5
        assert de.max() <= 1e-4
        assert _rel(got["grad"], ref["grad"]).max() < 1e-3


def test_dmc48_fp64_trajectory_matches_oracle(vb, orc, spec):
    mod, ctx = vb
    W, nsteps, tau = 6, 2, 0.005
    R = S.initial_walkers(spec, W, 9)
    e0 = float(np.mean(orc.evaluate(spec, R)["eloc"]))
    ref = orc.dmc(spec, R, nsteps, tau, e0, W, seed=21, step0=5)
    ctx.set_system(0, spec)
    buf = torch.zeros((4 * W, spec.N, 3), dtype=torch.float64, device="cuda")
    buf[:W] = torch.tensor(R, device="cuda")
    W1, et, hist = ctx.dmc_steps(0, 0, buf, W, nsteps, tau, e0, W, 21, step0=5)
    torch.cuda.synchronize()
    assert W1 == ref["W"]
    np.testing.assert_array_equal(hist["pop"], ref["pop"])
    np.testing.assert_allclose(hist["sum_w"], ref["sum_w"], rtol=1e-10)
    np.testing.assert_allclose(hist["sum_wE"], ref["sum_wE"], rtol=1e-10)
    np.testing.assert_allclose(buf[:W1].cpu().numpy(), ref["R"], atol=1e-9)


def test_dmc48_full_population(vb, orc, spec):
    """65536 walkers in the mixed form: every walker evaluates to finite values, the walkers
    with the most extreme E_L (next to the trial's nodes) and random ones match the oracle, and
    one DMC step (tau = 0.005, capacity 1.5x, E_T at the median E_L) keeps a nonempty
    population within the capacity whose sampled walkers match the oracle.  (The weight sums
    are not checked: from unequilibrated walkers, exp(-tau (E_L - E_T)) of a walker at
    E_L ~ -1e6 overflows; the plain step has no energy limits.)"""
    mod, ctx = vb
    target, tau = 65536, 0.005
    cap = target * 3 // 2
    ctx.set_system(0, spec)
    buf = torch.zeros((cap, spec.N, 3), dtype=torch.float64, device="cuda")
    buf[:target] = torch.tensor(S.initial_walkers(spec, target, 3), device="cuda")
    lp, sg, el = (torch.zeros(target, dtype=torch.float64, device="cuda") for _ in range(3))
    ctx.eval_walkers(0, 1, buf[:target], lp, sg, el)
    torch.cuda.synchronize()
    e, l = el.cpu().numpy(), lp.cpu().numpy()
    assert np.isfinite(e).all() and np.isfinite(l).all()
    order = np.argsort(e)
    idx = np.concatenate([order[:2], order[-2:], np.random.default_rng(2).choice(target, 3, replace=False)])
    ref = orc.evaluate(spec, buf[:target].cpu().numpy()[idx])
    assert np.abs(l[idx] - ref["logpsi"]).max() <= 1e-5
    assert _rel(e[idx], ref["eloc"]).max() <= 1e-4
    W1, et, hist = ctx.dmc_steps(0, 1, buf, target, 1, tau, float(np.median(e)), target, 77)
    torch.cuda.synchronize()
    pop = np.asarray(hist["pop"])
    print("dmc48 population", pop.tolist(), "acceptance", hist["accepted"] / target)
    assert len(pop) == 1 and 0 < pop[0] <= cap, pop
    idx = np.random.default_rng(1).choice(W1, 4, replace=False)
    R = buf[:W1].cpu().numpy()[idx]
    ref = orc.evaluate(spec, R)
    got = gpu_eval(vb, spec, R, 1)
    assert np.abs(got["logpsi"] - ref["logpsi"]).max() <= 1e-5
    assert _rel(got["eloc"], ref["eloc"]).max() <= 1e-4


def test_dmc48_reduced_population_220_steps(vb, spec):
    """The DMC workload at a reduced population: 1024 walkers equilibrated by VMC sweeps (table
    sweeps, mixed form), then 220 DMC steps at tau = 0.005 in each form, four independent
    replicas per form.  The population stays within +-20 % of the target in every step after
    the first 20, and the two forms' estimates (mean over steps 20..219 of sum w E_L / sum w)
    agree within 2 sigma (sigma from the replicas' spread).  The FP64 form's first steps match
    the oracle's step by step (test_dmc48_fp64_trajectory_matches_oracle)."""
    mod, ctx = vb
    ctx.set_system(0, spec)
    W, tau, steps, skip = 1024, 0.005, 220, 20
    R = torch.tensor(S.initial_walkers(spec, W, 6), device="cuda")
    ctx.vmc_steps(0, 1, R, 60, spec.step, 3, step0=0, refresh=10)
    lp, sg, el = (torch.zeros(W, dtype=torch.float64, device="cuda") for _ in range(3))
    ctx.eval_walkers(0, 1, R, lp, sg, el)
    e0 = float(el.mean())
    est = {0: [], 1: []}
    for prec in (1, 0):
        for rep in range(4):
            buf = torch.zeros((W * 3 // 2, spec.N, 3), dtype=torch.float64, device="cuda")
            buf[:W] = R
            _, _, h = ctx.dmc_steps(0, prec, buf, W, steps, tau, e0, W, 1000 + rep, step0=0)
            pop = np.asarray(h["pop"])
            assert len(pop) == steps, len(pop)
            assert np.all(np.abs(pop[skip:] / W - 1.0) <= 0.2), (pop.min(), pop.max())
            est[prec].append(float(np.mean(h["sum_wE"][skip:] / h["sum_w"][skip:])))
    m = {p: np.mean(v) for p, v in est.items()}
    s = {p: np.std(v, ddof=1) / np.sqrt(len(v)) for p, v in est.items()}
    print("dmc48 reduced: E_VMC %.3f, DMC mixed %.3f +- %.3f, fp64 %.3f +- %.3f" % (e0, m[1], s[1], m[0], s[0]))
    assert abs(m[1] - m[0]) < 2 * np.hypot(s[0], s[1]), (m, s)
