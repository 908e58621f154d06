"""Parity of the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances:
  FP64 form  : ln|Psi| and E_L within 1e-10 relative (|d| <= 1e-10 max(1, |x|)); gradients
               1e-9; parameter derivatives 1e-8 relative to max(1, |x|) (derivatives add one
               more cancellation level than E_L).
  mixed form : |d ln|Psi|| <= 1e-5 and |d E_L| <= 1e-4 max(1, |E_L|) per walker (worst walker
               reported); derivatives 2e-3 relative to max(1, |x|) (float bulk arithmetic,
               ~1e-7 relative rounding amplified by Slater conditioning).
"""
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


def gpu_eval(vb, spec, R, precision, derivs=False, grad=True):
    mod, ctx = vb
    ctx.set_system(0, spec)
    W = R.shape[0]
    P = spec.n_params
    dev = "cuda"
    Rt = torch.tensor(R, dtype=torch.float64, device=dev)
    lp = torch.zeros(W, dtype=torch.float64, device=dev)
    sg = torch.zeros_like(lp)
    el = torch.zeros_like(lp)
    g = torch.zeros_like(Rt) if grad else None
    O = torch.zeros((W, P), dtype=mod.deriv_dtype(precision), device=dev) if derivs and P else None
    dE = torch.zeros_like(O) if O is not None else None
    ctx.eval_walkers(0, precision, Rt, lp, sg, el, g, O, dE)
    torch.cuda.synchronize()
    out = {"logpsi": lp.cpu().numpy(), "sign": sg.cpu().numpy(), "eloc": el.cpu().numpy()}
    if grad:
        out["grad"] = g.cpu().numpy()
    if O is not None:
        out["O"], out["dEL"] = O.double().cpu().numpy(), dE.double().cpu().numpy()
    return out


def rel_err(a, b):
    return np.abs(a - b) / np.maximum(1.0, np.abs(b))


SYSTEMS = {
    "hydrogenic": (lambda: S.one_electron(3.0, 0.0, a1=-3.0, a2=-0.8), 10),
    "gauss_h": (lambda: S.one_electron(1.0, 0.4), 9),
    "two_electron": (lambda: S.two_electron_product(2.0, 0.9), 11),
    "h2_vb": (S.h2_vb, 50),
    "small_open_shell": (S.small_open_shell, 37),
    "ethylene_vb": (S.ethylene_vb, 5),
}


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_eval_fp64_matches_oracle(vb, orc, name):
    maker, W = SYSTEMS[name]
    spec = maker()
    R = S.initial_walkers(spec, W, 100 + W)
    ref = orc.evaluate(spec, R, grad=True)
    got = gpu_eval(vb, spec, R, 0)
    np.testing.assert_array_equal(got["sign"], ref["sign"])
    assert rel_err(got["logpsi"], ref["logpsi"]).max() < 1e-10
    assert rel_err(got["eloc"], ref["eloc"]).max() < 1e-10
    assert rel_err(got["grad"], ref["grad"]).max() < 1e-9


@pytest.mark.parametrize("name", ["small_open_shell", "ethylene_vb"])
def test_eval_fp64_derivatives_match_oracle(vb, orc, name):
    spec = SYSTEMS[name][0]()
    W = 4 if name == "small_open_shell" else 2
    R = S.initial_walkers(spec, W, 7)
    ref = orc.evaluate(spec, R, derivs=True)
    got = gpu_eval(vb, spec, R, 0, derivs=True)
    assert rel_err(got["O"], ref["O"]).max() < 1e-8
    scale = np.maximum(1.0, np.abs(ref["dEL"]))
    assert (np.abs(got["dEL"] - ref["dEL"]) / scale).max() < 1e-8


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_eval_mixed_within_tolerance(vb, orc, name):
    maker, W = SYSTEMS[name]
    spec = maker()
    R = S.initial_walkers(spec, W, 300 + W)
    ref = orc.evaluate(spec, R, grad=True)
    got = gpu_eval(vb, spec, R, 1)
    dl = np.abs(got["logpsi"] - ref["logpsi"])
    de = rel_err(got["eloc"], ref["eloc"])
    print("%s mixed: worst |dlnPsi| %.2e (walker %d), worst rel dE_L %.2e (walker %d)"
          % (name, dl.max(), dl.argmax(), de.max(), de.argmax()))
    assert dl.max() <= 1e-5
    assert de.max() <= 1e-4
    np.testing.assert_array_equal(got["sign"], ref["sign"])


@pytest.mark.parametrize("name", ["small_open_shell", "ethylene_vb"])
def test_eval_mixed_derivatives(vb, orc, name):
    """Mixed O_p and E_L,p on 24 walkers, element by element; the worst walker and parameter of
    each are reported."""
    spec = SYSTEMS[name][0]()
    R = S.initial_walkers(spec, 24, 17)
    ref = orc.evaluate(spec, R, derivs=True)
    got = gpu_eval(vb, spec, R, 1, derivs=True)
    for key in ("O", "dEL"):
        r = rel_err(got[key], ref[key])
        w, p = np.unravel_index(r.argmax(), r.shape)
        print("%s mixed %s: worst rel error %.2e at walker %d, parameter %d (median %.2e)"
              % (name, key, r.max(), w, p, np.median(r)))
        assert r.max() < 2e-3, key


def gpu_vmc(vb, spec, R, nsweeps, seed, precision=0, step0=0):
    mod, ctx = vb
    ctx.set_system(0, spec)
    Rt = torch.tensor(R, dtype=torch.float64, device="cuda")
    nacc = torch.zeros(R.shape[0], dtype=torch.int32, device="cuda")
    ctx.vmc_steps(0, precision, Rt, nsweeps, spec.step, seed, step0=step0, nacc=nacc)
    torch.cuda.synchronize()
    return Rt.cpu().numpy(), nacc.cpu().numpy()


@pytest.mark.parametrize("name,W,nsw", [("h2_vb", 64, 6), ("small_open_shell", 33, 3), ("hydrogenic", 8, 5),
                                        ("ethylene_vb", 3, 1)])
def test_vmc_fp64_trajectory_matches_oracle(vb, orc, name, W, nsw):
    """Same Philox streams, same proposals: FP64 trajectories agree move for move."""
    spec = SYSTEMS[name][0]()
    R0 = S.initial_walkers(spec, W, 5)
    Rg, ng = gpu_vmc(vb, spec, R0, nsw, seed=2024, step0=11)
    Ro, _, _, no = orc.vmc(spec, R0, nsw, spec.step, seed=2024, step0=11, eloc=False)
    np.testing.assert_array_equal(ng, no)
    np.testing.assert_allclose(Rg, Ro, rtol=0, atol=1e-12)


@pytest.mark.parametrize("name,W,nsw", [("small_open_shell", 19, 3), ("ethylene_vb", 3, 1)])
def test_vmc_fp64_from_saved_state_matches_oracle(vb, orc, name, W, nsw):
    """Sweeps that start from the walker state written by an evaluation (no LU refresh inside
    the call) follow the oracle's trajectory move for move; the evaluation after them (from the
    carried inverses) matches the oracle, and sweeps continued from the carried state move
    exactly as sweeps continued from a freshly factorised state."""
    mod, ctx = vb
    spec = SYSTEMS[name][0]()
    ctx.set_system(0, spec)
    R0 = S.initial_walkers(spec, W, 15)
    Rt = torch.tensor(R0, device="cuda")
    z = torch.zeros(W, dtype=torch.float64, device="cuda")
    state = torch.zeros((W, ctx.walker_state_size(0)), dtype=torch.float64, device="cuda")
    ctx.eval_walkers(0, 0, Rt, z.clone(), z.clone(), z.clone(), state_out=state)
    nacc = torch.zeros(W, dtype=torch.int32, device="cuda")
    lp, sg, el = z.clone(), z.clone(), z.clone()
    ctx.vmc_steps(0, 0, Rt, nsw, spec.step, 99, step0=3, refresh=0, state=state, state_valid=True, nacc=nacc,
                  logpsi=lp, sign=sg, eloc=el)
    state2 = torch.zeros_like(state)
    ctx.eval_walkers(0, 0, Rt, z.clone(), z.clone(), z.clone(), state_out=state2)
    torch.cuda.synchronize()
    Ro, _, _, no = orc.vmc(spec, R0, nsw, spec.step, seed=99, step0=3, eloc=False)
    np.testing.assert_array_equal(nacc.cpu().numpy(), no)
    np.testing.assert_allclose(Rt.cpu().numpy(), Ro, rtol=0, atol=1e-12)
    ref = orc.evaluate(spec, Ro)
    assert rel_err(el.cpu().numpy(), ref["eloc"]).max() < 1e-10
    assert rel_err(lp.cpu().numpy(), ref["logpsi"]).max() < 1e-10
    Ra, Rb = Rt.clone(), Rt.clone()
    na, nb = torch.zeros_like(nacc), torch.zeros_like(nacc)
    ctx.vmc_steps(0, 0, Ra, 2, spec.step, 99, step0=50, refresh=0, state=state, state_valid=True, nacc=na)
    ctx.vmc_steps(0, 0, Rb, 2, spec.step, 99, step0=50, refresh=0, state=state2, state_valid=True, nacc=nb)
    torch.cuda.synchronize()
    assert torch.equal(na, nb)
    np.testing.assert_allclose(Ra.cpu().numpy(), Rb.cpu().numpy(), rtol=0, atol=1e-12)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name,refresh", [("ethylene_vb", 0), ("small_open_shell", 4)])
def test_carried_evaluation_matches_fresh(vb, orc, name, refresh, precision):
    """Ten walker-steps (one sweep + evaluation with derivatives each) that carry the inverses,
    term ratios and ln|Phi| through the sweeps instead of factorising (refresh 0: never;
    refresh 4: every fourth step) give the evaluation a fresh factorisation gives at the same
    positions (FP64 1e-10 in ln|Psi| and E_L, 1e-8 in derivatives), and the mixed form stays
    within its bounds of the oracle."""
    mod, ctx = vb
    spec = SYSTEMS[name][0]()
    ctx.set_system(0, spec)
    W, P = 48, spec.n_params
    Rt = torch.tensor(S.initial_walkers(spec, W, 77), device="cuda")
    dt = mod.deriv_dtype(precision)
    z = lambda: torch.zeros(W, dtype=torch.float64, device="cuda")
    lp, sg, el = z(), z(), z()
    O = torch.zeros((W, P), dtype=dt, device="cuda")
    dE = torch.zeros_like(O)
    state = torch.zeros((W, ctx.walker_state_size(0)), dtype=torch.float64, device="cuda")
    ctx.eval_walkers(0, precision, Rt, z(), z(), z(), state_out=state)
    for k in range(10):
        ctx.vmc_steps(0, precision, Rt, 1, spec.step, 31, step0=k, refresh=refresh, state=state, state_valid=True,
                      logpsi=lp, sign=sg, eloc=el, O=O, dEL=dE)
    lp2, sg2, el2 = z(), z(), z()
    O2, dE2 = torch.zeros_like(O), torch.zeros_like(O)
    ctx.eval_walkers(0, precision, Rt, lp2, sg2, el2, O=O2, dEL=dE2)
    torch.cuda.synchronize()
    a = {k: v.double().cpu().numpy() for k, v in dict(lp=lp, sg=sg, el=el, O=O, dE=dE).items()}
    b = {k: v.double().cpu().numpy() for k, v in dict(lp=lp2, sg=sg2, el=el2, O=O2, dE=dE2).items()}
    np.testing.assert_array_equal(a["sg"], b["sg"])
    if precision == 0:
        assert rel_err(a["lp"], b["lp"]).max() < 1e-10
        assert rel_err(a["el"], b["el"]).max() < 1e-10
        for key in ("O", "dE"):
            assert np.abs(a[key] - b[key]).max() <= 1e-8 * max(1.0, np.abs(b[key]).max()), key
    else:
        ref = orc.evaluate(spec, Rt.cpu().numpy(), derivs=True)
        dl = np.abs(a["lp"] - ref["logpsi"]).max()
        de = rel_err(a["el"], ref["eloc"]).max()
        print("%s carried mixed: worst |dlnPsi| %.2e, worst rel dE_L %.2e" % (name, dl, de))
        assert dl <= 1e-5 and de <= 1e-4
        for key, rk in (("O", "O"), ("dE", "dEL")):
            assert np.abs(a[key] - ref[rk]).max() <= 2e-3 * max(1.0, np.abs(ref[rk]).max()), key


def _group_mean(E, groups):
    """Mean and standard error from independent groups of walkers: E [steps, walkers]; VMC
    walkers never interact, so the time averages of disjoint walker groups are independent."""
    g = E.reshape(E.shape[0], groups, -1).mean(axis=(0, 2))
    return g.mean(), g.std(ddof=1) / np.sqrt(groups)


def test_vmc_mixed_statistics_match_oracle(vb, orc):
    """Mixed-form VMC of the H2 system: mean E_L agrees with the oracle's within 2 sigma
    (sigma^2 = sigma_gpu^2 + sigma_oracle^2, each from 32 independent walker groups)."""
    spec = S.h2_vb()
    mod, ctx = vb
    ctx.set_system(0, spec)
    W = 8192
    Rt = torch.tensor(S.initial_walkers(spec, W, 9), device="cuda")
    lp = torch.zeros(W, dtype=torch.float64, device="cuda")
    sg, el = torch.zeros_like(lp), torch.zeros_like(lp)
    ctx.vmc_steps(0, 1, Rt, 100, spec.step, 5, step0=0)
    es = []
    for k in range(200):
        ctx.vmc_steps(0, 1, Rt, 1, spec.step, 5, step0=1000 + k, logpsi=lp, sign=sg, eloc=el)
        es.append(el.cpu().numpy().copy())
    g_mean, g_err = _group_mean(np.array(es), 32)
    Wo = 1024
    Ro, _, _, _ = orc.vmc(spec, S.initial_walkers(spec, Wo, 19), 100, spec.step, seed=77, eloc=False)
    _, hist, _, _ = orc.vmc(spec, Ro, 200, spec.step, seed=77, step0=500)
    o_mean, o_err = _group_mean(np.asarray(hist), 32)
    print("H2 VMC mixed: GPU %.5f +- %.5f, oracle %.5f +- %.5f" % (g_mean, g_err, o_mean, o_err))
    assert abs(g_mean - o_mean) < 2 * np.hypot(g_err, o_err), (g_mean, g_err, o_mean, o_err)


def test_zero_walkers_and_ragged_tail(vb, orc):
    mod, ctx = vb
    spec = S.small_open_shell()
    ctx.set_system(0, spec)
    empty = torch.zeros((0, spec.N, 3), dtype=torch.float64, device="cuda")
    z = torch.zeros(0, dtype=torch.float64, device="cuda")
    ctx.eval_walkers(0, 0, empty, z, z, z)
    assert ctx.last_launch_count() == 0
    for W in (1, 17, 31, 33):
        R = S.initial_walkers(spec, W, W)
        got = gpu_eval(vb, spec, R, 0, grad=False)
        ref = orc.evaluate(spec, R)
        assert rel_err(got["eloc"], ref["eloc"]).max() < 1e-10


def test_ethylene_launch_shape(vb):
    """The per-walker shared-memory footprint keeps several walkers per block."""
    mod, ctx = vb
    ctx.set_system(0, S.ethylene_vb())
    for prec, min_eval in ((0, 3), (1, 5)):
        li = ctx.launch_info(0, prec)
        assert li["eval_walkers_per_block"] >= min_eval and li["sweep_walkers_per_block"] >= 8, li
        assert li["eval_smem_per_walker"] * li["eval_walkers_per_block"] <= 232448


def test_full_size_ethylene_sampled(vb, orc):
    """16384 walkers in the benchmark's launch configuration; sampled walkers checked one by one."""
    spec = S.ethylene_vb()
    W = 16384
    R = S.initial_walkers(spec, W, 1)
    for precision, tol_l, tol_e in [(0, 1e-10, 1e-10), (1, 1e-5, 1e-4)]:
        got = gpu_eval(vb, spec, R, precision, derivs=True, grad=False)
        idx = np.array([0, 1, 4095, 8191, 12288, W - 1])
        ref = orc.evaluate(spec, R[idx])
        assert np.abs(got["logpsi"][idx] - ref["logpsi"]).max() <= tol_l * max(1.0, np.abs(ref["logpsi"]).max())
        assert rel_err(got["eloc"][idx], ref["eloc"]).max() <= tol_e
        assert np.all(np.isfinite(got["O"])) and np.all(np.isfinite(got["dEL"]))
        ref_d = orc.evaluate(spec, R[[W - 1]], derivs=True)
        tol_d = 1e-8 if precision == 0 else 2e-3
        assert rel_err(got["O"][W - 1], ref_d["O"][0]).max() < tol_d
