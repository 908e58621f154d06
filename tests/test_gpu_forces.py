"""Nucleus-position derivatives of ln|Psi| and E_L (the ingredients of forces) through the C
ABI against the FP64 oracle, element by element.

Tolerances: FP64 form 1e-9 (d ln|Psi|) and 1e-8 (dE_L) relative to max(1, |x|): the
derivative of E_L carries third derivatives of the Jastrow factor and of the Gaussians, one
cancellation level more than E_L.  Mixed form: 1e-4 and 2e-3 relative to max(1, largest
|x| of the walker), the bounds of the mixed parameter derivatives.
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


def gpu_nuclear(vb, spec, R, precision, eloc_deriv=True):
    mod, ctx = vb
    ctx.set_system(0, spec)
    W = R.shape[0]
    Rt = torch.tensor(R, dtype=torch.float64, device="cuda")
    lp, sg, el = (torch.zeros(W, dtype=torch.float64, device="cuda") for _ in range(3))
    dlp = torch.zeros((W, spec.Nn, 3), dtype=torch.float64, device="cuda")
    dE = torch.zeros_like(dlp) if eloc_deriv else None
    ctx.eval_nuclear_derivs(0, precision, Rt, lp, sg, el, dlp, dE)
    torch.cuda.synchronize()
    out = {"logpsi": lp.cpu().numpy(), "eloc": el.cpu().numpy(), "dlogpsi": dlp.cpu().numpy(),
           "launches": ctx.last_launch_count()}
    if eloc_deriv:
        out["dEL"] = dE.cpu().numpy()
    return out


SYSTEMS = {
    "hydrogenic": (lambda: S.one_electron(3.0, 0.0, a1=-3.0, a2=-0.8), 10),
    "gauss_h": (lambda: S.one_electron(1.0, 0.4), 9),
    "two_electron": (lambda: S.two_electron_product(2.0, 0.9), 11),
    "h2_vb": (S.h2_vb, 33),
    "small_open_shell": (S.small_open_shell, 37),
    "ethylene_vb": (S.ethylene_vb, 6),
}


def _scaled(a, b):
    return np.abs(a - b) / np.maximum(1.0, np.abs(b))


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_nuclear_derivs_fp64_match_oracle(vb, orc, name):
    maker, W = SYSTEMS[name]
    spec = maker()
    R = S.initial_walkers(spec, W, 300 + W)
    ref = orc.nuclear_derivs(spec, R)
    ev = orc.evaluate(spec, R)
    got = gpu_nuclear(vb, spec, R, 0)
    assert _scaled(got["eloc"], ev["eloc"]).max() < 1e-10
    assert _scaled(got["dlogpsi"], ref["dlogpsi"]).max() < 1e-9
    assert _scaled(got["dEL"], ref["dEL"]).max() < 1e-8
    # evaluation (four kernels, no Jastrow-parameter kernel) plus the derivative kernel
    assert got["launches"] == 4


@pytest.mark.parametrize("name", ["h2_vb", "small_open_shell", "ethylene_vb"])
def test_nuclear_derivs_mixed_match_oracle(vb, orc, name):
    maker, W = SYSTEMS[name]
    spec = maker()
    R = S.initial_walkers(spec, W, 400 + W)
    ref = orc.nuclear_derivs(spec, R)
    got = gpu_nuclear(vb, spec, R, 1)
    for key, tol in (("dlogpsi", 1e-4), ("dEL", 2e-3)):
        scale = np.maximum(1.0, np.abs(ref[key]).reshape(W, -1).max(1))[:, None, None]
        err = (np.abs(got[key] - ref[key]) / scale).max()
        assert err < tol, (key, err)


def test_nuclear_derivs_random_molecules(vb, orc):
    """Random molecules of the batched workload (s, p and d shells, 2-32 electrons): two small
    ones and the largest one the nucleus-derivative kernel takes (it refuses systems on
    reference-determinant tables and tables beyond its shared memory, with an error)."""
    mod, ctx = vb
    specs, _ = S.batched_workload(64)
    small = [sp for sp in specs if sp.N <= 10][:2]
    big = None
    for sp in sorted(specs, key=lambda sp: -sp.N):
        try:
            got_big = gpu_nuclear(vb, sp, S.initial_walkers(sp, 3, 72), 0)
        except mod.VbqmcError as e:
            assert "tables" in str(e) or "shared memory" in str(e), str(e)
            continue
        big = sp
        break
    assert big is not None and big.N >= 20, "no molecule of 20 or more electrons was taken"
    print("largest molecule taken: %d electrons" % big.N)
    for k, spec in enumerate(small + [big]):
        R = S.initial_walkers(spec, 3, 70 + k)
        ref = orc.nuclear_derivs(spec, R)
        got = gpu_nuclear(vb, spec, R, 0) if spec is not big else got_big
        assert _scaled(got["dlogpsi"], ref["dlogpsi"]).max() < 1e-9, spec.name
        scale = max(1.0, np.abs(ref["dEL"]).max())
        assert np.abs(got["dEL"] - ref["dEL"]).max() < 1e-8 * scale, spec.name


def test_nuclear_derivs_optional_output_and_empty(vb):
    mod, ctx = vb
    spec = S.h2_vb()
    R = S.initial_walkers(spec, 8, 1)
    a = gpu_nuclear(vb, spec, R, 0)
    b = gpu_nuclear(vb, spec, R, 0, eloc_deriv=False)
    np.testing.assert_array_equal(a["dlogpsi"], b["dlogpsi"])
    z = torch.zeros(0, dtype=torch.float64, device="cuda")
    ctx.eval_nuclear_derivs(0, 0, torch.zeros((0, spec.N, 3), dtype=torch.float64, device="cuda"), z, z, z,
                            torch.zeros((0, spec.Nn, 3), dtype=torch.float64, device="cuda"))


def test_nuclear_derivs_full_size_translation_and_samples(vb, orc):
    """16384 ethylene walkers in the mixed form: translation invariance sum_a d ln|Psi|/dR_a =
    -sum_i grad_i ln|Psi| against the evaluation's own gradient on every walker, and a sample
    of walkers against the oracle."""
    mod, ctx = vb
    spec = S.ethylene_vb()
    W = 16384
    R = S.initial_walkers(spec, W, 2024)
    got = gpu_nuclear(vb, spec, R, 1)
    Rt = torch.tensor(R, device="cuda")
    lp, sg, el = (torch.zeros(W, dtype=torch.float64, device="cuda") for _ in range(3))
    g = torch.zeros_like(Rt)
    ctx.eval_walkers(0, 1, Rt, lp, sg, el, g)
    torch.cuda.synchronize()
    gs = g.cpu().numpy().sum(1)
    scale = np.maximum(1.0, np.abs(got["dlogpsi"]).reshape(W, -1).max(1))[:, None]
    assert (np.abs(got["dlogpsi"].sum(1) + gs) / scale).max() < 1e-3
    assert np.isfinite(got["dEL"]).all()
    idx = np.random.default_rng(0).choice(W, 12, replace=False)
    ref = orc.nuclear_derivs(spec, R[idx])
    for key, tol in (("dlogpsi", 1e-4), ("dEL", 2e-3)):
        sc = np.maximum(1.0, np.abs(ref[key]).reshape(len(idx), -1).max(1))[:, None, None]
        assert (np.abs(got[key][idx] - ref[key]) / sc).max() < tol, key
