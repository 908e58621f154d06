"""Slater-type shells on the GPU (Sec. 2.1: the paper's all-electron basis, whose 1s shells carry
the nuclear cusp, so that the e-n Jastrow term has a_1 = 0), against the oracle.

Tolerances as for Gaussian systems: FP64 ln|Psi| and E_L within 1e-10 of max(1, |x|), parameter
derivatives 1e-8; mixed |d ln|Psi|| <= 1e-5, relative d E_L <= 1e-4 (worst walker printed),
derivatives 2e-3 of the largest entry.  Exact pins on the device: E_L = -Z^2/2 for the 1s Slater
orbital with zeta = Z, in both forms."""
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


def _eval(vb, spec, R, precision, derivs=False):
    mod, ctx = vb
    ctx.set_system(0, spec)
    W = R.shape[0]
    Rt = torch.tensor(R, device="cuda")
    lp, sg, el = (torch.zeros(W, dtype=torch.float64, device="cuda") for _ in range(3))
    O = dE = None
    if derivs:
        O = torch.zeros((W, spec.n_params), dtype=mod.deriv_dtype(precision), device="cuda")
        dE = torch.zeros_like(O)
    ctx.eval_walkers(0, precision, Rt, lp, sg, el, None, O, dE)
    torch.cuda.synchronize()
    out = {"logpsi": lp.cpu().numpy(), "sign": sg.cpu().numpy(), "eloc": el.cpu().numpy()}
    if derivs:
        out["O"] = O.double().cpu().numpy()
        out["dEL"] = dE.double().cpu().numpy()
    return out


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("Z", [1.0, 3.0, 8.0])
def test_slater_1s_exact_on_device(vb, precision, Z):
    spec = S.slater_1s(Z, Z)
    R = np.random.default_rng(int(Z)).normal(scale=1.0 / Z, size=(64, 1, 3))
    got = _eval(vb, spec, R, precision)
    tol = 1e-12 if precision == 0 else 1e-6
    np.testing.assert_allclose(got["eloc"], -0.5 * Z * Z, rtol=tol)


@pytest.mark.parametrize("precision", [0, 1])
def test_slater_h2_matches_oracle(vb, orc, precision):
    spec = S.slater_h2()
    R = S.initial_walkers(spec, 40, 21)
    ref = orc.evaluate(spec, R, derivs=True)
    got = _eval(vb, spec, R, precision, derivs=True)
    np.testing.assert_array_equal(got["sign"], ref["sign"])
    dl = np.abs(got["logpsi"] - ref["logpsi"])
    de = np.abs(got["eloc"] - ref["eloc"]) / np.maximum(1.0, np.abs(ref["eloc"]))
    print("slater_h2 %s: worst |d ln Psi| %.2e (walker %d), worst rel d E_L %.2e (walker %d)" % (
        "mixed" if precision else "fp64", dl.max(), dl.argmax(), de.max(), de.argmax()))
    if precision == 0:
        assert (dl / np.maximum(1.0, np.abs(ref["logpsi"]))).max() < 1e-10 and de.max() < 1e-10
        for k in ("O", "dEL"):
            assert (np.abs(got[k] - ref[k]) / np.maximum(1.0, np.abs(ref[k]))).max() < 1e-8, k
    else:
        assert dl.max() <= 1e-5 and de.max() <= 1e-4
        for k in ("O", "dEL"):
            assert np.abs(got[k] - ref[k]).max() <= 2e-3 * max(1.0, np.abs(ref[k]).max()), k


def test_slater_vmc_fp64_trajectory_matches_oracle(vb, orc):
    mod, ctx = vb
    spec = S.slater_h2()
    ctx.set_system(0, spec)
    R0 = S.initial_walkers(spec, 33, 2)
    Rt = torch.tensor(R0, device="cuda")
    nacc = torch.zeros(33, dtype=torch.int32, device="cuda")
    ctx.vmc_steps(0, 0, Rt, 4, spec.step, 61, step0=2, nacc=nacc)
    torch.cuda.synchronize()
    Ro, _, _, no = orc.vmc(spec, R0, 4, spec.step, seed=61, step0=2, eloc=False)
    np.testing.assert_array_equal(nacc.cpu().numpy(), no)
    np.testing.assert_allclose(Rt.cpu().numpy(), Ro, rtol=0, atol=1e-12)


def test_slater_nuclear_derivatives_refused(vb):
    mod, ctx = vb
    spec = S.slater_h2()
    ctx.set_system(0, spec)
    R = torch.tensor(S.initial_walkers(spec, 2, 1), device="cuda")
    z = torch.zeros(2, dtype=torch.float64, device="cuda")
    d = torch.zeros((2, 2, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(mod.VbqmcError, match="Slater"):
        ctx.eval_nuclear_derivs(0, 0, R, z, z, z, d)
