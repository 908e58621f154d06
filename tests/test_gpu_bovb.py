"""Breathing-orbital VB (Sec. 2.2, Eq. PsiJBOVB) on the GPU: every structure has its own orbitals,
so no determinant is shared between structures (the ethylene-shaped BOVB system has 24 unique
determinants per spin instead of 8) and each structure's orbital excitations are parameters of
their own.

Against the oracle: FP64 ln|Psi|, E_L within 1e-10 of max(1, |x|), parameter derivatives 1e-8;
mixed |d ln|Psi|| <= 1e-5, relative d E_L <= 1e-4, derivatives 2e-3 of the largest entry; FP64 VMC
trajectories move for move.  The reduction to VBSCF (exact copies of the orbitals) is checked on
the device: the same values, and each shared excitation's derivative equals the sum of its
per-structure copies'."""
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


def _eval(vb, spec, R, precision):
    mod, ctx = vb
    ctx.set_system(0, spec)
    W = R.shape[0]
    Rt = torch.tensor(R, device="cuda")
    lp, sg, el = (torch.zeros(W, dtype=torch.float64, device="cuda") for _ in range(3))
    O = torch.zeros((W, spec.n_params), dtype=mod.deriv_dtype(precision), device="cuda")
    dE = torch.zeros_like(O)
    ctx.eval_walkers(0, precision, Rt, lp, sg, el, None, O, dE)
    torch.cuda.synchronize()
    return {"logpsi": lp.cpu().numpy(), "sign": sg.cpu().numpy(), "eloc": el.cpu().numpy(),
            "O": O.double().cpu().numpy(), "dEL": dE.double().cpu().numpy()}


@pytest.mark.parametrize("precision", [0, 1])
def test_bovb_ethylene_matches_oracle(vb, orc, precision):
    spec = S.ethylene_bovb()
    R = S.initial_walkers(spec, 6, 17)
    ref = orc.evaluate(spec, R, derivs=True)
    got = _eval(vb, spec, R, precision)
    np.testing.assert_array_equal(got["sign"], ref["sign"])
    dl = np.abs(got["logpsi"] - ref["logpsi"])
    de = np.abs(got["eloc"] - ref["eloc"]) / np.maximum(1.0, np.abs(ref["eloc"]))
    print("ethylene BOVB %s: worst |d ln Psi| %.2e (walker %d), worst rel d E_L %.2e (walker %d)" % (
        "mixed" if precision else "fp64", dl.max(), dl.argmax(), de.max(), de.argmax()))
    if precision == 0:
        assert (dl / np.maximum(1.0, np.abs(ref["logpsi"]))).max() < 1e-10 and de.max() < 1e-10
        for k in ("O", "dEL"):
            assert (np.abs(got[k] - ref[k]) / np.maximum(1.0, np.abs(ref[k]))).max() < 1e-8, k
    else:
        assert dl.max() <= 1e-5 and de.max() <= 1e-4
        for k in ("O", "dEL"):
            assert np.abs(got[k] - ref[k]).max() <= 2e-3 * max(1.0, np.abs(ref[k]).max()), k


def test_bovb_reduces_to_vbscf_on_device(vb):
    sp = S.ethylene_vb()
    bo = S.bovb(sp, eps=0.0)
    R = S.initial_walkers(sp, 64, 3)
    a, b = _eval(vb, sp, R, 0), _eval(vb, bo, R, 0)
    np.testing.assert_allclose(b["logpsi"], a["logpsi"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(b["eloc"], a["eloc"], rtol=1e-10, atol=1e-10)
    nk = len(sp.kappa_kl)
    n0 = sp.n_params - nk
    np.testing.assert_allclose(b["O"][:, :n0], a["O"][:, :n0], rtol=1e-10, atol=1e-10)
    q = 0
    for j, (k, l) in enumerate(sp.kappa_kl):
        n = sum(int(l) in (set(sp.inact[sp.inact_off[I]:sp.inact_off[I + 1]]) |
                           set(sp.pairs[sp.pair_off[I]:sp.pair_off[I + 1]].ravel())) for I in range(sp.Nvb))
        cols = list(range(n0 + q, n0 + q + n))
        q += n
        np.testing.assert_allclose(b["O"][:, cols].sum(1), a["O"][:, n0 + j], rtol=1e-9, atol=1e-9)
    assert q == len(bo.kappa_kl)


def test_bovb_vmc_fp64_trajectory_matches_oracle(vb, orc):
    mod, ctx = vb
    spec = S.ethylene_bovb()
    ctx.set_system(0, spec)
    R0 = S.initial_walkers(spec, 4, 9)
    Rt = torch.tensor(R0, device="cuda")
    nacc = torch.zeros(4, dtype=torch.int32, device="cuda")
    ctx.vmc_steps(0, 0, Rt, 2, spec.step, 31, step0=1, nacc=nacc)
    torch.cuda.synchronize()
    Ro, _, _, no = orc.vmc(spec, R0, 2, spec.step, seed=31, step0=1, eloc=False)
    np.testing.assert_array_equal(nacc.cpu().numpy(), no)
    np.testing.assert_allclose(Rt.cpu().numpy(), Ro, rtol=0, atol=1e-12)
