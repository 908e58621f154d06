"""The autograd face and the weighted column sum through the C ABI.

Column sum: against the sums written out in numpy (FP64, 1e-12 relative).  Autograd: the
gradients of sum_w (a_w ln|Psi_w| + b_w E_L,w) with respect to the parameters and the nucleus
positions against the oracle's O_j, E_L,j and nucleus derivatives (FP64 form 1e-8 relative to
the largest entry; mixed form 2e-3), and the forward at moved parameters against the oracle
evaluated there."""
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


@pytest.mark.parametrize("W,K,dtype,two", [(1, 1, torch.float64, True), (37, 5, torch.float64, False),
                                          (1000, 33, torch.float32, True), (16384, 400, torch.float32, True),
                                          (70001, 57, torch.float64, True)])
def test_weighted_colsum(vb, W, K, dtype, two):
    mod, ctx = vb
    g = torch.Generator().manual_seed(W + K)
    Ja = torch.randn(W, K, generator=g, dtype=torch.float64).to(dtype)
    Jb = torch.randn(W, K, generator=g, dtype=torch.float64).to(dtype)
    ga = torch.randn(W, generator=g, dtype=torch.float64)
    gb = torch.randn(W, generator=g, dtype=torch.float64)
    want = ga.numpy() @ Ja.double().numpy() + (gb.numpy() @ Jb.double().numpy() if two else 0.0)
    out = torch.zeros(K, dtype=torch.float64, device="cuda")
    ctx.weighted_colsum(ga.cuda(), Ja.cuda(), out, gb.cuda() if two else None, Jb.cuda() if two else None)
    torch.cuda.synchronize()
    scale = np.abs(ga.numpy())[:, None] * np.abs(Ja.double().numpy())
    if two:
        scale = scale + np.abs(gb.numpy())[:, None] * np.abs(Jb.double().numpy())
    bound = 1e-12 * np.maximum(1.0, scale.sum(0))
    assert (np.abs(out.cpu().numpy() - want) <= bound).all()
    out2 = torch.zeros_like(out)
    ctx.weighted_colsum(ga.cuda(), Ja.cuda(), out2, gb.cuda() if two else None, Jb.cuda() if two else None)
    torch.cuda.synchronize()
    assert torch.equal(out, out2)  # fixed summation order


def test_weighted_colsum_empty(vb):
    mod, ctx = vb
    out = torch.full((7,), 3.0, dtype=torch.float64, device="cuda")
    e = torch.zeros((0, 7), dtype=torch.float64, device="cuda")
    ctx.weighted_colsum(torch.zeros(0, dtype=torch.float64, device="cuda"), e, out)
    torch.cuda.synchronize()
    assert (out.cpu() == 0).all()


@pytest.mark.parametrize("precision,maker,W", [(0, S.small_open_shell, 24), (1, S.ethylene_vb, 16)])
def test_autograd_matches_oracle(vb, orc, precision, maker, W):
    from paper_2207_14715_gb300 import autograd as A
    mod, ctx = vb
    spec = maker()
    R = S.initial_walkers(spec, W, 31)
    p = torch.tensor(A.parameter_vector(spec), requires_grad=True)
    X = torch.tensor(spec.nuc_xyz, requires_grad=True)
    lp, el = A.evaluate(ctx, 3, spec, torch.tensor(R, device="cuda"), precision, params=p, nuclei=X)
    rng = np.random.default_rng(5)
    a, b = rng.normal(size=W), rng.normal(size=W) / W
    loss = (torch.tensor(a, device="cuda") * lp + torch.tensor(b, device="cuda") * el).sum()
    loss.backward()
    ref = orc.evaluate(spec, R, derivs=True)
    nref = orc.nuclear_derivs(spec, R)
    gp = a @ ref["O"] + b @ ref["dEL"]
    gX = np.einsum("w,wad->ad", a, nref["dlogpsi"]) + np.einsum("w,wad->ad", b, nref["dEL"])
    tol = 1e-8 if precision == 0 else 2e-3
    assert np.abs(p.grad.numpy() - gp).max() <= tol * max(1.0, np.abs(gp).max())
    assert np.abs(X.grad.numpy() - gX).max() <= tol * max(1.0, np.abs(gX).max())
    if precision == 0:
        np.testing.assert_allclose(lp.detach().cpu().numpy(), ref["logpsi"], rtol=1e-10)


def test_autograd_forward_at_moved_parameters(vb, orc):
    from paper_2207_14715_gb300 import autograd as A
    mod, ctx = vb
    spec = S.small_open_shell()
    R = S.initial_walkers(spec, 9, 4)
    p = A.parameter_vector(spec)
    nk = len(spec.kappa_kl)
    p[: p.size - nk] += 0.01 * np.random.default_rng(2).normal(size=p.size - nk)
    X = spec.nuc_xyz + 0.05
    lp, el = A.evaluate(ctx, 4, spec, torch.tensor(R, device="cuda"), 0, params=torch.tensor(p),
                        nuclei=torch.tensor(X))
    ref = orc.evaluate(A.with_parameters(spec, p, X), R)
    np.testing.assert_allclose(lp.cpu().numpy(), ref["logpsi"], rtol=1e-10)
    np.testing.assert_allclose(el.cpu().numpy(), ref["eloc"], rtol=1e-10)
