"""VMC sweeps through the reference-determinant tables (Sec. 2.1: the determinants of a spin share
the inactive orbitals and differ from the first one in a few active columns; Sec. 2.3.1:
Metropolis sampling of |Psi|^2).  The sweep carries the reference inverse B, the tables
T = B Phi_X and the minors q_u = D_u/D_0, updated by Sherman-Morrison and a rank-1 change of T
per accepted move.

FP64 form against the oracle on the same Philox streams: accepted-move counts equal and positions
within 1e-12 (only a decision within rounding of its threshold could differ), on systems switched
to the tables (vbqmc_use_tables) and on the 48-electron system, which uses them by itself.  Mixed
form: the same proposals, so positions agree with the FP64 form's except where a decision falls
within float rounding of its threshold; after equilibration the 48-electron walkers evaluate to
finite values that match the oracle within the mixed bounds (|d ln|Psi|| <= 1e-5, relative
d E_L <= 1e-4)."""
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


def _sweeps(vb, spec, R0, precision, nsw, seed, step0, tables=True, refresh=0):
    mod, ctx = vb
    ctx.set_system(0, spec)
    if tables:
        ctx.use_tables(0, True)
    W = R0.shape[0]
    Rt = torch.tensor(R0, device="cuda")
    nacc = torch.zeros(W, dtype=torch.int32, device="cuda")
    ctx.vmc_steps(0, precision, Rt, nsw, spec.step, seed, step0=step0, refresh=refresh, nacc=nacc)
    torch.cuda.synchronize()
    return Rt.cpu().numpy(), nacc.cpu().numpy()


@pytest.mark.parametrize("maker, W, nsw, refresh", [(S.small_open_shell, 19, 3, 0), (S.h2_vb, 33, 4, 2),
                                                    (S.ethylene_vb, 5, 2, 0), (S.ethylene_vb, 4, 3, 1)])
def test_table_sweep_fp64_matches_oracle(vb, orc, maker, W, nsw, refresh):
    spec = maker()
    R0 = S.initial_walkers(spec, W, 31)
    Rg, ng = _sweeps(vb, spec, R0, 0, nsw, seed=404, step0=7, refresh=refresh)
    Ro, _, _, no = orc.vmc(spec, R0, nsw, spec.step, seed=404, step0=7, eloc=False)
    np.testing.assert_array_equal(ng, no)
    np.testing.assert_allclose(Rg, Ro, rtol=0, atol=1e-12)


def test_table_sweep_equals_inverse_sweep(vb):
    """The two ways of carrying the determinants make the same decisions (FP64 form)."""
    spec = S.ethylene_vb()
    R0 = S.initial_walkers(spec, 256, 8)
    Ra, na = _sweeps(vb, spec, R0, 0, 3, seed=5, step0=0, tables=True)
    Rb, nb = _sweeps(vb, spec, R0, 0, 3, seed=5, step0=0, tables=False)
    assert (na == nb).mean() > 0.99
    same = np.all(np.abs(Ra - Rb) < 1e-10, axis=(1, 2))
    assert same.mean() > 0.99, same.mean()


def test_table_sweep_mixed_follows_fp64(vb):
    spec = S.ethylene_vb()
    R0 = S.initial_walkers(spec, 512, 12)
    Ra, na = _sweeps(vb, spec, R0, 0, 2, seed=77, step0=3)
    Rb, nb = _sweeps(vb, spec, R0, 1, 2, seed=77, step0=3)
    same = np.all(np.abs(Ra - Rb) < 1e-9, axis=(1, 2))
    assert same.mean() > 0.97, same.mean()


def test_dmc48_sweep_fp64_matches_oracle(vb, orc):
    spec = S.dmc48()
    R0 = S.initial_walkers(spec, 12, 44)
    Rg, ng = _sweeps(vb, spec, R0, 0, 1, seed=9, step0=2, tables=False)
    Ro, _, _, no = orc.vmc(spec, R0, 1, spec.step, seed=9, step0=2, eloc=False)
    np.testing.assert_array_equal(ng, no)
    np.testing.assert_allclose(Rg, Ro, rtol=0, atol=1e-12)


def test_dmc48_equilibrates_by_vmc(vb, orc):
    """4096 walkers of the 48-electron system, mixed form, 40 sweeps refreshed every 10: every
    walker finite, moves accepted, the mean E_L rises from the initial configurations' outliers
    towards the VMC energy, and sampled walkers evaluate as in the oracle."""
    mod, ctx = vb
    spec = S.dmc48()
    ctx.set_system(0, spec)
    W = 4096
    R = torch.tensor(S.initial_walkers(spec, W, 3), device="cuda")
    lp, sg, el = (torch.zeros(W, dtype=torch.float64, device="cuda") for _ in range(3))
    ctx.eval_walkers(0, 1, R, lp, sg, el)
    e_start = el.cpu().numpy()
    nacc = torch.zeros(W, dtype=torch.int32, device="cuda")
    ctx.vmc_steps(0, 1, R, 40, spec.step, 123, step0=0, refresh=10, nacc=nacc, logpsi=lp, sign=sg, eloc=el)
    torch.cuda.synchronize()
    e_end = el.cpu().numpy()
    acc = nacc.cpu().numpy().sum() / (40.0 * W * spec.N)
    print("dmc48 VMC: acceptance %.3f, E_L median %.2f -> %.2f, min %.3g -> %.3g" % (
        acc, np.median(e_start), np.median(e_end), e_start.min(), e_end.min()))
    assert np.isfinite(e_end).all() and np.isfinite(lp.cpu().numpy()).all()
    assert 0.05 < acc < 0.98
    idx = np.random.default_rng(0).choice(W, 4, replace=False)
    ref = orc.evaluate(spec, R.cpu().numpy()[idx])
    assert np.abs(lp.cpu().numpy()[idx] - ref["logpsi"]).max() <= 1e-5
    assert (np.abs(e_end[idx] - ref["eloc"]) / np.maximum(1, np.abs(ref["eloc"]))).max() <= 1e-4
