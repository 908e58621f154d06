"""Overlap matrix and weights of the JVB structures (arXiv:2207.14715, Sec. 2.4) from samples
evaluated on the GPU (the structure-coefficient derivatives Psi_I/Psi_0 of the evaluation, then
vbqmc_structure_overlap: double products and sums on the device, the row of a structure left out
of the parameters rebuilt per sample from sum_I c_I Psi_I/Psi_0 = 1) against the oracle's ratios
on the same points.

Tolerances are derived, not fitted.  Each ratio R_I = Phi_I/Phi is within eps_R relative of the
oracle's, eps_R = 1e-10 in the FP64 form and 2e-5 in the mixed form (the bounds on ln|Psi|,
1e-10 and 1e-5, taken for ln|Phi_I| and ln|Phi| each); the rebuilt ratio inherits
eps_R sum_J |c_J R_J| / |c_I0|.  To first order that bounds each entry of S by
B_IJ = <E_I |R_J| + |R_I| E_J> (E the pointwise ratio bounds), the Chirgwin-Coulson weights by
perturbing c_I (Sc)_I / c^T S c with |dS| <= B, and the Loewdin weights through
|d S^1/2| <= |B|_F / (2 sqrt(lambda_min(S))) (so S's conditioning enters).  The FP64 weights
are in addition required within 1e-8 absolute."""
import dataclasses

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


def _derivs(vb, spec, R, precision):
    mod, ctx = vb
    ctx.set_system(0, spec)
    W = R.shape[0]
    Rt = torch.tensor(R, dtype=torch.float64, device="cuda")
    z = lambda: torch.zeros(W, dtype=torch.float64, device="cuda")
    O = torch.zeros((W, spec.n_params), dtype=mod.deriv_dtype(precision), device="cuda")
    dE = torch.zeros_like(O)
    ctx.eval_walkers(0, precision, Rt, z(), z(), z(), None, O, dE)
    torch.cuda.synchronize()
    return O


# (system, walkers, structure-coefficient parameters: None keeps the system's own, which leave
# out the first structure; a list replaces them -- all structures: no row to rebuild)
CASES = [("ethylene_vb", S.ethylene_vb, 256, None), ("h2_vb", S.h2_vb, 96, [1, 2]),
         ("small_open_shell_all", S.small_open_shell, 80, [0, 1, 2, 3])]


@pytest.mark.parametrize("name, maker, W, cparam", CASES)
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("weighted", [False, True])
def test_structure_overlap_and_weights_match_oracle(vb, orc, name, maker, W, cparam, precision, weighted):
    mod, ctx = vb
    spec = maker()
    if cparam is not None:
        spec = dataclasses.replace(spec, cparam=np.asarray(cparam, dtype=np.int32))
    R = S.initial_walkers(spec, W, 500 + W)
    w = np.random.default_rng(W).uniform(0.3, 1.7, W) if weighted else None
    O = _derivs(vb, spec, R, precision)
    wt = torch.tensor(w, device="cuda") if weighted else None
    S_gpu = ctx.structure_overlap(precision, O, spec.cparam, spec.c_vb, weights=wt)
    torch.cuda.synchronize()
    X = orc.structure_ratios(spec, R)
    S_ref = orc.structure_overlap(X, w)
    c = np.asarray(spec.c_vb, np.float64)
    eps = 1e-10 if precision == 0 else 2e-5
    E = eps * np.abs(X)
    missing = [I for I in range(len(c)) if I not in list(spec.cparam)]
    for I0 in missing:
        E[:, I0] = eps * (np.abs(X) * np.abs(c)).sum(1) / abs(c[I0])
    ww = np.ones(W) if w is None else w
    B = (ww[:, None, None] * (E[:, :, None] * np.abs(X)[:, None, :] + np.abs(X)[:, :, None] * E[:, None, :])).sum(0)
    B = B / ww.sum() + 1e-15 * np.abs(S_ref).max()
    err = np.abs(S_gpu - S_ref)
    assert (err <= B).all(), (err.max(), (err / B).max())
    w_cc, w_l = mod.structure_weights(S_gpu, c)
    r_cc, r_l = orc.structure_weights(S_ref, c)
    n = c @ S_ref @ c
    Bc = B @ np.abs(c)
    tol_cc = (np.abs(c) * Bc + np.abs(r_cc) * (np.abs(c) @ Bc)) / n + 1e-14
    lam_min = np.linalg.eigvalsh(0.5 * (S_ref + S_ref.T)).min()
    lam, U = np.linalg.eigh(0.5 * (S_ref + S_ref.T))
    cb = (U * np.sqrt(np.clip(lam, 0, None))) @ U.T @ c
    tol_l = 4.0 * np.linalg.norm(B) / (2.0 * np.sqrt(lam_min)) * np.linalg.norm(c) / np.linalg.norm(cb) + 1e-14
    assert (np.abs(w_cc - r_cc) <= tol_cc).all(), (np.abs(w_cc - r_cc).max(), tol_cc.max())
    assert np.abs(w_l - r_l).max() <= tol_l, (np.abs(w_l - r_l).max(), tol_l)
    if precision == 0:
        assert np.abs(w_cc - r_cc).max() <= 1e-8 and np.abs(w_l - r_l).max() <= 1e-8
    assert abs(w_cc.sum() - 1) < 1e-12 and abs(w_l.sum() - 1) < 1e-12
    print("%s %s: |dS| %.1e (bound %.1e), |dw_CC| %.1e, |dw_L| %.1e (bound %.1e), cond(S) %.1e" % (
        name, "fp64" if precision == 0 else "mixed", err.max(), B.max(), np.abs(w_cc - r_cc).max(),
        np.abs(w_l - r_l).max(), tol_l, lam.max() / lam_min))
