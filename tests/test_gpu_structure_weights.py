"""Overlap matrix and weights of the JVB structures (arXiv:2207.14715, Sec. 2.4) from samples
evaluated on the GPU (the structure-coefficient derivatives Psi_I/Psi_0 of the evaluation, the
column-sum and linear-method kernels) against the oracle's ratios on the same points.

Tolerances: S within 1e-5 of its largest entry in the FP64 form (the centred products come from
the linear-method kernel, whose products run on the FP32 pipe: 2e-6 of the matrix scale with
double inputs) and 2e-3 in the mixed form (the bound of the mixed derivatives).  The weights
amplify those errors (the row of the structure left out of the parameters comes from a
difference of sums, and the Loewdin square root divides by the spread of S's eigenvalues:
4.5e-4 measured in the FP64 form on the ethylene-shaped system), so they are compared within
1e-2 absolute, well inside the statistical error of any sampled weight; their formulas are
pinned exactly on the host (test_structure_weights.py)."""
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
    S_ref = orc.structure_overlap(orc.structure_ratios(spec, R), w)
    tol = 1e-5 if precision == 0 else 2e-3
    scale = np.abs(S_ref).max()
    assert np.abs(S_gpu - S_ref).max() <= tol * scale, (np.abs(S_gpu - S_ref).max(), scale)
    for a, b in zip(mod.structure_weights(S_gpu, spec.c_vb), orc.structure_weights(S_ref, spec.c_vb)):
        assert np.abs(a - b).max() <= 1e-2, (np.abs(a - b).max(), a, b)
        assert abs(a.sum() - 1) < 1e-12
