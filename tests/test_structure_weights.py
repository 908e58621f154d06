"""Structure overlap and weights of the JVB structures (arXiv:2207.14715, Sec. 2.4): the oracle's
ratios Psi_I/Psi_0, and the weight formulas of the oracle and of the library
(vbqmc_structure_weights, host code of the C ABI), against closed forms and identities.  (The
GPU side of the overlap is in test_gpu_structure_weights.py.)"""
import dataclasses
import math

import numpy as np
import pytest

from paper_2207_14715_gb300 import systems as S
from paper_2207_14715_gb300 import vbqmc


def _cc_closed(c1, c2, s):
    # two structures with unit self-overlap and mutual overlap s
    norm = c1 * c1 + c2 * c2 + 2 * s * c1 * c2
    return np.array([c1 * (c1 + s * c2), c2 * (c2 + s * c1)]) / norm


def _lowdin_closed(c1, c2, s):
    # S^(1/2) of [[1, s], [s, 1]] is [[a, b], [b, a]] with a, b from the eigenvalues 1 +- s
    a = 0.5 * (math.sqrt(1 + s) + math.sqrt(1 - s))
    b = 0.5 * (math.sqrt(1 + s) - math.sqrt(1 - s))
    cb = np.array([a * c1 + b * c2, b * c1 + a * c2])
    return cb ** 2 / np.sum(cb ** 2)


@pytest.mark.parametrize("c1, c2, s", [(1.0, 0.3, 0.4), (0.7, -0.5, 0.25), (1.0, 1.0, -0.6)])
def test_weights_two_structures_closed_form(orc, c1, c2, s):
    Sm = np.array([[1.0, s], [s, 1.0]])
    for fn in (orc.structure_weights, vbqmc.structure_weights):
        w_cc, w_l = fn(Sm, [c1, c2])
        np.testing.assert_allclose(w_cc, _cc_closed(c1, c2, s), rtol=0, atol=1e-13)
        np.testing.assert_allclose(w_l, _lowdin_closed(c1, c2, s), rtol=0, atol=1e-13)


def test_weights_orthogonal_structures_agree_and_sum_to_one(orc):
    rng = np.random.default_rng(5)
    d = rng.uniform(0.2, 2.0, 5)
    c = rng.uniform(-1, 1, 5)
    ref = c * c * d / np.sum(c * c * d)
    for fn in (orc.structure_weights, vbqmc.structure_weights):
        w_cc, w_l = fn(np.diag(d), c)
        np.testing.assert_allclose(w_cc, ref, atol=1e-14)
        np.testing.assert_allclose(w_l, ref, atol=1e-14)
    A = rng.normal(size=(6, 6))
    Sm = A @ A.T + 0.1 * np.eye(6)
    c = rng.normal(size=6)
    for fn in (orc.structure_weights, vbqmc.structure_weights):
        w_cc, w_l = fn(Sm, c)
        assert abs(w_cc.sum() - 1) < 1e-13 and abs(w_l.sum() - 1) < 1e-13
    np.testing.assert_allclose(vbqmc.structure_weights(Sm, c)[1], orc.structure_weights(Sm, c)[1], atol=1e-12)


@pytest.mark.parametrize("maker, W", [(S.h2_vb, 40), (S.small_open_shell, 24), (S.ethylene_vb, 6)])
def test_oracle_ratios_resolve_the_wave_function(orc, maker, W):
    """sum_I c_I Psi_I/Psi_0 = 1 at every point, and the sample overlap then satisfies
    c^T S c = 1 (the normalisation <Psi_0|Psi_0> of the estimator)."""
    spec = maker()
    R = S.initial_walkers(spec, W, 17)
    X = orc.structure_ratios(spec, R)
    c = np.asarray(spec.c_vb)
    assert np.abs(X @ c - 1).max() < 1e-10 * max(1.0, np.abs(X).max())
    Sm = orc.structure_overlap(X)
    assert abs(c @ Sm @ c - 1) < 1e-10


def test_oracle_single_structure(orc):
    """One structure: Psi_0 = c_0 Psi_1, so the ratio is 1/c_0 everywhere and the weight is 1."""
    spec = S.two_electron_product(2.0, 0.9)
    assert len(spec.c_vb) == 1
    R = S.initial_walkers(spec, 10, 3)
    X = orc.structure_ratios(spec, R)
    np.testing.assert_allclose(X, 1.0 / spec.c_vb[0], rtol=1e-13)
    w_cc, w_l = orc.structure_weights(orc.structure_overlap(X), spec.c_vb)
    np.testing.assert_allclose(w_cc, [1.0])
    np.testing.assert_allclose(w_l, [1.0])


@pytest.mark.parametrize("maker, keep", [(S.h2_vb, [0]), (S.h2_vb, [1, 2]), (S.ethylene_vb, [0, 2, 5]),
                                         (S.small_open_shell, [3, 1])])
def test_structure_subset_is_the_expansion_with_the_others_removed(orc, maker, keep):
    """A subset of structures (the wave function of a resonance-energy diabatic state) evaluates
    like the full expansion with the other coefficients set to zero: same ln|Psi|, sign and E_L."""
    spec = maker()
    sub = S.structure_subset(spec, keep)
    zeroed = dataclasses.replace(spec, c_vb=np.where(np.isin(np.arange(len(spec.c_vb)), keep), spec.c_vb, 0.0))
    R = S.initial_walkers(spec, 8, 4)
    a, b = orc.evaluate(sub, R), orc.evaluate(zeroed, R)
    np.testing.assert_allclose(a["logpsi"], b["logpsi"], rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(a["sign"], b["sign"])
    np.testing.assert_allclose(a["eloc"], b["eloc"], rtol=1e-10, atol=1e-10)
    assert len(sub.c_vb) == len(keep)
