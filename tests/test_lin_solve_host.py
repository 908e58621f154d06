"""The library's host FP64 solve of the linear method (vbqmc_lin_solve, Sec. 2.3.1 Eq.
geneigeqM) and its structure-weight routine (vbqmc_structure_weights, Sec. 2.4), run on the CPU:
both are host code of the C ABI and need no device.

Pins: the one-parameter pencil in closed form (a quadratic), the strong zero-variance limit of
the two-structure 1s system (exact state Delta c2 / (1 - Delta c2 <O>) = -c2, E = -Z^2/2), the
invariance of the update under a duplicated (redundant) parameter, and agreement with the
oracle's generalized eigensolver (LAPACK dggev through scipy) on random pencils up to P = 400."""
import math

import numpy as np
import pytest

from paper_2207_14715_gb300 import systems as S
from paper_2207_14715_gb300 import vbqmc


def _pencil(rng, P, M=None):
    M = M or max(4 * P, 60)
    O = rng.normal(size=(M, P)) * rng.uniform(0.1, 3.0, size=P)
    dE = 0.3 * rng.normal(size=(M, P))
    EL = -10.0 + rng.normal(size=M)
    return O, dE, EL


@pytest.mark.parametrize("E0, gL, gR, h, s", [(-1.0, 0.4, 0.6, -0.5, 2.0), (3.0, -1.0, 2.0, 5.0, 0.5),
                                             (-7.5, 0.01, 0.02, -7.4, 1.0)])
def test_one_parameter_closed_form(E0, gL, gR, h, s):
    """P = 1: det(A - E B) = (E0 - E)(h - E s) - gL gR / 4 = 0.  With d = E - E0 this is
    s d^2 - q d - gL gR / 4 = 0, q = h - E0 s; the lowest root d = (q - r) / (2 s),
    r = sqrt(q^2 + s gL gR), written without cancellation, and the eigenvector's ratio
    v1 / v0 = 2 d / gR from the first row."""
    q = h - E0 * s
    r = math.sqrt(q * q + s * gL * gR)
    d = -gL * gR / (2.0 * (q + r)) if q > 0 else (q - r) / (2.0 * s)
    dp, e = vbqmc.lin_solve(E0, [gL], [gR], [[h]], [[s]])
    assert e == pytest.approx(E0 + d, rel=1e-13, abs=1e-13)
    assert dp[0] == pytest.approx(2.0 * d / gR, rel=1e-11)


@pytest.mark.parametrize("Z, c2", [(1.0, 0.7), (2.0, -0.3), (3.0, -0.4)])
def test_strong_zero_variance(orc, Z, c2):
    """Psi = J (Phi_1 + c2 Phi_2) with J = exp(-Z r) exact: any sample gives the exact state."""
    spec = S.two_structure_1s(Z, 0.9, c2)
    R = np.random.default_rng(7).normal(scale=1.0 / Z, size=(25, 1, 3))
    ev = orc.evaluate(spec, R, derivs=True)
    m = orc.lin_matrices(ev["O"], ev["dEL"], ev["eloc"])
    dp, e = vbqmc.lin_solve(m["E0"], m["gL"], m["gR"], m["H"], m["S"])
    obar = ev["O"][:, 0].mean()
    assert dp[0] / (1.0 - dp[0] * obar) == pytest.approx(-c2, rel=1e-10, abs=1e-12)
    assert e == pytest.approx(-0.5 * Z * Z, rel=1e-10)


def test_duplicated_parameter_is_redundant(orc):
    """Appending a copy of a parameter's derivative column makes S singular; the solve must drop
    that direction and return the same energy, with the two copies' updates summing to the
    update of the single parameter."""
    rng = np.random.default_rng(11)
    O, dE, EL = _pencil(rng, 6)
    m = orc.lin_matrices(O, dE, EL)
    dp, e = vbqmc.lin_solve(m["E0"], m["gL"], m["gR"], m["H"], m["S"])
    O2 = np.concatenate([O, O[:, 2:3]], axis=1)
    dE2 = np.concatenate([dE, dE[:, 2:3]], axis=1)
    m2 = orc.lin_matrices(O2, dE2, EL)
    dp2, e2 = vbqmc.lin_solve(m2["E0"], m2["gL"], m2["gR"], m2["H"], m2["S"])
    assert e2 == pytest.approx(e, rel=1e-10)
    np.testing.assert_allclose(np.delete(dp2, [2, 6]), np.delete(dp, 2), rtol=0, atol=1e-8 * np.abs(dp).max())
    assert dp2[2] + dp2[6] == pytest.approx(dp[2], rel=1e-8, abs=1e-10)


@pytest.mark.parametrize("P, shift", [(1, 0.0), (3, 0.0), (17, 0.2), (64, 0.0), (150, 1.0), (400, 0.0)])
def test_matches_oracle_eigensolver(orc, P, shift):
    O, dE, EL = _pencil(np.random.default_rng(P), P)
    m = orc.lin_matrices(O, dE, EL)
    dp, e = vbqmc.lin_solve(m["E0"], m["gL"], m["gR"], m["H"], m["S"], shift=shift)
    dpo, eo = orc.lin_solve(m["E0"], m["gL"], m["gR"], m["H"], m["S"], shift=shift)
    assert e == pytest.approx(eo, rel=1e-11)
    np.testing.assert_allclose(dp, dpo, rtol=0, atol=1e-8 * np.abs(dpo).max())


def test_rejects_bad_input():
    with pytest.raises(vbqmc.VbqmcError):
        vbqmc.lin_solve(0.0, [np.nan], [0.0], [[1.0]], [[1.0]])
    with pytest.raises(vbqmc.VbqmcError):
        vbqmc.lin_solve(0.0, [1.0], [1.0], [[1.0]], [[0.0]])  # S has no positive eigenvalue
    with pytest.raises(vbqmc.VbqmcError):
        vbqmc.structure_weights([[1.0, 0.0], [0.0, 1.0]], [0.0, 0.0])


def test_structure_weights_match_oracle(orc):
    rng = np.random.default_rng(3)
    for n in (1, 2, 6, 20):
        A = rng.normal(size=(n, n))
        Sm = A @ A.T + 0.05 * np.eye(n)
        c = rng.normal(size=n)
        got, ref = vbqmc.structure_weights(Sm, c), orc.structure_weights(Sm, c)
        np.testing.assert_allclose(got[0], ref[0], rtol=0, atol=1e-12)
        np.testing.assert_allclose(got[1], ref[1], rtol=0, atol=1e-12)


def test_ill_conditioned_overlap_matches_oracle(orc):
    """64 samples of the small open-shell system with 57 parameters: S has eigenvalues from 1e-16
    to 1e2 (near-redundant parameters), the regime where a reduction by S^-1/2 alone loses the
    eigenvector.  The solve must still agree with the oracle's QZ-based solve on the same
    matrices: E to 1e-12 and the update in the S-norm (the change of the wave function) to 1e-10."""
    spec = S.small_open_shell()
    R = S.initial_walkers(spec, 64, 12)
    R, _, _, _ = orc.vmc(spec, R, 20, spec.step, seed=4, eloc=False)
    ev = orc.evaluate(spec, R, derivs=True)
    m = orc.lin_matrices(ev["O"], ev["dEL"], ev["eloc"])
    assert np.linalg.eigvalsh(m["S"]).min() < 1e-9 * np.linalg.eigvalsh(m["S"]).max()
    sn = lambda v: np.sqrt(max(v @ m["S"] @ v, 0.0))
    for shift in (0.1, 0.5, 1.0):
        dp, e = vbqmc.lin_solve(m["E0"], m["gL"], m["gR"], m["H"], m["S"], shift=shift)
        dpo, eo = orc.lin_solve(m["E0"], m["gL"], m["gR"], m["H"], m["S"], shift=shift)
        assert e == pytest.approx(eo, rel=1e-12)
        assert sn(dp - dpo) <= 1e-10 * sn(dpo)
