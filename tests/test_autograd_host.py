"""Host side of the autograd face (no GPU): the parameter vector follows the library's (and the
oracle's) parameter order, checked against the oracle's own derivatives O_j by finite
differences along each direction of with_parameters."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2207_14715_gb300 import autograd as A  # noqa: E402
from paper_2207_14715_gb300 import systems as S  # noqa: E402


@pytest.mark.parametrize("maker", [S.small_open_shell, S.ethylene_vb])
def test_parameter_order_matches_oracle(orc, maker):
    spec = maker()
    p0 = A.parameter_vector(spec)
    assert p0.size == spec.n_params == orc.num_params(spec)
    R = S.initial_walkers(spec, 2, 6)
    O = orc.evaluate(spec, R, derivs=True)["O"]
    nk = len(spec.kappa_kl)
    js = list(range(0, spec.n_params - nk, max(1, (spec.n_params - nk) // 12)))
    h = 1e-5
    for j in js:
        e = np.zeros_like(p0)
        e[j] = h
        lp = orc.evaluate(A.with_parameters(spec, p0 + e), R)["logpsi"]
        lm = orc.evaluate(A.with_parameters(spec, p0 - e), R)["logpsi"]
        np.testing.assert_allclose((lp - lm) / (2 * h), O[:, j], rtol=1e-5, atol=1e-7)


def test_with_parameters_round_trip_and_kappa_zero():
    spec = S.small_open_shell()
    p0 = A.parameter_vector(spec)
    s2 = A.with_parameters(spec, p0, spec.nuc_xyz + 0.5)
    np.testing.assert_array_equal(A.parameter_vector(s2), p0)
    np.testing.assert_array_equal(s2.nuc_xyz, spec.nuc_xyz + 0.5)
    np.testing.assert_array_equal(spec.nuc_xyz, S.small_open_shell().nuc_xyz)
    if len(spec.kappa_kl):
        bad = p0.copy()
        bad[-1] = 0.1
        with pytest.raises(ValueError, match="kappa"):
            A.with_parameters(spec, bad)
    with pytest.raises(ValueError):
        A.with_parameters(spec, p0[:-1])
