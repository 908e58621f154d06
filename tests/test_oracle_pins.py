"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: published known-answer
vectors, closed forms, exact quadrature, brute force in Fock space, finite differences,
invariants, and textbook limits.  Paper passages: arXiv:2207.14715, Sec. 2.
"""
import itertools
import math
import os

import numpy as np
import pytest

from paper_2207_14715_gb300 import systems as S

HERE = os.path.dirname(os.path.abspath(__file__))


# ----------------------------------------------------------------------------- RNG
def test_philox_known_answers(orc):
    """Philox4x32-10 against the vectors published with Random123 (Salmon et al., SC'11)."""
    n = 0
    for line in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        assert orc.philox4x32_10(v[:4], v[4:6]) == v[6:]
        n += 1
    assert n == 3


def test_uniform_stream_moments(orc):
    u = np.array([orc.uniforms2(1234, w, 5, 0, 0, 0) for w in range(4000)]).ravel()
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 4 * math.sqrt(1 / 12 / len(u))


# ----------------------------------------------------------------------------- basis
def _basis_exponents(l):
    return {0: [(0, 0, 0)], 1: [(1, 0, 0), (0, 1, 0), (0, 0, 1)],
            2: [(2, 0, 0), (0, 2, 0), (0, 0, 2), (1, 1, 0), (1, 0, 1), (0, 1, 1)]}[l]


def test_basis_normalisation_gauss_hermite(orc):
    """Each normalised cartesian Gaussian integrates to 1 (exact Gauss-Hermite quadrature)."""
    spec = S.small_open_shell()
    xg, wg = np.polynomial.hermite.hermgauss(20)
    mu = 0
    for sh, (c, l) in enumerate(zip(spec.sh_center, spec.sh_l)):
        z = spec.sh_zeta[sh]
        for (a, b, cc) in _basis_exponents(int(l)):
            # value of chi at a point reveals the normalisation: chi(r) = N x^a y^b z^c e^{-z r^2}
            r = spec.nuc_xyz[c] + np.array([0.31, -0.22, 0.17])
            chi, _, _ = orc.basis_eval(spec, r)
            d = r - spec.nuc_xyz[c]
            N = chi[mu] / (d[0] ** a * d[1] ** b * d[2] ** cc * math.exp(-z * d @ d))
            # integral of x^{2a} e^{-2 z x^2} dx with x = X / sqrt(2z)
            one_d = [np.sum(wg * (xg / math.sqrt(2 * z)) ** (2 * e)) / math.sqrt(2 * z) for e in (a, b, cc)]
            assert N * N * np.prod(one_d) == pytest.approx(1.0, rel=1e-12)
            mu += 1
    assert mu == spec.M


def test_basis_gradient_laplacian_finite_difference(orc):
    spec = S.small_open_shell()
    rng = np.random.default_rng(3)
    h = 1e-3
    for _ in range(6):
        r = spec.nuc_xyz[rng.integers(spec.Nn)] + rng.normal(scale=0.8, size=3)
        chi, dchi, lchi = orc.basis_eval(spec, r)
        g_fd = np.zeros_like(dchi)
        lap_fd = np.zeros_like(lchi)
        for d in range(3):
            e = np.zeros(3)
            e[d] = 1

            def f(hh):
                return orc.basis_eval(spec, r + hh * e)[0]
            d1 = (f(h) - f(-h)) / (2 * h)
            d2 = (f(h / 2) - f(-h / 2)) / h
            g_fd[:, d] = (4 * d2 - d1) / 3
            s1 = (f(h) - 2 * chi + f(-h)) / h ** 2
            s2 = (f(h / 2) - 2 * chi + f(-h / 2)) / (h / 2) ** 2
            lap_fd += (4 * s2 - s1) / 3
        scale = np.abs(chi).max() + np.abs(dchi).max()
        np.testing.assert_allclose(dchi, g_fd, rtol=1e-8, atol=1e-9 * scale)
        np.testing.assert_allclose(lchi, lap_fd, rtol=1e-6, atol=1e-6 * scale)


def test_s_gaussian_laplacian_closed_form(orc):
    """lap exp(-z r^2) = (4 z^2 r^2 - 6 z) exp(-z r^2)."""
    spec = S.one_electron(1.0, 0.7)
    for r in [np.array([0.3, 0.1, -0.2]), np.array([1.5, -0.7, 0.9])]:
        chi, dchi, lchi = orc.basis_eval(spec, r)
        r2 = r @ r
        assert lchi[0] == pytest.approx((4 * 0.49 * r2 - 6 * 0.7) * chi[0], rel=1e-13)
        np.testing.assert_allclose(dchi[0], -2 * 0.7 * r * chi[0], rtol=1e-13)


# ----------------------------------------------------------------------------- determinants
def test_det_lu_against_leibniz(orc):
    rng = np.random.default_rng(5)
    for n in (1, 2, 3, 4, 5):
        for _ in range(5):
            A = rng.normal(size=(n, n))
            assert orc.det_lu(A) == pytest.approx(orc.det_leibniz(A), rel=1e-12, abs=1e-14)


def test_det_lu_inverse_product_and_singular(orc):
    rng = np.random.default_rng(6)
    A = rng.normal(size=(8, 8))
    assert orc.det_lu(A) * orc.det_lu(np.linalg.inv(A)) == pytest.approx(1.0, rel=1e-12)
    A[3] = A[1]
    assert abs(orc.det_lu(A)) < 1e-12


# ----------------------------------------------------------------------------- structures
def _fock_apply_create(state, x):
    """a^dag_x on a Fock vector {sorted tuple of spin-orbital labels: coefficient}."""
    out = {}
    for occ, c in state.items():
        if x in occ:
            continue
        nsmall = sum(1 for y in occ if y < x)
        new = tuple(sorted(occ + (x,)))
        out[new] = out.get(new, 0.0) + c * (-1) ** nsmall
    return out


def _fock_apply_annihilate(state, x):
    out = {}
    for occ, c in state.items():
        if x not in occ:
            continue
        pos = occ.index(x)
        new = occ[:pos] + occ[pos + 1:]
        out[new] = out.get(new, 0.0) + c * (-1) ** pos
    return out


def _add(a, b, s=1.0):
    r = dict(a)
    for k, v in b.items():
        r[k] = r.get(k, 0.0) + s * v
    return {k: v for k, v in r.items() if abs(v) > 1e-14}


def _string(ops):
    """Product of creation operators (listed left to right) acting on the vacuum."""
    st = {(): 1.0}
    for x in reversed(ops):
        st = _fock_apply_create(st, x)
    return st


def _lab(orb, spin):
    return 2 * orb + spin


def _structure_fock(inactive, pairs, unpaired):
    """Eq. PhiI built directly in Fock space (the i = j factor 2 divided out)."""
    st = {(): 1.0}
    blocks = []
    for p in inactive:
        blocks.append([(1.0, [_lab(p, 0), _lab(p, 1)])])
    for (i, j) in pairs:
        blocks.append([(1.0, [_lab(i, 0), _lab(j, 1)]), (-1.0, [_lab(i, 1), _lab(j, 0)])])
    for q in unpaired:
        blocks.append([(1.0, [_lab(q, 0)])])
    for b in reversed(blocks):
        new = {}
        for w, ops in b:
            part = st
            for x in reversed(ops):
                part = _fock_apply_create(part, x)
            new = _add(new, part, w)
        st = new
    for (i, j) in pairs:
        if i == j:
            st = {k: v / 2.0 for k, v in st.items()}
    return st


def _S2(state, norb):
    def Splus(s):
        r = {}
        for p in range(norb):
            r = _add(r, _fock_apply_create(_fock_apply_annihilate(s, _lab(p, 1)), _lab(p, 0)))
        return r

    def Sminus(s):
        r = {}
        for p in range(norb):
            r = _add(r, _fock_apply_create(_fock_apply_annihilate(s, _lab(p, 0)), _lab(p, 1)))
        return r

    def Sz(s):
        return {k: v * 0.5 * (sum(1 for x in k if x % 2 == 0) - sum(1 for x in k if x % 2 == 1)) for k, v in s.items()}

    return _add(_add(Sminus(Splus(state)), Sz(Sz(state))), Sz(state))


def _det_terms_fock(terms, I):
    st = {}
    for (s_, d, up, dn) in terms:
        if s_ != I:
            continue
        st = _add(st, _string([_lab(o, 0) for o in up] + [_lab(o, 1) for o in dn]), d)
    return st


@pytest.mark.parametrize("maker", [S.h2_vb, S.small_open_shell, S.ethylene_vb])
def test_structure_expansion_fock_space(orc, maker):
    """The signed determinant list of every structure equals Eq. PhiI built in Fock space,
    N_det,I = 2^(pairs with i != j), all |d| equal, and Phi_I is a spin eigenfunction with
    S = N_unpaired/2 = M_S (brute force for the structures with <= 16 electrons)."""
    spec = maker()
    terms = orc.expand(spec)
    for I in range(spec.Nvb):
        ina = list(spec.inact[spec.inact_off[I]:spec.inact_off[I + 1]])
        prs = [tuple(p) for p in spec.pairs[spec.pair_off[I]:spec.pair_off[I + 1]]]
        unp = list(spec.unp[spec.unp_off[I]:spec.unp_off[I + 1]])
        direct = _structure_fock(ina, prs, unp)
        from_terms = _det_terms_fock(terms, I)
        assert set(direct) == set(from_terms)
        for k in direct:
            assert from_terms[k] == pytest.approx(direct[k], abs=1e-12)
        mine = [t for t in terms if t[0] == I]
        assert len(mine) == 2 ** sum(1 for (i, j) in prs if i != j)
        assert len({abs(t[1]) for t in mine}) == 1
        Sval = 0.5 * len(unp)
        s2 = _S2(direct, spec.Norb)
        for k, v in direct.items():
            assert s2.get(k, 0.0) == pytest.approx(Sval * (Sval + 1) * v, abs=1e-12)


def test_heitler_london_spatially_symmetric(orc):
    """Covalent structure (a, b): Psi(r1 up, r2 down) = phi_a(r1) phi_b(r2) + phi_b(r1) phi_a(r2)."""
    spec = S.h2_vb()
    spec.c_vb = np.array([1.0, 0.0, 0.0])
    spec.jas_a = np.zeros((1, 6))
    spec.jas_b = np.zeros(6)
    spec.b1_anti = spec.b1_par = 0.0
    rng = np.random.default_rng(9)
    R = rng.normal(size=(5, 2, 3))
    out = orc.evaluate(spec, R)
    for w in range(5):
        ph = [spec.orb_coef @ orc.basis_eval(spec, R[w, e])[0] for e in range(2)]
        want = ph[0][0] * ph[1][1] + ph[0][1] * ph[1][0]
        assert out["sign"][w] * math.exp(out["logpsi"][w]) == pytest.approx(want, rel=1e-12)


# ----------------------------------------------------------------------------- wave function invariants
def test_antisymmetry_same_spin_exchange(orc):
    for spec in (S.small_open_shell(), S.ethylene_vb(params=False)):
        R = S.initial_walkers(spec, 3, 21)
        a = orc.evaluate(spec, R)
        for (i, j) in [(0, 1), (spec.n_up, spec.n_up + 1)]:
            R2 = R.copy()
            R2[:, [i, j]] = R2[:, [j, i]]
            b = orc.evaluate(spec, R2)
            np.testing.assert_allclose(b["logpsi"], a["logpsi"], rtol=1e-12)
            np.testing.assert_array_equal(b["sign"], -a["sign"])
            np.testing.assert_allclose(b["eloc"], a["eloc"], rtol=1e-9)


@pytest.mark.parametrize("Z", list(range(1, 10)))
def test_hydrogen_like_exact(orc, Z):
    """Psi = exp(-Z r) (constant orbital, a1 = -Z, a2 = -kappa): E_L = -Z^2/2 everywhere."""
    spec = S.one_electron(Z, 0.0, a1=-Z, a2=-0.8)
    R = np.random.default_rng(Z).normal(scale=2.0 / Z, size=(20, 1, 3))
    out = orc.evaluate(spec, R, grad=True)
    np.testing.assert_allclose(out["eloc"], -0.5 * Z * Z, rtol=1e-12)
    r = np.linalg.norm(R[:, 0], axis=1)
    np.testing.assert_allclose(out["logpsi"], -Z * r, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(out["grad"][:, 0], -Z * R[:, 0] / r[:, None], rtol=1e-11)


def test_gaussian_hydrogen_pointwise(orc):
    """Psi = exp(-z r^2), no Jastrow: E_L = 3z - 2 z^2 r^2 - Z/r."""
    for Z, z in [(1.0, 0.28), (2.0, 1.1)]:
        spec = S.one_electron(Z, z)
        R = np.random.default_rng(1).normal(size=(10, 1, 3))
        r = np.linalg.norm(R[:, 0], axis=1)
        out = orc.evaluate(spec, R)
        np.testing.assert_allclose(out["eloc"], 3 * z - 2 * z * z * r * r - Z / r, rtol=1e-12)


def test_two_electron_product_pointwise(orc):
    """Two electrons in one s Gaussian, no Jastrow:
    E_L = sum_i (3z - 2 z^2 r_i^2 - Z/r_i) + 1/r12."""
    Z, z = 2.0, 0.9
    spec = S.two_electron_product(Z, z)
    R = np.random.default_rng(2).normal(size=(10, 2, 3))
    r = np.linalg.norm(R, axis=2)
    r12 = np.linalg.norm(R[:, 0] - R[:, 1], axis=1)
    want = (3 * z - 2 * z * z * r ** 2 - Z / r).sum(1) + 1 / r12
    np.testing.assert_allclose(orc.evaluate(spec, R)["eloc"], want, rtol=1e-12)


def test_vmc_gaussian_means(orc):
    """VMC averages of E_L: one electron 3z/2 - 2Z sqrt(2z/pi); two electrons
    3z - 4Z sqrt(2z/pi) + 2 sqrt(z/pi) (within 4 sigma by reblocking)."""
    cases = [(S.one_electron(1.0, 8 / (9 * math.pi)), 1.0, 8 / (9 * math.pi), 1),
             (S.two_electron_product(2.0, 1.2), 2.0, 1.2, 2)]
    for spec, Z, z, ne in cases:
        R = S.initial_walkers(spec, 256, 5, sigma=0.7)
        R, _, _, _ = orc.vmc(spec, R, 40, 0.8, seed=77, eloc=False)
        _, hist, _, nacc = orc.vmc(spec, R, 60, 0.8, seed=77, step0=1000)
        if ne == 1:
            exact = 1.5 * z - 2 * Z * math.sqrt(2 * z / math.pi)
        else:
            exact = 3 * z - 4 * Z * math.sqrt(2 * z / math.pi) + 2 * math.sqrt(z / math.pi)
        m, e = orc.reblock(hist.mean(axis=1))
        assert abs(m - exact) < 4 * e + 1e-3, (m, e, exact)
    # z = 8/(9 pi) gives -4/(3 pi) for Z = 1
    assert 1.5 * (8 / (9 * math.pi)) - 2 * math.sqrt(2 * 8 / (9 * math.pi) / math.pi) == pytest.approx(-4 / (3 * math.pi))


# ----------------------------------------------------------------------------- Jastrow
def test_een_term_count_and_cusp_rank(orc):
    """23 e-e-n terms (2, 4, 7, 10 for p = 2..5); 15 free coefficients after the cusp conditions."""
    t = orc.een_terms()
    assert len(t) == 23
    assert [int(np.sum(t[:, 0] == p)) for p in (2, 3, 4, 5)] == [2, 4, 7, 10]
    assert np.all((t[:, 0] - t[:, 1] - t[:, 2]) == 2 * t[:, 3])
    B = orc.een_basis()
    assert B.shape == (23, 15)
    assert np.linalg.matrix_rank(B) == 15


def _jastrow_only(spec):
    spec.orb_coef = np.ones((spec.Norb, spec.M)) * 0.0
    return spec


def test_jastrow_special_values(orc):
    """ln J at hand-picked configurations: (i) Pade e-e with b1 = 1/2, b2 = 1 at distance r is
    (1/2) R/(1 + R), R = r/(1 + 0.8 r); (ii) both electrons on the nucleus: every e-e-n term is
    2 c (u = s = t = 1), so f_een = 2 sum c; (iii) f_een is symmetric in the two electrons."""
    spec = S.small_open_shell()
    spec.jas_a = np.zeros_like(spec.jas_a)
    spec.jas_b = np.zeros(6)
    spec.b1_anti = spec.b1_par = 0.0
    spec.een_on = False
    # (i) two electrons only matter through f_ee: use the two-electron system
    sp2 = S.two_electron_product(1.0, 0.5)
    sp2.b1_anti, sp2.jas_b = 0.5, np.array([0, 1.0, 0, 0, 0, 0])
    for r in (0.3, 1.7):
        R = np.array([[[0, 0, 0], [0, 0, r]]], np.float64)
        Rs = r / (1 + 0.8 * r)
        assert orc.lnJ(sp2, R)[0] == pytest.approx(0.5 * Rs / (1 + Rs), rel=1e-14)
    # (ii) single nucleus, two electrons at the nucleus -> only e-e-n with u = s = t = 1
    sp3 = S.two_electron_product(1.0, 0.5)
    sp3.een_on = True
    theta = np.random.default_rng(3).uniform(-1, 1, (1, 15))
    sp3.een_theta = theta
    B = orc.een_basis()
    c = B @ theta[0]
    R = np.zeros((1, 2, 3))
    assert orc.lnJ(sp3, R)[0] == pytest.approx(2 * c.sum(), rel=1e-12, abs=1e-14)
    # (iii) symmetry under exchanging the two electrons of opposite spin
    R = np.array([[[0.2, -0.1, 0.4], [-0.7, 0.5, 0.1]]])
    assert orc.lnJ(sp3, R)[0] == pytest.approx(orc.lnJ(sp3, R[:, ::-1].copy())[0], rel=1e-13)


def _cusp_series(orc, spec, R0, i, target, direction):
    """E_L as electron i approaches 'target' (a point) along 'direction'."""
    vals = []
    for k in range(2, 7):
        eps = 10.0 ** (-k)
        R = R0.copy()
        R[0, i] = target + eps * direction
        vals.append(orc.evaluate(spec, R)["eloc"][0])
    return np.array(vals)


def test_cusps_bounded(orc):
    """E_L stays bounded as r_ij -> 0 (antiparallel with b1 = 1/2, parallel with b1 = 1/4) and as
    r_ia -> 0 (a1 = -Z), with the cusp-constrained e-e-n term switched on; the successive
    differences shrink linearly with the distance.  Breaking a constraint makes it diverge."""
    spec = S.small_open_shell()
    spec.een_theta = 4.0 * spec.een_theta  # make the e-e-n term matter
    R0 = S.initial_walkers(spec, 1, 4)
    d = np.array([0.6, -0.48, 0.64])
    for (i, j) in [(0, spec.n_up), (0, 1)]:
        v = _cusp_series(orc, spec, R0, i, R0[0, j], d)
        diffs = np.abs(np.diff(v))
        assert diffs[-1] < 1e-3 and diffs[-1] < 0.2 * diffs[0] + 1e-9, v
    v = _cusp_series(orc, spec, R0, 1, spec.nuc_xyz[0], d)
    diffs = np.abs(np.diff(v))
    assert diffs[-1] < 1e-3, v
    # a raw e-e-n coefficient that violates the e-e condition makes E_L diverge like 1/r_ij;
    # probe: put theta so that c = B theta + delta where delta breaks it -> emulate by a2 term
    bad = S.small_open_shell()
    bad.b1_anti = 0.3  # wrong antiparallel cusp
    v = _cusp_series(orc, bad, R0, 0, R0[0, bad.n_up], d)
    assert abs(v[-1] - v[-2]) > 100.0


# ----------------------------------------------------------------------------- parameter derivatives
def _perturb(spec, j, h):
    """Copy of spec with parameter j moved by h (same ordering as the oracle: c, a2..a6 per
    element, b2..b6, theta per element, orbital excitations)."""
    import copy
    s = copy.deepcopy(s0 := spec)
    s.c_vb = s0.c_vb.copy(); s.jas_a = s0.jas_a.copy(); s.jas_b = s0.jas_b.copy()
    s.een_theta = s0.theta().copy(); s.orb_coef = s0.orb_coef.copy()
    if j < len(s.cparam):
        s.c_vb[s.cparam[j]] += h
        return s
    j -= len(s.cparam)
    if s.jas_param:
        if j < 5 * s.n_elem:
            s.jas_a[j // 5, 1 + j % 5] += h
            return s
        j -= 5 * s.n_elem
        if j < 5:
            s.jas_b[1 + j] += h
            return s
        j -= 5
        if s.een_on:
            if j < 15 * s.n_elem:
                s.een_theta[j // 15, j % 15] += h
                return s
            j -= 15 * s.n_elem
    k, l = s.kappa_kl[j]
    s.orb_coef[l] += h * s0.orb_coef[k]
    return s


def _fd_params(orc, spec, R, js, h=1e-3):
    outO, outE = [], []
    for j in js:
        def f(hh):
            o = orc.evaluate(_perturb(spec, j, hh), R)
            return o["logpsi"], o["eloc"]
        a1, b1 = f(h); a2, b2 = f(-h); a3, b3 = f(h / 2); a4, b4 = f(-h / 2)
        outO.append((4 * (a3 - a4) / h - (a1 - a2) / (2 * h)) / 3)
        outE.append((4 * (b3 - b4) / h - (b1 - b2) / (2 * h)) / 3)
    return np.array(outO).T, np.array(outE).T


def test_parameter_derivatives_finite_difference(orc):
    spec = S.small_open_shell()
    R = S.initial_walkers(spec, 3, 8)
    out = orc.evaluate(spec, R, derivs=True)
    P = out["O"].shape[1]
    assert P == spec.n_params
    O_fd, E_fd = _fd_params(orc, spec, R, range(P))
    scaleE = 1.0 + np.abs(out["eloc"])[:, None]
    np.testing.assert_allclose(out["O"], O_fd, rtol=1e-7, atol=1e-8)
    np.testing.assert_allclose(out["dEL"], E_fd, rtol=1e-6, atol=1e-7 * scaleE.max())


def test_parameter_derivatives_finite_difference_ethylene_subset(orc):
    spec = S.ethylene_vb()
    R = S.initial_walkers(spec, 1, 3)
    out = orc.evaluate(spec, R, derivs=True)
    js = list(range(0, spec.n_params, 23)) + [4, 5, 20, 49, 50, spec.n_params - 1]
    O_fd, E_fd = _fd_params(orc, spec, R, js)
    np.testing.assert_allclose(out["O"][:, js], O_fd, rtol=1e-6, atol=1e-8)
    np.testing.assert_allclose(out["dEL"][:, js], E_fd, rtol=1e-5, atol=1e-6 * (1 + abs(out["eloc"][0])))


def test_structure_coefficient_sum_rule(orc):
    """sum_I c_I (Phi_I/Phi) = 1 per walker when every c_I is a parameter."""
    spec = S.small_open_shell(params=False)
    spec.cparam = np.arange(spec.Nvb, dtype=np.int32)
    R = S.initial_walkers(spec, 4, 2)
    O = orc.evaluate(spec, R, derivs=True)["O"]
    np.testing.assert_allclose(O @ spec.c_vb, 1.0, rtol=1e-13)


# ----------------------------------------------------------------------------- nucleus-position derivatives
def _moved(spec, q, h):
    """Copy of spec with nucleus coordinate q = 3 alpha + d moved by h (its shells move with it)."""
    import copy
    s = copy.deepcopy(spec)
    s.nuc_xyz = spec.nuc_xyz.copy()
    s.nuc_xyz[q // 3, q % 3] += h
    return s


def _fd_nuclei(orc, spec, R, qs, h=1e-3):
    outL, outE = [], []
    for q in qs:
        def f(hh):
            o = orc.evaluate(_moved(spec, q, hh), R)
            return o["logpsi"], o["eloc"]
        a1, b1 = f(h); a2, b2 = f(-h); a3, b3 = f(h / 2); a4, b4 = f(-h / 2)
        outL.append((4 * (a3 - a4) / h - (a1 - a2) / (2 * h)) / 3)
        outE.append((4 * (b3 - b4) / h - (b1 - b2) / (2 * h)) / 3)
    return np.array(outL).T, np.array(outE).T


def test_nuclear_derivatives_finite_difference(orc):
    """d ln|Psi|/dR_alpha and dE_L/dR_alpha against Richardson central differences of the
    oracle moved to displaced nuclei (basis centres, e-n and e-e-n Jastrow and V all move)."""
    spec = S.small_open_shell()
    R = S.initial_walkers(spec, 3, 8)
    out = orc.nuclear_derivs(spec, R)
    L_fd, E_fd = _fd_nuclei(orc, spec, R, range(3 * spec.Nn))
    W = R.shape[0]
    np.testing.assert_allclose(out["dlogpsi"].reshape(W, -1), L_fd, rtol=1e-7, atol=1e-8)
    scale = 1.0 + np.abs(E_fd).max()
    np.testing.assert_allclose(out["dEL"].reshape(W, -1), E_fd, rtol=1e-6, atol=1e-7 * scale)


def test_nuclear_derivatives_finite_difference_ethylene_subset(orc):
    spec = S.ethylene_vb()
    R = S.initial_walkers(spec, 1, 3)
    out = orc.nuclear_derivs(spec, R)
    qs = [0, 4, 8, 10, 17]
    L_fd, E_fd = _fd_nuclei(orc, spec, R, qs)
    np.testing.assert_allclose(out["dlogpsi"].reshape(1, -1)[:, qs], L_fd, rtol=1e-6, atol=1e-8)
    np.testing.assert_allclose(out["dEL"].reshape(1, -1)[:, qs], E_fd, rtol=1e-5,
                               atol=1e-6 * (1 + np.abs(E_fd).max()))


@pytest.mark.parametrize("Z", [1, 3, 6])
def test_nuclear_derivatives_hydrogen_like(orc, Z):
    """Psi = exp(-Z |r - R_a|): d ln Psi/dR_a = Z (r - R_a)/|r - R_a| and E_L = -Z^2/2 wherever
    the nucleus sits, so dE_L/dR_a = 0."""
    spec = S.one_electron(Z, 0.0, a1=-Z, a2=-0.8)
    spec.nuc_xyz = np.array([[0.3, -0.2, 0.5]])
    R = spec.nuc_xyz[None] + np.random.default_rng(Z).normal(scale=2.0 / Z, size=(12, 1, 3))
    out = orc.nuclear_derivs(spec, R)
    d = R[:, 0] - spec.nuc_xyz[0]
    np.testing.assert_allclose(out["dlogpsi"][:, 0], Z * d / np.linalg.norm(d, axis=1)[:, None], rtol=1e-12)
    assert np.abs(out["dEL"]).max() <= 1e-11 * Z * Z


def test_nuclear_derivatives_coulomb(orc):
    """A wave function that does not depend on the nuclei (constant orbital, no Jastrow):
    d ln Psi/dR = 0 and dE_L/dR_a = dV/dR_a, Coulomb's law for the electrons and the other
    nuclei: -Z_a sum_i (r_i - R_a)/|r_i - R_a|^3 - Z_a sum_b Z_b (R_a - R_b)/|R_a - R_b|^3."""
    spec = S.two_electron_product(2.0, 0.0)
    spec.nuc_xyz = np.array([[0.0, 0.0, 0.0], [1.3, -0.4, 0.2], [-0.7, 0.9, 1.1]])
    spec.nuc_Z = np.array([2.0, 1.0, 3.0])
    spec.nuc_elem = np.zeros(3, np.int32)
    R = np.random.default_rng(4).normal(scale=1.5, size=(6, 2, 3))
    out = orc.nuclear_derivs(spec, R)
    assert np.abs(out["dlogpsi"]).max() == 0.0
    X, Zs = spec.nuc_xyz, spec.nuc_Z
    want = np.zeros((6, 3, 3))
    for a in range(3):
        for i in range(2):
            d = R[:, i] - X[a]
            want[:, a] -= Zs[a] * d / (np.linalg.norm(d, axis=1) ** 3)[:, None]
        for b in range(3):
            if b != a:
                d = X[a] - X[b]
                want[:, a] -= Zs[a] * Zs[b] * d / np.linalg.norm(d) ** 3
    np.testing.assert_allclose(out["dEL"], want, rtol=1e-12, atol=1e-12)


def test_nuclear_derivatives_translation_sum(orc):
    """Moving every nucleus and every electron together changes nothing, so
    sum_a d/dR_a = -sum_i d/dr_i: against the electron gradient of ln|Psi|, and against a
    Richardson difference of E_L under a common shift of the electrons."""
    spec = S.small_open_shell()
    R = S.initial_walkers(spec, 3, 5)
    out = orc.nuclear_derivs(spec, R)
    g = orc.evaluate(spec, R, grad=True)["grad"]
    np.testing.assert_allclose(out["dlogpsi"].sum(1), -g.sum(1), rtol=1e-10, atol=1e-10)
    h = 1e-3
    for d in range(3):
        def el(hh):
            Rs = R.copy()
            Rs[:, :, d] += hh
            return orc.evaluate(spec, Rs)["eloc"]
        fd = (4 * (el(h / 2) - el(-h / 2)) / h - (el(h) - el(-h)) / (2 * h)) / 3
        np.testing.assert_allclose(out["dEL"][:, :, d].sum(1), -fd, rtol=1e-6, atol=1e-6 * (1 + np.abs(fd).max()))


# ----------------------------------------------------------------------------- linear method
def test_linear_method_strong_zero_variance(orc):
    """Psi = J (Phi_1 + c2 Phi_2) with J = exp(-Z r): the exact state exp(-Z r) = Psi - c2 Psi_c2 is
    in the span of Psi and dPsi/dc2, so the nonsymmetric estimators give E_lin = -Z^2/2 and the
    exact state from any small sample (Sec. 2.3.1, strong zero-variance principle).  With the
    semi-orthogonal derivative (Eq. semiorthog, sample mean <O>), Psi_lin/Psi = 1 + dp (O - <O>)
    is proportional to 1 - c2 O exactly when dp / (1 - dp <O>) = -c2."""
    for Z, c2 in [(1.0, 0.7), (3.0, -0.4)]:
        spec = S.two_structure_1s(Z, 0.9, c2)
        for W, seed in [(2, 1), (5, 2), (40, 3)]:
            R = np.random.default_rng(seed).normal(scale=1.0 / Z, size=(W, 1, 3))
            ev = orc.evaluate(spec, R, derivs=True)
            m = orc.lin_matrices(ev["O"], ev["dEL"], ev["eloc"])
            dp, E = orc.lin_solve(m["E0"], m["gL"], m["gR"], m["H"], m["S"])
            obar = ev["O"][:, 0].mean()
            assert dp[0] / (1.0 - dp[0] * obar) == pytest.approx(-c2, rel=1e-9, abs=1e-10)
            assert E == pytest.approx(-0.5 * Z * Z, rel=1e-10)


def test_linear_method_centered_identity(orc):
    """Eq. Hij equals <dO_i dO_j E_L> + <dO_i E_L,j> with dO = O - <O>; S_ij = <dO_i dO_j>."""
    rng = np.random.default_rng(4)
    O, dE, E = rng.normal(size=(50, 4)), rng.normal(size=(50, 4)), rng.normal(size=50)
    w = rng.uniform(0.5, 1.5, 50)
    m = orc.lin_matrices(O, dE, E, w)
    Oc = O - (w @ O) / w.sum()
    Hc = np.einsum("m,mi,mj->ij", w * E, Oc, Oc) / w.sum() + np.einsum("m,mi,mj->ij", w, Oc, dE) / w.sum()
    np.testing.assert_allclose(m["H"], Hc, atol=1e-12)
    np.testing.assert_allclose(m["S"], np.einsum("m,mi,mj->ij", w, Oc, Oc) / w.sum(), atol=1e-12)


# ----------------------------------------------------------------------------- DMC
def test_dmc_exact_trial_constant_weights(orc):
    """With Psi = exp(-Z r) and E_T = -Z^2/2 every weight is exactly 1, the population never
    changes and the mixed estimator is -Z^2/2 (Sec. 2.3.2, Eq. E0DMCweights)."""
    Z = 2.0
    spec = S.one_electron(Z, 0.0, a1=-Z, a2=-0.8)
    R = np.random.default_rng(1).normal(scale=0.6, size=(64, 1, 3))
    out = orc.dmc(spec, R, 30, 0.01, -0.5 * Z * Z, 64, seed=5)
    assert np.all(out["pop"] == 64)
    np.testing.assert_allclose(out["sum_w"], 64.0, rtol=1e-13)
    np.testing.assert_allclose(out["sum_wE"] / out["sum_w"], -0.5 * Z * Z, rtol=1e-13)


def test_dmc_hydrogen_ground_state(orc):
    """Nodeless non-exact trial for H: the DMC mixed estimate approaches -1/2 (within 4 sigma +
    a 2 mHa time-step allowance), and lies below the VMC energy of the same trial."""
    spec = S.one_electron(1.0, 0.3, a1=-1.0, a2=1.0)
    R = np.random.default_rng(2).normal(scale=1.0, size=(400, 1, 3))
    R, _, _, _ = orc.vmc(spec, R, 50, 1.0, seed=3, eloc=False)
    _, hist, _, _ = orc.vmc(spec, R, 50, 1.0, seed=3, step0=500)
    e_vmc = hist.mean()
    out = orc.dmc(spec, R, 600, 0.01, e_vmc, 400, seed=9)
    Eb = out["sum_wE"][100:] / out["sum_w"][100:]
    m, e = orc.reblock(Eb)
    assert abs(m + 0.5) < 4 * e + 2e-3, (m, e)
    assert m < e_vmc


def test_dmc_h2_nodeless(orc):
    """H2 at R = 1.4 bohr with a nodeless trial: DMC gives the exact Born-Oppenheimer energy
    -1.17447 Ha within 4 sigma + a 3 mHa time-step allowance; VMC lies above it."""
    spec = S.h2_nodeless()
    R = S.initial_walkers(spec, 400, 6, sigma=0.8)
    R, _, _, _ = orc.vmc(spec, R, 60, 0.6, seed=1, eloc=False)
    _, hist, _, _ = orc.vmc(spec, R, 40, 0.6, seed=1, step0=900)
    e_vmc, e_vmc_err = orc.reblock(hist.mean(axis=1))
    assert e_vmc > -1.17447 - 4 * e_vmc_err
    out = orc.dmc(spec, R, 1500, 0.01, e_vmc, 400, seed=13)
    Eb = out["sum_wE"][200:] / out["sum_w"][200:]
    m, e = orc.reblock(Eb)
    assert e < 3e-3
    assert abs(m + 1.17447) < 4 * e + 3e-3, (m, e, e_vmc)


def _ar1(rng, N, rho):
    """Stationary AR(1) series x_t = rho x_{t-1} + sqrt(1 - rho^2) e_t, unit variance."""
    from scipy.signal import lfilter
    e = rng.normal(size=N)
    return lfilter([np.sqrt(1.0 - rho * rho)], [1.0, -rho], e, zi=[rho * rng.normal()])[0]


def test_reblock_short_series_is_the_textbook_standard_error(orc):
    """Below 32 samples no blocking level is formed: the error is s / sqrt(n) with the sample
    standard deviation s (n - 1 in the denominator).  x = 1, 2, 3, 4: s^2 = 5/3, error
    sqrt(5/3) / 2."""
    m, e = orc.reblock([1.0, 2.0, 3.0, 4.0])
    assert m == 2.5
    assert e == pytest.approx(np.sqrt(5.0 / 3.0) / 2.0, rel=1e-15)


@pytest.mark.parametrize("rho", [0.0, 0.9, 0.98])
def test_reblock_recovers_the_ar1_error_of_the_mean(orc, rho):
    """For an AR(1) series the variance of the mean is known in closed form,
    Var = (1 + 2 sum_{k=1}^{N-1} (1 - k/N) rho^k) / N (integrated autocorrelation time
    (1 + rho)/(1 - rho) for large N).  Over 20 independent series the reblocked error must track
    it: a level-0 estimate would be sqrt((1 - rho)/(1 + rho)) too small (0.23 at rho = 0.9)."""
    N = 1 << 18
    k = np.arange(1, N)
    sd = np.sqrt((1.0 + 2.0 * np.sum((1.0 - k / N) * rho ** k)) / N)
    ratios = []
    for seed in range(20):
        x = _ar1(np.random.default_rng(seed), N, rho)
        m, e = orc.reblock(x)
        assert m == pytest.approx(x.mean(), rel=0, abs=1e-15)
        ratios.append(e / sd)
    ratios = np.array(ratios)
    assert 0.95 < ratios.mean() < 1.25, ratios.mean()
    assert ratios.min() > 0.8 and ratios.max() < 1.6, (ratios.min(), ratios.max())


def test_dmc_limits_bound_the_weights_at_a_node(orc):
    """Trial orbital (1 + c' z) exp(-zeta r^2) (an s and a p Gaussian shell on one nucleus with
    normalised coefficients 1 and c = 2, so c' = c sqrt(4 zeta)) with the e-n cusp in the Jastrow:
    its node is the plane z0 = -1 / c', where lap Psi != 0, so v = grad ln|Psi| and E_L grow
    like 1 / |z - z0|.  Walkers placed 1e-7 from the node would carry weights exp(-tau (E_L - E_T))
    of order exp(1e5) without limits.  With the drift and energy limits of the step (Umrigar,
    Nightingale and Runge 1993) the branching energy E_T + (E_L - E_T)|Vbar|/|V| stays bounded
    (tau |Vbar| <= sqrt(2 tau) per electron): every weight stays within exp(+-0.5) here, so the
    weight sum stays within a factor two of the population."""
    import dataclasses
    zeta, c = 0.5, 2.0
    base = S.one_electron(1.0, zeta, a1=-1.0, a2=1.0)
    spec = dataclasses.replace(base, sh_center=np.zeros(2, np.int32), sh_l=np.array([0, 1], np.int32),
                               sh_zeta=np.array([zeta, zeta]), orb_coef=np.array([[1.0, 0.0, 0.0, c]]))
    z0 = -1.0 / (c * np.sqrt(4.0 * zeta))
    rng = np.random.default_rng(4)
    W = 64
    R = np.zeros((W, 1, 3))
    R[:, 0, 0] = rng.uniform(-1.0, 1.0, W)
    R[:, 0, 1] = rng.uniform(-1.0, 1.0, W)
    R[:, 0, 2] = z0 + np.where(rng.uniform(size=W) < 0.5, -1e-7, 1e-7)
    ev = orc.evaluate(spec, R)
    assert np.abs(ev["eloc"]).min() > 1e5  # E_L ~ 1 / |z - z0| at the node
    out = orc.dmc(spec, R, 1, 0.01, -0.3, W, seed=3, cap=4 * W)
    assert 0.5 * W < out["sum_w"][0] < 2.0 * W, out["sum_w"][0]
    assert out["pop"][0] <= 2 * W


def test_dmc_energy_cutoff_bounds_every_weight(orc):
    """Far from any node a walker can still have a huge |E_L| (here: E_T set 1e4 Ha away from the
    exact energy of the 1s trial, every walker's E_L - E_T = -1e4).  The cutoff
    |E_b - E_T| <= 0.2 sqrt(N / tau) (Zen et al. 2016) bounds each weight to
    exp(tau 0.2 sqrt(N / tau)): with N = 1, tau = 0.01 that is exp(0.02) per walker, so the
    weight sum is exactly W exp(0.02) (without the cutoff it would be W exp(100))."""
    Z = 2.0
    spec = S.one_electron(Z, 0.0, a1=-Z, a2=-0.8)
    W, tau = 32, 0.01
    R = np.random.default_rng(3).normal(scale=0.6, size=(W, 1, 3))
    out = orc.dmc(spec, R, 1, tau, -0.5 * Z * Z + 1e4, W, seed=2, cap=8 * W)
    np.testing.assert_allclose(out["sum_w"][0], W * np.exp(tau * 0.2 * np.sqrt(1.0 / tau)), rtol=1e-12)


# ----------------------------------------------------------------------------- Slater shells
@pytest.mark.parametrize("Z", list(range(1, 10)))
def test_slater_1s_exact_without_jastrow(orc, Z):
    """A 1s Slater orbital exp(-Z r) carries the exact nuclear cusp itself (the paper's a1 = 0,
    Sec. 2.1): E_L = -Z^2/2 at every point, no Jastrow factor."""
    spec = S.slater_1s(float(Z), float(Z))
    R = np.random.default_rng(Z).normal(scale=1.0 / Z, size=(20, 1, 3))
    out = orc.evaluate(spec, R)
    np.testing.assert_allclose(out["eloc"], -0.5 * Z * Z, rtol=1e-12)


def test_slater_normalisation_quadrature():
    """Every Slater component N x^a y^b z^c exp(-zeta r) of the library's normalisation integrates
    to 1: Gauss-Laguerre in r times Gauss-Legendre in cos(theta) and the trapezoid rule in phi
    (exact for these polynomial-times-exponential integrands)."""
    from oracle import oracle as orc
    spec = S.slater_h2()
    xr, wr = np.polynomial.laguerre.laggauss(40)
    xc, wc = np.polynomial.legendre.leggauss(12)
    nphi = 16
    phi = 2 * np.pi * np.arange(nphi) / nphi
    mu = 0
    for sh in range(2 * 4):
        c, l, zt = spec.sh_center[sh], int(spec.sh_l[sh]), spec.sh_zeta[sh]
        for (a, b, cc) in _basis_exponents(l):
            r0 = spec.nuc_xyz[c] + np.array([0.31, -0.22, 0.17])
            chi, _, _ = orc.basis_eval(spec, r0)
            d = r0 - spec.nuc_xyz[c]
            N = chi[mu] / (d[0] ** a * d[1] ** b * d[2] ** cc * math.exp(-zt * np.linalg.norm(d)))
            # int r^(2l+2) e^{-2 zt r} dr with r = x / (2 zt), and the angular integral of the monomial
            rad = np.sum(wr * (xr / (2 * zt)) ** (2 * l + 2)) / (2 * zt)
            st = np.sqrt(1 - xc ** 2)
            ang = 0.0
            for p in phi:
                ux, uy, uz = st * np.cos(p), st * np.sin(p), xc
                ang += np.sum(wc * ux ** (2 * a) * uy ** (2 * b) * uz ** (2 * cc)) * (2 * np.pi / nphi)
            assert N * N * rad * ang == pytest.approx(1.0, rel=1e-12)
            mu += 1


def test_slater_gradient_laplacian_finite_difference(orc):
    spec = S.slater_h2()
    rng = np.random.default_rng(13)
    h = 1e-3
    for _ in range(6):
        r = spec.nuc_xyz[rng.integers(spec.Nn)] + rng.normal(scale=0.8, size=3)
        chi, dchi, lchi = orc.basis_eval(spec, r)
        g_fd = np.zeros_like(dchi)
        lap_fd = np.zeros_like(lchi)
        for d in range(3):
            e = np.zeros(3)
            e[d] = 1

            def f(hh):
                return orc.basis_eval(spec, r + hh * e)[0]
            d1 = (f(h) - f(-h)) / (2 * h)
            d2 = (f(h / 2) - f(-h / 2)) / h
            g_fd[:, d] = (4 * d2 - d1) / 3
            s1 = (f(h) - 2 * chi + f(-h)) / h ** 2
            s2 = (f(h / 2) - 2 * chi + f(-h / 2)) / (h / 2) ** 2
            lap_fd += (4 * s2 - s1) / 3
        scale = np.abs(chi).max() + np.abs(dchi).max()
        np.testing.assert_allclose(dchi, g_fd, rtol=1e-8, atol=1e-9 * scale)
        np.testing.assert_allclose(lchi, lap_fd, rtol=1e-6, atol=1e-6 * scale)


@pytest.mark.parametrize("Z, zeta", [(2.0, 2.0), (2.0, 1.6875), (3.0, 2.4)])
def test_slater_two_electron_closed_form(orc, Z, zeta):
    """He-like singlet in one 1s Slater orbital, no Jastrow: Psi = exp(-zeta (r1 + r2)) and
    E_L = -zeta^2 + (zeta - Z)(1/r1 + 1/r2) + 1/r12 pointwise; with zeta = Z the nuclear cusp is
    exact and E_L stays bounded as an electron reaches the nucleus."""
    spec = S.slater_1s(Z, zeta)
    spec.n_dn = 1
    spec.inact_off, spec.inact = np.array([0, 1], np.int32), np.array([0], np.int32)
    spec.unp_off, spec.unp = np.array([0, 0], np.int32), np.zeros(0, np.int32)
    R = np.random.default_rng(int(10 * zeta)).normal(scale=0.8, size=(12, 2, 3))
    out = orc.evaluate(spec, R)
    r1, r2 = np.linalg.norm(R[:, 0], axis=1), np.linalg.norm(R[:, 1], axis=1)
    r12 = np.linalg.norm(R[:, 0] - R[:, 1], axis=1)
    ref = -zeta ** 2 + (zeta - Z) * (1 / r1 + 1 / r2) + 1 / r12
    np.testing.assert_allclose(out["eloc"], ref, rtol=1e-12)
    v = _cusp_series(orc, spec, R[:1], 0, np.zeros(3), np.array([0.6, -0.48, 0.64]))
    if zeta == Z:
        assert np.abs(np.diff(v))[-1] < 1e-3, v
    else:
        assert abs(v[-1] - v[-2]) > 100.0 * abs(zeta - Z), v


def test_slater_parameter_and_nuclear_derivatives_finite_difference(orc):
    spec = S.slater_h2()
    R = S.initial_walkers(spec, 3, 8)
    out = orc.evaluate(spec, R, derivs=True)
    P = out["O"].shape[1]
    O_fd, E_fd = _fd_params(orc, spec, R, range(P))
    np.testing.assert_allclose(out["O"], O_fd, rtol=1e-7, atol=1e-8)
    np.testing.assert_allclose(out["dEL"], E_fd, rtol=1e-6, atol=1e-7 * (1.0 + np.abs(out["eloc"]).max()))
    nd = orc.nuclear_derivs(spec, R)
    L_fd, EN_fd = _fd_nuclei(orc, spec, R, range(3 * spec.Nn))
    np.testing.assert_allclose(nd["dlogpsi"].reshape(3, -1), L_fd, rtol=1e-7, atol=1e-8)
    np.testing.assert_allclose(nd["dEL"].reshape(3, -1), EN_fd, rtol=1e-6, atol=1e-7 * (1.0 + np.abs(EN_fd).max()))


# ----------------------------------------------------------------------------- BOVB
def _bovb_groups(spec):
    """For every VBSCF excitation j, the indices of the BOVB excitations made from it (one per
    structure that uses its orbital l), in the order systems.bovb emits them."""
    groups, q = [], 0
    for k, l in spec.kappa_kl:
        n = 0
        for I in range(spec.Nvb):
            used = set(spec.inact[spec.inact_off[I]:spec.inact_off[I + 1]]) | set(
                spec.pairs[spec.pair_off[I]:spec.pair_off[I + 1]].ravel()) | set(spec.unp[spec.unp_off[I]:spec.unp_off[I + 1]])
            n += int(l) in used
        groups.append(list(range(q, q + n)))
        q += n
    return groups


@pytest.mark.parametrize("maker", [S.small_open_shell, S.h2_vb])
def test_bovb_with_identical_orbitals_reduces_to_vbscf(orc, maker):
    """BOVB (Sec. 2.2) whose per-structure orbitals are exact copies of the shared ones is the
    VBSCF wave function: same ln|Psi|, sign, E_L, structure-coefficient and Jastrow derivatives;
    and a shared orbital's excitation acts in every structure, so its derivative is the sum of
    the per-structure excitations' derivatives (first-order variations add)."""
    spec = maker()
    if len(spec.kappa_kl) == 0:
        spec.kappa_kl = np.array([[1, 0], [0, 1]], np.int32)
    bo = S.bovb(spec, eps=0.0)
    R = S.initial_walkers(spec, 5, 13)
    a, b = orc.evaluate(spec, R, derivs=True), orc.evaluate(bo, R, derivs=True)
    np.testing.assert_allclose(b["logpsi"], a["logpsi"], rtol=1e-13, atol=1e-13)
    np.testing.assert_array_equal(b["sign"], a["sign"])
    np.testing.assert_allclose(b["eloc"], a["eloc"], rtol=1e-12, atol=1e-12)
    nk = len(spec.kappa_kl)
    n0 = spec.n_params - nk
    np.testing.assert_allclose(b["O"][:, :n0], a["O"][:, :n0], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(b["dEL"][:, :n0], a["dEL"][:, :n0], rtol=1e-10, atol=1e-10)
    for j, grp in enumerate(_bovb_groups(spec)):
        cols = [n0 + q for q in grp]
        np.testing.assert_allclose(b["O"][:, cols].sum(1), a["O"][:, n0 + j], rtol=1e-11, atol=1e-11)
        np.testing.assert_allclose(b["dEL"][:, cols].sum(1), a["dEL"][:, n0 + j], rtol=1e-9, atol=1e-9)


def test_bovb_derivatives_finite_difference(orc):
    """Breathing orbitals (eps = 0.1): the per-structure excitation derivatives against
    Richardson differences of the oracle (a subset of the parameters)."""
    bo = S.bovb(S.small_open_shell(), eps=0.1)
    R = S.initial_walkers(bo, 3, 6)
    out = orc.evaluate(bo, R, derivs=True)
    P = bo.n_params
    js = list(range(0, 4)) + list(range(P - 12, P))
    O_fd, E_fd = _fd_params(orc, bo, R, js)
    np.testing.assert_allclose(out["O"][:, js], O_fd, rtol=1e-7, atol=1e-8)
    np.testing.assert_allclose(out["dEL"][:, js], E_fd, rtol=1e-6, atol=1e-7 * (1.0 + np.abs(out["eloc"]).max()))
