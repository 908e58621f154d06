"""Host-side checks of the CUDA library that need no GPU: exported C ABI, system set-up
(structure expansion, e-e-n cusp basis, parameter count) against the oracle, and argument
validation."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2207_14715_gb300 import systems as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def vb():
    from paper_2207_14715_gb300 import build, vbqmc
    build.build()
    vbqmc.lib()
    return vbqmc


def _declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\s*(?:int|void|const char\*)\s+(vbqmc_\w+)\s*\(", txt, re.M))
    return names


def test_library_exports_every_declared_symbol(vb):
    names = _declared_symbols()
    assert {"vbqmc_create", "vbqmc_set_system", "vbqmc_eval_walkers", "vbqmc_vmc_steps"} <= names
    L = vb.lib()
    for n in sorted(names):
        assert hasattr(L, n), n
        assert ctypes.cast(getattr(L, n), ctypes.c_void_p).value


def _canonical(up, dn, sign):
    """Sort the orbital lists of a determinant, folding the sorting parities into the sign."""
    sgn = sign
    for v in (up, dn):
        inv = sum(1 for a in range(len(v)) for b in range(a + 1, len(v)) if v[a] > v[b])
        if inv % 2:
            sgn = -sgn
    return tuple(sorted(up)), tuple(sorted(dn)), sgn


@pytest.mark.parametrize("maker", [S.h2_vb, S.small_open_shell, S.ethylene_vb, S.h2_nodeless])
def test_structure_expansion_matches_oracle(vb, orc, maker):
    spec = maker()
    info, terms, _ = vb.inspect_system(spec)
    mine = {}
    for r in terms:
        up = tuple(int(x) for x in r[:spec.n_up])
        dn = tuple(int(x) for x in r[spec.n_up:spec.n_up + spec.n_dn])
        mine[(int(r[-2]), up, dn)] = int(r[-1])
    ref = {}
    for (I, d, up, dn) in orc.expand(spec):
        u, v, sg = _canonical(up, dn, d)
        ref[(I, u, v)] = ref.get((I, u, v), 0) + int(sg)
    assert mine == ref
    assert info["N"] == spec.N and info["M"] == spec.M
    assert info["P"] == spec.n_params == orc.num_params(spec)


def test_een_cusp_basis_matches_oracle(vb, orc):
    _, _, B = vb.inspect_system(S.small_open_shell())
    np.testing.assert_allclose(B, orc.een_basis(), atol=1e-13)


def test_ethylene_sizes(vb):
    info, _, _ = vb.inspect_system(S.ethylene_vb())
    assert info["nterm"] == 24 and info["U_up"] == 8 and info["U_dn"] == 8
    assert info["M"] == 126 and info["P"] == 216


def test_invalid_inputs_are_rejected(vb):
    spec = S.small_open_shell()
    bad = S.small_open_shell()
    bad.inact = np.array([99], np.int32)
    with pytest.raises(vb.VbqmcError, match="bad orbital"):
        vb.inspect_system(bad)
    bad = S.small_open_shell()
    bad.n_up = 4
    with pytest.raises(vb.VbqmcError):
        vb.inspect_system(bad)
    bad = S.small_open_shell()
    bad.sh_l = spec.sh_l.copy()
    bad.sh_l[0] = 3
    with pytest.raises(vb.VbqmcError, match="l must be"):
        vb.inspect_system(bad)
    bad = S.small_open_shell()
    bad.kappa_kl = np.array([[1, 1]], np.int32)
    with pytest.raises(vb.VbqmcError, match="excitation"):
        vb.inspect_system(bad)
    # the packed shell records hold the center index in 16 bits
    bad = S.h2_vb()
    n = 65536
    bad.nuc_xyz, bad.nuc_Z, bad.nuc_elem = np.zeros((n, 3)), np.ones(n), np.zeros(n, np.int32)
    with pytest.raises(vb.VbqmcError, match="65535 nuclei"):
        vb.inspect_system(bad)


def test_binding_exposes_the_entry_points(vb):
    """The Python binding has one method per C entry point (argument marshalling only)."""
    for name in ("set_system", "eval_walkers", "eval_nuclear_derivs", "vmc_steps", "dmc_steps",
                 "accumulate_lin_matrices", "walker_state_size", "launch_info", "last_launch_count", "close"):
        assert callable(getattr(vb.Context, name)), name
    for name in ("create", "inspect_system", "lin_solve", "deriv_dtype", "accumulate_lin_matrices_noalloc"):
        assert callable(getattr(vb, name)), name
    for sym in vb.EXPORTED:
        assert hasattr(vb.lib(), sym)


def test_slater_shells_in_the_host_setup(vb):
    """Slater shells are accepted (zeta > 0) and counted like Gaussian shells; a bad kind or a
    Slater zeta of 0 is refused."""
    from paper_2207_14715_gb300 import systems as S
    spec = S.slater_h2()
    info, _, _ = vb.inspect_system(spec)
    assert info["M"] == spec.M
    bad = S.slater_h2()
    bad.sh_kind = np.full(len(bad.sh_l), 2, np.int32)
    with pytest.raises(vb.VbqmcError, match="kind"):
        vb.inspect_system(bad)
    bad = S.slater_1s(1.0, 1.0)
    bad.sh_zeta = np.zeros(1)
    with pytest.raises(vb.VbqmcError, match="zeta"):
        vb.inspect_system(bad)
