"""Python face of the VB-QMC oracle.  TEST INFRASTRUCTURE ONLY.

Plain FP64 CPU restatement of arXiv:2207.14715, Sec. 2, used to check the CUDA library.
Only tests/, the package smoke check and the benchmark's CPU-baseline leg may import it.
The C++ part (vbqmc_oracle.cpp) evaluates the wave function; this module adds the
linear-method estimators (Sec. 2.3.1, Eqs. Hi0, H0j, Hij, Sij, geneigeqM) and the
statistics, in numpy FP64, written as the paper prints them.

Pins: see tests/test_oracle_*.py.  Parity of the linear-method eigenvector choice and of
the DMC step definition is unpinned beyond the checks listed in the design notes.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_c_int_p = ctypes.POINTER(ctypes.c_int)
_c_dbl_p = ctypes.POINTER(ctypes.c_double)


class _OrcSystem(ctypes.Structure):
    _fields_ = [
        ("Nn", ctypes.c_int), ("n_elem", ctypes.c_int),
        ("nuc_xyz", _c_dbl_p), ("nuc_Z", _c_dbl_p), ("nuc_elem", _c_int_p),
        ("S", ctypes.c_int), ("sh_center", _c_int_p), ("sh_l", _c_int_p), ("sh_zeta", _c_dbl_p),
        ("Norb", ctypes.c_int), ("orb_coef", _c_dbl_p),
        ("Nup", ctypes.c_int), ("Ndn", ctypes.c_int),
        ("Nvb", ctypes.c_int), ("c_vb", _c_dbl_p),
        ("inact_off", _c_int_p), ("inact", _c_int_p),
        ("pair_off", _c_int_p), ("pairs", _c_int_p),
        ("unp_off", _c_int_p), ("unp", _c_int_p),
        ("kappa", ctypes.c_double), ("jas_a", _c_dbl_p), ("jas_b", _c_dbl_p),
        ("b1_anti", ctypes.c_double), ("b1_par", ctypes.c_double),
        ("een_on", ctypes.c_int), ("een_theta", _c_dbl_p),
        ("n_cparam", ctypes.c_int), ("cparam", _c_int_p),
        ("jas_param", ctypes.c_int),
        ("n_kappa", ctypes.c_int), ("kappa_kl", _c_int_p),
        ("sh_kind", _c_int_p),
    ]


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_num_params.restype = ctypes.c_int
        L.orc_det_lu.restype = ctypes.c_double
        L.orc_det_leibniz.restype = ctypes.c_double
        L.orc_uniforms2.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                    ctypes.c_uint32, ctypes.c_uint32, _c_dbl_p]
        L.orc_vmc.argtypes = [ctypes.POINTER(_OrcSystem), ctypes.c_int, _c_dbl_p, ctypes.c_int, ctypes.c_double,
                              ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, _c_int_p, _c_dbl_p, _c_dbl_p,
                              _c_int_p, ctypes.c_int]
        L.orc_dmc.argtypes = [ctypes.POINTER(_OrcSystem), ctypes.c_int, _c_int_p, _c_dbl_p, ctypes.c_int,
                              ctypes.c_double, _c_dbl_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32,
                              ctypes.c_uint32, ctypes.c_uint32, _c_dbl_p, _c_dbl_p, _c_int_p, _c_dbl_p, ctypes.c_int]
        _LIB = L
    return _LIB


def _dp(a):
    return a.ctypes.data_as(_c_dbl_p) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(_c_int_p) if a is not None else None


def _pack(spec):
    """Build the C description; returns (struct, keep-alive list)."""
    keep = []

    def d(x):
        a = np.ascontiguousarray(x, dtype=np.float64)
        keep.append(a)
        return _dp(a)

    def i(x):
        a = np.ascontiguousarray(x, dtype=np.int32)
        if a.size == 0:
            a = np.zeros(1, np.int32)
        keep.append(a)
        return _ip(a)

    s = _OrcSystem()
    s.Nn, s.n_elem = spec.Nn, spec.n_elem
    s.nuc_xyz, s.nuc_Z, s.nuc_elem = d(spec.nuc_xyz), d(spec.nuc_Z), i(spec.nuc_elem)
    s.S = len(spec.sh_l)
    s.sh_center, s.sh_l, s.sh_zeta = i(spec.sh_center), i(spec.sh_l), d(spec.sh_zeta)
    s.Norb, s.orb_coef = spec.Norb, d(spec.orb_coef)
    s.Nup, s.Ndn = spec.n_up, spec.n_dn
    s.Nvb, s.c_vb = spec.Nvb, d(spec.c_vb)
    s.inact_off, s.inact = i(spec.inact_off), i(spec.inact)
    s.pair_off, s.pairs = i(spec.pair_off), i(spec.pairs)
    s.unp_off, s.unp = i(spec.unp_off), i(spec.unp)
    s.kappa, s.jas_a, s.jas_b = spec.kappa, d(spec.jas_a), d(spec.jas_b)
    s.b1_anti, s.b1_par = spec.b1_anti, spec.b1_par
    s.een_on, s.een_theta = int(spec.een_on), d(spec.theta())
    s.n_cparam, s.cparam = len(spec.cparam), i(spec.cparam)
    s.jas_param = int(spec.jas_param)
    s.n_kappa, s.kappa_kl = len(spec.kappa_kl), i(spec.kappa_kl)
    s.sh_kind = i(spec.sh_kind) if getattr(spec, "sh_kind", None) is not None else None
    return s, keep


def default_threads():
    return max(1, os.cpu_count() or 1)


def num_params(spec) -> int:
    s, keep = _pack(spec)
    return lib().orc_num_params(ctypes.byref(s))


def evaluate(spec, R, derivs: bool = False, grad: bool = False, nthreads: int | None = None):
    """ln|Psi|, sign, E_L (and grad ln|Psi|, O_p, E_L,p) at R (W, N, 3)."""
    R = np.ascontiguousarray(R, dtype=np.float64)
    W = R.shape[0]
    s, keep = _pack(spec)
    P = lib().orc_num_params(ctypes.byref(s))
    lp, sg, el = np.zeros(W), np.zeros(W), np.zeros(W)
    g = np.zeros((W, spec.N, 3)) if grad else None
    O = np.zeros((W, P)) if derivs else None
    dE = np.zeros((W, P)) if derivs else None
    rc = lib().orc_eval(ctypes.byref(s), W, _dp(R), _dp(lp), _dp(sg), _dp(el), _dp(g), _dp(O), _dp(dE),
                        nthreads or default_threads())
    if rc:
        raise RuntimeError("oracle eval failed: %d" % rc)
    out = {"logpsi": lp, "sign": sg, "eloc": el}
    if grad:
        out["grad"] = g
    if derivs:
        out["O"], out["dEL"] = O, dE
    return out


def nuclear_derivs(spec, R, eloc: bool = True, nthreads: int | None = None):
    """d ln|Psi| / dR_alpha and d E_L / dR_alpha, each (W, Nn, 3), at electron positions R."""
    R = np.ascontiguousarray(R, dtype=np.float64)
    W = R.shape[0]
    s, keep = _pack(spec)
    dlp = np.zeros((W, spec.Nn, 3))
    dE = np.zeros((W, spec.Nn, 3)) if eloc else None
    rc = lib().orc_nuclear_derivs(ctypes.byref(s), W, _dp(R), _dp(dlp), _dp(dE), nthreads or default_threads())
    if rc:
        raise RuntimeError("oracle nuclear derivatives failed: %d" % rc)
    return {"dlogpsi": dlp, "dEL": dE}


def lnJ(spec, R):
    R = np.ascontiguousarray(R, dtype=np.float64)
    s, keep = _pack(spec)
    out = np.zeros(R.shape[0])
    lib().orc_lnJ(ctypes.byref(s), R.shape[0], _dp(R), _dp(out))
    return out


def vmc(spec, R, nsweeps, step, seed, step0=0, system=0, walker_id=None, eloc=True, nthreads=None):
    """Run VMC sweeps; returns (R_final, eloc_hist (nsweeps, W) or None, logpsi, nacc)."""
    R = np.array(R, dtype=np.float64, copy=True, order="C")
    W = R.shape[0]
    s, keep = _pack(spec)
    hist = np.zeros((nsweeps, W)) if eloc else None
    lp = np.zeros(W)
    nacc = np.zeros(W, np.int32)
    wid = None if walker_id is None else np.ascontiguousarray(walker_id, dtype=np.int32)
    rc = lib().orc_vmc(ctypes.byref(s), W, _dp(R), int(nsweeps), float(step), ctypes.c_uint64(seed),
                       ctypes.c_uint32(step0), ctypes.c_uint32(system), _ip(wid), _dp(hist), _dp(lp), _ip(nacc),
                       nthreads or default_threads())
    if rc:
        raise RuntimeError("oracle vmc failed: %d" % rc)
    return R, hist, lp, nacc


def dmc(spec, R, nsteps, tau, e_trial, target, seed, step0=0, system=0, cap=None, nthreads=None, walker_offset=0):
    """Fixed-node DMC (the step of vbqmc_oracle.cpp: drift and branching energy limited near
    nodes as in Umrigar, Nightingale and Runge 1993); returns dict with final population and
    per-step sums."""
    R0 = np.ascontiguousarray(R, dtype=np.float64)
    W = R0.shape[0]
    cap = cap or 4 * max(W, target)
    buf = np.zeros((cap, spec.N, 3))
    buf[:W] = R0
    s, keep = _pack(spec)
    Wio = ctypes.c_int(W)
    et = ctypes.c_double(e_trial)
    swE, sw, et_hist = np.zeros(nsteps), np.zeros(nsteps), np.zeros(nsteps)
    pop = np.zeros(nsteps, np.int32)
    rc = lib().orc_dmc(ctypes.byref(s), cap, ctypes.byref(Wio), _dp(buf), int(nsteps), float(tau),
                       ctypes.byref(et), int(target), ctypes.c_uint64(seed), ctypes.c_uint32(step0),
                       ctypes.c_uint32(system), ctypes.c_uint32(walker_offset), _dp(swE), _dp(sw), _ip(pop),
                       _dp(et_hist),
                       nthreads or default_threads())
    if rc:
        raise RuntimeError("oracle dmc failed: %d" % rc)
    return {"R": buf[:Wio.value].copy(), "W": Wio.value, "e_trial": et.value, "sum_wE": swE, "sum_w": sw,
            "pop": pop, "e_trial_hist": et_hist}


def expand(spec):
    """Signed determinant expansion: list of (structure, d, up tuple, dn tuple)."""
    s, keep = _pack(spec)
    mx = 4096
    st = np.zeros(mx, np.int32)
    d = np.zeros(mx)
    up = np.zeros((mx, max(spec.n_up, 1)), np.int32)
    dn = np.zeros((mx, max(spec.n_dn, 1)), np.int32)
    n = lib().orc_expand(ctypes.byref(s), mx, _ip(st), _dp(d), _ip(up), _ip(dn))
    if n < 0:
        raise RuntimeError("oracle expand failed: %d" % n)
    return [(int(st[t]), float(d[t]), tuple(int(x) for x in up[t, :spec.n_up]),
             tuple(int(x) for x in dn[t, :spec.n_dn])) for t in range(n)]


def een_basis():
    B = np.zeros(23 * 23)
    nt = ctypes.c_int(0)
    nf = lib().orc_een_basis(_dp(B), ctypes.byref(nt))
    return B[:nt.value * nf].reshape(nt.value, nf)


def een_terms():
    t = np.zeros(23 * 4, np.int32)
    n = lib().orc_een_terms(_ip(t))
    return t[:4 * n].reshape(n, 4)


def basis_eval(spec, r):
    s, keep = _pack(spec)
    M = spec.M
    chi, dchi, lchi = np.zeros(M), np.zeros((M, 3)), np.zeros(M)
    r = np.ascontiguousarray(r, dtype=np.float64)
    lib().orc_basis_eval(ctypes.byref(s), _dp(r), _dp(chi), _dp(dchi), _dp(lchi))
    return chi, dchi, lchi


def det_lu(A):
    A = np.ascontiguousarray(A, dtype=np.float64)
    return lib().orc_det_lu(A.shape[0], _dp(A))


def det_leibniz(A):
    A = np.ascontiguousarray(A, dtype=np.float64)
    return lib().orc_det_leibniz(A.shape[0], _dp(A))


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def uniforms2(seed, walker, step, slot, system, purpose):
    u = np.zeros(2)
    lib().orc_uniforms2(ctypes.c_uint64(seed), walker, step, slot, system, purpose, _dp(u))
    return u


# ----------------------------------------------------------------------------------
# Linear method (Sec. 2.3.1), written term by term as Eqs. Hi0, H0j, Hij, Sij print them.
# ----------------------------------------------------------------------------------
def structure_ratios(spec, R, nthreads: int | None = None):
    """Psi_I/Psi_0 = Phi_I/Phi of every VB structure I at R (W, N, 3) -> (W, Nvb) (Sec. 2.4; the
    Jastrow factor cancels).  The c_I derivative of Eq. PsiJVBp is exactly this ratio, so the
    evaluation of a copy of the system with every structure coefficient as a parameter (and no
    Jastrow or orbital parameters) returns them as its first Nvb derivative columns."""
    import dataclasses
    nvb = len(spec.c_vb)
    allc = dataclasses.replace(spec, cparam=np.arange(nvb, dtype=np.int32), jas_param=False,
                               kappa_kl=np.zeros((0, 2), np.int32))
    return evaluate(allc, R, derivs=True, nthreads=nthreads)["O"][:, :nvb]


def structure_overlap(ratios, w=None):
    """S_IJ = <(Psi_I/Psi_0)(Psi_J/Psi_0)> over the samples (Sec. 2.4, the VMC estimate), with
    weights w (None: all 1), as the average of the products sample by sample."""
    X = np.asarray(ratios, np.float64)
    w = np.ones(X.shape[0]) if w is None else np.asarray(w, np.float64)
    S = np.zeros((X.shape[1], X.shape[1]))
    for m in range(X.shape[0]):
        S += w[m] * np.outer(X[m], X[m])
    return S / w.sum()


def structure_weights(S, c):
    """Chirgwin-Coulson and Loewdin weights of the JVB structures (Sec. 2.4) as defined there:
    w_CC_I = sum_J c_I c_J S_IJ / <Psi_0|Psi_0>, and with cbar_K = sum_I c_I (S^1/2)_IK,
    w_L_K = cbar_K^2 / sum_K cbar_K^2; S^1/2 by scipy.linalg.sqrtm."""
    import scipy.linalg
    S = np.asarray(S, np.float64)
    c = np.asarray(c, np.float64)
    n = len(c)
    norm = sum(c[I] * c[J] * S[I, J] for I in range(n) for J in range(n))
    w_cc = np.array([sum(c[I] * c[J] * S[I, J] for J in range(n)) for I in range(n)]) / norm
    half = np.real(scipy.linalg.sqrtm(S))
    cbar = np.array([sum(c[I] * half[I, K] for I in range(n)) for K in range(n)])
    w_l = cbar ** 2 / np.sum(cbar ** 2)
    return w_cc, w_l


def lin_matrices(O, dEL, EL, w=None):
    """Sample estimates from O[M][P] = Psi_j/Psi_0, dEL[M][P] = E_L,j, EL[M] (weights w optional).
    Returns dict E0, gL, gR, H (P x P, nonsymmetric), S (P x P)."""
    O = np.asarray(O, np.float64)
    dEL = np.asarray(dEL, np.float64)
    EL = np.asarray(EL, np.float64)
    M = O.shape[0]
    w = np.ones(M) if w is None else np.asarray(w, np.float64)
    W = w.sum()

    def avg(x):
        return np.tensordot(w, x, axes=(0, 0)) / W

    E = avg(EL)
    Oa = avg(O)
    OE = avg(O * EL[:, None])
    Ej = avg(dEL)
    OOE = np.einsum("m,mi,mj->ij", w * EL, O, O) / W
    OO = np.einsum("m,mi,mj->ij", w, O, O) / W
    OEj = np.einsum("m,mi,mj->ij", w, O, dEL) / W
    gL = 2.0 * (OE - Oa * E)
    gR = 2.0 * (OE - Oa * E + Ej)
    H = (OOE - np.outer(Oa, OE) - np.outer(OE, Oa) + np.outer(Oa, Oa) * E + OEj - np.outer(Oa, Ej))
    S = OO - np.outer(Oa, Oa)
    return {"E0": E, "gL": gL, "gR": gR, "H": H, "S": S}


def lin_solve(E0, gL, gR, H, S, shift=0.0):
    """Eq. geneigeqM: [[E0, gR^T/2], [gL/2, H]] x = E [[1, 0], [0, S]] x.  Picks the lowest real
    eigenvalue whose eigenvector's first component is >= 1e-3 of its norm; returns (dp, E_lin)."""
    import scipy.linalg

    P = len(gL)
    A = np.zeros((P + 1, P + 1))
    B = np.zeros((P + 1, P + 1))
    A[0, 0] = E0
    A[0, 1:] = 0.5 * np.asarray(gR)
    A[1:, 0] = 0.5 * np.asarray(gL)
    A[1:, 1:] = np.asarray(H) + shift * np.eye(P)
    B[0, 0] = 1.0
    B[1:, 1:] = S
    ev, vec = scipy.linalg.eig(A, B)
    best = None
    for k in range(P + 1):
        lam = ev[k]
        if not np.isfinite(lam) or abs(lam.imag) > 1e-8 * max(1.0, abs(lam.real)):
            continue
        v = vec[:, k].real
        if abs(v[0]) < 1e-3 * np.linalg.norm(v):
            continue
        if best is None or lam.real < best[0]:
            best = (lam.real, v / v[0])
    if best is None:
        raise RuntimeError("no admissible eigenvector")
    return best[1][1:], best[0]


def reblock(x):
    """Flyvbjerg-Petersen blocking: mean and the largest standard error over blocking levels
    that keep at least 16 blocks."""
    x = np.asarray(x, np.float64).ravel()
    mean = x.mean()
    best = x.std(ddof=1) / np.sqrt(len(x)) if len(x) > 1 else 0.0
    y = x
    while len(y) >= 32:
        y = 0.5 * (y[0:len(y) // 2 * 2:2] + y[1:len(y) // 2 * 2:2])
        err = y.std(ddof=1) / np.sqrt(len(y))
        best = max(best, err)
    return mean, best
