"""Python binding of the VB-QMC C ABI (include/vbqmc.h): argument marshalling only.

Every computation runs in the CUDA library paper_2207_14715_gb300/_lib/libvbqmc.so.  There is
no fallback: if the library is missing or cannot be loaded, every call raises.  Device arrays
are torch CUDA tensors (used only as device memory); streams are torch CUDA streams.

Names follow the C ABI: create / set_system / inspect_system / eval_walkers / vmc_steps.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .systems import SystemSpec

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libvbqmc.so")

FP64 = 0
MIXED = 1

_c_int_p = ctypes.POINTER(ctypes.c_int)
_c_dbl_p = ctypes.POINTER(ctypes.c_double)


class VbqmcError(RuntimeError):
    pass


class _Desc(ctypes.Structure):
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


EXPORTED = ["vbqmc_create", "vbqmc_destroy", "vbqmc_last_error", "vbqmc_set_system", "vbqmc_inspect_system",
            "vbqmc_walker_state_size", "vbqmc_eval_walkers", "vbqmc_vmc_steps", "vbqmc_accumulate_lin_matrices",
            "vbqmc_launch_info", "vbqmc_last_launch_count", "vbqmc_accumulate_lin_matrices_noalloc",
            "vbqmc_dmc_steps", "vbqmc_set_kernel_timing", "vbqmc_kernel_times", "vbqmc_batch_create",
            "vbqmc_batch_destroy", "vbqmc_batch_vmc_steps", "vbqmc_batch_tune", "vbqmc_batch_info",
            "vbqmc_eval_nuclear_derivs", "vbqmc_weighted_colsum", "vbqmc_lin_solve", "vbqmc_structure_overlap",
            "vbqmc_structure_weights", "vbqmc_measure_alu_peaks", "vbqmc_lin_merge", "vbqmc_use_tables"]

_LIB = None


def lib():
    """Loads libvbqmc.so (raises if it is missing: there is no CPU path)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise VbqmcError("CUDA library not built: %s (run __graft_entry__.build())" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        L.vbqmc_last_error.restype = ctypes.c_char_p
        L.vbqmc_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int]
        L.vbqmc_destroy.argtypes = [ctypes.c_void_p]
        L.vbqmc_set_system.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(_Desc)]
        L.vbqmc_inspect_system.argtypes = [ctypes.POINTER(_Desc), _c_int_p, _c_int_p, ctypes.c_int, _c_dbl_p]
        vp = ctypes.c_void_p
        L.vbqmc_walker_state_size.argtypes = [vp, ctypes.c_int, _c_int_p]
        L.vbqmc_eval_walkers.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp, vp, vp, vp,
                                         vp]
        L.vbqmc_eval_nuclear_derivs.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp, vp,
                                                vp]
        L.vbqmc_weighted_colsum.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp, vp]
        L.vbqmc_vmc_steps.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int,
                                      vp, ctypes.c_int, vp, vp, vp, vp, vp, vp, vp]
        L.vbqmc_last_launch_count.argtypes = [vp]
        L.vbqmc_launch_info.argtypes = [vp, ctypes.c_int, ctypes.c_int, _c_int_p]
        L.vbqmc_accumulate_lin_matrices.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int64, vp, vp, vp, vp,
                                                    vp, vp, vp, vp, vp, vp]
        L.vbqmc_dmc_steps.argtypes = [vp, ctypes.c_int, ctypes.c_int, _c_int_p, ctypes.c_int, vp, ctypes.c_int,
                                      ctypes.c_double, _c_dbl_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32,
                                      ctypes.c_uint32, ctypes.c_uint32, _c_dbl_p, _c_dbl_p, _c_dbl_p, _c_int_p,
                                      _c_dbl_p, ctypes.POINTER(ctypes.c_int64), vp]
        L.vbqmc_batch_create.argtypes = [vp, ctypes.c_int, _c_int_p, _c_int_p, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_void_p)]
        L.vbqmc_batch_destroy.argtypes = [vp]
        L.vbqmc_batch_vmc_steps.argtypes = [vp, vp, ctypes.c_int, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32,
                                            ctypes.c_int, vp, ctypes.c_int, vp, vp, vp, vp, vp, vp, vp]
        L.vbqmc_batch_tune.argtypes = [vp, vp, vp, vp, vp, vp]
        L.vbqmc_batch_info.argtypes = [vp, _c_int_p]
        L.vbqmc_set_kernel_timing.argtypes = [vp, ctypes.c_int]
        L.vbqmc_kernel_times.argtypes = [vp, _c_dbl_p, ctypes.c_int, _c_int_p]
        L.vbqmc_lin_solve.argtypes = [ctypes.c_int, ctypes.c_double, _c_dbl_p, _c_dbl_p, _c_dbl_p, _c_dbl_p,
                                      ctypes.c_double, _c_dbl_p, _c_dbl_p]
        L.vbqmc_structure_overlap.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, ctypes.c_int,
                                              _c_dbl_p, ctypes.c_int, _c_int_p, _c_dbl_p, vp]
        L.vbqmc_use_tables.argtypes = [vp, ctypes.c_int, ctypes.c_int]
        L.vbqmc_lin_merge.argtypes = [ctypes.c_int, ctypes.c_int] + [_c_dbl_p] * 13
        L.vbqmc_structure_weights.argtypes = [ctypes.c_int, _c_dbl_p, _c_dbl_p, _c_dbl_p, _c_dbl_p]
        L.vbqmc_measure_alu_peaks.argtypes = [ctypes.c_int, _c_dbl_p, ctypes.c_int, _c_int_p]
        L.vbqmc_accumulate_lin_matrices_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, vp, vp, vp,
                                                            vp, vp, vp, vp, vp, vp, vp]
        _LIB = L
    return _LIB


def _check(rc):
    if rc != 0:
        raise VbqmcError("vbqmc error %d: %s" % (rc, lib().vbqmc_last_error().decode()))


def _desc(spec: SystemSpec):
    keep = []

    def d(x):
        a = np.ascontiguousarray(x, dtype=np.float64)
        keep.append(a)
        return a.ctypes.data_as(_c_dbl_p)

    def i(x):
        a = np.ascontiguousarray(x, dtype=np.int32)
        if a.size == 0:
            a = np.zeros(1, np.int32)
        keep.append(a)
        return a.ctypes.data_as(_c_int_p)

    s = _Desc()
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


def inspect_system(spec: SystemSpec, max_terms: int = 4096):
    """Host-side set-up only (no device): sizes, the signed determinant terms per structure
    (up orbitals, down orbitals, structure, sign) and the 23x15 e-e-n free-parameter basis."""
    s, keep = _desc(spec)
    info = np.zeros(12, np.int32)
    row = spec.n_up + spec.n_dn + 2
    terms = np.zeros((max_terms, row), np.int32)
    B = np.zeros((23, 15))
    _check(lib().vbqmc_inspect_system(ctypes.byref(s), info.ctypes.data_as(_c_int_p),
                                      terms.ctypes.data_as(_c_int_p), max_terms, B.ctypes.data_as(_c_dbl_p)))
    keys = ["N", "P", "M", "Norb", "nterm", "U_up", "U_dn", "nsterm", "n_ev", "n_kappa_entries", "n_up", "n_dn"]
    d = dict(zip(keys, (int(x) for x in info)))
    return d, terms[:d["nsterm"]], B


def _dp(a):
    return a.ctypes.data_as(_c_dbl_p)


def _ip(a):
    return a.ctypes.data_as(_c_int_p)


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def deriv_dtype(precision):
    """Element type of O and dE_L/dp for a precision mode (the mode's bulk type)."""
    import torch
    return torch.float32 if precision == MIXED else torch.float64


def _check_deriv(precision, *ts):
    want = deriv_dtype(precision)
    for t in ts:
        if t is not None and t.dtype != want:
            raise VbqmcError("derivative arrays must be %s in this precision mode" % want)


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Context:
    """One library context on one CUDA device (vbqmc_create / vbqmc_destroy)."""

    def __init__(self, device: int = 0):
        h = ctypes.c_void_p()
        _check(lib().vbqmc_create(ctypes.byref(h), int(device)))
        self.h = h
        self.device = device
        self.specs = {}

    def close(self):
        if self.h:
            lib().vbqmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_system(self, sys_id: int, spec: SystemSpec):
        s, keep = _desc(spec)
        _check(lib().vbqmc_set_system(self.h, int(sys_id), ctypes.byref(s)))
        self.specs[sys_id] = spec

    def use_tables(self, sys_id: int, on: bool = True):
        """vbqmc_use_tables: carry the system's determinants through reference tables (on) or
        per-determinant inverses (off)."""
        _check(lib().vbqmc_use_tables(self.h, int(sys_id), 1 if on else 0))

    def last_launch_count(self) -> int:
        return int(lib().vbqmc_last_launch_count(self.h))

    def launch_info(self, sys_id, precision) -> dict:
        out = np.zeros(5, np.int32)
        _check(lib().vbqmc_launch_info(self.h, int(sys_id), int(precision), out.ctypes.data_as(_c_int_p)))
        return {"eval_walkers_per_block": int(out[0]), "eval_smem_per_walker": int(out[1]),
                "sweep_walkers_per_block": int(out[2]), "sweep_smem_per_walker": int(out[3]),
                "tables": bool(out[4])}

    def walker_state_size(self, sys_id) -> int:
        n = ctypes.c_int(0)
        _check(lib().vbqmc_walker_state_size(self.h, int(sys_id), ctypes.byref(n)))
        return int(n.value)

    def eval_walkers(self, sys_id, precision, R, logpsi, sign, eloc, grad=None, O=None, dEL=None, state_out=None,
                     stream=None):
        """R [W, N, 3] float64 CUDA tensor; outputs preallocated float64 CUDA tensors."""
        W = R.shape[0]
        _check_deriv(precision, O, dEL)
        _check(lib().vbqmc_eval_walkers(self.h, int(sys_id), int(precision), int(W), _ptr(R), _ptr(logpsi),
                                        _ptr(sign), _ptr(eloc), _ptr(grad), _ptr(O), _ptr(dEL), _ptr(state_out),
                                        _stream(stream)))

    def weighted_colsum(self, ga, Ja, out, gb=None, Jb=None, stream=None):
        """out[k] = sum_w ga[w] Ja[w, k] (+ gb[w] Jb[w, k]); Ja, Jb [W, K] float64 or float32 CUDA
        tensors of one dtype, ga, gb [W] float64, out [K] float64."""
        W = int(Ja.shape[0])
        K = int(np.prod(Ja.shape[1:])) if Ja.dim() > 1 else 1
        for t in (Ja, Jb, ga, gb, out):
            if t is not None and not t.is_contiguous():
                raise ValueError("weighted_colsum needs contiguous tensors")
        jtype = 1 if str(Ja.dtype) == "torch.float32" else 0
        if Jb is not None and Jb.dtype != Ja.dtype:
            raise ValueError("Ja and Jb must have one dtype")
        _check(lib().vbqmc_weighted_colsum(self.h, W, K, jtype, _ptr(ga), _ptr(Ja), _ptr(gb), _ptr(Jb), _ptr(out),
                                           _stream(stream)))

    def eval_nuclear_derivs(self, sys_id, precision, R, logpsi, sign, eloc, dlogpsi_dR, dEL_dR=None, stream=None):
        """Evaluation plus d ln|Psi|/dR_a and dE_L/dR_a ([W, Nn, 3] float64 CUDA tensors)."""
        W = R.shape[0]
        _check(lib().vbqmc_eval_nuclear_derivs(self.h, int(sys_id), int(precision), int(W), _ptr(R), _ptr(logpsi),
                                               _ptr(sign), _ptr(eloc), _ptr(dlogpsi_dR), _ptr(dEL_dR),
                                               _stream(stream)))

    def vmc_steps(self, sys_id, precision, R, nsweeps, step, seed, step0=0, system_tag=0, walker_offset=0,
                  refresh=1, state=None, state_valid=False, nacc=None, logpsi=None, sign=None, eloc=None, O=None,
                  dEL=None, stream=None):
        W = R.shape[0]
        _check_deriv(precision, O, dEL)
        _check(lib().vbqmc_vmc_steps(self.h, int(sys_id), int(precision), int(W), _ptr(R), int(nsweeps),
                                     float(step), ctypes.c_uint64(seed), ctypes.c_uint32(step0),
                                     ctypes.c_uint32(system_tag), ctypes.c_uint32(walker_offset), int(refresh),
                                     _ptr(state), int(bool(state_valid)), _ptr(nacc), _ptr(logpsi), _ptr(sign),
                                     _ptr(eloc), _ptr(O), _ptr(dEL), _stream(stream)))


    def dmc_steps(self, sys_id, precision, R, W, nsteps, tau, E_T, target, seed, step0=0, system_tag=0,
                  walker_offset=0, stream=None):
        """vbqmc_dmc_steps on the population R[:W] of a float64 CUDA tensor R [cap, N, 3] (updated
        in place).  Returns (W, E_T, history) with history the per-step host arrays sum_wE,
        sum_w, sum_wEb, pop, e_trial (truncated to the steps run) and the accepted-move count."""
        cap = R.shape[0]
        W_c = ctypes.c_int(int(W))
        et = ctypes.c_double(float(E_T))
        swe = np.zeros(max(nsteps, 1))
        sw = np.zeros(max(nsteps, 1))
        sweb = np.zeros(max(nsteps, 1))
        pop = np.full(max(nsteps, 1), -1, np.int32)
        etr = np.zeros(max(nsteps, 1))
        nacc = ctypes.c_int64(0)
        _check(lib().vbqmc_dmc_steps(self.h, int(sys_id), int(precision), ctypes.byref(W_c), int(cap), _ptr(R),
                                     int(nsteps), float(tau), ctypes.byref(et), int(target), int(seed) & (2**64 - 1),
                                     int(step0) & 0xffffffff, int(system_tag), int(walker_offset) & 0xffffffff,
                                     _dp(swe), _dp(sw), _dp(sweb), _ip(pop), _dp(etr), ctypes.byref(nacc),
                                     _stream(stream)))
        ran = int((pop >= 0).sum()) if nsteps > 0 else 0
        hist = {"sum_wE": swe[:ran], "sum_w": sw[:ran], "sum_wEb": sweb[:ran], "pop": pop[:ran],
                "e_trial": etr[:ran], "accepted": int(nacc.value)}
        return W_c.value, et.value, hist

    EVAL_KERNELS = ("jastrow", "orbitals", "det", "jastrow_deriv")

    def set_kernel_timing(self, on=True):
        """Record CUDA events around each evaluation kernel (vbqmc_set_kernel_timing)."""
        _check(lib().vbqmc_set_kernel_timing(self.h, 1 if on else 0))

    def kernel_times(self):
        """ms per evaluation kernel of the last timed evaluation, keyed by EVAL_KERNELS."""
        ms = np.zeros(len(self.EVAL_KERNELS))
        n = ctypes.c_int(0)
        _check(lib().vbqmc_kernel_times(self.h, _dp(ms), len(ms), ctypes.byref(n)))
        return dict(zip(self.EVAL_KERNELS, ms.tolist()))

    def accumulate_lin_matrices(self, precision, O, dEL, eloc, weights=None, stream=None):
        """Linear-method estimators (E0, gL, gR, S, H) from O, dEL [M, P] (mode's bulk type) and
        eloc [M] float64 CUDA tensors; returns float64 CUDA tensors."""
        import torch
        _check_deriv(precision, O, dEL)
        M, P = O.shape
        dev = O.device
        E0 = torch.empty(1, dtype=torch.float64, device=dev)
        gL = torch.empty(P, dtype=torch.float64, device=dev)
        gR = torch.empty(P, dtype=torch.float64, device=dev)
        S = torch.empty((P, P), dtype=torch.float64, device=dev)
        H = torch.empty((P, P), dtype=torch.float64, device=dev)
        _check(lib().vbqmc_accumulate_lin_matrices(self.h, int(precision), int(P), int(M), _ptr(O), _ptr(dEL),
                                                   _ptr(eloc), _ptr(weights), _ptr(E0), _ptr(gL), _ptr(gR), _ptr(S),
                                                   _ptr(H), _stream(stream)))
        return {"E0": E0, "gL": gL, "gR": gR, "S": S, "H": H}

    def lin_part(self, precision, O, dEL, eloc, weights=None, stream=None):
        """This rank's share of a multi-rank linear-method accumulation (ranks.merge_lin_parts):
        the estimators of vbqmc_accumulate_lin_matrices plus the weight sum and the mean row <O>
        (vbqmc_weighted_colsum), as host arrays."""
        import torch
        M, P = O.shape
        ones = torch.ones(M, dtype=torch.float64, device=O.device)
        ga = ones if weights is None else weights
        sums = torch.empty(P + 1, dtype=torch.float64, device=O.device)
        self.weighted_colsum(ga, O, sums[:P], stream=stream)
        self.weighted_colsum(ga, ones.reshape(M, 1), sums[P:], stream=stream)
        m = self.accumulate_lin_matrices(precision, O, dEL, eloc, weights=weights, stream=stream)
        out = {k: v.cpu().numpy() for k, v in m.items()}
        h = sums.cpu().numpy()
        out["wsum"] = float(h[P])
        out["mean"] = h[:P] / h[P]
        return out

    def structure_overlap(self, precision, O, cparam, c_vb, weights=None, stream=None):
        """vbqmc_structure_overlap: S_IJ = <(Psi_I/Psi_0)(Psi_J/Psi_0)> (Sec. 2.4) from derivative
        rows O [M, P] (the mode's bulk type) whose first len(cparam) columns are the c_I
        derivatives of the structures cparam.  weights [M] float64 CUDA tensor or None.
        Returns an [Nvb, Nvb] float64 numpy array (the call synchronizes the stream)."""
        M, P = O.shape
        _check_deriv(precision, O)
        c = np.ascontiguousarray(c_vb, np.float64)
        cp = np.ascontiguousarray(cparam, np.int32)
        if len(cp) > P:
            raise VbqmcError("cparam longer than the derivative rows")
        nvb = len(c)
        S = np.zeros((nvb, nvb), np.float64)
        _check(lib().vbqmc_structure_overlap(self.h, int(precision), int(M), int(P), _ptr(O), _ptr(weights), nvb,
                                             _dp(c), len(cp), _ip(cp) if len(cp) else None, _dp(S),
                                             _stream(stream)))
        return S


def structure_weights(S, c_vb):
    """vbqmc_structure_weights: Chirgwin-Coulson and Loewdin weights of the JVB structures
    (Sec. 2.4) from their overlap S [Nvb, Nvb] and coefficients c.  Returns (w_CC, w_L)."""
    S = np.ascontiguousarray(S, np.float64)
    c = np.ascontiguousarray(c_vb, np.float64)
    n = len(c)
    if S.shape != (n, n):
        raise VbqmcError("S must be [Nvb, Nvb]")
    w_cc, w_l = np.zeros(n), np.zeros(n)
    _check(lib().vbqmc_structure_weights(n, _dp(S), _dp(c), _dp(w_cc), _dp(w_l)))
    return w_cc, w_l


def lin_solve(E0, gL, gR, H, S, shift=0.0):
    """vbqmc_lin_solve: the parameter update of Eq. geneigeqM (host FP64 routine of the
    library).  Returns (dp [P], E_lin)."""
    gL = np.ascontiguousarray(gL, np.float64)
    gR = np.ascontiguousarray(gR, np.float64)
    H = np.ascontiguousarray(H, np.float64)
    S = np.ascontiguousarray(S, np.float64)
    P = len(gL)
    if gR.shape != (P,) or H.shape != (P, P) or S.shape != (P, P):
        raise VbqmcError("lin_solve: gL, gR [P] and H, S [P, P] expected")
    dp = np.zeros(P)
    e = ctypes.c_double(0.0)
    _check(lib().vbqmc_lin_solve(P, float(E0), _dp(gL), _dp(gR), _dp(H), _dp(S), float(shift), _dp(dp),
                                 ctypes.byref(e)))
    return dp, e.value


def lin_merge(parts):
    """vbqmc_lin_merge: estimators of the whole sample from per-part ones.  parts: list of dicts
    with 'wsum' (float), 'mean' [P], 'E0', 'gL' [P], 'gR' [P], 'S' [P, P], 'H' [P, P] (host
    values).  Returns a dict with E0 [1], mean [P], gL, gR [P], S, H [P, P] (numpy, float64)."""
    n = len(parts)
    P = len(np.asarray(parts[0]["gL"]))
    stack = lambda k, shape: np.ascontiguousarray(np.stack([np.asarray(p[k], np.float64).reshape(shape)
                                                             for p in parts]))
    ws = np.ascontiguousarray([float(p["wsum"]) for p in parts])
    e0 = np.ascontiguousarray([float(np.asarray(p["E0"]).ravel()[0]) for p in parts])
    mean, gL, gR = stack("mean", (P,)), stack("gL", (P,)), stack("gR", (P,))
    S, H = stack("S", (P, P)), stack("H", (P, P))
    out = {"E0": np.zeros(1), "mean": np.zeros(P), "gL": np.zeros(P), "gR": np.zeros(P), "S": np.zeros((P, P)),
           "H": np.zeros((P, P))}
    _check(lib().vbqmc_lin_merge(n, P, _dp(ws), _dp(mean), _dp(e0), _dp(gL), _dp(gR), _dp(S), _dp(H),
                                 _dp(out["E0"]), _dp(out["mean"]), _dp(out["gL"]), _dp(out["gR"]), _dp(out["S"]),
                                 _dp(out["H"])))
    return out


def measure_alu_peaks(device=0):
    """vbqmc_measure_alu_peaks: {'fp32_tflops', 'fp64_tflops', 'exp_tops', 'sms'} of a device."""
    out = np.zeros(4)
    n = ctypes.c_int(0)
    _check(lib().vbqmc_measure_alu_peaks(int(device), _dp(out), 4, ctypes.byref(n)))
    return {"fp32_tflops": float(out[0]), "fp64_tflops": float(out[1]), "exp_tops": float(out[2]),
            "sms": int(out[3])}


def accumulate_lin_matrices_noalloc(precision, O, dEL, eloc, weights, E0, gL, gR, S, H, stream=None):
    """vbqmc_accumulate_lin_matrices_noalloc: the linear-method estimators into caller-owned
    float64 CUDA tensors E0 [1], gL [P], gR [P], S [P, P], H [P, P], with no device allocation
    by the library or by this wrapper.  Runs on O's device (made current for the call)."""
    import torch
    _check_deriv(precision, O, dEL)
    M, P = O.shape
    for t, shape in ((E0, (1,)), (gL, (P,)), (gR, (P,)), (S, (P, P)), (H, (P, P))):
        if t.dtype != torch.float64 or tuple(t.shape) != shape or not t.is_contiguous() or t.device != O.device:
            raise VbqmcError("outputs must be contiguous float64 tensors on O's device with shapes "
                             "E0 [1], gL [P], gR [P], S [P, P], H [P, P]")
    with torch.cuda.device(O.device):
        _check(lib().vbqmc_accumulate_lin_matrices_noalloc(int(precision), int(P), int(M), _ptr(O), _ptr(dEL),
                                                           _ptr(eloc), _ptr(weights), _ptr(E0), _ptr(gL), _ptr(gR),
                                                           _ptr(S), _ptr(H), _stream(stream)))


def _ptr_array(ts):
    """Host array of device pointers (None -> NULL array)."""
    if ts is None:
        return None
    arr = (ctypes.c_void_p * len(ts))(*[t.data_ptr() if t is not None else None for t in ts])
    return arr


class Batch:
    """Several loaded systems run as one set of launches (vbqmc_batch_*).  Per-system arguments
    are lists of CUDA tensors in the order of sys_ids."""

    KINDS = ("sweep", "jastrow", "jastrow_deriv", "orbitals", "det", "fused")

    def __init__(self, ctx: "Context", sys_ids, walkers, precision):
        self.ctx = ctx
        self.n = len(sys_ids)
        ids = np.ascontiguousarray(sys_ids, np.int32)
        W = np.ascontiguousarray(walkers, np.int32)
        h = ctypes.c_void_p()
        _check(lib().vbqmc_batch_create(ctx.h, self.n, _ip(ids), _ip(W), int(precision), ctypes.byref(h)))
        self.h = h
        self.precision = precision

    def close(self):
        if self.h:
            lib().vbqmc_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def vmc_steps(self, R, nsweeps, step, seed, step0=0, refresh=1, state=None, state_valid=False, nacc=None,
                  logpsi=None, sign=None, eloc=None, O=None, dEL=None, stream=None):
        keep = [_ptr_array(x) for x in (R, state, nacc, logpsi, sign, eloc, O, dEL)]
        _check(lib().vbqmc_batch_vmc_steps(self.h, keep[0], int(nsweeps), float(step), int(seed) & (2**64 - 1),
                                           int(step0) & 0xffffffff, int(refresh), keep[1], 1 if state_valid else 0,
                                           keep[2], keep[3], keep[4], keep[5], keep[6], keep[7], _stream(stream)))

    def tune(self, R, logpsi, sign, eloc, stream=None):
        keep = [_ptr_array(x) for x in (R, logpsi, sign, eloc)]
        _check(lib().vbqmc_batch_tune(self.h, keep[0], keep[1], keep[2], keep[3], _stream(stream)))

    def info(self):
        out = np.zeros(33, np.int32)
        _check(lib().vbqmc_batch_info(self.h, _ip(out)))
        d = {k: dict(zip(("items", "grid", "warps", "persist", "cap"), out[5 * i:5 * i + 5].tolist()))
             for i, k in enumerate(self.KINDS)}
        d["one_launch"] = bool(out[30])
        d["tuned_eval_us"] = {"per_kind": int(out[31]), "one_launch": int(out[32])}
        return d


def create(device: int = 0) -> Context:
    return Context(device)
