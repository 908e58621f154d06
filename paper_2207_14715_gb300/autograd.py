"""torch.autograd face of the evaluation: ln|Psi| and E_L of a set of walkers as functions of
the wave-function parameters p (arXiv:2207.14715, Sec. 2.2, Eq. PsiJVBp) and of the nucleus
positions.  The backward pass uses the library's derivative kernels (O_j and E_L,j of
Sec. 2.3.1; the nucleus derivatives) and its weighted column sum over walkers, so that
d/dp of a loss sum_w (a_w ln|Psi_w| + b_w E_L,w) is sum_w (a_w O_w + b_w E_L,p,w).

Argument marshalling only: the forward reloads the system with the given values (host
set-up of the C ABI) and every number comes from the CUDA library.  The orbital-rotation
parameters kappa_kl are derivatives at the current orbitals (Sec. 2.2): their values must be
zero, and their gradient is the one at kappa = 0.  Electron positions get no gradient.
"""
from __future__ import annotations

import copy

import numpy as np
import torch

from . import vbqmc
from .systems import EEN_NFREE, SystemSpec


def parameter_vector(spec: SystemSpec) -> np.ndarray:
    """Current parameter values in the library's order: c_I (cparam), then if jas_param
    a_2..a_6 per element, b_2..b_6 and (with e-e-n) theta per element, then kappa_kl = 0."""
    v = [np.asarray(spec.c_vb, dtype=np.float64)[np.asarray(spec.cparam, dtype=np.int64)]]
    if spec.jas_param:
        v.append(np.asarray(spec.jas_a, dtype=np.float64)[:, 1:6].reshape(-1))
        v.append(np.asarray(spec.jas_b, dtype=np.float64)[1:6])
        if spec.een_on:
            v.append(spec.theta().reshape(-1))
    v.append(np.zeros(len(spec.kappa_kl)))
    return np.concatenate(v).astype(np.float64)


def with_parameters(spec: SystemSpec, p=None, nuclei=None) -> SystemSpec:
    """Copy of spec with parameter vector p (order of parameter_vector) and nucleus positions
    [Nn, 3] replaced; kappa entries of p must be zero."""
    out = copy.deepcopy(spec)
    if nuclei is not None:
        out.nuc_xyz = np.array(nuclei, dtype=np.float64).reshape(spec.Nn, 3)
    if p is None:
        return out
    p = np.asarray(p, dtype=np.float64).reshape(-1)
    if p.size != spec.n_params:
        raise ValueError("parameter vector has %d entries, the system %d" % (p.size, spec.n_params))
    o = 0
    out.c_vb = np.array(spec.c_vb, dtype=np.float64)
    nc = len(spec.cparam)
    out.c_vb[np.asarray(spec.cparam, dtype=np.int64)] = p[o:o + nc]
    o += nc
    if spec.jas_param:
        ne = spec.n_elem
        out.jas_a = np.array(spec.jas_a, dtype=np.float64)
        out.jas_a[:, 1:6] = p[o:o + 5 * ne].reshape(ne, 5)
        o += 5 * ne
        out.jas_b = np.array(spec.jas_b, dtype=np.float64)
        out.jas_b[1:6] = p[o:o + 5]
        o += 5
        if spec.een_on:
            out.een_theta = p[o:o + EEN_NFREE * ne].reshape(ne, EEN_NFREE).copy()
            o += EEN_NFREE * ne
    if np.any(p[o:] != 0.0):
        raise ValueError("orbital-rotation parameters are derivatives at kappa = 0: their values must be 0")
    return out


class _Evaluate(torch.autograd.Function):
    @staticmethod
    def forward(fctx, p, nuclei, R, ctx, sys_id, spec, precision):
        need_p = p.requires_grad and spec.n_params > 0
        need_n = nuclei.requires_grad
        ctx.set_system(sys_id, with_parameters(spec, p.detach().cpu().numpy(), nuclei.detach().cpu().numpy()))
        W = R.shape[0]
        dev = R.device
        lp, sg, el = (torch.zeros(W, dtype=torch.float64, device=dev) for _ in range(3))
        O = dE = None
        if need_p:
            O = torch.zeros((W, spec.n_params), dtype=vbqmc.deriv_dtype(precision), device=dev)
            dE = torch.zeros_like(O)
        ctx.eval_walkers(sys_id, precision, R, lp, sg, el, O=O, dEL=dE)
        dlp = dER = None
        if need_n:
            dlp = torch.zeros((W, spec.Nn, 3), dtype=torch.float64, device=dev)
            dER = torch.zeros_like(dlp)
            lp2, sg2, el2 = (torch.zeros_like(lp) for _ in range(3))
            ctx.eval_nuclear_derivs(sys_id, precision, R, lp2, sg2, el2, dlp, dER)
        fctx.vb = ctx
        fctx.saved = (O, dE, dlp, dER)
        fctx.p_meta = (p.dtype, p.device, tuple(p.shape))
        fctx.n_meta = (nuclei.dtype, nuclei.device, tuple(nuclei.shape))
        return lp, el

    @staticmethod
    def backward(fctx, g_lp, g_el):
        O, dE, dlp, dER = fctx.saved
        ctx = fctx.vb
        if O is None and dlp is None:
            return (None,) * 7
        ref = O if O is not None else dlp
        W = ref.shape[0]
        dev = ref.device
        ga = (g_lp if g_lp is not None else torch.zeros(W, device=dev)).to(torch.float64).contiguous()
        gb = (g_el if g_el is not None else torch.zeros(W, device=dev)).to(torch.float64).contiguous()
        grads = [None, None]
        if O is not None:
            out = torch.zeros(O.shape[1], dtype=torch.float64, device=dev)
            ctx.weighted_colsum(ga, O, out, gb, dE)
            dt, dv, sh = fctx.p_meta
            grads[0] = out.to(dtype=dt, device=dv).reshape(sh)
        if dlp is not None:
            out = torch.zeros(dlp.shape[1] * 3, dtype=torch.float64, device=dev)
            ctx.weighted_colsum(ga, dlp.reshape(W, -1), out, gb, dER.reshape(W, -1))
            dt, dv, sh = fctx.n_meta
            grads[1] = out.to(dtype=dt, device=dv).reshape(sh)
        return grads[0], grads[1], None, None, None, None, None


def evaluate(ctx: "vbqmc.Context", sys_id: int, spec: SystemSpec, R, precision: int = vbqmc.MIXED, params=None,
             nuclei=None):
    """ln|Psi| and E_L [W] of walkers R [W, N, 3] (float64 CUDA), differentiable in params [P]
    and nuclei [Nn, 3] (torch tensors; defaults: the values in spec, without gradient).  The
    system is (re)loaded under sys_id with those values."""
    if params is None:
        params = torch.tensor(parameter_vector(spec))
    if nuclei is None:
        nuclei = torch.tensor(np.asarray(spec.nuc_xyz, dtype=np.float64))
    return _Evaluate.apply(params, nuclei, R, ctx, int(sys_id), spec, int(precision))
