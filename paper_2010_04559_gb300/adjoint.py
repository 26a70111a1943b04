"""Detector response R(sigma_t, sigma_s, f_n) = sum_c w[c] int_cell phi_s dV
and its gradients through the adjoint, as a torch.autograd.Function.

Marshalling only: the forward solve A psi = f, the adjoint solve
A^T lambda = g (a context with amgt_set_adjoint(1) and the isotropic source
4 pi * w) and the gradient reductions run in libamgt (include/amgt.h:
amgt_solve, amgt_response, amgt_response_gradients).
"""
import numpy as np

from ._capi import AMGT_MODE_F64, AMGT_PREC_MG, context_from_problem


def response_problem(prob, weight):
    """The problem dict of the adjoint solve: source = isotropic emission
    4 pi * weight per cell, vacuum boundaries; cross sections and moments as
    in `prob`."""
    q = dict(prob)
    q["q"] = 4.0 * np.pi * np.asarray(weight, dtype=np.float64)
    q["boundary"] = [(0, 0.0)] * (2 * prob["dim"])
    return q


def solve_response(prob, weight, device=0, tol=1e-12, mode=AMGT_MODE_F64, precond=AMGT_PREC_MG):
    """Forward and adjoint solves on the GPU; returns (R, psi, lam,
    dR/dsigma_t, dR/dsigma_s, dR/df) with torch CUDA float64 tensors."""
    import torch
    dev = torch.device("cuda", device)
    fwd = context_from_problem(prob, device=device)
    adj = context_from_problem(response_problem(prob, weight), device=device)
    try:
        adj.amgt_set_adjoint(1)
        ns, na = fwd.amgt_query_sizes(0)
        psi = torch.empty((ns, na), device=dev, dtype=torch.float64)
        lam = torch.empty_like(psi)
        phi = torch.empty(ns, device=dev, dtype=torch.float64)
        fwd.amgt_solve(tol=tol, precond=precond, mode=mode, psi=psi, phi=phi, device_ptrs=True)
        adj.amgt_solve(tol=tol, precond=precond, mode=mode, psi=lam, phi=phi, device_ptrs=True)
        R = adj.amgt_response(psi)
        C = int(np.prod(prob["ncell"]))
        dt = torch.empty(C, device=dev, dtype=torch.float64)
        ds = torch.empty(C, device=dev, dtype=torch.float64)
        # one row of f_n per material (one row without mat_id)
        df = torch.empty(np.asarray(prob["fmom"]).shape, device=dev, dtype=torch.float64)
        fwd.amgt_response_gradients(psi, lam, dt, ds, df)
    finally:
        fwd.close()
        adj.close()
    return R, psi, lam, dt, ds, df


class DetectorResponse:
    """R = DetectorResponse.apply(sigma_t, sigma_s, fmom, prob, weight) for
    torch tensors sigma_t [C], sigma_s [C] (n = 0 scatter per cell) and
    fmom [N+1] (f_n, f_0 = 1), or [nmat][N+1] with prob["mat_id"]; backward
    returns the adjoint gradients."""

    _fn = None

    @classmethod
    def apply(cls, sigma_t, sigma_s, fmom, prob, weight, **solve_kw):
        if cls._fn is None:
            cls._fn = _make_function()
        return cls._fn.apply(sigma_t, sigma_s, fmom, prob, weight, solve_kw)


def _make_function():
    import torch

    class _Fn(torch.autograd.Function):
        @staticmethod
        def forward(fctx, sigma_t, sigma_s, fmom, prob, weight, solve_kw):
            p = dict(prob)
            p["sigma_t"] = sigma_t.detach().double().cpu().numpy()
            p["sigma_s"] = sigma_s.detach().double().cpu().numpy()
            p["fmom"] = fmom.detach().double().cpu().numpy()
            dev = sigma_t.device.index if sigma_t.is_cuda else 0
            R, _, _, dt, ds, df = solve_response(p, weight, device=dev, **solve_kw)
            fctx.save_for_backward(dt.to(sigma_t.device), ds.to(sigma_s.device),
                                   df.to(fmom.device))
            return torch.tensor(R, dtype=torch.float64, device=sigma_t.device)

        @staticmethod
        def backward(fctx, gR):
            dt, ds, df = fctx.saved_tensors
            return gR * dt, gR * ds, gR * df, None, None, None

    return _Fn
