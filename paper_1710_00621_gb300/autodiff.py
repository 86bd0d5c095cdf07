"""Differentiable Wiener / CR solve: a torch.autograd.Function over the library's solver.

The solution x of A(theta) x = b(theta) (Eq. A) is a function of the scalar mixing
matrix q_{nu,k} (Eq. P with constant mixing), of spatially variable mixing maps q_{nu,k}(p)
(Eq. Q, ``wiener_solution_maps``, gradients by ``cmbws_grad_mix_maps``) and of the prior
spectra; here the prior
of component k is parametrised by a log-scale t_k, C_{k,l} = exp(t_k) C0_{k,l}.  The
backward pass runs one more solve, A lambda = dL/dx (A is symmetric), and evaluates
lambda^T (db/dtheta - dA/dtheta x) with ``cmbws_grad_terms``.  Spectral indices and
amplitudes enter through ordinary torch arithmetic on q and t (e.g. ``power_law_q``).

Every transform and vector operation runs in libcmbws; this module only marshals
arguments (it builds the model for the current parameters, calls the solver, and
reshapes the gradient terms).
"""
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import binding as B


@dataclass
class WienerProblem:
    """Everything of the model except the differentiated parameters.

    grids: [nobs] band Grid; beams: [nobs] b_l; cl0: [ncomp] reference C_l (None = no
    prior); ninv: [nobs] CUDA float64 tau maps; d: [nobs] CUDA float64 data maps;
    omega1 / omega2: optional CR draws (as in cmbws_rhs)."""
    lmax_comp: Sequence[int]
    grids: list
    beams: list
    cl0: list
    ninv: list
    d: list
    omega1: Optional[list] = None
    omega2: Optional[torch.Tensor] = None
    prec: int = B.CMBWS_FP64
    tol: float = 1e-10
    adjoint_tol: Optional[float] = None
    maxiter: int = 2000
    inner_tol: float = 1e-3
    cert_prec: Optional[int] = None
    mix_grids: Optional[list] = None   # [nobs][ncomp] mixing Grid of a variable pair, or None

    @property
    def nobs(self):
        return len(self.grids)

    @property
    def ncomp(self):
        return len(self.lmax_comp)

    def model(self, q, t, mix_maps=None):
        """cmbws model for mixing q [nobs, ncomp] and prior log-scales t [ncomp] (host arrays),
        with the variable pairs' maps mix_maps [nobs][ncomp] (CUDA float64 or None)."""
        cls = [None if c is None else np.asarray(c, dtype=np.float64) * float(np.exp(t[k]))
               for k, c in enumerate(self.cl0)]
        return B.cmbws_model_create(list(self.lmax_comp), self.grids, self.beams, cls, self.ninv,
                                    np.asarray(q, dtype=np.float64), prec=self.prec,
                                    mix_grids=self.mix_grids if mix_maps is not None else None,
                                    mix_maps=mix_maps)

    def solve(self, model, b, tol):
        x = torch.zeros_like(b)
        cert = self.cert_prec
        if cert is None:
            cert = B.CMBWS_FP64 if self.prec == B.CMBWS_FP64 else B.CMBWS_FP32X2
        rep = B.cmbws_cg_solve(model, b, x, tol=tol, maxiter=self.maxiter, inner_tol=self.inner_tol,
                               cert_prec=cert)
        return x, rep


class WienerSolution(torch.autograd.Function):
    """x = A(q, t)^-1 b(q, t); differentiable in q [nobs, ncomp] and t [ncomp]."""

    @staticmethod
    def forward(ctx, q, t, prob):
        qh = q.detach().double().cpu().numpy().reshape(prob.nobs, prob.ncomp)
        th = t.detach().double().cpu().numpy().reshape(prob.ncomp)
        model = prob.model(qh, th)
        dev = prob.d[0].device
        b = torch.empty(model.nvec, dtype=torch.float64, device=dev)
        B.cmbws_rhs(model, prob.d, b, prob.omega1, prob.omega2)
        x, rep = prob.solve(model, b, prob.tol)
        ctx.prob, ctx.model, ctx.report = prob, model, rep
        ctx.save_for_backward(x)
        ctx.q_meta = (q.dtype, q.device, q.shape)
        ctx.t_meta = (t.dtype, t.device, t.shape)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        prob, model = ctx.prob, ctx.model
        lam, rep = prob.solve(model, gx.contiguous().double(), prob.adjoint_tol or prob.tol)
        ctx.adjoint_report = rep
        out = torch.empty(prob.nobs * prob.ncomp + prob.ncomp, dtype=torch.float64, device=x.device)
        B.cmbws_grad_terms(model, x, lam, prob.d, out, prob.omega1, prob.omega2)
        gq = out[:prob.nobs * prob.ncomp].reshape(prob.nobs, prob.ncomp)
        gt = out[prob.nobs * prob.ncomp:]
        qd, qdev, qs = ctx.q_meta
        td, tdev, ts = ctx.t_meta
        return gq.to(device=qdev, dtype=qd).reshape(qs), gt.to(device=tdev, dtype=td).reshape(ts), None


class WienerSolutionMaps(torch.autograd.Function):
    """x = A(q, t, maps)^-1 b(q, t, maps); differentiable in q, t and the mixing maps of the
    variable pairs (one tensor per pair, in the order of ``pairs``)."""

    @staticmethod
    def forward(ctx, q, t, prob, pairs, *maps):
        qh = q.detach().double().cpu().numpy().reshape(prob.nobs, prob.ncomp)
        th = t.detach().double().cpu().numpy().reshape(prob.ncomp)
        mm = [[None] * prob.ncomp for _ in range(prob.nobs)]
        for (nu, k), mp in zip(pairs, maps):
            mm[nu][k] = mp.detach().to(dtype=torch.float64).contiguous()
        model = prob.model(qh, th, mm)
        dev = prob.d[0].device
        b = torch.empty(model.nvec, dtype=torch.float64, device=dev)
        B.cmbws_rhs(model, prob.d, b, prob.omega1, prob.omega2)
        x, rep = prob.solve(model, b, prob.tol)
        ctx.prob, ctx.model, ctx.report, ctx.pairs = prob, model, rep, pairs
        ctx.save_for_backward(x)
        ctx.q_meta = (q.dtype, q.device, q.shape)
        ctx.t_meta = (t.dtype, t.device, t.shape)
        ctx.m_meta = [(mp.dtype, mp.device, mp.shape) for mp in maps]
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        prob, model = ctx.prob, ctx.model
        lam, rep = prob.solve(model, gx.contiguous().double(), prob.adjoint_tol or prob.tol)
        ctx.adjoint_report = rep
        out = torch.empty(prob.nobs * prob.ncomp + prob.ncomp, dtype=torch.float64, device=x.device)
        B.cmbws_grad_terms(model, x, lam, prob.d, out, prob.omega1, prob.omega2)
        gm = [[None] * prob.ncomp for _ in range(prob.nobs)]
        for (nu, k), (dt, dv, sh) in zip(ctx.pairs, ctx.m_meta):
            gm[nu][k] = torch.empty(sh, dtype=torch.float64, device=x.device).reshape(-1)
        B.cmbws_grad_mix_maps(model, x, lam, prob.d, gm, prob.omega1)
        gq = out[:prob.nobs * prob.ncomp].reshape(prob.nobs, prob.ncomp).clone()
        for nu, k in ctx.pairs:  # the scalar entry of a variable pair is not a parameter here
            gq[nu, k] = 0.0
        gt = out[prob.nobs * prob.ncomp:]
        qd, qdev, qs = ctx.q_meta
        td, tdev, ts = ctx.t_meta
        gmaps = [gm[nu][k].to(device=dv, dtype=dt).reshape(sh)
                 for (nu, k), (dt, dv, sh) in zip(ctx.pairs, ctx.m_meta)]
        return (gq.to(device=qdev, dtype=qd).reshape(qs), gt.to(device=tdev, dtype=td).reshape(ts),
                None, None, *gmaps)


def wiener_solution_maps(q, t, maps, prob: WienerProblem):
    """Differentiable solution x(q, t, maps); maps: [nobs][ncomp] CUDA tensors on the pairs'
    mixing grids (prob.mix_grids) or None for scalar pairs (which take q)."""
    pairs = [(nu, k) for nu in range(prob.nobs) for k in range(prob.ncomp) if maps[nu][k] is not None]
    return WienerSolutionMaps.apply(q, t, prob, pairs, *[maps[nu][k] for nu, k in pairs])


def wiener_solution(q, t, prob: WienerProblem):
    """Differentiable solution x(q, t) of the problem (see WienerSolution)."""
    return WienerSolution.apply(q, t, prob)


def power_law_q(freqs, nu0, beta, fixed: List[bool]):
    """q_{nu,k} = (nu / nu0_k)^beta_k as a torch expression (flat columns where fixed[k])."""
    f = torch.as_tensor(np.asarray(freqs, dtype=np.float64))[:, None]
    n0 = torch.as_tensor(np.asarray(nu0, dtype=np.float64))[None, :]
    q = (f / n0) ** beta[None, :]
    mask = torch.as_tensor(np.asarray(fixed, dtype=bool))[None, :]
    return torch.where(mask, torch.ones_like(q), q)


class SHTSynthesis(torch.autograd.Function):
    """map = Y alm (cmbws_sht_synth, Sec. 2.1) with its hand-written adjoint: the gradient of a
    loss with respect to alm is Y^T (dL/dmap), the adjoint synthesis of the library
    (cmbws_sht_analysis with weighted = 0, Sec. 3.2), the exact transpose of the synthesis.

    alm: CUDA float64 [nmaps, (L+1)^2] (CMBWS_ALM order) or [(L+1)^2]; returns [nmaps, npix]
    (or [npix])."""

    @staticmethod
    def forward(ctx, alm, grid, prec):
        a = alm.detach().contiguous()
        nmaps = 1 if a.dim() == 1 else a.shape[0]
        out = torch.empty((nmaps, grid.npix) if a.dim() > 1 else (grid.npix,), dtype=torch.float64,
                          device=a.device)
        B.cmbws_sht_synth(grid, prec, a, out, nmaps)
        ctx.grid, ctx.prec, ctx.nmaps, ctx.shape = grid, prec, nmaps, a.shape
        return out

    @staticmethod
    def backward(ctx, g):
        ga = torch.empty(ctx.shape, dtype=torch.float64, device=g.device)
        B.cmbws_sht_analysis(ctx.grid, ctx.prec, g.contiguous(), ga, ctx.nmaps, 0)
        return ga, None, None


class SHTAdjoint(torch.autograd.Function):
    """alm = Y^T map (adjoint synthesis, cmbws_sht_analysis with weighted = 0), whose own
    adjoint is the synthesis Y: the gradient with respect to the map is Y (dL/dalm)."""

    @staticmethod
    def forward(ctx, m, grid, prec):
        f = m.detach().contiguous()
        nmaps = 1 if f.dim() == 1 else f.shape[0]
        nalm = (grid.lmax + 1) ** 2
        out = torch.empty((nmaps, nalm) if f.dim() > 1 else (nalm,), dtype=torch.float64,
                          device=f.device)
        B.cmbws_sht_analysis(grid, prec, f, out, nmaps, 0)
        ctx.grid, ctx.prec, ctx.nmaps, ctx.shape = grid, prec, nmaps, f.shape
        return out

    @staticmethod
    def backward(ctx, g):
        gm = torch.empty(ctx.shape, dtype=torch.float64, device=g.device)
        B.cmbws_sht_synth(ctx.grid, ctx.prec, g.contiguous(), gm, ctx.nmaps)
        return gm, None, None


def sht_synth(alm, grid, prec=B.CMBWS_FP64):
    """Differentiable Y alm."""
    return SHTSynthesis.apply(alm, grid, prec)


def sht_adjoint(m, grid, prec=B.CMBWS_FP64):
    """Differentiable Y^T map."""
    return SHTAdjoint.apply(m, grid, prec)
