"""torch.autograd wrappers of the library's forward calls and their adjoints.

  columns(x, ...)              Eq. colden            backward: urchin_trace_columns_vjp
  shielded_rate(tau, w, s)     Eq. gamma_shld        backward: urchin_gamma_vjp
  equilibrium(gamma, ...)      App. C3 root          backward: urchin_equilibrium_vjp
  converged_x(w, ...)          Sec. 4 fixed point    backward: urchin_solve_vjp
                                                     (implicit function theorem)

Forward and backward both run in the library's CUDA kernels; these classes
only route tensors.  Composing shielded_rate(columns(x)) and calling
backward gives dGamma/dx products; converged_x followed by columns gives the
gradient of a column misfit with respect to the UV-background bin weights.
The recombination case, the frozen set and tau_eff are discrete or only used
for decisions: they carry no gradient.
"""
from __future__ import annotations

import torch

from . import urchin as U


class _Columns(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, bvh, dirs, l_ray, origins, kernel, precision):
        tau = U.urchin_trace_columns(bvh, x.detach().contiguous(), dirs, l_ray, origins, kernel, precision)
        ctx.args = (bvh, dirs, l_ray, origins, kernel, precision, tau.dtype)
        return tau

    @staticmethod
    def backward(ctx, tau_bar):
        bvh, dirs, l_ray, origins, kernel, precision, dt = ctx.args
        xb = U.urchin_trace_columns_vjp(bvh, dirs, l_ray, tau_bar.to(dt).contiguous(), origins, kernel, precision)
        return xb, None, None, None, None, None, None


class _Rate(torch.autograd.Function):
    @staticmethod
    def forward(ctx, tau, w, s):
        g, te = U.urchin_gamma(tau.detach().contiguous(), s, w.detach().contiguous())
        ctx.save_for_backward(tau, w, s)
        ctx.mark_non_differentiable(te)
        return g, te

    @staticmethod
    def backward(ctx, g_bar, te_bar):
        tau, w, s = ctx.saved_tensors
        want_tau, want_w = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (want_tau or want_w):
            return None, None, None
        tb, wb = U.urchin_gamma_vjp(tau.detach().contiguous(), s, w.detach().contiguous(),
                                    g_bar.to(torch.float64).contiguous(), want_tau=want_tau, want_w=want_w)
        return tb, wb, None


class _Equilibrium(torch.autograd.Function):
    @staticmethod
    def forward(ctx, gamma, tau_eff, nH, T, case_rule, y):
        x = U.urchin_equilibrium(gamma.detach().contiguous(), tau_eff, nH, T, case_rule, y)
        ctx.save_for_backward(gamma, tau_eff, nH, T)
        ctx.args = (case_rule, y)
        return x

    @staticmethod
    def backward(ctx, x_bar):
        gamma, tau_eff, nH, T = ctx.saved_tensors
        case_rule, y = ctx.args
        gb = U.urchin_equilibrium_vjp(gamma.detach().contiguous(), tau_eff, nH, T,
                                      x_bar.to(torch.float64).contiguous(), case_rule, y)
        return gb, None, None, None, None, None


class _ConvergedX(torch.autograd.Function):
    @staticmethod
    def forward(ctx, w, bvh, dirs, l_ray, s, nH, T, solve_kw, vjp_kw, info):
        state = torch.empty(bvh.n, dtype=torch.uint8, device=w.device)
        x, st = U.urchin_solve(bvh, dirs, l_ray, s, w.detach().contiguous(), nH, T, state=state, **solve_kw)
        ctx.save_for_backward(w, s, nH, T, x, state)
        ctx.args = (bvh, dirs, l_ray, solve_kw, vjp_kw, info)
        if info is not None:
            info["forward_stats"] = st
        return x

    @staticmethod
    def backward(ctx, x_bar):
        w, s, nH, T, x, state = ctx.saved_tensors
        bvh, dirs, l_ray, solve_kw, vjp_kw, info = ctx.args
        keep = {k: solve_kw[k] for k in ("y", "tau_skip", "segments", "kernel", "precision", "case_rule",
                                         "warm_start") if k in solve_kw}
        keep.update(vjp_kw)
        wb, st = U.urchin_solve_vjp(bvh, dirs, l_ray, s, w.detach().contiguous(), nH, T, x, state,
                                    x_bar.to(torch.float64).contiguous(), **keep)
        if info is not None:
            info["vjp_stats"] = st
        return wb, None, None, None, None, None, None, None, None, None


def columns(x, bvh, dirs, l_ray, origins=None, kernel=U.KERNEL_M4, precision=U.F32):
    """tau[o, k] of Eq. colden, differentiable in x (float64 [n])."""
    return _Columns.apply(x, bvh, dirs, l_ray, origins, kernel, precision)


def shielded_rate(tau, w, s):
    """(Gamma [n_orig] float64, tau_eff [n_orig] float32) of Eq. gamma_shld,
    differentiable in tau and in the spectrum weights w."""
    return _Rate.apply(tau, w, s)


def equilibrium(gamma, tau_eff, nH, T, case_rule=U.CASE_AUTO, y=0.0):
    """Equilibrium neutral fraction (App. C3), differentiable in gamma."""
    return _Equilibrium.apply(gamma, tau_eff, nH, T, case_rule, y)


def converged_x(w, bvh, dirs, l_ray, s, nH, T, solve_kw=None, vjp_kw=None, info=None):
    """x* of urchin_solve for spectrum weights w, differentiable in w by the
    implicit function theorem (urchin_solve_vjp).  solve_kw go to
    urchin_solve (tol should be tight: the gradient is that of the exact
    fixed point), vjp_kw (tol, max_iter, gmres_m) to urchin_solve_vjp.  A
    dict `info` receives the forward solve's statistics ("forward_stats")
    and, after backward, the adjoint's ("vjp_stats")."""
    return _ConvergedX.apply(w, bvh, dirs, l_ray, s, nH, T, dict(solve_kw or {}), dict(vjp_kw or {}), info)
