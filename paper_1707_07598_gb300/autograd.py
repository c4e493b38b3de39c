"""torch.autograd bindings of the MSFV path.

Two differentiable functions of the log-conductivity m, both backed by a Session (one
mesh, coarsening, sources and receivers on the current GPU):

* ``predict(m, session)`` -> d_pred (Ns x Nr), the predicted data of Sec. 2.2.  Its
  vector-Jacobian product is J^T w (msfv_jtvec) and its Jacobian-vector product, for
  forward-mode AD, is J v (msfv_jvec); J is the sensitivity of Sec. 4.3 through the
  model-dependent prolongation dP/dm (Sec. 4.5).
* ``misfit(m, d_obs, session)`` -> phi = 1/2 ||d_pred - d_obs||^2 (Sec. 4.1), with the
  gradient from the adjoint kernels (msfv_adjoint).

Every step runs in the library's CUDA kernels; this module only marshals tensors and
keeps the linearisation point consistent.  The derivative calls of a Session refer to
the m of its last forward, so a backward whose forward was superseded by a later forward
on the same session first runs the forward again at its own m.  Whether the session
stores the local factors or recomputes them in every derivative call is chosen by its
factor_mode (and HBM budget) at construction.
"""
from __future__ import annotations

import torch

from . import msfv as _msfv


def _relinearise(session, m, version):
    if session.version != version:
        session.forward(m)


class _Predict(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, session):
        d = session.forward(m.detach().contiguous())
        ctx.session = session
        ctx.version = session.version
        ctx.save_for_backward(m)
        ctx.save_for_forward(m)
        return d

    @staticmethod
    def backward(ctx, gd):
        (m,) = ctx.saved_tensors
        s = ctx.session
        _relinearise(s, m.detach().contiguous(), ctx.version)
        ctx.version = s.version
        return s.jtvec(gd.detach().to(torch.float64).contiguous()), None

    @staticmethod
    def jvp(ctx, dm, _session_tangent):
        s = ctx.session
        m = ctx.saved_tensors[0] if ctx.saved_tensors else None
        if m is not None:
            _relinearise(s, m.detach().contiguous(), ctx.version)
        return s.jvec(dm.detach().to(torch.float64).contiguous())


class _Misfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, d_obs, session):
        d = session.forward(m.detach().contiguous())
        dobs = d_obs.detach().to(torch.float64).contiguous()
        r = torch.empty_like(d)
        phi = _msfv.misfit_static(d, dobs, r=r)
        ctx.session = session
        ctx.version = session.version
        ctx.save_for_backward(m, dobs, r)
        return phi

    @staticmethod
    def backward(ctx, gphi):
        m, dobs, r = ctx.saved_tensors
        s = ctx.session
        _relinearise(s, m.detach().contiguous(), ctx.version)
        ctx.version = s.version
        _, g = s.adjoint(dobs, want_phi=False)
        gm = g * gphi if ctx.needs_input_grad[0] else None
        gobs = -r * gphi if ctx.needs_input_grad[1] else None
        return gm, gobs, None


def predict(m: torch.Tensor, session) -> torch.Tensor:
    """Predicted data d_pred(m) (Ns x Nr) with J^T / J v derivatives."""
    return _Predict.apply(m, session)


def misfit(m: torch.Tensor, d_obs: torch.Tensor, session) -> torch.Tensor:
    """phi(m) = 1/2 ||d_pred(m) - d_obs||^2 with the adjoint-kernel gradient."""
    return _Misfit.apply(m, d_obs, session)


class MSFVData(torch.nn.Module):
    """m -> d_pred as a module (the Session is created once for the problem)."""

    def __init__(self, prob, factor_mode: int = 0, hbm_budget_bytes: int = 0):
        super().__init__()
        self.session = _msfv.Session(prob, factor_mode=factor_mode,
                                     hbm_budget_bytes=hbm_budget_bytes)

    def forward(self, m):
        return predict(m, self.session)
