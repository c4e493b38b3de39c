"""Gauss-Newton-CG inversion driver (Sec. 5) on top of msfv_gn_step.

Each iteration solves (J^T J + alpha K) dm = -grad by conjugate gradients with the
library's J v / J^T w kernels and takes an Armijo-backtracked, bound-clipped step; all of
it runs inside the library.  This module only loops and records the history.
"""
from __future__ import annotations


def gauss_newton(session, m, d_obs, iters: int = 5, alpha: float = 1e-8, m_ref=None,
                 cg_iters: int = 10, cg_tol: float = 1e-2, max_backtracks: int = 8,
                 bounds=(-10.0, 10.0)):
    """Run `iters` Gauss-Newton iterations from m (updated in place).  Returns the list of
    per-iteration statistics (misfit and regulariser before / after, CG iterations,
    accepted step)."""
    hist = []
    for _ in range(iters):
        st = session.gn_step(m, d_obs, alpha, m_ref=m_ref, cg_iters=cg_iters, cg_tol=cg_tol,
                             max_backtracks=max_backtracks, bounds=bounds)
        hist.append(st)
        if st["step"] == 0.0:
            break
    return hist
