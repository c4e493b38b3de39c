"""Oracle of the Gauss-Newton-CG inversion step (Sec. 5).  TEST INFRASTRUCTURE ONLY.

Plain numpy/scipy, written from the definitions:

* regulariser R(m) = alpha/2 sum over interior faces f (cells x, y) of
  w_f ((m - m_ref)_y - (m - m_ref)_x)^2 with w_f = area_f / distance_f (the diffusion
  penalty of Sec. 5; the paper leaves its discretisation open), and its Hessian
  alpha K with K the weighted cell Laplacian, assembled as a sparse matrix L^T W L
  from the face-difference operator L;
* one Gauss-Newton step: gradient g = J^T r + alpha K (m - m_ref), conjugate gradients
  on (J^T J + alpha K) x = -g from x = 0 (products through the oracle's jvec / jtvec),
  then m <- clip(m + s x) with s = 1, 1/2, ... until the Armijo condition
  Phi(m + s x) <= Phi(m) + 1e-4 s g.x holds.

Pins: tests/test_oracle_pins.py (closed-form R of a linear field, symmetry and the
constant null vector of K, consistency of R and K, CG against a dense solve).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def face_difference(n):
    """Sparse L (faces x cells): row f = e_y - e_x for the face between cells x < y, with
    the faces of axis 0 first, then axis 1, then axis 2; and the weights w_f."""
    n = tuple(int(v) for v in n)
    N = int(np.prod(n))
    idx = np.arange(N).reshape(n[::-1])          # numpy axes reversed: axis 0 fastest
    rows, cols, vals, w = [], [], [], []
    f = 0
    for a in range(len(n)):
        ax = len(n) - 1 - a
        lo = np.take(idx, np.arange(n[a] - 1), axis=ax).ravel()
        hi = np.take(idx, np.arange(1, n[a]), axis=ax).ravel()
        k = lo.size
        fr = np.arange(f, f + k)
        rows += [fr, fr]
        cols += [hi, lo]
        vals += [np.ones(k), -np.ones(k)]
        area = 1.0
        for b in range(len(n)):
            if b != a:
                area /= n[b]
        w.append(np.full(k, area * n[a]))        # area / distance, distance = 1/n[a]
        f += k
    L = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(f, N))
    return L, np.concatenate(w)


def reg_matrix(n):
    """K = L^T W L."""
    L, w = face_difference(n)
    return (L.T @ sp.diags(w) @ L).tocsr()


def reg_value(n, m, m_ref=None, alpha=1.0):
    """alpha/2 sum_f w_f (L (m - m_ref))_f^2, summed face by face."""
    L, w = face_difference(n)
    x = m - (m_ref if m_ref is not None else 0.0)
    dl = L @ x
    return 0.5 * alpha * float(np.sum(w * dl * dl))


def gn_step(orc, m, d_obs, alpha, m_ref=None, cg_iters=10, cg_tol=1e-2, max_backtracks=8,
            bounds=(-10.0, 10.0)):
    """One Gauss-Newton-CG step of the regularised misfit; returns (m_new, stats)."""
    n = orc.prob.n
    K = reg_matrix(n)
    ref = m_ref if m_ref is not None else np.zeros_like(m)

    def objective(mm):
        st = orc.forward(mm)
        r = st['d'] - d_obs
        return st, 0.5 * float(np.sum(r * r)), reg_value(n, mm, ref, alpha)

    st0, phid0, phir0 = objective(m)
    r0 = st0['d'] - d_obs
    g = orc.jtvec(st0, r0) + alpha * (K @ (m - ref))
    x = np.zeros_like(m)
    res = -g
    p = res.copy()
    rr = float(res @ res)
    gnorm = np.sqrt(rr)
    it, rel = 0, (1.0 if gnorm > 0 else 0.0)
    while it < cg_iters and rr > 0:
        q = orc.jtvec(st0, orc.jvec(st0, p)) + alpha * (K @ p)
        pq = float(p @ q)
        if not pq > 0:
            break
        a = rr / pq
        x = x + a * p
        res = res - a * q
        rr1 = float(res @ res)
        it += 1
        rel = np.sqrt(rr1) / gnorm
        if rel <= cg_tol:
            break
        p = res + (rr1 / rr) * p
        rr = rr1
    slope = float(g @ x)
    phi0 = phid0 + phir0
    step = 1.0
    for bt in range(max_backtracks + 1):
        mt = np.clip(m + step * x, bounds[0], bounds[1])
        _, phid1, phir1 = objective(mt)
        if phid1 + phir1 <= phi0 + 1e-4 * step * slope:
            return mt, dict(phi_d0=phid0, phi_r0=phir0, phi_d1=phid1, phi_r1=phir1,
                            grad_norm=gnorm, cg_iters=it, cg_rel_res=rel, step=step,
                            backtracks=bt, x=x)
        step *= 0.5
    return m.copy(), dict(phi_d0=phid0, phi_r0=phir0, phi_d1=phid0, phi_r1=phir0,
                          grad_norm=gnorm, cg_iters=it, cg_rel_res=rel, step=0.0,
                          backtracks=max_backtracks, x=x)
