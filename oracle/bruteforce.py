"""Dense brute-force MSFV forward map for tiny meshes, differentiable by complex step.

TEST INFRASTRUCTURE ONLY (pins the oracle; shares no code with it).

It works from the definitions with a different organisation than the oracle:
instead of one local solve per entity it forms, for each level k = 1..d, the
global "tangential" operator of all cells with exactly k off-vertex axes and
solves one dense system for all basis functions at once (Sec. 3.2,
Eq. multiscaleBasis_step3 -- the block-diagonal structure over entities is not
used).  Then P, A_c = R A P, the pinned reduced solve and the data follow densely
(Sec. 3.1, Eq. fwdProbRed).  All arithmetic is written so that a complex model
m + i*eps*v flows through analytically (exp, harmonic means and dense solves are
analytic), which gives J v = Im(d(m + i eps v)) / eps to machine precision with no
derivative code at all.
"""
from __future__ import annotations

import numpy as np


def _coords(n):
    N = int(np.prod(n))
    out = np.zeros((N, len(n)), dtype=np.int64)
    rem = np.arange(N)
    for a, v in enumerate(n):
        out[:, a] = rem % v
        rem //= v
    return out


def forward_dense(m, n, c, src_pos, src_neg, src_amp, rec, source_bases=False, oversample=0):
    """Predicted data (Ns, Nr) for model m (real or complex), dense linear algebra.

    source_bases: also solve, level by level, the tangential systems with the source
    as forcing and zero vertex values (Sec. 3.2, source bases) and add that field
    with coefficient one, the reduced right-hand side becoming R (q - A C).

    oversample = w > 0 (Sec. 6 names oversampling without a construction; the reading
    is the oracle's): on the levels below d every piece of the level is solved on its
    own, on the cells that share its off-vertex intervals and lie within w of its
    vertex coordinates.  That system is cut out of the dense fine operator A: the rows
    and columns of those cells, with the flux across the sides normal to the piece
    taken off the diagonal; every neighbour across a tangential end contributes the
    already known basis row of its projection onto the piece's vertex coordinates.
    All Nc basis columns are solved at once, so no corner bookkeeping is needed."""
    n = tuple(int(v) for v in n)
    d = len(n)
    N = int(np.prod(n))
    X = _coords(n)
    stride = [int(np.prod(n[:a])) for a in range(d)]
    sig = np.exp(m)
    dt = np.result_type(sig.dtype, np.float64)
    # fine operator, face by face
    A = np.zeros((N, N), dtype=dt)
    Tface = {}
    for a in range(d):
        area = 1.0
        for b in range(d):
            if b != a:
                area *= 1.0 / n[b]
        geo = area * n[a]
        for x in range(N):
            if X[x, a] + 1 < n[a]:
                y = x + stride[a]
                t = geo * 2.0 * sig[x] * sig[y] / (sig[x] + sig[y])
                Tface[(x, y)] = t
                Tface[(y, x)] = t
                A[x, x] += t
                A[y, y] += t
                A[x, y] -= t
                A[y, x] -= t
    half = c // 2
    isvert = (X - half) % c == 0          # per axis: coordinate is a vertex coordinate
    level = (~isvert).sum(axis=1)         # number of off-vertex axes
    nc = tuple(v // c for v in n)
    Nc = int(np.prod(nc))
    cstride = [int(np.prod(nc[:a])) for a in range(d)]
    Ns = len(src_pos)
    Qm = np.zeros((N, Ns))
    for j in range(Ns):
        Qm[src_pos[j], j] += src_amp[j]
        Qm[src_neg[j], j] -= src_amp[j]
    Phi = np.zeros((N, Nc), dtype=dt)
    Csrc = np.zeros((N, Ns), dtype=dt)
    for x in np.nonzero(level == 0)[0]:
        J = sum(((X[x, a] - half) // c) * cstride[a] for a in range(d))
        Phi[x, J] = 1.0
    for k in range(1, d + 1):
        rows = np.nonzero(level == k)[0]
        if len(rows) == 0:
            continue
        if oversample and k < d:
            _oversampled_level(A, Tface, Phi, X, rows, isvert, n, c, stride, oversample)
            continue
        M = np.zeros((len(rows), N), dtype=dt)
        for r, x in enumerate(rows):
            for a in range(d):
                if isvert[x, a]:
                    continue                  # only fluxes along off-vertex axes
                for s in (-1, 1):
                    ca = X[x, a] + s
                    if 0 <= ca < n[a]:
                        y = x + s * stride[a]
                        t = Tface[(x, y)]
                        M[r, x] += t
                        M[r, y] -= t
        known = np.nonzero(level < k)[0]
        rhs = -M[:, known] @ Phi[known]
        Phi[rows] = np.linalg.solve(M[:, rows], rhs)
        if source_bases:
            Csrc[rows] = np.linalg.solve(M[:, rows], Qm[rows] - M[:, known] @ Csrc[known])
    # restriction, coarse operator, pinned solve
    R = np.zeros((Nc, N))
    for x in range(N):
        I = sum((X[x, a] // c) * cstride[a] for a in range(d))
        R[I, x] = 1.0
    Ac = R @ A @ Phi
    out = np.zeros((Ns, len(rec)), dtype=dt)
    for j in range(Ns):
        b = R @ (Qm[:, j] - A @ Csrc[:, j])
        t = np.zeros(Nc, dtype=dt)
        t[1:] = np.linalg.solve(Ac[1:, 1:], b[1:])
        u = Phi @ t + Csrc[:, j]
        out[j] = u[np.asarray(rec)]
    return out, Phi, Ac


def _oversampled_level(A, Tface, Phi, X, rows, isvert, n, c, stride, w):
    """Fill Phi on the cells `rows` of one level, piece by piece, by oversampled solves."""
    d = len(n)
    half = c // 2
    N = A.shape[0]
    interval = (X - half) // c            # per axis: which open interval (off-vertex axes)
    pieces = {}
    for x in rows:
        key = tuple(int(X[x, a]) if isvert[x, a] else ('I', int(interval[x, a]))
                    for a in range(d))
        pieces.setdefault(key, []).append(int(x))
    for key, own in pieces.items():
        x0 = own[0]
        vert = [a for a in range(d) if isvert[x0, a]]
        offv = [a for a in range(d) if not isvert[x0, a]]
        sel = np.ones(N, dtype=bool)
        for a in offv:
            sel &= (~isvert[:, a]) & (interval[:, a] == interval[x0, a])
        for b in vert:
            sel &= np.abs(X[:, b] - X[x0, b]) <= w
        box = np.nonzero(sel)[0]
        pos = {int(y): i for i, y in enumerate(box)}
        M = A[np.ix_(box, box)].copy()
        rhs = np.zeros((len(box), Phi.shape[1]), dtype=Phi.dtype)
        for i, x in enumerate(box):
            for a in range(d):
                for s in (-1, 1):
                    ca = X[x, a] + s
                    if not 0 <= ca < n[a]:
                        continue
                    y = int(x + s * stride[a])
                    if y in pos:
                        continue
                    t = Tface[(int(x), y)]
                    if a in vert:
                        M[i, i] -= t                  # normal side of the box: no flux
                    else:
                        yp = y - sum((X[y, b] - X[x0, b]) * stride[b] for b in vert)
                        rhs[i] += t * Phi[yp]         # Dirichlet value at the projection
        sol = np.linalg.solve(M, rhs)
        for x in own:
            Phi[x] = sol[pos[x]]


def data(m, prob):
    d, _, _ = forward_dense(m, prob.n, prob.coarsen, prob.src_pos, prob.src_neg,
                            prob.src_amp, prob.rec_cell,
                            source_bases=bool(getattr(prob, 'source_bases', False)),
                            oversample=int(getattr(prob, 'oversample', 0)))
    return d


def jvec_complex_step(m, prob, v, eps=1e-30):
    """J v by complex step: Im(d(m + i eps v)) / eps."""
    mc = np.asarray(m, dtype=np.complex128) + 1j * eps * np.asarray(v)
    return np.imag(data(mc, prob)) / eps


def misfit_gradient_complex_step(m, prob, d_obs, eps=1e-30):
    """Gradient of 1/2 ||d(m) - d_obs||^2, one complex-step evaluation per cell."""
    N = len(m)
    r = np.real(data(np.asarray(m, dtype=np.complex128), prob)) - d_obs
    g = np.zeros(N)
    for k in range(N):
        e = np.zeros(N)
        e[k] = 1.0
        g[k] = np.sum(r * jvec_complex_step(m, prob, e, eps))
    return g


# ---------------------------------------------------------------------------
# Nodal Galerkin variant (Sec. 3.1-3.2 with Lagrange boundary data on primal blocks)
# ---------------------------------------------------------------------------

def forward_dense_nodal(m, n, c, src_pos, src_neg, src_amp, rec):
    """Predicted data (Ns, Nr) of the nodal Galerkin multiscale model, dense, written
    cell by cell: A = sum_c sigma_c K_c where K_c couples the two ends of each of the
    cell's 2^(d-1) d edges with weight (area / length) / 2^(d-1).  All block-interior
    nodes are solved in one dense system at once; the other nodes carry multilinear
    hats.  Complex m flows through (complex-step derivatives)."""
    n = tuple(int(v) for v in n)
    d = len(n)
    nn = tuple(v + 1 for v in n)
    Nn = int(np.prod(nn))
    sn = [int(np.prod(nn[:a])) for a in range(d)]
    Xc = _coords(n)
    sig = np.exp(m)
    dt = np.result_type(sig.dtype, np.float64)
    A = np.zeros((Nn, Nn), dtype=dt)
    h = [1.0 / v for v in n]
    for cell in range(len(sig)):
        base = sum(Xc[cell, a] * sn[a] for a in range(d))
        for a in range(d):
            geo = np.prod([h[b] for b in range(d) if b != a]) / h[a] / 2 ** (d - 1)
            others = [b for b in range(d) if b != a]
            for offs in np.ndindex(*([2] * len(others))):
                lo = base + sum(o * sn[b] for b, o in zip(others, offs))
                hi = lo + sn[a]
                wgt = geo * sig[cell]
                A[lo, lo] += wgt
                A[hi, hi] += wgt
                A[lo, hi] -= wgt
                A[hi, lo] -= wgt
    Xn = _coords(nn)
    ncn = tuple(v // c + 1 for v in n)
    Ncn = int(np.prod(ncn))
    scn = [int(np.prod(ncn[:a])) for a in range(d)]
    # hats everywhere, then the interior nodes of all blocks replaced by one solve
    S = np.ones((Nn, Ncn), dtype=dt)
    for J in range(Ncn):
        Jc = [(J // scn[a]) % ncn[a] for a in range(d)]
        for a in range(d):
            S[:, J] *= np.maximum(0.0, 1.0 - np.abs(Xn[:, a] - c * Jc[a]) / c)
    inner = np.all(Xn % c != 0, axis=1) if c > 1 else np.zeros(Nn, dtype=bool)
    if inner.any():
        I = np.nonzero(inner)[0]
        O = np.nonzero(~inner)[0]
        S[I] = np.linalg.solve(A[np.ix_(I, I)], -A[np.ix_(I, O)] @ S[O])
    Ak = S.T @ A @ S
    Ns = len(src_pos)
    out = np.zeros((Ns, len(rec)), dtype=dt)
    for j in range(Ns):
        q = np.zeros(Nn)
        q[src_pos[j]] += src_amp[j]
        q[src_neg[j]] -= src_amp[j]
        b = S.T @ q
        t = np.zeros(Ncn, dtype=dt)
        t[1:] = np.linalg.solve(Ak[1:, 1:], b[1:])
        out[j] = (S @ t)[np.asarray(rec)]
    return out, S, Ak, A


def data_nodal(m, prob):
    d, _, _, _ = forward_dense_nodal(m, prob.n, prob.coarsen, prob.src_pos, prob.src_neg,
                                     prob.src_amp, prob.rec_cell)
    return d


def jvec_complex_step_nodal(m, prob, v, eps=1e-30):
    mc = np.asarray(m, dtype=np.complex128) + 1j * eps * np.asarray(v)
    return np.imag(data_nodal(mc, prob)) / eps


def misfit_gradient_complex_step_nodal(m, prob, d_obs, eps=1e-30):
    N = len(m)
    r = np.real(data_nodal(np.asarray(m, dtype=np.complex128), prob)) - d_obs
    g = np.zeros(N)
    for k in range(N):
        e = np.zeros(N)
        e[k] = 1.0
        g[k] = np.sum(r * jvec_complex_step_nodal(m, prob, e, eps))
    return g
