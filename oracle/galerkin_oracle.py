"""Plain FP64 CPU oracle of the paper's own multiscale variant: a nodal discretisation,
Lagrange boundary data on the primal coarse blocks, the Galerkin reduced operator
A_k = S^T A S, and the sensitivities of Eq. sensred including the X_k term.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU legs of ``bench.py``; never by the product path.

What is computed (notation of the paper):

(a) sigma = exp(m) per cell.  Nodal operator A(m) = G^T diag(w) G on the (n+1)^d node
    lattice (Sec. 2.2: fields, sources and receivers live on the nodes): every lattice
    edge e along axis a gets w_e = (prod_{b != a} h_b / h_a) * 2^(1-d) * sum of sigma over
    the cells that share the edge (2^(d-1) of them inside the domain, fewer on its
    boundary).  Equivalently A = sum_c sigma_c K_c with one fixed edge Laplacian K_c per
    cell; dA / dm_c = sigma_c K_c.
(b) Basis S_k(m) (Sec. 3.2, Eq. multiscaleBasis_step3 with the piecewise-Lagrange
    construction): coarse nodes are the fine nodes at multiples of c on every axis; on the
    faces, edges and corners of the primal blocks of c^d cells, basis function J is the
    multilinear hat of coarse node J; inside each block it solves the local nodal problem
    A_II x_I = -A_IB x_B (no source).
(c) A_k = S^T A S (Eq. reducedPDE), b_j = S^T q_j; "fix u at one grid point" (Sec. 2.2):
    coarse node 0 (the fine node at the origin) is pinned to zero; t_j = A_k^{-1} b_j,
    U_j = S t_j, d_j = U_j at the receiver nodes (Eq. fwdProbRed).
(d) Sensitivities (Sec. 4.3):  J v = Pr^T ( Y(t) + S dt ),
        dt = A_k^{-1} ( X(q - A U) - S^T (G(U) + A Y(t)) ),
    with Y(t) = grad_m(S t) v (Eq. Y), X(w) = grad_m(S^T w) v (Eq. X), G(U) = grad_m(A U) v.
    Local derivatives per block (Sec. 4.5, Eq. reducedDiscreteMSBasisPDE): the block
    boundary values are Lagrange hats and do not depend on m, so
        d x_I = -A_II^{-1} (dA x)_I .
    J^T w follows by transposition: with z = Pr w, mu = A_k^{-1} S^T z, lambda = S mu,
    y = z - A lambda and r = q - A U,
        J^T w = sum_j [ Y(t_j)^T y_j + Y(mu_j)^T r_j - G(U_j)^T lambda_j ],
    the middle term being the X_k term.  The Y^T terms are local adjoint solves per block
    with seeds collapsed over sources per corner v: sum_j t_j(v) y_j + mu_j(v) r_j.
(e) The fixed-basis Jacobian (Sec. 4.2, Eq. senssimple) keeps only -G(U)^T lambda.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def lattice_coords(nn):
    """Integer coordinates (N, d) of a lattice with nn[a] points per axis, axis 0 fastest."""
    N = int(np.prod(nn))
    idx = np.arange(N, dtype=np.int64)
    out = np.empty((N, len(nn)), dtype=np.int64)
    for a, v in enumerate(nn):
        out[:, a] = idx % v
        idx = idx // v
    return out


def strides(nn):
    s = [1]
    for v in nn[:-1]:
        s.append(s[-1] * v)
    return tuple(s)


class NodalOracle:
    """The nodal Galerkin multiscale oracle for one problem (cells n, coarsening c,
    node-indexed dipoles and receivers)."""

    def __init__(self, prob):
        self.prob = prob
        self.n = tuple(int(v) for v in prob.n)
        self.d = len(self.n)
        self.c = int(prob.coarsen)
        for v in self.n:
            if v % self.c:
                raise ValueError("coarsening factor must divide the mesh size")
        self.nn = tuple(v + 1 for v in self.n)              # nodes per axis
        self.ncn = tuple(v // self.c + 1 for v in self.n)   # coarse nodes per axis
        self.N = int(np.prod(self.n))
        self.Nn = int(np.prod(self.nn))
        self.Ncn = int(np.prod(self.ncn))
        self.sn = strides(self.nn)
        self.sc = strides(self.n)
        self.scn = strides(self.ncn)
        self.Xn = lattice_coords(self.nn)
        self.Xc = lattice_coords(self.n)
        h = [1.0 / v for v in self.n]
        self.geo = [np.prod([h[b] for b in range(self.d) if b != a]) / h[a] for a in range(self.d)]
        self._build_edges()
        self._build_blocks()
        pr = self.prob
        Q = np.zeros((pr.n_src, self.Nn))
        for j in range(pr.n_src):
            Q[j, pr.src_pos[j]] += pr.src_amp[j]
            Q[j, pr.src_neg[j]] -= pr.src_amp[j]
        self.Q = Q
        self.rec = np.asarray(pr.rec_cell, dtype=np.int64)

    # -- step (a): edges, their cells, the nodal operator -------------------------
    def _build_edges(self):
        """Edge list (lower node, axis) and the sparse map E (n_edges x N cells) with
        w = E sigma."""
        lo, ax, rows, cols, vals = [], [], [], [], []
        k0 = 0
        for a in range(self.d):
            xs = np.nonzero(self.Xn[:, a] < self.nn[a] - 1)[0]
            xc = self.Xn[xs]
            others = [b for b in range(self.d) if b != a]
            # cells sharing the edge: coordinate xc[a] along a, xc[b]-1 or xc[b] across
            for offs in itertools.product((0, 1), repeat=len(others)):
                cc = xc.copy()
                ok = np.ones(len(xs), dtype=bool)
                for b, o in zip(others, offs):
                    cc[:, b] = xc[:, b] - o
                    ok &= (cc[:, b] >= 0) & (cc[:, b] < self.n[b])
                cell = sum(cc[:, b] * self.sc[b] for b in range(self.d))
                rows.append(k0 + np.nonzero(ok)[0])
                cols.append(cell[ok])
                vals.append(np.full(int(ok.sum()), self.geo[a] / 2 ** (self.d - 1)))
            lo.append(xs)
            ax.append(np.full(len(xs), a))
            k0 += len(xs)
        self.e_lo = np.concatenate(lo).astype(np.int64)
        self.e_ax = np.concatenate(ax).astype(np.int64)
        self.e_hi = self.e_lo + np.array(self.sn, dtype=np.int64)[self.e_ax]
        ne = k0
        self.E = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(ne, self.N))
        self.G = sp.csr_matrix((np.concatenate([np.ones(ne), -np.ones(ne)]),
                                (np.concatenate([np.arange(ne)] * 2),
                                 np.concatenate([self.e_lo, self.e_hi]))), shape=(ne, self.Nn))

    def operator(self, w):
        """A = G^T diag(w) G for edge weights w."""
        return (self.G.T @ sp.diags(w) @ self.G).tocsr()

    # -- step (b): blocks, Lagrange hats, local solves ------------------------------
    def _build_blocks(self):
        c, d = self.c, self.d
        # Lagrange hats on every node (used on block boundaries): per axis the coarse
        # node at or below (weight 1 - r/c) and the one above (weight r/c)
        K = self.Xn // c
        r = self.Xn - K * c
        rows, cols, vals = [], [], []
        for bits in itertools.product((0, 1), repeat=d):
            wt = np.ones(self.Nn)
            J = np.zeros(self.Nn, dtype=np.int64)
            for a in range(d):
                wa = (r[:, a] / c) if bits[a] else (1.0 - r[:, a] / c)
                wt = wt * wa
                J += np.minimum(K[:, a] + bits[a], self.ncn[a] - 1) * self.scn[a]
            keep = wt != 0
            rows.append(np.nonzero(keep)[0])
            cols.append(J[keep])
            vals.append(wt[keep])
        rows, cols, vals = np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)
        self.Hat = sp.csr_matrix((vals, (rows, cols)), shape=(self.Nn, self.Ncn))
        self.interior = np.all(self.Xn % c != 0, axis=1) if c > 1 else np.zeros(self.Nn, bool)
        # blocks: interior nodes, closure nodes, corner coarse nodes
        self.blocks = []
        if c == 1:
            return
        nb = [v // c for v in self.n]
        for K in itertools.product(*[range(v) for v in nb]):
            rng = [np.arange(K[a] * c, K[a] * c + c + 1) for a in range(d)]
            grids = np.meshgrid(*rng[::-1], indexing='ij')
            nodes = np.zeros(grids[0].size, dtype=np.int64)
            for kk, gg in enumerate(grids):
                a = d - 1 - kk
                nodes += gg.reshape(-1) * self.sn[a]
            inner = nodes[self.interior[nodes]]
            corners = []
            for bits in itertools.product((0, 1), repeat=d):
                corners.append(sum((K[a] + bits[a]) * self.scn[a] for a in range(d)))
            self.blocks.append(dict(nodes=nodes, inner=inner,
                                    bnd=nodes[~self.interior[nodes]],
                                    corners=np.array(corners, dtype=np.int64)))

    def basis(self, A):
        """S (Nn x Ncn): hats on block boundaries, local solves inside the blocks; also
        the per-block factorisations of A_II."""
        S = self.Hat.tolil(copy=True)
        lus = []
        for B in self.blocks:
            I, Bn, C = B['inner'], B['bnd'], B['corners']
            AII = A[I][:, I].tocsc()
            AIB = A[I][:, Bn]
            lu = spla.splu(AII)
            xb = self.Hat[Bn][:, C].toarray()
            xi = lu.solve(np.asarray(-(AIB @ xb)))
            for k, J in enumerate(C):
                S[I, J] = xi[:, k].reshape(-1, 1)
            lus.append(lu)
        return S.tocsr(), lus

    # -- step (c): reduced solve --------------------------------------------------
    def forward(self, m):
        m = np.asarray(m, dtype=np.float64)
        sig = np.exp(m)
        w = self.E @ sig
        A = self.operator(w)
        S, lus = self.basis(A)
        Ak = (S.T @ A @ S).tocsr()
        lu_k = spla.splu(Ak[1:, 1:].tocsc())
        Ns = self.prob.n_src
        b = (S.T @ self.Q.T).T
        t = np.zeros((Ns, self.Ncn))
        for j in range(Ns):
            t[j, 1:] = lu_k.solve(b[j, 1:])
        U = (S @ t.T).T
        return dict(m=m, sig=sig, w=w, A=A, S=S, lus=lus, Ak=Ak, lu_k=lu_k, t=t, U=U,
                    d=U[:, self.rec].copy())

    def coarse_solve(self, st, rhs):
        out = np.zeros(self.Ncn)
        out[1:] = st['lu_k'].solve(np.asarray(rhs[1:], dtype=np.float64))
        return out

    # -- step (d): derivatives ----------------------------------------------------
    def dweights(self, st, v):
        """Directional derivative of the edge weights along v (dsigma = sigma v)."""
        return self.E @ (st['sig'] * np.asarray(v))

    def dbasis(self, st, dA):
        """dS: zero on block boundaries, -A_II^{-1} (dA S)_I inside each block."""
        S = st['S']
        dS = sp.lil_matrix((self.Nn, self.Ncn))
        for B, lu in zip(self.blocks, st['lus']):
            I, Nd, C = B['inner'], B['nodes'], B['corners']
            x = S[Nd][:, C]
            rhs = -(dA[I][:, Nd] @ x).toarray()
            dx = lu.solve(np.asarray(rhs))
            for k, J in enumerate(C):
                dS[I, J] = dx[:, k].reshape(-1, 1)
        return dS.tocsr()

    def jvec(self, st, v, with_x=True):
        """J v (Ns, Nr).  with_x=False leaves out the X_k term (for the pins)."""
        dA = self.operator(self.dweights(st, v))
        A, S = st['A'], st['S']
        dS = self.dbasis(st, dA)
        out = np.zeros((self.prob.n_src, len(self.rec)))
        for j in range(self.prob.n_src):
            tj = st['t'][j]
            # d(S^T A S) t = d(S^T q):  dt = A_k^{-1} (X(q - A U) - S^T (dA U + A dS t))
            rhs = -(S.T @ (dA @ st['U'][j] + A @ (dS @ tj)))
            if with_x:
                rhs = rhs + dS.T @ (self.Q[j] - A @ st['U'][j])
            dt = self.coarse_solve(st, rhs)
            du = dS @ tj + S @ dt
            out[j] = du[self.rec]
        return out

    def _edge_to_cells(self, st, gw):
        """Chain rule from edge weights to m: dw_e / dm_c = E_ec sigma_c."""
        return (self.E.T @ gw) * st['sig']

    def jtvec(self, st, w):
        """J^T w (N cells,)."""
        w = np.asarray(w, dtype=np.float64)
        Ns = self.prob.n_src
        A, S, t, U = st['A'], st['S'], st['t'], st['U']
        Z = np.zeros((Ns, self.Nn))
        for j in range(Ns):
            np.add.at(Z[j], self.rec, w[j])
        mu = np.array([self.coarse_solve(st, S.T @ Z[j]) for j in range(Ns)])
        Lam = (S @ mu.T).T
        Y = Z - (A @ Lam.T).T
        Rf = self.Q - (A @ U.T).T
        # -G(U)^T lambda: -sum_j (lambda_a - lambda_b)(U_a - U_b) per edge
        gw = -np.sum((Lam[:, self.e_lo] - Lam[:, self.e_hi]) * (U[:, self.e_lo] - U[:, self.e_hi]),
                     axis=0)
        # Y(t)^T y + Y(mu)^T r (the second is the X_k term), block by block
        for B, lu in zip(self.blocks, st['lus']):
            I, Nd, C = B['inner'], B['nodes'], B['corners']
            seeds = Y[:, I].T @ t[:, C] + Rf[:, I].T @ mu[:, C]          # (n_I, 2^d)
            eta = np.asarray(lu.solve(np.asarray(seeds)))
            # -eta^T dA x = -sum_e dw_e (eta_a - eta_b)(x_a - x_b) over the block's edges
            full = np.zeros((self.Nn, len(C)))
            full[I] = eta
            x = S[:, C].toarray()
            inside = np.isin(self.e_lo, Nd) & np.isin(self.e_hi, Nd)
            touch = inside & (np.isin(self.e_lo, I) | np.isin(self.e_hi, I))
            el, eh = self.e_lo[touch], self.e_hi[touch]
            gw[touch] -= np.sum((full[el] - full[eh]) * (x[el] - x[eh]), axis=1)
        return self._edge_to_cells(st, gw)

    def misfit_gradient(self, st, d_obs):
        r = st['d'] - np.asarray(d_obs)
        return 0.5 * float(np.sum(r * r)), self.jtvec(st, r)

    def jtvec_fixed_basis(self, st, w):
        """Eq. senssimple: only -G(U)^T lambda."""
        w = np.asarray(w, dtype=np.float64)
        Ns = self.prob.n_src
        S, U = st['S'], st['U']
        Z = np.zeros((Ns, self.Nn))
        for j in range(Ns):
            np.add.at(Z[j], self.rec, w[j])
        mu = np.array([self.coarse_solve(st, S.T @ Z[j]) for j in range(Ns)])
        Lam = (S @ mu.T).T
        gw = -np.sum((Lam[:, self.e_lo] - Lam[:, self.e_hi]) * (U[:, self.e_lo] - U[:, self.e_hi]),
                     axis=0)
        return self._edge_to_cells(st, gw)
