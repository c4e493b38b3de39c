"""Plain FP64 CPU oracle of the MSFV reduced solve and its derivative.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU legs of ``bench.py``; never by the product path.

What is computed, step by step (notation of the paper where it has one):

(a) sigma = exp(m) (Sec. 2.1, the parametrisation below Eq. DCR); face
    transmissibilities T_f = harmonic mean of the two cell conductivities times
    (face area / cell distance); no flux through the outer boundary (Neumann,
    Eq. DCR second line).  The fine operator is A(m) = sum_f T_f (e_a-e_b)(e_a-e_b)^T,
    i.e. the cell-centred finite-volume form of -div(sigma grad u).
(b) Multiscale basis by local solves (Sec. 3.2, Eq. multiscaleBasis_step3): the
    fine mesh is cut along the dual-coarse grid whose vertices are the coarse-cell
    centres.  Every piece ("entity") of that grid -- dual edges (1D), dual faces
    (2D, in 3D) and dual-cell interiors -- gets its own local problem, solved with
    Dirichlet data from its lower-dimensional boundary and no source.  The local
    operator keeps only the fluxes tangential to the entity (reduced boundary
    conditions).  One right-hand side per corner vertex of the entity.
(c) Prolongation P (the basis S_k(m) of Sec. 3.1): column J holds basis function
    phi_J, assembled from the entity solutions.
(d) Coarse operator A_c = R A P with the finite-volume restriction R (sum over
    each primal coarse cell): the projection of Eq. reducedPDE with R in place of
    S_k^T on the left.
(e) Reduced solve with the gauge "fix one value" (Sec. 2.2): coarse unknown 0 is
    pinned to zero (row and column 0 removed); u_j = P t_j; data = point samples
    of u_j at the receiver cells (the receiver matrix of Eq. forwardProbFine).
(f) Sensitivities of the adaptive reduced model (Sec. 4.3, Eq. sensred):
    J = Pr^T ( Y(t) + P dt/dm ),  dt/dm = -A_c^{-1} R ( G(u) + A Y(t) ),
    with G(u) = grad_m(A u) (Eq. G) and Y(t) = grad_m(P t) (Eq. Y).  The X term of
    the paper's derivation vanishes because R does not depend on m.  Y is formed
    from local derivative solves (Sec. 4.5, Eq. reducedDiscreteMSBasisPDE):
    d phi_E = -L_E^{-1} ( dL_E phi_E + dB_E phi_dE + B_E d phi_dE ), where the
    boundary values phi_dE themselves depend on m and are differentiated first
    (edges -> faces -> interiors).  J^T w runs the same chain in reverse.

Source bases (Sec. 3.2, the second construction listed there), when the problem asks
for them: every entity also solves its local problem once per source j with the
restricted source q_j as forcing and zero data on the coarse vertices; the boundary
data of a face or interior are the source-basis values of its lower-dimensional
boundary (edges -> faces -> interiors, as for the vertex bases).  The assembled
source basis C_j enters with coefficient one: u_j = P t_j + C_j, and the reduced
system keeps the finite-volume restriction, A_c t_j = R (q_j - A C_j).  Its
sensitivity adds the chain d C_j (same local operators, no new matrices):
J = Pr^T ( Y(t) + dC + P dt/dm ),  dt/dm = -A_c^{-1} R ( G(u) + A Y(t) + A dC ).

Oversampling (with width w > 0; Sec. 6 names it as a way to lessen the effect of the
local boundary conditions on the basis but gives no construction, so this reading is
ours): every dual edge and dual face solves its local problem on a box widened by w
cells on both sides along its normal (vertex) axes, clipped to the mesh.  Inside that
box all fluxes count, tangential and normal; across its normal sides none passes;
across its tangential ends the Dirichlet value of a cell is the basis value already
computed at the cell's projection onto the entity's own vertex planes (vertex values for
an edge, edge values for a face).  Only the values on the entity's own cells enter P, so
each cell still takes its basis values from exactly one local problem and the basis
stays conforming; the dual-cell interiors are unchanged.  w = 0 is the plain method.
Source bases are not defined with oversampling.

Readings of the paper where it is silent or garbled are listed in the design
notes of the repository; the ones that matter here: cell-centred FV with
harmonic face averages, coarse vertex at fine index c*I + floor(c/2) per axis,
partial dual cells at the outer boundary keep the no-flux condition there, and
the gauge pins coarse unknown 0.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


# ---------------------------------------------------------------------------
# Step (a): conductivity and face transmissibilities
# ---------------------------------------------------------------------------

def strides_of(n):
    s = [1]
    for v in n[:-1]:
        s.append(s[-1] * v)
    return tuple(s)


def cell_coords(n):
    """Integer coordinates of every cell, shape (N, d), axis 0 fastest."""
    N = int(np.prod(n))
    idx = np.arange(N, dtype=np.int64)
    out = np.empty((N, len(n)), dtype=np.int64)
    for a, v in enumerate(n):
        out[:, a] = idx % v
        idx = idx // v
    return out


def transmissibility(m, n):
    """T[a][x] for the face between cell x and x+e_a (0 where x is on the last layer).

    sigma = exp(m); T = 2 s_x s_y / (s_x + s_y) * (prod_{b != a} h_b) / h_a.
    Returns (T, dT_dmx, dT_dmy): the derivative of T_f with respect to the
    log-conductivity of the lower cell x and of the upper cell y.
    """
    n = tuple(n)
    d = len(n)
    h = [1.0 / v for v in n]
    sig = np.exp(m)
    coords = cell_coords(n)
    st = strides_of(n)
    T, Dx, Dy = [], [], []
    for a in range(d):
        geo = np.prod([h[b] for b in range(d) if b != a]) / h[a]
        has = coords[:, a] < n[a] - 1
        x = np.nonzero(has)[0]
        y = x + st[a]
        sx, sy = sig[x], sig[y]
        Ta = np.zeros(len(m), dtype=sig.dtype)
        dx = np.zeros(len(m), dtype=sig.dtype)
        dy = np.zeros(len(m), dtype=sig.dtype)
        Ta[x] = geo * 2.0 * sx * sy / (sx + sy)
        # d/dm_x of 2 s_x s_y/(s_x+s_y) with ds_x/dm_x = s_x  ->  T * s_y/(s_x+s_y)
        dx[x] = Ta[x] * sy / (sx + sy)
        dy[x] = Ta[x] * sx / (sx + sy)
        T.append(Ta)
        Dx.append(dx)
        Dy.append(dy)
    return T, Dx, Dy


def fine_operator(T, n):
    """A = sum_f T_f (e_x - e_y)(e_x - e_y)^T over all interior faces (sparse CSR)."""
    n = tuple(n)
    N = int(np.prod(n))
    st = strides_of(n)
    coords = cell_coords(n)
    rows, cols, vals = [], [], []
    diag = np.zeros(N, dtype=T[0].dtype)
    for a in range(len(n)):
        x = np.nonzero(coords[:, a] < n[a] - 1)[0]
        y = x + st[a]
        t = T[a][x]
        rows += [x, y]
        cols += [y, x]
        vals += [-t, -t]
        np.add.at(diag, x, t)
        np.add.at(diag, y, t)
    rows.append(np.arange(N))
    cols.append(np.arange(N))
    vals.append(diag)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(N, N))


# ---------------------------------------------------------------------------
# Step (b): the dual-coarse grid and its entities
# ---------------------------------------------------------------------------

def axis_pieces(n_a, c):
    """Split one axis into vertex coordinates and the open intervals between them.

    Coarse vertex K sits at fine coordinate c*K + floor(c/2) (the centre of coarse
    cell K).  Returns a list of pieces in coordinate order:
      ('V', K, pos)                      a vertex coordinate
      ('I', lo, hi, start, length)       an open interval; lo / hi are the coarse
                                         vertices at its ends, None at the outer
                                         boundary (a partial dual cell).
    """
    half = c // 2
    ncoarse = n_a // c
    pieces = []
    if half > 0:
        pieces.append(('I', None, 0, 0, half))
    for K in range(ncoarse):
        pos = c * K + half
        pieces.append(('V', K, pos))
        if K + 1 < ncoarse:
            if c - 1 > 0:
                pieces.append(('I', K, K + 1, pos + 1, c - 1))
        else:
            right = n_a - 1 - pos
            if right > 0:
                pieces.append(('I', K, None, pos + 1, right))
    return pieces


@dataclass
class Entity:
    dim: int                 # number of interval axes
    axes: tuple              # tangential (interval) axes
    cells: np.ndarray        # global cell indices, axis 0 fastest
    corners: np.ndarray      # global coarse-vertex indices of its corner vertices
    # local problem description (filled by Oracle._describe)
    bnd: np.ndarray = None           # boundary cells (Dirichlet data)
    f_axis: np.ndarray = None        # tangential faces touching the entity
    f_idx: np.ndarray = None         # face index (= lower cell)
    f_a: np.ndarray = None           # local index of the entity-side cell
    f_b: np.ndarray = None           # local index of the other cell, -1 if on the boundary
    f_q: np.ndarray = None           # boundary index of the other cell, -1 if inside
    g_ent: np.ndarray = None         # entity id of each boundary cell
    g_loc: np.ndarray = None         # local index of each boundary cell in its entity
    g_pos: np.ndarray = None         # (n_bnd, n_corners) corner position in that entity or -1
    # oversampling: the cells the local problem is solved on (the entity itself unless it
    # is widened), the positions of the entity's own cells among them, and the vertex
    # coordinate of each normal axis (-1 on tangential axes)
    solve_cells: np.ndarray = None
    keep: np.ndarray = None
    centre: tuple = None


class Oracle:
    """The MSFV oracle for one problem (mesh, coarsening, sources, receivers)."""

    def __init__(self, prob):
        self.prob = prob
        self.n = tuple(int(v) for v in prob.n)
        self.d = len(self.n)
        self.c = int(prob.coarsen)
        for v in self.n:
            if v % self.c:
                raise ValueError("coarsening factor must divide the mesh size")
        self.N = int(np.prod(self.n))
        self.nc = tuple(v // self.c for v in self.n)
        self.Nc = int(np.prod(self.nc))
        self.st = strides_of(self.n)
        self.cst = strides_of(self.nc)
        self.source_bases = bool(getattr(prob, 'source_bases', False))
        self.w = int(getattr(prob, 'oversample', 0))
        if self.w < 0:
            raise ValueError("oversampling width must be >= 0")
        if self.w and self.source_bases:
            raise ValueError("source bases are not defined with oversampling")
        self._build_entities()
        self._build_restriction_and_sources()

    # -- geometry ----------------------------------------------------------
    def _build_entities(self):
        per_axis = [axis_pieces(v, self.c) for v in self.n]
        ents = []
        for combo in itertools.product(*per_axis):
            ranges, corner_lists, axes = [], [], []
            for a, pc in enumerate(combo):
                if pc[0] == 'V':
                    ranges.append(np.array([pc[2]]))
                    corner_lists.append([pc[1]])
                else:
                    ranges.append(np.arange(pc[3], pc[3] + pc[4]))
                    corner_lists.append([k for k in (pc[1], pc[2]) if k is not None])
                    axes.append(a)
            cells = self._box_cells(ranges)
            corners = []
            for ks in itertools.product(*corner_lists[::-1]):
                ks = ks[::-1]
                corners.append(sum(ks[a] * self.cst[a] for a in range(self.d)))
            # oversampled box of an edge or face: +-w cells along its normal axes
            centre = tuple(int(pc[2]) if pc[0] == 'V' else -1 for pc in combo)
            solve_cells, keep = cells, np.arange(len(cells))
            if self.w and 0 < len(axes) < self.d:
                wide = [np.arange(max(0, centre[a] - self.w), min(self.n[a], centre[a] + self.w + 1))
                        if centre[a] >= 0 else ranges[a] for a in range(self.d)]
                solve_cells = self._box_cells(wide)
                where = {int(x): i for i, x in enumerate(solve_cells)}
                keep = np.array([where[int(x)] for x in cells], dtype=np.int64)
            ents.append(Entity(dim=len(axes), axes=tuple(axes), cells=cells,
                               corners=np.array(corners, dtype=np.int64),
                               solve_cells=solve_cells, keep=keep, centre=centre))
        ents.sort(key=lambda e: e.dim)
        self.entities = ents
        self.cell2ent = np.full(self.N, -1, dtype=np.int64)
        self.cell2loc = np.full(self.N, -1, dtype=np.int64)
        for eid, e in enumerate(ents):
            self.cell2ent[e.cells] = eid
            self.cell2loc[e.cells] = np.arange(len(e.cells))
        assert (self.cell2ent >= 0).all()
        coords = cell_coords(self.n)
        for e in ents:
            if e.dim > 0:
                self._describe(e, coords)

    def _box_cells(self, ranges):
        """Global indices of the box ranges[0] x ranges[1] (x ranges[2]), axis 0 fastest."""
        grids = np.meshgrid(*ranges[::-1], indexing='ij')
        cells = np.zeros(grids[0].size, dtype=np.int64)
        for k, g in enumerate(grids):
            a = self.d - 1 - k
            cells += g.reshape(-1) * self.st[a]
        return cells

    def _project(self, e, y, coords):
        """Cell y moved onto the entity's vertex planes (its normal coordinates set to
        the entity's vertex coordinates): the source of y's Dirichlet value."""
        for a in range(self.d):
            if e.centre[a] >= 0:
                y = y + (e.centre[a] - coords[y, a]) * self.st[a]
        return int(y)

    def _describe(self, e, coords):
        """Faces, boundary cells and gather indices of one local problem (on e.solve_cells:
        the entity, or its oversampled box).  A face leaving the box along a tangential
        axis couples to a Dirichlet cell; along a normal axis it is dropped (no flux)."""
        loc = {int(x): i for i, x in enumerate(e.solve_cells)}
        fa, fb, fq, fax, fidx, bnd = [], [], [], [], [], {}
        for p, x in enumerate(e.solve_cells):
            for a in range(self.d):
                tangential = a in e.axes
                for sgn in (+1, -1):
                    ca = coords[x, a] + sgn
                    if ca < 0 or ca >= self.n[a]:
                        continue                       # outer boundary: no flux
                    y = int(x + sgn * self.st[a])
                    inside = y in loc
                    if inside and sgn < 0:
                        continue                       # internal faces once
                    if not inside and not tangential:
                        continue                       # normal side of the box: no flux
                    fax.append(a)
                    fidx.append(min(int(x), y))
                    fa.append(p)
                    if inside:
                        fb.append(loc[y])
                        fq.append(-1)
                    else:
                        yb = self._project(e, y, coords)
                        if yb not in bnd:
                            bnd[yb] = len(bnd)
                        fb.append(-1)
                        fq.append(bnd[yb])
        e.f_axis = np.array(fax, dtype=np.int64)
        e.f_idx = np.array(fidx, dtype=np.int64)
        e.f_a = np.array(fa, dtype=np.int64)
        e.f_b = np.array(fb, dtype=np.int64)
        e.f_q = np.array(fq, dtype=np.int64)
        e.bnd = np.array(sorted(bnd, key=bnd.get), dtype=np.int64)
        e.g_ent = self.cell2ent[e.bnd]
        e.g_loc = self.cell2loc[e.bnd]
        e.g_pos = np.full((len(e.bnd), len(e.corners)), -1, dtype=np.int64)
        for q in range(len(e.bnd)):
            other = self.entities[e.g_ent[q]].corners
            for i, v in enumerate(e.corners):
                hit = np.nonzero(other == v)[0]
                if len(hit):
                    e.g_pos[q, i] = hit[0]

    def _build_restriction_and_sources(self):
        coords = cell_coords(self.n)
        cidx = np.zeros(self.N, dtype=np.int64)
        for a in range(self.d):
            cidx += (coords[:, a] // self.c) * self.cst[a]
        self.coarse_of_cell = cidx
        # R: sum over each primal coarse cell
        self.R = sp.csr_matrix((np.ones(self.N), (cidx, np.arange(self.N))),
                               shape=(self.Nc, self.N))
        pr = self.prob
        Ns = pr.n_src
        Q = np.zeros((Ns, self.N))
        for j in range(Ns):
            Q[j, pr.src_pos[j]] += pr.src_amp[j]
            Q[j, pr.src_neg[j]] -= pr.src_amp[j]
        self.Q = Q
        self.rec = np.asarray(pr.rec_cell, dtype=np.int64)

    # -- local problems ------------------------------------------------------
    def local_matrices(self, e, Tface):
        """L_E and B_E of one entity for face values Tface (list per axis).

        (L_E phi_E + B_E phi_bnd)_a = sum over tangential faces (a,b) of
        T_ab (phi_a - phi_b); linear in T, so the same routine gives dL, dB.
        """
        nE, nB = len(e.solve_cells), len(e.bnd)
        t = np.array([Tface[a][i] for a, i in zip(e.f_axis, e.f_idx)],
                     dtype=Tface[0].dtype) if len(e.f_axis) else np.zeros(0)
        inner = e.f_b >= 0
        ai, bi, ti = e.f_a[inner], e.f_b[inner], t[inner]
        ao, qo, to = e.f_a[~inner], e.f_q[~inner], t[~inner]
        rows = np.concatenate([ai, bi, ai, bi, ao])
        cols = np.concatenate([ai, bi, bi, ai, ao])
        vals = np.concatenate([ti, ti, -ti, -ti, to])
        L = sp.csc_matrix((vals, (rows, cols)), shape=(nE, nE))
        B = sp.csr_matrix((-to, (ao, qo)), shape=(nE, nB))
        return L, B

    def gather_boundary(self, e, vals):
        """Values on the boundary cells of e of the basis functions of e's corners."""
        out = np.zeros((len(e.bnd), len(e.corners)), dtype=vals[0].dtype)
        for q in range(len(e.bnd)):
            blk = vals[e.g_ent[q]]
            for i in range(len(e.corners)):
                p = e.g_pos[q, i]
                if p >= 0:
                    out[q, i] = blk[e.g_loc[q], p]
        return out

    def gather_source_boundary(self, e, cvals):
        """Source-basis values (n_bnd, Ns) on the boundary cells of e (zero on vertices)."""
        out = np.zeros((len(e.bnd), self.prob.n_src), dtype=cvals[0].dtype)
        for q in range(len(e.bnd)):
            out[q] = cvals[e.g_ent[q]][e.g_loc[q]]
        return out

    def scatter_source_boundary(self, e, seeds, contrib):
        """Add contrib (n_bnd, Ns) to the source-basis seeds of the boundary entities."""
        for q in range(len(e.bnd)):
            f = e.g_ent[q]
            if self.entities[f].dim == 0:
                continue
            seeds[f][e.g_loc[q]] += contrib[q]

    def scatter_boundary(self, e, seeds, contrib):
        """Add contrib (n_bnd, n_corners) to the seeds of the boundary entities."""
        for q in range(len(e.bnd)):
            f = e.g_ent[q]
            if self.entities[f].dim == 0:
                continue                 # vertex values are fixed: no derivative
            for i in range(len(e.corners)):
                p = e.g_pos[q, i]
                if p >= 0:
                    seeds[f][e.g_loc[q], p] += contrib[q, i]

    # -- forward: steps (a)-(e) ----------------------------------------------
    def forward(self, m):
        """Basis, coarse operator, reduced solve and predicted data for model m."""
        m = np.asarray(m, dtype=np.float64)
        st = {}
        T, Dx, Dy = transmissibility(m, self.n)
        st['m'], st['T'], st['Dx'], st['Dy'] = m, T, Dx, Dy
        Ns = self.prob.n_src
        vals, lus, cvals, fulls = [], [], [], []
        for e in self.entities:
            if e.dim == 0:
                vals.append(np.ones((1, 1)))
                fulls.append(vals[-1])
                lus.append(None)
                cvals.append(np.zeros((1, Ns)))
                continue
            L, B = self.local_matrices(e, T)
            lu = spla.splu(L)
            phib = self.gather_boundary(e, vals)
            rhs = -(B @ phib)
            full = np.asarray(lu.solve(np.asarray(rhs))).reshape(len(e.solve_cells), len(e.corners))
            fulls.append(full)                         # the whole (oversampled) solution
            vals.append(full[e.keep])                  # its values on the entity's cells
            lus.append(lu)
            if self.source_bases:
                # L_E c_E = q_E - B_E c_bnd, one column per source
                cb = self.gather_source_boundary(e, cvals)
                rhs_c = self.Q[:, e.cells].T - B @ cb
                cvals.append(np.asarray(lu.solve(np.asarray(rhs_c))).reshape(len(e.cells), Ns))
            else:
                cvals.append(np.zeros((len(e.cells), Ns)))
        st['vals'], st['lus'], st['cvals'], st['fulls'] = vals, lus, cvals, fulls
        P = self.assemble_P(vals)
        A = fine_operator(T, self.n)
        Ac = (self.R @ A @ P).tocsr()
        lu_c = spla.splu(Ac[1:, 1:].tocsc())
        C = self.assemble_sources(cvals)               # (Ns, N): source bases C_j
        b = (self.R @ (self.Q - (A @ C.T).T).T).T      # (Ns, Nc): R (q_j - A C_j)
        t = np.zeros((Ns, self.Nc))
        for j in range(Ns):
            t[j, 1:] = lu_c.solve(b[j, 1:])
        U = (P @ t.T).T + C                            # (Ns, N): u_j = P t_j + C_j
        st.update(P=P, A=A, Ac=Ac, lu_c=lu_c, t=t, C=C, U=U, d=U[:, self.rec].copy())
        return st

    def assemble_sources(self, cvals):
        """Source bases as fine fields (Ns, N) from the per-entity values."""
        C = np.zeros((self.prob.n_src, self.N), dtype=cvals[0].dtype)
        for e, cv in zip(self.entities, cvals):
            if e.dim > 0:
                C[:, e.cells] = cv.T
        return C

    def assemble_P(self, vals):
        rows = np.concatenate([np.repeat(e.cells, len(e.corners)) for e in self.entities])
        cols = np.concatenate([np.tile(e.corners, len(e.cells)) for e in self.entities])
        data = np.concatenate([v.reshape(-1) for v in vals])
        keep = data != 0
        return sp.csr_matrix((data[keep], (rows[keep], cols[keep])), shape=(self.N, self.Nc))

    def coarse_solve(self, st, rhs, transpose=False):
        """Pinned coarse solve: unknown 0 fixed to zero, equation 0 dropped."""
        out = np.zeros(self.Nc)
        out[1:] = st['lu_c'].solve(np.asarray(rhs[1:], dtype=np.float64),
                                   trans='T' if transpose else 'N')
        return out

    # -- derivative: step (f) --------------------------------------------------
    def dT_of(self, st, v):
        """Directional derivative of the face transmissibilities along v."""
        st_ = self.st
        out = []
        for a in range(self.d):
            da = np.zeros(self.N)
            x = np.nonzero(st['T'][a])[0]
            da[x] = st['Dx'][a][x] * v[x] + st['Dy'][a][x] * v[x + st_[a]]
            out.append(da)
        return out

    def jvec(self, st, v):
        """J v (Ns, Nr): tangent of the predicted data along model direction v."""
        v = np.asarray(v, dtype=np.float64)
        T = st['T']
        dT = self.dT_of(st, v)
        Ns = self.prob.n_src
        dvals, dcvals = [], []
        for e, full, cval, lu in zip(self.entities, st['fulls'], st['cvals'], st['lus']):
            if e.dim == 0:
                dvals.append(np.zeros((1, 1)))
                dcvals.append(np.zeros((1, Ns)))
                continue
            L, B = self.local_matrices(e, T)
            dL, dB = self.local_matrices(e, dT)
            phib = self.gather_boundary(e, st['vals'])
            dphib = self.gather_boundary(e, dvals)
            rhs = -(dL @ full + dB @ phib + B @ dphib)
            dfull = np.asarray(lu.solve(np.asarray(rhs))).reshape(full.shape)
            dvals.append(dfull[e.keep])
            if self.source_bases:
                cb = self.gather_source_boundary(e, st['cvals'])
                dcb = self.gather_source_boundary(e, dcvals)
                rhs_c = -(dL @ cval + dB @ cb + B @ dcb)
                dcvals.append(np.asarray(lu.solve(np.asarray(rhs_c))).reshape(cval.shape))
            else:
                dcvals.append(np.zeros(cval.shape))
        dP = self.assemble_P(dvals)
        dC = self.assemble_sources(dcvals)
        dA = fine_operator(dT, self.n)
        dAc = self.R @ dA @ st['P'] + self.R @ st['A'] @ dP
        out = np.zeros((Ns, len(self.rec)))
        for j in range(Ns):
            tj = st['t'][j]
            # d(R (q - A C)) = -R (dA C + A dC)
            rhs = -(dAc @ tj) - self.R @ (dA @ st['C'][j] + st['A'] @ dC[j])
            dtj = self.coarse_solve(st, rhs)
            du = dP @ tj + st['P'] @ dtj + dC[j]
            out[j] = du[self.rec]
        return out

    def jtvec(self, st, w):
        """J^T w (N,): adjoint of the predicted data map applied to w (Ns, Nr)."""
        w = np.asarray(w, dtype=np.float64)
        Ns = self.prob.n_src
        T, P, A = st['T'], st['P'], st['A']
        Z = np.zeros((Ns, self.N))
        for j in range(Ns):
            np.add.at(Z[j], self.rec, w[j])              # z_j = Pr w_j
        lam_c = np.zeros((Ns, self.Nc))
        for j in range(Ns):
            lam_c[j] = self.coarse_solve(st, P.T @ Z[j], transpose=True)
        Lam = (self.R.T @ lam_c.T).T                      # lambda_j = R^T lambda_c,j
        Y = Z - (A @ Lam.T).T                             # y_j = z_j - A lambda_j
        gT = [np.zeros(self.N) for _ in range(self.d)]
        # G(u)^T lambda: -lambda^T dA u = -sum_f dT_f (l_a - l_b)(u_a - u_b)
        coords = cell_coords(self.n)
        for a in range(self.d):
            x = np.nonzero(coords[:, a] < self.n[a] - 1)[0]
            y = x + self.st[a]
            gT[a][x] -= np.sum((Lam[:, x] - Lam[:, y]) * (st['U'][:, x] - st['U'][:, y]), axis=0)
        # Y(t)^T y: seeds W_v = sum_j t_j(v) y_j on each entity, then reverse sweep
        t = st['t']
        seeds = [None if e.dim == 0 else Y[:, e.cells].T @ t[:, e.corners]
                 for e in self.entities]
        # source bases enter with coefficient one: their seeds are y_j itself
        seeds_c = [None if e.dim == 0 else Y[:, e.cells].T for e in self.entities]
        for eid in range(len(self.entities) - 1, -1, -1):
            e = self.entities[eid]
            if e.dim == 0:
                continue
            full, lu = st['fulls'][eid], st['lus'][eid]
            L, B = self.local_matrices(e, T)
            parts = [(full, self.gather_boundary(e, st['vals']), seeds, self.scatter_boundary)]
            if self.source_bases:
                parts.append((st['cvals'][eid], self.gather_source_boundary(e, st['cvals']),
                              seeds_c, self.scatter_source_boundary))
            for sol, solb, sd, scatter in parts:
                # the seeds live on the entity's own cells; zero elsewhere in its box
                seed = np.zeros(sol.shape)
                seed[e.keep] = sd[eid]
                mu = np.asarray(lu.solve(seed)).reshape(sol.shape)
                # -mu^T d(L x + B x_b)/dT_f = -(mu_a - mu_b)(x_a - x_b)
                inner = e.f_b >= 0
                mu_b = np.zeros((len(e.f_a), mu.shape[1]))
                x_b = np.zeros((len(e.f_a), mu.shape[1]))
                mu_b[inner] = mu[e.f_b[inner]]
                x_b[inner] = sol[e.f_b[inner]]
                x_b[~inner] = solb[e.f_q[~inner]]
                contrib = -np.sum((mu[e.f_a] - mu_b) * (sol[e.f_a] - x_b), axis=1)
                for k in range(len(e.f_a)):
                    gT[e.f_axis[k]][e.f_idx[k]] += contrib[k]
                # boundary seeds: -B^T mu
                scatter(e, sd, -(B.T @ mu))
        # chain rule through T(m)
        g = np.zeros(self.N)
        for a in range(self.d):
            x = np.nonzero(st['T'][a])[0]
            y = x + self.st[a]
            np.add.at(g, x, gT[a][x] * st['Dx'][a][x])
            np.add.at(g, y, gT[a][x] * st['Dy'][a][x])
        return g

    def misfit_gradient(self, st, d_obs):
        """phi = 1/2 ||d_pred - d_obs||_F^2 and its gradient J^T r."""
        r = st['d'] - np.asarray(d_obs)
        return 0.5 * float(np.sum(r * r)), self.jtvec(st, r)

    # -- fixed-basis variant (Sec. 4.2, Eq. senssimple), used as a contrast -----
    def jtvec_fixed_basis(self, st, w):
        """J^T w when the dependence of P on m is ignored (Eq. senssimple)."""
        Ns = self.prob.n_src
        P = st['P']
        Z = np.zeros((Ns, self.N))
        for j in range(Ns):
            np.add.at(Z[j], self.rec, w[j])
        gT = [np.zeros(self.N) for _ in range(self.d)]
        coords = cell_coords(self.n)
        for j in range(Ns):
            lam = self.R.T @ self.coarse_solve(st, P.T @ Z[j], transpose=True)
            for a in range(self.d):
                x = np.nonzero(coords[:, a] < self.n[a] - 1)[0]
                y = x + self.st[a]
                gT[a][x] -= (lam[x] - lam[y]) * (st['U'][j, x] - st['U'][j, y])
        g = np.zeros(self.N)
        for a in range(self.d):
            x = np.nonzero(st['T'][a])[0]
            y = x + self.st[a]
            np.add.at(g, x, gT[a][x] * st['Dx'][a][x])
            np.add.at(g, y, gT[a][x] * st['Dy'][a][x])
        return g

    # -- convenience -----------------------------------------------------------
    def basis_weights(self, st):
        """Dense P restricted to its non-zeros, as a scipy CSR matrix (N, Nc)."""
        return st['P']
