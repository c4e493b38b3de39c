"""Pins of the oracle's source bases (Sec. 3.2: local solves forced by the restricted
source with zero vertex data, added to the vertex bases with coefficient one).

* the dense brute-force map (a different organisation: one tangential system per level)
  with source bases, forward and, by complex step, J v and the misfit gradient;
* exactness for problems that are one-dimensional (sigma varying along x only, line or
  sheet dipoles off the vertex columns): the reduced boundary conditions are then exact
  and u = P t + C reproduces the fine solution to rounding, which the vertex bases
  alone do not;
* conservation R A u_j = R q_j, the local equations of every entity, c = 1.
CPU only."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import bruteforce as BF
from oracle.msfv_oracle import Oracle, cell_coords, fine_operator, transmissibility
from paper_1707_07598_gb300 import workloads as W

TINY = [
    ((8, 8), 2, 2, 5),
    ((12, 8), 4, 3, 6),
    ((9, 9), 3, 2, 4),
    ((10, 5), 5, 2, 4),
    ((6, 4, 4), 2, 2, 5),
    ((8, 8, 8), 4, 3, 7),
    ((6, 6, 6), 3, 2, 5),
    ((4, 4, 8), 4, 2, 4),
]


def _tiny(n, c, ns, nr, seed=31):
    prob = W.make_problem(n, c, ns, nr, seed=seed, top_layer=False, source_bases=True)
    m = W.gaussian_random_field(n, 0.3, seed + 2)
    return prob, m


def _problem(n, c, pos, neg, rec, amp=None):
    pos = np.asarray(pos, dtype=np.int64)
    return W.Problem(n=tuple(n), coarsen=c, src_pos=pos, src_neg=np.asarray(neg, dtype=np.int64),
                     src_amp=np.ones(len(pos)) if amp is None else np.asarray(amp, dtype=float),
                     rec_cell=np.asarray(rec, dtype=np.int64), source_bases=True)


def _idx(n, *xs):
    s, out = 1, 0
    for a, x in enumerate(xs):
        out += x * s
        s *= n[a]
    return out


@pytest.mark.parametrize("n,c,ns,nr", TINY)
def test_forward_matches_dense_brute_force(n, c, ns, nr):
    prob, m = _tiny(n, c, ns, nr)
    st = Oracle(prob).forward(m)
    d_bf, Phi, Ac = BF.forward_dense(m, n, c, prob.src_pos, prob.src_neg, prob.src_amp,
                                     prob.rec_cell, source_bases=True)
    d_plain, _, _ = BF.forward_dense(m, n, c, prob.src_pos, prob.src_neg, prob.src_amp,
                                     prob.rec_cell)
    assert np.abs(st['P'].toarray() - Phi).max() < 1e-12
    assert np.linalg.norm(st['d'] - d_bf) <= 1e-12 * np.linalg.norm(d_bf)
    if c > 1:   # the source bases change the answer
        assert np.linalg.norm(d_plain - d_bf) > 1e-6 * np.linalg.norm(d_bf)


def test_every_kind_of_source_cell_3d():
    """Source ends on a coarse vertex, a dual edge, a dual face and a dual-cell interior
    (and a partial boundary dual cell), against the brute force."""
    n, c = (8, 8, 8), 4               # vertex coordinates 2 and 6 on every axis
    cells = {
        'vertex': _idx(n, 2, 6, 2), 'edge': _idx(n, 4, 2, 6), 'face': _idx(n, 3, 6, 5),
        'interior': _idx(n, 4, 4, 4), 'boundary': _idx(n, 0, 7, 1), 'edge2': _idx(n, 6, 0, 2),
    }
    pos = [cells['vertex'], cells['edge'], cells['face'], cells['interior']]
    neg = [cells['boundary'], cells['interior'], cells['edge2'], cells['face']]
    rec = np.arange(0, 512, 7)
    prob = _problem(n, c, pos, neg, rec, amp=[1.0, -0.5, 2.0, 0.75])
    m = W.gaussian_random_field(n, 0.3, 5)
    st = Oracle(prob).forward(m)
    d_bf, _, _ = BF.forward_dense(m, n, c, prob.src_pos, prob.src_neg, prob.src_amp, rec,
                                  source_bases=True)
    assert np.linalg.norm(st['d'] - d_bf) <= 1e-12 * np.linalg.norm(d_bf)
    C = st['C']
    # zero on the coarse vertices, non-zero around every off-vertex source end
    X = cell_coords(n)
    vert = np.all((X - c // 2) % c == 0, axis=1)
    assert np.all(C[:, vert] == 0)
    assert np.all(np.abs(C[1:, cells['interior']]) > 0)
    v = W.noise_like(prob.N, 1.0, 6)
    ref = BF.jvec_complex_step(m, prob, v)
    o = Oracle(prob)
    assert np.linalg.norm(o.jvec(st, v) - ref) <= 1e-11 * np.linalg.norm(ref)


@pytest.mark.parametrize("n,c,ns,nr", [TINY[0], TINY[1], TINY[4], TINY[5], TINY[7]])
def test_jvec_matches_complex_step(n, c, ns, nr):
    prob, m = _tiny(n, c, ns, nr)
    o = Oracle(prob)
    st = o.forward(m)
    v = W.noise_like(prob.N, 1.0, 17)
    ref = BF.jvec_complex_step(m, prob, v)
    assert np.linalg.norm(o.jvec(st, v) - ref) <= 1e-11 * np.linalg.norm(ref)


@pytest.mark.parametrize("n,c,ns,nr", [((8, 8), 2, 2, 5), ((9, 6), 3, 2, 4), ((4, 4, 4), 2, 2, 4),
                                       ((6, 4, 4), 2, 2, 3)])
def test_gradient_matches_complex_step(n, c, ns, nr):
    prob, m = _tiny(n, c, ns, nr)
    o = Oracle(prob)
    st = o.forward(m)
    d_obs = st['d'] + W.noise_like(st['d'].shape, 0.05 * np.abs(st['d']).max(), 5)
    _, g = o.misfit_gradient(st, d_obs)
    g_ref = BF.misfit_gradient_complex_step(m, prob, d_obs)
    assert np.linalg.norm(g - g_ref) <= 1e-11 * np.linalg.norm(g_ref)


@pytest.mark.parametrize("n,c,ns,nr", TINY)
def test_dot_product(n, c, ns, nr):
    prob, m = _tiny(n, c, ns, nr)
    o = Oracle(prob)
    st = o.forward(m)
    v = W.noise_like(prob.N, 1.0, 21)
    w = W.noise_like((prob.n_src, prob.n_rec), 1.0, 23)
    lhs = np.sum(w * o.jvec(st, v))
    rhs = np.dot(o.jtvec(st, w), v)
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + np.linalg.norm(w) * np.linalg.norm(v) * 1e-3)


def _fine_solution(m, n, q, pin):
    """Fine FV solve A u = q with u[pin] = 0 (scipy's sparse LU)."""
    T, _, _ = transmissibility(m, n)
    A = fine_operator(T, n).tocsc()
    keep = np.setdiff1d(np.arange(len(q)), [pin])
    u = np.zeros(len(q))
    u[keep] = spla.splu(A[keep][:, keep]).solve(q[keep])
    return u


@pytest.mark.parametrize("n,c,x1,x2", [((16, 8), 4, 4, 12), ((24, 12), 6, 1, 16),
                                       ((12, 4, 4), 4, 4, 9), ((16, 8, 8), 4, 0, 11)])
def test_exact_for_one_dimensional_problems(n, c, x1, x2):
    """sigma = sigma(x) and a dipole pair of planes x = x1, x = x2 (one point dipole
    per transverse cell, both planes off the vertex columns): the fine solution is
    independent of y (and z), the tangential local problems are then exact, and the
    sum of the point-dipole solutions equals the fine solution to rounding."""
    d = len(n)
    assert (x1 - c // 2) % c and (x2 - c // 2) % c
    rng = np.random.default_rng(7)
    prof = rng.normal(0.0, 1.0, n[0])
    X = cell_coords(n)
    m = prof[X[:, 0]]
    trans = [X[:, 0] == 0]
    sel = np.nonzero(X[:, 0] == 0)[0]            # transverse cells (x = 0)
    pos = sel + x1
    neg = sel + x2
    rec = np.arange(0, int(np.prod(n)), 3)
    prob = _problem(n, c, pos, neg, rec)
    st = Oracle(prob).forward(m)
    u_ms = st['U'].sum(axis=0)
    q = np.zeros(prob.N)
    q[pos] += 1.0
    q[neg] -= 1.0
    pin = _idx(n, *([c // 2] * d))                # coarse vertex 0
    u_f = _fine_solution(m, n, q, pin)
    assert np.abs(u_ms - u_f).max() <= 1e-11 * np.abs(u_f).max()
    # the vertex bases alone are not exact here
    prob0 = _problem(n, c, pos, neg, rec)
    prob0.source_bases = False
    u0 = Oracle(prob0).forward(m)['U'].sum(axis=0)
    assert np.abs(u0 - u_f).max() > 1e-3 * np.abs(u_f).max()


@pytest.mark.parametrize("n,c,ns,nr", [((16, 16), 4, 3, 8), ((12, 12, 12), 4, 3, 8)])
def test_conservation_and_local_equations(n, c, ns, nr):
    """R A u_j = R q_j on every coarse cell; on every entity, the tangential operator
    applied to C_j (with C_j on the entity's boundary) equals q_j there; C_j = 0 on the
    vertices."""
    prob, m = _tiny(n, c, ns, nr, seed=41)
    o = Oracle(prob)
    st = o.forward(m)
    A, R = st['A'], o.R
    for j in range(prob.n_src):
        lhs = R @ (A @ st['U'][j])
        rhs = R @ o.Q[j]
        assert np.abs(lhs - rhs).max() <= 1e-12 * (1 + np.abs(rhs).max())
    for e, cv in zip(o.entities, st['cvals']):
        if e.dim == 0:
            assert np.all(st['C'][:, e.cells] == 0)
            continue
        L, B = o.local_matrices(e, st['T'])
        res = L @ cv + B @ o.gather_source_boundary(e, st['cvals']) - o.Q[:, e.cells].T
        assert np.abs(res).max() <= 1e-12 * (1 + np.abs(cv).max() * 1e3)


def test_coarsening_one_has_no_source_bases():
    """c = 1: every cell is a vertex, the source bases vanish and the answer is the
    plain one (the fine solve)."""
    prob, m = _tiny((6, 5), 1, 2, 6)
    st = Oracle(prob).forward(m)
    prob0 = W.make_problem((6, 5), 1, 2, 6, seed=31, top_layer=False)
    st0 = Oracle(prob0).forward(m)
    assert np.all(st['C'] == 0)
    assert np.array_equal(st['d'], st0['d'])


@pytest.mark.parametrize("c", [4, 8])
def test_source_bases_reduce_the_error_against_the_fine_solve(c):
    """The reason for source bases (Sec. 3.2): near the sources the vertex bases alone
    cannot represent the field.  On the 32^3 two-box model with surface dipoles the
    receiver data move closer to the fine solve (c = 1: P = I, A_c = A) with them.
    Both gauges pin the cell of coarse vertex 0."""
    n = (32, 32, 32)
    prob = W.make_problem(n, c, 4, 64, seed=131, top_layer=True)
    m = W.gaussian_random_field(n, 0.15, 132)
    m = W.add_box(m, n, (0.3, 0.5, 0.6), 0.2, 2.0)
    m = W.add_box(m, n, (0.7, 0.5, 0.6), 0.2, -2.0)
    pin = _idx(n, c // 2, c // 2, c // 2)
    fine = W.Problem(n=n, coarsen=1, src_pos=prob.src_pos, src_neg=prob.src_neg,
                     src_amp=prob.src_amp, rec_cell=prob.rec_cell)
    Uf = Oracle(fine).forward(m)['U']
    d_f = (Uf - Uf[:, [pin]])[:, prob.rec_cell]
    err = {}
    for sb in (False, True):
        prob.source_bases = sb
        d = Oracle(prob).forward(m)['d']
        err[sb] = np.linalg.norm(d - d_f) / np.linalg.norm(d_f)
    assert err[True] < 0.8 * err[False], err
