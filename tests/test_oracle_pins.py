"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test names the part of the oracle it pins; together they are chosen so that
a dropped term, a wrong sign or index, or a transposed operand in any oracle
step fails at least one of them.  CPU only.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import bruteforce as BF
from oracle.msfv_oracle import Oracle, axis_pieces, cell_coords, transmissibility
from paper_1707_07598_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

TINY = [
    ((8, 8), 2, 2, 5),
    ((12, 8), 4, 2, 6),
    ((9, 9), 3, 1, 4),
    ((10, 5), 5, 2, 4),
    ((8, 8), 1, 1, 3),
    ((6, 4, 4), 2, 2, 5),
    ((8, 8, 8), 4, 2, 7),
    ((6, 6, 6), 3, 2, 5),
    ((4, 4, 8), 4, 1, 4),
]


def _tiny(n, c, ns, nr, seed=3, corr=0.3):
    prob = W.make_problem(n, c, ns, nr, seed=seed, top_layer=False)
    m = W.gaussian_random_field(n, corr, seed + 2)
    return prob, m


# ---------------------------------------------------------------------------
# (a) face transmissibilities
# ---------------------------------------------------------------------------

def test_transmissibility_special_cases():
    """Constant sigma gives sigma * area / distance; two cells give the series value."""
    n = (4, 3, 2)
    m = np.full(24, 0.7)
    T, Dx, Dy = transmissibility(m, n)
    s = np.exp(0.7)
    X = cell_coords(n)
    geo = [(1 / 3) * (1 / 2) * 4, (1 / 4) * (1 / 2) * 3, (1 / 4) * (1 / 3) * 2]
    for a in range(3):
        inner = X[:, a] < n[a] - 1
        assert np.allclose(T[a][inner], s * geo[a], rtol=1e-15)
        assert np.all(T[a][~inner] == 0)          # no flux through the outer boundary
    # two cells: 1/T = (h/2)/s1 + (h/2)/s2 for a unit-area face at distance h
    m2 = np.array([np.log(2.0), np.log(6.0)])
    T2, D2x, D2y = transmissibility(m2, (2, 1))
    h = 0.5
    assert np.isclose(T2[0][0], 1.0 / (h / 2 / 2.0 + h / 2 / 6.0), rtol=1e-15)
    # derivative wrt log-conductivity by finite difference of the two-cell formula
    eps = 1e-6
    Tp, _, _ = transmissibility(m2 + np.array([eps, 0]), (2, 1))
    Tm, _, _ = transmissibility(m2 - np.array([eps, 0]), (2, 1))
    assert np.isclose(D2x[0][0], (Tp[0][0] - Tm[0][0]) / (2 * eps), rtol=1e-8)


# ---------------------------------------------------------------------------
# (b) local solves: closed forms
# ---------------------------------------------------------------------------

def _read_golden_edge():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "edge_series.txt"))
            if l.strip() and not l.startswith("#")]
    Tf = np.array(rows[0], dtype=float)
    lo = np.array(rows[1], dtype=float) / 11.0
    hi = np.array(rows[2], dtype=float) / 11.0
    return Tf, lo, hi


def test_edge_problem_matches_hand_derived_series_resistances():
    """The oracle's 1D local solve reproduces the hand-derived fixture."""
    Tf, lo, hi = _read_golden_edge()
    prob = W.Problem(n=(8, 4), coarsen=4, src_pos=np.array([0]), src_neg=np.array([1]),
                     src_amp=np.array([1.0]), rec_cell=np.array([0]))
    o = Oracle(prob)
    # the x-edge between vertices (2,2) and (6,2): inner cells x = 3, 4, 5 at y = 2
    cells = np.array([3 + 8 * 2, 4 + 8 * 2, 5 + 8 * 2])
    e = o.entities[o.cell2ent[cells[0]]]
    assert e.dim == 1 and np.array_equal(e.cells, cells)
    Tface = [np.zeros(32), np.zeros(32)]
    Tface[0][np.arange(2, 6) + 8 * 2] = Tf
    L, B = o.local_matrices(e, Tface)
    phib = np.zeros((len(e.bnd), len(e.corners)))
    for q, b in enumerate(e.bnd):
        J = o.cell2ent[b]
        vert = o.entities[J].corners[0]
        phib[q] = (e.corners == vert).astype(float)
    sol = spla.splu(L).solve(-(B @ phib))
    lo_col = int(np.argmin(e.corners))
    assert np.allclose(sol[:, lo_col], lo, atol=1e-15)
    assert np.allclose(sol[:, 1 - lo_col], hi, atol=1e-15)


@pytest.mark.parametrize("n,c,ns,nr", TINY + [((16, 12), 4, 1, 3), ((12, 12, 6), 3, 1, 3)])
def test_edge_profiles_are_series_resistances(n, c, ns, nr):
    """Every full dual edge: phi_lo(i) = resistance(i -> hi) / resistance(lo -> hi)."""
    prob, m = _tiny(n, c, ns, nr)
    o = Oracle(prob)
    st = o.forward(m)
    T = st['T']
    st_ = o.st
    for e, val in zip(o.entities, st['vals']):
        if e.dim != 1 or len(e.corners) != 2:
            continue
        a = e.axes[0]
        faces = np.concatenate([[e.cells[0] - st_[a]], e.cells])   # lower cell of each face
        res = 1.0 / T[a][faces]
        right = np.cumsum(res[::-1])[::-1][1:]                     # resistance right of each cell
        phi_lo = right / res.sum()
        lo_col = int(np.argmin(e.corners))
        assert np.allclose(val[:, lo_col], phi_lo, rtol=1e-12, atol=1e-14)


def _hat(x, K, c, nK):
    """1D interpolation weight of vertex K at coordinate x (partial ends are constant)."""
    pos = np.array([c * k + c // 2 for k in range(nK)])
    if x <= pos[0]:
        return 1.0 if K == 0 else 0.0
    if x >= pos[-1]:
        return 1.0 if K == nK - 1 else 0.0
    return max(0.0, 1.0 - abs(x - pos[K]) / c)


@pytest.mark.parametrize("n,c", [((12, 8), 4), ((9, 6), 3), ((8, 8, 4), 4), ((6, 9, 3), 3),
                                 ((8, 4, 6), 2), ((10, 10), 5)])
def test_constant_sigma_gives_multilinear_basis(n, c):
    """Constant sigma (anisotropic cells allowed): phi_J = product of 1D hats in index space."""
    prob = W.make_problem(n, c, 1, 2, seed=1, top_layer=False)
    o = Oracle(prob)
    st = o.forward(np.full(prob.N, -0.4))
    P = st['P'].toarray()
    X = cell_coords(n)
    nc = tuple(v // c for v in n)
    Jc = cell_coords(nc)
    expect = np.ones_like(P)
    for a in range(len(n)):
        w = np.array([[_hat(X[x, a], Jc[J, a], c, nc[a]) for J in range(o.Nc)]
                      for x in range(o.N)])
        expect *= w
    assert np.abs(P - expect).max() < 1e-13


@pytest.mark.parametrize("n,c,ns,nr", TINY)
def test_partition_of_unity(n, c, ns, nr):
    prob, m = _tiny(n, c, ns, nr)
    o = Oracle(prob)
    st = o.forward(m)
    assert np.abs(st['P'] @ np.ones(o.Nc) - 1.0).max() < 1e-13


def test_axis_pieces_cover_each_axis_once():
    for n_a, c in [(8, 1), (8, 2), (12, 3), (16, 4), (15, 5), (64, 8), (48, 16)]:
        cov = np.zeros(n_a, dtype=int)
        for pc in axis_pieces(n_a, c):
            if pc[0] == 'V':
                cov[pc[2]] += 1
                assert pc[2] == c * pc[1] + c // 2
            else:
                cov[pc[3]:pc[3] + pc[4]] += 1
        assert np.all(cov == 1)


# ---------------------------------------------------------------------------
# (c)-(e) coarse operator and reduced solve
# ---------------------------------------------------------------------------

def _fv_matrix(m, n):
    """Cell-centred FV matrix written out face by face (independent of the oracle)."""
    n = tuple(n)
    N = int(np.prod(n))
    X = cell_coords(n)
    sig = np.exp(m)
    A = sp.lil_matrix((N, N))
    stride = [1, n[0], n[0] * (n[1] if len(n) > 1 else 1)]
    for x in range(N):
        for a in range(len(n)):
            if X[x, a] + 1 < n[a]:
                y = x + stride[a]
                area = np.prod([1.0 / n[b] for b in range(len(n)) if b != a])
                t = area * n[a] / (0.5 / sig[x] + 0.5 / sig[y])
                A[x, x] += t
                A[y, y] += t
                A[x, y] -= t
                A[y, x] -= t
    return A.tocsc()


@pytest.mark.parametrize("n", [(8, 8), (6, 5, 4)])
def test_coarsening_one_is_the_fine_solve(n):
    """c = 1: P = I and A_c = A; data equal a library solve of the pinned fine system."""
    prob = W.make_problem(n, 1, 3, 6, seed=4, top_layer=False)
    m = W.gaussian_random_field(n, 0.3, 6)
    o = Oracle(prob)
    st = o.forward(m)
    A = _fv_matrix(m, n)
    for j in range(prob.n_src):
        q = np.zeros(prob.N)
        q[prob.src_pos[j]] += 1
        q[prob.src_neg[j]] -= 1
        u = np.zeros(prob.N)
        u[1:] = spla.spsolve(A[1:, 1:], q[1:])
        assert np.allclose(st['d'][j], u[prob.rec_cell], rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("n,c,ns,nr", TINY)
def test_conservation_RAPt_equals_Rq(n, c, ns, nr):
    """The reduced solution conserves mass on every primal coarse cell, incl. the pinned one."""
    prob, m = _tiny(n, c, ns, nr)
    o = Oracle(prob)
    st = o.forward(m)
    for j in range(prob.n_src):
        res = o.R @ (st['A'] @ (st['P'] @ st['t'][j])) - o.R @ o.Q[j]
        assert np.abs(res).max() < 1e-12 * max(1.0, np.abs(o.R @ o.Q[j]).max())
        assert st['t'][j][0] == 0.0


def _mms_error(n, c):
    nn = (n, n)
    X = (cell_coords(nn) + 0.5) / n
    m = 0.5 * np.sin(2 * np.pi * X[:, 0]) * np.cos(np.pi * X[:, 1])
    sig = np.exp(m)
    gm = np.stack([np.pi * np.cos(2 * np.pi * X[:, 0]) * np.cos(np.pi * X[:, 1]),
                   -0.5 * np.pi * np.sin(2 * np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1])], 1)
    u = np.cos(np.pi * X[:, 0]) * np.cos(np.pi * X[:, 1])
    gu = np.stack([-np.pi * np.sin(np.pi * X[:, 0]) * np.cos(np.pi * X[:, 1]),
                   -np.pi * np.cos(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1])], 1)
    q = -sig * (np.sum(gm * gu, axis=1) - 2 * np.pi ** 2 * u)   # -div(sigma grad u)
    q = q / n ** 2
    q -= q.mean()
    prob = W.Problem(n=nn, coarsen=c, src_pos=np.array([0]), src_neg=np.array([1]),
                     src_amp=np.array([1.0]), rec_cell=np.arange(n * n))
    o = Oracle(prob)
    o.Q = q[None, :]
    uh = o.forward(m)['U'][0]
    e = (uh - uh.mean()) - (u - u.mean())
    return np.sqrt(np.mean(e ** 2))


@pytest.mark.parametrize("c,ns,lo", [(1, (16, 32, 64), 1.9), (3, (12, 24, 48), 1.9),
                                     (4, (16, 32, 64), 0.9)])
def test_manufactured_solution_convergence(c, ns, lo):
    """u = cos(pi x) cos(pi y), smooth sigma: O(h^2) for c = 1 and odd c; even c is O(h)
    because the coarse vertex sits half a cell off the coarse-cell centre."""
    errs = [_mms_error(n, c) for n in ns]
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert min(rates) >= lo, rates


# ---------------------------------------------------------------------------
# everything forward: dense brute force
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,c,ns,nr", TINY)
def test_forward_matches_dense_brute_force(n, c, ns, nr):
    prob, m = _tiny(n, c, ns, nr)
    o = Oracle(prob)
    st = o.forward(m)
    d_bf, Phi, Ac = BF.forward_dense(m, n, c, prob.src_pos, prob.src_neg, prob.src_amp,
                                     prob.rec_cell)
    assert np.abs(st['P'].toarray() - Phi).max() < 1e-12
    assert np.abs(st['Ac'].toarray() - Ac).max() < 1e-12 * np.abs(Ac).max()
    assert np.linalg.norm(st['d'] - d_bf) <= 1e-12 * np.linalg.norm(d_bf)


# ---------------------------------------------------------------------------
# (f) derivatives
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,c,ns,nr", TINY)
def test_jvec_matches_complex_step(n, c, ns, nr):
    prob, m = _tiny(n, c, ns, nr)
    o = Oracle(prob)
    st = o.forward(m)
    v = W.noise_like(prob.N, 1.0, 17)
    jv = o.jvec(st, v)
    ref = BF.jvec_complex_step(m, prob, v)
    assert np.linalg.norm(jv - ref) <= 1e-11 * np.linalg.norm(ref)


@pytest.mark.parametrize("n,c,ns,nr", [((8, 8), 2, 2, 5), ((9, 6), 3, 2, 4), ((4, 4, 4), 2, 2, 4),
                                       ((6, 4, 4), 2, 1, 3)])
def test_gradient_matches_complex_step(n, c, ns, nr):
    """Full misfit gradient vs one complex-step derivative per cell."""
    prob, m = _tiny(n, c, ns, nr)
    o = Oracle(prob)
    st = o.forward(m)
    d_obs = st['d'] + W.noise_like(st['d'].shape, 0.05 * np.abs(st['d']).max(), 5)
    phi, g = o.misfit_gradient(st, d_obs)
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


@pytest.mark.parametrize("n,c", [((32, 32), 8), ((16, 16, 16), 4)])
def test_gradient_central_differences(n, c):
    """Central differences (step 1e-6) along 20 random directions agree with J^T r."""
    prob = W.make_problem(n, c, 2, 16, seed=8, top_layer=len(n) == 3)
    m = W.gaussian_random_field(n, 0.15, 9)
    o = Oracle(prob)
    st = o.forward(m)
    d_obs = st['d'] * 1.01 + W.noise_like(st['d'].shape, 1e-3, 4)
    phi, g = o.misfit_gradient(st, d_obs)
    for k in range(20):
        v = W.noise_like(prob.N, 1.0, 100 + k)
        fp, _ = 0.5 * np.sum((o.forward(m + 1e-6 * v)['d'] - d_obs) ** 2), None
        fm = 0.5 * np.sum((o.forward(m - 1e-6 * v)['d'] - d_obs) ** 2)
        fd = (fp - fm) / 2e-6
        assert abs(fd - g @ v) <= 1e-6 * max(abs(fd), 1e-3 * np.linalg.norm(g) * np.linalg.norm(v))


def test_adaptive_basis_gradient_beats_fixed_basis():
    """Ignoring dP/dm (Sec. 4.2, Eq. senssimple) gives visibly wrong directional
    derivatives, while the adaptive gradient (Eq. sensred) matches central differences.
    A constant direction would not show it: uniform scaling of sigma leaves every
    local problem, hence P, unchanged."""
    n, c = (32, 32), 8
    prob = W.make_problem(n, c, 1, 64, seed=12, top_layer=False)
    X = (cell_coords(n) + 0.5) / 32
    inside = (np.abs(X[:, 0] - 0.5) < 0.2) & (np.abs(X[:, 1] - 0.5) < 0.2)
    m = np.where(inside, np.log(0.1), np.log(0.01))     # conductive block (Sec. 4.4)
    o = Oracle(prob)
    st = o.forward(m)
    w = W.noise_like((1, prob.n_rec), 1.0, 3)
    g_ada = o.jtvec(st, w)
    g_fix = o.jtvec_fixed_basis(st, w)
    # constant direction: both agree (basis invariant to uniform scaling)
    one = np.ones(prob.N)
    assert abs(g_ada @ one - g_fix @ one) <= 1e-10 * abs(g_ada @ one)
    for k in range(3):
        v = W.noise_like(prob.N, 1.0, 40 + k)
        s = 1e-5
        ref = np.sum(w * (o.forward(m + s * v)['d'] - o.forward(m - s * v)['d'])) / (2 * s)
        err_ada = abs(g_ada @ v - ref) / abs(ref)
        err_fix = abs(g_fix @ v - ref) / abs(ref)
        assert err_ada < 1e-6, (err_ada, err_fix)
        assert err_fix > 1e-2, (err_ada, err_fix)


def test_golden_oracle_outputs_are_reproduced():
    """Regression fixtures written by tests/golden/make_golden.py (oracle only)."""
    import json
    with open(os.path.join(GOLDEN, "oracle_tiny.json")) as f:
        gold = json.load(f)
    from oracle.galerkin_oracle import NodalOracle
    assert len(gold) >= 8 and any(c.get('sb') for c in gold) and any(c.get('nodal') for c in gold)
    assert any(c.get('ov') for c in gold)
    for case in gold:
        prob = W.make_problem(tuple(case['n']), case['c'], case['ns'], case['nr'],
                              seed=case['seed'], top_layer=False,
                              source_bases=case.get('sb', False), nodal=case.get('nodal', False),
                              oversample=case.get('ov', 0))
        m = W.gaussian_random_field(prob.n, case['corr'], case['seed'] + 2)
        o = NodalOracle(prob) if case.get('nodal') else Oracle(prob)
        st = o.forward(m)
        phi, g = o.misfit_gradient(st, np.array(case['d_obs']))
        assert np.allclose(st['d'], np.array(case['d']), rtol=1e-12, atol=1e-14)
        assert np.allclose(g, np.array(case['grad']), rtol=1e-10, atol=1e-14)


# ---------------------------------------------------------------------------------
# Gauss-Newton-CG driver oracle (Sec. 5)
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("n", [(5, 4), (4, 3, 5), (6, 6, 6)])
def test_regulariser_of_a_linear_field_closed_form(n):
    """m = x-coordinate of the cell centre: every x-face jumps by 1/n_x, so
    R = alpha/2 (n_x - 1)/n_x (faces of the other axes see no jump)."""
    from oracle.gn_oracle import reg_value
    N = int(np.prod(n))
    x = (np.arange(N) % n[0] + 0.5) / n[0]
    assert abs(reg_value(n, x, alpha=3.0) - 1.5 * (n[0] - 1) / n[0]) < 1e-13
    # the same along the last axis
    last = (np.arange(N) // int(np.prod(n[:-1])) + 0.5) / n[-1]
    assert abs(reg_value(n, last, alpha=2.0) - (n[-1] - 1) / n[-1]) < 1e-13


@pytest.mark.parametrize("n", [(5, 4), (4, 3, 5)])
def test_regulariser_matrix_is_the_hessian(n):
    from oracle.gn_oracle import reg_matrix, reg_value
    K = reg_matrix(n)
    N = K.shape[0]
    assert abs(K - K.T).max() < 1e-14                     # symmetric
    assert np.abs(K @ np.ones(N)).max() < 1e-12           # constants are free
    rng = np.random.default_rng(3)
    m, ref = rng.standard_normal(N), rng.standard_normal(N)
    # R(m) = alpha/2 (m - ref)^T K (m - ref) and grad R = alpha K (m - ref) (central FD)
    assert abs(reg_value(n, m, ref, 2.0) - (m - ref) @ (K @ (m - ref))) < 1e-10
    v = rng.standard_normal(N)
    fd = (reg_value(n, m + 1e-6 * v, ref, 2.0) - reg_value(n, m - 1e-6 * v, ref, 2.0)) / 2e-6
    assert abs(fd - 2.0 * v @ (K @ (m - ref))) < 1e-6 * max(1.0, abs(fd))
    # positive semi-definite
    assert np.linalg.eigvalsh(K.toarray()).min() > -1e-12


def test_gauss_newton_cg_direction_equals_a_dense_solve():
    """With as many CG iterations as unknowns the CG direction is the dense solution of
    (J^T J + alpha K) x = -g (J assembled column by column from the oracle's jvec)."""
    from oracle.gn_oracle import gn_step, reg_matrix
    prob = W.make_problem((6, 6), 3, 2, 8, seed=5, top_layer=False)
    m = W.gaussian_random_field(prob.n, 0.3, 6)
    orc = Oracle(prob)
    st = orc.forward(m)
    d_obs = st['d'] * 1.05 + 1e-3
    alpha = 1e-2
    m1, info = gn_step(orc, m, d_obs, alpha, cg_iters=200, cg_tol=1e-14, max_backtracks=0,
                       bounds=(-1e9, 1e9))
    N = prob.N
    J = np.stack([orc.jvec(st, e).ravel() for e in np.eye(N)], axis=1)
    K = reg_matrix(prob.n).toarray()
    g = J.T @ (st['d'] - d_obs).ravel() + alpha * K @ m
    x = np.linalg.solve(J.T @ J + alpha * K, -g)
    assert np.linalg.norm(info['x'] - x) <= 1e-8 * np.linalg.norm(x)
    assert info['phi_d1'] + info['phi_r1'] < info['phi_d0'] + info['phi_r0']
