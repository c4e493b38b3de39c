"""Pins of the nodal Galerkin oracle (the paper's own variant: nodal operator, Lagrange
boundary data on primal blocks, A_k = S^T A S, sensitivities with the X_k term).

* the dense brute force (cell-by-cell assembly, all block interiors in one system):
  operator, basis and data; J v and the misfit gradient by complex step; dot product;
* the X_k term: leaving it out breaks J v whenever a source sits inside a block;
* constant sigma: the basis is exactly the multilinear (Lagrange) interpolation;
* Galerkin properties: S^T (q - A U) = 0 off the pinned row, A_k symmetric, and U has
  the smallest energy error against the fine solve over the span of S;
* c = 1: S = I and the model is the fine nodal solve;
* identity receivers (Sec. 4.4): the adaptive Jacobian matches complex step, the
  fixed-basis one does not.
CPU only."""
import numpy as np
import pytest

from oracle import bruteforce as BF
from oracle.galerkin_oracle import NodalOracle
from paper_1707_07598_gb300 import workloads as W

TINY = [((8, 8), 2, 2, 5), ((8, 8), 4, 2, 6), ((6, 9), 3, 2, 5), ((12, 8), 4, 3, 7),
        ((4, 4, 4), 2, 2, 5), ((8, 4, 4), 4, 2, 6), ((6, 6, 6), 3, 2, 5), ((6, 6), 1, 2, 4)]


def _tiny(n, c, ns, nr, seed=3):
    prob = W.make_problem(n, c, ns, nr, seed=seed, top_layer=False, nodal=True)
    m = W.gaussian_random_field(n, 0.3, seed + 2)
    return prob, m


def _node(nn, *xs):
    s, o = 1, 0
    for a, x in enumerate(xs):
        o += x * s
        s *= nn[a]
    return o


@pytest.mark.parametrize("n,c,ns,nr", TINY)
def test_forward_matches_dense_brute_force(n, c, ns, nr):
    prob, m = _tiny(n, c, ns, nr)
    st = NodalOracle(prob).forward(m)
    d_bf, S, Ak, A = BF.forward_dense_nodal(m, n, c, prob.src_pos, prob.src_neg, prob.src_amp,
                                            prob.rec_cell)
    assert np.abs(st['A'].toarray() - A).max() <= 1e-13 * np.abs(A).max()
    assert np.abs(st['S'].toarray() - S).max() <= 1e-12
    assert np.abs(st['Ak'].toarray() - Ak).max() <= 1e-12 * np.abs(Ak).max()
    assert np.linalg.norm(st['d'] - d_bf) <= 1e-12 * np.linalg.norm(d_bf)


@pytest.mark.parametrize("n,c,ns,nr", TINY)
def test_jvec_matches_complex_step_and_dot_product(n, c, ns, nr):
    prob, m = _tiny(n, c, ns, nr)
    o = NodalOracle(prob)
    st = o.forward(m)
    v = W.noise_like(prob.N, 1.0, 17)
    jv = o.jvec(st, v)
    ref = BF.jvec_complex_step_nodal(m, prob, v)
    assert np.linalg.norm(jv - ref) <= 1e-11 * np.linalg.norm(ref)
    w = W.noise_like((prob.n_src, prob.n_rec), 1.0, 19)
    lhs, rhs = np.sum(w * jv), o.jtvec(st, w) @ v
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + np.linalg.norm(w) * np.linalg.norm(v) * 1e-3)


@pytest.mark.parametrize("n,c,ns,nr", [((8, 8), 4, 2, 6), ((6, 6), 3, 2, 5), ((4, 4, 4), 2, 2, 4)])
def test_gradient_matches_complex_step(n, c, ns, nr):
    prob, m = _tiny(n, c, ns, nr, seed=5)
    o = NodalOracle(prob)
    st = o.forward(m)
    d_obs = st['d'] + W.noise_like(st['d'].shape, 0.05 * np.abs(st['d']).max(), 6)
    _, g = o.misfit_gradient(st, d_obs)
    g_ref = BF.misfit_gradient_complex_step_nodal(m, prob, d_obs)
    assert np.linalg.norm(g - g_ref) <= 1e-11 * np.linalg.norm(g_ref)


def test_the_x_term_is_needed_when_a_source_is_inside_a_block():
    n, c = (12, 12), 4
    nn = (13, 13)
    prob = W.Problem(n=n, coarsen=c, src_pos=np.array([_node(nn, 5, 6)]),   # block interior
                     src_neg=np.array([_node(nn, 8, 3)]), src_amp=np.array([1.0]),
                     rec_cell=np.arange(0, 169, 4, dtype=np.int64), nodal=True)
    m = W.gaussian_random_field(n, 0.3, 9)
    o = NodalOracle(prob)
    st = o.forward(m)
    v = W.noise_like(prob.N, 1.0, 10)
    ref = BF.jvec_complex_step_nodal(m, prob, v)
    assert np.linalg.norm(o.jvec(st, v) - ref) <= 1e-11 * np.linalg.norm(ref)
    assert np.linalg.norm(o.jvec(st, v, with_x=False) - ref) > 1e-3 * np.linalg.norm(ref)


@pytest.mark.parametrize("n,c", [((12, 8), 4), ((6, 6, 9), 3)])
def test_constant_sigma_gives_the_lagrange_interpolation(n, c):
    prob = W.make_problem(n, c, 1, 3, seed=1, top_layer=False, nodal=True)
    o = NodalOracle(prob)
    st = o.forward(np.full(prob.N, 0.4))
    assert np.abs(st['S'].toarray() - o.Hat.toarray()).max() <= 1e-13


@pytest.mark.parametrize("n,c,ns,nr", [((16, 16), 4, 3, 10), ((8, 8, 8), 4, 2, 9)])
def test_galerkin_orthogonality_symmetry_and_energy_optimality(n, c, ns, nr):
    prob, m = _tiny(n, c, ns, nr, seed=11)
    o = NodalOracle(prob)
    st = o.forward(m)
    A, S, Ak = st['A'], st['S'], st['Ak']
    assert abs(Ak - Ak.T).max() <= 1e-14 * abs(Ak).max()
    for j in range(ns):
        res = S.T @ (o.Q[j] - A @ st['U'][j])
        assert np.abs(res[1:]).max() <= 1e-12 * np.abs(S.T @ o.Q[j]).max()
    # energy error against the fine solve (same pinned node 0) is smallest at t
    fine = W.Problem(n=n, coarsen=1, src_pos=prob.src_pos, src_neg=prob.src_neg,
                     src_amp=prob.src_amp, rec_cell=prob.rec_cell, nodal=True)
    Uf = NodalOracle(fine).forward(m)['U']
    rng = np.random.default_rng(0)
    for j in range(ns):
        e0 = Uf[j] - st['U'][j]
        E0 = e0 @ (A @ e0)
        for _ in range(5):
            dt = rng.normal(size=o.Ncn)
            dt[0] = 0.0
            e1 = e0 - S @ (1e-3 * dt * np.abs(st['t'][j]).max())
            assert e1 @ (A @ e1) >= E0 * (1 - 1e-12)


def test_coarsening_one_is_the_fine_nodal_solve():
    n = (6, 5)
    prob = W.make_problem(n, 1, 2, 6, seed=13, top_layer=False, nodal=True)
    m = W.gaussian_random_field(n, 0.3, 14)
    st = NodalOracle(prob).forward(m)
    assert np.array_equal(st['S'].toarray(), np.eye(42))
    _, _, _, A = BF.forward_dense_nodal(m, n, 1, prob.src_pos, prob.src_neg, prob.src_amp,
                                        prob.rec_cell)
    for j in range(2):
        q = np.zeros(42)
        q[prob.src_pos[j]] += 1.0
        q[prob.src_neg[j]] -= 1.0
        u = np.zeros(42)
        u[1:] = np.linalg.solve(A[1:, 1:], q[1:])
        assert np.abs(st['U'][j] - u).max() <= 1e-12 * np.abs(u).max()


def test_identity_receivers_adaptive_matches_fixed_does_not():
    """Sec. 4.4: one dipole, every node a receiver, a conductive block; along a smooth
    non-constant direction the adaptive Jacobian equals complex step while the
    fixed-basis one misses by far more than rounding."""
    n, c = (12, 12, 6), 3
    nn = tuple(v + 1 for v in n)
    Nn = int(np.prod(nn))
    prob = W.Problem(n=n, coarsen=c, src_pos=np.array([_node(nn, 2, 6, 6)]),
                     src_neg=np.array([_node(nn, 10, 6, 6)]), src_amp=np.array([1.0]),
                     rec_cell=np.arange(Nn, dtype=np.int64), nodal=True)
    X = np.stack(np.unravel_index(np.arange(prob.N), n[::-1])[::-1], axis=1)
    box = np.all((X >= [4, 4, 2]) & (X < [8, 8, 4]), axis=1)
    m = np.where(box, np.log(0.1), np.log(0.01))
    o = NodalOracle(prob)
    st = o.forward(m)
    v = np.sin(np.pi * X[:, 0] / n[0]) * np.cos(np.pi * X[:, 1] / n[1])
    w = W.noise_like((1, Nn), 1.0, 3)
    ref = BF.jvec_complex_step_nodal(m, prob, v)
    g_ad = o.jtvec(st, w)
    g_fx = o.jtvec_fixed_basis(st, w)
    fd = np.sum(w * ref)
    assert abs(g_ad @ v - fd) <= 1e-10 * abs(fd)
    assert abs(g_fx @ v - fd) > 1e-4 * abs(fd)


@pytest.mark.parametrize("d", [2, 3])
def test_nodal_operator_converges_at_second_order(d):
    """The nodal operator (reading R13: arithmetic edge averages of sigma, area/length
    weights, no flux through the outer boundary) against -div(sigma grad u) = f for the
    manufactured u = prod cos(pi x_a) and a smooth sigma, with f integrated over each
    node's dual volume: the nodal error falls at second order.  This pins the geometric
    factors and the averaging independently of the brute force, which shares the reading."""
    import scipy.sparse.linalg as spla
    errs = []
    sizes = (8, 16, 32) if d == 2 else (4, 8, 16)
    for n in sizes:
        nn = (n,) * d
        prob = W.Problem(n=nn, coarsen=1, src_pos=np.array([0]), src_neg=np.array([1]),
                         src_amp=np.array([1.0]), rec_cell=np.array([0]), nodal=True)
        o = NodalOracle(prob)
        h = 1.0 / n
        Xc = (o.Xc + 0.5) * h                       # cell centres
        m = 0.5 * np.sin(2 * np.pi * Xc[:, 0]) * np.cos(np.pi * Xc[:, -1])
        A = o.operator(o.E @ np.exp(m))
        Xn = o.Xn * h                               # node positions
        # sigma and its gradient at the nodes from the same analytic model
        s_m = 0.5 * np.sin(2 * np.pi * Xn[:, 0]) * np.cos(np.pi * Xn[:, -1])
        sig = np.exp(s_m)
        dm = np.zeros_like(Xn)
        dm[:, 0] += np.pi * np.cos(2 * np.pi * Xn[:, 0]) * np.cos(np.pi * Xn[:, -1])
        dm[:, -1] += -0.5 * np.pi * np.sin(2 * np.pi * Xn[:, 0]) * np.sin(np.pi * Xn[:, -1])
        u = np.prod(np.cos(np.pi * Xn), axis=1)
        grad_u = np.stack([-np.pi * np.sin(np.pi * Xn[:, a]) *
                           np.prod(np.cos(np.pi * np.delete(Xn, a, axis=1)), axis=1)
                           for a in range(d)], axis=1)
        lap_u = -d * np.pi ** 2 * u
        f = -(sig * lap_u + sig * np.sum(dm * grad_u, axis=1))   # -div(sigma grad u)
        vol = np.prod(np.where((o.Xn == 0) | (o.Xn == n), 0.5, 1.0), axis=1) * h ** d
        q = f * vol
        q -= (q.sum() / vol.sum()) * vol            # compatible with the Neumann problem
        keep = np.arange(1, o.Nn)
        uh = np.zeros(o.Nn)
        uh[keep] = spla.spsolve(A[keep][:, keep].tocsc(), q[keep])
        e = (uh - uh.mean()) - (u - u.mean())
        errs.append(np.abs(e).max())
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert min(rates) >= 1.8, (errs, rates)


def test_constant_direction_leaves_the_lagrange_basis_unchanged():
    """Sec. 4.4 uses a constant perturbation dm = -0.001 * 1.  The Lagrange-data basis is
    invariant under a uniform scaling of sigma (the block problems are homogeneous in
    sigma and their boundary data are fixed), so dS = 0 along it and the adaptive and
    fixed-basis J v coincide; along a non-constant direction they differ."""
    n, c = (12, 12, 6), 3
    nn = tuple(v + 1 for v in n)
    Nn = int(np.prod(nn))
    prob = W.Problem(n=n, coarsen=c, src_pos=np.array([_node(nn, 2, 6, 6)]),
                     src_neg=np.array([_node(nn, 10, 6, 6)]), src_amp=np.array([1.0]),
                     rec_cell=np.arange(Nn, dtype=np.int64), nodal=True)
    m = W.gaussian_random_field(n, 0.3, 17)
    o = NodalOracle(prob)
    st_ = o.forward(m)

    def fixed_jv(v):
        dA = o.operator(o.dweights(st_, v))
        S = st_['S']
        dt = o.coarse_solve(st_, -(S.T @ (dA @ st_['U'][0])))
        return (S @ dt)[prob.rec_cell]

    v0 = -0.001 * np.ones(prob.N)
    ja = o.jvec(st_, v0)[0]
    assert np.linalg.norm(ja - fixed_jv(v0)) <= 1e-12 * np.linalg.norm(ja)
    X = np.stack(np.unravel_index(np.arange(prob.N), n[::-1])[::-1], axis=1)
    v1 = 0.001 * np.sin(np.pi * (X[:, 0] + 0.5) / n[0])
    j1 = o.jvec(st_, v1)[0]
    assert np.linalg.norm(j1 - fixed_jv(v1)) > 1e-4 * np.linalg.norm(j1)


# The sizes the paper prints for its two test meshes (Sec. 5.1, Tab. 1; Sec. 5.2, Tab. 2):
# the fine nodal systems have k = 17,797 (36 x 36 x 12 cells) and 139,425 (64 x 64 x 32)
# unknowns, and each multiscale k is the number of Lagrange coarse nodes plus the
# augmented bases the text lists (25 global-skeleton + 93 / 400 local bases for the block
# model's 12^3 / 6^3 blocks; 72 + 862 / 3938 for the SEG model's 16^3 / 8^3 blocks).
PAPER_SIZES = [
    ((36, 36, 12), 12, 17797, 150, 25 + 93),
    ((36, 36, 12), 6, 17797, 572, 25 + 400),
    ((64, 64, 32), 16, 139425, 1009, 72 + 862),
    ((64, 64, 32), 8, 139425, 4415, 72 + 3938),
]


@pytest.mark.parametrize("n,c,k_fine,k_ms,augmented", PAPER_SIZES)
def test_node_and_basis_counts_match_the_paper(n, c, k_fine, k_ms, augmented):
    prob = W.make_problem(n, c, 2, 4, seed=1, nodal=True)
    orc = NodalOracle(prob)
    assert orc.Nn == k_fine
    assert orc.Ncn + augmented == k_ms
    assert orc.Hat.shape == (k_fine, k_ms - augmented)
