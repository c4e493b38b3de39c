"""Source bases (Sec. 3.2) on the GPU, through the C ABI, against the CPU oracle.

Bar: 1e-9 relative 2-norm on d, u, the misfit gradient, J v, J^T w and the fixed-basis
J^T w.  Cases: 2D and 3D, odd and even c, partial dual cells, sources on every kind of
cell (coarse vertex, dual edge, dual face, dual-cell interior, several sources in one
entity), shared- and global-memory factor windows (c = 16), both coarse solvers, the
128^3 c = 8 workload.  Also: the one-dimensional exactness pin on the GPU alone,
bitwise repeatability and the rejected recompute mode."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.msfv_oracle import Oracle  # noqa: E402
from paper_1707_07598_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-9


def rel(a, b):
    """Relative error in the 2-norm and in the max-norm, whichever is larger: a bound on
    rel() holds for the whole array and for its largest entries alike."""
    a = np.asarray(a)
    b = np.asarray(b)
    r2 = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
    rinf = np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300) if b.size else 0.0
    return max(r2, rinf)


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1707_07598_gb300 import build
    build.build()
    return torch.device("cuda:0")


def _idx(n, *xs):
    s, out = 1, 0
    for a, x in enumerate(xs):
        out += x * s
        s *= n[a]
    return out


def check_all(prob, m, dev, seed=0, factor_mode=0, derivs=True):
    from paper_1707_07598_gb300.msfv import Session
    orc = Oracle(prob)
    st = orc.forward(m)
    d_obs = st['d'] * 1.02 + W.noise_like(st['d'].shape, 1e-3 * np.abs(st['d']).max(), seed + 1)
    phi_ref, g_ref = orc.misfit_gradient(st, d_obs)
    s = Session(prob, factor_mode=factor_mode)
    assert s.info()["source_slots"] > 0
    mt = torch.from_numpy(m).to(dev)
    u = torch.empty((prob.n_src, prob.N), dtype=torch.float64, device=dev)
    d = s.forward(mt, u=u)
    phi, g = s.adjoint(torch.from_numpy(d_obs).to(dev))
    assert rel(d.cpu().numpy(), st['d']) < TOL
    assert rel(u.cpu().numpy(), st['U']) < TOL
    assert abs(phi - phi_ref) <= TOL * abs(phi_ref)
    assert rel(g.cpu().numpy(), g_ref) < TOL
    if derivs:
        v = W.noise_like(prob.N, 1.0, seed + 5)
        w = W.noise_like((prob.n_src, prob.n_rec), 1.0, seed + 6)
        jv = s.jvec(torch.from_numpy(v).to(dev)).cpu().numpy()
        jtw = s.jtvec(torch.from_numpy(w).to(dev)).cpu().numpy()
        assert rel(jv, orc.jvec(st, v)) < TOL
        assert rel(jtw, orc.jtvec(st, w)) < TOL
        jtf = s.jtvec_fixed_basis(torch.from_numpy(w).to(dev)).cpu().numpy()
        assert rel(jtf, orc.jtvec_fixed_basis(st, w)) < TOL
    s.close()
    return st


CASES = [
    ((16, 16), 4, 3, 9),
    ((24, 16), 8, 3, 12),
    ((18, 18), 3, 4, 10),
    ((20, 15), 5, 2, 8),
    ((16, 12), 2, 3, 7),
    ((8, 8, 8), 4, 3, 9),
    ((12, 8, 8), 4, 2, 9),
    ((9, 9, 6), 3, 3, 7),
    ((16, 16, 16), 8, 4, 20),
    ((10, 10, 10), 5, 2, 8),
    ((8, 6, 4), 2, 3, 6),
    ((24, 16, 16), 8, 5, 30),
]


@pytest.mark.parametrize("n,c,ns,nr", CASES)
def test_source_bases_match_oracle(dev, n, c, ns, nr):
    prob = W.make_problem(n, c, ns, nr, seed=61, top_layer=False, source_bases=True)
    m = W.gaussian_random_field(n, 0.2, 62)
    check_all(prob, m, dev, seed=63)


def test_every_kind_of_source_cell(dev):
    """Source ends on a coarse vertex, dual edges, faces, interiors, the partial dual
    cells at the boundary, and two sources sharing entities; receivers on source cells."""
    n, c = (16, 16, 16), 4               # vertex coordinates 2, 6, 10, 14
    cells = [_idx(n, 2, 6, 10), _idx(n, 4, 2, 6), _idx(n, 3, 6, 5), _idx(n, 4, 4, 4),
             _idx(n, 0, 15, 1), _idx(n, 6, 0, 2), _idx(n, 5, 5, 5), _idx(n, 4, 2, 7),
             _idx(n, 14, 14, 13), _idx(n, 15, 15, 15)]
    pos = np.array(cells[0::2], dtype=np.int64)
    neg = np.array(cells[1::2], dtype=np.int64)
    rec = np.unique(np.concatenate([np.array(cells), np.arange(0, 4096, 37)])).astype(np.int64)
    prob = W.Problem(n=n, coarsen=c, src_pos=pos, src_neg=neg,
                     src_amp=np.array([1.0, -0.5, 2.0, 0.75, 1.25]), rec_cell=rec,
                     source_bases=True)
    m = W.gaussian_random_field(n, 0.25, 71)
    check_all(prob, m, dev, seed=72)


@pytest.mark.parametrize("window", ["shared", "global"])
def test_coarsening_16_and_factor_windows(dev, monkeypatch, window):
    """c = 16 in 3D factors in global memory; c = 8 with MSFV_LOCAL_WINDOW=global too."""
    if window == "global":
        monkeypatch.setenv("MSFV_LOCAL_WINDOW", "global")
        n, c = (24, 16, 16), 8
    else:
        n, c = (32, 32, 32), 16
    prob = W.make_problem(n, c, 3, 24, seed=81, top_layer=False, source_bases=True)
    m = W.gaussian_random_field(n, 0.2, 82)
    check_all(prob, m, dev, seed=83)


@pytest.mark.parametrize("solver", ["band", "mg", "nd"])
def test_both_coarse_solvers(dev, monkeypatch, solver):
    monkeypatch.setenv("MSFV_COARSE_SOLVER", solver)
    prob = W.make_problem((32, 32, 32), 4, 4, 40, seed=91, top_layer=True, source_bases=True)
    m = W.gaussian_random_field(prob.n, 0.2, 92)
    check_all(prob, m, dev, seed=93, derivs=False)


def test_workload_128_c8_with_source_bases(dev):
    """The 128^3, c = 8, 16-dipole, 512-receiver workload with source bases: data,
    fields and gradient against the oracle."""
    prob, m = W.config_3d_128()
    prob.source_bases = True
    check_all(prob, m, dev, seed=101, derivs=False)


def test_one_dimensional_problem_is_exact_on_gpu(dev):
    """sigma = sigma(x), one dipole per transverse cell between two planes off the
    vertex columns: the summed fields equal the fine solution (pinned gauge) computed by
    scipy, with no oracle involved."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    from paper_1707_07598_gb300.msfv import Session
    n, c, x1, x2 = (32, 16, 16), 8, 9, 22
    rng = np.random.default_rng(5)
    prof = rng.normal(0.0, 1.0, n[0])
    N = int(np.prod(n))
    X = np.stack(np.unravel_index(np.arange(N), n[::-1])[::-1], axis=1)
    m = prof[X[:, 0]]
    sel = np.nonzero(X[:, 0] == 0)[0]
    prob = W.Problem(n=n, coarsen=c, src_pos=sel + x1, src_neg=sel + x2,
                     src_amp=np.ones(len(sel)), rec_cell=np.arange(0, N, 5, dtype=np.int64),
                     source_bases=True)
    s = Session(prob)
    u = torch.empty((prob.n_src, N), dtype=torch.float64, device=dev)
    s.forward(torch.from_numpy(m).to(dev), u=u)
    u_ms = u.sum(dim=0).cpu().numpy()
    s.close()
    # fine finite-volume solve with harmonic face averages, u = 0 on coarse vertex 0
    sig = np.exp(m)
    st = [1, n[0], n[0] * n[1]]
    rows, cols, vals = [], [], []
    diag = np.zeros(N)
    for a in range(3):
        x = np.nonzero(X[:, a] < n[a] - 1)[0]
        y = x + st[a]
        geo = n[a] / np.prod([n[b] for b in range(3) if b != a])
        t = geo * 2 * sig[x] * sig[y] / (sig[x] + sig[y])
        rows += [x, y]
        cols += [y, x]
        vals += [-t, -t]
        np.add.at(diag, x, t)
        np.add.at(diag, y, t)
    A = sp.csc_matrix((np.concatenate(vals + [diag]),
                       (np.concatenate(rows + [np.arange(N)]), np.concatenate(cols + [np.arange(N)]))),
                      shape=(N, N))
    q = np.zeros(N)
    q[sel + x1] += 1.0
    q[sel + x2] -= 1.0
    pin = _idx(n, c // 2, c // 2, c // 2)
    keep = np.setdiff1d(np.arange(N), [pin])
    u_f = np.zeros(N)
    u_f[keep] = spla.splu(A[keep][:, keep]).solve(q[keep])
    assert np.abs(u_ms - u_f).max() <= 1e-10 * np.abs(u_f).max()


def test_repeatable_bitwise_and_recompute_rejected(dev):
    from paper_1707_07598_gb300.msfv import MSFVError, Session
    prob = W.make_problem((16, 16, 16), 4, 4, 20, seed=111, top_layer=False, source_bases=True)
    m = torch.from_numpy(W.gaussian_random_field(prob.n, 0.2, 112)).to(dev)
    s = Session(prob)
    d1 = s.forward(m).clone()
    _, g1 = s.adjoint(d1 * 1.01)
    g1 = g1.clone()
    d2 = s.forward(m)
    _, g2 = s.adjoint(d1 * 1.01)
    assert torch.equal(d1, d2) and torch.equal(g1, g2)
    s.close()
    with pytest.raises(MSFVError) as e:
        Session(prob, factor_mode=2)
    assert e.value.code == 1
