"""The paper's own variant on the GPU (nodal operator, Lagrange data on primal blocks,
Galerkin A_k = S^T A S, X_k term), through the C ABI, against the nodal oracle.

Bar: 1e-9 relative 2-norm on d, the nodal fields u, the misfit gradient, J v, J^T w and
the fixed-basis J^T w.  Cases: 2D and 3D, c in {1, 2, 3, 4, 5, 8}, non-cubic meshes,
sources and receivers inside blocks (the X_k term is live there) and on block faces,
both coarse solvers, a 64^3 surface survey; bitwise repeatability."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.galerkin_oracle import NodalOracle  # noqa: E402
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


def check_all(prob, m, dev, seed=0, derivs=True):
    from paper_1707_07598_gb300.msfv import Session
    orc = NodalOracle(prob)
    st = orc.forward(m)
    d_obs = st['d'] * 1.02 + W.noise_like(st['d'].shape, 1e-3 * np.abs(st['d']).max(), seed + 1)
    phi_ref, g_ref = orc.misfit_gradient(st, d_obs)
    s = Session(prob)
    mt = torch.from_numpy(m).to(dev)
    u = torch.empty((prob.n_src, s.Nf), dtype=torch.float64, device=dev)
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


CASES = [
    ((16, 16), 4, 3, 12),
    ((24, 16), 8, 2, 12),
    ((18, 18), 3, 3, 10),
    ((20, 15), 5, 2, 8),
    ((16, 12), 2, 3, 9),
    ((8, 8), 1, 2, 6),
    ((8, 8, 8), 4, 3, 12),
    ((12, 8, 8), 4, 2, 9),
    ((9, 9, 6), 3, 3, 9),
    ((16, 16, 16), 8, 4, 20),
    ((8, 6, 4), 2, 3, 8),
    ((4, 4, 4), 1, 2, 6),
]


@pytest.mark.parametrize("n,c,ns,nr", CASES)
def test_nodal_variant_matches_oracle(dev, n, c, ns, nr):
    prob = W.make_problem(n, c, ns, nr, seed=71, top_layer=False, nodal=True)
    m = W.gaussian_random_field(n, 0.2, 72)
    check_all(prob, m, dev, seed=73)


def test_surface_survey_64(dev):
    """64^3 cells, c = 8, 8 dipoles and 128 receivers on the top surface."""
    prob = W.make_problem((64, 64, 64), 8, 8, 128, seed=81, top_layer=True, nodal=True)
    m = W.gaussian_random_field(prob.n, 0.15, 82)
    check_all(prob, m, dev, seed=83, derivs=False)


@pytest.mark.parametrize("solver", ["band", "mg", "nd"])
def test_both_coarse_solvers(dev, monkeypatch, solver):
    monkeypatch.setenv("MSFV_COARSE_SOLVER", solver)
    prob = W.make_problem((32, 32, 32), 4, 3, 40, seed=91, top_layer=False, nodal=True)
    m = W.gaussian_random_field(prob.n, 0.2, 92)
    check_all(prob, m, dev, seed=93, derivs=False)


def test_repeatable_bitwise(dev):
    from paper_1707_07598_gb300.msfv import Session
    prob = W.make_problem((16, 16, 16), 4, 3, 20, seed=101, top_layer=False, nodal=True)
    m = torch.from_numpy(W.gaussian_random_field(prob.n, 0.2, 102)).to(dev)
    s = Session(prob)
    d1 = s.forward(m).clone()
    _, g1 = s.adjoint(d1 * 1.01)
    g1 = g1.clone()
    d2 = s.forward(m)
    _, g2 = s.adjoint(d1 * 1.01)
    assert torch.equal(d1, d2) and torch.equal(g1, g2)
    s.close()


@pytest.mark.parametrize("n,c,k_fine,k_lagrange", [((36, 36, 12), 12, 17797, 32),
                                                   ((36, 36, 12), 6, 17797, 147),
                                                   ((64, 64, 32), 16, 139425, 75),
                                                   ((64, 64, 32), 8, 139425, 405)])
def test_session_sizes_match_the_paper(dev, n, c, k_fine, k_lagrange):
    """The library's nodal sessions on the paper's two meshes have its fine system sizes
    (Sec. 5.1, Tab. 1: 17,797; Sec. 5.2, Tab. 2: 139,425) and as many coarse unknowns as
    the Lagrange part of its k (150 - 25 - 93 = 32 and 572 - 25 - 400 = 147 on the block
    model; 1009 - 72 - 862 = 75 and 4415 - 72 - 3938 = 405 on the SEG model)."""
    from paper_1707_07598_gb300.msfv import Session
    prob = W.make_problem(n, c, 2, 4, seed=1, nodal=True)
    s = Session(prob)
    info = s.info()
    assert info["N"] == k_fine and info["Nc"] == k_lagrange
    s.close()
