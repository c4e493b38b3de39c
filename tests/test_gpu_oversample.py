"""GPU path with oversampled dual edge and face problems against the CPU oracle.

Oversampling is named in Sec. 6 as a way to lessen the effect of the local boundary
conditions on the basis; the library and the oracle implement the same reading (a dual
edge or face solved on its box widened by w cells along its normal axes, only its own
cells kept).  Bar: 1e-9 relative error in the 2-norm and the max-norm on predicted
data, fields u, misfit, gradient, J v and J^T w.  Cases: 2D and 3D, several dual cells
per axis with partial dual cells at the boundary, widths from 1 to c - 1 (boxes that
reach the neighbouring vertex planes' cells and boxes clipped by the mesh), c = 4, 8
and 16, and a 64^3 case with c = 8; the shared-memory box kernels and the global-memory
ones (boxes too large for shared memory, or forced).  Also: the gradient is bitwise
repeatable (the overlapping boxes' contributions are gathered in a fixed order), a batch
graph with oversampled instances gives the plain path's bits, invalid widths are
rejected, and the benchmark's own 128^3 configuration passes checks that hold at any
size."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.msfv_oracle import Oracle  # noqa: E402
from paper_1707_07598_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-9


def rel(a, b):
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


CASES = [
    ((48, 40), 8, 1, 3, 20),
    ((48, 40), 8, 3, 2, 20),
    ((40, 24), 8, 7, 2, 16),
    ((20, 15), 5, 2, 2, 8),
    ((12, 8, 8), 4, 1, 2, 9),
    ((24, 16, 16), 8, 2, 3, 24),
    ((24, 24, 16), 8, 7, 2, 20),
    ((16, 16, 12), 4, 3, 2, 12),
    ((32, 32, 32), 16, 3, 2, 24),
    # face boxes too large for shared memory (global-memory kernels), edge boxes in it
    ((32, 32, 32), 16, 5, 2, 24),
]


@pytest.mark.parametrize("n,c,w,ns,nr", CASES)
def test_oversampled_forward_gradient_jvec_jtvec_match_oracle(dev, n, c, w, ns, nr):
    from paper_1707_07598_gb300.msfv import Session
    prob = W.make_problem(n, c, ns, nr, seed=31, top_layer=len(n) == 3, oversample=w)
    m = 1.5 * W.gaussian_random_field(n, 0.15, 32)
    orc = Oracle(prob)
    st = orc.forward(m)
    d_obs = st['d'] * 1.02 + W.noise_like(st['d'].shape, 1e-3 * np.abs(st['d']).max(), 33)
    phi_ref, g_ref = orc.misfit_gradient(st, d_obs)
    s = Session(prob)
    u = torch.empty((prob.n_src, prob.N), dtype=torch.float64, device=dev)
    d = s.forward(torch.from_numpy(m).to(dev), u=u)
    phi, g = s.adjoint(torch.from_numpy(d_obs).to(dev))
    assert rel(d.cpu().numpy(), st['d']) < TOL
    assert rel(u.cpu().numpy(), st['U']) < TOL
    assert abs(phi - phi_ref) <= TOL * abs(phi_ref)
    assert rel(g.cpu().numpy(), g_ref) < TOL
    v = W.noise_like(prob.N, 1.0, 34)
    wt = W.noise_like((prob.n_src, prob.n_rec), 1.0, 35)
    jv = s.jvec(torch.from_numpy(v).to(dev)).cpu().numpy()
    jtw = s.jtvec(torch.from_numpy(wt).to(dev)).cpu().numpy()
    assert rel(jv, orc.jvec(st, v)) < TOL
    assert rel(jtw, orc.jtvec(st, wt)) < TOL
    s.close()


@pytest.mark.parametrize("n,c,w", [((24, 16, 16), 8, 2), ((40, 24), 8, 3)])
def test_oversampled_global_memory_kernels_match_oracle(dev, n, c, w, monkeypatch):
    """MSFV_OVER_GLOBAL=1 at set-up: the global-memory box kernels where the shared-memory
    ones would run."""
    from paper_1707_07598_gb300.msfv import Session
    monkeypatch.setenv("MSFV_OVER_GLOBAL", "1")
    prob = W.make_problem(n, c, 2, 16, seed=81, top_layer=False, oversample=w)
    m = W.gaussian_random_field(n, 0.15, 82)
    orc = Oracle(prob)
    st = orc.forward(m)
    d_obs = st['d'] * 1.01
    _, g_ref = orc.misfit_gradient(st, d_obs)
    s = Session(prob)
    d = s.forward(torch.from_numpy(m).to(dev))
    _, g = s.adjoint(torch.from_numpy(d_obs).to(dev))
    v = W.noise_like(prob.N, 1.0, 83)
    jv = s.jvec(torch.from_numpy(v).to(dev)).cpu().numpy()
    assert rel(d.cpu().numpy(), st['d']) < TOL
    assert rel(g.cpu().numpy(), g_ref) < TOL
    assert rel(jv, orc.jvec(st, v)) < TOL
    s.close()


def test_oversampled_64cube_matches_oracle(dev):
    from paper_1707_07598_gb300.msfv import Session
    n, c, w = (64, 64, 64), 8, 2
    prob = W.make_problem(n, c, 4, 64, seed=41, top_layer=True, oversample=w)
    m = W.gaussian_random_field(n, 0.1, 42)
    orc = Oracle(prob)
    st = orc.forward(m)
    d_obs = st['d'] * 1.01
    phi_ref, g_ref = orc.misfit_gradient(st, d_obs)
    s = Session(prob)
    d = s.forward(torch.from_numpy(m).to(dev))
    phi, g = s.adjoint(torch.from_numpy(d_obs).to(dev))
    assert rel(d.cpu().numpy(), st['d']) < TOL
    assert abs(phi - phi_ref) <= TOL * abs(phi_ref)
    assert rel(g.cpu().numpy(), g_ref) < TOL
    # the contributions of overlapping boxes are summed in a fixed order: same bits
    _, g2 = s.adjoint(torch.from_numpy(d_obs).to(dev))
    assert torch.equal(g, g2)
    s.close()


def test_oversampled_instances_in_a_batch_graph_match_the_plain_path(dev):
    from paper_1707_07598_gb300.msfv import Batch, Session
    probs = [W.make_problem((32, 32, 32), 8, 3, 24, seed=51, top_layer=True, oversample=2),
             W.make_problem((48, 40), 8, 2, 16, seed=52, top_layer=False, oversample=3),
             W.make_problem((32, 32, 32), 8, 3, 24, seed=53, top_layer=True)]
    ms = [torch.from_numpy(W.gaussian_random_field(p.n, 0.15, 60 + k)).to(dev)
          for k, p in enumerate(probs)]
    dobs = [torch.from_numpy(W.noise_like((p.n_src, p.n_rec), 1e-3, 70 + k)).to(dev)
            for k, p in enumerate(probs)]
    sessions = [Session(p, stream=torch.cuda.Stream(dev)) for p in probs]
    torch.cuda.synchronize()
    b = Batch(sessions, ms, dobs)
    b.run()
    b.check()
    for s in sessions:
        s.set_stream(torch.cuda.current_stream(dev))
    for k, s in enumerate(sessions):
        d = s.forward(ms[k])
        _, g = s.adjoint(dobs[k], want_phi=False)
        assert torch.equal(d, b.d_pred[k]) and torch.equal(g, b.grad[k]), k
    b.close()
    for s in sessions:
        s.close()


def test_invalid_oversampling_is_rejected(dev):
    from paper_1707_07598_gb300.msfv import MSFVError, Session
    for kw in (dict(oversample=8), dict(oversample=-1),
               dict(oversample=1, source_bases=True), dict(oversample=1, nodal=True)):
        prob = W.make_problem((16, 16), 8, 1, 4, seed=1, top_layer=False, **kw)
        with pytest.raises(MSFVError):
            Session(prob)


def test_oversampled_bench_configuration_properties(dev):
    """The configuration the oversampled benchmark line times (128^3, c = 8, 16 dipoles,
    512 receivers, w = 2), checked by properties that hold at any size (the oracle takes
    minutes here; it is compared element by element up to 64^3 above):

    * a conductivity that varies along one axis only gives the plain method's data (the
      widened solutions are constant along the normal axes; pinned on the oracle in
      tests/test_oracle_oversample.py);
    * on the benchmark's model the gradient equals J^T r and <w, J v> = <J^T w, v>
      (Sec. 4.3, Eq. sensred);
    * the gradient is bitwise repeatable."""
    from paper_1707_07598_gb300.msfv import Session
    prob, m_np = W.config_3d_128()
    N = prob.N
    z = np.arange(N) // (prob.n[0] * prob.n[1])
    layer = np.random.default_rng(91).normal(0.0, 1.5, prob.n[2])
    m1 = torch.from_numpy(layer[z]).to(dev)
    s0 = Session(prob)
    d_plain = s0.forward(m1).clone()
    s0.close()
    prob.oversample = 2
    s = Session(prob)
    d_over = s.forward(m1)
    # the same basis up to rounding; the coarse solve amplifies rounding by its condition
    assert rel(d_over.cpu().numpy(), d_plain.cpu().numpy()) < 1e-8
    m = torch.from_numpy(m_np).to(dev)
    d = s.forward(m)
    d_obs = d * 1.01
    _, g = s.adjoint(d_obs, want_phi=False)
    _, g2 = s.adjoint(d_obs, want_phi=False)
    assert torch.equal(g, g2)
    jtr = s.jtvec((d - d_obs).contiguous())
    assert float((jtr - g).norm()) <= 1e-12 * float(g.norm())
    v = torch.from_numpy(W.noise_like(N, 1.0, 92)).to(dev)
    w = torch.from_numpy(W.noise_like((prob.n_src, prob.n_rec), 1.0, 93)).to(dev)
    jv = s.jvec(v)
    jtw = s.jtvec(w)
    lhs, rhs = float((w * jv).sum()), float(jtw @ v)
    assert abs(lhs - rhs) <= 1e-10 * float(w.norm() * jv.norm())
    s.close()
