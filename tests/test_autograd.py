"""torch.autograd.Function bindings (misfit gradient, J^T w, forward-mode J v) against the
CPU oracle, central finite differences on the GPU, and the linearisation-point
bookkeeping.  Stored and recomputed local factors, c = 8 (shared-memory factor windows)
and c = 16 (global-memory windows)."""
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


@pytest.mark.parametrize("fm", [1, 2])
@pytest.mark.parametrize("n,c,ns,nr", [((16, 16, 16), 8, 3, 20), ((32, 32, 32), 16, 2, 16),
                                       ((24, 20), 4, 2, 12)])
def test_autograd_matches_oracle(dev, fm, n, c, ns, nr):
    from paper_1707_07598_gb300.autograd import misfit, predict
    from paper_1707_07598_gb300.msfv import Session
    prob = W.make_problem(n, c, ns, nr, seed=101, top_layer=len(n) == 3)
    m_np = W.gaussian_random_field(n, 0.2, 102)
    orc = Oracle(prob)
    st = orc.forward(m_np)
    d_obs_np = st['d'] * 1.03
    phi_ref, g_ref = orc.misfit_gradient(st, d_obs_np)
    s = Session(prob, factor_mode=fm)
    m = torch.from_numpy(m_np).to(dev).requires_grad_(True)
    d_obs = torch.from_numpy(d_obs_np).to(dev).requires_grad_(True)
    phi = misfit(m, d_obs, s)
    phi.backward()
    assert abs(phi.item() - phi_ref) <= TOL * abs(phi_ref)
    assert rel(m.grad.cpu().numpy(), g_ref) < TOL
    assert rel(d_obs.grad.cpu().numpy(), -(st['d'] - d_obs_np)) < TOL
    # vector-Jacobian product of the data map
    w_np = W.noise_like((prob.n_src, prob.n_rec), 1.0, 103)
    m2 = torch.from_numpy(m_np).to(dev).requires_grad_(True)
    d = predict(m2, s)
    assert rel(d.detach().cpu().numpy(), st['d']) < TOL
    d.backward(torch.from_numpy(w_np).to(dev))
    assert rel(m2.grad.cpu().numpy(), orc.jtvec(st, w_np)) < TOL
    # forward-mode Jacobian-vector product
    import torch.autograd.forward_ad as fwAD
    v_np = W.noise_like(prob.N, 1.0, 104)
    with fwAD.dual_level():
        md = fwAD.make_dual(torch.from_numpy(m_np).to(dev), torch.from_numpy(v_np).to(dev))
        jv = fwAD.unpack_dual(predict(md, s)).tangent
    assert rel(jv.cpu().numpy(), orc.jvec(st, v_np)) < TOL
    s.close()


def test_backward_after_a_later_forward_relinearises(dev):
    """A backward whose forward was superseded on the same session uses its own m."""
    from paper_1707_07598_gb300.autograd import predict
    from paper_1707_07598_gb300.msfv import Session
    prob = W.make_problem((16, 16, 16), 8, 2, 12, seed=111, top_layer=True)
    m1_np = W.gaussian_random_field(prob.n, 0.2, 112)
    m2_np = W.gaussian_random_field(prob.n, 0.2, 113)
    orc = Oracle(prob)
    st1 = orc.forward(m1_np)
    s = Session(prob)
    m1 = torch.from_numpy(m1_np).to(dev).requires_grad_(True)
    d1 = predict(m1, s)
    s.forward(torch.from_numpy(m2_np).to(dev))        # moves the session to m2
    w_np = W.noise_like((prob.n_src, prob.n_rec), 1.0, 114)
    d1.backward(torch.from_numpy(w_np).to(dev))
    assert rel(m1.grad.cpu().numpy(), orc.jtvec(st1, w_np)) < TOL
    s.close()


@pytest.mark.parametrize("fm", [1, 2])
def test_misfit_gradient_central_differences_c16(dev, fm):
    """Central differences (step 1e-6) along 20 random directions, 64^3, c = 16."""
    from paper_1707_07598_gb300.autograd import misfit
    from paper_1707_07598_gb300.msfv import Session
    prob = W.make_problem((64, 64, 64), 16, 8, 128, seed=121, top_layer=True)
    m_np = W.gaussian_random_field(prob.n, 0.15, 122)
    s = Session(prob, factor_mode=fm)
    m0 = torch.from_numpy(m_np).to(dev)
    d_obs = s.forward(m0) * 1.05
    m = m0.clone().requires_grad_(True)
    phi = misfit(m, d_obs, s)
    phi.backward()
    g = m.grad.detach()

    def f(mm):
        with torch.no_grad():
            return misfit(mm, d_obs, s).item()
    for k in range(20):
        v = torch.from_numpy(W.noise_like(prob.N, 1.0, 200 + k)).to(dev)
        fd = (f(m0 + 1e-6 * v) - f(m0 - 1e-6 * v)) / 2e-6
        an = float(g @ v)
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3 * float(g.norm() * v.norm()))
    s.close()
