"""Gauss-Newton-CG inversion step (msfv_gn_step) against the oracle's step, and an
end-to-end inversion of the two-block model with 1% noise (Sec. 5)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.gn_oracle import gn_step  # noqa: E402
from oracle.msfv_oracle import Oracle  # noqa: E402
from paper_1707_07598_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1707_07598_gb300 import build
    build.build()
    return torch.device("cuda:0")


@pytest.mark.parametrize("n,c,ns,nr,alpha", [((16, 16), 4, 2, 12, 1e-3),
                                             ((12, 12, 8), 4, 3, 16, 1e-4)])
def test_gn_step_matches_oracle(dev, n, c, ns, nr, alpha):
    from paper_1707_07598_gb300.msfv import Session
    prob = W.make_problem(n, c, ns, nr, seed=171, top_layer=len(n) == 3)
    m_true = W.block_model(n)
    orc = Oracle(prob)
    d_obs = orc.forward(m_true)['d']
    d_obs = d_obs + 0.01 * np.abs(d_obs) * W.noise_like(d_obs.shape, 1.0, 172)
    m0 = np.zeros(prob.N)
    mref = W.noise_like(prob.N, 0.1, 173)
    m_or, st_or = gn_step(orc, m0, d_obs, alpha, m_ref=mref, cg_iters=6, cg_tol=1e-12)
    s = Session(prob)
    m = torch.from_numpy(m0).to(dev)
    st = s.gn_step(m, torch.from_numpy(d_obs).to(dev), alpha,
                   m_ref=torch.from_numpy(mref).to(dev), cg_iters=6, cg_tol=1e-12)
    for k in ("phi_d0", "phi_r0", "grad_norm"):
        assert abs(st[k] - st_or[k]) <= 1e-9 * abs(st_or[k])
    assert st["cg_iters"] == st_or["cg_iters"] and st["step"] == st_or["step"]
    assert rel(m.cpu().numpy(), m_or) < 1e-7
    assert abs(st["phi_d1"] - st_or["phi_d1"]) <= 1e-7 * abs(st_or["phi_d1"])
    s.close()


def test_two_block_inversion_reduces_the_misfit(dev):
    """Five Gauss-Newton iterations from a homogeneous start recover enough of the two
    conductive blocks to reduce the data misfit by more than 10x."""
    from paper_1707_07598_gb300.inversion import gauss_newton
    from paper_1707_07598_gb300.msfv import Session
    n = (32, 32, 32)
    prob = W.make_problem(n, 8, 8, 256, seed=181, top_layer=True)
    s = Session(prob)
    d_true = s.forward(torch.from_numpy(W.block_model(n)).to(dev))
    noise = torch.from_numpy(W.noise_like(tuple(d_true.shape), 1.0, 182)).to(dev)
    d_obs = (d_true + 0.01 * d_true.abs() * noise).contiguous()
    m = torch.zeros(prob.N, dtype=torch.float64, device=dev)
    hist = gauss_newton(s, m, d_obs, iters=5, alpha=1e-8, cg_iters=10)
    assert len(hist) >= 3
    phis = [h["phi_d0"] for h in hist] + [hist[-1]["phi_d1"]]
    assert all(b <= a for a, b in zip(phis, phis[1:]))      # monotone (Armijo)
    assert phis[-1] < 0.1 * phis[0]
    assert float(m.abs().max()) <= 10.0
    s.close()
