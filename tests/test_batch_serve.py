"""Batched (one CUDA graph over several instances) and served (continuous batching)
execution against the plain one-instance path and the oracle: each result must be the
same alone and in the mix."""
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


MIX = [((16, 16, 16), 8, 3, 20), ((24, 20), 4, 2, 12), ((32, 32, 32), 16, 2, 16),
       ((16, 16, 8), 4, 4, 10), ((20, 15), 5, 1, 8)]


def test_batch_graph_matches_plain_sessions_and_oracle(dev):
    from paper_1707_07598_gb300.msfv import Batch, Session
    probs, ms, dobs, refs, sessions = [], [], [], [], []
    for k, (n, c, ns, nr) in enumerate(MIX):
        prob = W.make_problem(n, c, ns, nr, seed=150 + k, top_layer=len(n) == 3)
        m = W.gaussian_random_field(n, 0.2, 160 + k)
        orc = Oracle(prob)
        st = orc.forward(m)
        d_obs = st['d'] * 1.02
        refs.append((st['d'], orc.misfit_gradient(st, d_obs)[1]))
        probs.append(prob)
        ms.append(torch.from_numpy(m).to(dev))
        dobs.append(torch.from_numpy(d_obs).to(dev))
        sessions.append(Session(prob, stream=torch.cuda.Stream(dev)))
    b = Batch(sessions, ms, dobs)
    for rep in range(2):                            # replays are identical
        b.run()
        b.check()
        for k in range(len(MIX)):
            assert rel(b.d_pred[k].cpu().numpy(), refs[k][0]) < TOL
            assert rel(b.grad[k].cpu().numpy(), refs[k][1]) < TOL
    # the same instances run alone on fresh sessions give the same bits
    for k, prob in enumerate(probs):
        s = Session(prob)
        d = s.forward(ms[k])
        _, g = s.adjoint(dobs[k], want_phi=False)
        assert torch.equal(d, b.d_pred[k]) and torch.equal(g, b.grad[k])
        s.close()
    # inputs refreshed in place are picked up by the next replay
    m2 = W.gaussian_random_field(MIX[0][0], 0.3, 199)
    ms[0].copy_(torch.from_numpy(m2).to(dev))
    b.run()
    b.check()
    st2 = Oracle(probs[0]).forward(m2)
    assert rel(b.d_pred[0].cpu().numpy(), st2['d']) < TOL
    b.close()
    for s in sessions:
        s.close()


FUSE_MIX = [((16, 16, 16), 8, 3, 20, {}), ((24, 16, 16), 8, 2, 12, {}),
            ((16, 16, 8), 8, 4, 10, {}), ((32, 32, 32), 16, 2, 16, {}),
            ((32, 16, 16), 16, 3, 16, {}), ((16, 16, 16), 4, 2, 9, {}),
            ((16, 16, 16), 8, 2, 12, {"source_bases": True}),
            ((16, 16, 16), 8, 2, 12, {"nodal": True})]


@pytest.mark.parametrize("fuse", ["1", "0"])
def test_fused_interior_launches_match_sessions_alone(dev, monkeypatch, fuse):
    """Instances that share a kernel shape have their dual-cell interiors (forward and
    adjoint) in one fused persistent launch; source-basis and nodal instances stay
    unfused in the same graph.  Every instance's data and gradient are the bits of the
    same session run alone, with and without fusion, and match the oracle."""
    from paper_1707_07598_gb300.msfv import Batch, Session
    monkeypatch.setenv("MSFV_BATCH_FUSE", fuse)
    probs, ms, dobs, sessions = [], [], [], []
    for k, (n, c, ns, nr, kw) in enumerate(FUSE_MIX):
        prob = W.make_problem(n, c, ns, nr, seed=170 + k, top_layer=True, **kw)
        probs.append(prob)
        ms.append(torch.from_numpy(W.gaussian_random_field(n, 0.2, 180 + k)).to(dev))
        sessions.append(Session(prob, stream=torch.cuda.Stream(dev)))
        dobs.append(torch.from_numpy(W.noise_like((ns, nr), 1e-3, 190 + k)).to(dev))
    torch.cuda.synchronize()
    b = Batch(sessions, ms, dobs)
    for _ in range(2):
        b.run()
        b.check()
    for k, prob in enumerate(probs):
        s = Session(prob)
        d = s.forward(ms[k])
        _, g = s.adjoint(dobs[k], want_phi=False)
        assert torch.equal(d, b.d_pred[k]) and torch.equal(g, b.grad[k]), k
        s.close()
    for k in (0, 3, 5):
        orc = Oracle(probs[k])
        st = orc.forward(ms[k].cpu().numpy())
        _, g_ref = orc.misfit_gradient(st, W.noise_like(st['d'].shape, 1e-3, 190 + k))
        assert rel(b.d_pred[k].cpu().numpy(), st['d']) < TOL
        assert rel(b.grad[k].cpu().numpy(), g_ref) < TOL
    b.close()
    for s in sessions:
        s.close()


def test_served_results_are_the_same_alone_and_in_the_mix(dev):
    from paper_1707_07598_gb300.serve import GpuBackend, Server
    reqs = W.served_requests(rate=400.0, duration=0.08, seed=11, sizes=(16, 32),
                             coarsenings=(4, 8), max_src=6, p_new_client=0.4)
    assert len(reqs) >= 10 and len({q.client for q in reqs}) >= 3
    mixed = Server(GpuBackend(dev), budget_bytes=8 << 30, max_inflight=8,
                   keep_results=True).run(reqs)
    alone = Server(GpuBackend(dev, use_graph=False), budget_bytes=8 << 30, max_inflight=1,
                   keep_results=True).run(reqs)
    a = {r.rid: r for r in alone.records}
    assert all(r.status == "done" for r in mixed.records)
    for r in mixed.records:
        (d1, g1), (d2, g2) = r.result, a[r.rid].result
        assert rel(d1, d2) <= 1e-12 and rel(g1, g2) <= 1e-12
    # the one-at-a-time run never overlaps two requests
    iv = sorted((r.start, r.finish) for r in alone.records)
    assert all(s1 >= f0 for (s0, f0), (s1, f1) in zip(iv, iv[1:]))


def test_served_request_matches_oracle(dev):
    """One served request's inputs, rebuilt on the host, against the oracle."""
    from paper_1707_07598_gb300.serve import GpuBackend, Server
    reqs = W.served_requests(rate=200.0, duration=0.03, seed=12, sizes=(16,),
                             coarsenings=(4,), max_src=3, p_new_client=1.0)
    st = Server(GpuBackend(dev), budget_bytes=4 << 30, keep_results=True).run(reqs[:2])
    r0 = st.records[0]
    spec = reqs[0].instance
    prob = spec.problem()
    m0 = W.gaussian_random_field_device(prob.n, spec.corr_len, spec.seed, dev)
    g = torch.Generator(device=dev)
    g.manual_seed(spec.seed + 1)
    dm = torch.randn(prob.N, generator=g, device=dev, dtype=torch.float64)
    d_obs = 1e-3 * torch.randn((prob.n_src, prob.n_rec), generator=g, device=dev,
                               dtype=torch.float64)
    m = (m0 + 0.01 * reqs[0].iteration * dm).cpu().numpy()
    orc = Oracle(prob)
    sto = orc.forward(m)
    _, gref = orc.misfit_gradient(sto, d_obs.cpu().numpy())
    assert rel(r0.result[0], sto['d']) < TOL and rel(r0.result[1], gref) < TOL


def test_batch_and_autograd_carry_the_variants(dev):
    """A graph batch mixing a plain session, one with source bases and one of the nodal
    variant gives each the bits it gets alone; the autograd binding's gradient on the
    variants matches their oracles."""
    from oracle.galerkin_oracle import NodalOracle
    from paper_1707_07598_gb300.autograd import misfit
    from paper_1707_07598_gb300.msfv import Batch, Session
    probs = [W.make_problem((16, 16, 16), 8, 3, 20, seed=170, top_layer=True),
             W.make_problem((16, 16, 16), 4, 3, 20, seed=171, top_layer=False, source_bases=True),
             W.make_problem((16, 16, 16), 4, 3, 20, seed=172, top_layer=False, nodal=True)]
    ms, dobs, sessions, refs = [], [], [], []
    for k, prob in enumerate(probs):
        m = W.gaussian_random_field(prob.n, 0.2, 180 + k)
        orc = NodalOracle(prob) if prob.nodal else Oracle(prob)
        st = orc.forward(m)
        d_obs = st['d'] * 1.02
        refs.append((st['d'], orc.misfit_gradient(st, d_obs)[1]))
        ms.append(torch.from_numpy(m).to(dev))
        dobs.append(torch.from_numpy(d_obs).to(dev))
        sessions.append(Session(prob, stream=torch.cuda.Stream(dev)))
    b = Batch(sessions, ms, dobs)
    b.run()
    b.check()
    for k, prob in enumerate(probs):
        assert rel(b.d_pred[k].cpu().numpy(), refs[k][0]) < TOL
        assert rel(b.grad[k].cpu().numpy(), refs[k][1]) < TOL
        s = Session(prob)
        d = s.forward(ms[k])
        _, g = s.adjoint(dobs[k], want_phi=False)
        assert torch.equal(d, b.d_pred[k]) and torch.equal(g, b.grad[k])
        mm = ms[k].clone().requires_grad_(True)
        misfit(mm, dobs[k], s).backward()
        assert rel(mm.grad.cpu().numpy(), refs[k][1]) < TOL
        s.close()
    b.close()
    for s in sessions:
        s.close()
