"""Full-size checks of the batched path on the largest instances of the default benchmark
line (192^3 with c = 16 and c = 8, 128^3 with c = 4), run as one batch graph with the fused
dual-cell interior launches the benchmark times.  The oracle takes hours at these sizes,
so the checks are properties that hold at any size:

* conservation of the reduced solution: R (A u_j - q_j) = 0 on every primal coarse cell
  (Sec. 3.1, Eq. reducedPDE with the finite-volume restriction R; the pinned row follows
  from the zero column sums of A and sum q_j = 0), with A assembled by the oracle's own
  fine operator from the oracle's transmissibilities;
* bit-equality of the batch's data and gradient with the plain one-instance path;
* the gradient equals J^T r, and <w, J v> = <J^T w, v> (Sec. 4.3, Eq. sensred);
* central differences of the misfit along random directions (step 1e-6)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.msfv_oracle import cell_coords, fine_operator, strides_of, transmissibility  # noqa: E402
from paper_1707_07598_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

INSTANCES = [((192, 192, 192), 16, 8, 256), ((192, 192, 192), 8, 8, 256),
             ((128, 128, 128), 4, 8, 256)]


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1707_07598_gb300 import build
    build.build()
    return torch.device("cuda:0")


def coarse_residual(prob, m, U):
    """max_j ||R (A u_j - q_j)|| / ||R q_j|| with the oracle's operator (host, FP64)."""
    n = tuple(prob.n)
    T, _, _ = transmissibility(m, n)
    A = fine_operator(T, n)
    coords = cell_coords(n)
    cst = strides_of(tuple(v // prob.coarsen for v in n))
    cidx = np.zeros(prob.N, dtype=np.int64)
    for a in range(len(n)):
        cidx += (coords[:, a] // prob.coarsen) * cst[a]
    Nc = int(np.prod([v // prob.coarsen for v in n]))
    worst = 0.0
    for j in range(prob.n_src):
        q = np.zeros(prob.N)
        q[prob.src_pos[j]] += prob.src_amp[j]
        q[prob.src_neg[j]] -= prob.src_amp[j]
        Rq = np.bincount(cidx, weights=q, minlength=Nc)
        res = np.bincount(cidx, weights=A @ U[j] - q, minlength=Nc)
        worst = max(worst, float(np.linalg.norm(res) / np.linalg.norm(Rq)))
    return worst


def test_batched_full_size_instances(dev):
    from paper_1707_07598_gb300.msfv import Batch, Session
    probs, ms, dobs, sessions = [], [], [], []
    for k, (n, c, ns, nr) in enumerate(INSTANCES):
        prob = W.make_problem(n, c, ns, nr, seed=300 + k, top_layer=True)
        probs.append(prob)
        ms.append(W.gaussian_random_field_device(prob.n, 0.1, 310 + k, dev))
        sessions.append(Session(prob, stream=torch.cuda.Stream(dev)))
        dobs.append(torch.from_numpy(W.noise_like((ns, nr), 1e-3, 320 + k)).to(dev))
    torch.cuda.synchronize()
    b = Batch(sessions, ms, dobs)
    b.run()
    b.check()
    info = b.info()
    assert info["fused_instances"] == len(INSTANCES) and info["fused_groups"] == 3
    # the checks below use torch ops on the current stream: run the sessions there too
    for s in sessions:
        s.set_stream(torch.cuda.current_stream(dev))
    for k, prob in enumerate(probs):
        s = sessions[k]
        u = torch.empty((prob.n_src, prob.N), dtype=torch.float64, device=dev)
        d = s.forward(ms[k], u=u)
        _, g = s.adjoint(dobs[k], want_phi=False)
        # the batch graph (fused launches) and the plain path give the same bits
        assert torch.equal(d, b.d_pred[k]) and torch.equal(g, b.grad[k]), k
        # conservation of the reduced solution on every primal coarse cell
        assert coarse_residual(prob, ms[k].cpu().numpy(), u.cpu().numpy()) < 1e-9, k
        # the gradient is J^T r, and J and J^T are adjoint
        jtr = s.jtvec((d - dobs[k]).contiguous())
        assert float((jtr - g).norm()) <= 1e-12 * float(g.norm()), k
        v = torch.from_numpy(W.noise_like(prob.N, 1.0, 330 + k)).to(dev)
        w = torch.from_numpy(W.noise_like((prob.n_src, prob.n_rec), 1.0, 340 + k)).to(dev)
        jv = s.jvec(v)
        jtw = s.jtvec(w)
        lhs, rhs = float((w * jv).sum()), float(jtw @ v)
        assert abs(lhs - rhs) <= 1e-10 * float(w.norm() * jv.norm()), k
    # central differences of the misfit on the c = 16 instance (the dominant kernel)
    s, prob, m0, d_obs = sessions[0], probs[0], ms[0], dobs[0]
    s.forward(m0)
    _, g = s.adjoint(d_obs, want_phi=False)

    def misfit(mm):
        dd = s.forward(mm)
        return 0.5 * float(((dd - d_obs) ** 2).sum())

    for r in range(2):
        v = torch.from_numpy(W.noise_like(prob.N, 1.0, 350 + r)).to(dev)
        fd = (misfit(m0 + 1e-6 * v) - misfit(m0 - 1e-6 * v)) / 2e-6
        an = float(g @ v)
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3 * float(g.norm() * v.norm()))
    b.close()
    for s in sessions:
        s.close()
