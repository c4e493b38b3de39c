"""GPU path (through the C ABI) against the CPU oracle, element by element.

Bar: 1e-9 relative error, in the 2-norm and in the max-norm, on predicted data, fields
u, misfit, gradient, J v and J^T w (all FP64 on both sides).  Cases span several dual cells per axis, partial
dual cells at the boundary, odd and even coarsening, c = 1, non-cubic meshes,
repeated receivers, sources and receivers on vertex / edge cells, and the full
2D 64x64 and 3D 128^3 workloads."""
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


CASES = [
    ((16, 16), 4, 2, 9),
    ((24, 16), 8, 3, 12),
    ((18, 18), 3, 2, 10),
    ((20, 15), 5, 2, 8),
    ((16, 12), 2, 2, 7),
    ((8, 8), 1, 2, 5),
    ((32, 32), 8, 1, 32),
    ((8, 8, 8), 4, 2, 9),
    ((12, 8, 8), 4, 2, 9),
    ((9, 9, 6), 3, 2, 7),
    ((16, 16, 16), 8, 3, 20),
    ((10, 10, 10), 5, 2, 8),
    ((8, 6, 4), 2, 2, 6),
    ((4, 4, 4), 1, 1, 4),
    ((24, 16, 16), 8, 4, 30),
]


def run_pair(prob, m, dev, seed=0, factor_mode=0):
    orc = Oracle(prob)
    st = orc.forward(m)
    d_obs = st['d'] * 1.02 + W.noise_like(st['d'].shape, 1e-3 * np.abs(st['d']).max(), seed + 1)
    phi_ref, g_ref = orc.misfit_gradient(st, d_obs)
    from paper_1707_07598_gb300.msfv import Session
    s = Session(prob, factor_mode=factor_mode)
    mt = torch.from_numpy(m).to(dev)
    u = torch.empty((prob.n_src, prob.N), dtype=torch.float64, device=dev)
    d = s.forward(mt, u=u)
    phi, g = s.adjoint(torch.from_numpy(d_obs).to(dev))
    torch.cuda.synchronize()
    return orc, st, s, d.cpu().numpy(), u.cpu().numpy(), phi, g.cpu().numpy(), d_obs, phi_ref, g_ref


@pytest.mark.parametrize("n,c,ns,nr", CASES)
def test_forward_and_gradient_match_oracle(dev, n, c, ns, nr):
    prob = W.make_problem(n, c, ns, nr, seed=11, top_layer=len(n) == 3)
    m = W.gaussian_random_field(n, 0.2, 12)
    orc, st, s, d, u, phi, g, d_obs, phi_ref, g_ref = run_pair(prob, m, dev)
    assert rel(d, st['d']) < TOL
    assert rel(u, st['U']) < TOL
    assert abs(phi - phi_ref) <= TOL * abs(phi_ref)
    assert rel(g, g_ref) < TOL
    s.close()


@pytest.mark.parametrize("n,c,ns,nr", [((16, 16), 4, 2, 9), ((20, 15), 5, 2, 8),
                                       ((8, 8, 8), 4, 2, 9), ((9, 9, 6), 3, 2, 7),
                                       ((16, 16, 16), 8, 3, 20)])
def test_jvec_and_jtvec_match_oracle(dev, n, c, ns, nr):
    prob = W.make_problem(n, c, ns, nr, seed=13, top_layer=False)
    m = W.gaussian_random_field(n, 0.25, 14)
    orc = Oracle(prob)
    st = orc.forward(m)
    from paper_1707_07598_gb300.msfv import Session
    s = Session(prob)
    s.forward(torch.from_numpy(m).to(dev))
    v = W.noise_like(prob.N, 1.0, 15)
    w = W.noise_like((prob.n_src, prob.n_rec), 1.0, 16)
    jv = s.jvec(torch.from_numpy(v).to(dev)).cpu().numpy()
    jtw = s.jtvec(torch.from_numpy(w).to(dev)).cpu().numpy()
    assert rel(jv, orc.jvec(st, v)) < TOL
    assert rel(jtw, orc.jtvec(st, w)) < TOL
    # adjoint consistency on the GPU alone
    assert abs(np.sum(w * jv) - jtw @ v) <= 1e-12 * np.linalg.norm(w) * np.linalg.norm(jv) * 10
    s.close()


def test_repeated_receivers_and_vertex_sources(dev):
    n, c = (16, 16, 8), 4
    base = W.make_problem(n, c, 2, 6, seed=3, top_layer=False)
    # vertex cell (2,2,2): c*0 + 2 on each axis; an edge cell next to it
    vert = 2 + 16 * 2 + 256 * 2
    rec = np.array([vert, vert, vert + 1, 5, 5, 77, 200], dtype=np.int64)
    prob = W.Problem(n=n, coarsen=c, src_pos=np.array([vert, 9]), src_neg=np.array([100, vert + 1]),
                     src_amp=np.array([1.0, 2.5]), rec_cell=rec)
    m = W.gaussian_random_field(n, 0.2, 4)
    orc, st, s, d, u, phi, g, d_obs, phi_ref, g_ref = run_pair(prob, m, dev, seed=7)
    assert rel(d, st['d']) < TOL
    assert rel(g, g_ref) < TOL
    s.close()


def test_solve_host_matches_device_path(dev):
    prob = W.make_problem((16, 16, 16), 8, 2, 12, seed=21)
    m = W.gaussian_random_field(prob.n, 0.2, 22)
    from paper_1707_07598_gb300.msfv import Session
    s = Session(prob)
    d_dev = s.forward(torch.from_numpy(m).to(dev)).cpu().numpy()
    d_obs = d_dev * 1.01
    phi_dev, g_dev = s.adjoint(torch.from_numpy(d_obs).to(dev))
    d_h, g_h, phi_h = s.solve_host(m, d_obs)
    assert np.array_equal(d_h, d_dev)
    assert np.array_equal(g_h, g_dev.cpu().numpy())
    assert phi_h == phi_dev
    s.close()


def test_repeatable_bitwise(dev):
    """Deterministic reductions: two runs give identical bits."""
    prob = W.make_problem((16, 16, 16), 4, 3, 20, seed=31)
    m = W.gaussian_random_field(prob.n, 0.2, 32)
    from paper_1707_07598_gb300.msfv import Session
    s = Session(prob)
    mt = torch.from_numpy(m).to(dev)
    d1 = s.forward(mt).clone()
    _, g1 = s.adjoint(d1 * 1.01)
    g1 = g1.clone()
    d2 = s.forward(mt)
    _, g2 = s.adjoint(d1 * 1.01)
    assert torch.equal(d1, d2) and torch.equal(g1, g2)
    s.close()


def test_gradient_central_differences_on_gpu(dev):
    """Central differences (step 1e-6) along 20 random directions (GPU only)."""
    prob = W.make_problem((32, 32, 32), 8, 4, 64, seed=41)
    m = W.gaussian_random_field(prob.n, 0.15, 42)
    from paper_1707_07598_gb300.msfv import Session
    s = Session(prob)
    mt = torch.from_numpy(m).to(dev)
    d0 = s.forward(mt)
    d_obs = d0 * 1.05
    _, g = s.adjoint(d_obs)
    g = g.clone()

    def misfit(mm):
        dd = s.forward(mm)
        return 0.5 * float(torch.sum((dd - d_obs) ** 2))
    for k in range(20):
        v = torch.from_numpy(W.noise_like(prob.N, 1.0, 100 + k)).to(dev)
        fd = (misfit(mt + 1e-6 * v) - misfit(mt - 1e-6 * v)) / 2e-6
        an = float(g @ v)
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3 * float(g.norm() * v.norm()))
    s.close()


def test_config_2d_64_full(dev):
    prob, m = W.config_2d_64()
    orc, st, s, d, u, phi, g, d_obs, phi_ref, g_ref = run_pair(prob, m, dev)
    assert rel(d, st['d']) < TOL and rel(u, st['U']) < TOL and rel(g, g_ref) < TOL
    s.close()


def test_config_3d_128_full(dev):
    """The full 128^3, c = 8, 16-dipole, 512-receiver workload the benchmark times."""
    prob, m = W.config_3d_128()
    orc, st, s, d, u, phi, g, d_obs, phi_ref, g_ref = run_pair(prob, m, dev)
    assert rel(d, st['d']) < TOL
    assert rel(u, st['U']) < TOL
    assert abs(phi - phi_ref) <= TOL * abs(phi_ref)
    assert rel(g, g_ref) < TOL
    s.close()


@pytest.mark.parametrize("solver", ["band", "mg", "nd"])
@pytest.mark.parametrize("n,c,ns,nr", [((32, 32), 4, 2, 16), ((20, 15), 5, 2, 8),
                                       ((16, 16, 16), 4, 3, 20), ((24, 16, 16), 8, 4, 30),
                                       ((12, 10, 6), 2, 2, 9), ((128, 128), 4, 3, 24),
                                       ((320, 256), 4, 2, 20), ((48, 48, 48), 4, 3, 30)])
def test_both_coarse_solvers_match_oracle(dev, monkeypatch, solver, n, c, ns, nr):
    """Banded LU, multigrid GMRES and the nested-dissection LU all reproduce the oracle's
    pinned coarse solve (forward, transposed in the gradient, and again in J v)."""
    monkeypatch.setenv("MSFV_COARSE_SOLVER", solver)
    prob = W.make_problem(n, c, ns, nr, seed=51, top_layer=len(n) == 3)
    m = W.gaussian_random_field(n, 0.2, 52)
    orc, st, s, d, u, phi, g, d_obs, phi_ref, g_ref = run_pair(prob, m, dev)
    assert s.info()["coarse_solver"] == {"band": 0, "mg": 1, "nd": 2}[solver]
    assert rel(d, st['d']) < TOL and rel(u, st['U']) < TOL and rel(g, g_ref) < TOL
    v = W.noise_like(prob.N, 1.0, 53)
    assert rel(s.jvec(torch.from_numpy(v).to(dev)).cpu().numpy(), orc.jvec(st, v)) < TOL
    s.close()


@pytest.mark.parametrize("window", ["shared", "global"])
@pytest.mark.parametrize("fm", [1, 2])
@pytest.mark.parametrize("n,c,ns,nr", [((20, 15), 5, 2, 8), ((32, 32), 8, 2, 16),
                                       ((9, 9, 6), 3, 2, 7), ((16, 16, 16), 8, 3, 20),
                                       ((24, 16, 16), 8, 4, 30)])
def test_factor_modes_and_windows_match_oracle(dev, monkeypatch, window, fm, n, c, ns, nr):
    """Stored or recomputed local factors, shared- or global-memory factor windows."""
    if window == "global":
        monkeypatch.setenv("MSFV_LOCAL_WINDOW", "global")
    prob = W.make_problem(n, c, ns, nr, seed=71, top_layer=len(n) == 3)
    m = W.gaussian_random_field(n, 0.2, 72)
    orc, st, s, d, u, phi, g, d_obs, phi_ref, g_ref = run_pair(prob, m, dev, factor_mode=fm)
    info = s.info()
    assert info["recompute"] == (1 if fm == 2 else 0)
    assert (info["global_window_mask"] != 0) == (window == "global")
    assert (info["factor_bytes"] == 0) == (fm == 2)
    assert rel(d, st['d']) < TOL and rel(u, st['U']) < TOL and rel(g, g_ref) < TOL
    assert abs(phi - phi_ref) <= TOL * abs(phi_ref)
    v = W.noise_like(prob.N, 1.0, 73)
    w = W.noise_like((prob.n_src, prob.n_rec), 1.0, 74)
    assert rel(s.jvec(torch.from_numpy(v).to(dev)).cpu().numpy(), orc.jvec(st, v)) < TOL
    assert rel(s.jtvec(torch.from_numpy(w).to(dev)).cpu().numpy(), orc.jtvec(st, w)) < TOL
    s.close()


@pytest.mark.parametrize("fm", [1, 2])
@pytest.mark.parametrize("n,ns,nr", [((32, 32, 32), 2, 16), ((48, 32, 16), 3, 20),
                                     ((64, 64, 64), 4, 64)])
def test_coarsening_16_in_3d_matches_oracle(dev, fm, n, ns, nr):
    """c = 16 in 3D: dual-cell interiors of up to 15^3 unknowns, half bandwidth 225,
    factored in global memory."""
    prob = W.make_problem(n, 16, ns, nr, seed=81, top_layer=True)
    m = W.gaussian_random_field(n, 0.15, 82)
    orc, st, s, d, u, phi, g, d_obs, phi_ref, g_ref = run_pair(prob, m, dev, factor_mode=fm)
    assert s.info()["global_window_mask"] & (1 << 3)
    assert rel(d, st['d']) < TOL and rel(u, st['U']) < TOL and rel(g, g_ref) < TOL
    v = W.noise_like(prob.N, 1.0, 83)
    assert rel(s.jvec(torch.from_numpy(v).to(dev)).cpu().numpy(), orc.jvec(st, v)) < TOL
    s.close()


def test_auto_factor_mode_recomputes_under_a_tight_budget(dev):
    """Automatic factor mode: stores the factors when they fit, recomputes them when the
    budget is a quarter of the factor bytes short of the stored-factor workspace
    (recompute keeps one largest factor per resident thread group, 63 MB for 456 groups,
    against 0.2 GB of stored factors for the 2197 interiors at 96^3)."""
    prob = W.make_problem((96, 96, 96), 8, 4, 32, seed=91, top_layer=True)
    m = W.gaussian_random_field(prob.n, 0.2, 92)
    orc, st, s, d, u, phi, g, d_obs, phi_ref, g_ref = run_pair(prob, m, dev)
    info = s.info()
    assert info["recompute"] == 0 and info["factor_bytes"] > 0
    budget = info["workspace_bytes"] - info["factor_bytes"] // 4
    s.close()
    from paper_1707_07598_gb300.msfv import Session
    s2 = Session(prob, factor_mode=0, hbm_budget_bytes=budget)
    assert s2.info()["recompute"] == 1 and s2.info()["workspace_bytes"] <= budget
    mt = torch.from_numpy(m).to(dev)
    d2 = s2.forward(mt).cpu().numpy()
    phi2, g2 = s2.adjoint(torch.from_numpy(d_obs).to(dev))
    assert rel(d2, st['d']) < TOL and rel(g2.cpu().numpy(), g_ref) < TOL
    s2.close()


@pytest.mark.parametrize("n,c,ns,nr", [((16, 16, 16), 4, 3, 20), ((24, 16, 16), 8, 4, 30),
                                       ((32, 32), 4, 2, 16)])
def test_multigrid_with_coarse_levels_in_global_memory(dev, monkeypatch, n, c, ns, nr):
    """The multigrid levels >= 1 kept in global memory (as for coarse meshes whose level
    vectors do not fit in one CTA's shared memory) reproduce the oracle."""
    monkeypatch.setenv("MSFV_COARSE_SOLVER", "mg")
    monkeypatch.setenv("MSFV_MG_COARSE_GLOBAL", "1")
    prob = W.make_problem(n, c, ns, nr, seed=131, top_layer=len(n) == 3)
    m = W.gaussian_random_field(n, 0.2, 132)
    orc, st, s, d, u, phi, g, d_obs, phi_ref, g_ref = run_pair(prob, m, dev)
    assert rel(d, st['d']) < TOL and rel(u, st['U']) < TOL and rel(g, g_ref) < TOL
    s.close()


def test_large_coarse_mesh_192_c4(dev):
    """192^3, c = 4: 110592 coarse unknowns, multigrid levels in global memory.  Too large
    for the oracle; checked by the adjoint identity <w, J v> = <J^T w, v> and by the
    gradient matching J^T r."""
    from paper_1707_07598_gb300.msfv import Session
    prob = W.make_problem((192, 192, 192), 4, 8, 64, seed=141, top_layer=True)
    m = torch.from_numpy(W.gaussian_random_field(prob.n, 0.1, 142)).to(dev)
    s = Session(prob)
    info = s.info()
    assert info["Nc"] == 48 ** 3 and info["coarse_solver"] == 1
    d = s.forward(m)
    assert torch.isfinite(d).all()
    d_obs = d * 1.02
    phi, g = s.adjoint(d_obs)
    assert s.info()["coarse_iters"] > 0
    v = torch.from_numpy(W.noise_like(prob.N, 1.0, 143)).to(dev)
    w = torch.from_numpy(W.noise_like((prob.n_src, prob.n_rec), 1.0, 144)).to(dev)
    jv = s.jvec(v)
    jtw = s.jtvec(w)
    lhs, rhs = float((w * jv).sum()), float(jtw @ v)
    assert abs(lhs - rhs) <= 1e-10 * float(w.norm() * jv.norm())
    jtr = s.jtvec((d - d_obs).contiguous())
    assert float((jtr - g).norm()) <= 1e-12 * float(g.norm())
    s.close()


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("n,c,ns,nr", [((20, 15), 5, 2, 8), ((16, 16, 16), 8, 3, 20),
                                       ((9, 9, 6), 3, 2, 7)])
def test_every_kernel_shape_matches_oracle(dev, monkeypatch, variant, n, c, ns, nr):
    """Each local-kernel shape (warp x4, warp x8, 128- and 256-thread blocks) is exact."""
    monkeypatch.setenv("MSFV_LOCAL_VARIANT", str(variant))
    prob = W.make_problem(n, c, ns, nr, seed=191, top_layer=len(n) == 3)
    m = W.gaussian_random_field(n, 0.2, 192)
    orc, st, s, d, u, phi, g, d_obs, phi_ref, g_ref = run_pair(prob, m, dev, factor_mode=2)
    assert rel(d, st['d']) < TOL and rel(u, st['U']) < TOL and rel(g, g_ref) < TOL
    v = W.noise_like(prob.N, 1.0, 193)
    assert rel(s.jvec(torch.from_numpy(v).to(dev)).cpu().numpy(), orc.jvec(st, v)) < TOL
    s.close()


def test_autotune_picks_a_shape_and_stays_exact(dev):
    from paper_1707_07598_gb300.msfv import Session
    prob = W.make_problem((32, 32, 32), 8, 4, 32, seed=195, top_layer=True)
    m = W.gaussian_random_field(prob.n, 0.15, 196)
    s = Session(prob)
    res = s.autotune(torch.from_numpy(m).to(dev))
    assert set(res) == {1, 2, 3}
    for k, (choice, times) in res.items():
        if choice == "mixed":       # mixed-precision interiors: nothing to choose
            continue
        assert choice in times and times[choice] == min(times.values())
    orc = Oracle(prob)
    st = orc.forward(m)
    d = s.forward(torch.from_numpy(m).to(dev)).cpu().numpy()
    assert rel(d, st['d']) < TOL
    # a later session of the same shapes starts with the tuned shapes
    s2 = Session(prob)
    d2 = s2.forward(torch.from_numpy(m).to(dev)).cpu().numpy()
    assert rel(d2, st['d']) < TOL
    s.close()
    s2.close()


@pytest.mark.parametrize("n,c,ns,nr", [((16, 16), 4, 2, 9), ((16, 16, 16), 8, 3, 20)])
def test_fixed_basis_jtvec_matches_oracle_and_is_the_worse_gradient(dev, n, c, ns, nr):
    """J^T w with the basis held fixed (Sec. 4.2) against the oracle, and the contrast the
    paper draws: the adaptive-basis gradient matches central differences, the fixed-basis
    one does not (Sec. 4.2's study of the gradient error)."""
    prob = W.make_problem(n, c, ns, nr, seed=201, top_layer=len(n) == 3)
    m = W.gaussian_random_field(n, 0.2, 202)
    orc = Oracle(prob)
    st = orc.forward(m)
    from paper_1707_07598_gb300.msfv import Session
    s = Session(prob)
    mt = torch.from_numpy(m).to(dev)
    d = s.forward(mt)
    w = W.noise_like((prob.n_src, prob.n_rec), 1.0, 203)
    gf = s.jtvec_fixed_basis(torch.from_numpy(w).to(dev)).cpu().numpy()
    assert rel(gf, orc.jtvec_fixed_basis(st, w)) < TOL
    # gradients of phi = <w, d(m)> along random directions: adaptive vs fixed vs FD
    ga = s.jtvec(torch.from_numpy(w).to(dev)).cpu().numpy()
    err_a, err_f = [], []
    wt = torch.from_numpy(w).to(dev)
    for k in range(5):
        v = W.noise_like(prob.N, 1.0, 210 + k)
        vt = torch.from_numpy(v).to(dev)
        fd = (float((s.forward(mt + 1e-6 * vt) * wt).sum()) -
              float((s.forward(mt - 1e-6 * vt) * wt).sum())) / 2e-6
        err_a.append(abs(ga @ v - fd) / abs(fd))
        err_f.append(abs(gf @ v - fd) / abs(fd))
    assert max(err_a) < 1e-6 and min(err_f) > 1e-4
    s.close()


def test_error_paths_report_status_without_faulting(dev):
    """A model with a NaN cell gives MSFV_ERR_NUMERIC (non-positive / NaN local pivot) at
    the next status read; derivative calls before any forward give MSFV_ERR_STATE; the
    session stays usable afterwards."""
    from paper_1707_07598_gb300.msfv import MSFVError, Session
    prob = W.make_problem((16, 16, 16), 8, 2, 12, seed=221, top_layer=True)
    s = Session(prob)
    d_obs = torch.zeros((prob.n_src, prob.n_rec), dtype=torch.float64, device=dev)
    with pytest.raises(MSFVError) as e:
        s.adjoint(d_obs)
    assert e.value.code == 6
    with pytest.raises(MSFVError) as e:
        s.jvec(torch.zeros(prob.N, dtype=torch.float64, device=dev))
    assert e.value.code == 6
    m = torch.zeros(prob.N, dtype=torch.float64, device=dev)
    m[1234] = float("nan")
    s.forward(m)
    with pytest.raises(MSFVError) as e:
        s.adjoint(d_obs)
    assert e.value.code == 3
    # the next forward with a valid model clears the status: the session recovers
    m_ok = W.gaussian_random_field(prob.n, 0.2, 222)
    st = Oracle(prob).forward(m_ok)
    assert rel(s.forward(torch.from_numpy(m_ok).to(dev)).cpu().numpy(), st['d']) < TOL
    s.adjoint(d_obs)
    s.close()
    # a fresh session on the same device works
    s2 = Session(prob)
    assert rel(s2.forward(torch.from_numpy(m_ok).to(dev)).cpu().numpy(), st['d']) < TOL
    s2.close()


def test_grid_barrier_wait_expires_with_timeout_status(dev, monkeypatch):
    """The all-SM coarse solver's software grid barrier waits at most the session's wait
    limit.  With a limit of 1 ns a wait runs out: every CTA leaves the solve, the status
    read reports MSFV_ERR_TIMEOUT (4) and nothing faults; with the default limit
    restored, the next forward and gradient on the same session match the oracle."""
    from paper_1707_07598_gb300.msfv import MSFVError, Session
    monkeypatch.setenv("MSFV_COARSE_SOLVER", "mg")
    monkeypatch.setenv("MSFV_MG_SOLVER", "all")
    prob = W.make_problem((32, 32, 32), 4, 3, 20, seed=251, top_layer=True)
    m = W.gaussian_random_field(prob.n, 0.2, 252)
    orc = Oracle(prob)
    st = orc.forward(m)
    d_obs = st['d'] * 1.02
    phi_ref, g_ref = orc.misfit_gradient(st, d_obs)
    s = Session(prob)
    assert s.info()["coarse_group_ctas"] > 8            # one cooperative grid over the SMs
    mt = torch.from_numpy(m).to(dev)
    dt = torch.from_numpy(d_obs).to(dev)
    s.set_wait_limit(1)
    s.forward(mt)
    with pytest.raises(MSFVError) as e:
        s.adjoint(dt)
    assert e.value.code == 4
    with pytest.raises(MSFVError):
        s.set_wait_limit(-1)
    s.set_wait_limit(0)
    d = s.forward(mt).cpu().numpy()
    phi, g = s.adjoint(dt)
    assert rel(d, st['d']) < TOL and rel(g.cpu().numpy(), g_ref) < TOL
    assert abs(phi - phi_ref) <= TOL * abs(phi_ref)
    s.close()


@pytest.mark.parametrize("cycle", ["1,1,1,1", "2,1,2,1", "1,2,1,2"])
@pytest.mark.parametrize("n,c,ns,nr", [((128, 128), 4, 3, 24), ((48, 48, 48), 4, 3, 30),
                                       ((24, 16, 16), 8, 4, 30)])
def test_multigrid_smoothing_variants_match_oracle(dev, monkeypatch, cycle, n, c, ns, nr):
    """V(1,1), V(2,1) and V(1,2) cycles (distributed and local levels) give the same
    pinned coarse solution (the preconditioner changes, the solve does not)."""
    monkeypatch.setenv("MSFV_COARSE_SOLVER", "mg")
    monkeypatch.setenv("MSFV_MG_CYCLE", cycle)
    prob = W.make_problem(n, c, ns, nr, seed=231, top_layer=len(n) == 3)
    m = W.gaussian_random_field(n, 0.2, 232)
    orc, st, s, d, u, phi, g, d_obs, phi_ref, g_ref = run_pair(prob, m, dev)
    assert rel(d, st['d']) < TOL and rel(u, st['U']) < TOL and rel(g, g_ref) < TOL
    s.close()


@pytest.mark.parametrize("variant", ["all", "cluster"])
@pytest.mark.parametrize("n,c,ns,nr", [((16, 16, 16), 4, 3, 20), ((24, 16, 16), 8, 4, 30),
                                       ((48, 48, 48), 4, 5, 30), ((128, 128), 4, 3, 24),
                                       ((32, 32), 4, 1, 16)])
def test_multigrid_solver_variants_match_oracle(dev, monkeypatch, variant, n, c, ns, nr):
    """The all-SM cooperative multigrid GMRES and the cluster-per-right-hand-side one give
    the oracle's pinned coarse solution, forward and transposed."""
    monkeypatch.setenv("MSFV_COARSE_SOLVER", "mg")
    monkeypatch.setenv("MSFV_MG_SOLVER", variant)
    prob = W.make_problem(n, c, ns, nr, seed=241, top_layer=len(n) == 3)
    m = W.gaussian_random_field(n, 0.2, 242)
    orc, st, s, d, u, phi, g, d_obs, phi_ref, g_ref = run_pair(prob, m, dev)
    assert rel(d, st['d']) < TOL and rel(u, st['U']) < TOL and rel(g, g_ref) < TOL
    info = s.info()
    assert 0 < info["coarse_iters"] < 100 and 0 < info["coarse_iters_T"] < 100
    s.close()


@pytest.mark.parametrize("n,c,ns,nr", [((16, 16, 16), 8, 3, 20), ((24, 16, 16), 8, 4, 30),
                                       ((9, 9, 6), 3, 2, 7), ((32, 32), 8, 2, 16),
                                       ((64, 64, 64), 8, 8, 64)])
def test_mixed_precision_interiors_match_oracle(dev, monkeypatch, n, c, ns, nr):
    """MSFV_LOCAL_PRECISION=mixed: the top-dimensional local problems factored in FP32 and
    solved with two FP64 refinement steps reach the same 1e-9 bar on d, u, the gradient,
    J v and J^T w."""
    monkeypatch.setenv("MSFV_LOCAL_PRECISION", "mixed")
    from paper_1707_07598_gb300.msfv import Session
    prob = W.make_problem(n, c, ns, nr, seed=211, top_layer=len(n) == 3)
    m = W.gaussian_random_field(n, 0.2, 212)
    orc, st, s, d, u, phi, g, d_obs, phi_ref, g_ref = run_pair(prob, m, dev)
    assert rel(d, st['d']) < TOL and rel(u, st['U']) < TOL and rel(g, g_ref) < TOL
    v = W.noise_like(prob.N, 1.0, 213)
    w = W.noise_like((prob.n_src, prob.n_rec), 1.0, 214)
    assert rel(s.jvec(torch.from_numpy(v).to(dev)).cpu().numpy(), orc.jvec(st, v)) < TOL
    assert rel(s.jtvec(torch.from_numpy(w).to(dev)).cpu().numpy(), orc.jtvec(st, w)) < TOL
    s.close()


def test_mixed_precision_nodal_variant(dev, monkeypatch):
    monkeypatch.setenv("MSFV_LOCAL_PRECISION", "mixed")
    from oracle.galerkin_oracle import NodalOracle
    from paper_1707_07598_gb300.msfv import Session
    prob = W.make_problem((16, 16, 16), 4, 3, 20, seed=221, top_layer=False, nodal=True)
    m = W.gaussian_random_field(prob.n, 0.2, 222)
    orc = NodalOracle(prob)
    st = orc.forward(m)
    d_obs = st['d'] * 1.02
    _, g_ref = orc.misfit_gradient(st, d_obs)
    s = Session(prob)
    d = s.forward(torch.from_numpy(m).to(dev)).cpu().numpy()
    _, g = s.adjoint(torch.from_numpy(d_obs).to(dev))
    v = W.noise_like(prob.N, 1.0, 223)
    assert rel(d, st['d']) < TOL and rel(g.cpu().numpy(), g_ref) < TOL
    assert rel(s.jvec(torch.from_numpy(v).to(dev)).cpu().numpy(), orc.jvec(st, v)) < TOL
    s.close()
