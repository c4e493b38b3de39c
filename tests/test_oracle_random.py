"""Randomised cross-checks of both oracles against their independent dense brute forces
(hypothesis, derandomised so every run draws the same cases): small 2D and 3D meshes,
every coarsening that divides them, random source and receiver cells (any kind of cell,
repeats allowed for receivers), with and without source bases, and the nodal variant.
CPU only; skipped where hypothesis is not installed."""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
from hypothesis import given, settings  # noqa: E402

from oracle import bruteforce as BF  # noqa: E402
from oracle.galerkin_oracle import NodalOracle  # noqa: E402
from oracle.msfv_oracle import Oracle  # noqa: E402
from paper_1707_07598_gb300 import workloads as W  # noqa: E402


@st.composite
def problems(draw, nodal=False):
    d = draw(st.sampled_from([2, 3]))
    c = draw(st.sampled_from([1, 2, 3, 4]))
    # coarse cells per axis; every axis has at least 2 fine cells and the mesh at least
    # 2 coarse cells
    k = [draw(st.integers(1, 3 if d == 3 else 4)) for _ in range(d)]
    k = [max(ka, 2) if c == 1 else ka for ka in k]
    if int(np.prod(k)) < 2:
        k[0] = 2
    n = tuple(c * ka for ka in k)
    lat = tuple(v + 1 for v in n) if nodal else n
    N = int(np.prod(lat))
    ns = draw(st.integers(1, min(3, N // 2)))
    cells = draw(st.lists(st.integers(0, N - 1), min_size=2 * ns, max_size=2 * ns, unique=True))
    rec = draw(st.lists(st.integers(0, N - 1), min_size=1, max_size=6))
    amp = draw(st.lists(st.floats(0.5, 2.0), min_size=ns, max_size=ns))
    sb = (not nodal) and draw(st.booleans())
    seed = draw(st.integers(0, 10 ** 6))
    prob = W.Problem(n=n, coarsen=c, src_pos=np.array(cells[:ns], dtype=np.int64),
                     src_neg=np.array(cells[ns:], dtype=np.int64), src_amp=np.array(amp),
                     rec_cell=np.array(rec, dtype=np.int64), source_bases=sb, nodal=nodal)
    m = W.gaussian_random_field(n, 0.3, seed % 1000)
    return prob, m


@settings(max_examples=60, deadline=None, derandomize=True)
@given(problems())
def test_cell_centred_oracle_equals_brute_force(pm):
    prob, m = pm
    st_ = Oracle(prob).forward(m)
    d_bf, _, _ = BF.forward_dense(m, prob.n, prob.coarsen, prob.src_pos, prob.src_neg,
                                  prob.src_amp, prob.rec_cell, source_bases=prob.source_bases)
    assert np.linalg.norm(st_['d'] - d_bf) <= 1e-11 * max(np.linalg.norm(d_bf), 1e-300)


@settings(max_examples=40, deadline=None, derandomize=True)
@given(problems(nodal=True))
def test_nodal_oracle_equals_brute_force(pm):
    prob, m = pm
    st_ = NodalOracle(prob).forward(m)
    d_bf, _, _, _ = BF.forward_dense_nodal(m, prob.n, prob.coarsen, prob.src_pos,
                                           prob.src_neg, prob.src_amp, prob.rec_cell)
    assert np.linalg.norm(st_['d'] - d_bf) <= 1e-11 * max(np.linalg.norm(d_bf), 1e-300)


@settings(max_examples=30, deadline=None, derandomize=True)
@given(problems())
def test_cell_centred_adjoint_identity(pm):
    prob, m = pm
    o = Oracle(prob)
    s_ = o.forward(m)
    rng = np.random.default_rng(1)
    v = rng.normal(size=prob.N)
    w = rng.normal(size=(prob.n_src, prob.n_rec))
    lhs, rhs = np.sum(w * o.jvec(s_, v)), o.jtvec(s_, w) @ v
    assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + np.linalg.norm(w) * np.linalg.norm(v))


@settings(max_examples=25, deadline=None, derandomize=True)
@given(problems(nodal=True))
def test_nodal_adjoint_identity(pm):
    prob, m = pm
    o = NodalOracle(prob)
    s_ = o.forward(m)
    rng = np.random.default_rng(2)
    v = rng.normal(size=prob.N)
    w = rng.normal(size=(prob.n_src, prob.n_rec))
    lhs, rhs = np.sum(w * o.jvec(s_, v)), o.jtvec(s_, w) @ v
    assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + np.linalg.norm(w) * np.linalg.norm(v))


@settings(max_examples=20, deadline=None, derandomize=True)
@given(problems())
def test_cell_centred_jvec_complex_step(pm):
    """J v (with or without source bases) against complex step of the brute force."""
    prob, m = pm
    if prob.N > 200:
        return                                    # keep the dense complex step cheap
    o = Oracle(prob)
    s_ = o.forward(m)
    v = np.random.default_rng(3).normal(size=prob.N)
    ref = BF.jvec_complex_step(m, prob, v)
    assert np.linalg.norm(o.jvec(s_, v) - ref) <= 1e-10 * max(np.linalg.norm(ref), 1e-300)
