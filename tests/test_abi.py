"""The C-ABI library builds, loads and exports every symbol include/msfv.h
declares; descriptor validation runs on the host (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1707_07598_gb300 import build as B
from paper_1707_07598_gb300 import msfv as M

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return M.load()


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "msfv.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(msfv_[a-z_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def _desc(**kw):
    pos = np.array([0], dtype=np.int64)
    neg = np.array([5], dtype=np.int64)
    rec = np.array([3, 7], dtype=np.int64)
    d = M._Desc()
    d.dim = kw.get("dim", 2)
    n = kw.get("n", (16, 16, 1))
    for a in range(3):
        d.n[a] = n[a]
    d.coarsen = kw.get("c", 4)
    d.n_src = kw.get("ns", 1)
    d.src_pos = pos.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    d.src_neg = (np.array([0], dtype=np.int64) if kw.get("same") else neg).ctypes.data_as(
        ctypes.POINTER(ctypes.c_int64))
    d.src_amp = None
    d.n_rec = kw.get("nr", 2)
    r = np.array([3, 10 ** 9], dtype=np.int64) if kw.get("badrec") else rec
    d.rec_cell = r.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    d.factor_mode = kw.get("fm", 0)
    d.hbm_budget_bytes = kw.get("budget", 0)
    d.source_bases = kw.get("sb", 0)
    d.discretization = kw.get("disc", 0)
    d.oversample = kw.get("ov", 0)
    d._keep = (pos, neg, rec, r)
    return d


@pytest.mark.parametrize("kw,frag", [
    (dict(dim=4), "dim"),
    (dict(c=0), "coarsen"),
    (dict(c=3), "divide"),
    (dict(n=(4, 4, 1), c=4), "2 coarse"),
    (dict(ns=0), "n_src"),
    (dict(nr=0), "n_rec"),
    (dict(same=True), "pos == neg"),
    (dict(badrec=True), "receiver"),
    (dict(fm=3), "factor_mode"),
    (dict(dim=3, n=(34, 34, 34), c=17), "too wide"),
    (dict(budget=1000), "hbm_budget"),
    (dict(sb=2), "source_bases"),
    (dict(sb=1, fm=2), "stored local factors"),
    (dict(sb=1, budget=1000), "stored local factors"),
    (dict(disc=2), "discretization"),
    (dict(disc=1, sb=1), "not available for the nodal"),
    (dict(disc=1, fm=2), "stored local factors"),
    (dict(disc=1, budget=1000), "stored local factors"),
    (dict(ov=-1), "oversample must be >= 0"),
    (dict(ov=4), "oversample must be <= coarsen - 1"),
    (dict(ov=1, sb=1), "source bases are not defined with oversampling"),
    (dict(ov=1, disc=1), "oversampling is not available for the nodal"),
])
def test_setup_rejects_bad_descriptors_on_the_host(lib, kw, frag):
    d = _desc(**kw)
    h = ctypes.c_void_p()
    rc = lib.msfv_setup(ctypes.byref(d), None, ctypes.byref(h))
    assert rc in (1, 2)      # MSFV_ERR_ARG, or MSFV_ERR_OOM for the budget case
    assert not h.value
    assert frag in lib.msfv_last_error(None).decode()


def test_null_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.msfv_setup(None, None, ctypes.byref(h)) == 1
    assert lib.msfv_forward(None, None, None, None) == 1
    assert lib.msfv_destroy(None) == 0
    assert lib.msfv_phase_name(4).decode() == "basis_interiors"


def _desc3(n, c, pos, neg, rec, **kw):
    d = M._Desc()
    d.dim = 3
    for a in range(3):
        d.n[a] = n[a]
    d.coarsen = c
    pos = np.asarray(pos, dtype=np.int64)
    neg = np.asarray(neg, dtype=np.int64)
    rec = np.asarray(rec, dtype=np.int64)
    d.n_src = len(pos)
    d.src_pos = pos.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    d.src_neg = neg.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    d.src_amp = None
    d.n_rec = len(rec)
    d.rec_cell = rec.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    d.factor_mode = 0
    d.hbm_budget_bytes = kw.get("budget", 1000)
    d.source_bases = kw.get("sb", 0)
    d.discretization = kw.get("disc", 0)
    d.oversample = kw.get("ov", 0)
    d._keep = (pos, neg, rec)
    return d


def test_host_tables_of_source_bases_and_nodal_variant_build_on_the_host(lib):
    """Setup builds every host-side table (source-basis support, slots, side links to
    the neighbouring entities, flux rows, receiver map; the nodal seed points and
    block-interior subset) before it checks the budget.  With a tiny budget the call
    runs that logic on the CPU and stops with MSFV_ERR_OOM: a broken side link would
    surface as MSFV_ERR_ARG ("inconsistent dual-grid sides")."""
    n, c = (16, 16, 16), 4                 # vertex coordinates 2, 6, 10, 14

    def idx(x, y, z):
        return x + 16 * (y + 16 * z)
    # source ends on a vertex, dual edges, faces, interiors and partial boundary cells
    pos = [idx(2, 6, 10), idx(4, 2, 6), idx(3, 6, 5), idx(4, 4, 4), idx(0, 15, 1)]
    neg = [idx(6, 0, 2), idx(5, 5, 5), idx(4, 2, 7), idx(14, 14, 13), idx(15, 15, 15)]
    rec = [idx(1, 2, 3), idx(4, 2, 6), idx(15, 15, 15)]
    for kw, frag in [(dict(sb=1), "source bases need the stored local factors"),
                     (dict(disc=1), "nodal variant needs the stored local factors")]:
        d = _desc3(n, c, pos, neg, rec, **kw)
        h = ctypes.c_void_p()
        rc = lib.msfv_setup(ctypes.byref(d), None, ctypes.byref(h))
        assert rc == 2 and not h.value, lib.msfv_last_error(None).decode()
        assert frag in lib.msfv_last_error(None).decode()
    # the nodal lattice has 17^3 nodes: a node index beyond the cell count is valid there
    d = _desc3(n, c, [4500], [0], [17 ** 3 - 1], disc=1)
    h = ctypes.c_void_p()
    assert lib.msfv_setup(ctypes.byref(d), None, ctypes.byref(h)) == 2
    d = _desc3(n, c, [17 ** 3], [0], [1], disc=1)
    assert lib.msfv_setup(ctypes.byref(d), None, ctypes.byref(h)) == 1
    assert "out of range" in lib.msfv_last_error(None).decode()


@pytest.mark.parametrize("dim,n,c,w", [(3, (16, 16, 16), 4, 1), (3, (16, 16, 16), 4, 3),
                                       (3, (24, 16, 8), 8, 7), (3, (32, 32, 32), 16, 5),
                                       (2, (48, 40, 1), 8, 3), (2, (20, 15, 1), 5, 4),
                                       (3, (128, 128, 128), 8, 2)])
def test_oversampling_plan_builds_on_the_host(lib, dim, n, c, w):
    """Setup plans the oversampled edge and face boxes (widened boxes, offsets, receivers
    re-indexed in the box, the fixed-order gathers of the face gradient and of the faces'
    seeds of the edges, with their range checks) before it checks the budget: with a tiny
    budget the whole plan runs on the CPU and setup stops with MSFV_ERR_OOM.  A plan that
    failed would return MSFV_ERR_ARG with its reason."""
    N = int(np.prod(n[:dim]))
    rng = np.random.default_rng(7)
    cells = rng.choice(N, 14, replace=False)
    d = M._Desc()
    d.dim = dim
    for a in range(3):
        d.n[a] = n[a]
    d.coarsen = c
    pos, neg, rec = (np.asarray(cells[:3], dtype=np.int64), np.asarray(cells[3:6], dtype=np.int64),
                     np.asarray(cells[6:], dtype=np.int64))
    d.n_src = 3
    d.src_pos = pos.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    d.src_neg = neg.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    d.src_amp = None
    d.n_rec = len(rec)
    d.rec_cell = rec.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    d.factor_mode = 1
    d.hbm_budget_bytes = 1000
    d.source_bases = 0
    d.discretization = 0
    d.oversample = w
    h = ctypes.c_void_p()
    rc = lib.msfv_setup(ctypes.byref(d), None, ctypes.byref(h))
    msg = lib.msfv_last_error(None).decode()
    assert rc == 2 and not h.value, msg
    assert "exceeds hbm_budget_bytes" in msg
