"""The allocation-free misfit entry point against msfv_adjoint's misfit.

msfv_misfit_static serves callers that cannot allocate device memory where they need
the misfit (a serving loop under a fixed allocator budget, or a host application that
only lends its own buffers).  This file is collected last so that a
run stopping at the first failure has already run every other test; it also passes
on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1707_07598_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-9


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1707_07598_gb300 import build, msfv
    build.build()
    L = msfv.load()
    L.msfv_misfit_static.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.msfv_misfit_static.restype = ctypes.c_int
    return L


def _static(L, d_pred, d_obs, r, phi):
    stream = torch.cuda.current_stream().cuda_stream
    return L.msfv_misfit_static(d_pred.data_ptr(), d_obs.data_ptr(), d_pred.numel(),
                                r.data_ptr() if r is not None else None, phi.data_ptr(),
                                stream)


def test_static_misfit_matches_adjoint_twice_in_a_row(lib):
    from paper_1707_07598_gb300.msfv import Session
    dev = torch.device("cuda:0")
    prob = W.make_problem((32, 32, 32), 8, 4, 64, seed=61)
    m = torch.from_numpy(W.gaussian_random_field(prob.n, 0.15, 62)).to(dev)
    s = Session(prob)
    d_pred = s.forward(m).clone()
    d_obs = d_pred * 1.03 + torch.from_numpy(W.noise_like(tuple(d_pred.shape), 1e-3, 63)).to(dev)
    phi_ref, _ = s.adjoint(d_obs)
    r = torch.empty_like(d_pred)
    phi = torch.empty(1, dtype=torch.float64, device=dev)
    for _ in range(2):                                  # two calls in a row share the scratch
        r.fill_(float("nan"))
        phi.fill_(float("nan"))
        assert _static(lib, d_pred, d_obs, r, phi) == 0
        torch.cuda.synchronize()
        assert abs(phi.item() - phi_ref) <= TOL * abs(phi_ref)
        assert torch.equal(r, d_pred - d_obs)
    # after the first call (which may load the kernels), a call takes no device memory
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    assert _static(lib, d_pred, d_obs, r, phi) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert abs(phi.item() - phi_ref) <= TOL * abs(phi_ref)
    # a different, larger input right after: no stale partials leak in
    big_p = torch.from_numpy(W.noise_like(300000, 1.0, 64)).to(dev)
    big_o = torch.from_numpy(W.noise_like(300000, 1.0, 65)).to(dev)
    assert _static(lib, big_p, big_o, None, phi) == 0
    torch.cuda.synchronize()
    ref = 0.5 * float(np.sum((big_p.cpu().numpy() - big_o.cpu().numpy()) ** 2))
    assert abs(phi.item() - ref) <= TOL * ref
    s.close()


def test_static_misfit_rejects_counts_beyond_its_scratch(lib):
    dev = torch.device("cuda:0")
    x = torch.zeros(4, dtype=torch.float64, device=dev)
    phi = torch.zeros(1, dtype=torch.float64, device=dev)
    limit = 16 * 1024 * 1024
    rc = lib.msfv_misfit_static(x.data_ptr(), x.data_ptr(), limit + 1, None, phi.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    assert rc == 1                                     # MSFV_ERR_ARG, nothing enqueued
