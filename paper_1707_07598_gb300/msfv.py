"""Thin Python binding of the MSFV C ABI (include/msfv.h).

Argument marshalling only: every step of the path runs in the CUDA kernels of
``libmsfv.so``.  PyTorch supplies device memory (CUDA tensors) and the stream.
There is no CPU fallback: if the library or a GPU is missing the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import build as _build

MSFV_OK = 0
_ERR = {1: "MSFV_ERR_ARG", 2: "MSFV_ERR_OOM", 3: "MSFV_ERR_NUMERIC", 4: "MSFV_ERR_TIMEOUT",
        5: "MSFV_ERR_CUDA", 6: "MSFV_ERR_STATE"}

_lib = None


class MSFVError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERR.get(code, code)}: {msg}")
        self.code = code


class _GNOpts(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("m_ref_dev", ctypes.c_void_p),
                ("cg_iters", ctypes.c_int), ("cg_tol", ctypes.c_double),
                ("max_backtracks", ctypes.c_int), ("m_min", ctypes.c_double),
                ("m_max", ctypes.c_double)]


class _GNStats(ctypes.Structure):
    _fields_ = [("phi_d0", ctypes.c_double), ("phi_r0", ctypes.c_double),
                ("phi_d1", ctypes.c_double), ("phi_r1", ctypes.c_double),
                ("grad_norm", ctypes.c_double), ("cg_iters", ctypes.c_int),
                ("cg_rel_res", ctypes.c_double), ("step", ctypes.c_double),
                ("backtracks", ctypes.c_int)]


class _Desc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("coarsen", ctypes.c_int),
                ("n_src", ctypes.c_int), ("src_pos", ctypes.POINTER(ctypes.c_int64)),
                ("src_neg", ctypes.POINTER(ctypes.c_int64)),
                ("src_amp", ctypes.POINTER(ctypes.c_double)),
                ("n_rec", ctypes.c_int), ("rec_cell", ctypes.POINTER(ctypes.c_int64)),
                ("factor_mode", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_size_t),
                ("source_bases", ctypes.c_int), ("discretization", ctypes.c_int),
                ("oversample", ctypes.c_int)]


def lib_path() -> str:
    return _build.lib_path()


def load(path: Optional[str] = None):
    """Load libmsfv.so (built in-tree by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or lib_path()
    if not os.path.exists(p):
        raise RuntimeError(f"libmsfv.so not found at {p}: run __graft_entry__.build() first "
                           "(there is no CPU fallback)")
    L = ctypes.CDLL(p)
    vp, i64p, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)
    L.msfv_setup.argtypes = [ctypes.POINTER(_Desc), vp, ctypes.POINTER(vp)]
    L.msfv_forward.argtypes = [vp, vp, vp, vp]
    L.msfv_adjoint.argtypes = [vp, vp, vp, dp]
    L.msfv_jvec.argtypes = [vp, vp, vp]
    L.msfv_jtvec.argtypes = [vp, vp, vp]
    L.msfv_jtvec_fixed_basis.argtypes = [vp, vp, vp]
    L.msfv_jtvec_fixed_basis.restype = ctypes.c_int
    L.msfv_solve_host.argtypes = [vp, vp, vp, vp, vp, dp]
    L.msfv_destroy.argtypes = [vp]
    L.msfv_last_error.argtypes = [vp]
    L.msfv_last_error.restype = ctypes.c_char_p
    L.msfv_set_stream.argtypes = [vp, vp]
    L.msfv_info.argtypes = [vp, i64p, ctypes.c_int]
    L.msfv_profile.argtypes = [vp, ctypes.c_int]
    L.msfv_phase_times.argtypes = [vp, dp, i64p, ctypes.c_int, ctypes.c_int]
    L.msfv_phase_name.argtypes = [ctypes.c_int]
    L.msfv_phase_name.restype = ctypes.c_char_p
    L.msfv_interior_flops.argtypes = [vp]
    L.msfv_interior_flops.restype = ctypes.c_double
    L.msfv_coarse_trace.argtypes = [vp, i64p, ctypes.c_int]
    L.msfv_launch_count.argtypes = [vp]
    L.msfv_launch_count.restype = ctypes.c_int64
    L.msfv_misfit_static.argtypes = [vp, vp, ctypes.c_int64, vp, vp, vp]
    L.msfv_misfit_static.restype = ctypes.c_int
    L.msfv_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp),
                                    ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                    vp, ctypes.POINTER(vp)]
    L.msfv_batch_create.restype = ctypes.c_int
    L.msfv_batch_run_host.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                      ctypes.POINTER(vp), ctypes.POINTER(vp)]
    L.msfv_batch_run_host.restype = ctypes.c_int
    L.msfv_nd_analyse.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), i64p, ctypes.c_int]
    L.msfv_nd_analyse.restype = ctypes.c_int
    L.msfv_batch_run_timed.argtypes = [vp, dp, dp, i64p, ctypes.c_int]
    L.msfv_batch_run_timed.restype = ctypes.c_int
    L.msfv_batch_info.argtypes = [vp, i64p, ctypes.c_int]
    L.msfv_batch_info.restype = ctypes.c_int
    for f in ("msfv_batch_run", "msfv_batch_check", "msfv_batch_destroy"):
        getattr(L, f).argtypes = [vp]
        getattr(L, f).restype = ctypes.c_int
    L.msfv_batch_last_error.argtypes = [vp]
    L.msfv_batch_last_error.restype = ctypes.c_char_p
    L.msfv_gn_step.argtypes = [vp, vp, vp, ctypes.POINTER(_GNOpts), ctypes.POINTER(_GNStats)]
    L.msfv_gn_step.restype = ctypes.c_int
    L.msfv_autotune.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
    L.msfv_autotune.restype = ctypes.c_int
    L.msfv_fp64_probe.argtypes = [vp, dp, dp]
    L.msfv_set_wait_limit.argtypes = [vp, ctypes.c_int64]
    L.msfv_status.argtypes = [vp]
    L.msfv_status.restype = ctypes.c_int
    L.msfv_set_wait_limit.restype = ctypes.c_int
    L.msfv_fp64_probe.restype = ctypes.c_int
    for f in ("msfv_setup", "msfv_forward", "msfv_adjoint", "msfv_jvec", "msfv_jtvec",
              "msfv_solve_host", "msfv_destroy", "msfv_set_stream", "msfv_info", "msfv_profile",
              "msfv_phase_times", "msfv_phase_name", "msfv_coarse_trace"):
        if getattr(L, f).restype is None and f != "msfv_phase_name":
            getattr(L, f).restype = ctypes.c_int
    _lib = L
    return L


def _ptr(t) -> int:
    """Device pointer of a contiguous float64 CUDA tensor."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return t.data_ptr()


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class Session:
    """One MSFV problem (mesh, coarsening, sources, receivers) on the current GPU.

    Mirrors the C ABI: ``forward`` (steps a-e), ``adjoint`` (misfit and gradient),
    ``jvec`` / ``jtvec`` (Sec. 4.3 sensitivities), ``solve_host``.  ``prob.source_bases``
    adds the source bases of Sec. 3.2; ``prob.nodal`` selects the nodal Galerkin
    discretisation (fields of ``Nf`` node values per source; m and gradients stay on the
    ``N`` cells).
    """

    def __init__(self, prob, stream=None, factor_mode: int = 0, hbm_budget_bytes: int = 0):
        L = load()
        self._lib = L
        self.prob = prob
        n = tuple(int(v) for v in prob.n)
        self.dim = len(n)
        self.N = int(np.prod(n))                      # model cells
        self.nodal = bool(getattr(prob, "nodal", False))
        # field values per source: nodes of the (n+1)^d lattice in the nodal variant
        self.Nf = int(np.prod([v + 1 for v in n])) if self.nodal else self.N
        self.Ns = int(prob.n_src)
        self.Nr = int(prob.n_rec)
        self._src_pos = np.ascontiguousarray(prob.src_pos, dtype=np.int64)
        self._src_neg = np.ascontiguousarray(prob.src_neg, dtype=np.int64)
        self._src_amp = np.ascontiguousarray(prob.src_amp, dtype=np.float64)
        self._rec = np.ascontiguousarray(prob.rec_cell, dtype=np.int64)
        d = _Desc()
        d.dim = self.dim
        for a in range(3):
            d.n[a] = n[a] if a < self.dim else 1
        d.coarsen = int(prob.coarsen)
        d.n_src = self.Ns
        d.src_pos = self._src_pos.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        d.src_neg = self._src_neg.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        d.src_amp = self._src_amp.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.n_rec = self.Nr
        d.rec_cell = self._rec.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        d.factor_mode = int(factor_mode)
        d.hbm_budget_bytes = int(hbm_budget_bytes)
        d.source_bases = 1 if getattr(prob, "source_bases", False) else 0
        d.oversample = int(getattr(prob, "oversample", 0))
        d.discretization = 1 if getattr(prob, "nodal", False) else 0
        h = ctypes.c_void_p()
        self._h = None
        rc = L.msfv_setup(ctypes.byref(d), ctypes.c_void_p(_stream_handle(stream)), ctypes.byref(h))
        if rc != MSFV_OK:
            raise MSFVError(rc, L.msfv_last_error(None).decode())
        self._h = h
        self.version = 0   # bumped by every forward: derivative calls refer to the last one

    # -- helpers ------------------------------------------------------------------
    def _check(self, rc):
        if rc != MSFV_OK:
            raise MSFVError(rc, self._lib.msfv_last_error(self._h).decode())

    def set_stream(self, stream=None):
        self._check(self._lib.msfv_set_stream(self._h, ctypes.c_void_p(_stream_handle(stream))))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.msfv_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- the path -------------------------------------------------------------------
    def forward(self, m, d_pred=None, u=None):
        import torch
        if d_pred is None:
            d_pred = torch.empty((self.Ns, self.Nr), dtype=torch.float64, device=m.device)
        self._check(self._lib.msfv_forward(self._h, _ptr(m), _ptr(d_pred),
                                           _ptr(u) if u is not None else None))
        self.version += 1
        return d_pred

    def adjoint(self, d_obs, grad=None, want_phi: bool = True):
        import torch
        if grad is None:
            grad = torch.empty(self.N, dtype=torch.float64, device=d_obs.device)
        phi = ctypes.c_double(0.0)
        self._check(self._lib.msfv_adjoint(self._h, _ptr(d_obs), _ptr(grad),
                                           ctypes.byref(phi) if want_phi else None))
        return (phi.value if want_phi else None), grad

    def jvec(self, v, out=None):
        import torch
        if out is None:
            out = torch.empty((self.Ns, self.Nr), dtype=torch.float64, device=v.device)
        self._check(self._lib.msfv_jvec(self._h, _ptr(v), _ptr(out)))
        return out

    def jtvec(self, w, out=None):
        import torch
        if out is None:
            out = torch.empty(self.N, dtype=torch.float64, device=w.device)
        self._check(self._lib.msfv_jtvec(self._h, _ptr(w), _ptr(out)))
        return out

    def jtvec_fixed_basis(self, w, out=None):
        """J^T w with the basis held fixed (the Sec. 4.2 contrast)."""
        import torch
        if out is None:
            out = torch.empty(self.N, dtype=torch.float64, device=w.device)
        self._check(self._lib.msfv_jtvec_fixed_basis(self._h, _ptr(w), _ptr(out)))
        return out

    def solve_host(self, m_host: np.ndarray, d_obs_host: np.ndarray, d_pred_host=None,
                   grad_host=None):
        """Forward + gradient through host buffers (copies inside the call)."""
        m_host = np.ascontiguousarray(m_host, dtype=np.float64)
        d_obs_host = np.ascontiguousarray(d_obs_host, dtype=np.float64)
        if d_pred_host is None:
            d_pred_host = np.empty((self.Ns, self.Nr))
        if grad_host is None:
            grad_host = np.empty(self.N)
        phi = ctypes.c_double(0.0)
        self._check(self._lib.msfv_solve_host(
            self._h, m_host.ctypes.data, d_obs_host.ctypes.data, d_pred_host.ctypes.data,
            grad_host.ctypes.data, ctypes.byref(phi)))
        return d_pred_host, grad_host, phi.value

    VARIANTS = ("warp x4", "warp x8", "cta128", "cta256")

    def autotune(self, m=None) -> dict:
        """Time every shape of the local basis kernel per entity class and keep the
        fastest (msfv_autotune).  Returns {class: (chosen shape, {shape: ms})}."""
        var = (ctypes.c_int * 4)()
        ms = (ctypes.c_double * 16)()
        self._check(self._lib.msfv_autotune(self._h, _ptr(m) if m is not None else None, var, ms))
        out = {}
        for k in range(1, self.dim + 1):
            if var[k] < 0:      # the mixed-precision top class has a single kernel shape
                out[k] = ("mixed", {})
                continue
            times = {self.VARIANTS[v]: ms[4 * (k - 1) + v] for v in range(4) if ms[4 * (k - 1) + v] >= 0}
            out[k] = (self.VARIANTS[var[k]], times)
        return out

    def gn_step(self, m, d_obs, alpha: float, m_ref=None, cg_iters: int = 10,
                cg_tol: float = 1e-2, max_backtracks: int = 8, bounds=(-10.0, 10.0)) -> dict:
        """One Gauss-Newton-CG iteration (msfv_gn_step); m is updated in place."""
        o = _GNOpts(float(alpha), _ptr(m_ref) if m_ref is not None else None, int(cg_iters),
                    float(cg_tol), int(max_backtracks), float(bounds[0]), float(bounds[1]))
        st = _GNStats()
        self._check(self._lib.msfv_gn_step(self._h, _ptr(m), _ptr(d_obs), ctypes.byref(o),
                                           ctypes.byref(st)))
        self.version += 1
        return {k: getattr(st, k) for k, _ in _GNStats._fields_}

    # -- introspection ----------------------------------------------------------------
    def info(self) -> dict:
        out = (ctypes.c_int64 * 21)()
        self._check(self._lib.msfv_info(self._h, out, 21))
        keys = ["N", "Nc", "Ns", "Nr", "n_local_problems", "workspace_bytes", "factor_bytes",
                "coarse_solver", "coarse_iters", "coarse_iters_T", "coarse_group_ctas",
                "recompute", "global_window_mask", "source_slots", "source_values",
                "oversample", "oversampled_boxes", "oversampled_edge_flops",
                "oversampled_face_flops", "oversampled_smem_bytes", "oversampled_grid"]
        return dict(zip(keys, list(out)))

    def check(self):
        """Wait for the session's stream and raise MSFVError when the last forward or a
        derivative call after it failed numerically or timed out (msfv_status)."""
        self._check(self._lib.msfv_status(self._h))

    def set_wait_limit(self, ns: int = 0):
        """Bound (ns; 0 = the default) on a grid-barrier wait of the all-SM coarse solver;
        an expired wait is reported as MSFV_ERR_TIMEOUT (msfv_set_wait_limit)."""
        self._check(self._lib.msfv_set_wait_limit(self._h, int(ns)))

    def profile(self, enable: bool = True):
        self._check(self._lib.msfv_profile(self._h, int(enable)))

    def phase_times(self, reset: bool = False) -> dict:
        ms = (ctypes.c_double * 32)()
        calls = (ctypes.c_int64 * 32)()
        n = self._lib.msfv_phase_times(self._h, ms, calls, 32, int(reset))
        return {self._lib.msfv_phase_name(k).decode(): (ms[k], calls[k]) for k in range(n)}

    def coarse_trace(self, cap: int = 65536):
        """(tag, ns) barrier stamps of the multigrid coarse solver (MSFV_TRACE_COARSE=1)."""
        buf = (ctypes.c_int64 * cap)()
        n = self._lib.msfv_coarse_trace(self._h, buf, cap)
        if n < 0:
            raise MSFVError(-n, "msfv_coarse_trace failed")
        return [(int(v) >> 48, int(v) & ((1 << 48) - 1)) for v in buf[:n]]

    def interior_flops(self) -> float:
        return float(self._lib.msfv_interior_flops(self._h))

    def launch_count(self) -> int:
        return int(self._lib.msfv_launch_count(self._h))


def misfit_static(d_pred, d_obs, r=None, phi=None, stream=None):
    """phi = 1/2 ||d_pred - d_obs||^2 (device scalar) and optionally r = d_pred - d_obs,
    through msfv_misfit_static: no device allocation inside the call."""
    import torch
    L = load()
    if phi is None:
        phi = torch.empty((), dtype=torch.float64, device=d_pred.device)
    if d_pred.shape != d_obs.shape:
        raise ValueError("d_pred and d_obs must have the same shape")
    rc = L.msfv_misfit_static(_ptr(d_pred), _ptr(d_obs), d_pred.numel(),
                              _ptr(r) if r is not None else None, _ptr(phi),
                              ctypes.c_void_p(_stream_handle(stream)))
    if rc != MSFV_OK:
        raise MSFVError(rc, L.msfv_last_error(None).decode())
    return phi


def nd_analyse(nc) -> dict:
    """Host-side plan of the nested-dissection coarse LU for a coarse grid of nc nodes per
    axis (msfv_nd_analyse; no GPU needed)."""
    L = load()
    nc = [int(v) for v in nc]
    arr = (ctypes.c_int * 3)(*(nc + [1] * (3 - len(nc))))
    out = (ctypes.c_int64 * 7)()
    rc = L.msfv_nd_analyse(len(nc), arr, out, 7)
    if rc != MSFV_OK:
        raise MSFVError(rc, "msfv_nd_analyse failed")
    keys = ["fronts", "levels", "pool_doubles", "update_rows", "max_front", "factor_flops", "ok"]
    return dict(zip(keys, list(out)))


def fp64_probe(stream=None):
    """(TFLOP/s, ms) of the device's FP64 FMA pipe, measured by msfv_fp64_probe."""
    L = load()
    tf, ms = ctypes.c_double(), ctypes.c_double()
    rc = L.msfv_fp64_probe(ctypes.c_void_p(_stream_handle(stream)), ctypes.byref(tf),
                           ctypes.byref(ms))
    if rc != MSFV_OK:
        raise MSFVError(rc, "msfv_fp64_probe failed")
    return tf.value, ms.value


class Batch:
    """One forward + gradient step of several sessions captured as one CUDA graph
    (msfv_batch_*).  The graph reads m[k] / d_obs[k] and writes d_pred[k] / grad[k] in
    place at every run, so refresh the inputs in place between runs."""

    def __init__(self, sessions, m, d_obs, d_pred=None, grad=None, stream=None):
        import torch
        L = load()
        self._lib = L
        K = len(sessions)
        if not (len(m) == len(d_obs) == K):
            raise ValueError("one m and one d_obs per session")
        self.sessions = list(sessions)
        self.m = list(m)
        self.d_obs = list(d_obs)
        self.d_pred = list(d_pred) if d_pred is not None else [
            torch.empty((s.Ns, s.Nr), dtype=torch.float64, device=mm.device)
            for s, mm in zip(sessions, m)]
        self.grad = list(grad) if grad is not None else [
            torch.empty(s.N, dtype=torch.float64, device=mm.device) for s, mm in zip(sessions, m)]
        arr = lambda xs: (ctypes.c_void_p * K)(*[ctypes.c_void_p(v) for v in xs])  # noqa: E731
        h = ctypes.c_void_p()
        self._h = None
        self._stream = stream
        rc = L.msfv_batch_create(arr([s._h.value for s in sessions]), K,
                                 arr([_ptr(t) for t in self.m]), arr([_ptr(t) for t in self.d_obs]),
                                 arr([_ptr(t) for t in self.d_pred]),
                                 arr([_ptr(t) for t in self.grad]),
                                 ctypes.c_void_p(_stream_handle(stream)), ctypes.byref(h))
        if rc != MSFV_OK:
            raise MSFVError(rc, L.msfv_batch_last_error(None).decode())
        self._h = h
        for s in sessions:
            s.version += 1

    def run(self):
        rc = self._lib.msfv_batch_run(self._h)
        if rc != MSFV_OK:
            raise MSFVError(rc, self._lib.msfv_batch_last_error(self._h).decode())
        for s in self.sessions:
            s.version += 1

    def run_host(self, m_host, d_obs_host, d_pred_host, grad_host):
        """One step through host buffers (msfv_batch_run_host): lists of C-contiguous
        float64 numpy arrays (pinned memory gives the fastest copies), one per instance;
        the outputs are written in place.  Synchronises the batch's stream."""
        K = len(self.sessions)
        arrs = []
        for xs, n_of, writable in ((m_host, lambda s: s.N, False),
                                   (d_obs_host, lambda s: s.Ns * s.Nr, False),
                                   (d_pred_host, lambda s: s.Ns * s.Nr, True),
                                   (grad_host, lambda s: s.N, True)):
            if len(xs) != K:
                raise ValueError("one host array per instance")
            for s, x in zip(self.sessions, xs):
                if (x.dtype != np.float64 or not x.flags["C_CONTIGUOUS"] or x.size != n_of(s)
                        or (writable and not x.flags["WRITEABLE"])):
                    raise ValueError("host arrays must be C-contiguous float64 of the "
                                     "instance's size")
            arrs.append((ctypes.c_void_p * K)(*[ctypes.c_void_p(x.ctypes.data) for x in xs]))
        rc = self._lib.msfv_batch_run_host(self._h, *arrs)
        for s in self.sessions:
            s.version += 1
        if rc != MSFV_OK:
            raise MSFVError(rc, self._lib.msfv_batch_last_error(self._h).decode())

    def run_timed(self) -> list:
        """One step enqueued eagerly with CUDA events around the fused interior launches
        (msfv_batch_run_timed): per fused group a dict of the forward and adjoint launch
        times (ms), the forward flops, the entities and their largest size and half
        bandwidth.  Synchronises."""
        ng = self.info()["fused_groups"]
        n = max(1, ng)
        ms = (ctypes.c_double * (2 * n))()
        fl = (ctypes.c_double * n)()
        sh = (ctypes.c_int64 * (3 * n))()
        rc = self._lib.msfv_batch_run_timed(self._h, ms, fl, sh, n)
        for s in self.sessions:
            s.version += 1
        if rc != MSFV_OK:
            raise MSFVError(rc, self._lib.msfv_batch_last_error(self._h).decode())
        return [{"fwd_ms": ms[2 * g], "adj_ms": ms[2 * g + 1], "flops": fl[g],
                 "entities": int(sh[3 * g]), "nmax": int(sh[3 * g + 1]), "bmax": int(sh[3 * g + 2])}
                for g in range(ng)]

    def info(self) -> dict:
        out = (ctypes.c_int64 * 5)()
        rc = self._lib.msfv_batch_info(self._h, out, 5)
        if rc != MSFV_OK:
            raise MSFVError(rc, "msfv_batch_info failed")
        return dict(zip(["instances", "fused_groups", "fused_instances", "fused_entities",
                         "device_bytes"], list(out)))

    def check(self):
        rc = self._lib.msfv_batch_check(self._h)
        if rc != MSFV_OK:
            raise MSFVError(rc, self._lib.msfv_batch_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.msfv_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
