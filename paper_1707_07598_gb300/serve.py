"""Request loop for served MSFV forward + gradient solves (continuous batching).

Requests (``workloads.RequestSpec``) arrive over time; each is one forward + gradient
solve of a client's instance.  A client's requests are successive Gauss-Newton
iterations on one mesh and survey, so they reuse one device-resident session (its stored
local factors, coarse hierarchy and buffers) and run in order.  The loop

* admits a request as soon as its client's session is idle and an in-flight slot is
  free, or, for a new client, as soon as its session fits the HBM budget (idle sessions
  are evicted least recently used first to make room; a session that cannot fit even in
  an empty budget is rejected);
* runs every admitted request on its session's own CUDA stream, so requests that arrive
  while others are on the GPU overlap with them on the device;
* records arrival, start and finish times, so it reports p50 / p99 latency and the
  throughput beside those of the plain one-at-a-time path.

The scheduling logic is independent of the GPU: ``Server`` drives a backend object
(``GpuBackend`` here, a simulated one in the CPU tests).
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional

import numpy as np


class DoesNotFit(Exception):
    """The backend cannot open a session within the given byte budget."""


@dataclass
class Slot:
    client: int
    handle: object
    nbytes: int
    busy: bool = False
    last_used: float = 0.0


@dataclass
class Record:
    rid: int
    client: int
    arrival: float
    start: float = float("nan")
    finish: float = float("nan")
    status: str = "queued"      # queued / running / done / failed / rejected
    result: object = None

    @property
    def latency(self) -> float:
        return self.finish - self.arrival


@dataclass
class Stats:
    records: List[Record]
    makespan: float
    evictions: int
    opened: int
    peak_bytes: int

    def done(self) -> List[Record]:
        """Requests that finished with a valid result (the throughput and latencies)."""
        return [r for r in self.records if r.status == "done"]

    def failed(self) -> List[Record]:
        """Requests whose solve finished with a numerical or device-wait error."""
        return [r for r in self.records if r.status == "failed"]

    @property
    def throughput(self) -> float:
        d = self.done()
        return len(d) / self.makespan if self.makespan > 0 else 0.0

    def percentile(self, q: float) -> float:
        lat = [r.latency for r in self.done()]
        return float(np.percentile(lat, q)) if lat else float("nan")


def estimated_work(spec) -> float:
    """Relative cost of one forward + gradient request.  The local solves cost about
    n b^2 per dual cell, n ~ (c-1)^d unknowns and half bandwidth b ~ (c-1)^(d-1), over
    N / c^d dual cells; the coarse solve about 400 flops per coarse node and source."""
    d = len(spec.n)
    N = float(np.prod(spec.n))
    c = max(int(spec.coarsen), 1)
    cells = N / c ** d
    local = cells * float(max(c - 1, 1)) ** (3 * d - 2)
    coarse = cells * 400.0 * spec.n_src
    return local + coarse


class Server:
    """Continuous-batching request loop over a backend with open / launch / done / close.

    max_inflight = 1 gives the plain one-at-a-time path (no overlap), with the same
    admission and eviction rules.  policy "fifo" admits in arrival order; "sjf" admits
    the queued requests with the smallest estimated work first (a client's requests
    still run in order), which keeps small requests from waiting behind large ones."""

    def __init__(self, backend, budget_bytes: int, max_inflight: int = 8,
                 clock: Callable[[], float] = time.perf_counter, idle_sleep: float = 2e-4,
                 keep_results: bool = False, sleep: Callable[[float], None] = time.sleep,
                 policy: str = "fifo"):
        if policy not in ("fifo", "sjf"):
            raise ValueError("policy must be 'fifo' or 'sjf'")
        self.policy = policy
        self.backend = backend
        self.budget = int(budget_bytes)
        self.max_inflight = max(1, int(max_inflight))
        self.clock = clock
        self.sleep = sleep
        self.idle_sleep = idle_sleep
        self.keep_results = keep_results

    # -- memory ---------------------------------------------------------------------
    def _used(self, slots: Dict[int, Slot]) -> int:
        return sum(s.nbytes for s in slots.values())

    def _open(self, slots: Dict[int, Slot], req, now: float):
        """Open a session for req's client, evicting idle sessions (LRU) as needed.
        Returns the slot, None when it must wait, or 'reject' when it can never fit."""
        while True:
            try:
                h, nb = self.backend.open(req.instance, self.budget - self._used(slots))
                s = Slot(client=req.client, handle=h, nbytes=nb, last_used=now)
                slots[req.client] = s
                self.opened += 1
                return s
            except DoesNotFit:
                idle = [s for s in slots.values() if not s.busy]
                if idle:
                    victim = min(idle, key=lambda s: s.last_used)
                    self.backend.close(victim.handle)
                    del slots[victim.client]
                    self.evictions += 1
                    continue
                if not slots:
                    return "reject"       # does not fit even in an empty budget
                return None               # wait for running sessions to finish

    # -- loop -----------------------------------------------------------------------
    def run(self, requests, horizon: Optional[float] = None) -> Stats:
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        recs = {r.rid: Record(r.rid, r.client, r.arrival) for r in reqs}
        slots: Dict[int, Slot] = {}
        inflight = []            # (req, slot, token)
        queue = []               # arrived, not started (arrival order)
        nxt = 0
        self.evictions = 0
        self.opened = 0
        peak = 0
        t0 = self.clock()
        last_finish = 0.0
        while nxt < len(reqs) or queue or inflight:
            now = self.clock() - t0
            if horizon is not None and now > horizon and not inflight:
                break
            while nxt < len(reqs) and reqs[nxt].arrival <= now:
                queue.append(reqs[nxt])
                nxt += 1
            progressed = False
            # completions
            still = []
            for req, s, tok in inflight:
                if self.backend.done(tok):
                    r = recs[req.rid]
                    r.finish = self.clock() - t0
                    # a solve whose local pivots or coarse solve failed is not a result
                    ok = self.backend.ok(tok) if hasattr(self.backend, "ok") else True
                    r.status = "done" if ok else "failed"
                    if self.keep_results and ok:
                        r.result = self.backend.result(tok)
                    last_finish = max(last_finish, r.finish)
                    s.busy = False
                    s.last_used = r.finish
                    progressed = True
                else:
                    still.append((req, s, tok))
            inflight = still
            # admissions, in arrival order (or smallest work first); a client's requests
            # stay in order
            blocked = set()
            rest = []
            order = queue
            if self.policy == "sjf":
                first = {}
                for q in queue:                    # each client's earliest queued request
                    first.setdefault(q.client, q)
                heads = sorted(first.values(), key=lambda q: (estimated_work(q.instance), q.arrival))
                head_ids = {id(q) for q in heads}
                order = heads + [q for q in queue if id(q) not in head_ids]
            for req in order:
                if req.client in blocked or len(inflight) >= self.max_inflight:
                    rest.append(req)
                    blocked.add(req.client)
                    continue
                s = slots.get(req.client)
                if s is not None and s.busy:
                    rest.append(req)
                    blocked.add(req.client)
                    continue
                if s is None:
                    s = self._open(slots, req, now)
                    if s == "reject":
                        recs[req.rid].status = "rejected"
                        progressed = True
                        continue
                    if s is None:
                        rest.append(req)
                        blocked.add(req.client)
                        continue
                peak = max(peak, self._used(slots))
                s.busy = True
                r = recs[req.rid]
                r.start = self.clock() - t0
                r.status = "running"
                inflight.append((req, s, self.backend.launch(s.handle, req)))
                progressed = True
            queue = sorted(rest, key=lambda r: (r.arrival, r.rid))
            if not progressed:
                if nxt < len(reqs) and not inflight and not queue:
                    wait = reqs[nxt].arrival - (self.clock() - t0)
                    if wait > 0:
                        self.sleep(min(wait, 0.05))
                        continue
                self.sleep(self.idle_sleep)
        for s in list(slots.values()):
            self.backend.close(s.handle)
        return Stats(records=[recs[r.rid] for r in reqs], makespan=last_finish,
                     evictions=self.evictions, opened=self.opened, peak_bytes=peak)


class GpuBackend:
    """Sessions of the MSFV library on one GPU, one CUDA stream each.  A client's model
    at Gauss-Newton iteration k is m_0 + 0.01 k dm (m_0 a seeded lognormal field's log,
    dm seeded noise); its observed data are seeded noise.  Each request copies nothing
    from the host: the inputs are generated on the device, the step runs as a captured
    CUDA graph of msfv_forward + msfv_adjoint, and d_pred / grad are copied back to
    pinned host buffers."""

    def __init__(self, device=None, factor_mode: int = 0, use_graph: bool = True,
                 copy_back: bool = True):
        import torch
        self.torch = torch
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.factor_mode = factor_mode
        self.use_graph = use_graph
        self.copy_back = copy_back
        # the inputs of every new client are drawn on this one stream: torch caches the
        # temporaries of the field synthesis (up to ~10 GB at 256^3) per stream, so one
        # stream keeps that cache bounded instead of growing with the number of clients
        self.setup_stream = None

    def open(self, spec, budget_bytes: int):
        from . import workloads as W
        from .msfv import MSFV_OK, Batch, MSFVError, Session  # noqa: F401
        torch = self.torch
        if budget_bytes <= 0:
            raise DoesNotFit()
        stream = torch.cuda.Stream(device=self.device)
        prob = spec.problem()
        # this backend's own device buffers: m_0, dm, m, d_obs and the graph's outputs
        own = 8 * (4 * prob.N + 2 * prob.n_src * prob.n_rec)
        if budget_bytes <= own:
            raise DoesNotFit()
        try:
            sess = Session(prob, stream=stream, factor_mode=self.factor_mode,
                           hbm_budget_bytes=int(budget_bytes - own))
        except MSFVError as e:
            if e.code == 2:
                raise DoesNotFit() from e
            raise
        if int(sess.info()["workspace_bytes"]) + own > budget_bytes:
            # the library's up-front estimate was short of what it allocated
            sess.close()
            raise DoesNotFit()
        if self.setup_stream is None:
            self.setup_stream = torch.cuda.Stream(device=self.device)
        with torch.cuda.stream(self.setup_stream):
            m0_t = W.gaussian_random_field_device(prob.n, spec.corr_len, spec.seed, self.device)
            g = torch.Generator(device=self.device)
            g.manual_seed(spec.seed + 1)
            dm_t = torch.randn(prob.N, generator=g, device=self.device, dtype=torch.float64)
            dobs_t = 1e-3 * torch.randn((prob.n_src, prob.n_rec), generator=g,
                                        device=self.device, dtype=torch.float64)
        self.setup_stream.synchronize()
        # the client's own buffers live on its stream; the set-up temporaries are released
        # only after the copies that read them have run
        with torch.cuda.stream(stream):
            m0, dm, d_obs = m0_t.clone(), dm_t.clone(), dobs_t.clone()
            m = m0.clone()
        stream.synchronize()
        del m0_t, dm_t, dobs_t
        h = {"sess": sess, "stream": stream, "prob": prob, "m0": m0, "dm": dm, "m": m,
             "d_obs": d_obs, "batch": None}
        extra = 0
        if self.use_graph:
            try:
                with torch.cuda.stream(stream):
                    h["batch"] = Batch([sess], [m], [d_obs], stream=stream)
            except MSFVError as e:
                sess.close()
                if e.code == 2:          # its fused-launch buffers do not fit right now
                    raise DoesNotFit() from e
                raise
            # the batch's own buffers (fused work lists and scratch) count against the
            # budget like the session's
            extra = int(h["batch"].info()["device_bytes"])
        else:
            with torch.cuda.stream(stream):
                h["d_pred"] = torch.empty((prob.n_src, prob.n_rec), dtype=torch.float64,
                                          device=self.device)
                h["grad"] = torch.empty(prob.N, dtype=torch.float64, device=self.device)
        nbytes = int(sess.info()["workspace_bytes"]) + own + extra
        if nbytes > budget_bytes:
            if h["batch"] is not None:
                h["batch"].close()
            sess.close()
            raise DoesNotFit()
        return h, nbytes

    def launch(self, h, req):
        torch = self.torch
        st = h["stream"]
        with torch.cuda.stream(st):
            torch.add(h["m0"], h["dm"], alpha=0.01 * req.iteration, out=h["m"])
            if h["batch"] is not None:
                h["batch"].run()
                d_pred, grad = h["batch"].d_pred[0], h["batch"].grad[0]
            else:
                h["sess"].forward(h["m"], h["d_pred"])
                h["sess"].adjoint(h["d_obs"], h["grad"], want_phi=False)
                d_pred, grad = h["d_pred"], h["grad"]
            out = None
            if self.copy_back:
                out = (torch.empty(d_pred.shape, dtype=torch.float64, pin_memory=True),
                       torch.empty(grad.shape, dtype=torch.float64, pin_memory=True))
                out[0].copy_(d_pred, non_blocking=True)
                out[1].copy_(grad, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        return (ev, out, h)

    def done(self, tok) -> bool:
        return tok[0].query()

    def ok(self, tok) -> bool:
        """Numerical status of a finished request (its event has completed, so reading the
        status waits for nothing but a few bytes): False when the session's local pivots
        or coarse solve failed or a device-side wait expired.  Any other error (a CUDA
        error: the context is no longer usable) is raised, not counted as a failed
        request."""
        from .msfv import MSFVError
        h = tok[2]
        try:
            if h["batch"] is not None:
                h["batch"].check()
            else:
                h["sess"].check()
        except MSFVError as e:
            if e.code in (3, 4):          # MSFV_ERR_NUMERIC, MSFV_ERR_TIMEOUT
                return False
            raise
        return True

    def result(self, tok):
        if tok[1] is None:
            return None
        return tok[1][0].numpy().copy(), tok[1][1].numpy().copy()

    def close(self, h):
        h["stream"].synchronize()
        if h["batch"] is not None:
            h["batch"].check()
            h["batch"].close()
        h["sess"].close()
