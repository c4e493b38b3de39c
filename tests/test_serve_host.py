"""Host logic of the request loop (CPU): admission by HBM budget, LRU eviction of idle
sessions, in-order Gauss-Newton iterations per client, rejection of sessions larger
than the budget, overlap limits and latency accounting, on a simulated backend."""
import pytest

from paper_1707_07598_gb300 import workloads as W
from paper_1707_07598_gb300.serve import DoesNotFit, Server


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-6)


class FakeBackend:
    """Session bytes = cells; a request takes cells * 1e-7 s after its launch."""

    def __init__(self, clock):
        self.clock = clock
        self.open_now = {}
        self.launched = []
        self.closed = 0

    def open(self, spec, budget):
        nb = spec.n[0] * spec.n[1] * spec.n[2]
        if nb > budget:
            raise DoesNotFit()
        h = object()
        self.open_now[id(h)] = nb
        return h, nb

    def launch(self, h, req):
        assert id(h) in self.open_now
        self.launched.append(req.rid)
        spec = req.instance
        return (self.clock() + spec.n[0] * spec.n[1] * spec.n[2] * 1e-7, req.rid)

    def done(self, tok):
        return self.clock() >= tok[0]

    def result(self, tok):
        return tok[1]

    def close(self, h):
        del self.open_now[id(h)]
        self.closed += 1


def reqs(seed=5, duration=2.0, rate=40.0):
    return W.served_requests(rate=rate, duration=duration, seed=seed, sizes=(16, 32, 64),
                             coarsenings=(4, 8), max_src=8)


@pytest.mark.parametrize("inflight", [1, 4])
def test_all_complete_in_client_order_within_budget(inflight):
    clk = FakeClock()
    be = FakeBackend(clk)
    rs = reqs()
    budget = 3 * 64 ** 3
    st = Server(be, budget, max_inflight=inflight, clock=clk, sleep=clk.sleep,
                keep_results=True).run(rs)
    assert all(r.status == "done" for r in st.records)
    assert st.peak_bytes <= budget
    assert be.open_now == {}                      # every session closed at the end
    by_client = {}
    for q in rs:
        by_client.setdefault(q.client, []).append(q)
    rec = {r.rid: r for r in st.records}
    for qs in by_client.values():
        qs.sort(key=lambda q: q.iteration)
        for a, b in zip(qs, qs[1:]):              # iteration k+1 starts after k finished
            assert rec[b.rid].start >= rec[a.rid].finish
    for r in st.records:
        assert r.start >= r.arrival and r.finish > r.start and r.result == r.rid
    if inflight == 1:                              # plain path: no two requests overlap
        iv = sorted((r.start, r.finish) for r in st.records)
        for (s0, f0), (s1, f1) in zip(iv, iv[1:]):
            assert s1 >= f0


def test_eviction_under_a_tight_budget_and_rejection():
    clk = FakeClock()
    be = FakeBackend(clk)
    rs = reqs(seed=7)
    budget = 64 ** 3 + 32 ** 3                    # at most one 64^3 session resident
    st = Server(be, budget, max_inflight=4, clock=clk, sleep=clk.sleep).run(rs)
    assert all(r.status == "done" for r in st.records)
    assert st.evictions > 0 and st.peak_bytes <= budget
    # a budget smaller than the largest session rejects its requests, serves the rest
    clk2 = FakeClock()
    st2 = Server(FakeBackend(clk2), 32 ** 3, max_inflight=4, clock=clk2,
                 sleep=clk2.sleep).run(rs)
    big = {q.rid for q in rs if q.instance.n[0] == 64}
    for r in st2.records:
        assert r.status == ("rejected" if r.rid in big else "done")


def test_overlap_raises_throughput_and_latency_stats():
    rs = reqs(seed=9, rate=200.0)
    out = {}
    for k in (1, 8):
        clk = FakeClock()
        out[k] = Server(FakeBackend(clk), 10 ** 9, max_inflight=k, clock=clk,
                        sleep=clk.sleep).run(rs)
    assert out[8].throughput > out[1].throughput
    assert out[8].percentile(50) <= out[1].percentile(50)
    assert out[8].percentile(99) >= out[8].percentile(50)


def test_served_request_stream_shape():
    rs = W.served_requests(rate=50.0, duration=60.0, seed=5)
    assert 2500 < len(rs) < 3500                   # Poisson(3000)
    assert all(0 <= q.arrival < 60.0 for q in rs)
    seen = {}
    for q in rs:                                    # iterations count up per client
        assert q.iteration == seen.get(q.client, 0)
        seen[q.client] = q.iteration + 1
        assert q.instance.n[0] in (32, 64, 128, 256) and q.instance.coarsen in (4, 8, 16)
        assert 1 <= q.instance.n_src <= 64


def test_smallest_work_first_cuts_the_median_latency_under_overload():
    rs = W.served_requests(rate=400.0, duration=1.0, seed=13, sizes=(16, 32, 64),
                           coarsenings=(4, 8), max_src=8)
    out = {}
    for pol in ("fifo", "sjf"):
        clk = FakeClock()
        out[pol] = Server(FakeBackend(clk), 10 ** 9, max_inflight=2, clock=clk,
                          sleep=clk.sleep, policy=pol).run(rs)
        assert all(r.status == "done" for r in out[pol].records)
    assert out["sjf"].percentile(50) < out["fifo"].percentile(50)
    # client order is still respected under sjf
    rec = {r.rid: r for r in out["sjf"].records}
    by_client = {}
    for q in rs:
        by_client.setdefault(q.client, []).append(q)
    for qs in by_client.values():
        qs.sort(key=lambda q: q.iteration)
        for a, b in zip(qs, qs[1:]):
            assert rec[b.rid].start >= rec[a.rid].finish


class FailingBackend(FakeBackend):
    """FakeBackend whose solves for the listed request ids finish with a bad status."""

    def __init__(self, clock, bad):
        super().__init__(clock)
        self.bad = set(bad)

    def ok(self, tok):
        return tok[1] not in self.bad


def test_a_failed_solve_is_not_counted_and_the_loop_goes_on():
    clock = FakeClock()
    rs = reqs(seed=8)
    bad = {rs[1].rid, rs[4].rid}
    be = FailingBackend(clock, bad)
    st = Server(be, budget_bytes=10 ** 9, max_inflight=4, clock=clock, sleep=clock.sleep,
                keep_results=True).run(rs)
    failed = {r.rid for r in st.failed()}
    assert failed == bad
    done = st.done()
    assert len(done) == len(rs) - len(bad)
    assert all(r.rid not in bad for r in done) and all(r.result == r.rid for r in done)
    assert all(r.result is None for r in st.failed())
    # throughput and latencies count the good results only
    assert st.throughput == pytest.approx(len(done) / st.makespan)
    lat = sorted(r.latency for r in done)
    assert st.percentile(100) == pytest.approx(lat[-1])
    # every request was launched once, in order per client, and every session closed
    assert sorted(be.launched) == sorted(r.rid for r in rs)
    assert not be.open_now
