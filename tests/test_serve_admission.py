"""Host logic of the serving loop (serve.run) against a fake server, on the
CPU: requests are admitted in arrival order while their device memory fits
the budget and the server has free task slots; a refused request's ligand
is released; every request completes with its own results; the memory in
use never exceeds the budget while more than one request is in flight."""
import numpy as np
import pytest

from paper_2203_02096_gb300 import capi, serve


class FakeLigand:
    live = 0

    def __init__(self, lig):
        self.n_genes = 7 + lig["torsions"]
        self.bytes = lig["bytes"]
        self.name = lig["name"]
        FakeLigand.live += 1

    def device_bytes(self):
        return self.bytes

    def free(self):
        FakeLigand.live -= 1


class FakeServer:
    """Task slots with a fixed capacity; a request's runs finish after a
    fixed number of polls."""

    def __init__(self, capacity, polls_to_finish=3):
        self.capacity, self.polls = capacity, polls_to_finish
        self.next_task = 0
        self.active = {}            # first task -> [nruns, polls left, ligand name]
        self.order = []             # ligand names in submit order
        self.in_use = 0

    def submit(self, grids, lig, params, seed):
        if self.in_use + params.nruns > self.capacity:
            return None
        first = self.next_task
        self.next_task += params.nruns
        self.in_use += params.nruns
        self.active[first] = [params.nruns, self.polls, lig.name]
        self.order.append(lig.name)
        return first

    def done(self, first, nruns):
        rec = self.active[first]
        rec[1] -= 1
        return rec[1] <= 0

    def result(self, first, nruns, n_genes):
        rec = self.active.pop(first)
        self.in_use -= rec[0]
        g = np.full((nruns, n_genes), float(first), np.float32)
        return g, np.full(nruns, -float(first)), np.full(nruns, 100, np.int64)


@pytest.fixture
def fake_capi(monkeypatch):
    FakeLigand.live = 0
    monkeypatch.setattr(capi, "ligand_from", lambda ctx, lig: FakeLigand(lig))
    yield


def _requests(n, seed=0):
    rng = np.random.default_rng(seed)
    arrivals = np.sort(rng.uniform(0.0, 0.02, size=n))
    return [serve.Request({"name": k, "torsions": int(rng.integers(0, 8)), "bytes": int(rng.integers(1, 5)) << 20},
                          0, seed=k, arrival=float(a)) for k, a in enumerate(arrivals)]


def test_all_requests_complete_in_arrival_order(fake_capi):
    reqs = _requests(24)
    params = capi.default_params(nruns=4)
    srv = FakeServer(capacity=16)
    rep = serve.run(None, srv, [None], reqs, params, mem_budget=64 << 20, poll_sleep=1e-4, timeout=30.0)
    assert len(rep.done) == len(reqs)
    assert srv.order == [r.ligand["name"] for r in sorted(reqs, key=lambda r: r.arrival)]
    assert FakeLigand.live == 0                      # every ligand handle released
    assert 1 <= rep.max_in_flight <= 4               # 16 slots / 4 runs per request
    for d in rep.done:
        assert d.latency >= 0.0
        assert d.best_geno.shape == (4, d.request.ligand["torsions"] + 7)
        assert np.all(d.evals == 100)
    s = rep.summary()
    assert s["requests"] == len(reqs) and s["p99_s"] >= s["p50_s"] >= 0.0


def test_memory_budget_bounds_the_requests_in_flight(fake_capi, monkeypatch):
    reqs = _requests(20, seed=1)
    params = capi.default_params(nruns=2)
    budget = 9 << 20
    srv = FakeServer(capacity=1 << 10, polls_to_finish=5)
    peak = {"bytes": 0, "in_flight": 0}
    submit = srv.submit

    def watched_submit(grids, lig, p, seed):
        first = submit(grids, lig, p, seed)
        if first is not None:
            live = sum(r.ligand["bytes"] + p.nruns * serve.ROW_BYTES for r in reqs
                       if r.ligand["name"] in [v[2] for v in srv.active.values()])
            if len(srv.active) > 1:
                assert live <= budget, (live, budget)
            peak["bytes"] = max(peak["bytes"], live)
            peak["in_flight"] = max(peak["in_flight"], len(srv.active))
        return first

    monkeypatch.setattr(srv, "submit", watched_submit)
    rep = serve.run(None, srv, [None], reqs, params, mem_budget=budget, poll_sleep=1e-4, timeout=30.0)
    assert len(rep.done) == len(reqs)
    assert peak["in_flight"] >= 2                    # the budget admits several 1-4 MB requests at once
    assert FakeLigand.live == 0


def test_a_request_larger_than_the_budget_runs_alone(fake_capi):
    reqs = [serve.Request({"name": 0, "torsions": 2, "bytes": 1 << 20}, 0, seed=0, arrival=0.0),
            serve.Request({"name": 1, "torsions": 2, "bytes": 64 << 20}, 0, seed=1, arrival=0.0),
            serve.Request({"name": 2, "torsions": 2, "bytes": 1 << 20}, 0, seed=2, arrival=0.0)]
    params = capi.default_params(nruns=1)
    srv = FakeServer(capacity=64)
    rep = serve.run(None, srv, [None], reqs, params, mem_budget=8 << 20, poll_sleep=1e-4, timeout=30.0)
    assert [d.request.ligand["name"] for d in rep.done] == [0, 1, 2]
    assert srv.order == [0, 1, 2]
    assert FakeLigand.live == 0


def test_steady_throughput_counts_completions_while_requests_arrive():
    """Served rate without ramp-up and drain: 1 request/s arriving for 20 s,
    each done 5 s after it arrives -> completions at 5..24 s, of which those
    in [5, 19] (first completion to last arrival) give 14 in 14 s."""
    from paper_2203_02096_gb300 import serve
    rep = serve.ServiceReport()
    for k in range(20):
        r = serve.Request(ligand=None, grid_index=0, seed=k, arrival=float(k))
        rep.done.append(serve.Done(r, 5.0, None, None, None))
    rep.wall = 24.0
    assert rep.steady_throughput() == pytest.approx(14 / 14)
    assert rep.summary()["throughput_per_s"] == pytest.approx(20 / 24)
    # a stream shorter than a second of overlap has no steady rate
    short = serve.ServiceReport(done=rep.done[:1], wall=5.0)
    assert short.steady_throughput() is None


class FakePlain:
    """A plain-form docking that finishes after a fixed number of polls."""
    started = []
    polls = 3

    def __init__(self, ctx, grids, lig, params, seed):
        self.lig, self.params, self.left = lig, params, FakePlain.polls
        FakePlain.started.append((lig.name, params.ls_threads))

    def done(self):
        self.left -= 1
        return self.left <= 0

    def result(self):
        R = self.params.nruns
        return (np.full((R, self.lig.n_genes), -1.0, np.float32), np.full(R, -7.0), np.full(R, 100, np.int64))


@pytest.fixture
def fake_plain(monkeypatch):
    FakePlain.started, FakePlain.polls = [], 3
    monkeypatch.setattr(serve, "PlainDocking", FakePlain)
    yield


def _spaced(n, gap):
    return [serve.Request({"name": k, "torsions": 3, "bytes": 1 << 20}, 0, seed=k, arrival=k * gap) for k in range(n)]


def test_idle_gpu_requests_take_the_plain_route(fake_capi, fake_plain):
    """Requests that arrive one at a time, each after the previous one is
    done, are all docked in the plain form with the asked team width;
    nothing reaches the server."""
    params = capi.default_params(nruns=4, ls_threads=128)
    srv = FakeServer(capacity=64)
    rep = serve.run(None, srv, [None], _spaced(6, 0.02), params, poll_sleep=1e-4, timeout=30.0, idle_plain=True,
                    plain_threads=32)
    assert [d.route for d in rep.done] == ["plain"] * 6
    assert [n for n, _ in FakePlain.started] == list(range(6))
    assert all(t == 32 for _, t in FakePlain.started)
    assert params.ls_threads == 128                   # the caller's parameters are untouched
    assert srv.order == [] and FakeLigand.live == 0
    assert rep.summary()["plain_route"] == 6
    assert all(d.best_geno.shape == (4, 10) and np.all(d.best_E == -7.0) for d in rep.done)


def test_a_short_queue_waits_for_the_plain_slot_a_long_one_goes_to_the_server(fake_capi, fake_plain):
    params = capi.default_params(nruns=2)
    # three at once: the first docks plain, two wait for it (queue <= 4)
    srv = FakeServer(capacity=64)
    FakePlain.polls = 3
    rep = serve.run(None, srv, [None], _spaced(3, 0.0), params, poll_sleep=1e-4, timeout=30.0, idle_plain=True)
    assert sorted(d.route for d in rep.done) == ["plain"] * 3 and srv.order == []
    # one request, then nineteen more while it docks plain: the queue (19 >
    # 4) goes to the persistent kernel, in arrival order, once the plain
    # docking is done (the two never share the GPU)
    FakePlain.started, FakePlain.polls = [], 400     # the plain docking outlasts the arrivals
    reqs = _spaced(20, 0.0)
    for r in reqs[1:]:
        r.arrival = 0.005
    srv = FakeServer(capacity=64, polls_to_finish=5)
    submit, plain_done = srv.submit, []

    def watched_submit(grids, lig, p, seed):
        assert plain_done, "a server submission beside a running plain docking"
        return submit(grids, lig, p, seed)

    srv.submit = watched_submit
    done = FakePlain.done

    def watched_done(self):
        d = done(self)
        if d:
            plain_done.append(True)
        return d

    FakePlain.done = watched_done
    try:
        rep = serve.run(None, srv, [None], reqs, params, poll_sleep=1e-4, timeout=30.0, idle_plain=True,
                        plain_queue=4)
    finally:
        FakePlain.done = done
    routes = {d.request.ligand["name"]: d.route for d in rep.done}
    assert len(routes) == 20 and routes[0] == "plain"
    assert all(routes[k] == "served" for k in range(1, 20))
    assert srv.order == list(range(1, 20))
    # twenty at once: the queue is long from the start, all are served
    FakePlain.started, FakePlain.polls = [], 3
    srv = FakeServer(capacity=64, polls_to_finish=5)
    rep = serve.run(None, srv, [None], _spaced(20, 0.0), params, poll_sleep=1e-4, timeout=30.0, idle_plain=True)
    assert [d.route for d in rep.done] == ["served"] * 20 and FakePlain.started == []
    assert FakeLigand.live == 0


def test_idle_plain_needs_adadelta(fake_capi, fake_plain):
    params = capi.default_params(nruns=2, ls_method=1)
    with pytest.raises(ValueError):
        serve.run(None, FakeServer(capacity=8), [None], _spaced(1, 0.0), params, idle_plain=True)
