"""Host logic of the continuous-batching server (no GPU): admission by HBM
budget, arrival-order admission, batching of everything ready into one work
list, the one-at-a-time baseline, rejection of requests that can never fit."""
import numpy as np

from paper_2103_14024_gb300 import synth as S
from paper_2103_14024_gb300.serve import Admission, RenderServer, Request, summarize


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-4          # every reading advances simulated time by 0.1 ms
        return self.t


class FakeEvent:
    def __init__(self, clock, done_at):
        self.clock, self.done_at = clock, done_at

    def query(self):
        return self.clock.t >= self.done_at


class Recorder:
    """Fake launcher: a launch takes 0.5 ms + 1 ns per ray of simulated time."""

    def __init__(self, clock, server):
        self.clock, self.server, self.launches, self.max_used = clock, server, [], 0

    def __call__(self, reqs, stream):
        self.launches.append([r.rid for r in reqs])
        self.max_used = max(self.max_used, self.server.adm.resident + self.server.adm.used)
        return FakeEvent(self.clock, self.clock.t + 5e-4 + 1e-9 * sum(r.rays for r in reqs))


def _requests(n, rate, seed=5):
    arr, tree, cams = S.serve_requests(seed, n, rate_hz=rate)
    return [Request(i, float(arr[i]), int(tree[i]), cams[i]) for i in range(n)]


def _server(budget, mode_streams=3):
    clock = FakeClock()
    srv = RenderServer(trees=[None] * 4, hbm_budget_bytes=budget, streams=mode_streams, clock=clock,
                       launcher=lambda *a: None, allocator=lambda r: None, stream_factory=lambda n: [None] * n)
    rec = Recorder(clock, srv)
    srv.launcher = rec
    return srv, rec


def test_admission_accounting():
    a = Admission(100, 30)
    assert a.take(50) and not a.take(21) and a.take(20)
    a.release(50)
    assert a.used == 20 and a.fits(50)


def test_batch_mode_respects_budget_and_order():
    reqs = _requests(200, rate=3000.0)
    budget = 200_000_000            # outputs only (resident = 0 with a fake launcher)
    srv, rec = _server(budget)
    srv.run(reqs, mode="batch")
    assert all(r.t_done >= r.t_launch >= r.t_admit >= r.arrival for r in reqs)
    assert rec.max_used <= budget
    flat = [i for launch in rec.launches for i in launch]
    assert flat == sorted(flat) == list(range(200))          # FIFO admission and launch
    assert max(len(l) for l in rec.launches) > 1                # several requests share a launch
    s = summarize(reqs)
    assert s["requests"] == 200 and s["p99_ms"] >= s["p50_ms"] > 0


def test_alone_mode_one_request_per_launch():
    reqs = _requests(50, rate=3000.0)
    srv, rec = _server(10 ** 10)
    srv.run(reqs, mode="alone")
    assert all(len(l) == 1 for l in rec.launches)
    # one launch at a time: each starts after the previous finished
    order = sorted(reqs, key=lambda r: r.t_launch)
    assert all(b.t_launch >= a.t_done for a, b in zip(order, order[1:]))


def test_batching_lowers_latency_under_load():
    reqs_a = _requests(300, rate=5000.0, seed=9)
    reqs_b = _requests(300, rate=5000.0, seed=9)
    s1, _ = _server(10 ** 10)
    s1.run(reqs_a, mode="batch")
    s2, _ = _server(10 ** 10)
    s2.run(reqs_b, mode="alone")
    assert summarize(reqs_a)["p99_ms"] < summarize(reqs_b)["p99_ms"]


def test_oversized_request_rejected_not_stuck():
    reqs = _requests(20, rate=1000.0)
    big = max(r.rays for r in reqs) * 12
    srv, rec = _server(big - 1)
    srv.run(reqs, mode="batch")
    rej = [r for r in reqs if r.rejected]
    assert rej and all(r.rays * 12 > big - 1 for r in rej)
    assert all(r.t_done >= 0 for r in reqs)


def test_summary_breakdowns_are_consistent():
    """Per-resolution groups partition the requests, and the queue/run split
    adds up to the latency of each request."""
    reqs = _requests(200, rate=3000.0, seed=11)
    srv, _ = _server(10 ** 10)
    srv.run(reqs, mode="batch")
    s = summarize(reqs)
    assert sum(v["n"] for v in s["by_resolution"].values()) == s["requests"] == 200
    for key, v in s["by_resolution"].items():
        w, h = (int(x) for x in key.split("x"))
        lat = [(r.t_done - r.arrival) * 1e3 for r in reqs if (int(r.cam["width"]), int(r.cam["height"])) == (w, h)]
        assert v["n"] == len(lat) and abs(v["p50_ms"] - float(np.percentile(lat, 50))) < 1e-3
    for r in reqs:
        assert r.arrival <= r.t_admit <= r.t_launch <= r.t_done
    assert s["p50_wait_ms"] >= 0 and s["p50_run_ms"] > 0


def test_on_done_hands_over_each_output_once_and_drops_it():
    """With on_done, every finished output is handed over exactly once, after
    completion, and the server keeps no reference to it afterwards: the bytes
    returned to the budget are free."""
    reqs = _requests(60, 5000.0)
    clock = FakeClock()
    live = set()
    srv = RenderServer(trees=[None] * 4, hbm_budget_bytes=30_000_000, streams=3, clock=clock,
                       launcher=lambda *a: None, allocator=lambda r: (live.add(r.rid), ("img", r.rid))[1],
                       stream_factory=lambda n: [None] * n)
    rec = Recorder(clock, srv)
    srv.launcher = rec
    seen = []

    def on_done(r):
        assert r.rgb == ("img", r.rid) and r.t_done >= r.t_launch >= r.t_admit >= r.arrival
        seen.append(r.rid)
        live.discard(r.rid)

    srv.run(reqs, mode="batch", on_done=on_done)
    done = [r.rid for r in reqs if not r.rejected]
    assert sorted(seen) == sorted(done) and len(seen) == len(set(seen))
    assert all(r.rgb is None for r in reqs) and not live
    assert rec.max_used <= 30_000_000 and srv.adm.used == 0


def test_small_requests_go_to_the_priority_stream():
    """With priority_pixels, every launch on the high-priority stream slot holds
    only requests of at most that many pixels, each request is launched once,
    and everything completes within the budget."""
    reqs = _requests(120, 3000.0)
    clock = FakeClock()
    made = []

    def factory(n, high=False):
        made.append((n, high))
        return [("hi" if high else "lo", i) for i in range(n)]

    srv = RenderServer(trees=[None] * 4, hbm_budget_bytes=60_000_000, streams=2, clock=clock,
                       launcher=lambda *a: None, allocator=lambda r: None, stream_factory=factory,
                       priority_pixels=512 * 512)
    launches = []

    def launcher(batch, stream):
        launches.append((stream, [r.rid for r in batch], [r.rays for r in batch]))
        return FakeEvent(clock, clock.t + 5e-4 + 1e-9 * sum(r.rays for r in batch))

    srv.launcher = launcher
    srv.run(reqs, mode="batch")
    assert made == [(2, False), (1, True)]
    hi = [l for l in launches if l[0][0] == "hi"]
    assert hi and all(max(rays) <= 512 * 512 for _, _, rays in hi)
    ids = [i for _, rids, _ in launches for i in rids]
    done = [r.rid for r in reqs if not r.rejected]
    assert sorted(ids) == sorted(done) and len(ids) == len(set(ids))
    assert all(r.t_done >= r.t_launch >= r.t_admit >= r.arrival for r in reqs if not r.rejected)
    # one request at a time ignores the priority stream
    made.clear()
    launches.clear()
    reqs = _requests(20, 3000.0)
    srv.run(reqs, mode="alone")
    assert made == [(1, False)] and all(len(r) == 1 for _, r, _ in launches)
