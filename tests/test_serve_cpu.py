"""Scheduling logic of the continuous-batching server, against a fake pool
on the CPU (no GPU): admission by footprint, backfill with a bound on how
long the head of the queue can be bypassed, collection of finished jobs and
their latency."""
import pytest

pytest.importorskip("numpy")


class FakePool:
    """Arena of `budget` units; a job of nx*ny sites takes nx*ny units."""

    def __init__(self, budget, lb):
        self.budget, self.used, self.lb = budget, 0, lb
        self.jobs = {}
        self.next = 0
        self.peak = 0
        self.runs = []

    def admit(self, p, seed, steps):
        need = p["nx"] * p["ny"]
        if self.used + need > self.budget:
            raise self.lb.LbError(self.lb.LB_ERR_NOMEM, "admit")
        if p["nx"] < 8:
            raise self.lb.LbError(self.lb.LB_ERR_INVALID, "admit")
        j = self.next
        self.next += 1
        self.jobs[j] = dict(need=need, steps=steps, done=0)
        self.used += need
        self.peak = max(self.peak, self.used)
        return j

    def run(self, q):
        self.runs.append(sorted(self.jobs))
        for j in self.jobs.values():
            j["done"] += min(q, j["steps"] - j["done"])
        return sum(1 for j in self.jobs.values() if j["done"] < j["steps"])

    def poll(self, j):
        return self.jobs[j]["done"], self.jobs[j]["done"] >= self.jobs[j]["steps"]

    def stress(self, j):
        return {"step": self.jobs[j]["done"]}

    def release(self, j):
        self.used -= self.jobs.pop(j)["need"]


@pytest.fixture
def lb():
    import paper_0807_4471_gb300 as lb
    from paper_0807_4471_gb300 import build
    build.build()
    return lb


def make(spec):
    return dict(nx=spec["nx"], ny=spec["ny"])


def test_all_jobs_finish_within_budget(lb):
    from paper_0807_4471_gb300.serve import Server
    pool = FakePool(budget=100 * 100, lb=lb)
    srv = Server(pool, make, quantum=10, clock=iter(range(10 ** 6)).__next__)
    sizes = [(64, 64), (96, 96), (32, 32), (80, 80), (16, 16), (100, 100), (48, 48)]
    jobs = [srv.submit(dict(nx=a, ny=b, steps=25 + 7 * k, seed=k)) for k, (a, b) in enumerate(sizes)]
    srv.run_until_idle(1000)
    assert all(j.done and j.error is None for j in jobs)
    assert pool.peak <= pool.budget
    assert [j.result["step"] for j in jobs] == [25 + 7 * k for k in range(len(sizes))]
    assert all(j.latency > 0 for j in jobs)
    assert srv.stats.finished == len(sizes)
    assert srv.stats.site_updates == sum(a * b * (25 + 7 * k) for k, (a, b) in enumerate(sizes))


def test_backfill_and_head_of_line_bound(lb):
    from paper_0807_4471_gb300.serve import Server
    pool = FakePool(budget=10000, lb=lb)
    srv = Server(pool, make, quantum=10, max_bypass=2, clock=iter(range(10 ** 6)).__next__)
    big_running = srv.submit(dict(nx=90, ny=90, steps=100))     # 8100 units
    head = srv.submit(dict(nx=60, ny=60, steps=10))             # 3600: must wait
    small = [srv.submit(dict(nx=20, ny=20, steps=10)) for _ in range(6)]
    srv.step()
    # the small jobs backfill around the waiting head
    assert big_running.admitted is not None and head.admitted is None
    assert sum(1 for s in small if s.admitted is not None) >= 1
    srv.run_until_idle(1000)
    assert head.done and all(s.done for s in small)


def test_invalid_job_fails_without_blocking(lb):
    from paper_0807_4471_gb300.serve import Server
    pool = FakePool(budget=10000, lb=lb)
    srv = Server(pool, make, quantum=10, clock=iter(range(10 ** 6)).__next__)
    bad = srv.submit(dict(nx=4, ny=64, steps=10))
    good = srv.submit(dict(nx=32, ny=32, steps=10))
    srv.run_until_idle(100)
    assert bad.done and bad.error is not None
    assert good.done and good.error is None


def test_percentile():
    from paper_0807_4471_gb300.serve import percentile
    assert percentile([1, 2, 3, 4, 5], 50) == 3
    assert percentile(range(101), 99) == 99


def test_cancel_queued_and_running_jobs_and_log(lb, tmp_path):
    """A queued job is withdrawn, a running one is stopped and its memory
    freed for the next admission; each ended job leaves one JSON line."""
    import json
    from paper_0807_4471_gb300.serve import Server
    pool = FakePool(budget=2 * 64 * 64, lb=lb)
    log = tmp_path / "jobs.jsonl"
    srv = Server(pool, make, quantum=10, log_path=str(log))
    a = srv.submit(dict(nx=64, ny=64, steps=1000))
    b = srv.submit(dict(nx=64, ny=64, steps=30))
    c = srv.submit(dict(nx=64, ny=64, steps=20))      # does not fit yet
    srv.step()
    assert a._slot in srv.running and b._slot in srv.running and c in srv.queue
    assert srv.cancel(a)                              # running: memory freed
    assert pool.used == 64 * 64
    d = srv.submit(dict(nx=64, ny=64, steps=10))
    assert srv.cancel(d)                              # queued: withdrawn
    assert not srv.cancel(d)
    srv.run_until_idle()
    assert b.result and c.result and a.error == "cancelled" and d.error == "cancelled"
    assert srv.stats.cancelled == 2 and srv.stats.finished == 2
    recs = [json.loads(line) for line in log.read_text().splitlines()]
    assert sorted(r["id"] for r in recs) == sorted([a.id, b.id, c.id, d.id])
    assert {r["id"]: r["error"] for r in recs}[a.id] == "cancelled"
    assert all(r["latency"] is not None for r in recs)


def test_failed_result_is_not_counted_as_finished(lb):
    """A job whose result cannot be read (a latched device error) counts as
    failed only: not as finished, and its steps add no site updates."""
    from paper_0807_4471_gb300.serve import Server

    class BadStressPool(FakePool):
        def stress(self, j):
            if self.jobs[j]["need"] == 16 * 16:
                raise self.lb.LbError(self.lb.LB_ERR_NONFINITE, "stress")
            return super().stress(j)

    pool = BadStressPool(10 ** 6, lb)
    srv = Server(pool, make, quantum=10)
    good = srv.submit(dict(nx=8, ny=8, steps=20), arrival=0.0)
    bad = srv.submit(dict(nx=16, ny=16, steps=20), arrival=0.0)
    srv.run_until_idle()
    assert good.result is not None and good.error is None
    assert bad.result is None and bad.error is not None and "status -4" in bad.error
    assert srv.stats.finished == 1 and srv.stats.failed == 1
    assert srv.stats.site_updates == 8 * 8 * 20
    assert pool.used == 0
