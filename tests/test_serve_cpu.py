"""Host-side serving logic on the CPU: HBM-budget admission, FIFO order and latency
bookkeeping of the open-loop driver, against a simulated single-queue server and clock."""
import pytest

from paper_2005_01442_gb300 import serve


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-4)


class FakeServer:
    """FIFO server that needs `service` seconds per request, one at a time."""
    name = "fake"

    def __init__(self, clock, service):
        self.clock, self.service = clock, service
        self.busy_until = 0.0
        self.order = []

    def submit(self, req, out):
        start = max(self.clock(), self.busy_until)
        self.busy_until = start + self.service
        self.order.append(req.arrival)
        return self.busy_until

    def pump(self):
        return True

    def done(self, handle):
        return self.clock() >= handle


class Cam:
    def __init__(self, w, h):
        self.width, self.height = w, h


def test_open_loop_latencies_and_fifo():
    clock = Clock()
    srv = FakeServer(clock, 0.010)
    reqs = [serve.Request(0.1 * k, 0, 0, Cam(32, 32)) for k in range(20)]
    budget = serve.ImageBudget(10 ** 9, lambda h, w: object())
    res = serve.run_open_loop(srv, reqs, budget, clock=clock, sleep=clock.sleep)
    assert srv.order == [r.arrival for r in reqs]
    # an idle server answers every request after one service time (to the polling step)
    assert all(0.010 <= x <= 0.0102 for x in res["latencies_s"])
    assert res["requests"] == 20 and budget.used == 0


def test_budget_admission_queues_requests():
    clock = Clock()
    srv = FakeServer(clock, 0.010)
    img = 64 * 64 * 16
    reqs = [serve.Request(0.0, 0, 0, Cam(64, 64)) for _ in range(6)]
    budget = serve.ImageBudget(2 * img, lambda h, w: object())  # two images at a time
    peak = []
    orig = budget.try_acquire

    def spy(h, w):
        b = orig(h, w)
        peak.append(budget.used)
        return b

    budget.try_acquire = spy
    res = serve.run_open_loop(srv, reqs, budget, clock=clock, sleep=clock.sleep)
    assert max(peak) <= 2 * img
    lat = sorted(res["latencies_s"])
    # served one after another: the k-th waits k service times
    for k, x in enumerate(lat):
        assert abs(x - 0.010 * (k + 1)) < 2e-3
    with pytest.raises(ValueError):
        budget.try_acquire(1024, 1024)


def test_poisson_arrivals_rate_and_determinism():
    mk = lambda rng, v, w, h: Cam(w, h)  # noqa: E731
    a = serve.poisson_requests(5, 200.0, 20.0, [1, 2, 3], [7, 8], [(512, 512), (1024, 1024)], mk)
    b = serve.poisson_requests(5, 200.0, 20.0, [1, 2, 3], [7, 8], [(512, 512), (1024, 1024)], mk)
    assert [r.arrival for r in a] == [r.arrival for r in b]
    assert abs(len(a) / 20.0 - 200.0) < 15.0
    assert {r.vol_id for r in a} == {1, 2, 3} and {r.tf_id for r in a} == {7, 8}
    assert all(x.arrival < y.arrival for x, y in zip(a, a[1:]))
    assert serve.percentile([3, 1, 2, 4], 50) == 2 and serve.percentile([3, 1, 2, 4], 99) == 4
