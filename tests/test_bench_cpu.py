"""bench.py's result assembly on the CPU, with fakes for the device parts: the roofline of a
render call, the measured peaks and the serving sweep's summary (best images/s under the p99
cap)."""
import types

import pytest

import bench


class FakeR:
    def microbench(self, kind):
        return {0: 70e12, 1: 30e12, 2: 31e12, 3: 2e12}[kind]

    def build_occupancy(self, v, t, b):
        pass


def test_peaks_take_the_lower_of_measured_and_unit_count():
    p = bench.measure_peaks(FakeR(), 152)
    assert p["fp32_tflops"] == pytest.approx(70.0)
    assert p["l1_gbs"] == pytest.approx(30000.0)
    fast = FakeR()
    fast.microbench = lambda k: 1e18
    p = bench.measure_peaks(fast, 152)
    assert p["fp32_tflops"] == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)
    assert p["l1_gbs"] == pytest.approx(152 * 128 * 2.07e9 / 1e9)


def test_roofline_terms_and_binding_term():
    peaks = {"fp32_tflops": 80.0, "l1_gbs": 40000.0}
    # 1e9 executed samples in 10 ms: ALU 230e9 / 0.01 = 23 TFLOP/s, gather 128e9 / 0.01 =
    # 12.8 TB/s of 40 TB/s
    r = bench.roofline(10 ** 9, 5 * 10 ** 8, 10.0, peaks, "k")
    assert r["alu_frac"] == pytest.approx(23.0 / 80.0)
    assert r["gather_frac"] == pytest.approx(12800.0 / 40000.0)
    assert r["frac"] == pytest.approx(max(r["alu_frac"], r["gather_frac"]))
    assert r["bound"] == "l1_gather" and r["unit"] == "GB/s"
    assert r["frac_resampled"] == pytest.approx(r["frac"] / 2)
    assert r["traffic"] is None


def test_serve_sweep_summary(monkeypatch):
    from paper_2005_01442_gb300 import serve
    results = {("plain", 200.0): (190.0, 12.0), ("batched", 200.0): (195.0, 10.0),
               ("plain", 800.0): (600.0, 80.0), ("batched", 800.0): (780.0, 30.0),
               ("launching", 200.0): (200.0, 8.0), ("launching", 800.0): (790.0, 40.0)}

    class Srv:
        extra_bytes_per_pixel = 0

        def __init__(self, kind):
            self.name = kind

        def close(self):
            pass

    monkeypatch.setattr(serve, "BatchedServer", lambda R, max_slots, mode=0:
                        Srv("launching" if mode == 1 else "batched"))
    monkeypatch.setattr(serve, "PlainServer", lambda R: Srv("plain"))
    monkeypatch.setattr(serve, "poisson_requests", lambda *a, **k: [a[1]])

    def run(srv, reqs, budget, warmup):
        ips, p99 = results[(srv.name, reqs[0])]
        return {"server": srv.name, "images_per_s": ips, "p99_ms": p99, "p50_ms": p99 / 2,
                "latencies_s": [], "records": []}
    monkeypatch.setattr(serve, "run_open_loop", run)
    fake_torch = types.SimpleNamespace(cuda=types.SimpleNamespace(synchronize=lambda: None),
                                       empty=None, float32=None)
    out = bench.serve_bench(FakeR(), fake_torch, {1: (8, 8, 8)}, [0],
                            [(200.0, 1.0, 0.1), (800.0, 1.0, 0.1)], 8, seed=5, p99_cap_ms=33.0)
    assert out["best_at_p99_cap"]["plain"]["images_per_s"] == 190.0  # 800/s broke the cap
    assert out["best_at_p99_cap"]["batched"]["images_per_s"] == 780.0
    assert out["batched_over_plain_at_p99_cap"] == pytest.approx(780.0 / 190.0)
    assert out["best_at_p99_cap"]["launching"]["images_per_s"] == 200.0  # 800/s broke the cap
    assert out["launching_over_plain_at_p99_cap"] == pytest.approx(200.0 / 190.0)
    assert len(out["runs"]) == 6
