"""Continuous-batching server: scheduling on CPU (fake library), results on GPU."""
import threading
import time
import types

import numpy as np
import pytest

import fh_inputs as fi
from paper_1807_02718_gb300 import fh as F
from paper_1807_02718_gb300 import serve as S


def _fake_lib(record, solve_s=0.02):
    fake = types.SimpleNamespace()
    fake.FH_FP64, fake.FH_MIXED_FP32 = 0, 1
    fake.FHError = F.FHError
    lock = threading.Lock()
    live = {"n": 0, "max": 0}

    def footprint(Js, Ns, precision):
        return int(sum(int(np.sum(np.asarray(n[1:], dtype=np.int64) ** 2)) * 16 for n in Ns))

    def create(dev, prec):  # one context per slot
        with lock:
            live["n"] += 1
            live["max"] = max(live["max"], live["n"])
        return object()

    def destroy(ctx):
        with lock:
            live["n"] -= 1

    def discretize_batch(ctx, curves, omegas, Ns, ps=None):
        record.append(len(curves))

    fake.fh_footprint = footprint
    fake.fh_create = create
    fake.fh_destroy = destroy
    fake.fh_discretize_batch = discretize_batch
    fake.fh_solve_frequencies = lambda ctx: time.sleep(solve_s)
    fake.fh_window_spectra_p = lambda ctx, q, a, t0, dt, H: None
    fake.fh_sample_p = lambda ctx, q, x, T: np.zeros((len(x) // 2, len(T)))
    fake.fh_resample_p = lambda ctx, q, T, n_x: np.zeros((n_x, len(T)))
    fake.fh_device_memory = lambda dev: (8 << 30, 16 << 30)
    return fake, live


def _req(rng, n=64, J=5, arrival=0.0):
    om = fi.frequency_mesh(J, 4.0)
    N = np.full(J, n, dtype=np.int32)
    q = [np.linspace(0, 10, 5), np.linspace(20, 30, 3)]
    return S.Request(fi.circle(1.0), om, N, (1.0, 0.0), np.zeros(10), -10.0, 0.01,
                     fi.targets_on_circle(8, 3.0), q, arrival=arrival)


def test_scheduler_respects_memory_budget_and_batch_limit(monkeypatch):
    record = []
    fake, live = _fake_lib(record)
    monkeypatch.setattr(S, "F", fake)
    rng = np.random.default_rng(0)
    reqs = [_req(rng, arrival=0.002 * i) for i in range(24)]
    one = reqs[0].footprint(0)
    srv = S.Server(precision=0, slots=4, max_batch=3, mem_budget=int(5.5 * one))
    for r in reqs:
        srv.submit(r)
    srv.drain(timeout=60)
    srv.close()
    st = srv.stats()
    assert st["requests"] == 24 and st["errors"] == 0
    assert max(record) <= 3
    assert srv.mem_peak <= 5.5 * one
    assert live["max"] >= 2                 # slots worked concurrently
    assert live["n"] == 0                   # every slot context released on close
    assert srv.mem_used == 0
    assert st["p99_ms"] >= st["p50_ms"] > 0


def test_scheduler_rejects_oversize_request(monkeypatch):
    record = []
    fake, _ = _fake_lib(record)
    monkeypatch.setattr(S, "F", fake)
    rng = np.random.default_rng(1)
    big = _req(rng, n=512)
    srv = S.Server(precision=0, slots=1, max_batch=2, mem_budget=big.footprint(0) // 2)
    srv.submit(big)
    srv.submit(_req(rng, n=16))
    srv.drain(timeout=30)
    srv.close()
    assert big.error is not None and big.results == []
    assert srv.stats()["requests"] == 1


def test_budget_defaults_to_free_device_memory(monkeypatch):
    fake, _ = _fake_lib([])
    monkeypatch.setattr(S, "F", fake)
    srv = S.Server(precision=0, slots=1, max_batch=1)
    srv.close()
    assert srv.mem_budget == int(0.8 * (8 << 30))


@pytest.mark.gpu
def test_result_same_alone_and_in_the_mix():
    from paper_1807_02718_gb300 import build
    build.build()
    rng = np.random.default_rng(11)
    mk = lambda: S.synthetic_request(rng, wmax_lo=8.0, wmax_hi=20.0, J=12, n_cap=256,
                                     n_queries=(3, 3), n_targets=(40, 60), n_times=16)
    probe = mk()
    alone = S.Server(slots=1, max_batch=1)
    alone.submit(probe)
    alone.drain()
    alone.close()
    assert probe.error is None and len(probe.results) == 3
    ref = [u.copy() for u in probe.results]

    others = [mk() for _ in range(7)]
    probe.results, probe.done, probe.admitted = [], None, None
    mix = S.Server(slots=3, max_batch=3)
    for i, r in enumerate(others[:4] + [probe] + others[4:]):
        r.arrival = 0.001 * i
        mix.submit(r)
    mix.drain()
    mix.close()
    assert all(r.error is None for r in others + [probe])
    assert mix.peak_active >= 2
    for a, b in zip(ref, probe.results):
        assert np.array_equal(a, b)
    st = mix.stats()
    assert st["requests"] == 8 and st["p99_ms"] >= st["p50_ms"] > 0


@pytest.mark.gpu
def test_served_request_against_the_oracle():
    """One request served in a mix of three: every query's u (the first with
    fresh target fields, the later ones on the resident fields) against the
    oracle's full run of the same problem (1e-10 relative L2)."""
    import oracle as O
    from paper_1807_02718_gb300 import build
    build.build()
    rng = np.random.default_rng(17)
    reqs = [S.synthetic_request(rng, wmax_lo=8.0, wmax_hi=16.0, J=16, n_cap=256, n_queries=(3, 3),
                                n_targets=(20, 30), n_times=12) for _ in range(3)]
    srv = S.Server(slots=2, max_batch=2)
    for i, r in enumerate(reqs):
        r.arrival = 0.001 * i
        srv.submit(r)
    srv.drain()
    srv.close()
    r = reqs[1]
    assert r.error is None and len(r.results) == 3
    wl = fi.Workload("served", r.curve, r.omega, r.N, 1.0, r.p, r.a, r.t0, r.dt, r.H, r.x,
                     np.concatenate(r.queries))
    ref = O.run(wl)["u"]
    got = np.concatenate(r.results, axis=1)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-10
