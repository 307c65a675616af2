"""Continuous-batching server for fast-hybrid scattering requests.

A request is one scattering problem (obstacle, frequency mesh, incidence
direction, incident signal), one set of targets x and a list of sample
queries (times T).  The server keeps a FIFO of arrived requests and a fixed
number of slots.  Each slot is a worker thread that owns one libfh context on
its own CUDA stream: it takes as many waiting requests as fit (batch size and
device memory: the footprint of the batch, counted with fh_footprint, within
the budget, which is a fraction of the device's free memory at start-up
(fh_device_memory) unless given), discretises and solves them in shared
launches (fh_discretize_batch / fh_solve_frequencies), keeps their densities
and window spectra resident, and answers every query of the batch: the first
query of a request evaluates its target fields (fh_sample_p), the later ones
reuse them (fh_resample_p: the time side only, any T, no re-solve).  Then it
takes the next batch into the same context (its buffers are reused).
Requests that arrive while other slots are busy are admitted as soon as a
slot and memory are free; the slots' kernels run concurrently on the device.
Every result is computed by the same kernels with the same per-problem
arithmetic whatever the batch, so it is the same alone and in the mix.

    python -m paper_1807_02718_gb300.serve --rate 50 --requests 64 --slots 4
"""
from __future__ import annotations

import argparse
import json
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import fh as F


@dataclass
class Request:
    curve: object
    omega: np.ndarray
    N: np.ndarray
    p: tuple
    a: np.ndarray
    t0: float
    dt: float
    x: np.ndarray                      # targets, interleaved
    queries: list                      # [T], sample times per query
    H: float = 10.0
    arrival: float = 0.0               # seconds after server start
    rid: int = -1
    results: list = field(default_factory=list)
    admitted: float = None
    done: float = None
    error: str = None

    @property
    def solves(self) -> int:
        return len(self.omega) - 1

    @property
    def samples(self) -> int:
        return len(self.x) // 2 * sum(len(T) for T in self.queries)

    def footprint(self, precision: int) -> int:
        base = F.fh_footprint([len(self.omega)], [self.N], precision)
        n_items = int(np.sum(np.ceil(np.asarray(self.N[1:]) / 64.0)))
        n_x = len(self.x) // 2
        n_T = max((len(T) for T in self.queries), default=0)
        work = (16 * (len(self.omega) + 8 * n_items) * n_x + 16 * len(self.omega) * n_T
                + 8 * n_x * n_T)
        return base + work


class Server:
    def __init__(self, device: int = 0, precision: int = F.FH_MIXED_BF16, slots: int = 4,
                 max_batch: int = 8, mem_budget: int | None = None, mem_fraction: float = 0.8):
        self.device = device
        self.precision = precision
        self.max_batch = max_batch
        if mem_budget is None:   # what the device has free now, less a margin
            free, _ = F.fh_device_memory(device)
            mem_budget = int(mem_fraction * free)
        self.mem_budget = mem_budget
        self.mem_used = 0
        self.mem_peak = 0
        self.batch_sizes: list[int] = []
        self._next_id = 0
        self.pending: list[Request] = []
        self.finished: list[Request] = []
        self.lock = threading.Condition()
        self.closed = False
        self.t_start = time.perf_counter()
        self.active = 0
        self.peak_active = 0
        self.workers = [threading.Thread(target=self._worker, args=(i,), daemon=True)
                        for i in range(slots)]
        for w in self.workers:
            w.start()

    def now(self) -> float:
        return time.perf_counter() - self.t_start

    def submit(self, req: Request):
        with self.lock:
            if req.rid < 0:
                self._next_id += 1
                req.rid = self._next_id
            if req.footprint(self.precision) > self.mem_budget:
                req.error = "request larger than the memory budget"
                req.done = self.now()
                self.finished.append(req)
            else:
                self.pending.append(req)
            self.lock.notify_all()

    def close(self):
        with self.lock:
            self.closed = True
            self.lock.notify_all()
        for w in self.workers:
            w.join()

    def drain(self, timeout: float = 600.0):
        t_end = time.perf_counter() + timeout
        with self.lock:
            while (self.pending or self.active) and time.perf_counter() < t_end:
                self.lock.wait(timeout=0.05)

    # ------------------------------------------------------------- workers

    def _take_batch(self):
        """FIFO requests that have arrived and fit the memory budget (blocking)."""
        with self.lock:
            while True:
                if self.closed and not self.pending:
                    return None, 0
                now = self.now()
                batch, need = [], 0
                for r in self.pending:
                    if r.arrival > now or len(batch) >= self.max_batch:
                        break
                    fp = r.footprint(self.precision)
                    if self.mem_used + need + fp > self.mem_budget:
                        break
                    batch.append(r)
                    need += fp
                if batch:
                    for r in batch:
                        self.pending.remove(r)
                        r.admitted = now
                    self.mem_used += need
                    self.mem_peak = max(self.mem_peak, self.mem_used)
                    self.batch_sizes.append(len(batch))
                    self.active += 1
                    self.peak_active = max(self.peak_active, self.active)
                    return batch, need
                wait = 0.05
                if self.pending and self.pending[0].arrival > now:
                    wait = min(wait, self.pending[0].arrival - now)
                self.lock.wait(timeout=max(wait, 1e-4))

    def _worker(self, slot: int):
        # one context per slot: its device buffers grow to the largest batch
        # seen and are reused by later batches (no allocation per request)
        ctx = None
        while True:
            batch, need = self._take_batch()
            if batch is None:
                if ctx is not None:
                    F.fh_destroy(ctx)
                return
            try:
                if ctx is None:
                    ctx = F.fh_create(self.device, self.precision)
                F.fh_discretize_batch(ctx, [r.curve for r in batch], [r.omega for r in batch],
                                      [r.N for r in batch], ps=[r.p for r in batch])
                F.fh_solve_frequencies(ctx)
                for q, r in enumerate(batch):
                    F.fh_window_spectra_p(ctx, q, r.a, r.t0, r.dt, r.H)
                    for i, T in enumerate(r.queries):
                        if i == 0:   # target fields of the request, then resident
                            r.results.append(F.fh_sample_p(ctx, q, r.x, T))
                        else:
                            r.results.append(F.fh_resample_p(ctx, q, T, len(r.x) // 2))
                    r.done = self.now()
            except F.FHError as e:
                for r in batch:
                    if r.done is None:
                        r.error = str(e)
                        r.done = self.now()
            finally:
                with self.lock:
                    self.mem_used -= need
                    self.active -= 1
                    self.finished.extend(batch)
                    self.lock.notify_all()

    # --------------------------------------------------------------- stats

    def stats(self) -> dict:
        ok = [r for r in self.finished if r.error is None]
        lat = np.array([r.done - r.arrival for r in ok]) if ok else np.zeros(1)
        span = max((r.done for r in ok), default=0.0) - min((r.arrival for r in ok), default=0.0)
        solves = sum(r.solves for r in ok)
        samples = sum(r.samples for r in ok)
        return {"requests": len(ok), "errors": len(self.finished) - len(ok),
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "solves_per_s": solves / span if span > 0 else 0.0,
                "time_samples_per_s": samples / span if span > 0 else 0.0,
                "peak_concurrent_batches": self.peak_active}


def synthetic_request(rng: np.random.Generator, wmax_lo=10.0, wmax_hi=120.0, J=128, n_cap=2048,
                      n_queries=(1, 100), n_targets=(256, 4096), n_times=16, t_max=1.0e4) -> Request:
    """A serving request of the paper's shapes: a random star obstacle
    r = 1 + sum_{k<=5} a_k cos(k t + phi_k), J frequencies on [0, w_max],
    w_max ~ U(wmax_lo, wmax_hi), N by 8 points per wavelength (capped at
    n_cap), a random pulse-train or linear-chirp signal, n_targets ~ U targets
    on a circle of radius 3, and n_queries ~ U queries of n_times random times
    in [0, t_max]."""
    import fh_inputs as fi
    cur = fi.random_star(rng)
    W = float(rng.uniform(wmax_lo, wmax_hi))
    om = fi.frequency_mesh(J, W)
    N = fi.boundary_sizes(cur, om, n_max=n_cap)
    ang = float(rng.uniform(0, 2 * np.pi))
    if rng.random() < 0.5:
        sig = fi.pulse_train(int(rng.integers(1, 1 << 30)), n=int(rng.integers(2, 8)), span=60.0,
                             fmin=0.2 * W, fmax=0.6 * W)
    else:
        sig = fi.Chirp(0.0, float(rng.uniform(30, 80)), 5.0)
    t0, dt = -10.0, 0.01
    a = fi.sample_signal(sig, t0, dt, int(np.ceil((sig.t_end - t0) / dt)) + 1)
    nx = int(rng.integers(n_targets[0], n_targets[1] + 1))
    queries = [np.sort(rng.uniform(0.0, t_max, n_times))
               for _ in range(int(rng.integers(n_queries[0], n_queries[1] + 1)))]
    return Request(cur, om, N, (np.cos(ang), np.sin(ang)), a, t0, dt, fi.targets_on_circle(nx, 3.0), queries)


def run_stream(rate: float, n_requests: int, seed: int = 5, slots: int = 4, max_batch: int = 8,
               precision: int = F.FH_MIXED_BF16, **request_kw) -> dict:
    """Serve n_requests synthetic requests arriving as a Poisson process of
    the given rate; returns the server's statistics."""
    rng = np.random.default_rng(seed)
    reqs = [synthetic_request(rng, **request_kw) for _ in range(n_requests)]
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_requests))
    srv = Server(precision=precision, slots=slots, max_batch=max_batch)
    for r, t in zip(reqs, arrivals):
        r.arrival = float(t) + 0.2
        srv.submit(r)
    srv.drain()
    srv.close()
    out = {"rate": rate, "slots": slots, "max_batch": max_batch}
    out.update(srv.stats())
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rate", type=float, default=50.0, help="Poisson arrival rate (requests/s)")
    ap.add_argument("--requests", type=int, default=48)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--max-batch", type=int, default=8)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--precision", default="bf16", choices=["fp64", "fp32", "tf32", "bf16"])
    args = ap.parse_args()
    from . import build
    build.build()
    prec = {"fp64": F.FH_FP64, "fp32": F.FH_MIXED_FP32, "tf32": F.FH_MIXED_TF32,
            "bf16": F.FH_MIXED_BF16}[args.precision]
    out = run_stream(args.rate, args.requests, args.seed, args.slots, args.max_batch, prec)
    out["precision"] = args.precision
    print(json.dumps(out))


if __name__ == "__main__":
    main()
