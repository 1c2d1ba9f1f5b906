"""Request serving for Poisson solves: continuous batching over the C ABI.

Requests (grid size, order, coarse operator, tolerance, right-hand side) arrive
over time. Each of `slots` workers owns a CUDA stream and runs one request at a
time through `mg_solve` (the library's kernels; ctypes releases the GIL during the
call, so the workers' solves overlap on the GPU). A request is admitted when a
worker is free and its device memory fits the HBM budget: hierarchies (one
`mg_handle` per problem shape) are cached on the device and reused by later
requests of the same shape; idle cached hierarchies are evicted, least recently
used first, when a new shape needs room. Latency is measured from arrival to the
moment the solution is back in host memory.

This module is plumbing around the CUDA library: it performs no arithmetic of the
method itself.
"""
from __future__ import annotations

import collections
import dataclasses
import queue
import threading
import time

import numpy as np
import torch

import paper_2008_03885_gb300 as mg
import synth


@dataclasses.dataclass
class Request:
    rid: int
    n: int
    order: int
    coarse_op: str  # "galerkin" or "nongalerkin"
    rtol: float
    f: np.ndarray | None  # (n+1, n+1) float64 right-hand side in host memory, or None:
    #                       N(0,1) from `seed`, generated on the device (synth.rhs_normal_torch)
    arrival: float = 0.0  # seconds after the stream starts
    seed: int = 0


@dataclasses.dataclass
class Result:
    rid: int
    u: np.ndarray | None  # None when the server runs with keep_u=False
    cycles: int
    rel_res: float
    arrival: float
    start: float
    done: float

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class Hierarchy:
    """A cached problem shape: the library handle plus device arrays for u and f whose
    addresses stay fixed, so the handle's captured CUDA graph is reused."""

    def __init__(self, key, opts):
        n, order, op = key
        self.key = key
        self.handle = mg.mg_setup(n, order, opts.get("coarsening", "redblack"), op,
                                  **{k: v for k, v in opts.items() if k != "coarsening"})
        # no fill kernel here: the worker's stream zeroes u and overwrites f before use
        # (a fill on this thread's current stream would not be ordered with it)
        self.u = torch.empty((n + 1, n + 1), dtype=torch.float64, device="cuda")
        self.f = torch.empty_like(self.u)

    def close(self):
        self.handle.close()


class HierarchyCache:
    """Device hierarchies keyed by problem shape, with an HBM byte budget."""

    def __init__(self, budget_bytes: float, opts: dict):
        self.budget = float(budget_bytes)
        self.opts = opts
        self.idle = collections.OrderedDict()  # key -> list of idle hierarchies (LRU order)
        self.in_use = 0.0  # bytes of all hierarchies, idle and busy
        self.peak = 0.0
        self.cv = threading.Condition()
        self.created = 0
        self.evicted = 0

    def key_bytes(self, key) -> int:
        n, order, op = key
        ws = mg.mg_workspace_bytes(n, order, self.opts.get("coarsening", "redblack"), op,
                                   **{k: v for k, v in self.opts.items() if k != "coarsening"})
        return ws + 2 * (n + 1) ** 2 * 8

    def acquire(self, key) -> Hierarchy:
        """An idle hierarchy of `key`, or a new one once it fits the budget (waits)."""
        with self.cv:
            while True:
                lst = self.idle.get(key)
                if lst:
                    hi = lst.pop()
                    if not lst:
                        del self.idle[key]
                    return hi
                need = self.key_bytes(key)
                if need > self.budget:
                    raise mg.MGError(mg.MG_ERR_BUDGET, f"request needs {need / 1e9:.2f} GB")
                if self.in_use + need <= self.budget or self._evict(need):
                    self.in_use += need
                    self.peak = max(self.peak, self.in_use)
                    break
                self.cv.wait(timeout=0.05)
        try:
            hi = Hierarchy(key, self.opts)
        except Exception:
            with self.cv:
                self.in_use -= need
                self.cv.notify_all()
            raise
        hi.nbytes = need
        self.created += 1
        return hi

    def _evict(self, need: float) -> bool:
        """Free idle hierarchies, least recently used first, until `need` fits."""
        for k in list(self.idle.keys()):
            lst = self.idle[k]
            while lst and self.in_use + need > self.budget:
                hi = lst.pop(0)
                self.in_use -= hi.nbytes
                hi.close()
                self.evicted += 1
            if not lst:
                del self.idle[k]
            if self.in_use + need <= self.budget:
                break
        return self.in_use + need <= self.budget

    def release(self, hi: Hierarchy):
        with self.cv:
            self.idle.setdefault(hi.key, []).append(hi)
            self.idle.move_to_end(hi.key)
            self.cv.notify_all()

    def close(self):
        with self.cv:
            for lst in self.idle.values():
                for hi in lst:
                    hi.close()
            self.idle.clear()


class Server:
    """Continuous-batching solver service (see the module docstring)."""

    def __init__(self, slots: int = 8, budget_bytes: float = 120e9, max_cycles: int = 60, **opts):
        self.slots = slots
        self.max_cycles = max_cycles
        self.cache = HierarchyCache(budget_bytes, opts)
        self.queue_depth_max = 0

    def warm(self, keys, per_key: int = 1):
        """Create hierarchies ahead of time (creation synchronises the device)."""
        his = [self.cache.acquire(key) for key in keys for _ in range(per_key)]
        for hi in his:
            self.cache.release(hi)
        torch.cuda.synchronize()

    def run(self, requests, realtime: bool = True, keep_u: bool = True):
        """Serve `requests` (sorted by arrival). Returns (results by rid, stats).
        keep_u=False: each solution is still copied back to host memory (the latency
        includes it) but into a buffer the worker reuses, and not kept."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        q: queue.Queue = queue.Queue()
        results = {}
        errors = []
        lock = threading.Lock()
        t0 = time.perf_counter()

        def worker():
            stream = torch.cuda.Stream()
            host_bufs = {}  # n -> pinned buffer reused for the copy-back (keep_u=False)
            while True:
                r = q.get()
                if r is None:
                    return
                try:
                    res = self._solve(r, stream, t0, None if keep_u else host_bufs)
                    with lock:
                        results[r.rid] = res
                except Exception as e:  # reported after the run
                    with lock:
                        errors.append((r.rid, repr(e)))

        threads = [threading.Thread(target=worker, daemon=True) for _ in range(self.slots)]
        for t in threads:
            t.start()
        for r in reqs:
            if realtime:
                wait = r.arrival - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(wait)
            q.put(r)
            self.queue_depth_max = max(self.queue_depth_max, q.qsize())
        for _ in threads:
            q.put(None)
        for t in threads:
            t.join()
        wall = time.perf_counter() - t0
        if errors:
            raise RuntimeError(f"{len(errors)} requests failed, first: {errors[0]}")
        lat = np.array([results[r.rid].latency for r in reqs])
        stats = {
            "requests": len(reqs),
            "wall_s": wall,
            "throughput_rps": len(reqs) / wall,
            "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3),
            "max_queue_depth": self.queue_depth_max,
            "hbm_peak_gb": self.cache.peak / 1e9,
            "hierarchies_created": self.cache.created,
            "hierarchies_evicted": self.cache.evicted,
        }
        return results, stats

    def _solve(self, r: Request, stream, t0: float, host_bufs=None) -> Result:
        hi = self.cache.acquire((r.n, r.order, r.coarse_op))
        start = time.perf_counter() - t0
        try:
            with torch.cuda.stream(stream):
                if r.f is None:
                    synth.rhs_normal_torch(r.n, r.seed, out=hi.f)
                else:
                    f_host = torch.from_numpy(r.f).pin_memory()
                    hi.f.copy_(f_host, non_blocking=True)
                hi.u.zero_()
                k, hist = mg.mg_solve(hi.handle, hi.u, hi.f, rtol=r.rtol, max_cycles=self.max_cycles,
                                      stream=stream, raise_not_converged=False)
                if host_bufs is None:
                    u_host = torch.empty(hi.u.shape, dtype=torch.float64).pin_memory()
                else:
                    u_host = host_bufs.get(r.n)
                    if u_host is None:
                        u_host = host_bufs[r.n] = torch.empty(hi.u.shape, dtype=torch.float64).pin_memory()
                u_host.copy_(hi.u, non_blocking=True)
                stream.synchronize()
        finally:
            self.cache.release(hi)
        return Result(r.rid, u_host.numpy() if host_bufs is None else None, k, hist[-1], r.arrival, start,
                      time.perf_counter() - t0)

    def close(self):
        self.cache.close()


def poisson_stream(seed: int, count: int, rate: float, k_lo: int, k_hi: int, rtol: float = 1e-8,
                   rhs=None, device_rhs: bool = False):
    """Seeded request stream: exponential inter-arrival times at `rate` per second,
    sides 2^k + 1 with k uniform in [k_lo, k_hi], order 2/4 and Galerkin/non-Galerkin
    50/50, one right-hand side per request from `rhs(n, seed)` (default N(0,1)), seeded
    by the request id. device_rhs=True: the requests carry only the seed and the server
    generates each N(0,1) right-hand side on the device (a 20 000-request stream of
    sides up to 4097 would need ~0.7 TB of host memory for its right-hand sides)."""
    rhs = rhs or synth.rhs_normal
    u = synth.uniform01(seed, 4 * count)
    t = 0.0
    out = []
    for i in range(count):
        t += -np.log(1.0 - u[4 * i]) / rate
        k = k_lo + int(u[4 * i + 1] * (k_hi - k_lo + 1))
        order = 2 if u[4 * i + 2] < 0.5 else 4
        op = "galerkin" if u[4 * i + 3] < 0.5 else "nongalerkin"
        n = 2 ** k
        rs = seed * 100003 + i
        out.append(Request(i, n, order, op, rtol, None if device_rhs else rhs(n, rs), t, rs))
    return out
