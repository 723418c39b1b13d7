"""Registration serving loop with continuous batching.

Requests (a static/moving pair, a force law, a schedule) arrive over time.  The
server keeps a fixed number of slots, one CUDA stream each.  A waiting request
is admitted as soon as a slot is free and its device footprint fits the HBM
budget left by the jobs already resident; it then gets its own context
(dir_create: images uploaded once, pyramid and fields resident on the device)
and its registration is enqueued on the slot's stream (dir_register_async).
Jobs on different slots overlap on the GPU; a job's completion is detected
without blocking by a CUDA event recorded behind its work, after which its
field is read back, its context freed and the slot handed to the next waiting
request.  Every step of a registration runs in the library's kernels; this
module only schedules.

    python -m paper_0909_0928_gb300.serve --rates 1 2 5 10 20 --jobs 40

prints one JSON line per arrival rate with p50/p99 latency and volumes/s, for
the same request stream served one job at a time and with continuous batching.
"""
from __future__ import annotations

import argparse
import collections
import json
import math
import time
from dataclasses import dataclass
from dataclasses import field as dc_field

import numpy as np

from . import (DIR_F32, DIR_I16, DirParams, dir_create, dir_destroy, dir_get_field, dir_params_default,
               dir_register_async, dir_sync)


def footprint_bytes(dims, levels: int, elem: int = 4) -> int:
    """Device bytes one context holds: pyramid images (2 per level), two fields
    of the finest size, plus a margin for staging and pitch padding."""
    nx, ny, nz = dims
    total = 0
    n0 = 0
    for lv in range(levels):
        px = (nx + 31) // 32 * 32
        n = px * ny * nz
        if lv == 0:
            n0 = n
        total += 2 * n
        nx, ny, nz = (nx + 1) // 2, (ny + 1) // 2, (nz + 1) // 2
    total += 6 * n0
    return int(total * elem * 1.05) + (4 << 20)


@dataclass
class Request:
    rid: int
    S: np.ndarray            # (nz, ny, nx) float32 or int16 HU, host (pinned or not)
    M: np.ndarray
    spacing: tuple
    variant: int
    params: DirParams
    arrival: float = 0.0     # seconds on the server clock
    # filled by the server
    admitted: float = 0.0
    done: float = 0.0
    field: np.ndarray | None = None
    iters_run: list = dc_field(default_factory=list)

    @property
    def dims(self):
        nz, ny, nx = self.S.shape
        return (nx, ny, nz)

    @property
    def voxels(self):
        return int(self.S.size)


class Server:
    """Continuous-batching scheduler over `slots` CUDA streams."""

    def __init__(self, slots: int = 8, hbm_budget_bytes: int | None = None, keep_fields=True):
        import torch
        self.torch = torch
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        free, _total = torch.cuda.mem_get_info()
        self.budget = hbm_budget_bytes if hbm_budget_bytes is not None else int(free * 0.8)
        self.in_use = 0
        self.waiting: collections.deque[Request] = collections.deque()
        self.running: dict[int, tuple] = {}  # slot -> (request, ctx, event, bytes)
        self.finished: list[Request] = []
        self.keep_fields = keep_fields
        self.t0 = time.perf_counter()

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def submit(self, req: Request):
        self.waiting.append(req)

    def _admit(self):
        while self.waiting:
            free_slots = [s for s in range(len(self.streams)) if s not in self.running]
            if not free_slots:
                return
            req = self.waiting[0]
            need = footprint_bytes(req.dims, req.params.levels)
            if need > self.budget:
                raise ValueError(f"request {req.rid} needs {need} bytes, more than the budget")
            if self.in_use + need > self.budget:
                return  # wait for memory, keep arrival order
            self.waiting.popleft()
            slot = free_slots[0]
            stream = self.streams[slot]
            req.admitted = self.now()
            dtype = DIR_I16 if req.S.dtype == np.int16 else DIR_F32
            ctx = dir_create(req.S, req.M, req.dims, req.spacing, dtype, False, req.variant,
                             req.params, stream)
            dir_register_async(ctx)
            ev = self.torch.cuda.Event()
            ev.record(stream)
            self.running[slot] = (req, ctx, ev, need)
            self.in_use += need

    def _reap(self):
        for slot in list(self.running):
            req, ctx, ev, need = self.running[slot]
            if not ev.query():
                continue
            st = dir_sync(ctx)
            req.iters_run = list(st.iters_run[: req.params.levels])
            if self.keep_fields:
                nx, ny, nz = req.dims
                out = np.empty((3, nz, ny, nx), dtype=np.float32)
                dir_get_field(ctx, out)
                req.field = out
            req.done = self.now()
            dir_destroy(ctx)
            del self.running[slot]
            self.in_use -= need
            self.finished.append(req)

    def step(self):
        self._reap()
        self._admit()

    def idle(self) -> bool:
        return not self.waiting and not self.running

    def run(self, requests: list[Request], realtime: bool = True):
        """Feed requests at their arrival times and serve until all finished."""
        pending = sorted(requests, key=lambda r: r.arrival)
        self.t0 = time.perf_counter()
        i = 0
        while i < len(pending) or not self.idle():
            t = self.now()
            while i < len(pending) and (not realtime or pending[i].arrival <= t):
                if not realtime:
                    pending[i].arrival = t
                self.submit(pending[i])
                i += 1
            self.step()
            if self.running or self.waiting:
                time.sleep(0.0002)
            elif i < len(pending):
                time.sleep(max(0.0, min(0.002, pending[i].arrival - self.now())))
        return self.finished


def latency_stats(done: list[Request]) -> dict:
    lat = np.array([r.done - r.arrival for r in done])
    span = max(r.done for r in done) - min(r.arrival for r in done)
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "volumes_per_s": len(done) / span,
            "voxels_per_s": sum(r.voxels for r in done) / span, "jobs": len(done)}


_POOL: dict = {}


def phantom_pool(sizes, seed: int, a_max_mm: float):
    """One seeded lung phantom per size (cached), stored as int16 HU: requests
    reuse them."""
    from phantom import PhantomSpec, make_lung_phantom
    out = []
    for k, dims in enumerate(sizes):
        key = (tuple(dims), seed, a_max_mm)
        if key not in _POOL:
            spec = PhantomSpec(dims=tuple(dims), spacing=(0.9, 0.9, 2.5), seed=seed * 100 + k,
                               a_max_mm=a_max_mm, compression=0.15, compression_region="lower",
                               n_landmarks=10)
            ph = make_lung_phantom(spec)
            _POOL[key] = (np.round(ph["S"]).astype(np.int16), np.round(ph["M"]).astype(np.int16),
                          spec.spacing)
        out.append(_POOL[key])
    return out


DEFAULT_SIZES = [(128, 128, 64), (192, 192, 96), (256, 256, 128), (384, 384, 128),
                 (512, 512, 160)]


def make_requests(n: int, rate: float, seed: int, sizes=DEFAULT_SIZES,
                  a_max_mm: float = 15.0, iters=(200, 100, 50), use_graph: int = 0) -> list[Request]:
    """Poisson arrivals at `rate` jobs/s; each request takes one of the pooled
    phantoms (sizes spanning 128x128x64 .. 512x512x160, up to a_max_mm of RBF
    motion) and a force law uniform over the six, 3-level pyramid."""
    from phantom import SplitMix64Stream
    pool = phantom_pool(sizes, seed, a_max_mm)
    rng = SplitMix64Stream(seed, sid=11)
    t = 0.0
    out = []
    for k in range(n):
        t += -math.log(1.0 - float(rng.uniform(1)[0])) / rate
        S, M, spacing = pool[int(float(rng.uniform(1)[0]) * len(pool)) % len(pool)]
        variant = int(float(rng.uniform(1)[0]) * 6) % 6
        # one registration per context: launching directly costs less host time
        # than capturing a graph that would be replayed only once
        params = dir_params_default(levels=3, iters=list(iters), use_graph=use_graph)
        out.append(Request(rid=k, S=S, M=M, spacing=spacing, variant=variant, params=params,
                           arrival=t))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rates", type=float, nargs="+", default=[1, 2, 5, 10, 20, 40])
    ap.add_argument("--jobs", type=int, default=30)
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--graph", type=int, default=0, help="capture each job's registration")
    args = ap.parse_args()
    import torch
    torch.cuda.init()
    warm = make_requests(4, 100.0, args.seed + 1, use_graph=args.graph)  # first contexts
    Server(slots=2, keep_fields=False).run(warm, realtime=False)
    for rate in args.rates:
        line = {"mode": "serve", "rate_jobs_per_s": rate, "jobs": args.jobs}
        # the same Poisson stream, served one job at a time (a plain queue of
        # per-pair registrations) and with continuous batching over the slots
        for name, slots in (("plain_queue", 1), ("continuous_batching", args.slots)):
            reqs = make_requests(args.jobs, rate, args.seed, use_graph=args.graph)
            done = Server(slots=slots, keep_fields=False).run(reqs, realtime=True)
            line[name] = {"slots": slots, **latency_stats(done)}
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
