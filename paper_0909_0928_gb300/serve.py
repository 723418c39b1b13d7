"""Registration serving loop with continuous batching and resident contexts.

Requests (a static/moving pair, a force law, a schedule) arrive over time.  The
server runs at most `slots` registrations at once.  A waiting request is
admitted as soon as a slot is free and its device footprint fits the HBM
budget: if an idle context of the same volume size, image type, force law and
schedule is resident, the pair is loaded into it (dir_load: the images are
copied in, the pyramid, fields and captured registration graph stay on the
device); otherwise a new context is created on a stream of its own
(dir_create), after evicting idle contexts of other shapes, least recently
used first, while the budget requires it.  The registration is enqueued on
the context's stream (dir_register_async); jobs on different streams overlap
on the GPU.  A job's completion is detected without blocking by a CUDA event
recorded behind its work, after which its field is read back and its context
returns to the idle pool for the next request of its shape.  Every step of a
registration runs in the library's kernels; this module only schedules.

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

from . import (DIR_BF16, DIR_F32, DIR_F64, DIR_I16, DirParams, dir_create, dir_destroy,
               dir_get_field, dir_load, dir_params_default, dir_register_async, dir_sync)


def footprint_bytes(dims, levels: int, elem: int = 4, field_elem: int | None = None,
                    scratch_planes: int = 0) -> int:
    """Device bytes one context holds: pyramid images (2 per level, pitched
    rows), two fields of the finest size, scratch_planes more finest-size
    float volumes (the u + D scratch of Eqs. 3-6), the staging buffer of the
    host field read-back (3 N floats), plus a margin for reduction rows and
    padding."""
    nx, ny, nz = dims
    fe = elem if field_elem is None else field_elem
    total = 0
    n0 = 0
    for lv in range(levels):
        px = (nx + 31) // 32 * 32
        n = px * ny * nz
        if lv == 0:
            n0 = n
        total += 2 * n * elem
        nx, ny, nz = (nx + 1) // 2, (ny + 1) // 2, (nz + 1) // 2
    total += 6 * n0 * fe + scratch_planes * n0 * 4
    stage = 3 * dims[0] * dims[1] * dims[2] * 4
    return int((total + stage) * 1.05) + (4 << 20)


def _params_key(p: DirParams) -> tuple:
    return (p.levels, tuple(p.iters[: p.levels]), p.sigma, p.alpha, p.stop_mode, p.eps,
            p.stop_window, p.field_dtype, p.use_graph, p.precision, p.fuse, p.plain_kernels,
            p.correlation, p.pdl)


def request_footprint(req) -> int:
    p = req.params
    elem = 8 if p.precision == DIR_F64 else 4
    fe = 2 if p.field_dtype == DIR_BF16 else elem
    # Eqs. 3-6 under the default schedule (and fuse = 4): u and D = W - S of
    # the finest level (Eq. 6: both warped differences); counted whenever the
    # schedule may take it
    planes = 0
    if (req.variant >= 2 and p.precision != DIR_F64 and p.field_dtype != DIR_BF16
            and p.fuse in (2, 4) and not p.plain_kernels):
        planes = 5 if req.variant == 5 else 4
    return footprint_bytes(req.dims, p.levels, elem, fe, planes)


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
    """Continuous-batching scheduler: at most `slots` registrations at once,
    contexts resident between requests of the same shape."""

    def __init__(self, slots: int = 8, hbm_budget_bytes: int | None = None, keep_fields=True,
                 reuse: bool = True):
        import torch
        self.torch = torch
        self.slots = slots
        free, _total = torch.cuda.mem_get_info()
        self.budget = hbm_budget_bytes if hbm_budget_bytes is not None else int(free * 0.8)
        self.in_use = 0           # bytes of every resident context, busy or idle
        self.waiting: collections.deque[Request] = collections.deque()
        self.running: list[tuple] = []   # (request, entry, event)
        # idle contexts by shape key, least recently used first: entry =
        # [ctx, stream, bytes, key]
        self.idle: collections.OrderedDict[int, list] = collections.OrderedDict()
        self.finished: list[Request] = []
        self.keep_fields = keep_fields
        self.reuse = reuse
        self.created = 0
        self.reused = 0
        self.evicted = 0
        self._next_id = 0
        self.t0 = time.perf_counter()

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def submit(self, req: Request):
        self.waiting.append(req)

    @staticmethod
    def _key(req) -> tuple:
        return (req.dims, req.S.dtype == np.int16, req.variant, _params_key(req.params))

    def _take_idle(self, key):
        for eid, entry in self.idle.items():
            if entry[3] == key:
                del self.idle[eid]
                return entry
        return None

    def _evict_for(self, need: int) -> bool:
        """Free idle contexts, least recently used first, until `need` more
        bytes fit; False if they cannot."""
        while self.in_use + need > self.budget and self.idle:
            _eid, (ctx, _stream, nbytes, _key) = self.idle.popitem(last=False)
            dir_destroy(ctx)
            self.in_use -= nbytes
            self.evicted += 1
        return self.in_use + need <= self.budget

    def _admit(self):
        while self.waiting and len(self.running) < self.slots:
            req = self.waiting[0]
            dtype = DIR_I16 if req.S.dtype == np.int16 else DIR_F32
            key = self._key(req)
            entry = self._take_idle(key) if self.reuse else None
            if entry is not None:
                dir_load(entry[0], req.S, req.M, dtype, False)
                self.reused += 1
            else:
                need = request_footprint(req)
                if need > self.budget:
                    raise ValueError(f"request {req.rid} needs {need} bytes, more than the budget")
                if not self._evict_for(need):
                    return  # wait for memory, keep arrival order
                stream = self.torch.cuda.Stream()
                ctx = dir_create(req.S, req.M, req.dims, req.spacing, dtype, False, req.variant,
                                 req.params, stream)
                entry = [ctx, stream, need, key]
                self.in_use += need
                self.created += 1
            self.waiting.popleft()
            req.admitted = self.now()
            dir_register_async(entry[0])
            ev = self.torch.cuda.Event()
            ev.record(entry[1])
            self.running.append((req, entry, ev))

    def _reap(self):
        still = []
        for req, entry, ev in self.running:
            if not ev.query():
                still.append((req, entry, ev))
                continue
            ctx = entry[0]
            st = dir_sync(ctx)
            req.iters_run = list(st.iters_run[: req.params.levels])
            if self.keep_fields:
                nx, ny, nz = req.dims
                out = np.empty((3, nz, ny, nx), dtype=np.float32)
                dir_get_field(ctx, out)
                req.field = out
            req.done = self.now()
            if self.reuse:
                self.idle[self._next_id] = entry
                self._next_id += 1
            else:
                dir_destroy(ctx)
                self.in_use -= entry[2]
            self.finished.append(req)
        self.running = still

    def step(self):
        self._reap()
        self._admit()

    def idle_now(self) -> bool:
        return not self.waiting and not self.running

    def close(self):
        """Frees every idle context (the running ones finish first)."""
        while self.running:
            self._reap()
            time.sleep(0.0002)
        while self.idle:
            _eid, (ctx, _s, nbytes, _k) = self.idle.popitem(last=False)
            dir_destroy(ctx)
            self.in_use -= nbytes

    def run(self, requests: list[Request], realtime: bool = True):
        """Feed requests at their arrival times and serve until all finished."""
        pending = sorted(requests, key=lambda r: r.arrival)
        self.finished = []
        self.t0 = time.perf_counter()
        i = 0
        while i < len(pending) or not self.idle_now():
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
                  a_max_mm: float = 15.0, iters=(200, 100, 50), use_graph: int = 1) -> list[Request]:
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
        # contexts stay resident between requests of the same shape, so the
        # registration graph captured by the first one is replayed by the next
        params = dir_params_default(levels=3, iters=list(iters), use_graph=use_graph)
        out.append(Request(rid=k, S=S, M=M, spacing=spacing, variant=variant, params=params,
                           arrival=t))
    return out


def warm_shapes(srv: Server, seed: int, sizes=DEFAULT_SIZES, iters=(200, 100, 50)):
    """Serves one request of every (size, force law) shape so that the server
    holds a resident context, with its captured graph, for each."""
    pool = phantom_pool(sizes, seed, 15.0)
    reqs = []
    for k, (S, M, spacing) in enumerate(pool):
        for v in range(6):
            params = dir_params_default(levels=3, iters=list(iters), use_graph=1)
            reqs.append(Request(rid=-1 - len(reqs), S=S, M=M, spacing=spacing, variant=v,
                                params=params))
    srv.run(reqs, realtime=False)


def sweep(rates, jobs: int, slots: int, seed: int) -> list[dict]:
    """The same Poisson request streams served three ways: one job at a time
    with a fresh context each (the plain per-pair form), continuous batching
    with fresh contexts, and continuous batching with resident contexts."""
    forms = (("plain_queue", 1, False), ("batching_fresh_contexts", slots, False),
             ("batching_resident_contexts", slots, True))
    servers = {}
    for name, n, reuse in forms:
        servers[name] = Server(slots=n, keep_fields=False, reuse=reuse)
        if reuse:
            warm_shapes(servers[name], seed)
    lines = []
    for rate in rates:
        line = {"mode": "serve", "rate_jobs_per_s": rate, "jobs": jobs}
        for name, n, reuse in forms:
            srv = servers[name]
            reqs = make_requests(jobs, rate, seed)
            c0, r0 = srv.created, srv.reused
            done = srv.run(reqs, realtime=True)
            line[name] = {"slots": n, **latency_stats(done), "contexts_created": srv.created - c0,
                          "contexts_reused": srv.reused - r0}
        lines.append(line)
    for srv in servers.values():
        srv.close()
    return lines


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rates", type=float, nargs="+", default=[1, 2, 5, 10, 20])
    ap.add_argument("--jobs", type=int, default=30)
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--seed", type=int, default=5)
    args = ap.parse_args()
    import torch
    torch.cuda.init()
    for line in sweep(args.rates, args.jobs, args.slots, args.seed):
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
