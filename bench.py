#!/usr/bin/env python3
"""Benchmark: demons registration of a 256 x 256 x 100 synthetic lung phantom.

One step = one whole registration through the C ABI (pyramid build, 3 levels
at 200/100/50 iterations coarse to fine, sigma 1 voxel, passive force by
default) plus the final warp of the moving image by the registered field.
The metric is voxel-updates/s (sum over levels of voxels x iterations, per
second of device time) with s per registration p50/p99 beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--variant passive]
  python bench.py --impl reference   # FP64 CPU oracle on the host cores
  python bench.py --form batch       # 32 uneven int16 pairs: one graph vs 32 plain runs
  python bench.py --form study       # landmark accuracy per force law, alpha sweep, stop test
  python bench.py --form precision   # int16 images / BF16 field against the FP64 kernels
  python bench.py --form serve       # Poisson request streams: plain queue vs continuous batching

Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (256, 256, 100)
SPACING = (0.9, 0.9, 2.5)
LEVELS = 3
ITERS = [200, 100, 50]            # coarsest first
METRIC = "voxel-updates/s and s per 256x256x100 registration (% HBM roofline); p50/p99"
UNIT = "voxel-updates/s"
VARIANT_NAMES = ["passive", "evolved_passive", "active", "double", "adjusted_double",
                 "inverse_consistent"]
# algorithmic bytes per voxel and launch at the finest level (fp32 volumes):
# force: read u (12) + S (4) + M (4), write v (12); smoothing: read v (12), write u (12)
FORCE_BYTES = {0: 32, 1: 36, 2: 32, 3: 32, 4: 32, 5: 32}
SMOOTH_BYTES = 24


def level_dims(dims, levels):
    out = [tuple(dims)]
    for _ in range(1, levels):
        out.append(tuple((d + 1) // 2 for d in out[-1]))
    return out


def max_over_ranks(x: float, dist, device) -> float:
    """The largest value of x over all ranks (timing rule: max over ranks)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step: float, steps: int, world: int, max_ms: float) -> float:
    """Units all ranks processed (replicas: each rank does the same work) per
    second of the slowest rank's timed region."""
    return world * units_per_rank_step * steps / (max_ms / 1e3)


def voxel_updates(dims, levels, iters):
    lv = level_dims(dims, levels)
    return sum(lv[levels - 1 - lc][0] * lv[levels - 1 - lc][1] * lv[levels - 1 - lc][2] * iters[lc]
               for lc in range(levels))


def workload_config(variant, alpha, n_gpus):
    return {"workload": f"{DIMS[0]}x{DIMS[1]}x{DIMS[2]} f32 synthetic lung phantom, "
                        f"{LEVELS}-level pyramid {'/'.join(map(str, ITERS))} coarse to fine, "
                        f"sigma 1 voxel, {VARIANT_NAMES[variant]} force",
            "dims": list(DIMS), "spacing_mm": list(SPACING), "levels": LEVELS,
            "iters_coarse_to_fine": ITERS, "variant": VARIANT_NAMES[variant], "alpha": alpha,
            "l2": "flushed between steps (256 MiB write)",
            "parallelism": f"replicas x{n_gpus}" if n_gpus > 1 else "single GPU"}


def measured_peak_gbs():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# source files each timed kernel is built from (its traffic figure in profiles/
# is valid only while their combined sha256 is unchanged)
KERNEL_SOURCES = {
    "force_kernel": ["dir_force_kernel.cuh", "dir_force_law.cuh", "dir_common.cuh"],
    "force_tma_kernel": ["dir_force_tma.cu", "dir_force_gm.cuh", "dir_force_kernel.cuh",
                         "dir_force_law.cuh", "dir_stencil.cuh", "dir_common.cuh"],
    "force_tma_gm_kernel": ["dir_force_tma.cu", "dir_force_gm.cuh", "dir_force_kernel.cuh",
                            "dir_force_law.cuh", "dir_stencil.cuh", "dir_common.cuh"],
    "smooth2_kernel": ["dir_smooth.cu", "dir_smooth2.cuh", "dir_common.cuh"],
    "fused_kernel": ["dir_fused.cu", "dir_stencil.cuh", "dir_force_law.cuh", "dir_common.cuh"],
    "fused2_kernel": ["dir_fused.cu", "dir_smooth2.cuh", "dir_force_kernel.cuh",
                      "dir_force_law.cuh", "dir_common.cuh"],
    "fused_small_kernel": ["dir_fused.cu", "dir_smooth2.cuh", "dir_force_kernel.cuh",
                           "dir_force_law.cuh", "dir_common.cuh"],
    "smooth_xy_kernel": ["dir_smooth.cu", "dir_split.cuh", "dir_smooth2.cuh", "dir_common.cuh"],
    "force_zs_kernel": ["dir_force_zs.cu", "dir_split.cuh", "dir_force_gm.cuh",
                        "dir_force_kernel.cuh", "dir_force_law.cuh", "dir_stencil.cuh",
                        "dir_common.cuh"],
    "force_zd_kernel": ["dir_force_d.cu", "dir_split_d.cuh", "dir_split.cuh",
                        "dir_force_kernel.cuh", "dir_stencil.cuh", "dir_common.cuh"],
    "force_st_kernel": ["dir_force_d.cu", "dir_split_d.cuh", "dir_force_kernel.cuh",
                        "dir_force_law.cuh", "dir_stencil.cuh", "dir_common.cuh"],
}


def _code_only(text: str) -> str:
    """Source text without comments and blank lines: a change of comments
    alone leaves a kernel, and so its recorded ncu counters, as they were."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(line.rstrip() for line in text.splitlines() if line.strip())


def sources_sha256(kernel: str) -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        path = os.path.join(ROOT, "paper_0909_0928_gb300", "csrc", f)
        h.update(_code_only(open(path, encoding="utf-8").read()).encode())
    return h.hexdigest()


def profiled_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, valid only while
    the kernel's sources are unchanged since the capture (sha256 recorded)."""
    summ = os.path.join(ROOT, "profiles", f"{kernel}_traffic.txt")
    try:
        vals = {}
        for line in open(summ):
            if ":" in line:
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
        if vals.get("source_sha256") == sources_sha256(kernel):
            return float(vals["dram_bytes_per_launch_full_size"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi samples during the timed region (median SM clock under load)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = None
        self.gpu = gpu_index

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu),
                                          f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "50"], stdout=self.out,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        loaded = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def cpu_baseline(phantom, variant, alpha, iters_sample, single_thread_sample=None):
    """The FP64 oracle as it stands, threaded over z-slices on the host cores
    (and, if asked, single-threaded on a smaller sample)."""
    import oracle
    t0 = time.perf_counter()
    r = oracle.register(phantom["S"], phantom["M"], variant=variant, levels=LEVELS,
                        iters=iters_sample, alpha=alpha, threaded=True)
    dt = time.perf_counter() - t0
    vu = voxel_updates(DIMS, LEVELS, iters_sample)
    out = {"value": vu / dt, "unit": UNIT, "cores": oracle.num_threads(True), "kind": "oracle",
           "sample": f"full-size phantom, {LEVELS} levels at {'/'.join(map(str, iters_sample))} "
                     f"iterations coarse to fine ({vu} voxel-updates, {dt:.1f} s)",
           "seconds": dt, "iters_run": r["iters_run"]}
    if single_thread_sample:
        t0 = time.perf_counter()
        oracle.register(phantom["S"], phantom["M"], variant=variant, levels=LEVELS,
                        iters=single_thread_sample, alpha=alpha, threaded=False)
        d1 = time.perf_counter() - t0
        v1 = voxel_updates(DIMS, LEVELS, single_thread_sample)
        out["single_thread"] = {"value": v1 / d1, "unit": UNIT, "cores": 1,
                                "sample": f"{'/'.join(map(str, single_thread_sample))} iterations "
                                          f"({v1} voxel-updates, {d1:.1f} s)"}
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from phantom import FULL, make_lung_phantom
    ph = make_lung_phantom(FULL)
    sample = [20, 10, 5]
    for _ in range(args.warmup):
        cpu_baseline(ph, args.variant_id, args.alpha, sample)
    times = []
    last = None
    for _ in range(args.steps):
        last = cpu_baseline(ph, args.variant_id, args.alpha, sample)
        times.append(last["seconds"])
    vu = voxel_updates(DIMS, LEVELS, sample)
    value = vu * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.variant_id, args.alpha, args.gpus),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": last["cores"],
                             "kind": "oracle", "sample": last["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


BATCH_PAIRS = 32


def _batch_pair(k):
    """Pair k of the batched form: seed 100 + k, dims drawn per axis uniformly
    on multiples of 16 (96..256 x 96..256 x 48..128), RBF motion up to 12 mm
    with 20% compression of the lower lung, int16 HU; passive for even k,
    inverse consistent for odd k."""
    import numpy as np
    from phantom import PhantomSpec, SplitMix64Stream, make_lung_phantom
    r = SplitMix64Stream(100 + k, sid=21).uniform(3)
    dims = (96 + 16 * int(r[0] * 11), 96 + 16 * int(r[1] * 11), 48 + 16 * int(r[2] * 6))
    ph = make_lung_phantom(PhantomSpec(dims=dims, spacing=SPACING, seed=100 + k, a_max_mm=12.0,
                                       compression=0.2, compression_region="lower",
                                       n_landmarks=10))
    return (np.round(ph["S"]).astype(np.int16), np.round(ph["M"]).astype(np.int16),
            0 if k % 2 == 0 else 5)


SMALL_PAIRS = 64
SMALL_DIMS = (64, 64, 32)


def _small_pair(k):
    """Pair k of the small-volume batch: the 64x64x32 phantom shape (1 x 1 x 2.5
    mm, RBF motion up to 4 mm) with seed 300 + k, int16 HU; passive for even k,
    inverse consistent for odd k."""
    import numpy as np
    from phantom import PhantomSpec, make_lung_phantom
    ph = make_lung_phantom(PhantomSpec(dims=SMALL_DIMS, spacing=(1.0, 1.0, 2.5), seed=300 + k,
                                       a_max_mm=4.0, compression=0.05, n_landmarks=10))
    return (np.round(ph["S"]).astype(np.int16), np.round(ph["M"]).astype(np.int16),
            0 if k % 2 == 0 else 5)


def batch_pairs(n=BATCH_PAIRS, small=False):
    """The 32 seeded pairs of uneven sizes, generated on the host cores by a
    pool started with spawn before any GPU work."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(min(n, os.cpu_count() or 1)) as pool:
        return pool.map(_small_pair if small else _batch_pair, range(n))


def run_batch(args):
    """Batched form against the plain per-pair form on the same 32 contexts."""
    import numpy as np
    import torch
    import paper_0909_0928_gb300 as dl
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.current_stream()
    pairs = batch_pairs()
    small = batch_pairs(SMALL_PAIRS, small=True)
    ctxs, dev, vu = [], [], 0
    for S, M, v in pairs:
        nz, ny, nx = S.shape
        St, Mt = torch.from_numpy(S).cuda(), torch.from_numpy(M).cuda()
        dev.append((St, Mt))
        p = dl.dir_params_default(levels=LEVELS, iters=ITERS)
        ctxs.append(dl.dir_create(St, Mt, (nx, ny, nz), SPACING, dl.DIR_I16, True, v, p, stream))
        vu += voxel_updates((nx, ny, nz), LEVELS, ITERS)
    n = len(ctxs)

    def sequential(reps):
        done = []   # completion time of each pair after the start of its round
        t_all = 0.0
        for _ in range(reps):
            t = 0.0
            for c in ctxs:
                t += dl.dir_register(c).ms_total
                done.append(t)
            t_all += t
        return t_all / reps, done

    sequential(1)
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    plain_ms, plain_done = sequential(args.steps)
    ref = []
    for (S, _, _), c in zip(pairs, ctxs):
        f = np.empty((3,) + S.shape, np.float32)
        dl.dir_get_field(c, f)
        ref.append(f)
    t0 = time.perf_counter()
    shapes = [dl.dir_autotune(c, reps=3, levels=LEVELS) for c in ctxs]
    tune_s = time.perf_counter() - t0
    sequential(1)
    tuned_ms, _ = sequential(args.steps)
    def fields_same():
        ok = True
        for (S, _, _), c, f0 in zip(pairs, ctxs, ref):
            f = np.empty((3,) + S.shape, np.float32)
            dl.dir_get_field(c, f)
            ok = ok and bool(np.array_equal(f, f0))
        return ok

    # branch form: each registration on one of `br` concurrent graph branches
    best = None
    per_branches = {}
    for br in (4, 8, 16, 32):
        b = dl.dir_batch_create(ctxs, branches=br, stream=stream, grouped=False)
        for _ in range(args.warmup):
            dl.dir_batch_run(b)
        ms = statistics.median([dl.dir_batch_run(b) for _ in range(args.steps)])
        per_branches[br] = ms
        if best is None or ms < per_branches[best]:
            best = br
        dl.dir_batch_destroy(b)
    same = fields_same()
    # grouped form (the default): one x/y and one z + force launch per
    # iteration over all the pairs of a pyramid level
    b = dl.dir_batch_create(ctxs, stream=stream)
    grouped = dl.dir_batch_grouped(b)
    for _ in range(args.warmup):
        dl.dir_batch_run(b)
    gms = statistics.median([dl.dir_batch_run(b) for _ in range(args.steps)])
    dl.dir_batch_destroy(b)
    same = same and fields_same()
    for c in ctxs:
        dl.dir_destroy(c)

    # many small volumes: one registration alone is bound by launch latencies
    sctx, sdev, svu = [], [], 0
    for S, M, v in small:
        nz, ny, nx = S.shape
        St, Mt = torch.from_numpy(S).cuda(), torch.from_numpy(M).cuda()
        sdev.append((St, Mt))
        p = dl.dir_params_default(levels=LEVELS, iters=ITERS)
        sctx.append(dl.dir_create(St, Mt, (nx, ny, nz), (1.0, 1.0, 2.5), dl.DIR_I16, True, v, p,
                                  stream))
        svu += voxel_updates((nx, ny, nz), LEVELS, ITERS)
    for c in sctx:
        dl.dir_register(c)
    s_plain = statistics.median([sum(dl.dir_register(c).ms_total for c in sctx)
                                 for _ in range(max(1, args.steps // 2))])
    s_ref = []
    for (S, _, _), c in zip(small, sctx):
        f = np.empty((3,) + S.shape, np.float32)
        dl.dir_get_field(c, f)
        s_ref.append(f)
    s_forms = {}
    for name, kw in (("grouped", {}), ("branches_16", {"branches": 16, "grouped": False}),
                     ("branches_32", {"branches": 32, "grouped": False})):
        b = dl.dir_batch_create(sctx, stream=stream, **kw)
        for _ in range(args.warmup):
            dl.dir_batch_run(b)
        s_forms[name] = statistics.median([dl.dir_batch_run(b) for _ in range(args.steps)])
        dl.dir_batch_destroy(b)
        for (S, _, _), c, f0 in zip(small, sctx, s_ref):
            f = np.empty((3,) + S.shape, np.float32)
            dl.dir_get_field(c, f)
            same = same and bool(np.array_equal(f, f0))
    for c in sctx:
        dl.dir_destroy(c)
    small_line = {"pairs": len(small), "dims": list(SMALL_DIMS),
                  "sizes": "seeds 300-363, 64x64x32 int16 HU, passive / inverse consistent "
                           "alternating, 3 levels 200/100/50",
                  "voxel_updates": svu,
                  "plain_sequential_ms": s_plain,
                  "forms_ms": s_forms,
                  "volumes_per_s": {k: len(small) / (v / 1e3) for k, v in
                                    dict(s_forms, plain_sequential=s_plain).items()},
                  "speedup_grouped_vs_plain": s_plain / s_forms["grouped"],
                  "speedup_grouped_vs_best_branches": min(s_forms["branches_16"],
                                                          s_forms["branches_32"]) /
                                                      s_forms["grouped"]}
    clk = clocks.stop()
    bms = per_branches[best]
    q = lambda xs, p: float(np.quantile(np.asarray(xs), p))
    line = {"mode": "batch", "pairs": n, "variants": {"passive": sum(v == 0 for *_, v in pairs),
                                                      "inverse_consistent": sum(v == 5 for *_, v in pairs)},
            "sizes": "seeds 100-131, dims uniform on multiples of 16 in 96..256 x 96..256 x "
                     "48..128, int16 HU, FP32 fields, 3 levels 200/100/50",
            "dims": [list(S.shape[::-1]) for S, _, _ in pairs],
            "voxel_updates": vu,
            "plain_sequential": {"ms": plain_ms, "volumes_per_s": n / (plain_ms / 1e3),
                                 "voxel_updates_per_s": vu / (plain_ms / 1e3),
                                 "completion_p50_ms": q(plain_done, 0.5),
                                 "completion_p99_ms": q(plain_done, 0.99)},
            "tuned_sequential": {"ms": tuned_ms, "volumes_per_s": n / (tuned_ms / 1e3)},
            "batched": {"ms": gms, "form": "grouped" if grouped else "branches (not groupable)",
                        "volumes_per_s": n / (gms / 1e3), "voxel_updates_per_s": vu / (gms / 1e3),
                        "completion_p50_ms": gms, "completion_p99_ms": gms},
            "batched_branches": {"ms": bms, "branches": best, "volumes_per_s": n / (bms / 1e3),
                                 "voxel_updates_per_s": vu / (bms / 1e3),
                                 "per_branch_count_ms": per_branches},
            "speedup_vs_plain": plain_ms / gms, "speedup_branches_vs_plain": plain_ms / bms,
            "fields_identical": same,
            "autotune_s": tune_s, "tuned_shapes_first_pair": shapes[0],
            "small_volumes": small_line, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0 if same else 1



def landmark_error_mm(u_vox, landmarks, u_true_mm, spacing):
    """Trilinear field at the landmark voxel positions (x, y, z), in mm, against
    the known field: mean and SD of the 3-D error (the form of Table 3)."""
    import numpy as np
    from scipy.ndimage import map_coordinates
    coords = np.stack([landmarks[:, 2], landmarks[:, 1], landmarks[:, 0]])  # (z, y, x)
    ue = np.stack([map_coordinates(u_vox[c], coords, order=1, mode="nearest")
                   for c in range(3)], 1) * np.asarray(spacing)
    err = np.linalg.norm(ue - u_true_mm, axis=1)
    return float(err.mean()), float(err.std())


def run_study(args):
    """Accuracy studies on the full-size phantom with its known deformation
    (Sec. 3.2 evaluation on synthetic landmarks): every force law, the alpha
    of Eq. (5) from 0.1 to 5, the relative-norm stop test of Sec. 2.4 and the
    same test on the correlation coefficient (reduced on the device every
    iteration), and the finest level iteration by iteration, each with the
    correlation of the deformed moving image with S beside the landmark error
    (Sec. 3.3)."""
    import numpy as np
    import torch
    import paper_0909_0928_gb300 as dl
    from phantom import FULL, make_lung_phantom
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.current_stream()
    ph = make_lung_phantom(FULL)
    S_d, M_d = torch.from_numpy(ph["S"]).cuda(), torch.from_numpy(ph["M"]).cuda()
    lm, ut = ph["landmarks"], ph["u_true_mm"]
    init = np.linalg.norm(ut, axis=1)
    out = {"mode": "study", "workload": workload_config(0, 0.4, 1)["workload"],
           "landmarks": int(lm.shape[0]),
           "initial_mm": {"mean": float(init.mean()), "sd": float(init.std())}}

    S_np = ph["S"].astype(np.float64)

    def correlation(W):
        """Pearson correlation of the deformed moving image with S (the image
        similarity the paper contrasts with spatial accuracy, Sec. 3.3)."""
        a = S_np - S_np.mean()
        b = W.astype(np.float64) - W.mean()
        return float((a * b).sum() / np.sqrt((a * a).sum() * (b * b).sum()))

    def run(variant, alpha=0.4, stop_mode=0, eps=1e-4, iters=ITERS, reps=3, curve=False):
        # correlation = 1: the device reduces the correlation coefficient of the
        # warped image with S every iteration, in the force pass
        p = dl.dir_params_default(levels=LEVELS, iters=list(iters), alpha=alpha,
                                  stop_mode=stop_mode, eps=eps, stop_window=10, correlation=1)
        ctx = dl.dir_create(S_d, M_d, DIMS, SPACING, dl.DIR_F32, True, variant, p, stream)
        try:
            st = dl.dir_register(ctx)
            ms = [dl.dir_register(ctx).ms_total for _ in range(reps)]
            u = np.empty((3,) + ph["S"].shape, np.float32)
            dl.dir_get_field(ctx, u)
            W = np.empty(ph["S"].shape, np.float32)
            dl.dir_warp(ctx, ph["M"], W)
            rho = dl.dir_get_correlation(ctx, sum(iters))
            hist = dl.dir_get_history(ctx, sum(iters))
        finally:
            dl.dir_destroy(ctx)
        m, sd = landmark_error_mm(u, lm, ut, SPACING)
        runs = list(st.iters_run[:LEVELS])
        fine = slice(sum(runs[:-1]), sum(runs))
        out = {"landmark_mm": {"mean": m, "sd": sd}, "ms": statistics.median(ms) if ms else None,
               "iters_run": runs, "mse_final": st.mse_final, "relnorm_final": st.relnorm_final,
               "correlation": correlation(W),
               "correlation_device_last": float(rho[-1]) if rho.size else None}
        if curve:  # the finest level, iteration by iteration (Fig. 3a)
            h = hist[fine]
            out["finest_curve"] = {
                "correlation": [round(float(r), 6) for r in rho[fine]],
                "relative_norm": [round(float(a / b), 6) if b > 0 else None for a, b in
                                  zip(h[:, 1], h[:, 2])]}
        return out

    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    out["variants"] = {VARIANT_NAMES[v]: run(v, curve=(v == 0)) for v in range(6)}
    out["alpha_sweep_adjusted_double"] = {str(a): run(4, alpha=a)
                                          for a in (0.1, 0.2, 0.4, 0.5, 1.0, 2.0, 3.0, 5.0)}
    out["stop_test_passive"] = {f"{e:g}": run(0, stop_mode=1, eps=e)
                                for e in (1e-2, 1e-3, 1e-4, 1e-5)}
    # the similarity criterion Sec. 2.4 argues against: the same windowed test
    # on the correlation coefficient, decided on the device
    out["stop_test_correlation_passive"] = {f"{e:g}": run(0, stop_mode=2, eps=e)
                                            for e in (1e-3, 1e-4, 1e-5, 1e-6)}
    # the finest level iteration by iteration (Fig. 3a): a registration stopped
    # after k finest iterations is the state of iteration k of a longer one
    out["finest_iterations_passive"] = {
        str(k): run(0, iters=[ITERS[0], ITERS[1], k], reps=0)
        for k in (0, 5, 10, 20, 30, 50, 70, 90)}
    out["clocks"] = clocks.stop()
    print(json.dumps(out), flush=True)
    return 0


def run_precision(args):
    """Storage forms of the full-size passive registration (NEXT-1): images as
    float or int16 HU, field as FP32 or BF16, arithmetic FP32, reductions FP64.
    Error against the FP64 form of the same kernels (precision = DIR_F64, which
    matches the FP64 oracle to 1e-9 voxel on this workload), landmark error,
    algorithmic bytes per voxel-update and time.  Schedules: single scale, 50
    iterations (the 64^3-style parity schedule on the full-size inputs), and the
    3-level 200/100/50 pyramid."""
    import numpy as np
    import torch
    import paper_0909_0928_gb300 as dl
    from phantom import FULL, make_lung_phantom
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.current_stream()
    ph = make_lung_phantom(FULL)
    S16 = np.round(ph["S"]).astype(np.int16)
    M16 = np.round(ph["M"]).astype(np.int16)
    imgs = {"f32": (torch.from_numpy(S16.astype(np.float32)).cuda(),
                    torch.from_numpy(M16.astype(np.float32)).cuda(), dl.DIR_F32),
            "i16": (torch.from_numpy(S16).cuda(), torch.from_numpy(M16).cuda(), dl.DIR_I16)}
    lm, ut = ph["landmarks"], ph["u_true_mm"]
    # bytes per voxel-update of the finest-level two-kernel iteration
    bpv = {("f32", "f32"): 56, ("i16", "f32"): 52, ("f32", "bf16"): 32, ("i16", "bf16"): 28}
    out = {"mode": "precision", "workload": "256x256x100 lung phantom rounded to int16 HU, passive"}
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    for sched_name, levels, iters in (("single_scale_50", 1, [50]), ("pyramid_200_100_50", 3, ITERS)):
        def run(img, field, precision=dl.DIR_F32):
            S_d, M_d, dt = imgs[img]
            p = dl.dir_params_default(levels=levels, iters=iters, precision=precision,
                                      field_dtype=dl.DIR_BF16 if field == "bf16" else dl.DIR_F32)
            ctx = dl.dir_create(S_d, M_d, DIMS, SPACING, dt, True, 0, p, stream)
            try:
                dl.dir_register(ctx)
                ms = statistics.median([dl.dir_register(ctx).ms_total for _ in range(5)])
                u = np.empty((3,) + ph["S"].shape, np.float64)
                dl.dir_get_field_f64(ctx, u)
            finally:
                dl.dir_destroy(ctx)
            return u, ms
        ref, ms64 = run("f32", "f32", dl.DIR_F64)
        res = {"reference": {"precision": "f64 kernels", "ms": ms64}}
        for img, field in (("f32", "f32"), ("i16", "f32"), ("f32", "bf16"), ("i16", "bf16")):
            u, ms = run(img, field)
            err = np.abs(u - ref).max(axis=0)
            m, sd = landmark_error_mm(u.astype(np.float32), lm, ut, SPACING)
            res[f"images_{img}_field_{field}"] = {
                "ms": ms, "bytes_per_voxel_update_finest": bpv[(img, field)],
                "max_du_vs_f64": float(err.max()), "q99_du_vs_f64": float(np.quantile(err, 0.99)),
                "median_du_vs_f64": float(np.median(err)),
                "landmark_mm": {"mean": m, "sd": sd}}
        out[sched_name] = res
    out["clocks"] = clocks.stop()
    print(json.dumps(out), flush=True)
    return 0


def run_serve(args):
    """Serving sweep (config 5): Poisson arrivals at 1 to 20 jobs/s of int16 HU
    registrations, 128x128x64 .. 512x512x160, force law uniform over the six,
    3 levels; a plain queue (one job at a time, fresh context each) against
    continuous batching with fresh and with resident contexts.  One JSON line
    per rate, clocks sampled over the whole sweep."""
    import torch
    from paper_0909_0928_gb300 import serve
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    lines = serve.sweep([1, 2, 5, 10, 20], jobs=args.steps, slots=8, seed=5)
    clk = clocks.stop()
    for line in lines:
        line["clocks"] = clk
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--variant", default="passive", choices=VARIANT_NAMES)
    ap.add_argument("--alpha", type=float, default=0.4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--form", default="plain",
                    choices=["plain", "batch", "study", "precision", "serve"])
    ap.add_argument("--fuse", type=int, default=2, choices=[0, 1, 2, 3, 4],
                    help="iteration schedule: 0 force + smoothing kernels, 1 fused, "
                         "3 split Gaussian (x/y kernel, z pass inside the force kernel), "
                         "4 as 3 with Eqs. 3-6 split after the difference image, "
                         "2 the library default (split where it applies)")
    args = ap.parse_args()
    args.variant_id = VARIANT_NAMES.index(args.variant)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.form == "batch":
        return run_batch(args)
    if args.form == "study":
        return run_study(args)
    if args.form == "precision":
        return run_precision(args)
    if args.form == "serve":
        return run_serve(args)

    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import paper_0909_0928_gb300 as dl
    from phantom import FULL, make_lung_phantom

    ph = make_lung_phantom(FULL)
    S_h, M_h = ph["S"], ph["M"]
    n0 = S_h.size
    stream = torch.cuda.current_stream()
    S_d = torch.from_numpy(S_h).cuda()
    M_d = torch.from_numpy(M_h).cuda()
    W_d = torch.empty_like(S_d)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    # the timed steps run the registration exactly as a user does (no event
    # records inside the graph); the per-kernel times come from a separate
    # context with timing = 1 afterwards
    params = dl.dir_params_default(levels=LEVELS, iters=ITERS, alpha=args.alpha, timing=0,
                                   fuse=args.fuse)
    ctx = dl.dir_create(S_d, M_d, DIMS, SPACING, dl.DIR_F32, True, args.variant_id, params, stream)
    vu_step = voxel_updates(DIMS, LEVELS, ITERS)

    def step():
        st = dl.dir_register(ctx)
        dl.dir_warp(ctx, M_d, W_d, dl.DIR_F32, True)
        return st

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    step_ms, launches = [], 0
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        st = step()
        ev[i][1].record(stream)
        launches += st.kernel_launches + 1
    torch.cuda.synchronize()
    clk = clocks.stop()

    # finest-level kernel times: the same registration with event records
    # around every force and smoothing launch of the finest level
    tparams = dl.dir_params_default(levels=LEVELS, iters=ITERS, alpha=args.alpha, timing=1,
                                    fuse=args.fuse)
    tctx = dl.dir_create(S_d, M_d, DIMS, SPACING, dl.DIR_F32, True, args.variant_id, tparams,
                         stream)
    kt = {"force": [0.0, 0], "fused": [0.0, 0], "smooth": [0.0, 0]}
    schedule = 0
    for i in range(args.warmup + max(3, min(args.steps, 10))):
        flush.zero_()
        st = dl.dir_register(tctx)
        schedule = st.schedule_finest
        if i < args.warmup:
            continue
        for k, ms, n in (("force", st.ms_force_finest, st.n_force_finest),
                         ("fused", st.ms_fused_finest, st.n_fused_finest),
                         ("smooth", st.ms_smooth_finest, st.n_smooth_finest)):
            kt[k][0] += ms
            kt[k][1] += n
    dl.dir_destroy(tctx)

    # the finest-level iteration without event records in the graph: the same
    # registration iterating only the finest level, less the one iterating
    # nowhere (pyramid, upsampling and the last smoothing are in both)
    def untimed_ms(iters, reps=8, variant=None, fuse=None):
        p = dl.dir_params_default(levels=LEVELS, iters=iters, alpha=args.alpha,
                                  fuse=args.fuse if fuse is None else fuse)
        c = dl.dir_create(S_d, M_d, DIMS, SPACING, dl.DIR_F32, True,
                          args.variant_id if variant is None else variant, p, stream)
        ms = []
        for i in range(reps + 3):
            flush.zero_()
            st = dl.dir_register(c)
            if i >= 3:
                ms.append(st.ms_total)
        dl.dir_destroy(c)
        return statistics.median(ms)
    fine_only = [0] * (LEVELS - 1) + [ITERS[-1]]
    finest_untimed_ms = (untimed_ms(fine_only) - untimed_ms([0] * LEVELS)) / ITERS[-1]
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    total_ms = max_over_ranks(total_ms, dist, "cuda")
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    value = whole_job_rate(vu_step, args.steps, world, total_ms)

    # end to end through the public API with host buffers: upload (pinned) ->
    # register -> field download, every step
    S_p = torch.from_numpy(S_h).pin_memory()
    M_p = torch.from_numpy(M_h).pin_memory()
    U_p = torch.empty(3 * n0, dtype=torch.float32).pin_memory()
    e2e_s = []
    for i in range(args.warmup + min(args.steps, 10)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dl.dir_load(ctx, S_p, M_p, dl.DIR_F32, False)
        dl.dir_register(ctx)
        dl.dir_get_field(ctx, U_p, False, False)
        e2e_s.append(time.perf_counter() - t0)
    e2e_s = e2e_s[args.warmup:]
    e2e_serial = world * vu_step / statistics.mean(e2e_s)

    # the same, as a user streaming registrations would run it: two contexts
    # on their own streams, so that one registration's upload and readback
    # overlap the other's kernels; every step still uploads its pair, runs its
    # registration and reads its field back inside the timed region
    streams2 = [torch.cuda.Stream(), torch.cuda.Stream()]
    ctx2 = [dl.dir_create(S_d, M_d, DIMS, SPACING, dl.DIR_F32, True, args.variant_id, params,
                          st2) for st2 in streams2]
    U2 = [torch.empty(3 * n0, dtype=torch.float32).pin_memory() for _ in range(2)]
    for c2 in ctx2:  # capture both graphs before timing
        dl.dir_register(c2)

    def pipelined(k):
        for i in range(k):
            c2 = ctx2[i % 2]
            dl.dir_load(c2, S_p, M_p, dl.DIR_F32, False)
            dl.dir_register_async(c2)
            if i > 0:
                prev = ctx2[(i - 1) % 2]
                dl.dir_sync(prev)
                dl.dir_get_field(prev, U2[(i - 1) % 2], False, False)
        last = ctx2[(k - 1) % 2]
        dl.dir_sync(last)
        dl.dir_get_field(last, U2[(k - 1) % 2], False, False)

    pipelined(args.warmup)
    k_e2e = max(4, min(args.steps, 20))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pipelined(k_e2e)
    e2e_pipe_s = (time.perf_counter() - t0) / k_e2e
    for c2 in ctx2:
        dl.dir_destroy(c2)
    e2e_value = world * vu_step / e2e_pipe_s

    # roofline of the dominant kernel (finest-level launches, timed live);
    # algorithmic bytes per voxel: force and fused iteration read the field
    # (12), S (4) and M (4) and write the field (12); smoothing reads and writes
    # the field (24)
    peak, peak_kind = measured_peak_gbs()
    n_fine = n0
    bytes_pv = {"force": FORCE_BYTES[args.variant_id], "fused": FORCE_BYTES[args.variant_id],
                "smooth": SMOOTH_BYTES}
    kernel_of = {"force": "force_tma_kernel" if args.variant_id in (0, 1) else "force_tma_gm_kernel",
                 "fused": "fused2_kernel", "smooth": "smooth2_kernel"}
    if schedule == 2:  # split Gaussian: x/y kernel, then z pass + force (same bytes per voxel)
        kernel_of.update(force="force_zs_kernel", smooth="smooth_xy_kernel")
    if schedule == 3:  # Eqs. 3-6: x/y kernel, z + D kernel, stencil force kernel
        kernel_of.update(force="force_zd_kernel+force_st_kernel", smooth="smooth_xy_kernel")
        # z + D: t 12, S 4, M 4, u 12, D 4 (Eq. 6: + d 4); force: D 4, S 4, u 12, v 12 (+ d 4)
        bytes_pv["force"] = 68 if args.variant_id != 5 else 76
    per_kernel = {}
    for k, (ms, n) in kt.items():
        if n:
            avg = ms / n
            per_kernel[k] = {"launches": n, "total_ms": ms, "avg_ms": avg,
                             "achieved_gbs": n_fine * bytes_pv[k] / (avg / 1e3) / 1e9,
                             "frac": n_fine * bytes_pv[k] / (avg / 1e3) / 1e9 / peak}
    if "force" in per_kernel and "smooth" in per_kernel and "fused" not in per_kernel:
        # one finest-level iteration of the two-kernel schedule (force, then
        # smoothing, gaps between them included)
        it_ms = per_kernel["force"]["avg_ms"] + per_kernel["smooth"]["avg_ms"]
        it_b = n_fine * (bytes_pv["force"] + bytes_pv["smooth"])
        per_kernel["iteration"] = {"avg_ms": it_ms, "bytes_per_voxel": bytes_pv["force"] +
                                   bytes_pv["smooth"], "achieved_gbs": it_b / (it_ms / 1e3) / 1e9,
                                   "frac": it_b / (it_ms / 1e3) / 1e9 / peak}
        per_kernel["iteration_untimed"] = {
            "avg_ms": finest_untimed_ms, "bytes_per_voxel": bytes_pv["force"] + bytes_pv["smooth"],
            "achieved_gbs": it_b / (finest_untimed_ms / 1e3) / 1e9,
            "frac": it_b / (finest_untimed_ms / 1e3) / 1e9 / peak,
            "method": f"(registration with 0/../{ITERS[-1]} iterations - with none) / {ITERS[-1]}, "
                      "no event records in the graph, median of 8"}
    kname = max((k for k in per_kernel if not k.startswith("iteration")),
                key=lambda k: per_kernel[k]["total_ms"])
    kk = per_kernel[kname]
    traffic = profiled_traffic(kernel_of[kname])
    roofline = {"bound": "hbm", "kernel": kernel_of[kname], "achieved": kk["achieved_gbs"],
                "peak": peak, "unit": "GB/s", "frac": kk["frac"], "traffic": traffic,
                "algorithmic_bytes_per_launch": n_fine * bytes_pv[kname],
                "avg_launch_ms": kk["avg_ms"],
                "peak_source": f"{peak_kind} hbm_gbs (copy bandwidth)",
                "finest_level_kernels": per_kernel}

    per_variant = None
    if not args.no_variants:
        per_variant = {}
        # the library's default schedule (fuse = 2: the split Gaussian for
        # Eqs. 1-2) for every force law, plus Eqs. 1-2 with the two-kernel
        # schedule everywhere (0) and passive fused everywhere (1)
        for vid, alpha, fuse in ((0, 0.4, 2), (0, 0.4, 0), (0, 0.4, 1), (1, 0.4, 2), (1, 0.4, 0),
                                 (2, 0.4, 2), (2, 0.4, 0), (3, 0.4, 2), (4, 0.4, 2), (4, 2.0, 2),
                                 (5, 0.4, 2), (5, 0.4, 0)):
            p2 = dl.dir_params_default(levels=LEVELS, iters=ITERS, alpha=alpha, fuse=fuse)
            c2 = dl.dir_create(S_d, M_d, DIMS, SPACING, dl.DIR_F32, True, vid, p2, stream)
            ms = []
            for k in range(8):
                flush.zero_()
                st = dl.dir_register(c2)
                if k >= 3:
                    ms.append(st.ms_total)
            dl.dir_destroy(c2)
            name = VARIANT_NAMES[vid] + (f"_alpha{alpha}" if vid == 4 else "") + \
                {2: "", 0: "_two_kernel", 1: "_fused_all_levels", 3: "_split_gaussian"}[fuse]
            med = statistics.median(ms)
            per_variant[name] = {"ms_p50": med, "voxel_updates_per_s": vu_step / (med / 1e3)}
        # the finest-level iteration of Eqs. 3 and 6 in the default schedule
        # (x/y kernel, z + D kernel, stencil force kernel), untimed as above.
        # Algorithmic bytes per voxel: x/y 24, z + D 36 (t 12, S 4, M 4, u 12,
        # D 4; Eq. 6 + d 4), force 32 (D 4, S 4, u 12, v 12; Eq. 6 + d 4)
        try:
            for vid, bpv in ((2, 92), (5, 100)):
                it_ms = (untimed_ms(fine_only, variant=vid, fuse=2) -
                         untimed_ms([0] * LEVELS, variant=vid, fuse=2)) / ITERS[-1]
                gbs = n0 * bpv / (it_ms / 1e3) / 1e9
                per_variant[VARIANT_NAMES[vid] + "_finest_iteration"] = {
                    "avg_ms": it_ms, "bytes_per_voxel": bpv, "achieved_gbs": gbs,
                    "frac": gbs / peak, "method": "as roofline.finest_level_kernels."
                                                  "iteration_untimed, default schedule"}
        except Exception as e:  # reported, never fatal to the bench line
            per_variant["eqs3_6_finest_iteration_error"] = repr(e)

    dl.dir_destroy(ctx)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(ph, args.variant_id, args.alpha, [40, 20, 10], [8, 4, 2])
        cpu = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample", "single_thread")}

    if rank == 0:
        srt = sorted(step_ms)
        p50 = statistics.median(srt)
        p99 = srt[min(len(srt) - 1, int(round(0.99 * (len(srt) - 1))))]
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic lung phantom (seeded), stands in for the "
                                        "paper's DIR-lab 4DCT cases",
                "config": workload_config(args.variant_id, args.alpha, world),
                "s_per_registration": {"p50": p50 / 1e3, "p99": p99 / 1e3,
                                       "mean": total_ms / args.steps / 1e3},
                "voxel_updates_per_step": vu_step,
                "roofline": roofline, "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * n0 * 4,
                        "d2h_bytes_per_step": 3 * n0 * 4,
                        "s_per_registration": e2e_pipe_s,
                        "method": f"{k_e2e} steps through dir_load (pinned host pair) -> "
                                  "dir_register_async -> dir_sync -> dir_get_field (pinned host "
                                  "field), alternating two contexts on two streams so one step's "
                                  "copies overlap the other's kernels; wall clock",
                        "serial_one_context": {"value": e2e_serial, "unit": UNIT,
                                               "s_per_registration_mean": statistics.mean(e2e_s)}},
                "gpu_launches": launches, "clocks": clk, "per_variant": per_variant,
                "paper_context": "7.02-11.10 s per 256x256x94-112 registration on a GeForce GTX "
                                 "285 (Table 2; iteration counts not reported)"}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
