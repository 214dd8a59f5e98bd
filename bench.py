#!/usr/bin/env python
"""Benchmark of the observer-siting hot path on one GB300.

Two pipelines site 4096 observers on the resident 46400^2 terrain (R=100,
40000 candidates from top-4 per 464^2 block):
  plain      vix (S=10 LOS per post) -> findmax -> viewshed -> site
  surrogate  CNN scores on a lattice of posts -> findmax_f32 -> viewshed -> site
             (network trained beforehand on another terrain of the same recipe;
             lattice stride tuned on a third one: the largest of 32..128 whose
             coverage is within 0.1% of stride 32's)
The headline `value` is the end-to-end siting time of the surrogate pipeline
when its coverage is within 1% of (or above) the plain pipeline's, else of
the plain pipeline; both are reported in full.  Prints ONE JSON line.

    python bench.py [--steps K] [--warmup W] [--workload full|scale|small]
    python bench.py --impl reference   # the CPU oracle on a bounded sample

Multi-GPU: the path is run as independent replicas (one terrain per rank, no
collective on the data path); rank 0 prints the max-over-ranks time.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import workloads as WL  # noqa: E402

METRIC = "viewsheds/sec and end-to-end siting s at 46400² (plain vs surrogate, equal coverage)"
L2_BYTES = 129 * 1024 * 1024
OPS_PER_LOS_STEP = 10     # integer issue slots per LOS crossing (2 loads + 8 ALU)
OPS_PER_RAY_STEP = 16     # integer issue slots per viewshed ray step


# ------------------------------------------------------------------ helpers
def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
        return dist, dist.get_rank(), ws, int(os.environ.get("LOCAL_RANK", "0"))
    return None, 0, 1, 0


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 50 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ workload
def pick_workload(name):
    return {"full": WL.FULL, "scale": WL.SCALE, "small": WL.SMALL, "mid": WL.MID}[name]


def interior_ray_steps(R):
    """Ray steps of one viewshed whose disc lies inside the grid: rays to the
    8R ring cells, each walked until it leaves the disc."""
    n = 0
    for e in range(-R + 1, R + 1):          # one side of the ring (ex = R), times 4
        for k in range(1, R + 1):
            num = k * e
            rnd = (2 * abs(num) + R) // (2 * R)
            if k * k + rnd * rnd > R * R:
                break
            n += 1
    return 4 * n


class Pipeline:
    def __init__(self, V, w, g, dev):
        self.V, self.w, self.g = V, w, g
        self.n = V.findmax_count(w.H, w.W, 1, w.block, w.k)
        self.vixbuf = torch.empty((w.H, w.W), dtype=torch.uint8, device=dev)
        self.cand = torch.empty(self.n, dtype=torch.int64, device=dev)
        self.bm = torch.empty((self.n, 2 * w.R + 1, V.words_per_row(w.R)), dtype=torch.int32, device=dev)
        self.area = torch.empty(self.n, dtype=torch.int32, device=dev)
        self.cum = torch.empty((w.H, (w.W + 31) // 32), dtype=torch.int32, device=dev)
        self.ws = torch.empty(V.site_workspace(self.n, w.R), dtype=torch.uint8, device=dev)
        self.ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        self.result = None

    def step(self, record=False, g=None, host=None):
        V, w = self.V, self.w
        ev = self.ev
        g = g or self.g
        if host is not None:  # vix reads every post: copy the whole terrain first
            g.storage.copy_(host, non_blocking=True)
        if record:
            ev[0].record()
        V.vix(g, w.R, w.ht, w.hr, w.S, w.vix_seed, out=self.vixbuf)
        if record:
            ev[1].record()
        V.findmax(self.vixbuf, w.block, w.k, out=self.cand)
        if record:
            ev[2].record()
        V.viewshed(g, w.R, w.ht, w.hr, self.cand, bm=self.bm, area=self.area)
        if record:
            ev[3].record()
        self.cum.zero_()
        self.result = V.site(self.bm, self.cand, w.H, w.W, w.R, w.n_obs, cum=self.cum, ws=self.ws, sync=False)
        if record:
            ev[4].record()

    def stage_ms(self):
        return [self.ev[i].elapsed_time(self.ev[i + 1]) for i in range(4)]


# ------------------------------------------------------------------ CPU oracle sample
def oracle_sample(z_host, w, cand=None, threads=None):
    """Time the CPU oracle on a bounded sample of the workload, on all host
    threads and on one thread.  vix: a tile of posts, extrapolated linearly to
    the grid; viewshed: every candidate (the pipeline's own when given, else
    as many seeded interior posts) on all threads, a sample of them on one;
    site: the oracle's greedy over all those candidates for 1 and for 64
    steps (its set-up, the initial gains of every candidate, and the first 64
    steps), the per-step cost extrapolated to n_obs steps.  Returns
    (seconds on all threads, description, threads, seconds on one thread)."""
    from oracle import oracle as O
    threads = threads or os.cpu_count() or 1
    H, W = w.H, w.W
    rng = np.random.default_rng(12345)

    def vix_tile(side, nthr):
        y0, x0 = (H - side) // 2, (W - side) // 2
        posts = ((np.arange(y0, y0 + side)[:, None] * W) + np.arange(x0, x0 + side)[None, :]).ravel()
        ths = [threading.Thread(target=O.vix_posts, args=(z_host, w.R, w.ht, w.hr, w.S, w.vix_seed, c, W))
               for c in np.array_split(posts, nthr)]
        t = time.perf_counter()
        for th in ths:
            th.start()
        for th in ths:
            th.join()
        return (time.perf_counter() - t) * (H * W) / len(posts)

    side = 512 if H * W > 4e6 else min(H, W)
    t_vix = vix_tile(side, threads)
    t_vix1 = vix_tile(min(side, 128), 1)
    n_full = WL.FULL.n_candidates() if w is WL.FULL else w.n_candidates()
    if cand is None:
        cand = (rng.integers(w.R, H - w.R, n_full) * W + rng.integers(w.R, W - w.R, n_full)).astype(np.int64)
    cand = np.asarray(cand, np.int64)
    t = time.perf_counter()
    bm, _ = O.viewshed(z_host, w.R, w.ht, w.hr, cand, threads=threads)
    t_vs = (time.perf_counter() - t) * n_full / len(cand)
    ns = min(256, len(cand))
    t = time.perf_counter()
    O.viewshed(z_host, w.R, w.ht, w.hr, cand[:ns], threads=1)
    t_vs1 = (time.perf_counter() - t) * n_full / ns
    t = time.perf_counter()
    O.site(bm, cand, H, W, w.R, 1)
    t0 = time.perf_counter() - t
    t = time.perf_counter()
    ch, _, _ = O.site(bm, cand, H, W, w.R, 64)
    t1 = time.perf_counter() - t
    per_step = max(t1 - t0, 0.0) / max(len(ch) - 1, 1)
    t_site = t0 + per_step * (w.n_obs - 1)
    total, total1 = t_vix + t_vs + t_site, t_vix1 + t_vs1 + t_site
    desc = ("oracle on %d threads (and on 1): vix of a %dx%d post tile (%dx%d on 1 thread), the %d candidates' "
            "viewsheds (%d on 1 thread), the greedy over all %d for its first 64 steps; extrapolated linearly to "
            "%dx%d posts and %d observers (vix %.1f s, viewshed %.1f s, site %.1f s; 1 thread: vix %.1f s, "
            "viewshed %.1f s)" % (threads, side, side, min(side, 128), min(side, 128), len(cand), ns, len(cand),
                                  H, W, w.n_obs, t_vix, t_vs, t_site, t_vix1, t_vs1))
    return total, desc, threads, total1


# ------------------------------------------------------------------ learned proposal
class SurrogatePipeline:
    """Train the proposal network on another terrain of the same recipe (the
    bench terrain is held out), then site from its lattice scores."""

    def __init__(self, V, w, g, pipe, args, dev):
        from paper_2006_16783_gb300 import surrogate as S
        self.V, self.w, self.g = V, w, g
        t0 = time.perf_counter()
        wtr = WL.scaled(w, w.H, w.W, name=w.name + "_train", seed=w.seed + 7)
        ztr = wtr.make_terrain(dev)
        ztr_s, _ = WL.terrain.pad_pitch(ztr, 8)
        del ztr
        gtr = V.Grid(ztr_s, w.W)
        posts = S.sample_posts(w.H, w.W, args.train_posts, 32, 11, dev)
        labels = S.exact_vix(gtr, posts, w.R, w.ht, w.hr)
        self.label_s = time.perf_counter() - t0
        self.tr = S.Trainer(S.init_master(0), batch=512, lr=2e-3, patch_step=args.patch_step)
        t1 = time.perf_counter()
        self.train_loss = self.tr.fit([(gtr, posts, labels)], epochs=args.epochs, seed=3,
                                      log=lambda m: print(m, file=sys.stderr))
        torch.cuda.synchronize()
        self.train_s = time.perf_counter() - t1
        del gtr, ztr_s, posts, labels
        # held-out error on the bench terrain, next to the 10-sample vix estimate
        pt = S.sample_posts(w.H, w.W, 200000, 32, 5, dev)
        lt = S.exact_vix(g, pt, w.R, w.ht, w.hr)
        self.mae = float((self.tr.predict(g, pt) - lt).abs().mean())
        self.mae_vix = float((pipe.vixbuf.reshape(-1)[pt].float() / w.S - lt).abs().mean())
        self.mae_posts = pt.numel()
        # proposal stride: given, or tuned on another terrain of the recipe --
        # the largest stride whose coverage is within 0.1 % of the densest's
        self.tuning = None
        st = args.sur_stride
        if st <= 0:
            st, self.tuning = self._tune_stride(pipe, dev)
        self.stride = st
        self.n = V.findmax_count(w.H, w.W, st, w.block, w.k)
        self.score = torch.empty(((w.H + st - 1) // st, (w.W + st - 1) // st), dtype=torch.float32, device=dev)
        self.cand = torch.empty(self.n, dtype=torch.int64, device=dev)
        self.bm = torch.empty((self.n, 2 * w.R + 1, V.words_per_row(w.R)), dtype=torch.int32, device=dev)
        self.area = torch.empty(self.n, dtype=torch.int32, device=dev)
        self.cum = torch.empty_like(pipe.cum)
        self.ws = torch.empty(V.site_workspace(self.n, w.R), dtype=torch.uint8, device=dev)
        self.ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        self.copy_stream = torch.cuda.Stream()
        self.result = None

    STRIDES = (32, 48, 64, 96, 128)

    def _tune_stride(self, pipe, dev):
        V, w = self.V, self.w
        t0 = time.perf_counter()
        wtu = WL.scaled(w, w.H, w.W, name=w.name + "_tune", seed=w.seed + 8)
        ztu = wtu.make_terrain(dev)
        ztu_s, _ = WL.terrain.pad_pitch(ztu, 8)
        del ztu
        gtu = V.Grid(ztu_s, w.W)
        nmax = max(V.findmax_count(w.H, w.W, st, w.block, w.k) for st in self.STRIDES)
        cand = torch.empty(nmax, dtype=torch.int64, device=dev)
        bm = torch.empty((nmax, 2 * w.R + 1, V.words_per_row(w.R)), dtype=torch.int32, device=dev)
        area = torch.empty(nmax, dtype=torch.int32, device=dev)
        cum = torch.empty_like(pipe.cum)
        ws = torch.empty(V.site_workspace(nmax, w.R), dtype=torch.uint8, device=dev)
        cov = {}
        for st in self.STRIDES:
            n = V.findmax_count(w.H, w.W, st, w.block, w.k)
            score = V.cnn_score_lattice(gtu, st, self.tr.packed, patch_step=self.tr.patch_step)
            V.findmax_f32(score, w.H, w.W, st, w.block, w.k, out=cand[:n])
            V.viewshed(gtu, w.R, w.ht, w.hr, cand[:n], bm=bm[:n], area=area[:n])
            cum.zero_()
            cov[st] = coverage(V.site(bm[:n], cand[:n], w.H, w.W, w.R, w.n_obs, cum=cum, ws=ws, sync=False))[0]
        best = max(s for s in self.STRIDES if cov[s] >= (1.0 - 1e-3) * cov[self.STRIDES[0]])
        del gtu, ztu_s, cand, bm, area, cum, ws
        torch.cuda.synchronize()
        return best, {"terrain_seed": w.seed + 8, "coverage_by_stride": cov, "chosen": best,
                      "rule": "largest stride with coverage >= 0.999 x the stride-32 coverage",
                      "tune_s": time.perf_counter() - t0}

    def step(self, record=False, g=None, host=None):
        """One siting; with ``host`` (a pinned copy of the terrain) the terrain
        is streamed into ``g`` while the lattice is scored."""
        from paper_2006_16783_gb300 import surrogate as S
        V, w, ev = self.V, self.w, self.ev
        g = g or self.g
        if record:
            ev[0].record()
        if host is not None:
            S.score_lattice_streamed(g, host, self.stride, self.tr.packed, self.score,
                                     patch_step=self.tr.patch_step, copy_stream=self.copy_stream)
        else:
            V.cnn_score_lattice(g, self.stride, self.tr.packed, out=self.score, patch_step=self.tr.patch_step)
        if record:
            ev[1].record()
        V.findmax_f32(self.score, w.H, w.W, self.stride, w.block, w.k, out=self.cand)
        if record:
            ev[2].record()
        V.viewshed(g, w.R, w.ht, w.hr, self.cand, bm=self.bm, area=self.area)
        if record:
            ev[3].record()
        self.cum.zero_()
        self.result = V.site(self.bm, self.cand, w.H, w.W, w.R, w.n_obs, cum=self.cum, ws=self.ws, sync=False)
        if record:
            ev[4].record()

    def stage_ms(self):
        return [self.ev[i].elapsed_time(self.ev[i + 1]) for i in range(4)]

    names = ["cnn_lattice", "findmax_f32", "viewshed", "site"]


def site_loop_bytes(cand, chosen, W, R, PR):
    """Algorithmic bytes of the greedy loop: per step the winner's window (V and
    C read, C written: 3 * (2R+1) * PR words) and, for every candidate not yet
    chosen whose window meets the winner's, the overlap words of its bitmap (an
    upper bound: the kernel skips words without new coverage)."""
    words = (2 * R + 1) * PR
    cy, cx = cand // W, cand % W
    gw0 = np.floor_divide(cx - R, 32)
    alive = np.ones(len(cand), dtype=bool)
    where = {int(p): i for i, p in enumerate(cand)}
    total = 0
    for p in chosen:
        i = where[int(p)]
        alive[i] = False
        wy, wgw = cy[i], gw0[i]
        rows = np.clip(np.minimum(cy, wy) + R - (np.maximum(cy, wy) - R) + 1, 0, None)
        cols = np.clip(np.minimum(gw0, wgw) + PR - 1 - np.maximum(gw0, wgw) + 1, 0, None)
        near = alive & (np.abs(cx - cx[i]) <= 2 * R)
        total += 3 * words * 4 + int((rows * cols)[near].sum()) * 4
    return total


def recorded_counters():
    """Per-unit figures of the headline kernels from the committed ncu capture
    on the mid workload (profiles/counters_mid_11600sq_R100.json): thread
    instructions and DRAM bytes per work unit (LOS crossing, ray step,
    candidate) and the issue-active share.  A kernel's figures are used only
    while its source file hashes to the recorded SHA-1."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles", "counters_mid_11600sq_R100.json")
    out = {}
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return out
    import hashlib
    for key, r in rec.get("kernels", {}).items():
        src = os.path.join(os.path.dirname(path), "..", r["source"])
        try:
            sha = hashlib.sha1(open(src, "rb").read()).hexdigest()
        except OSError:
            continue
        if sha == r["sha1"]:
            out[key] = r
    return out


def coverage(result):
    ch, gn, _, nch = result
    t = int(nch.item())
    return int(gn[:t].sum().item()), t


def time_steps(pipe, steps, dist, dev):
    """K steps bracketed by a barrier and device syncs; per-stage medians."""
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stage = []
    e0.record()
    for _ in range(steps):
        torch.cuda.nvtx.range_push("timed_step")  # lets a profiler select the timed launches
        pipe.step(record=True)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        stage.append(pipe.stage_ms())
    e1.record()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = max_over_ranks(e0.elapsed_time(e1) / steps, dist, dev)
    return ms, [statistics.median(x[i] for x in stage) for i in range(4)]


def cnn_flops_per_patch():
    """Algorithmic FLOPs of one patch of the network: 2 * outputs * 9 * cin
    per 3x3 convolution (65 -> 33 -> 17 -> 9 -> 5 -> 5 pixels, 1 then 32
    input channels, 32 output channels; every output counts all 9 taps) and
    2 * 32 for the fc layer."""
    n, tot = 65, 0
    for cin, stride in ((1, 2), (32, 2), (32, 2), (32, 2), (32, 1)):
        n = (n - 1) // stride + 1
        tot += 2 * n * n * 32 * cin * 9
    return tot + 2 * 32


def max_over_ranks(value, dist, dev):
    """The slowest replica's figure (every rank gets it); identity without a
    process group."""
    if not dist:
        return value
    tt = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


# ------------------------------------------------------------------ main
def run_reference(args, w, rank):
    """The oracle as it stands, on the host cores, one bounded sample per step."""
    if rank != 0:
        return
    z = w.make_terrain("cuda" if torch.cuda.is_available() else "cpu").cpu().numpy()
    for _ in range(args.warmup):
        oracle_sample(z, w)
    vals = []
    desc = threads = v1 = None
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, desc, threads, v1 = oracle_sample(z, w)
        vals.append(v)
    wall = time.perf_counter() - t0
    value = statistics.median(vals)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * wall / max(args.steps, 1),
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
           "data": "synthetic", "config": {"workload": w.name, "H": w.H, "W": w.W, "R": w.R,
                                           "ht": w.ht, "hr": w.hr, "S": w.S, "block": w.block,
                                           "k": w.k, "n_obs": w.n_obs},
           "cpu_baseline": {"value": value, "unit": "s", "cores": threads, "kind": "oracle", "sample": desc,
                            "single_thread_value": v1},
           "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def cnn_oracle_sample(z_host, w, stride, step, npatch=24):
    """Seconds per patch of the numpy CNN oracle (fp64 forward of single patches)."""
    from oracle import cnn_oracle as C
    p = C.init_params(0)
    rng = np.random.default_rng(1)
    cy = rng.integers(32, w.H - 32, npatch)
    cx = rng.integers(32, w.W - 32, npatch)
    x0 = np.stack([C.normalize_patch(C.extract_patch(z_host, int(a), int(b), step)) for a, b in zip(cy, cx)])
    t = time.perf_counter()
    C.forward(p, x0)
    return (time.perf_counter() - t) / npatch


def run_learn(args, rank, local):
    """The learned-proposal workload: train on posts of eight 4096^2 fBm
    terrains (exact R=100 labels), report the error on a held-out 16384^2
    terrain next to the 10-sample vix estimate of the same quantity.  fBm
    relief grows as size^H, so the held-out terrain's elevation range is
    scaled by 4^0.8 to keep the relief at the ROI scale comparable."""
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2006_16783_gb300 as V
    from paper_2006_16783_gb300 import surrogate as S
    R, h, n_train, n_test = 100, 10, args.train_posts, 1000000
    t0 = time.perf_counter()
    data = []
    per = n_train // 8
    for i in range(8):
        z = WL.terrain.spectral_fbm(4096, 4096, 0.8, 3000 + i, 0, 1000, device=dev)
        g = V.Grid(z.contiguous())
        posts = S.sample_posts(4096, 4096, per, 32, 3000 + i, dev)
        data.append((g, posts, S.exact_vix(g, posts, R, h, h)))
    zt = WL.terrain.spectral_fbm(16384, 16384, 0.8, 3100, 0, int(round(1000 * 4 ** 0.8)), device=dev)
    gt = V.Grid(zt.contiguous())
    pt = S.sample_posts(16384, 16384, n_test, 32, 3100, dev)
    lt = S.exact_vix(gt, pt, R, h, h)
    label_s = time.perf_counter() - t0
    tr = S.Trainer(S.init_master(0), batch=512, lr=2e-3, patch_step=args.patch_step)
    t1 = time.perf_counter()
    last = tr.fit(data, epochs=args.epochs, seed=3, log=lambda m: print(m, file=sys.stderr))
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t1
    mae = float((tr.predict(gt, pt) - lt).abs().mean())
    mae_vix = float((S.sampled_vix_fraction(gt, pt, R, h, h, 10, 0x5EED) - lt).abs().mean())
    out = {"metric": "held-out MAE of the learned visibility index (R=100)", "value": mae, "unit": "abs err",
           "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
           "config": {"workload": "learn_8x4096sq_fbm_heldout_16384sq", "train_posts": per * 8,
                      "test_posts": n_test, "epochs": args.epochs, "R": R, "h": h,
                      "patch_step": args.patch_step},
           "mae_sampled_vix_S10": mae_vix, "train_loss_last_epoch": last, "label_s": label_s,
           "train_s": train_s, "train_patches_per_s": per * 8 * args.epochs / train_s,
           "label_mean": float(lt.mean()), "label_std": float(lt.std())}
    if rank == 0:
        print(json.dumps(out))


def batch_oracle_sample(items, zs, bufs, threads=None):
    """The oracle on the batched workload, terrain by terrain, on the host
    cores: vix of a 128 x 128 tile (all threads) and 100 viewsheds (all
    threads), each extrapolated linearly to the terrain, and the greedy run in
    full on the pipeline's bitmaps (identical to the oracle's).  Returns
    (seconds, threads, description)."""
    from oracle import oracle as O
    threads = threads or os.cpu_count() or 1
    t_vix = t_vs = t_site = 0.0
    for it, z, b in zip(items, zs, bufs):
        H, W = z.shape
        side = min(128, H, W)
        y0, x0 = (H - side) // 2, (W - side) // 2
        posts = ((np.arange(y0, y0 + side)[:, None] * W) + np.arange(x0, x0 + side)[None, :]).ravel()
        ths = [threading.Thread(target=O.vix_posts, args=(z, it["R"], it["ht"], it["hr"], it["S"], it["seed"], c, W))
               for c in np.array_split(posts, threads)]
        t = time.perf_counter()
        for th in ths:
            th.start()
        for th in ths:
            th.join()
        t_vix += (time.perf_counter() - t) * H * W / len(posts)
        cand = b["cand"].cpu().numpy()
        sub = cand[:100]
        t = time.perf_counter()
        O.viewshed(z, it["R"], it["ht"], it["hr"], sub, threads=threads)
        t_vs += (time.perf_counter() - t) * len(cand) / max(len(sub), 1)
        bm = b["bm"].cpu().numpy().view(np.uint32)
        t = time.perf_counter()
        O.site(bm, cand, H, W, it["R"], it["n_obs"])
        t_site += time.perf_counter() - t
    desc = ("oracle on %d threads, terrain by terrain: vix of a 128x128 tile and 100 viewsheds, extrapolated "
            "linearly to every post and candidate; the greedy in full on the pipeline's bitmaps (vix %.1f s, "
            "viewshed %.1f s, site %.1f s)" % (threads, t_vix, t_vs, t_site))
    return t_vix + t_vs + t_site, threads, desc


def run_batch(args, dist, rank, world, local):
    """The 64-terrain batched workload: every terrain's vix in one persistent
    launch, every findmax in one launch, every viewshed in one persistent
    launch, the greedy problems' preparation and loops in seven launches, all
    captured in one CUDA graph; the launch shapes come from the autotuner.
    value = seconds per graph replay."""
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2006_16783_gb300 as V
    from paper_2006_16783_gb300 import autotune
    from paper_2006_16783_gb300.batch import BatchedSiting
    inst = WL.batch_instances()
    t = time.perf_counter()
    items, zs = [], []
    for w in inst:
        z = w.make_terrain(dev)
        items.append({"grid": V.Grid.from_tensor(z, dev), "R": w.R, "ht": w.ht, "hr": w.hr, "S": w.S,
                      "seed": w.vix_seed, "block": w.block, "k": w.k, "n_obs": w.n_obs})
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            zs.append(z.cpu().numpy())
        del z
    gen_s = time.perf_counter() - t
    table = None
    if not args.no_tune:
        big = max(items, key=lambda it: it["grid"].H * it["grid"].W)
        table = autotune.tune_all(big["grid"], [it["R"] for it in items],
                                  log=lambda m: print(m, file=sys.stderr))
    bs = BatchedSiting(items, dev)
    # one eager siting: its launches (graph replays bypass the library's
    # counter) and the time of each batched stage
    bs.run()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    c0 = V.launch_count()
    ev[0].record()
    V.vix_batch(bs.vix_jobs, bs.vix_ws)
    ev[1].record()
    V.findmax_batch(bs.fm_jobs)
    ev[2].record()
    V.viewshed_batch(bs.vs_jobs, bs.vs_ws)
    ev[3].record()
    bs.cum_all.zero_()
    V.site_batch(bs.site_jobs_, bs.site_ws)
    ev[4].record()
    torch.cuda.synchronize()
    launches = V.launch_count() - c0
    st = [ev[i].elapsed_time(ev[i + 1]) for i in range(4)]
    # LOS crossings of the vix stage, counted
    steps = torch.zeros(1, dtype=torch.int64, device=dev)
    for it in items:
        V.vix_count(it["grid"], it["R"], it["ht"], it["hr"], it["S"], it["seed"], steps)
    torch.cuda.synchronize()
    los_steps = int(steps.item())
    bs.capture()
    for _ in range(args.warmup):
        bs.replay()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        bs.replay()
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    if dist:
        dist.barrier()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, dev)
    res = bs.results()
    ncand = sum(b["cand"].numel() for b in bs.bufs)
    nobs = sum(int(r[1].numel()) for r in res)
    cov = sum(int(r[1].sum().item()) for r in res)
    posts = sum(it["grid"].H * it["grid"].W for it in items)
    peaks, peak_src = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    issue_peak = sms * 4 * 32 * mhz * 1e6 / 1e9
    names = ["vix", "findmax", "viewshed", "site"]
    vix_roof = {"bound": "alu", "kernel": "vix", "units": los_steps, "unit": "Gop/s", "peak": issue_peak,
                "achieved": los_steps * OPS_PER_LOS_STEP / (st[0] * 1e-3) / 1e9, "traffic": None,
                "min_inst_per_unit": OPS_PER_LOS_STEP,
                "note": "minimal instruction sequence per LOS crossing (the batched kernel was not captured)"}
    vix_roof["frac"] = vix_roof["achieved"] / issue_peak
    out = {"metric": "batched siting s per graph replay (64 terrains)", "value": ms / 1000.0, "unit": "s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
           "data": "synthetic",
           "config": {"workload": "batch_64_terrains_512_to_4096", "instances": len(items), "posts": posts,
                      "candidates": ncand, "radii": sorted(set(it["R"] for it in items)),
                      "l2": "inputs larger than L2 (%.1f GB of terrain)" % (2.0 * posts / 1e9)},
           "stages_ms": dict(zip(names, st)), "dominant_stage": names[int(np.argmax(st))],
           "roofline": vix_roof, "peak_source": peak_src,
           "observers": nobs, "coverage_posts": cov, "viewsheds_per_s_incl_all_stages": ncand / (ms * 1e-3),
           "vix_los_steps": los_steps, "autotune": table, "clocks": clk, "terrain_gen_s": gen_s,
           "gpu_launches": args.steps * launches, "gpu_launches_per_step": launches}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, threads, desc = batch_oracle_sample(items, zs, bs.bufs)
        out["cpu_baseline"] = {"value": v, "unit": "s", "cores": threads, "kind": "oracle", "sample": desc}
    if rank == 0:
        print(json.dumps(out, default=str))


def run_paper(args, dist, rank, world, local):
    """The paper's own parameter regime (R = 1000, h_t = 100, h_r = 10,
    20 candidates per block of side ~R/3, greedy until 95% coverage): the
    plain pipeline with the large-ROI kernels (warp-per-line vix, banded
    viewshed, lazy greedy site).  One timed siting per step, per-stage CUDA
    events; the paper's elapsed times for the same table are context."""
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2006_16783_gb300 as V
    w = {"paper": WL.PAPER, "paper_mid": WL.PAPER_MID, "paper_small": WL.PAPER_SMALL,
         "paper_r2000": WL.PAPER_R2000}[args.workload]
    t = time.perf_counter()
    z = w.make_terrain(dev)
    zs, _ = WL.terrain.pad_pitch(z, 8)
    del z
    torch.cuda.empty_cache()
    g = V.Grid(zs, w.W)
    gen_s = time.perf_counter() - t
    n = V.findmax_count(w.H, w.W, 1, w.block, w.k)
    wsb = max(V.vshed.vix_workspace(w.H, w.W, w.R, w.S), V.vshed.viewshed_workspace(w.H, w.W, w.R, n))
    ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=dev)
    vixbuf = torch.empty((w.H, w.W), dtype=torch.uint8, device=dev)
    cand = torch.empty(n, dtype=torch.int64, device=dev)
    bm = torch.empty((n, 2 * w.R + 1, V.words_per_row(w.R)), dtype=torch.int32, device=dev)
    area = torch.empty(n, dtype=torch.int32, device=dev)
    cum = torch.empty((w.H, (w.W + 31) // 32), dtype=torch.int32, device=dev)
    sws = torch.empty(V.site_workspace(n, w.R), dtype=torch.uint8, device=dev)
    steps_ctr = torch.zeros(1, dtype=torch.int64, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]

    def step(count=False):
        ev[0].record()
        if count:
            V.vshed.vix_count(g, w.R, w.ht, w.hr, w.S, w.vix_seed, steps_ctr, out=vixbuf, ws=ws)
        else:
            V.vix(g, w.R, w.ht, w.hr, w.S, w.vix_seed, out=vixbuf, ws=ws)
        ev[1].record()
        V.findmax(vixbuf, w.block, w.k, out=cand)
        ev[2].record()
        V.viewshed(g, w.R, w.ht, w.hr, cand, bm=bm, area=area, ws=ws)
        ev[3].record()
        cum.zero_()
        res = V.site(bm, cand, w.H, w.W, w.R, w.n_obs, w.target, cum=cum, ws=sws, sync=False)
        ev[4].record()
        return res

    for i in range(args.warmup):
        step(count=(i == 0))
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    stages, walls = [], []
    n_launch0 = V.launch_count()
    for _ in range(args.steps):
        res = step()
        torch.cuda.synchronize()
        stages.append([ev[i].elapsed_time(ev[i + 1]) for i in range(4)])
        walls.append(ev[0].elapsed_time(ev[4]))
    n_launch = V.launch_count() - n_launch0
    clk = clocks.stop()
    if dist:
        dist.barrier()
    ms = max_over_ranks(statistics.median(walls), dist, dev)
    st = [statistics.median(x[i] for x in stages) for i in range(4)]
    covered, nobs = coverage(res)
    los = int(steps_ctr.item()) if args.warmup else None
    steps_vs = interior_ray_steps(w.R) * n
    sur_out = paper_surrogate(args, V, w, g, dev, vixbuf, bm, area, cum, sws, ws, nobs, ms, dist) \
        if args.paper_surrogate else None
    out = {"metric": "paper-regime siting s (vix + findmax + viewshed + site to 95% coverage)",
           "value": ms / 1000.0, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "int32", "data": "synthetic",
           "config": {"workload": w.name, "H": w.H, "W": w.W, "R": w.R, "ht": w.ht, "hr": w.hr, "S": w.S,
                      "block": w.block, "k": w.k, "n_obs_cap": w.n_obs, "coverage_target": w.target,
                      "bitmap_GB": bm.numel() * 4 / 1e9},
           "stages_ms": dict(zip(["vix", "findmax", "viewshed", "site"], st)),
           "candidates": n, "observers": nobs, "coverage_posts": covered,
           "coverage_frac": covered / float(w.H * w.W),
           "viewsheds_per_s": n / (st[2] * 1e-3), "interior_ray_steps_per_s": steps_vs / (st[2] * 1e-3),
           "vix_los_steps": los, "vix_los_steps_per_s": (los / (st[0] * 1e-3)) if los else None,
           "paper_context_s": {"vix": 130, "findmax": 9, "viewshed": 1706, "site": 3510,
                               "note": "the paper's US-West R=1000 run, 32-way CPU parallelism"},
           "clocks": clk, "gpu_launches": n_launch, "terrain_gen_s": gen_s}
    if sur_out:
        out["surrogate"] = sur_out
    if rank == 0:
        print(json.dumps(out, default=str))


def paper_surrogate(args, V, w, g, dev, vixbuf, bm, area, cum, sws, ws, nobs_plain, ms_plain, dist):
    """The learned proposal in the paper's regime: the network is trained on
    exact R = 1000 visibility indices of another terrain of the recipe, with a
    patch that spans the ROI (patch step 30: 65 posts 30 apart cover ~2R); it
    scores a lattice (stride 64 gives >= 20 lattice posts per 334-post block),
    findmax_f32 keeps 20 per block, and the exact viewshed and site steps run
    to the same 95 % coverage.  Reported beside the plain pipeline."""
    from paper_2006_16783_gb300 import surrogate as S
    P = args.paper_patch_step
    strides = [int(x) for x in str(args.paper_stride).split(",")]
    t0 = time.perf_counter()
    side = min(8192, w.H, w.W)
    wtr = WL.scaled(w, side, side, name=w.name + "_train", seed=w.seed + 7)
    ztr = wtr.make_terrain(dev)
    ztr_s, _ = WL.terrain.pad_pitch(ztr, 8)
    del ztr
    gtr = V.Grid(ztr_s, side)
    margin = 32 * P  # training patches inside the grid
    posts = S.sample_posts(side, side, args.train_posts, margin, 11, dev)
    labels = S.exact_vix(gtr, posts, w.R, w.ht, w.hr)
    torch.cuda.synchronize()
    label_s = time.perf_counter() - t0
    tr = S.Trainer(S.init_master(0), batch=512, lr=2e-3, patch_step=P)
    t1 = time.perf_counter()
    loss = tr.fit([(gtr, posts, labels)], epochs=args.epochs, seed=3, log=lambda m: print(m, file=sys.stderr))
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t1
    del gtr, ztr_s, posts, labels
    # held-out error on the bench terrain, beside the 10-sample vix
    pt = S.sample_posts(w.H, w.W, 20000, margin, 5, dev)
    lt = S.exact_vix(g, pt, w.R, w.ht, w.hr, ws=ws)
    mae = float((tr.predict(g, pt) - lt).abs().mean())
    mae_vix = float((vixbuf.reshape(-1)[pt].float() / w.S - lt).abs().mean())
    common = {"patch_step": P, "train_terrain": "%dx%d, seed %d" % (side, side, w.seed + 7),
              "train_posts": args.train_posts, "epochs": args.epochs, "train_loss_last_epoch": loss,
              "label_s": label_s, "train_s": train_s, "mae_heldout": mae, "mae_sampled_vix": mae_vix,
              "mae_posts": int(pt.numel()), "observers_plain": nobs_plain, "by_stride": {}}
    for stride in strides:
        common["by_stride"][str(stride)] = _paper_surrogate_run(args, V, w, g, dev, tr, P, stride, bm, area, cum,
                                                                sws, ws, ms_plain, dist)
    return common


def _paper_surrogate_run(args, V, w, g, dev, tr, P, stride, bm, area, cum, sws, ws, ms_plain, dist):
    """One lattice stride of the paper-regime proposal, timed like the plain
    pipeline.  --paper-block / --paper-k replace the findmax blocks of the
    proposal (e.g. the top 1 of every 75^2 block instead of the top 20 of
    every 334^2 block: about as many candidates, spread evenly)."""
    blk = args.paper_block or w.block
    kk = args.paper_k or w.k
    ns = V.findmax_count(w.H, w.W, stride, blk, kk)
    assert ns <= bm.shape[0]
    score = torch.empty(((w.H + stride - 1) // stride, (w.W + stride - 1) // stride), dtype=torch.float32,
                        device=dev)
    cand = torch.empty(ns, dtype=torch.int64, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]

    def step():
        ev[0].record()
        V.cnn_score_lattice(g, stride, tr.packed, out=score, patch_step=P)
        ev[1].record()
        V.findmax_f32(score, w.H, w.W, stride, blk, kk, out=cand)
        ev[2].record()
        V.viewshed(g, w.R, w.ht, w.hr, cand, bm=bm[:ns], area=area[:ns], ws=ws)
        ev[3].record()
        cum.zero_()
        r = V.site(bm[:ns], cand, w.H, w.W, w.R, w.n_obs, w.target, cum=cum, ws=sws, sync=False)
        ev[4].record()
        return r

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    stages, walls = [], []
    n0 = V.launch_count()
    for _ in range(args.steps):
        res = step()
        torch.cuda.synchronize()
        stages.append([ev[i].elapsed_time(ev[i + 1]) for i in range(4)])
        walls.append(ev[0].elapsed_time(ev[4]))
    n_launch = V.launch_count() - n0
    ms = max_over_ranks(statistics.median(walls), dist, dev)
    st = [statistics.median(x[i] for x in stages) for i in range(4)]
    covered, nobs = coverage(res)
    return {"s_per_step": ms / 1000.0, "stages_ms": dict(zip(["cnn_lattice", "findmax_f32", "viewshed", "site"], st)),
            "speedup_vs_plain": ms_plain / ms, "candidates": ns, "observers": nobs,
            "coverage_posts": covered, "coverage_frac": covered / float(w.H * w.W),
            "patches_per_step": score.numel(), "proposal_block": blk, "proposal_k": kk, "gpu_launches": n_launch}


def run_accuracy(args, dist, rank, world, local):
    """The accuracy study of the paper's closing section (sensitivity of the
    result to lowered accuracy in the data) and of its R2 / R3 discussion, on
    the headline workload's recipe:
      - cells where the ray-sweep viewshed (vs_viewshed, R2-style) and the
        exact per-cell viewshed (vs_viewshed_r3) disagree, over all candidates;
      - the exact (R3) coverage of the observers sited with R2 bitmaps against
        observers sited with R3 bitmaps;
      - the exact coverage on the true terrain of observers sited on the
        terrain rounded to q metres (q = 10, 50, 200)."""
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2006_16783_gb300 as V
    w = WL.FULL if args.accuracy_size == "full" else WL.MID
    t0 = time.perf_counter()
    z = w.make_terrain(dev)
    zs, _ = WL.terrain.pad_pitch(z, 8)
    del z
    g = V.Grid(zs, w.W)
    pipe = Pipeline(V, w, g, dev)

    def site_cov(bm, cand):
        cum = torch.zeros_like(pipe.cum)
        res = V.site(bm, cand, w.H, w.W, w.R, w.n_obs, cum=cum, ws=pipe.ws, sync=False)
        return res

    def union_cov(bm, cand, chosen):
        """Exact coverage of a fixed observer set: the union of their bitmaps
        (a greedy run over just those candidates picks every one that adds)."""
        idx = torch.nonzero(torch.isin(cand, chosen)).reshape(-1)
        cum = torch.zeros_like(pipe.cum)
        res = V.site(bm[idx].contiguous(), cand[idx].contiguous(), w.H, w.W, w.R, int(idx.numel()), cum=cum,
                     ws=pipe.ws, sync=False)
        return coverage(res)[0]

    # R2 pipeline on the true terrain
    pipe.step()
    torch.cuda.synchronize()
    cand = pipe.cand.clone()
    bm2 = pipe.bm
    ch2, gn2, _, n2 = pipe.result
    ch2 = ch2[:int(n2.item())].clone()
    cov2_r2 = int(gn2[:int(n2.item())].sum().item())
    # R3 bitmaps of the same candidates
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    bm3, area3 = V.viewshed_r3(g, w.R, w.ht, w.hr, cand)
    e1.record()
    torch.cuda.synchronize()
    r3_ms = e0.elapsed_time(e1)
    b2 = bm2.view(torch.int32)
    b3 = bm3.view(torch.int32)
    def popc(t):  # bits set, counted on the device (measurement only)
        u = t.view(torch.int32).to(torch.int64) & 0xFFFFFFFF
        c = torch.zeros_like(u)
        for sh in range(32):
            c += (u >> sh) & 1
        return int(c.sum().item())
    only2 = popc(b2 & ~b3)
    only3 = popc(b3 & ~b2)
    both = popc(b2 & b3)
    res3 = site_cov(bm3, cand)
    cov3_r3, n3 = coverage(res3)
    cov2_r3 = union_cov(bm3, cand, ch2)
    out_q = {}
    for q in (10, 50, 200):
        zq = (torch.round(zs.float() / q) * q).clamp(-32768, 32767).to(torch.int16)
        gq = V.Grid(zq, w.W)
        pq = Pipeline(V, w, gq, dev)
        pq.step()
        torch.cuda.synchronize()
        chq, gnq, _, nq = pq.result
        chq = chq[:int(nq.item())]
        # exact coverage on the true terrain of the observers sited on the rounded one
        bq3, _ = V.viewshed_r3(g, w.R, w.ht, w.hr, chq.contiguous())
        cum = torch.zeros_like(pipe.cum)
        resq = V.site(bq3, chq.contiguous(), w.H, w.W, w.R, int(chq.numel()), cum=cum, ws=pipe.ws, sync=False)
        out_q[str(q)] = {"observers": int(chq.numel()), "exact_coverage_posts": coverage(resq)[0],
                         "vs_true_terrain_R2_sited": coverage(resq)[0] / max(cov2_r3, 1)}
        del pq, gq, zq, bq3
    out = {"metric": "accuracy study (R2 vs exact R3 viewsheds; rounded elevations)", "workload": w.name,
           "config": {"H": w.H, "W": w.W, "R": w.R, "ht": w.ht, "hr": w.hr, "candidates": int(cand.numel()),
                      "n_obs": w.n_obs},
           "cells": {"R2_and_R3": both, "R2_only": only2, "R3_only": only3,
                     "disagree_frac": (only2 + only3) / max(both + only2 + only3, 1)},
           "coverage": {"R2_sited_R2_counted": cov2_r2, "R2_sited_exact": cov2_r3, "R3_sited_exact": cov3_r3,
                        "R2_sited_vs_R3_sited_exact": cov2_r3 / max(cov3_r3, 1),
                        "observers_R2": int(ch2.numel()), "observers_R3": n3},
           "rounded_terrain": out_q, "r3_viewsheds_ms": r3_ms,
           "r3_viewsheds_per_s": cand.numel() / (r3_ms * 1e-3), "wall_s": time.perf_counter() - t0}
    if rank == 0:
        print(json.dumps(out, default=str))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="full",
                    choices=["full", "mid", "scale", "small", "batch", "learn", "paper", "paper_mid",
                             "paper_small", "paper_r2000", "accuracy"])
    ap.add_argument("--paper-surrogate", action="store_true",
                    help="--workload paper*: also run the learned proposal trained on exact R-vix labels")
    ap.add_argument("--paper-patch-step", type=int, default=30,
                    help="post spacing of the CNN patch in the paper regime (65 posts 30 apart span ~2R)")
    ap.add_argument("--paper-block", type=int, default=0,
                    help="findmax block of the paper-regime proposal (0 = the workload's)")
    ap.add_argument("--paper-k", type=int, default=0, help="candidates per block of that proposal (0 = the workload's)")
    ap.add_argument("--paper-stride", default="64",
                    help="lattice stride(s) of the paper-regime proposal, comma-separated")
    ap.add_argument("--accuracy-size", default="full", choices=["full", "mid"],
                    help="terrain of --workload accuracy: the headline recipe at 46400^2 or 11600^2")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--sur-stride", type=int, default=0,
                    help="proposal lattice stride; 0 = tuned on another terrain of the recipe")
    ap.add_argument("--patch-step", type=int, default=3,
                    help="post spacing inside the CNN's 65x65 input patch")
    ap.add_argument("--train-posts", type=int, default=None,
                    help="training posts (default 4000000; 500000 for the paper-regime proposal)")
    ap.add_argument("--epochs", type=int, default=None, help="default 6; 3 for the paper-regime proposal")
    args = ap.parse_args()
    paper = args.workload.startswith("paper")
    if args.train_posts is None:
        args.train_posts = 500000 if paper else 4000000
    if args.epochs is None:
        args.epochs = 3 if paper else 6
    dist, rank, world, local = dist_init()
    if args.workload == "batch":
        run_batch(args, dist, rank, world, local)
        return
    if args.workload == "learn":
        run_learn(args, rank, local)
        return
    if args.workload == "accuracy":
        if args.impl == "reference":
            if rank == 0:
                print(json.dumps({"impl": "reference", "unavailable": "the accuracy study has no oracle arm"}))
            return
        run_accuracy(args, dist, rank, world, local)
        return
    if args.workload in ("paper", "paper_mid", "paper_small", "paper_r2000"):
        if args.impl == "reference":
            if rank == 0:
                print(json.dumps({"impl": "reference", "unavailable": "the paper-regime workload has no bounded "
                                  "oracle sample; the oracle arm times the headline workload"}))
            return
        run_paper(args, dist, rank, world, local)
        return
    w = pick_workload(args.workload)
    if args.impl == "reference":
        run_reference(args, w, rank)
        if dist:
            dist.barrier()
        return

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2006_16783_gb300 as V

    # ---- inputs: terrain resident in HBM (larger than L2)
    t = time.perf_counter()
    z_dev = w.make_terrain(dev)
    zs, pitch = WL.terrain.pad_pitch(z_dev, 8)
    del z_dev
    g = V.Grid(zs, w.W)
    gen_s = time.perf_counter() - t
    plain = Pipeline(V, w, g, dev)
    plain.names = ["vix", "findmax", "viewshed", "site"]

    # work accounting for the roofline (untimed): LOS crossings of one vix pass
    steps_ctr = torch.zeros(1, dtype=torch.int64, device=dev)
    V.vix_count(g, w.R, w.ht, w.hr, w.S, w.vix_seed, steps_ctr, out=plain.vixbuf)
    los_steps = int(steps_ctr.item())
    for _ in range(args.warmup):
        plain.step()
    torch.cuda.synchronize()
    cov_plain, nobs_plain = coverage(plain.result)

    sur = None
    if not args.no_surrogate:
        sur = SurrogatePipeline(V, w, g, plain, args, dev)
        for _ in range(args.warmup):
            sur.step()
        torch.cuda.synchronize()
    cov_sur = coverage(sur.result)[0] if sur else 0
    head = sur if (sur and cov_sur >= 0.99 * cov_plain) else plain
    other = plain if head is sur else sur

    # ---- timed region: K steps of the headline pipeline, clocks sampled
    clocks = ClockSampler(local)
    clocks.start()
    n_launch0 = V.launch_count()
    ms, st = time_steps(head, args.steps, dist, dev)
    n_launch = V.launch_count() - n_launch0   # the library's kernels in the timed region
    clk = clocks.stop()
    n_launch1 = V.launch_count()
    o_ms, o_st = time_steps(other, args.steps, dist, dev) if other else (None, None)
    o_launch = V.launch_count() - n_launch1
    p_ms, p_st = (ms, st) if head is plain else (o_ms, o_st)
    s_ms, s_st = ((ms, st) if head is sur else (o_ms, o_st)) if sur else (None, None)

    # ---- dense gain pass on its own (HBM roofline of the site step)
    zero = torch.zeros_like(plain.cum)
    gbuf = torch.empty(plain.n, dtype=torch.int32, device=dev)
    for _ in range(3):
        V.site_gains(plain.bm, plain.cand, w.H, w.W, w.R, zero, out=gbuf)
    ga, gb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ga.record()
    for _ in range(5):
        V.site_gains(plain.bm, plain.cand, w.H, w.W, w.R, zero, out=gbuf)
    gb.record()
    torch.cuda.synchronize()
    gains_ms = ga.elapsed_time(gb) / 5
    cand_h = plain.cand.cpu().numpy()
    cyh, cxh = cand_h // w.W, cand_h % w.W
    PR = V.words_per_row(w.R)
    rows_in = np.minimum(cyh + w.R, w.H - 1) - np.maximum(cyh - w.R, 0) + 1
    gw0 = np.floor_divide(cxh - w.R, 32)
    WWc = (w.W + 31) // 32
    words_in = np.minimum(gw0 + PR - 1, WWc - 1) - np.maximum(gw0, 0) + 1
    # algorithmic bytes of the dense pass: every bitmap, the cumulative
    # viewshed under the union of the candidates' windows (each word read
    # once), and 8 bytes of key per candidate
    cover = np.zeros((w.H, WWc), bool)
    for y_, x_ in zip(cyh, cxh):
        g0 = (int(x_) - w.R) // 32
        cover[max(0, int(y_) - w.R):min(w.H, int(y_) + w.R + 1), max(0, g0):min(WWc, g0 + PR)] = True
    union_words = int(cover.sum())
    del cover
    gain_bytes = plain.n * (2 * w.R + 1) * PR * 4 + union_words * 4 + plain.n * 8

    # ---- e2e: the headline pipeline through the same C-ABI calls on a terrain
    # copied in from pinned host memory every step, results copied back
    e2e = None
    if not args.no_e2e:
        zh = torch.empty_like(zs, device="cpu").pin_memory()
        zh.copy_(zs)
        out_ch = torch.empty(w.n_obs, dtype=torch.int64).pin_memory()
        out_gn = torch.empty(w.n_obs, dtype=torch.int64).pin_memory()
        out_n = torch.empty(1, dtype=torch.int32).pin_memory()
        zs2 = torch.empty_like(zs)
        g2 = V.Grid(zs2, w.W)
        for _ in range(2):
            head.step(g=g2, host=zh)
        torch.cuda.synchronize()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
        walls = []
        for i in range(args.steps):
            t0 = time.perf_counter()
            evs[i][0].record()
            head.step(g=g2, host=zh)  # the terrain's copy-in is part of the step
            evs[i][1].record()
            c2, g2_, _, n2 = head.result
            out_ch.copy_(c2[:w.n_obs], non_blocking=True)
            out_gn.copy_(g2_[:w.n_obs], non_blocking=True)
            out_n.copy_(n2, non_blocking=True)
            evs[i][2].record()
            torch.cuda.synchronize()
            walls.append(time.perf_counter() - t0)
        e2e_s = statistics.median(walls)  # wall clock of one synchronised step
        parts = [statistics.median(e[j].elapsed_time(e[j + 1]) for e in evs) for j in range(2)]
        e2e = {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": zs.numel() * 2,
               "d2h_bytes_per_step": w.n_obs * 16 + 4,
               "parts_ms": {"h2d_and_pipeline": parts[0], "d2h": parts[1]},
               "h2d": ("terrain streamed in row bands on a side stream while the lattice is scored"
                       if head is sur else "terrain copied before the pipeline")}
        del zs2, g2

    # ---- rooflines
    peaks, peak_src = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    issue_peak = sms * 4 * 32 * mhz * 1e6 / 1e9            # G thread-instr / s
    # vix and viewshed: thread instructions issued per work unit counted by
    # ncu on the mid workload (the current kernel sources), times this run's
    # units, over the live stage time, against the issue peak; beside it the
    # same rate for a minimal instruction sequence (OPS_PER_*)
    cnt = recorded_counters()

    def issue_roof(key, units, t_ms, min_ops):
        r = {"bound": "alu", "peak": issue_peak, "unit": "Gop/s", "units": units,
             "min_inst_per_unit": min_ops,
             "algorithmic_frac": units * min_ops / (t_ms * 1e-3) / 1e9 / issue_peak}
        c = cnt.get(key)
        if c:
            r["inst_per_unit"] = c["thread_inst_per_unit"]
            r["achieved"] = units * c["thread_inst_per_unit"] / (t_ms * 1e-3) / 1e9
            r["issue_active_mid_pct"] = c["issue_active_pct"]
            r["traffic"] = units * c["dram_bytes_per_unit"]
            r["traffic_source"] = "ncu on the mid workload, scaled by units"
        else:  # the kernel changed since the capture: the minimal sequence only
            r["achieved"] = units * min_ops / (t_ms * 1e-3) / 1e9
            r["traffic"] = None
        return r

    roof = {
        "vix": issue_roof("vix", los_steps, p_st[0], OPS_PER_LOS_STEP),
        "viewshed": issue_roof("viewshed", plain.n * interior_ray_steps(w.R), p_st[2], OPS_PER_RAY_STEP),
        "site_gains": {"bound": "hbm", "achieved": gain_bytes / (gains_ms * 1e-3) / 1e9,
                       "peak": peaks["hbm_gbs"], "unit": "GB/s", "bytes": gain_bytes,
                       "traffic": (plain.n * cnt["site_gains"]["dram_bytes_per_unit"]) if "site_gains" in cnt else None},
        "findmax": {"bound": "hbm", "achieved": (w.H * w.W + plain.n * 8) / (p_st[1] * 1e-3) / 1e9,
                    "peak": peaks["hbm_gbs"], "unit": "GB/s", "traffic": None},
    }
    # the greedy loop of the headline pipeline: bytes per step (window V + C
    # read + C write, and the refresh's overlap words) over the site stage time
    hres = head.result
    nsel = int(hres[3].item())
    loop_bytes = site_loop_bytes(head.cand.cpu().numpy(), hres[0][:nsel].cpu().numpy(), w.W, w.R,
                                 V.words_per_row(w.R))
    roof["site_loop"] = {"bound": "hbm", "achieved": loop_bytes / (st[3] * 1e-3) / 1e9,
                         "peak": peaks["hbm_gbs"], "unit": "GB/s", "traffic": None,
                         "note": "sequential greedy (one CTA or a leader cluster): bound by the "
                                 "latency of its dependent memory rounds and barriers, not by bandwidth"}
    if sur:
        flops = sur.score.numel() * cnn_flops_per_patch()
        roof["cnn_lattice"] = {"bound": "tensor", "achieved": flops / (s_st[0] * 1e-3) / 1e12,
                               "peak": peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]),
                               "unit": "TFLOP/s", "traffic": None}
        c = cnt.get("cnn_forward")
        # DRAM bytes per patch from a capture with the same lattice stride and
        # patch step (the windows of neighbouring patches overlap in L2)
        if c and c.get("stride") == sur.stride and c.get("patch_step") == sur.tr.patch_step:
            roof["cnn_lattice"]["traffic"] = sur.score.numel() * c["dram_bytes_per_unit"]
            roof["cnn_lattice"]["traffic_source"] = "ncu on %s, scaled by patches" % c["workload"]
    for r in roof.values():
        r["frac"] = r["achieved"] / r["peak"]
    stage_roof = {"vix": "vix", "findmax": "findmax", "viewshed": "viewshed", "site": "site_loop",
                  "cnn_lattice": "cnn_lattice", "findmax_f32": "findmax", }
    dom = head.names[int(np.argmax(st))]
    dom_roof = dict(roof[stage_roof[dom]])
    dom_roof["kernel"] = dom

    plain_obj = {"s_per_step": p_ms / 1000.0, "stages_ms": dict(zip(plain.names, p_st)),
                 "coverage_posts": cov_plain, "observers": nobs_plain, "candidates": plain.n,
                 "viewsheds_per_s": plain.n / (p_st[2] * 1e-3), "vix_los_steps": los_steps,
                 "gpu_launches_per_step": (n_launch if head is plain else o_launch) / args.steps}
    out = {
        "metric": METRIC, "value": ms / 1000.0, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32+bf16" if head is sur else "int32",
        "data": "synthetic",
        "config": {"workload": w.name, "H": w.H, "W": w.W, "R": w.R, "ht": w.ht, "hr": w.hr,
                   "S": w.S, "block": w.block, "k": w.k, "n_obs": w.n_obs, "candidates": plain.n,
                   "pipeline": ("surrogate (CNN on a stride-%d lattice, findmax, viewshed, site)" % sur.stride
                                if head is sur else "plain (vix, findmax, viewshed, site)"),
                   "l2": "inputs larger than L2 (%.1f GB terrain, %.0f MB bitmaps)" % (
                       zs.numel() * 2 / 1e9, plain.bm.numel() * 4 / 1e6),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "viewsheds_per_s": plain.n / (st[2] * 1e-3),
        "stages_ms": dict(zip(head.names, st)),
        "coverage_posts": cov_sur if head is sur else cov_plain,
        "coverage_frac": (cov_sur if head is sur else cov_plain) / (w.H * w.W),
        "plain": plain_obj,
        "site_gains_ms": gains_ms,
        "roofline": dom_roof, "rooflines": roof, "peak_source": peak_src,
        "clocks": clk, "gpu_launches": n_launch, "terrain_gen_s": gen_s,
    }
    if sur:
        out["surrogate"] = {
            "s_per_step": s_ms / 1000.0, "stages_ms": dict(zip(sur.names, s_st)),
            "coverage_posts": cov_sur, "coverage_ratio_vs_plain": cov_sur / max(cov_plain, 1),
            "speedup_vs_plain": p_ms / s_ms, "lattice_stride": sur.stride, "stride_tuning": sur.tuning,
            "candidates": sur.n,
            "patch_step": sur.tr.patch_step,
            "patches_per_step": sur.score.numel(), "train_posts": args.train_posts, "epochs": args.epochs,
            "train_loss_last_epoch": sur.train_loss, "label_s": sur.label_s, "train_s": sur.train_s,
            "train_patches_per_s": args.train_posts * args.epochs / max(sur.train_s, 1e-9),
            "mae_heldout": sur.mae, "mae_sampled_vix": sur.mae_vix, "mae_posts": sur.mae_posts,
            "gpu_launches_per_step": (n_launch if head is sur else o_launch) / args.steps}
    if e2e:
        out["e2e"] = e2e
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        zh_np = zs[:, :w.W].cpu().numpy() if pitch != w.W else zs.cpu().numpy()
        v, desc, threads, v1 = oracle_sample(zh_np, w, cand=head.cand.cpu().numpy())
        if head is sur:
            # the surrogate pipeline's oracle: numpy CNN per lattice patch instead of vix
            per_patch = cnn_oracle_sample(zh_np, w, sur.stride, args.patch_step)
            t_vix = float(desc.split("(vix ")[1].split(" s")[0])
            t_vix1 = float(desc.split("1 thread: vix ")[1].split(" s")[0])
            v = v - t_vix + per_patch * sur.score.numel()
            v1 = v1 - t_vix1 + per_patch * sur.score.numel()
            desc += ("; surrogate pipeline: vix replaced by the numpy CNN oracle on %d lattice patches "
                     "(%.2f ms per patch on one thread, 24 patches timed; one thread in both figures)"
                     % (sur.score.numel(), per_patch * 1e3))
        out["cpu_baseline"] = {"value": v, "unit": "s", "cores": threads, "kind": "oracle", "sample": desc,
                               "single_thread_value": v1}
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
