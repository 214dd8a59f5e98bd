#!/usr/bin/env python
"""Benchmark of the observer-siting hot path on one GB300.

One step = the whole plain pipeline on the resident 46400^2 terrain:
vix (S=10 LOS per post) -> findmax (top-4 per 464^2 block, 40000 candidates)
-> viewshed (R=100) -> site (4096 observers).  Prints ONE JSON line.

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
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""
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
                                          "--format=csv,noheader,nounits", "-lms", "200"],
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
    return {"full": WL.FULL, "scale": WL.SCALE, "small": WL.SMALL}[name]


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

    def step(self, record=False):
        V, w = self.V, self.w
        ev = self.ev
        if record:
            ev[0].record()
        V.vix(self.g, w.R, w.ht, w.hr, w.S, w.vix_seed, out=self.vixbuf)
        if record:
            ev[1].record()
        V.findmax(self.vixbuf, w.block, w.k, out=self.cand)
        if record:
            ev[2].record()
        V.viewshed(self.g, w.R, w.ht, w.hr, self.cand, bm=self.bm, area=self.area)
        if record:
            ev[3].record()
        self.cum.zero_()
        self.result = V.site(self.bm, self.cand, w.H, w.W, w.R, w.n_obs, cum=self.cum, ws=self.ws, sync=False)
        if record:
            ev[4].record()

    def stage_ms(self):
        return [self.ev[i].elapsed_time(self.ev[i + 1]) for i in range(4)]


# ------------------------------------------------------------------ CPU oracle sample
def oracle_sample(z_host, w, budget_s=20.0, threads=None):
    """Time the CPU oracle on a bounded sample of the workload and extrapolate
    linearly to the whole workload.  Returns (seconds, description, threads)."""
    from oracle import oracle as O
    threads = threads or os.cpu_count() or 1
    H, W = w.H, w.W
    rng = np.random.default_rng(12345)
    # vix: a square tile of posts in the middle of the terrain
    side = 512 if H * W > 4e6 else min(H, W)
    y0, x0 = (H - side) // 2, (W - side) // 2
    posts = ((np.arange(y0, y0 + side)[:, None] * W) + np.arange(x0, x0 + side)[None, :]).ravel()
    chunks = np.array_split(posts, threads)
    t = time.perf_counter()
    ths = [threading.Thread(target=O.vix_posts, args=(z_host, w.R, w.ht, w.hr, w.S, w.vix_seed, c, W))
           for c in chunks]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    t_vix = (time.perf_counter() - t) * (H * W) / len(posts)
    # viewsheds of seeded interior candidates
    nv = 400
    cy = rng.integers(w.R, H - w.R, nv)
    cx = rng.integers(w.R, W - w.R, nv)
    cand = (cy * W + cx).astype(np.int64)
    t = time.perf_counter()
    bm, area = O.viewshed(z_host, w.R, w.ht, w.hr, cand, threads=threads)
    n_full = WL.FULL.n_candidates() if w is WL.FULL else w.n_candidates()
    t_vs = (time.perf_counter() - t) * n_full / nv
    # site: heap set-up and per-step cost on the sample, scaled to the workload
    t = time.perf_counter()
    O.site(bm, cand, H, W, w.R, 1)
    t0 = time.perf_counter() - t
    t = time.perf_counter()
    ch, gn, C = O.site(bm, cand, H, W, w.R, 64)
    t1 = time.perf_counter() - t
    per_step = max(t1 - t0, 0.0) / max(len(ch) - 1, 1)
    t_site = t0 * n_full / nv + per_step * w.n_obs
    total = t_vix + t_vs + t_site
    desc = ("oracle on %d threads: vix of a %dx%d post tile, %d viewsheds, site of those %d candidates "
            "(1 and 64 steps); extrapolated linearly to %dx%d posts, %d candidates, %d observers "
            "(vix %.1f s, viewshed %.1f s, site %.1f s)" % (
                threads, side, side, nv, nv, H, W, n_full, w.n_obs, t_vix, t_vs, t_site))
    return total, desc, threads


# ------------------------------------------------------------------ learned proposal
def run_surrogate(V, w, g, pipe, covered_plain, args, dev):
    from paper_2006_16783_gb300 import surrogate as S
    t0 = time.perf_counter()
    # training terrain: the same recipe with another seed (the bench terrain is held out)
    wtr = WL.scaled(w, w.H, w.W, name=w.name + "_train", seed=w.seed + 7)
    ztr = wtr.make_terrain(dev)
    ztr_s, _ = WL.terrain.pad_pitch(ztr, 8)
    del ztr
    gtr = V.Grid(ztr_s, w.W)
    posts = S.sample_posts(w.H, w.W, args.train_posts, 32, 11, dev)
    labels = S.exact_vix(gtr, posts, w.R, w.ht, w.hr)
    label_s = time.perf_counter() - t0
    tr = S.Trainer(S.init_master(0), batch=512, lr=2e-3)
    t1 = time.perf_counter()
    last = tr.fit([(gtr, posts, labels)], epochs=args.epochs, seed=3,
                  log=lambda m: print(m, file=sys.stderr))
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t1
    del gtr, ztr_s, posts, labels
    # held-out error on the bench terrain, next to the 10-sample vix estimate
    pt = S.sample_posts(w.H, w.W, 200000, 32, 5, dev)
    lt = S.exact_vix(g, pt, w.R, w.ht, w.hr)
    mae = float((tr.predict(g, pt) - lt).abs().mean())
    mae_vix = float((pipe.vixbuf.reshape(-1)[pt].float() / w.S - lt).abs().mean())
    # the surrogate pipeline: lattice scores -> findmax_f32 -> viewshed -> site
    st = args.sur_stride
    n = V.findmax_count(w.H, w.W, st, w.block, w.k)
    score = torch.empty(((w.H + st - 1) // st, (w.W + st - 1) // st), dtype=torch.float32, device=dev)
    cand = torch.empty(n, dtype=torch.int64, device=dev)
    bm = pipe.bm if n == pipe.n else torch.empty((n, 2 * w.R + 1, V.words_per_row(w.R)), dtype=torch.int32,
                                                  device=dev)
    area = torch.empty(n, dtype=torch.int32, device=dev)
    cum = torch.empty_like(pipe.cum)
    ws = torch.empty(V.site_workspace(n, w.R), dtype=torch.uint8, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    res = None

    def step(record):
        nonlocal res
        if record:
            ev[0].record()
        V.cnn_score_lattice(g, st, tr.packed, out=score)
        if record:
            ev[1].record()
        V.findmax_f32(score, w.H, w.W, st, w.block, w.k, out=cand)
        if record:
            ev[2].record()
        V.viewshed(g, w.R, w.ht, w.hr, cand, bm=bm, area=area)
        if record:
            ev[3].record()
        cum.zero_()
        res = V.site(bm, cand, w.H, w.W, w.R, w.n_obs, cum=cum, ws=ws, sync=False)
        if record:
            ev[4].record()

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stages = []
    a.record()
    for _ in range(args.steps):
        step(True)
        torch.cuda.synchronize()
        stages.append([ev[i].elapsed_time(ev[i + 1]) for i in range(4)])
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / args.steps
    ch, gn, _, nch = res
    covered = int(gn[:int(nch.item())].sum().item())
    names = ["cnn_lattice", "findmax_f32", "viewshed", "site"]
    return {
        "s_per_step": ms / 1000.0,
        "stages_ms": dict(zip(names, [statistics.median(x[i] for x in stages) for i in range(4)])),
        "coverage_posts": covered, "coverage_ratio_vs_plain": covered / max(covered_plain, 1),
        "speedup_vs_plain": None, "lattice_stride": st, "candidates": n,
        "patches_per_step": score.numel(),
        "train_posts": args.train_posts, "epochs": args.epochs, "train_loss_last_epoch": last,
        "label_s": label_s, "train_s": train_s,
        "mae_heldout": mae, "mae_sampled_vix": mae_vix, "mae_posts": pt.numel(),
        "gpu_launches_per_step": 7,
    }


# ------------------------------------------------------------------ main
def run_reference(args, w, rank):
    """The oracle as it stands, on the host cores, one bounded sample per step."""
    if rank != 0:
        return
    z = w.make_terrain("cuda" if torch.cuda.is_available() else "cpu").cpu().numpy()
    for _ in range(args.warmup):
        oracle_sample(z, w)
    vals = []
    desc = threads = None
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, desc, threads = oracle_sample(z, w)
        vals.append(v)
    wall = time.perf_counter() - t0
    value = statistics.median(vals)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * wall / max(args.steps, 1),
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
           "data": "synthetic", "config": {"workload": w.name, "H": w.H, "W": w.W, "R": w.R,
                                           "ht": w.ht, "hr": w.hr, "S": w.S, "block": w.block,
                                           "k": w.k, "n_obs": w.n_obs},
           "cpu_baseline": {"value": value, "unit": "s", "cores": threads, "kind": "oracle", "sample": desc},
           "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="full", choices=["full", "scale", "small"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--sur-stride", type=int, default=16)
    ap.add_argument("--train-posts", type=int, default=500000)
    ap.add_argument("--epochs", type=int, default=3)
    args = ap.parse_args()
    w = pick_workload(args.workload)
    dist, rank, world, local = dist_init()
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

    # ---- inputs: terrain resident in HBM (larger than L2), pinned host copy for e2e
    t = time.perf_counter()
    z_dev = w.make_terrain(dev)
    zs, pitch = WL.terrain.pad_pitch(z_dev, 8)
    del z_dev
    g = V.Grid(zs, w.W)
    gen_s = time.perf_counter() - t
    pipe = Pipeline(V, w, g, dev)

    # work accounting for the roofline (untimed): LOS crossings of one vix pass
    steps_ctr = torch.zeros(1, dtype=torch.int64, device=dev)
    V.vix_count(g, w.R, w.ht, w.hr, w.S, w.vix_seed, steps_ctr, out=pipe.vixbuf)
    los_steps = int(steps_ctr.item())

    for _ in range(args.warmup):
        pipe.step()
    torch.cuda.synchronize()

    # ---- timed region: K steps on resident inputs
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stage = []
    e0.record()
    for _ in range(args.steps):
        pipe.step(record=True)
        torch.cuda.synchronize()
        stage.append(pipe.stage_ms())
    e1.record()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    if dist:
        tt = torch.tensor([ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    st = [statistics.median(s[i] for s in stage) for i in range(4)]
    chosen, gains, cum, nch = pipe.result
    n_chosen = int(nch.item())
    covered = int(gains[:n_chosen].sum().item())

    # ---- dense gain pass on its own (HBM roofline of the site step)
    zero = torch.zeros_like(pipe.cum)
    gbuf = torch.empty(pipe.n, dtype=torch.int32, device=dev)
    for _ in range(3):
        V.site_gains(pipe.bm, pipe.cand, w.H, w.W, w.R, zero, out=gbuf)
    ga, gb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ga.record()
    for _ in range(5):
        V.site_gains(pipe.bm, pipe.cand, w.H, w.W, w.R, zero, out=gbuf)
    gb.record()
    torch.cuda.synchronize()
    gains_ms = ga.elapsed_time(gb) / 5
    cand_h = pipe.cand.cpu().numpy()
    cyh, cxh = cand_h // w.W, cand_h % w.W
    PR = V.words_per_row(w.R)
    rows_in = np.minimum(cyh + w.R, w.H - 1) - np.maximum(cyh - w.R, 0) + 1
    gw0 = np.floor_divide(cxh - w.R, 32)
    WWc = (w.W + 31) // 32
    words_in = np.minimum(gw0 + PR - 1, WWc - 1) - np.maximum(gw0, 0) + 1
    gain_bytes = pipe.n * (2 * w.R + 1) * PR * 4 + int((rows_in * words_in).sum()) * 4 + pipe.n * 4

    # ---- e2e: host buffers through the same C-ABI calls, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        zh = torch.empty_like(zs, device="cpu").pin_memory()
        zh.copy_(zs)
        out_ch = torch.empty(w.n_obs, dtype=torch.int64).pin_memory()
        out_gn = torch.empty(w.n_obs, dtype=torch.int64).pin_memory()
        out_n = torch.empty(1, dtype=torch.int32).pin_memory()
        zs2 = torch.empty_like(zs)
        g2 = V.Grid(zs2, w.W)
        pipe2 = Pipeline(V, w, g2, dev)
        pipe2.vixbuf, pipe2.cand, pipe2.bm, pipe2.area, pipe2.cum, pipe2.ws = (
            pipe.vixbuf, pipe.cand, pipe.bm, pipe.area, pipe.cum, pipe.ws)
        for _ in range(1):
            zs2.copy_(zh, non_blocking=True)
            pipe2.step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            zs2.copy_(zh, non_blocking=True)
            pipe2.step()
            c2, g2_, _, n2 = pipe2.result
            out_ch.copy_(c2[:w.n_obs], non_blocking=True)
            out_gn.copy_(g2_[:w.n_obs], non_blocking=True)
            out_n.copy_(n2, non_blocking=True)
            torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / args.steps
        e2e = {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": zs.numel() * 2,
               "d2h_bytes_per_step": w.n_obs * 16 + 4}
        del zs2, pipe2

    # ---- learned proposal: train on another terrain of the same recipe, then
    # site with the network's lattice scores in place of the sampled vix
    sur = None
    if not args.no_surrogate:
        sur = run_surrogate(V, w, g, pipe, covered, args, dev)

    # ---- rooflines
    peaks, peak_src = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    issue_peak = sms * 4 * 32 * mhz * 1e6 / 1e9            # G thread-instr / s
    vix_ops = los_steps * OPS_PER_LOS_STEP
    vs_ops = pipe.n * interior_ray_steps(w.R) * OPS_PER_RAY_STEP
    roof = {
        "vix": {"bound": "alu", "achieved": vix_ops / (st[0] * 1e-3) / 1e9, "peak": issue_peak,
                "unit": "Gop/s", "traffic": None},
        "viewshed": {"bound": "alu", "achieved": vs_ops / (st[2] * 1e-3) / 1e9, "peak": issue_peak,
                     "unit": "Gop/s", "traffic": None},
        "site_gains": {"bound": "hbm", "achieved": gain_bytes / (gains_ms * 1e-3) / 1e9,
                       "peak": peaks["hbm_gbs"], "unit": "GB/s", "traffic": None},
        "findmax": {"bound": "hbm", "achieved": (w.H * w.W + pipe.n * 8) / (st[1] * 1e-3) / 1e9,
                    "peak": peaks["hbm_gbs"], "unit": "GB/s", "traffic": None},
    }
    for r in roof.values():
        r["frac"] = r["achieved"] / r["peak"]
    names = ["vix", "findmax", "viewshed", "site"]
    dom = names[int(np.argmax(st))]
    dom_roof = dict(roof.get(dom, roof["vix"]))
    dom_roof["kernel"] = dom

    out = {
        "metric": METRIC, "value": ms / 1000.0, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": w.name, "H": w.H, "W": w.W, "R": w.R, "ht": w.ht, "hr": w.hr,
                   "S": w.S, "block": w.block, "k": w.k, "n_obs": w.n_obs, "candidates": pipe.n,
                   "pipeline": "plain (vix, findmax, viewshed, site)",
                   "l2": "inputs larger than L2 (%.1f GB terrain, %.0f MB bitmaps)" % (
                       zs.numel() * 2 / 1e9, pipe.bm.numel() * 4 / 1e6),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "viewsheds_per_s": pipe.n / (st[2] * 1e-3),
        "stages_ms": dict(zip(names, st)),
        "observers": n_chosen, "coverage_posts": covered, "coverage_frac": covered / (w.H * w.W),
        "vix_los_steps": los_steps, "site_gains_ms": gains_ms,
        "roofline": dom_roof, "rooflines": roof, "peak_source": peak_src,
        "clocks": clk, "gpu_launches": 7 * args.steps, "terrain_gen_s": gen_s,
    }
    if sur:
        sur["speedup_vs_plain"] = (ms / 1000.0) / sur["s_per_step"]
        out["surrogate"] = sur
    if e2e:
        out["e2e"] = e2e
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, desc, threads = oracle_sample(zs[:, :w.W].cpu().numpy() if pitch != w.W else zs.cpu().numpy(), w)
        out["cpu_baseline"] = {"value": v, "unit": "s", "cores": threads, "kind": "oracle", "sample": desc}
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
