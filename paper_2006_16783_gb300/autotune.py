"""Project autotuner: times the candidate launch shapes of the viewshed
(threads per CTA, i.e. rays walked at once per candidate) and of vix (post
tile) for each ROI on a representative terrain, with CUDA events, and stores
the fastest in the library's tuning table (vs_tune_set).  Results of every
call are independent of the chosen shapes; only their speed changes."""
import torch

from . import vshed as V


def _time(fn, reps=3):
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def tune_viewshed(g, R, ht, hr, n=2000, seed=0, choices=(128, 256, 512)):
    gen = torch.Generator(device="cpu").manual_seed(seed)
    cand = (torch.randint(0, g.H, (n,), generator=gen) * g.W + torch.randint(0, g.W, (n,), generator=gen)).to(
        g.storage.device)
    bm = torch.empty((n, 2 * R + 1, V.words_per_row(R)), dtype=torch.int32, device=g.storage.device)
    area = torch.empty(n, dtype=torch.int32, device=g.storage.device)
    times = {}
    for t in choices:
        V.tune_set(V.VS_TUNE_VIEWSHED_THREADS, R, t)
        times[t] = _time(lambda: V.viewshed(g, R, ht, hr, cand, bm=bm, area=area))
    best = min(times, key=times.get)
    V.tune_set(V.VS_TUNE_VIEWSHED_THREADS, R, best)
    return best, times


def tune_vix(g, R, ht, hr, S, seed=1, choices=(1, 2)):
    out = torch.empty((g.H, g.W), dtype=torch.uint8, device=g.storage.device)
    times = {}
    for t in choices:
        V.tune_set(V.VS_TUNE_VIX_TILE, R, t)
        times[t] = _time(lambda: V.vix(g, R, ht, hr, S, seed, out=out), reps=2)
    best = min(times, key=times.get)
    V.tune_set(V.VS_TUNE_VIX_TILE, R, best)
    return best, times


def tune_all(g, radii, ht=10, hr=10, S=10, log=None):
    table = {}
    for R in sorted(set(radii)):
        bv, tv = tune_viewshed(g, R, ht, hr)
        bx, tx = tune_vix(g, R, ht, hr, S)
        table[R] = {"viewshed_threads": bv, "viewshed_ms": tv, "vix_tile": bx, "vix_ms": tx}
        if log:
            log("R=%d: viewshed threads %d %s, vix tile %d %s" % (R, bv, tv, bx, tx))
    return table
