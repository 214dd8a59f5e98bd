"""Many terrains sited together in a constant number of launches, whatever
the number of terrains: every terrain's vix in one persistent launch
(vs_vix_batch), every findmax in one launch (vs_findmax_batch), every
viewshed in one persistent launch (vs_viewshed_batch), every greedy problem's
preparation in six launches and every greedy loop in one (vs_site_batch), the
cumulative viewsheds zeroed by one fill; the whole sequence captured once in a
CUDA graph and replayed.  Launch shapes come from the autotuner (autotune.py)."""
import torch

from . import vshed as V


class BatchedSiting:
    """instances: list of dicts with keys grid (vshed.Grid), R, ht, hr, S,
    seed, block, k, n_obs.  Buffers are allocated once; run() enqueues one
    whole siting of every instance on the current stream."""

    def __init__(self, instances, device="cuda"):
        self.inst = instances
        dev = torch.device(device)
        self.vs_jobs, self.site_jobs_, self.bufs = [], [], []
        self.vix_jobs, self.fm_jobs = [], []
        # every terrain's cumulative viewshed in one buffer (zeroed by one fill)
        sizes = [it["grid"].H * ((it["grid"].W + 31) // 32) for it in instances]
        self.cum_all = torch.zeros(max(sum(sizes), 1), dtype=torch.int32, device=dev)
        offs = [sum(sizes[:i]) for i in range(len(sizes))]
        for it, o, sz in zip(instances, offs, sizes):
            g, R = it["grid"], it["R"]
            n = V.findmax_count(g.H, g.W, 1, it["block"], it["k"])
            b = {
                "vix": torch.empty((g.H, g.W), dtype=torch.uint8, device=dev),
                "cand": torch.empty(n, dtype=torch.int64, device=dev),
                "bm": torch.empty((n, 2 * R + 1, V.words_per_row(R)), dtype=torch.int32, device=dev),
                "area": torch.empty(n, dtype=torch.int32, device=dev),
                "cum": self.cum_all[o:o + sz].view(g.H, (g.W + 31) // 32),
                "chosen": torch.empty(max(it["n_obs"], 1), dtype=torch.int64, device=dev),
                "gains": torch.empty(max(it["n_obs"], 1), dtype=torch.int64, device=dev),
                "n_chosen": torch.zeros(1, dtype=torch.int32, device=dev),
            }
            self.bufs.append(b)
            self.vix_jobs.append({"g": g, "R": R, "ht": it["ht"], "hr": it["hr"], "S": it["S"], "seed": it["seed"],
                                  "out": b["vix"]})
            self.fm_jobs.append({"vix": b["vix"], "block": it["block"], "k": it["k"], "out": b["cand"]})
            self.vs_jobs.append({"g": g, "R": R, "ht": it["ht"], "hr": it["hr"], "cand": b["cand"],
                                 "bm": b["bm"], "area": b["area"]})
            self.site_jobs_.append({"bm": b["bm"], "cand": b["cand"], "H": g.H, "W": g.W, "R": R,
                                    "n_obs": it["n_obs"], "chosen": b["chosen"], "gains": b["gains"],
                                    "cum": b["cum"], "n_chosen": b["n_chosen"]})
        self.vs_ws = torch.empty(max(V.lib().vs_viewshed_batch_workspace(len(instances)), 256),
                                 dtype=torch.uint8, device=dev)
        self.vix_ws = torch.empty(max(V.lib().vs_vix_batch_workspace(len(instances)), 256),
                                  dtype=torch.uint8, device=dev)
        self.site_ws = torch.empty(max(V.site_batch_workspace(self.site_jobs_), 256), dtype=torch.uint8,
                                   device=dev)
        self.graph = None

    def run(self):
        V.vix_batch(self.vix_jobs, self.vix_ws)
        V.findmax_batch(self.fm_jobs)
        V.viewshed_batch(self.vs_jobs, self.vs_ws)
        self.cum_all.zero_()
        V.site_batch(self.site_jobs_, self.site_ws)

    def capture(self):
        """Record run() once into a CUDA graph (after one eager warm-up run)."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.run()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.run()
        return self.graph

    def replay(self):
        self.graph.replay()

    def results(self):
        out = []
        for b in self.bufs:
            t = int(b["n_chosen"].item())
            out.append((b["chosen"][:t], b["gains"][:t], b["cum"]))
        return out
