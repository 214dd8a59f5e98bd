"""The five synthetic workloads, each shaped like a run of the paper
(Sec. "Testing": DEM1000, US East, US West) with seeded fBm terrain standing in
for the unavailable datasets.  Parameters only -- no siting arithmetic.

    small   1000^2 spectral fBm (Hurst 0.8, 0..1000 m), R=50, h=10, S=10,
            top-1 per 25x25 block (1600 candidates), 100 observers
    scale   16384^2 spectral fBm (Hurst 0.75, 0..3000 m, lowest 10% flattened
            to 0), R=200, h=10, S=20, top-2 per 256x256 block (8192
            candidates), 2048 observers
    batch   64 instances: side U{512..4096}, Hurst 0.8, 0..1000*U{1..3} m,
            R in {50,100,150,250}, h in U{5..30}, n_obs in U{16..512}, S=10,
            block ceil(R/2), k=1
    learn   eight 4096^2 training terrains (seeds 3000..3007), a held-out
            16384^2 terrain (seed 3100), labels = exact vix at R=100
    full    46400^2 ridged multifractal (base wavelength 640 posts, 10 octaves,
            0..4000 m, lowest 5% flattened), R=100, h=10, S=10, top-4 per
            464x464 block (40000 candidates), 4096 observers
    paper   the paper's own US-West regime on the full recipe's terrain:
            46400^2, R=1000, h_t=100, h_r=10, S=10, top-20 per 334x334 block
            (386,420 candidates), greedy until 95% coverage
"""
import math
from dataclasses import dataclass, field

import numpy as np

from . import terrain


@dataclass
class Workload:
    name: str
    H: int
    W: int
    R: int
    ht: int
    hr: int
    S: int
    block: int
    k: int
    n_obs: int
    seed: int
    kind: str = "fbm"          # "fbm" or "ridged"
    hurst: float = 0.8
    zmax: int = 1000
    lake_frac: float = 0.0
    vix_seed: int = 0x5EED
    target: float = 0.0        # coverage stop of the site step (0 = off)
    extra: dict = field(default_factory=dict)

    def make_terrain(self, device="cpu"):
        """int16 (H, W) tensor on ``device``."""
        if self.kind == "ridged":
            return terrain.ridged_multifractal(self.H, self.W, self.seed, 0, self.zmax, self.lake_frac,
                                               device=device, **self.extra)
        return terrain.spectral_fbm(self.H, self.W, self.hurst, self.seed, 0, self.zmax,
                                    self.lake_frac, device=device)

    def n_candidates(self):
        nby, nbx = math.ceil(self.H / self.block), math.ceil(self.W / self.block)
        return nby * nbx * self.k  # exact when every block holds >= k posts


SMALL = Workload("small_1000sq_R50", 1000, 1000, 50, 10, 10, 10, 25, 1, 100, seed=1000,
                 hurst=0.8, zmax=1000)
SCALE = Workload("scale_16384sq_R200", 16384, 16384, 200, 10, 10, 20, 256, 2, 2048, seed=1001,
                 hurst=0.75, zmax=3000, lake_frac=0.10)
# base wavelength 640 posts, 10 octaves: relief at the ROI scale like mountainous
# 1-arc-second terrain (mean |dz| between neighbouring posts ~8 m, exact vix at
# R = 100 spread over [0, 1]); a wavelength near the grid size would make the
# terrain almost planar within any ROI
FULL = Workload("full_46400sq_R100", 46400, 46400, 100, 10, 10, 10, 464, 4, 4096, seed=1004,
                kind="ridged", zmax=4000, lake_frac=0.05,
                extra={"octaves": 10, "base_wavelength": 640})


# the full recipe on 1/16 of the area (11600^2, 2500 candidates): a size for
# profiler captures that keeps the terrain larger than L2
MID = Workload("mid_11600sq_R100", 11600, 11600, 100, 10, 10, 10, 464, 4, 1024, seed=1004,
               kind="ridged", zmax=4000, lake_frac=0.05,
               extra={"octaves": 10, "base_wavelength": 640})


# The paper's own US-West run (Sec. "Experiments", Table of the US-West
# dataset, first column): 46400^2 posts, R = 1000, h_t = 100, h_r = 10, the
# terrain cut into 139 x 139 blocks (side 334, about R/3) with 20 candidates
# each (386,420), greedy siting until 95% of the terrain is covered.  The full
# recipe's ridged terrain stands in for NASADEM US West.  Bitmaps: 386,420 x
# 2001 rows x 64 words = 198 GB.
PAPER = Workload("paper_uswest_46400sq_R1000", 46400, 46400, 1000, 100, 10, 10, 334, 20, 20000,
                 seed=1004, kind="ridged", zmax=4000, lake_frac=0.05, target=0.95,
                 extra={"octaves": 10, "base_wavelength": 640})
# the paper's second US-West column: R = 2000, 70 x 70 blocks (side 667 ~ R/3) of 20
# candidates (98,000), 95 % coverage.  Bitmaps: 98,000 x 4001 rows x 127 words = 199 GB.
PAPER_R2000 = Workload("paper_uswest_46400sq_R2000", 46400, 46400, 2000, 100, 10, 10, 667, 20, 20000,
                       seed=1004, kind="ridged", zmax=4000, lake_frac=0.05, target=0.95,
                       extra={"octaves": 10, "base_wavelength": 640})
# the same regime on 4096^2 (13 x 13 blocks, 3,380 candidates, 1.7 GB of bitmaps): a
# size for profiler captures (the terrain fits in L2; the kernels it is used for
# are bound by issue and cache latency, not DRAM)
PAPER_SMALL = Workload("paper_regime_4096sq_R1000", 4096, 4096, 1000, 100, 10, 10, 334, 20, 20000,
                       seed=1004, kind="ridged", zmax=4000, lake_frac=0.05, target=0.95,
                       extra={"octaves": 10, "base_wavelength": 640})
# the same regime on 16384^2 (49 x 50 blocks, 49,000 candidates, 25 GB of bitmaps)
PAPER_MID = Workload("paper_regime_16384sq_R1000", 16384, 16384, 1000, 100, 10, 10, 334, 20, 20000,
                     seed=1004, kind="ridged", zmax=4000, lake_frac=0.05, target=0.95,
                     extra={"octaves": 10, "base_wavelength": 640})


def batch_instances(seed=1002, count=64, max_side=4096):
    """The batched workload's 64 instances (parameters drawn from ``seed``)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        side = int(rng.integers(512, max_side + 1))
        R = int(rng.choice([50, 100, 150, 250]))
        h = int(rng.integers(5, 31))
        out.append(Workload("batch_%02d" % i, side, side, R, h, h, 10, (R + 1) // 2, 1,
                            int(rng.integers(16, 513)), seed=seed * 1000 + i, hurst=0.8,
                            zmax=1000 * int(rng.integers(1, 4))))
    return out


def scaled(w, H, W, name=None, **kw):
    """The same recipe at another size (used for parity cases the oracle can
    finish in seconds)."""
    d = dict(w.__dict__)
    d.update(kw)
    d["H"], d["W"] = H, W
    d["name"] = name or ("%s_at_%dx%d" % (w.name, H, W))
    return Workload(**d)
