"""The siting pipeline with its data split over ranks, one process per GPU
(the paper's parallel loops over posts and candidates, Sec. "Implementation",
divided between processes).

Rank r owns the contiguous block rows [y0, y1) of the grid (block rows of the
Findmax stage divided evenly, so every block lies on one rank):

- Vix: the rank computes its strip on a local grid holding rows
  [y0 - R - 1, y1 + R + 1) (every line of sight from a strip post stays
  inside).  Sample s of post p uses SplitMix64 output number p*S + s of the
  seed, and the local grid numbers posts from its first row ya, so the
  local call's seed is seed + 0x9E3779B97F4A7C15 * ya * W * S (mod 2^64):
  the generator's state for local post p - ya*W is then the global one.
- Findmax: the strip's blocks; concatenated in rank order the ranks' lists
  are the global list (blocks ordered row-major).
- Viewshed: the rank's candidates on the same local grid (the window of a
  strip post and every post its rays read lie inside); the bitmaps are the
  single-GPU ones (words are aligned to global columns).
- Site: every rank holds its candidates' bitmaps and gains and a full copy of
  the cumulative viewshed.  Per greedy step: each rank's best key
  (gain << 32) | (0xFFFFFFFF - post) -> all-reduce MAX of one 8-byte value ->
  the rank whose strip holds the winning post broadcasts the winner's bitmap
  -> every rank ORs it in and refreshes its own candidates
  (vs_site_shard_step).  The observers, gains and coverage are the single-rank
  greedy's, ties and stops included.

No data-path collective other than the site step's key and bitmap is needed.
The backend object does the per-rank computation: GPUBackend calls the
library's kernels; the tests pass a CPU backend to check the protocol.
"""
import math

import numpy as np
import torch

GAMMA = 0x9E3779B97F4A7C15


def strip_rows(H, block, rank, world):
    """Rows [y0, y1) of rank's strip: whole block rows, divided evenly."""
    nby = (H + block - 1) // block
    b0, b1 = nby * rank // world, nby * (rank + 1) // world
    return min(H, b0 * block), min(H, b1 * block)


def local_rows(H, y0, y1, R):
    """Rows [ya, yb) of the rank's local grid: the strip and R + 1 rows of halo."""
    return max(0, y0 - R - 1), min(H, y1 + R + 1)


def local_vix_seed(seed, ya, W, S):
    """Seed of the local vix call whose post numbering starts at global row ya."""
    return (seed + GAMMA * ya * W * S) % (1 << 64)


def owner_of(post, W, H, block, world):
    """Rank whose strip holds the post."""
    y = post // W
    for r in range(world):
        y0, y1 = strip_rows(H, block, r, world)
        if y0 <= y < y1:
            return r
    raise ValueError("post outside the grid")


class GPUBackend:
    """Per-rank computation on this process's GPU through the library."""

    def __init__(self, device="cuda"):
        from . import vshed as V
        self.V = V
        self.dev = device

    def grid(self, z_rows):
        return self.V.Grid.from_tensor(torch.as_tensor(z_rows), self.dev)

    def vix(self, g, R, ht, hr, S, seed):
        return self.V.vix(g, R, ht, hr, S, seed)

    def findmax(self, vmap_rows, block, k):
        return self.V.findmax(vmap_rows.contiguous(), block, k)

    def viewshed(self, g, R, ht, hr, posts_local):
        return self.V.viewshed(g, R, ht, hr, posts_local)[0]

    def site_init(self, bm, cand, H, W, R, cum):
        self.ws = torch.empty(self.V.lib().vs_site_shard_workspace(R), dtype=torch.uint8, device=self.dev)
        self.key = torch.zeros(1, dtype=torch.int64, device=self.dev)
        return self.V.site_gains(bm, cand, H, W, R, cum) if cand.numel() else \
            torch.zeros(0, dtype=torch.int32, device=self.dev)

    def site_step(self, bm, cand, H, W, R, gains, cum, win_bm, win_post, win_local):
        self.V.site_shard_step(bm, cand, H, W, R, gains, cum, win_bm, win_post, win_local, self.key, self.ws)
        return int(self.key.item())

    def cand_to_host(self, cand):
        return cand.cpu().numpy()

    def bitmap(self, bm, i):
        return bm[i].contiguous()


class ShardedSiting:
    """The whole pipeline (vix -> findmax -> viewshed -> site) with the grid
    split over the ranks of a torch.distributed process group."""

    def __init__(self, dist, backend, comm_device="cpu"):
        self.dist = dist
        self.be = backend
        self.rank = dist.get_rank() if dist else 0
        self.world = dist.get_world_size() if dist else 1
        self.comm_device = comm_device

    def _allreduce_max(self, v):
        if self.world == 1:
            return v
        t = torch.tensor([v], dtype=torch.int64, device=self.comm_device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return int(t.item())

    def _broadcast(self, arr, src):
        if self.world == 1:
            return arr
        t = arr.to(self.comm_device) if torch.is_tensor(arr) else torch.as_tensor(arr, device=self.comm_device)
        self.dist.broadcast(t, src)
        return t

    def run(self, z, R, ht, hr, S, seed, block, k, n_obs, target=0.0):
        """z: the whole terrain (H x W int16, host), read only for this rank's
        rows.  Returns (candidates of this rank (global posts), chosen posts,
        gains, this rank's cumulative viewshed, this rank's vix strip)."""
        be = self.be
        H, W = z.shape
        y0, y1 = strip_rows(H, block, self.rank, self.world)
        ya, yb = local_rows(H, y0, y1, R)
        g = be.grid(np.ascontiguousarray(z[ya:yb]))
        vloc = be.vix(g, R, ht, hr, S, local_vix_seed(seed, ya, W, S))
        vstrip = vloc[y0 - ya:y1 - ya]
        if y1 > y0:
            cand_strip = be.findmax(vstrip, block, k)
            cand = cand_strip + y0 * W                  # global posts
            bm = be.viewshed(g, R, ht, hr, cand_strip + (y0 - ya) * W)
        else:
            cand = torch.zeros(0, dtype=torch.int64)
            bm = None
        chosen, gains_out, cum = self._site(bm, cand, H, W, R, n_obs, target, block)
        return cand, chosen, gains_out, cum, vstrip

    def _site(self, bm, cand, H, W, R, n_obs, target, block):
        be = self.be
        WWc = (W + 31) // 32
        cum = be.zeros_cum(H, WWc) if hasattr(be, "zeros_cum") else \
            torch.zeros((H, WWc), dtype=torch.int32, device=getattr(be, "dev", "cpu"))
        need = -1
        if target > 0:
            need = math.ceil(target * H * W)
        gains = be.site_init(bm, cand, H, W, R, cum)
        cand_h = be.cand_to_host(cand)
        chosen, gains_out = [], []
        covered = 0
        win_bm, win_post, win_local = None, -1, -1
        words = (2 * R + 1) * ((2 * R) // 32 + 2)
        for t in range(n_obs + 1):
            key = be.site_step(bm, cand, H, W, R, gains, cum, win_bm, win_post, win_local)
            if t == n_obs:
                break                                   # the last winner is applied; no more steps
            if need >= 0 and covered >= need:
                break
            key = self._allreduce_max(key)
            if key == 0:
                break
            gain = key >> 32
            post = 0xFFFFFFFF - (key & 0xFFFFFFFF)
            owner = owner_of(post, W, H, block, self.world)
            if owner == self.rank:
                win_local = int(np.flatnonzero(cand_h == post)[0])   # the lowest index holding the post
                wb = be.bitmap(bm, win_local)
            else:
                win_local = -1
                wb = torch.zeros(words, dtype=torch.int32)
            wb = self._broadcast(wb.reshape(-1) if torch.is_tensor(wb) else wb, owner)
            win_bm = be.to_backend(wb) if hasattr(be, "to_backend") else wb.to(getattr(be, "dev", "cpu"))
            win_post = post
            chosen.append(post)
            gains_out.append(gain)
            covered += gain
        return np.array(chosen, np.int64), np.array(gains_out, np.int64), cum
