"""Learned candidate proposal: labels, training loop and proposal on top of
the C-ABI kernels (every step of the computation runs in libvshed).

The label of a post is its exact visibility index at ROI R (Sec.
"Definitions": the fraction of the receivers within the ROI that are
visible), here the area of its ray-sweep viewshed (vs_viewshed) over the
number of lattice points of the disc inside the grid.  The network is
trained by Adam on the mean L1 error (vs_cnn_forward with saved activations,
vs_cnn_backward, vs_cnn_adam, vs_cnn_pack).
"""
import math
import time

import numpy as np
import torch

from . import vshed as V


def exact_vix(g, posts, R, ht, hr, chunk=1 << 20, ws=None):
    """Exact visibility index of every listed post (fp32 in [0, 1]), computed
    by vs_exact_vix in chunks of ``chunk`` posts (one workspace reused)."""
    out = torch.empty(posts.numel(), dtype=torch.float32, device=posts.device)
    wsb = V.lib().vs_exact_vix_workspace(g.H, g.W, R, min(chunk, posts.numel()))
    if ws is None or ws.numel() < wsb:
        ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=posts.device)
    for i in range(0, posts.numel(), chunk):
        p = posts[i:i + chunk].contiguous()
        V.exact_vix(g, R, ht, hr, p, out=out[i:i + p.numel()], ws=ws)
    return out


def sample_posts(H, W, n, margin, seed, device):
    """n posts drawn uniformly at least ``margin`` from every edge."""
    gen = torch.Generator(device="cpu").manual_seed(seed)
    y = torch.randint(margin, H - margin, (n,), generator=gen)
    x = torch.randint(margin, W - margin, (n,), generator=gen)
    return (y * W + x).to(device)


def init_master(seed=0, device="cuda"):
    """He-normal conv weights, zero biases, small fc: the flat fp32 layout."""
    gen = torch.Generator(device="cpu").manual_seed(seed)
    parts = []
    for l, cin in enumerate([1, 32, 32, 32, 32]):
        parts.append(torch.randn(32 * cin * 9, generator=gen) * math.sqrt(2.0 / (9 * cin)))
        parts.append(torch.zeros(32))
    parts.append(torch.randn(32, generator=gen) * math.sqrt(1.0 / 32))
    parts.append(torch.zeros(1))
    w = torch.cat(parts).float().to(device)
    assert w.numel() == V.cnn_param_count()
    return w


class Trainer:
    """Mini-batch Adam on (grid, post, label) triples drawn from several grids."""

    def __init__(self, master, batch=512, lr=2e-3, patch_step=1):
        self.master = master
        self.patch_step = patch_step
        self.batch = batch
        self.lr = lr
        dev = master.device
        self.grads = torch.zeros_like(master)
        self.m = torch.zeros_like(master)
        self.v = torch.zeros_like(master)
        self.packed = V.cnn_pack(master)
        self.save = torch.empty(batch * V.cnn_save_bytes(), dtype=torch.uint8, device=dev)
        self.out = torch.empty(batch, dtype=torch.float32, device=dev)
        self.loss = torch.zeros(1, dtype=torch.float32, device=dev)
        self.ws = None
        self.step = 0
        self.epochs_done = 0

    def train_step(self, g, posts, labels):
        B = posts.numel()
        V.cnn_forward(g, posts, self.packed, out=self.out[:B], save=self.save[:B * V.cnn_save_bytes()],
                      patch_step=self.patch_step)
        self.ws = V.cnn_backward(self.save[:B * V.cnn_save_bytes()], labels, self.master, self.grads,
                                 self.loss, ws=self.ws)
        self.step += 1
        lr = self.lr
        V.cnn_adam(self.master, self.grads, self.m, self.v, self.step, lr=lr)
        V.cnn_pack(self.master, self.packed)

    def fit(self, data, epochs, seed=0, lr_decay=0.5, log=None, first_epoch=0):
        """data: list of (grid, posts, labels).  Epochs first_epoch .. epochs-1
        run with learning rate lr * lr_decay^epoch, each on a shuffle drawn
        from its own seed (seed, epoch), so that training resumed at an
        epoch boundary from a checkpoint (checkpoint / from_checkpoint) continues
        exactly as an uninterrupted run.  Returns the mean training loss of
        the last epoch."""
        last = None
        base_lr = self.lr
        for ep in range(first_epoch, epochs):
            gen = torch.Generator(device="cpu").manual_seed(seed * 1000003 + ep)
            self.lr = base_lr * (lr_decay ** ep)
            self.loss.zero_()
            seen = 0
            t0 = time.time()
            order = []
            for gi, (g, posts, labels) in enumerate(data):
                perm = torch.randperm(posts.numel(), generator=gen)
                for i in range(0, posts.numel() - self.batch + 1, self.batch):
                    order.append((gi, perm[i:i + self.batch]))
            sel = torch.randperm(len(order), generator=gen).tolist()
            for j in sel:
                gi, idx = order[j]
                g, posts, labels = data[gi]
                idx = idx.to(posts.device)
                self.train_step(g, posts[idx].contiguous(), labels[idx].contiguous())
                seen += idx.numel()
            last = float(self.loss.item()) / max(seen, 1)
            self.epochs_done = ep + 1
            if log:
                log("epoch %d: mean |y - label| = %.4f (%.1f s)" % (ep, last, time.time() - t0))
        self.lr = base_lr
        return last

    def checkpoint(self):
        """Checkpoint of the training state (host copies): fp32 master
        weights, Adam moments, Adam step, learning rate, batch size, patch
        step and the number of epochs done."""
        return {"master": self.master.cpu().clone(), "m": self.m.cpu().clone(), "v": self.v.cpu().clone(),
                "step": self.step, "lr": self.lr, "batch": self.batch, "patch_step": self.patch_step,
                "epochs_done": self.epochs_done}

    def save_checkpoint(self, path):
        torch.save(self.checkpoint(), path)

    @classmethod
    def from_checkpoint(cls, st, device="cuda"):
        """A trainer that continues from a checkpoint made by checkpoint()."""
        tr = cls(st["master"].to(device).clone(), batch=st["batch"], lr=st["lr"], patch_step=st["patch_step"])
        tr.m.copy_(st["m"].to(device))
        tr.v.copy_(st["v"].to(device))
        tr.step = int(st["step"])
        tr.epochs_done = int(st["epochs_done"])
        return tr

    @classmethod
    def load_checkpoint(cls, path, device="cuda"):
        return cls.from_checkpoint(torch.load(path, map_location="cpu"), device)

    def predict(self, g, posts, chunk=1 << 20):
        out = torch.empty(posts.numel(), dtype=torch.float32, device=posts.device)
        for i in range(0, posts.numel(), chunk):
            V.cnn_forward(g, posts[i:i + chunk].contiguous(), self.packed, out=out[i:i + chunk],
                          patch_step=self.patch_step)
        return out


def sampled_vix_fraction(g, posts, R, ht, hr, S, seed):
    """The plain method's estimate of the same quantity: vix count / S,
    evaluated only at the listed posts (one vs_vix pass over the grid)."""
    v = V.vix(g, R, ht, hr, S, seed)
    return v.reshape(-1)[posts].float() / float(S)


def propose(g, packed, stride, block, k, score=None, patch_step=1):
    """Candidate posts from the network's scores on a stride lattice:
    top-k per block (vs_cnn_score_lattice then vs_findmax_f32)."""
    score = V.cnn_score_lattice(g, stride, packed, out=score, patch_step=patch_step)
    return V.findmax_f32(score, g.H, g.W, stride, block, k), score


def score_lattice_streamed(g, host, stride, packed, out, patch_step=1, chunks=8, copy_stream=None):
    """Score the stride lattice of a terrain that is still in host memory.

    ``host`` is a pinned CPU tensor laid out like ``g.storage`` ([H][pitch]
    int16); it is copied into ``g.storage`` in ``chunks`` row bands on a side
    stream, and every band of lattice rows is scored on the current stream as
    soon as the terrain rows its patches read (within 32 * patch_step rows)
    have arrived, so the copy overlaps the network.  On return the current
    stream is ordered after the whole copy (later stages see the full
    terrain); nothing is synchronised with the host."""
    H, W = g.H, g.W
    Hs, Ws = (H + stride - 1) // stride, (W + stride - 1) // stride
    if tuple(host.shape) != tuple(g.storage.shape) or host.dtype != g.storage.dtype or not host.is_pinned():
        raise ValueError("host must be a pinned tensor shaped like the grid's storage")
    cur = torch.cuda.current_stream()
    cs = copy_stream or torch.cuda.Stream()
    cs.wait_stream(cur)  # earlier work on the device buffer is done
    bounds = [(i * H) // chunks for i in range(chunks + 1)]
    done = []
    with torch.cuda.stream(cs):
        for i in range(chunks):
            a, b = bounds[i], bounds[i + 1]
            if b > a:
                g.storage[a:b].copy_(host[a:b], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(cs)
            done.append((b, ev))
    reach = 32 * patch_step
    r = 0
    for b, ev in done:
        # lattice rows i whose patches read only rows below b
        last = Hs if b >= H else max(0, min(Hs, (b - 1 - reach) // stride + 1))
        if last > r:
            cur.wait_event(ev)
            V.cnn_score_lattice_rows(g, stride, packed, r, last - r, out[r:last], patch_step=patch_step)
            r = last
    cur.wait_stream(cs)
    return out


def _main():
    """python -m paper_2006_16783_gb300.surrogate score-lattice --size N --stride S
    scores an N x N ridged terrain with randomly initialised weights
    (--patch-step P: patches sampled every P posts);
    python -m paper_2006_16783_gb300.surrogate train-steps --size N --batch B --reps K
    runs K training steps (forward with saved activations, backward, Adam)
    on B random posts of that terrain with labels from vs_exact_vix.  Both
    are for timing and profiling the network's kernels."""
    import argparse
    import sys

    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["score-lattice", "train-steps"])
    ap.add_argument("--size", type=int, default=2048)
    ap.add_argument("--stride", type=int, default=16)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--batch", type=int, default=512)
    ap.add_argument("--patch-step", type=int, default=1)
    a = ap.parse_args()
    root = __file__.rsplit("/", 2)[0]
    if root not in sys.path:
        sys.path.insert(0, root)
    from synth import terrain as T
    from . import _build
    _build.build()
    z = T.ridged_multifractal(a.size, a.size, 5, 0, 4000, 0.05, octaves=10, base_wavelength=640, device="cuda")
    g = V.Grid(z.contiguous())
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    if a.cmd == "train-steps":
        margin = 32 * a.patch_step
        posts = sample_posts(a.size, a.size, a.batch, margin, 1, "cuda")
        labels = exact_vix(g, posts, 100, 10, 10)
        tr = Trainer(init_master(0), batch=a.batch, patch_step=a.patch_step)
        for i in range(a.reps):
            if i == a.reps - 1:
                ev[0].record()
            tr.train_step(g, posts, labels)
        ev[1].record()
        torch.cuda.synchronize()
        print("batch %d, last step %.3f ms, mean |y - label| %.4f" % (a.batch, ev[0].elapsed_time(ev[1]),
                                                                     float(tr.loss.item()) / (a.batch * a.reps)))
        return
    packed = V.cnn_pack(init_master(0))
    sc = None
    for i in range(a.reps):
        if i == a.reps - 1:
            ev[0].record()
        sc = V.cnn_score_lattice(g, a.stride, packed, patch_step=a.patch_step)
    ev[1].record()
    torch.cuda.synchronize()
    print("patches %d, last launch %.3f ms, mean score %.4f" % (sc.numel(), ev[0].elapsed_time(ev[1]),
                                                               float(sc.mean())))


if __name__ == "__main__":
    _main()
