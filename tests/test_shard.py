"""The siting pipeline split over ranks (paper_2006_16783_gb300.shard) on CPU:
two gloo ranks run the protocol -- strips with halos, the vix seed offset,
per-strip findmax, per-rank viewsheds, and the site step's all-reduce of the
8-byte key and broadcast of the winner's bitmap -- with a backend that does
each rank's work with the oracle and plain numpy (gains recomputed from
their definition).  The outcome must equal the single-rank oracle pipeline
exactly.  No GPU needed."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleBackend:
    """Each rank's computation with the CPU oracle (test infrastructure)."""

    def __init__(self):
        from oracle import oracle as O
        self.O = O

    def grid(self, z_rows):
        return np.ascontiguousarray(z_rows, np.int16)

    def vix(self, g, R, ht, hr, S, seed):
        return self.O.vix(g, R, ht, hr, S, seed)

    def findmax(self, vrows, block, k):
        return self.O.findmax(np.ascontiguousarray(vrows), block, k)

    def viewshed(self, g, R, ht, hr, posts):
        return self.O.viewshed(g, R, ht, hr, np.asarray(posts, np.int64))[0]

    def zeros_cum(self, H, WWc):
        return np.zeros((H, WWc), np.uint32)

    def _gains(self, bm, cand, H, W, R, cum):
        PR = (2 * R) // 32 + 2
        WWc = cum.shape[1]
        out = np.zeros(len(cand), np.int64)
        for i, p in enumerate(cand):
            cx, cy = int(p) % W, int(p) // W
            gw0 = (cx - R) // 32
            V = bm[i].reshape(2 * R + 1, PR)
            y0, y1 = max(0, cy - R), min(H - 1, cy + R)
            g0, g1 = max(0, gw0), min(WWc - 1, gw0 + PR - 1)
            v = V[y0 - (cy - R):y1 - (cy - R) + 1, g0 - gw0:g1 - gw0 + 1]
            c = cum[y0:y1 + 1, g0:g1 + 1]
            out[i] = int(np.unpackbits((v & ~c).view(np.uint8)).sum())
        return out

    def site_init(self, bm, cand, H, W, R, cum):
        self.geom = (H, W, R)
        return self._gains(bm, cand, H, W, R, cum)

    def site_step(self, bm, cand, H, W, R, gains, cum, win_bm, win_post, win_local):
        if win_post >= 0:                          # C |= V_win over its window
            PR = (2 * R) // 32 + 2
            WWc = cum.shape[1]
            cx, cy = win_post % W, win_post // W
            gw0 = (cx - R) // 32
            V = win_bm.reshape(2 * R + 1, PR)
            y0, y1 = max(0, cy - R), min(H - 1, cy + R)
            g0, g1 = max(0, gw0), min(WWc - 1, gw0 + PR - 1)
            cum[y0:y1 + 1, g0:g1 + 1] |= V[y0 - (cy - R):y1 - (cy - R) + 1, g0 - gw0:g1 - gw0 + 1]
        gains[:] = self._gains(bm, cand, H, W, R, cum)
        keys = [(int(g) << 32) | (0xFFFFFFFF - int(p)) for g, p in zip(gains, cand) if g > 0]
        return max(keys) if keys else 0

    def cand_to_host(self, cand):
        return np.asarray(cand)

    def bitmap(self, bm, i):
        return torch.as_tensor(np.ascontiguousarray(bm[i]).view(np.int32).reshape(-1))

    def to_backend(self, t):
        return t.numpy().view(np.uint32)


CASES = {
    "plain": dict(H=97, W=83, R=8, ht=10, hr=10, S=10, seed=5, block=10, k=2, n_obs=25, target=0.0),
    "coverage_stop": dict(H=90, W=70, R=6, ht=5, hr=3, S=7, seed=11, block=9, k=3, n_obs=200, target=0.6),
    "edge_rows": dict(H=61, W=64, R=3, ht=10, hr=10, S=10, seed=2, block=6, k=1, n_obs=400, target=0.0),
}


def _rank_main(rank, world, port, case, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2006_16783_gb300 import shard
    from synth import terrain as T
    c = CASES[case]
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    z = T.spectral_fbm(c["H"], c["W"], 0.8, 100 + c["seed"], 0, 400).numpy()
    ss = shard.ShardedSiting(dist, OracleBackend())
    cand, chosen, gains, cum, vstrip = ss.run(z, c["R"], c["ht"], c["hr"], c["S"], c["seed"], c["block"], c["k"],
                                              c["n_obs"], c["target"])
    q.put((rank, np.asarray(cand).tolist(), chosen.tolist(), gains.tolist(), cum.tobytes(),
           np.asarray(vstrip).tobytes()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("case", sorted(CASES))
def test_sharded_pipeline_equals_single_rank(O, case):
    from synth import terrain as T
    c = CASES[case]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, 2, port, case, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = {}
    for _ in range(2):
        r = q.get(timeout=300)
        res[r[0]] = r[1:]
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    z = T.spectral_fbm(c["H"], c["W"], 0.8, 100 + c["seed"], 0, 400).numpy()
    v = O.vix(z, c["R"], c["ht"], c["hr"], c["S"], c["seed"])
    cand = O.findmax(v, c["block"], c["k"])
    bm, _ = O.viewshed(z, c["R"], c["ht"], c["hr"], cand)
    ch, gn, C = O.site(bm, cand, c["H"], c["W"], c["R"], c["n_obs"], target=c["target"])
    # the vix strips and candidate lists, concatenated in rank order
    vs = np.concatenate([np.frombuffer(res[r][4], np.uint8) for r in (0, 1)])
    assert (vs == v.ravel()).all()
    assert res[0][0] + res[1][0] == cand.tolist()
    for r in (0, 1):
        assert res[r][1] == ch.tolist() and res[r][2] == gn.tolist()
        assert (np.frombuffer(res[r][3], np.uint32).reshape(C.shape) == C).all()
    assert len(ch) > 3


def test_strips_partition_block_rows():
    sys.path.insert(0, ROOT)
    from paper_2006_16783_gb300 import shard
    for H, b, world in [(97, 10, 2), (46400, 464, 8), (61, 6, 3), (100, 7, 4)]:
        rows = [shard.strip_rows(H, b, r, world) for r in range(world)]
        assert rows[0][0] == 0 and rows[-1][1] == H
        for (a0, a1), (b0, b1) in zip(rows, rows[1:]):
            assert a1 == b0 and a1 % b == 0
    # the seed offset makes the local counter equal the global one
    seed, ya, W, S = 12345, 37, 83, 10
    s2 = shard.local_vix_seed(seed, ya, W, S)
    for p_local, s in [(0, 0), (5, 3), (1000, 9)]:
        p = p_local + ya * W
        assert (s2 + shard.GAMMA * (p_local * S + s + 1)) % (1 << 64) == \
               (seed + shard.GAMMA * (p * S + s + 1)) % (1 << 64)
