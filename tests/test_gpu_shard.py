"""The sharded pipeline with the library's kernels (shard.GPUBackend): two
ranks as two processes on one GPU -- their kernels never wait on each other;
the site step's key all-reduce and bitmap broadcast go through gloo on the
host -- and one rank, against the single-process pipeline and the oracle."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CASE = dict(H=700, W=650, R=40, ht=10, hr=10, S=10, seed=3, block=50, k=2, n_obs=120)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _terrain():
    from synth import terrain as T
    return T.spectral_fbm(CASE["H"], CASE["W"], 0.8, 404, 0, 900).numpy()


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2006_16783_gb300 import _build, shard
    _build.build()
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    c = CASE
    ss = shard.ShardedSiting(dist, shard.GPUBackend("cuda:0"))
    cand, chosen, gains, cum, _ = ss.run(_terrain(), c["R"], c["ht"], c["hr"], c["S"], c["seed"], c["block"],
                                         c["k"], c["n_obs"])
    torch.cuda.synchronize()
    q.put((rank, cand.cpu().numpy().tolist(), chosen.tolist(), gains.tolist(), cum.cpu().numpy().tobytes()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_16783_gb300 import _build
    _build.build()
    import paper_2006_16783_gb300 as V
    return V


def _single(V):
    c = CASE
    g = V.Grid.from_tensor(torch.as_tensor(_terrain()), "cuda")
    v = V.vix(g, c["R"], c["ht"], c["hr"], c["S"], c["seed"])
    cand = V.findmax(v, c["block"], c["k"])
    bm, _ = V.viewshed(g, c["R"], c["ht"], c["hr"], cand)
    ch, gn, cum, t = V.site(bm, cand, c["H"], c["W"], c["R"], c["n_obs"])
    return cand.cpu().numpy(), ch.cpu().numpy(), gn.cpu().numpy(), cum.cpu().numpy()


def test_sharded_two_ranks_on_the_gpu(V, O):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = {}
    for _ in range(2):
        r = q.get(timeout=600)
        res[r[0]] = r[1:]
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    cand, ch, gn, cum = _single(V)
    assert res[0][0] + res[1][0] == cand.tolist()
    for r in (0, 1):
        assert res[r][1] == ch.tolist() and res[r][2] == gn.tolist()
        assert (np.frombuffer(res[r][3], np.int32).reshape(cum.shape) == cum).all()
    # and the single-process pipeline is the oracle's
    z = _terrain()
    c = CASE
    ov = O.vix(z, c["R"], c["ht"], c["hr"], c["S"], c["seed"])
    oc = O.findmax(ov, c["block"], c["k"])
    assert oc.tolist() == cand.tolist()
    obm, _ = O.viewshed(z, c["R"], c["ht"], c["hr"], oc, threads=8)
    och, ogn, oC = O.site(obm, oc, c["H"], c["W"], c["R"], c["n_obs"])
    assert och.tolist() == ch.tolist() and ogn.tolist() == gn.tolist()


def test_sharded_one_rank(V):
    from paper_2006_16783_gb300 import shard
    c = CASE
    ss = shard.ShardedSiting(None, shard.GPUBackend("cuda"))
    cand, chosen, gains, cum, _ = ss.run(_terrain(), c["R"], c["ht"], c["hr"], c["S"], c["seed"], c["block"],
                                         c["k"], c["n_obs"])
    s_cand, s_ch, s_gn, s_cum = _single(V)
    assert cand.cpu().numpy().tolist() == s_cand.tolist()
    assert chosen.tolist() == s_ch.tolist() and gains.tolist() == s_gn.tolist()
    assert (cum.cpu().numpy() == s_cum).all()
