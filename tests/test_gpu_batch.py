"""Batched multi-terrain siting (one persistent vix launch, one findmax
launch, one persistent viewshed launch, the greedy problems' preparation in
six launches and their loops in one, the whole sequence captured in a CUDA
graph) against the oracle run terrain by terrain; the launch count does not
grow with the number of terrains; the autotuner's launch shapes leave results
unchanged."""
import numpy as np
import pytest
import torch

from synth import terrain as T

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_16783_gb300 import _build
    _build.build()
    import paper_2006_16783_gb300 as V
    return V


def _instances(V):
    rng = np.random.default_rng(1002)
    out, zs = [], []
    for i in range(6):
        side = int(rng.integers(90, 260))
        H, W = side, side + int(rng.integers(0, 13))
        R = int(rng.choice([5, 10, 20, 40]))
        h = int(rng.integers(5, 31))
        z = T.spectral_fbm(H, W, 0.8, 500 + i, 0, 1000 * int(rng.integers(1, 4))).numpy()
        zs.append(z)
        out.append({"grid": V.Grid.from_tensor(torch.as_tensor(z), "cuda"), "R": R, "ht": h, "hr": h,
                    "S": 10, "seed": 77 + i, "block": (R + 1) // 2, "k": 1,
                    "n_obs": int(rng.integers(16, 120))})
    return out, zs


def _oracle(O, z, it):
    v = O.vix(z, it["R"], it["ht"], it["hr"], it["S"], it["seed"], threads=8)
    cand = O.findmax(v, it["block"], it["k"])
    bm, area = O.viewshed(z, it["R"], it["ht"], it["hr"], cand, threads=8)
    H, W = z.shape
    ch, gn, C = O.site(bm, cand, H, W, it["R"], it["n_obs"])
    return v, cand, bm, ch, gn, C


def _check(V, O, bs, zs):
    for it, z, b, (ch, gn, C) in zip(bs.inst, zs, bs.bufs, bs.results()):
        v, cand, bm, och, ogn, oC = _oracle(O, z, it)
        assert (b["vix"].cpu().numpy() == v).all()
        assert b["cand"].cpu().numpy().tolist() == cand.tolist()
        assert (b["bm"].cpu().numpy().view(np.uint32) == bm).all()
        assert ch.cpu().numpy().tolist() == och.tolist()
        assert gn.cpu().numpy().tolist() == ogn.tolist()
        assert (C.cpu().numpy().view(np.uint32) == oC).all()


def test_batched_pipeline_and_graph(V, O):
    from paper_2006_16783_gb300.batch import BatchedSiting
    inst, zs = _instances(V)
    bs = BatchedSiting(inst)
    bs.run()
    torch.cuda.synchronize()
    _check(V, O, bs, zs)
    bs.capture()
    for b in bs.bufs:
        for key in ("bm", "chosen", "gains", "cum", "cand"):
            b[key].fill_(-3)
    bs.replay()
    torch.cuda.synchronize()
    _check(V, O, bs, zs)


def test_autotuner_keeps_results(V):
    from paper_2006_16783_gb300 import autotune
    z = T.spectral_fbm(300, 320, 0.8, 3, 0, 900).numpy()
    g = V.Grid.from_tensor(torch.as_tensor(z), "cuda")
    cand = torch.arange(0, 300 * 320, 211, dtype=torch.int64, device="cuda")
    outs = []
    for t in (128, 256, 512):
        V.tune_set(V.VS_TUNE_VIEWSHED_THREADS, 30, t)
        bm, area = V.viewshed(g, 30, 10, 10, cand)
        outs.append(bm.cpu().numpy())
    assert all((o == outs[0]).all() for o in outs)
    v1 = []
    for t in (1, 2):
        V.tune_set(V.VS_TUNE_VIX_TILE, 30, t)
        v1.append(V.vix(g, 30, 10, 10, 10, 5).cpu().numpy())
    assert (v1[0] == v1[1]).all()
    best, times = autotune.tune_viewshed(g, 30, 10, 10, n=500)
    assert best in (128, 256, 512) and V.tune_get(V.VS_TUNE_VIEWSHED_THREADS, 30) == best
    V.tune_set(V.VS_TUNE_VIEWSHED_THREADS, 30, 0)
    V.tune_set(V.VS_TUNE_VIX_TILE, 30, 0)


def test_batch_launch_count_is_constant(V):
    """One siting of 3 terrains and of 6 terrains issue the same number of launches."""
    from paper_2006_16783_gb300.batch import BatchedSiting
    inst, _ = _instances(V)
    counts = []
    for m in (3, 6):
        bs = BatchedSiting(inst[:m])
        bs.run()
        torch.cuda.synchronize()
        c0 = V.launch_count()
        bs.run()
        counts.append(V.launch_count() - c0)
    assert counts[0] == counts[1] <= 10, counts


def test_site_batch_global_gains_job(V, O):
    """A job whose gains exceed one CTA's shared memory (55,000 candidates)
    runs inside the batched launch with its gains in global memory, beside a
    small job with a coverage stop; both equal the oracle."""
    H, W = 400, 380
    jobs, want = [], []
    for n, R, seed, target in ((55000, 3, 1, 0.0), (700, 12, 2, 0.3)):
        z = T.spectral_fbm(H, W, 0.8, 90 + seed, 0, 600).numpy()
        rng = np.random.default_rng(seed)
        cand = rng.choice(H * W, n, replace=False).astype(np.int64)
        bm, _ = O.viewshed(z, R, 10, 10, cand, threads=8)
        want.append(O.site(bm, cand, H, W, R, 400, target=target))
        jobs.append({"bm": torch.as_tensor(bm.view(np.int32)).cuda(), "cand": torch.as_tensor(cand).cuda(),
                     "H": H, "W": W, "R": R, "n_obs": 400, "target": target,
                     "chosen": torch.empty(400, dtype=torch.int64, device="cuda"),
                     "gains": torch.empty(400, dtype=torch.int64, device="cuda"),
                     "cum": torch.zeros((H, (W + 31) // 32), dtype=torch.int32, device="cuda"),
                     "n_chosen": torch.zeros(1, dtype=torch.int32, device="cuda")})
    ws = torch.empty(V.site_batch_workspace(jobs), dtype=torch.uint8, device="cuda")
    V.site_batch(jobs, ws)
    torch.cuda.synchronize()
    for j, (ch, gn, C) in zip(jobs, want):
        t = int(j["n_chosen"].item())
        assert t == len(ch)
        assert j["chosen"][:t].cpu().numpy().tolist() == ch.tolist()
        assert j["gains"][:t].cpu().numpy().tolist() == gn.tolist()
        assert (j["cum"].cpu().numpy().view(np.uint32) == C).all()
