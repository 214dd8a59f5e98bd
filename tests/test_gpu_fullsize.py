"""Parity at the workloads' full sizes, in the launch configurations the
benchmark uses, on outputs the oracle can compute one by one: sampled vix
posts, viewsheds of seeded candidates, findmax over a seeded full-size map,
and the greedy site over oracle-made bitmaps of seeded candidates.  The
terrains are generated on the GPU and copied to the host for the oracle."""
import numpy as np
import pytest
import torch

from synth import workloads as WL

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_16783_gb300 import _build
    _build.build()
    import paper_2006_16783_gb300 as V
    return V


def _terrain(V, w):
    z = w.make_terrain("cuda")
    zs, pitch = WL.terrain.pad_pitch(z, 8)
    g = V.Grid(zs, w.W)
    zh = z.cpu().numpy()
    del z
    return g, zh


def _seeded_posts(H, W, n, seed, margin=0):
    rng = np.random.default_rng(seed)
    return (rng.integers(margin, H - margin, n) * W + rng.integers(margin, W - margin, n)).astype(np.int64)


@pytest.mark.parametrize("name", ["full", "scale"])
def test_full_size_sampled_parity(V, O, name):
    w = {"full": WL.FULL, "scale": WL.SCALE}[name]
    g, zh = _terrain(V, w)
    H, W = w.H, w.W
    # vix: the bench's launch over the whole grid, sampled posts (edges included)
    v = V.vix(g, w.R, w.ht, w.hr, w.S, w.vix_seed)
    posts = np.concatenate([_seeded_posts(H, W, 600, 1), np.array([0, W - 1, (H - 1) * W, H * W - 1])])
    want = O.vix_posts(zh, w.R, w.ht, w.hr, w.S, w.vix_seed, posts)
    got = v.reshape(-1)[torch.as_tensor(posts).cuda()].cpu().numpy()
    assert (got == want).all()
    # viewsheds of seeded candidates (some at the border)
    cand = np.concatenate([_seeded_posts(H, W, 150, 2), np.array([0, H * W - 1, (H // 2) * W])])
    bm, area = V.viewshed(g, w.R, w.ht, w.hr, torch.as_tensor(cand).cuda())
    obm, oarea = O.viewshed(zh, w.R, w.ht, w.hr, cand, threads=16)
    assert (area.cpu().numpy() == oarea).all()
    assert (bm.cpu().numpy().view(np.uint32) == obm).all()
    del zh


def test_full_size_findmax(V, O):
    w = WL.FULL
    rng = np.random.default_rng(9)
    vmap = rng.integers(0, w.S + 1, (w.H, w.W), dtype=np.uint8)
    got = V.findmax(torch.as_tensor(vmap).cuda(), w.block, w.k).cpu().numpy()
    want = O.findmax(vmap, w.block, w.k)
    assert len(want) == 40000 and (got == want).all()


def test_full_size_site(V, O):
    """The greedy over 6000 seeded candidates of the 46400^2 terrain (bitmaps
    made by the oracle), 4096 observers, against the oracle's lazy greedy."""
    w = WL.FULL
    g, zh = _terrain(V, w)
    cand = _seeded_posts(w.H, w.W, 6000, 3)
    obm, _ = O.viewshed(zh, w.R, w.ht, w.hr, cand, threads=16)
    ch, gn, C = O.site(obm, cand, w.H, w.W, w.R, w.n_obs)
    gch, ggn, gC, t = V.site(torch.as_tensor(obm.view(np.int32)).cuda(), torch.as_tensor(cand).cuda(),
                             w.H, w.W, w.R, w.n_obs)
    assert gch.cpu().numpy().tolist() == ch.tolist()
    assert ggn.cpu().numpy().tolist() == gn.tolist()
    assert (gC.cpu().numpy().view(np.uint32) == C).all()


def test_batch_full_size_sampled(V, O):
    """The 64-instance batched workload at its full sizes: one persistent
    viewshed launch over seeded candidates of every instance, compared with
    the oracle on a sample of each instance's candidates."""
    inst = WL.batch_instances()
    jobs, keep = [], []
    for i, w in enumerate(inst):
        z = w.make_terrain("cuda")
        g = V.Grid.from_tensor(z, "cuda")
        cand = torch.as_tensor(_seeded_posts(w.H, w.W, 60, 100 + i)).cuda()
        bm = torch.empty((cand.numel(), 2 * w.R + 1, V.words_per_row(w.R)), dtype=torch.int32, device="cuda")
        area = torch.empty(cand.numel(), dtype=torch.int32, device="cuda")
        jobs.append({"g": g, "R": w.R, "ht": w.ht, "hr": w.hr, "cand": cand, "bm": bm, "area": area})
        keep.append((w, z.cpu().numpy()))
    ws = torch.empty(256, dtype=torch.uint8, device="cuda")
    V.viewshed_batch(jobs, ws)
    torch.cuda.synchronize()
    for (w, zh), j in zip(keep, jobs):
        sel = np.arange(0, 60, 6)
        c = j["cand"].cpu().numpy()[sel]
        obm, oarea = O.viewshed(zh, w.R, w.ht, w.hr, c, threads=16)
        assert (j["area"].cpu().numpy()[sel] == oarea).all(), w.name
        assert (j["bm"].cpu().numpy()[sel].view(np.uint32) == obm).all(), w.name


def _downstream_matches_oracle(O, zh, w, cand, bm, area, res):
    """Every candidate's bitmap and area, then the whole greedy (observers,
    gains, cumulative viewshed) against the oracle on the oracle's bitmaps."""
    c = cand.cpu().numpy()
    obm, oarea = O.viewshed(zh, w.R, w.ht, w.hr, c, threads=16)
    assert (area.cpu().numpy() == oarea).all()
    assert (bm.cpu().numpy().view(np.uint32) == obm).all()
    och, ogn, oC = O.site(obm, c, w.H, w.W, w.R, w.n_obs)
    chosen, gains, cum, t = res
    t = int(t.item()) if torch.is_tensor(t) else t
    assert t == len(och)
    assert chosen[:t].cpu().numpy().tolist() == och.tolist()
    assert gains[:t].cpu().numpy().tolist() == ogn.tolist()
    assert (cum.cpu().numpy().view(np.uint32) == oC).all()


def _plain(V, O, w, g, zh):
    v = V.vix(g, w.R, w.ht, w.hr, w.S, w.vix_seed)
    cand = V.findmax(v, w.block, w.k)
    ocand = O.findmax(v.cpu().numpy(), w.block, w.k)
    del v
    assert cand.cpu().numpy().tolist() == ocand.tolist()
    bm, area = V.viewshed(g, w.R, w.ht, w.hr, cand)
    res = V.site(bm, cand, w.H, w.W, w.R, w.n_obs)
    torch.cuda.synchronize()
    _downstream_matches_oracle(O, zh, w, cand, bm, area, res)


def test_headline_pipelines_full_size(V, O):
    """The 46400^2 headline configuration end to end, in the bench's launch
    configuration: the plain pipeline (vix map -> findmax over the whole map
    compared with the oracle's findmax on the same map -> 40,000 viewsheds ->
    4096 observers) and the surrogate pipeline (CNN scores of the stride-64
    lattice, patch step 3 -> findmax_f32 compared with the oracle's on the
    same scores -> 40,000 viewsheds -> 4096 observers).  Every candidate,
    bitmap, area, observer, gain and the cumulative viewshed is compared; only
    the vix map itself is sampled (test_full_size_sampled_parity)."""
    from paper_2006_16783_gb300 import surrogate as S
    w = WL.FULL
    g, zh = _terrain(V, w)
    _plain(V, O, w, g, zh)
    packed = V.cnn_pack(S.init_master(0))
    stride, step = 64, 3
    score = V.cnn_score_lattice(g, stride, packed, patch_step=step)
    cand = V.findmax_f32(score, w.H, w.W, stride, w.block, w.k)
    ocand = O.findmax_f32(score.cpu().numpy(), w.H, w.W, stride, w.block, w.k)
    assert len(ocand) == 40000 and cand.cpu().numpy().tolist() == ocand.tolist()
    bm, area = V.viewshed(g, w.R, w.ht, w.hr, cand)
    res = V.site(bm, cand, w.H, w.W, w.R, w.n_obs)
    torch.cuda.synchronize()
    _downstream_matches_oracle(O, zh, w, cand, bm, area, res)


def test_scale_pipeline_full_size(V, O):
    """16384^2, R = 200, S = 20, top-2 per 256^2 block (8192 candidates, bitmap
    rows of 14 words: the one-CTA greedy), 2048 observers: the whole plain
    pipeline against the oracle as above."""
    w = WL.SCALE
    g, zh = _terrain(V, w)
    _plain(V, O, w, g, zh)


def test_batch_pipeline_full_size(V, O):
    """The 64-terrain batched workload at its full sizes through BatchedSiting
    (the bench's launch configuration): per terrain the vix map on 300
    sampled posts, findmax over the whole map, and the greedy (observers,
    gains, cumulative viewshed) against the oracle on the pipeline's bitmaps
    (whose viewsheds test_batch_full_size_sampled checks)."""
    from paper_2006_16783_gb300.batch import BatchedSiting
    ws_ = WL.batch_instances()
    inst, zs = [], []
    for w in ws_:
        z = w.make_terrain("cuda")
        g = V.Grid.from_tensor(z, "cuda")
        inst.append({"grid": g, "R": w.R, "ht": w.ht, "hr": w.hr, "S": w.S, "seed": w.vix_seed,
                     "block": w.block, "k": w.k, "n_obs": w.n_obs})
        zs.append(z.cpu().numpy())
        del z
    bs = BatchedSiting(inst)
    bs.run()
    torch.cuda.synchronize()
    for w, it, zh, b, (ch, gn, C) in zip(ws_, inst, zs, bs.bufs, bs.results()):
        v = b["vix"].cpu().numpy()
        posts = _seeded_posts(w.H, w.W, 300, 7)
        assert (v.reshape(-1)[posts] == O.vix_posts(zh, w.R, w.ht, w.hr, w.S, w.vix_seed, posts)).all(), w.name
        cand = O.findmax(v, w.block, w.k)
        assert b["cand"].cpu().numpy().tolist() == cand.tolist(), w.name
        bm = b["bm"].cpu().numpy().view(np.uint32)
        och, ogn, oC = O.site(bm, cand, w.H, w.W, w.R, w.n_obs)
        assert ch.cpu().numpy().tolist() == och.tolist(), w.name
        assert gn.cpu().numpy().tolist() == ogn.tolist(), w.name
        assert (C.cpu().numpy().view(np.uint32) == oC).all(), w.name
