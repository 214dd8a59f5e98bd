"""Bit-exact parity of the CUDA path (through the C ABI) with the CPU oracle,
on seeded inputs that span several tiles and ragged tails, every ROI regime
(single window, halves, quadrants, 32- and 64-bit products) and the edge
cases (borders, corners, H != W, odd widths, empty and invalid inputs)."""
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


def _grid(V, z):
    return V.Grid.from_tensor(torch.as_tensor(z), "cuda")


def _np(t):
    return t.cpu().numpy()


# ------------------------------------------------------------------ vix
@pytest.mark.parametrize("H,W,R,S,ht,hr,zr", [
    (67, 45, 7, 10, 10, 10, 200),       # ragged tails in both directions
    (130, 200, 50, 10, 10, 10, 1000),   # several tiles, single window
    (96, 170, 100, 10, 5, 12, 2000),    # one-window R=100
    (90, 75, 150, 12, 10, 10, 3000),    # halves
    (70, 66, 200, 20, 10, 10, 3000),    # halves, R larger than the grid
    (80, 90, 250, 10, 20, 3, 1000),     # quadrants
    (33, 41, 3, 255, 0, 0, 50),         # S = 255
    (40, 40, 5, 0, 10, 10, 100),        # S = 0
])
def test_vix_parity(V, O, H, W, R, S, ht, hr, zr):
    z = T.spectral_fbm(H, W, 0.8, 100 + R + H, 0, zr).numpy()
    seed = 0xABCDEF + R
    want = O.vix(z, R, ht, hr, S, seed, threads=8)
    got = _np(V.vix(_grid(V, z), R, ht, hr, S, seed))
    assert (got == want).all(), np.argwhere(got != want)[:10]


def test_vix_extreme_elevations(V, O):
    rng = np.random.default_rng(3)
    z = rng.integers(-32768, 32768, (50, 61)).astype(np.int16)
    want = O.vix(z, 9, 100000, -100000, 16, 5)
    got = _np(V.vix(_grid(V, z), 9, 100000, -100000, 16, 5))
    assert (got == want).all()


def test_vix_flat_interior(V):
    z = np.full((120, 140), 300, np.int16)
    got = _np(V.vix(_grid(V, z), 20, 10, 10, 10, 1))
    assert (got[20:-20, 20:-20] == 10).all()


# ------------------------------------------------------------------ findmax
@pytest.mark.parametrize("H,W,b,k", [(100, 100, 25, 1), (130, 77, 16, 3), (64, 64, 7, 20),
                                     (33, 100, 40, 2), (5, 5, 1, 1), (300, 257, 64, 4),
                                     # rows and blocks on 16-byte boundaries: the 16-post kernel
                                     (320, 480, 48, 4), (96, 256, 16, 8), (200, 496, 64, 5),
                                     (70, 1600, 800, 3), (50, 1056, 544, 8)])
def test_findmax_parity(V, O, H, W, b, k):
    rng = np.random.default_rng(H + W + b + k)
    v = rng.integers(0, 6, (H, W)).astype(np.uint8)   # heavy ties
    want = O.findmax(v, b, k)
    got = _np(V.findmax(torch.as_tensor(v).cuda(), b, k))
    assert got.tolist() == want.tolist()


@pytest.mark.parametrize("H,W,s,b,k", [(200, 150, 8, 40, 2), (97, 131, 5, 23, 3), (64, 64, 16, 64, 1)])
def test_findmax_f32_parity(V, O, H, W, s, b, k):
    rng = np.random.default_rng(7)
    sc = rng.random(((H + s - 1) // s, (W + s - 1) // s)).astype(np.float32)
    sc[::3, ::2] = 0.5                                     # ties
    sc[1, 1] = -0.0
    sc[2, 2] = 0.0
    sc[0, 1] = 0.0                                         # +0 beside -0 in one block
    hs, ws = sc.shape
    bits = sc.view(np.uint32)
    bits[hs - 1, ws - 1] = 0x7FC00000                      # +NaN: above +inf
    bits[hs - 1, 0] = 0xFFC00000                           # -NaN: below -inf
    sc[0, ws - 1] = np.inf
    sc[hs - 2, 1] = -np.inf
    want = O.findmax_f32(sc, H, W, s, b, k)
    got = _np(V.findmax_f32(torch.as_tensor(sc).cuda(), H, W, s, b, k))
    assert got.tolist() == want.tolist()


# ------------------------------------------------------------------ viewshed
def _cands(H, W, n, seed):
    rng = np.random.default_rng(seed)
    edge = [0, W - 1, (H - 1) * W, H * W - 1, (H // 2) * W, (H // 2) * W + W - 1, W // 2,
            (H - 1) * W + W // 2, 1 * W + 1, (H - 2) * W + W - 2]
    return np.array(edge + rng.integers(0, H * W, n).tolist(), np.int64)


@pytest.mark.parametrize("H,W,R,ht,hr,zr", [
    (40, 37, 1, 10, 10, 100), (40, 37, 2, 10, 10, 100), (41, 39, 3, 0, 0, 100),
    (63, 71, 7, 10, 10, 300), (250, 237, 50, 10, 10, 1000), (300, 333, 100, 10, 10, 2000),
    (320, 301, 150, 10, 10, 3000), (420, 411, 200, 10, 10, 3000), (530, 517, 250, 30, 5, 1000),
    (150, 90, 100, 10, 10, 500),        # grid narrower than the window
])
def test_viewshed_parity(V, O, H, W, R, ht, hr, zr):
    z = T.spectral_fbm(H, W, 0.8, 7 * R + H, 0, zr).numpy()
    cand = _cands(H, W, 40, R)
    bw, aw = O.viewshed(z, R, ht, hr, cand, threads=8)
    bm, area = V.viewshed(_grid(V, z), R, ht, hr, torch.as_tensor(cand).cuda())
    got = _np(bm).view(np.uint32)
    assert (_np(area) == aw).all()
    assert (got == bw).all(), np.argwhere(got != bw)[:5]


def test_viewshed_spiky_extremes(V, O):
    rng = np.random.default_rng(11)
    z = rng.integers(-32768, 32768, (90, 95)).astype(np.int16)
    cand = _cands(90, 95, 20, 5)
    for R, ht, hr in [(12, 0, 0), (30, 100000, -100000), (45, -5, 7)]:
        bw, aw = O.viewshed(z, R, ht, hr, cand)
        bm, area = V.viewshed(_grid(V, z), R, ht, hr, torch.as_tensor(cand).cuda())
        assert (_np(bm).view(np.uint32) == bw).all() and (_np(area) == aw).all()


def test_viewshed_invalid_and_empty(V):
    z = np.zeros((30, 30), np.int16)
    g = _grid(V, z)
    cand = torch.tensor([-1, 900, 5], dtype=torch.int64, device="cuda")
    bm, area = V.viewshed(g, 4, 1, 1, cand)
    a = _np(area)
    assert a[0] == -1 and a[1] == -1 and a[2] > 0
    assert (_np(bm)[:2] == 0).all()
    bm, area = V.viewshed(g, 4, 1, 1, torch.zeros(0, dtype=torch.int64, device="cuda"))
    assert area.numel() == 0


# ------------------------------------------------------------------ site
def _site_case(O, seed, H, W, R, ncand, zr=500):
    z = T.spectral_fbm(H, W, 0.8, seed, 0, zr).numpy()
    rng = np.random.default_rng(seed)
    cand = rng.choice(H * W, ncand, replace=False).astype(np.int64)
    bm, area = O.viewshed(z, R, 10, 10, cand, threads=8)
    return cand, bm


@pytest.mark.parametrize("seed,H,W,R,ncand,nobs", [
    (1, 60, 70, 8, 40, 30), (2, 200, 190, 20, 300, 120), (3, 257, 301, 50, 500, 200),
    (4, 150, 130, 7, 2000, 2000), (5, 400, 420, 100, 150, 40)])
def test_site_parity(V, O, seed, H, W, R, ncand, nobs):
    cand, bm = _site_case(O, seed, H, W, R, ncand)
    ch, gn, C = O.site(bm, cand, H, W, R, nobs)
    gch, ggn, gC, t = V.site(torch.as_tensor(bm.view(np.int32)).cuda(), torch.as_tensor(cand).cuda(),
                             H, W, R, nobs)
    assert t == len(ch)
    assert _np(gch).tolist() == ch.tolist()
    assert _np(ggn).tolist() == gn.tolist()
    assert (_np(gC).view(np.uint32) == C).all()


@pytest.mark.slow
def test_site_parity_many_candidates(V, O):
    """More candidates than one CTA's shared memory holds: the cluster path."""
    H, W, R = 600, 620, 3
    cand, bm = _site_case(O, 31, H, W, R, 70000)
    ch, gn, C = O.site(bm, cand, H, W, R, 3000)
    gch, ggn, gC, t = V.site(torch.as_tensor(bm.view(np.int32)).cuda(), torch.as_tensor(cand).cuda(),
                             H, W, R, 3000)
    assert _np(gch).tolist() == ch.tolist() and _np(ggn).tolist() == gn.tolist()
    assert (_np(gC).view(np.uint32) == C).all()


@pytest.fixture(scope="module")
def r100_case(O):
    """R = 100 (bitmap rows of 8 words: the leader-cluster loop's vector
    refresh), 2600 candidates on a 600 x 620 grid, so that a winner's band
    (slots within 2R rows) spans more than 1024 slots and a step takes several
    rounds."""
    H, W, R = 600, 620, 100
    cand, bm = _site_case(O, 41, H, W, R, 2600, zr=900)
    return H, W, R, cand, bm


@pytest.mark.parametrize("q", [0, 1, 2, 4, 16])
def test_site_leader_cluster_by_tuning(V, O, r100_case, q):
    """Every cluster size of the leader-cluster loop (0 = default, 1 = one
    CTA) gives the oracle's observers, gains and cumulative viewshed."""
    H, W, R, cand, bm = r100_case
    ch, gn, C = O.site(bm, cand, H, W, R, 300)
    V.tune_set(V.VS_TUNE_SITE_CLUSTER, R, q)
    try:
        gch, ggn, gC, t = V.site(torch.as_tensor(bm.view(np.int32)).cuda(), torch.as_tensor(cand).cuda(),
                                 H, W, R, 300)
    finally:
        V.tune_set(V.VS_TUNE_SITE_CLUSTER, R, 0)
    assert t == len(ch)
    assert _np(gch).tolist() == ch.tolist() and _np(ggn).tolist() == gn.tolist()
    assert (_np(gC).view(np.uint32) == C).all()


def test_site_leader_cluster_target_and_resume(V, O, r100_case):
    H, W, R, cand, bm = r100_case
    tb = torch.as_tensor(bm.view(np.int32)).cuda()
    tc = torch.as_tensor(cand).cuda()
    for target in (0.4, 0.9):
        ch, gn, C = O.site(bm, cand, H, W, R, 2600, target=target)
        gch, ggn, gC, t = V.site(tb, tc, H, W, R, 2600, target=target)
        assert _np(gch).tolist() == ch.tolist() and (_np(gC).view(np.uint32) == C).all()
    full = O.site(bm, cand, H, W, R, 90)
    a = V.site(tb, tc, H, W, R, 40)
    b = V.site(tb, tc, H, W, R, 50, cum=a[2].clone())
    assert _np(a[0]).tolist() + _np(b[0]).tolist() == full[0].tolist()
    assert (_np(b[2]).view(np.uint32) == full[2]).all()


def test_site_duplicate_and_invalid_candidates(V, O):
    H, W, R = 90, 110, 6
    cand, bm = _site_case(O, 41, H, W, R, 80)
    cand2 = np.concatenate([cand, cand[:10]])             # duplicated posts
    bm2 = np.concatenate([bm, bm[:10]])
    ch, gn, C = O.site(bm2, cand2, H, W, R, 50)
    gch, ggn, gC, t = V.site(torch.as_tensor(bm2.view(np.int32)).cuda(), torch.as_tensor(cand2).cuda(),
                             H, W, R, 50)
    assert _np(gch).tolist() == ch.tolist() and (_np(gC).view(np.uint32) == C).all()


def test_site_coverage_target_and_resume(V, O):
    H, W, R = 180, 200, 15
    cand, bm = _site_case(O, 9, H, W, R, 400)
    tb = torch.as_tensor(bm.view(np.int32)).cuda()
    tc = torch.as_tensor(cand).cuda()
    for target in (0.3, 0.6, 0.95):
        ch, gn, C = O.site(bm, cand, H, W, R, 400, target=target)
        gch, ggn, gC, t = V.site(tb, tc, H, W, R, 400, target=target)
        assert _np(gch).tolist() == ch.tolist() and (_np(gC).view(np.uint32) == C).all()
    # resume: 25 observers then 35 more from the returned cumulative viewshed
    full = O.site(bm, cand, H, W, R, 60)
    a = V.site(tb, tc, H, W, R, 25)
    b = V.site(tb, tc, H, W, R, 35, cum=a[2].clone())
    assert _np(a[0]).tolist() + _np(b[0]).tolist() == full[0].tolist()
    assert (_np(b[2]).view(np.uint32) == full[2]).all()


def test_site_gains_dense(V, O):
    H, W, R = 120, 150, 20
    cand, bm = _site_case(O, 13, H, W, R, 200)
    ch, gn, C = O.site(bm, cand, H, W, R, 10)
    g = _np(V.site_gains(torch.as_tensor(bm.view(np.int32)).cuda(), torch.as_tensor(cand).cuda(),
                         H, W, R, torch.as_tensor(C.view(np.int32)).cuda()))
    # popcount(V_c AND NOT C) in plain numpy
    PR = (2 * R) // 32 + 2
    for c in range(len(cand)):
        cx, cy = cand[c] % W, cand[c] // W
        gw0 = (cx - R) // 32
        s = 0
        for r in range(2 * R + 1):
            y = cy - R + r
            if not 0 <= y < H:
                continue
            for w in range(PR):
                gw = gw0 + w
                if 0 <= gw < C.shape[1]:
                    s += bin(int(bm[c, r, w]) & ~int(C[y, gw]) & 0xFFFFFFFF).count("1")
        assert g[c] == s


def test_site_no_candidates(V):
    cum = torch.zeros((10, 1), dtype=torch.int32, device="cuda")
    ch, gn, C, t = V.site(torch.zeros((0, 3, 2), dtype=torch.int32, device="cuda"),
                          torch.zeros(0, dtype=torch.int64, device="cuda"), 10, 10, 1, 5, cum=cum)
    assert t == 0


# ------------------------------------------------------------------ whole pipeline
@pytest.mark.slow
def test_pipeline_small_workload_bit_exact(V, O):
    """The 1000^2 / R=50 workload end to end: vix -> findmax -> viewshed -> site."""
    from synth import workloads as WL
    w = WL.SMALL
    z = w.make_terrain().numpy()
    g = _grid(V, z)
    v = V.vix(g, w.R, w.ht, w.hr, w.S, w.vix_seed)
    ov = O.vix(z, w.R, w.ht, w.hr, w.S, w.vix_seed, threads=16)
    assert (_np(v) == ov).all()
    cand = V.findmax(v, w.block, w.k)
    ocand = O.findmax(ov, w.block, w.k)
    assert _np(cand).tolist() == ocand.tolist() and len(ocand) == 1600
    bm, area = V.viewshed(g, w.R, w.ht, w.hr, cand)
    obm, oarea = O.viewshed(z, w.R, w.ht, w.hr, ocand, threads=16)
    assert (_np(bm).view(np.uint32) == obm).all() and (_np(area) == oarea).all()
    ch, gn, C, t = V.site(bm, cand, w.H, w.W, w.R, w.n_obs)
    och, ogn, oC = O.site(obm, ocand, w.H, w.W, w.R, w.n_obs)
    assert _np(ch).tolist() == och.tolist() and _np(gn).tolist() == ogn.tolist()
    assert (_np(C).view(np.uint32) == oC).all()


def test_bounded_wait_reports_timeout_and_context_survives(V):
    """A barrier nothing completes: the kernel's bounded wait gives up, the
    status word says VS_ERR_TIMEOUT, and the next launches still work."""
    assert V.selftest_wait_timeout(4096) == V.VS_ERR_TIMEOUT
    z = np.zeros((20, 20), np.int16)
    bm, area = V.viewshed(_grid(V, z), 3, 1, 1, torch.tensor([210], dtype=torch.int64, device="cuda"))
    assert int(area.item()) == 29
