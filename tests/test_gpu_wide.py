"""Large ROIs: the banded viewshed kernel (windows that do not fit in shared
memory, the paper's R = 500..2000 regime of Sec. "Experiments") and the lazy
greedy site loop (gains or windows that do not fit in one cluster's shared
memory), bit-exact with the CPU oracle through the C ABI."""
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


def _posts(H, W, extra, seed):
    """Corners, edges, word-boundary columns and random interior posts."""
    pts = [(0, 0), (W - 1, 0), (0, H - 1), (W - 1, H - 1), (W // 2, H // 2), (1, H // 3),
           (W - 2, 2 * H // 3), (W // 3, 0), (31, 5), (32, H - 1), (33, 7)]
    rng = np.random.default_rng(seed)
    out = [y * W + x for x, y in pts if 0 <= x < W and 0 <= y < H]
    out += rng.integers(0, H * W, extra).tolist()
    return np.array(out, np.int64)


def _viewshed_vs_oracle(V, O, z, R, ht, hr, cand):
    bm, area = V.viewshed(_grid(V, z), R, ht, hr, torch.as_tensor(cand).cuda())
    wbm, warea = O.viewshed(z, R, ht, hr, cand, threads=8)
    assert (_np(area) == warea).all(), np.argwhere(_np(area) != warea)[:8]
    assert (_np(bm).view(np.uint32) == wbm).all()


@pytest.mark.parametrize("H,W,R,ht,hr,zr", [
    (700, 650, 300, 100, 10, 900),    # first ROI past the shared-memory quadrant
    (500, 900, 450, 10, 10, 2000),    # R close to the grid size
    (420, 380, 600, 100, 10, 1500),   # R larger than the grid
])
def test_wide_viewshed_parity(V, O, H, W, R, ht, hr, zr):
    assert V.vshed.viewshed_workspace(H, W, R, 1) > 0  # the banded path
    z = T.spectral_fbm(H, W, 0.8, 300 + R, 0, zr).numpy()
    _viewshed_vs_oracle(V, O, z, R, ht, hr, _posts(H, W, 13, R))


def test_wide_viewshed_r1000(V, O):
    """The paper's US-West ROI (R = 1000, h_t = 100, h_r = 10) on a ridged
    terrain larger than the window."""
    H, W, R = 2300, 2100, 1000
    z = T.ridged_multifractal(H, W, 17, 0, 2800, octaves=8).numpy()
    cand = np.array([0, (H // 2) * W + W // 2, (H - 1) * W + W - 1, 777 * W + 5, 1500 * W + 1999],
                    np.int64)
    _viewshed_vs_oracle(V, O, z, R, 100, 10, cand)


@pytest.mark.parametrize("R", [1, 2, 7, 33, 100, 150])
def test_wide_viewshed_forced_matches_staged(V, O, R):
    """The banded kernel forced on ROIs whose window fits gives the staged
    kernel's bitmaps (and the oracle's)."""
    H, W = 260, 310
    z = T.spectral_fbm(H, W, 0.8, 40 + R, 0, 1200).numpy()
    cand = _posts(H, W, 40, R)
    g = _grid(V, z)
    c = torch.as_tensor(cand).cuda()
    bm0, a0 = V.viewshed(g, R, 10, 10, c)
    V.tune_set(V.VS_TUNE_VIEWSHED_WIDE, R, 1)
    try:
        assert V.vshed.viewshed_workspace(H, W, R, 1) > 0
        bm1, a1 = V.viewshed(g, R, 10, 10, c)
    finally:
        V.tune_set(V.VS_TUNE_VIEWSHED_WIDE, R, 0)
    assert (_np(a0) == _np(a1)).all() and (_np(bm0) == _np(bm1)).all()
    wbm, warea = O.viewshed(z, R, 10, 10, cand)
    assert (_np(a1) == warea).all() and (_np(bm1).view(np.uint32) == wbm).all()


def test_wide_viewshed_invalid_and_empty(V):
    H, W, R = 300, 320, 300
    z = T.spectral_fbm(H, W, 0.8, 5, 0, 500).numpy()
    g = _grid(V, z)
    bm, area = V.viewshed(g, R, 10, 10, torch.tensor([-1, H * W, 5], dtype=torch.int64).cuda())
    a = _np(area)
    assert a[0] == -1 and a[1] == -1 and a[2] > 0
    assert not _np(bm[:2]).any()
    bm, area = V.viewshed(g, R, 10, 10, torch.empty(0, dtype=torch.int64).cuda())
    assert bm.shape[0] == 0


def test_wide_viewshed_workspace_checked(V):
    import ctypes
    H, W, R = 300, 320, 300
    z = T.spectral_fbm(H, W, 0.8, 5, 0, 500).numpy()
    g = _grid(V, z)
    need = V.vshed.viewshed_workspace(H, W, R, 1)
    cand = torch.tensor([5], dtype=torch.int64).cuda()
    bm = torch.empty((1, 2 * R + 1, V.vshed.words_per_row(R)), dtype=torch.int32, device="cuda")
    area = torch.empty(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(need - 1, dtype=torch.uint8, device="cuda")
    L = V.vshed.lib()
    rc = L.vs_viewshed(g.c(), R, 10, 10, ctypes.c_void_p(cand.data_ptr()), 1, ctypes.c_void_p(bm.data_ptr()),
                       ctypes.c_void_p(area.data_ptr()), ctypes.c_void_p(ws.data_ptr()), need - 1, None)
    assert rc == V.vshed.VS_ERR_WS


# ------------------------------------------------------------------ vix, warp-per-line kernel
@pytest.mark.parametrize("H,W,R,S,ht,hr,zr", [
    (150, 170, 300, 12, 100, 10, 1500),   # first ROI past the staged windows
    (120, 130, 500, 10, 100, 10, 2500),   # R larger than the grid
    (260, 240, 700, 10, 10, 10, 3000),
])
def test_wide_vix_parity(V, O, H, W, R, S, ht, hr, zr):
    assert V.vshed.vix_workspace(H, W, R, S) > 0
    z = T.spectral_fbm(H, W, 0.8, 500 + R, 0, zr).numpy()
    want = O.vix(z, R, ht, hr, S, 0x5EED + R, threads=8)
    g = _grid(V, z)
    got = _np(V.vix(g, R, ht, hr, S, 0x5EED + R))                    # transposed terrain in ws
    assert (got == want).all(), np.argwhere(got != want)[:8]
    out = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    V.vshed._check("vs_vix", V.vshed.lib().vs_vix(g.c(), R, ht, hr, S, 0x5EED + R, V.vshed._ptr(out),
                                                   V.vshed._stream()))  # no workspace: strided reads
    assert (_np(out) == want).all()


@pytest.mark.parametrize("R", [3, 50, 100])
def test_wide_vix_forced_matches_staged(V, R):
    """The warp-per-line kernel forced on ROIs the staged kernels cover gives
    the same counts and the same number of LOS crossings."""
    H, W, S = 300, 280, 10
    z = T.spectral_fbm(H, W, 0.8, 900 + R, 0, 1500).numpy()
    g = _grid(V, z)
    s0 = torch.zeros(1, dtype=torch.int64, device="cuda")
    a = V.vshed.vix_count(g, R, 10, 10, S, 99, s0)
    V.tune_set(V.VS_TUNE_VIX_TILE, R, 3)
    try:
        assert V.vshed.vix_workspace(H, W, R, S) > 0
        s1 = torch.zeros(1, dtype=torch.int64, device="cuda")
        b = V.vshed.vix_count(g, R, 10, 10, S, 99, s1)
    finally:
        V.tune_set(V.VS_TUNE_VIX_TILE, R, 0)
    assert (_np(a) == _np(b)).all()
    assert int(s0.item()) == int(s1.item()) > 0


# ------------------------------------------------------------------ lazy greedy
def _site_case(O, seed, H, W, R, n, zr=900, ht=10, hr=10):
    z = T.spectral_fbm(H, W, 0.8, seed, 0, zr).numpy()
    rng = np.random.default_rng(seed)
    cand = rng.choice(H * W, n, replace=False).astype(np.int64)
    cand[:3] = [0, H * W - 1, (H // 2) * W]
    cand[7] = cand[8]                     # a duplicate post
    bm, _ = O.viewshed(z, R, ht, hr, cand, threads=8)
    return z, cand, bm


def _site(V, bm, cand, H, W, R, n_obs, target=0.0, cum=None):
    return V.site(torch.as_tensor(bm.view(np.int32)).cuda(), torch.as_tensor(cand).cuda(), H, W, R, n_obs,
                  target, cum=cum)


@pytest.mark.parametrize("mode", [1, 2])   # the whole GPU, one CTA
@pytest.mark.parametrize("H,W,R,n,n_obs,target", [
    (300, 340, 20, 900, 200, 0.0),
    (600, 620, 100, 2600, 300, 0.0),
    (600, 620, 100, 2600, 400, 0.55),
    (90, 100, 9, 300, 500, 0.0),      # runs until the best gain is 0
    (40, 50, 6, 100, 30, 0.0),        # fewer candidates than SMs
])
def test_site_lazy_forced(V, O, H, W, R, n, n_obs, target, mode):
    _, cand, bm = _site_case(O, 11 + R, H, W, R, n)
    ch, gn, C = O.site(bm, cand, H, W, R, n_obs, target)
    V.tune_set(V.VS_TUNE_SITE_LAZY, R, mode)
    try:
        gch, ggn, gC, t = _site(V, bm, cand, H, W, R, n_obs, target)
    finally:
        V.tune_set(V.VS_TUNE_SITE_LAZY, R, 0)
    assert t == len(ch)
    assert _np(gch).tolist() == ch.tolist() and _np(ggn).tolist() == gn.tolist()
    assert (_np(gC).view(np.uint32) == C).all()


@pytest.mark.parametrize("mode", [1, 2])
def test_site_lazy_resume(V, O, mode):
    """Checkpoint / resume: two calls continuing from the returned cum give
    the sequence of one call."""
    H, W, R = 400, 380, 40
    _, cand, bm = _site_case(O, 23, H, W, R, 1200)
    ch, gn, C = O.site(bm, cand, H, W, R, 150)
    V.tune_set(V.VS_TUNE_SITE_LAZY, R, mode)
    try:
        c1, g1, cum, t1 = _site(V, bm, cand, H, W, R, 60)
        c2, g2, cum2, t2 = _site(V, bm, cand, H, W, R, 90, cum=cum)
    finally:
        V.tune_set(V.VS_TUNE_SITE_LAZY, R, 0)
    assert _np(c1).tolist() + _np(c2).tolist() == ch.tolist()
    assert _np(g1).tolist() + _np(g2).tolist() == gn.tolist()
    assert (_np(cum2).view(np.uint32) == C).all()


def test_site_lazy_auto_r1000(V, O):
    """R = 1000 bitmaps (512 KB each) do not fit any shared-memory loop: the
    call takes the lazy greedy by itself.  The paper's 95% coverage stop."""
    H, W, R = 2600, 2500, 1000
    z = T.ridged_multifractal(H, W, 29, 0, 2800, octaves=8).numpy()
    rng = np.random.default_rng(29)
    cand = rng.choice(H * W, 60, replace=False).astype(np.int64)
    bm, _ = O.viewshed(z, R, 100, 10, cand, threads=8)
    ch, gn, C = O.site(bm, cand, H, W, R, 60, 0.95)
    gch, ggn, gC, t = _site(V, bm, cand, H, W, R, 60, 0.95)
    assert t == len(ch)
    assert _np(gch).tolist() == ch.tolist() and _np(ggn).tolist() == gn.tolist()
    assert (_np(gC).view(np.uint32) == C).all()


def test_paper_regime_pipeline(V, O):
    """The paper's parameter regime on a small terrain: R = 500, h_t = 100,
    h_r = 10, blocks of side R/3 with 20 candidates each, 95% coverage target.
    Candidates come from the GPU's vix and findmax; viewsheds and sites are
    checked against the oracle."""
    H, W, R = 1000, 1000, 500
    z = T.ridged_multifractal(H, W, 31, 0, 1500, octaves=8).numpy()
    g = _grid(V, z)
    vix = V.vix(g, R, 100, 10, 10, 77)
    v = _np(vix)
    rng = np.random.default_rng(5)
    posts = np.concatenate([[0, W - 1, H * W - 1], rng.integers(0, H * W, 400)]).astype(np.int64)
    want = O.vix_posts(z, R, 100, 10, 10, 77, posts)
    assert (v.reshape(-1)[posts] == want).all()
    cand = V.findmax(vix, R // 3, 20)
    assert cand.numel() == V.vshed.lib().vs_findmax_count(H, W, 1, R // 3, 20)
    assert (_np(cand) == O.findmax(v, R // 3, 20)).all()
    bm, area = V.viewshed(g, R, 100, 10, cand)
    c = _np(cand)
    wbm, warea = O.viewshed(z, R, 100, 10, c, threads=8)
    assert (_np(area) == warea).all() and (_np(bm).view(np.uint32) == wbm).all()
    ch, gn, C = O.site(wbm, c, H, W, R, 400, 0.95)
    gch, ggn, gC, t = V.site(bm, cand, H, W, R, 400, 0.95)
    assert t == len(ch)
    assert _np(gch).tolist() == ch.tolist() and _np(ggn).tolist() == gn.tolist()
    assert (_np(gC).view(np.uint32) == C).all()


# ------------------------------------------------------------------ exact per-cell viewshed (R3)
@pytest.mark.parametrize("H,W,R,ht,hr,zr", [
    (70, 90, 7, 10, 10, 300),
    (160, 150, 30, 10, 10, 1200),
    (260, 300, 100, 100, 10, 2000),
    (420, 380, 300, 10, 10, 1500),    # beyond the staged windows
])
def test_viewshed_r3_parity(V, O, H, W, R, ht, hr, zr):
    z = T.spectral_fbm(H, W, 0.8, 700 + R, 0, zr).numpy()
    cand = _posts(H, W, 6, R)
    g = _grid(V, z)
    bm, area = V.viewshed_r3(g, R, ht, hr, torch.as_tensor(cand).cuda())
    got = _np(bm).view(np.uint32)
    for i, p in enumerate(cand):
        want = O.viewshed_brute(z, R, ht, hr, int(p))
        assert (got[i] == want).all(), (i, int(p))
        assert int(_np(area)[i]) == int(np.unpackbits(want.view(np.uint8)).sum())
    # without the transposed copy (strided reads): same bitmaps
    bm2 = torch.empty_like(bm)
    area2 = torch.empty_like(area)
    c = torch.as_tensor(cand).cuda()
    V.vshed._check("vs_viewshed_r3", V.vshed.lib().vs_viewshed_r3(
        g.c(), R, ht, hr, V.vshed._ptr(c), c.numel(), V.vshed._ptr(bm2), V.vshed._ptr(area2), None, 0,
        V.vshed._stream()))
    assert (_np(bm2) == _np(bm)).all() and (_np(area2) == _np(area)).all()


def test_viewshed_r3_flat_and_invalid(V, O):
    """Flat terrain: every disc cell in the grid is visible (grazing lines
    count); invalid candidates give empty bitmaps and area -1."""
    H, W, R = 120, 140, 25
    z = np.full((H, W), 300, np.int16)
    cand = np.array([60 * W + 70, 0, -1, H * W], np.int64)
    bm, area = V.viewshed_r3(_grid(V, z), R, 0, 0, torch.as_tensor(cand).cuda())
    a = _np(area)
    disc = sum(1 for dy in range(-R, R + 1) for dx in range(-R, R + 1) if dx * dx + dy * dy <= R * R)
    assert a[0] == disc
    assert a[1] == sum(1 for dy in range(0, R + 1) for dx in range(0, R + 1) if dx * dx + dy * dy <= R * R)
    assert a[2] == -1 and a[3] == -1 and not _np(bm[2:]).any()


# ------------------------------------------------------------------ extreme values
@pytest.mark.parametrize("R,ht,hr", [(4096, 100000, -100000), (700, -100000, 100000), (1500, 100000, 100000)])
def test_wide_extreme_values(V, O, R, ht, hr):
    """int16 extremes, the largest heights and the largest ROI: the 32-bit
    values with 64-bit products of the large-ROI kernels stay exact."""
    H, W = 150, 170
    rng = np.random.default_rng(R)
    z = rng.integers(-32768, 32768, (H, W)).astype(np.int16)
    z[:, 40] = 32767                       # a wall of the highest posts
    z[70, :] = -32768                      # a trench of the lowest
    cand = _posts(H, W, 5, R)
    _viewshed_vs_oracle(V, O, z, R, ht, hr, cand)
    want = O.vix(z, R, ht, hr, 10, 99, threads=8)
    got = _np(V.vix(_grid(V, z), R, ht, hr, 10, 99))
    assert (got == want).all()
    bm, _ = V.viewshed_r3(_grid(V, z), min(R, 200), ht, hr, torch.as_tensor(cand[:4]).cuda())
    for i, p in enumerate(cand[:4]):
        assert (_np(bm[i]).view(np.uint32) == O.viewshed_brute(z, min(R, 200), ht, hr, int(p))).all()


def test_launch_count_counts_library_kernels(V):
    """vs_launch_count grows by the kernels one call issues (a staged
    viewshed: one launch)."""
    H, W, R = 120, 130, 20
    z = T.spectral_fbm(H, W, 0.8, 3, 0, 500).numpy()
    g = _grid(V, z)
    c = torch.tensor([5, 700, 4000], dtype=torch.int64).cuda()
    V.viewshed(g, R, 10, 10, c)
    n0 = V.launch_count()
    V.viewshed(g, R, 10, 10, c)
    assert V.launch_count() - n0 == 1
