"""vs_site_ex -- intervisible transmitters and weighted receivers (the
extensions named in Sec. "Prior art") -- bit-exact with the oracle's plain
greedy, through the C ABI."""
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


def _np(t):
    return t.cpu().numpy()


def _case(O, seed, H, W, R, n, zr=900, ht=10, hr=10):
    z = T.spectral_fbm(H, W, 0.8, seed, 0, zr).numpy()
    rng = np.random.default_rng(seed)
    cand = rng.choice(H * W, n, replace=False).astype(np.int64)
    cand[:3] = [0, H * W - 1, (H // 2) * W]
    cand[7] = cand[8]                       # a duplicate post
    bm, _ = O.viewshed(z, R, ht, hr, cand, threads=8)
    # a candidate outside the grid (empty bitmap): never chosen
    cand = np.concatenate([cand[:5], [H * W + 3], cand[5:]]).astype(np.int64)
    bm = np.concatenate([bm[:5], np.zeros_like(bm[:1]), bm[5:]])
    return z, cand, bm


@pytest.mark.parametrize("H,W,R,n,n_obs,target,con,wtd", [
    (200, 230, 20, 500, 80, 0.0, True, False),
    (200, 230, 20, 500, 80, 0.0, False, True),
    (200, 230, 20, 500, 120, 0.0, True, True),
    (260, 240, 40, 700, 200, 0.5, True, False),   # coverage stop
    (260, 240, 40, 700, 200, 0.4, False, True),   # weighted coverage stop
    (600, 620, 100, 2600, 150, 0.0, True, True),
    (60, 70, 9, 80, 60, 0.0, True, False),        # runs out of eligible candidates
])
def test_site_ex_parity(V, O, H, W, R, n, n_obs, target, con, wtd):
    z, cand, bm = _case(O, 31 + R + n, H, W, R, n)
    rng = np.random.default_rng(R)
    wt = rng.integers(0, 256, (H, W)).astype(np.uint8) if wtd else None
    if wtd:
        wt[: H // 3, :] = 0                 # a third of the terrain weighs nothing
    ch, gn, C = O.site_ex(bm, cand, H, W, R, n_obs, target, z=z if con else None, ht=25,
                          weight=wt)
    grid = V.Grid.from_tensor(torch.as_tensor(z), "cuda") if con else None
    gch, ggn, gC, t = V.site_ex(torch.as_tensor(bm.view(np.int32)).cuda(), torch.as_tensor(cand).cuda(), H, W, R,
                                n_obs, target, grid=grid, ht=25,
                                weight=torch.as_tensor(wt).cuda() if wtd else None)
    assert t == len(ch)
    assert _np(gch).tolist() == ch.tolist() and _np(ggn).tolist() == gn.tolist()
    assert (_np(gC).view(np.uint32) == C).all()


def test_site_ex_without_options_is_vs_site(V, O):
    H, W, R = 200, 230, 20
    z, cand, bm = _case(O, 5, H, W, R, 400)
    b = torch.as_tensor(bm.view(np.int32)).cuda()
    c = torch.as_tensor(cand).cuda()
    a = V.site(b, c, H, W, R, 60)
    e = V.site_ex(b, c, H, W, R, 60)
    assert a[3] == e[3] and (_np(a[0]) == _np(e[0])).all() and (_np(a[2]) == _np(e[2])).all()


def test_site_ex_wall(V, O):
    """A wall splits the terrain: after the first transmitter nothing behind
    the wall may be chosen."""
    H, W, R = 9, 42, 40
    z = np.zeros((H, W), np.int16)
    z[:, 20] = 1000
    cand = np.array([4 * W + 5, 4 * W + 35, 4 * W + 12], np.int64)
    bm, _ = O.viewshed(z, R, 10, 0, cand)
    grid = V.Grid.from_tensor(torch.as_tensor(z), "cuda")
    b = torch.as_tensor(bm.view(np.int32)).cuda()
    c = torch.as_tensor(cand).cuda()
    ch, gn, _, t = V.site_ex(b, c, H, W, R, 3)
    assert _np(ch).tolist() == [4 * W + 35, 4 * W + 5] and _np(gn).tolist() == [198, 180]
    ch, gn, _, t = V.site_ex(b, c, H, W, R, 3, grid=grid, ht=10)
    assert _np(ch).tolist() == [4 * W + 35] and _np(gn).tolist() == [198]
