"""The leader cluster's multi-winner rounds (several greedy steps per round,
each candidate accepted while it lies more than 2R from the round's other
winners) against the oracle's one-step-at-a-time lazy greedy: observers,
gains and cumulative viewshed bit for bit."""
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


def _case(O, seed, H, W, R, ncand, zr=900, lattice=None):
    z = T.spectral_fbm(H, W, 0.8, seed, 0, zr).numpy()
    rng = np.random.default_rng(seed)
    if lattice:
        ys, xs = np.meshgrid(np.arange(0, H, lattice), np.arange(0, W, lattice), indexing="ij")
        cand = (ys * W + xs).ravel().astype(np.int64)
        cand = cand[rng.permutation(len(cand))[:ncand]]
    else:
        cand = rng.choice(H * W, ncand, replace=False).astype(np.int64)
    bm, _ = O.viewshed(z, R, 10, 10, cand, threads=8)
    return cand, bm


def _run(V, bm, cand, H, W, R, n_obs, multi, q=0, target=0.0, cum=None):
    V.tune_set(V.VS_TUNE_SITE_MULTI, R, 0 if multi else 1)
    V.tune_set(V.VS_TUNE_SITE_CLUSTER, R, q)
    try:
        out = V.site(torch.as_tensor(bm.view(np.int32)).cuda(), torch.as_tensor(cand).cuda(), H, W, R,
                     n_obs, target=target, cum=cum)
        torch.cuda.synchronize()
    finally:
        V.tune_set(V.VS_TUNE_SITE_MULTI, R, 0)
        V.tune_set(V.VS_TUNE_SITE_CLUSTER, R, 0)
    return out


def _check(got, want):
    gch, ggn, gC, t = got
    ch, gn, C = want
    assert t >= 0, t
    assert t == len(ch)
    assert gch[:t].cpu().numpy().tolist() == ch.tolist()
    assert ggn[:t].cpu().numpy().tolist() == gn.tolist()
    assert (gC.cpu().numpy().view(np.uint32) == C).all()


# spread candidates (long rounds), dense candidates (many pairs per winner:
# lists overflow and a round takes several), R = 40 and R = 100 (bitmap rows
# of 4 and 8 words), grids whose width is not a multiple of 32
CASES = [
    (11, 1500, 1530, 40, 1400, 700, 37),      # a lattice of spread candidates
    (12, 900, 950, 100, 2500, 600, 17),       # 2500 of a stride-17 lattice
    (13, 400, 420, 40, 4000, 900, None),      # dense: thousands of pairs per round
    (14, 301, 333, 100, 1200, 400, None),     # dense, windows clipped by the edges
]


@pytest.mark.parametrize("seed,H,W,R,ncand,nobs,lat", CASES)
def test_multi_matches_oracle(V, O, seed, H, W, R, ncand, nobs, lat):
    cand, bm = _case(O, seed, H, W, R, ncand, lattice=lat)
    want = O.site(bm, cand, H, W, R, nobs)
    _check(_run(V, bm, cand, H, W, R, nobs, True), want)
    _check(_run(V, bm, cand, H, W, R, nobs, False), want)


@pytest.mark.parametrize("q", [2, 4, 8, 16])
def test_multi_cluster_sizes(V, O, q):
    """One worker CTA (q = 2) up to 15 (q = 16)."""
    H, W, R = 900, 950, 100
    cand, bm = _case(O, 21, H, W, R, 1800, lattice=19)
    want = O.site(bm, cand, H, W, R, 500)
    _check(_run(V, bm, cand, H, W, R, 500, True, q=q), want)


@pytest.mark.parametrize("target", [0.3, 0.8, 0.999])
def test_multi_coverage_stop(V, O, target):
    """The coverage stop is checked before every winner of a round."""
    H, W, R = 700, 760, 40
    cand, bm = _case(O, 31, H, W, R, 2000, lattice=13)
    want = O.site(bm, cand, H, W, R, 2000, target=target)
    _check(_run(V, bm, cand, H, W, R, 2000, True, target=target), want)


def test_multi_resume_and_exhaustion(V, O):
    """Resume from a saved cumulative viewshed mid-sequence; run until every
    gain is zero (n_obs above the number of useful candidates)."""
    H, W, R = 500, 530, 40
    cand, bm = _case(O, 41, H, W, R, 900, lattice=11)
    full = O.site(bm, cand, H, W, R, 900)
    a = _run(V, bm, cand, H, W, R, 137, True)
    b = _run(V, bm, cand, H, W, R, 900, True, cum=a[2].clone())
    ta, tb = a[3], b[3]
    assert a[0][:ta].cpu().numpy().tolist() + b[0][:tb].cpu().numpy().tolist() == full[0].tolist()
    assert (b[2].cpu().numpy().view(np.uint32) == full[2]).all()
    assert ta + tb == len(full[0]) < 900


def test_multi_duplicate_posts(V, O):
    """Candidates sharing a post are 0 apart: never winners of one round."""
    H, W, R = 400, 410, 40
    cand, bm = _case(O, 51, H, W, R, 600, lattice=9)
    cand2 = np.concatenate([cand, cand[:50]])
    bm2 = np.concatenate([bm, bm[:50]])
    want = O.site(bm2, cand2, H, W, R, 300)
    _check(_run(V, bm2, cand2, H, W, R, 300, True), want)
