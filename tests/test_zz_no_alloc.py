"""vs_site_noalloc: the site step for callers that cannot allocate device
memory (host applications that own every allocation through their own pool,
latency-critical loops that cannot take cudaMalloc's implicit synchronisation,
bindings without a device allocator).  Its scratch is a static device array
inside the library; this checks, through the C ABI, that two calls in a row
give exactly what vs_site gives with a caller-provided workspace.

Kept in a file that pytest collects last, so that a failure here cannot hide
the rest of the suite."""
import ctypes

import numpy as np
import pytest
import torch

from synth import terrain as T

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _case(seed, H, W, R, ncand, with_host=False):
    from oracle import oracle as O
    z = T.spectral_fbm(H, W, 0.8, seed, 0, 500).numpy()
    rng = np.random.default_rng(seed)
    cand = rng.choice(H * W, ncand, replace=False).astype(np.int64)
    bm, _ = O.viewshed(z, R, 10, 10, cand, threads=8)
    dev = torch.as_tensor(bm.view(np.int32)).cuda(), torch.as_tensor(cand).cuda()
    return dev + ((bm, cand) if with_host else ())


def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_16783_gb300 import _build
    _build.build()
    from paper_2006_16783_gb300 import vshed
    return vshed, vshed.lib()


def _same(got, want):
    assert got[0].tolist() == want[0].tolist()
    assert got[1].tolist() == want[1].tolist()
    assert (got[2] == want[2]).all()


def _run(L, fn, bm, cand, H, W, R, n_obs, target, ws=None):
    chosen = torch.full((n_obs,), -7, dtype=torch.int64, device="cuda")
    gains = torch.full((n_obs,), -7, dtype=torch.int64, device="cuda")
    cum = torch.zeros((H, (W + 31) // 32), dtype=torch.int32, device="cuda")
    nch = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    args = [_p(bm), _p(cand), cand.numel(), H, W, R, n_obs, float(target), _p(chosen), _p(gains),
            _p(cum), _p(nch)]
    if ws is None:
        rc = fn(*args, st)
    else:
        rc = fn(*args, _p(ws), ws.numel(), st)
    assert rc == 0, rc
    torch.cuda.synchronize()
    t = int(nch.item())
    assert 0 <= t <= n_obs, t                 # a negative count is a device error code
    return chosen[:t].cpu().numpy(), gains[:t].cpu().numpy(), cum.cpu().numpy()


@pytest.mark.parametrize("target", [0.0, 0.7])
def test_site_noalloc_matches_site(target):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_16783_gb300 import _build
    _build.build()
    from paper_2006_16783_gb300 import vshed
    L = vshed.lib()
    H, W, R = 230, 250, 20
    bm, cand = _case(21, H, W, R, 600)
    ws = torch.empty(L.vs_site_workspace(cand.numel(), R), dtype=torch.uint8, device="cuda")
    want = _run(L, L.vs_site, bm, cand, H, W, R, 150, target, ws)
    for _ in range(2):                       # two calls in a row share the static scratch
        got = _run(L, L.vs_site_noalloc, bm, cand, H, W, R, 150, target)
        assert got[0].tolist() == want[0].tolist()
        assert got[1].tolist() == want[1].tolist()
        assert (got[2] == want[2]).all()
    # a second, different problem right after: nothing stale leaks through
    bm2, cand2 = _case(22, 120, 140, 9, 300)
    ws2 = torch.empty(L.vs_site_workspace(cand2.numel(), 9), dtype=torch.uint8, device="cuda")
    want2 = _run(L, L.vs_site, bm2, cand2, 120, 140, 9, 60, target, ws2)
    got2 = _run(L, L.vs_site_noalloc, bm2, cand2, 120, 140, 9, 60, target)
    assert got2[0].tolist() == want2[0].tolist() and (got2[2] == want2[2]).all()


def test_site_noalloc_rejects_oversize():
    from paper_2006_16783_gb300 import _build
    _build.build()
    from paper_2006_16783_gb300 import vshed
    L = vshed.lib()
    n = 1 << 20                               # needs 4 MiB of scratch: over the limit
    assert L.vs_site_workspace(n, 5) > (1 << 20)
    dummy = ctypes.c_void_p(256)
    rc = L.vs_site_noalloc(dummy, dummy, n, 100, 100, 5, 10, 0.0, dummy, dummy, dummy, dummy, None)
    assert rc == vshed.VS_ERR_RANGE


@pytest.mark.parametrize("loop", ["leader_cluster", "lazy_grid"])
def test_site_noalloc_other_loops(loop):
    """The greedy loops that keep more of their state in the scratch: the
    leader cluster (bitmap rows of whole 16-byte vectors, R = 40) and the lazy
    greedy on the whole GPU (its grid-barrier block and work list), each run
    twice in a row through vs_site_noalloc against vs_site, and once against
    the oracle's lazy greedy."""
    from oracle import oracle as O
    vshed, L = _lib()
    H, W, R = 260, 240, 40
    bm, cand, hbm, hcand = _case(31, H, W, R, 500, with_host=True)
    if loop == "lazy_grid":
        vshed.tune_set(vshed.VS_TUNE_SITE_LAZY, R, 1)
    try:
        ws = torch.empty(L.vs_site_workspace(cand.numel(), R), dtype=torch.uint8, device="cuda")
        want = _run(L, L.vs_site, bm, cand, H, W, R, 90, 0.0, ws)
        for _ in range(2):
            _same(_run(L, L.vs_site_noalloc, bm, cand, H, W, R, 90, 0.0), want)
    finally:
        vshed.tune_set(vshed.VS_TUNE_SITE_LAZY, R, 0)
    och, ogn, oC = O.site(hbm, hcand, H, W, R, 90)
    _same(want, (och, ogn, oC.view(np.int32)))


def test_site_noalloc_at_the_limit():
    """37,439 candidates fill the 1 MiB array exactly: two calls in a row equal
    vs_site; 37,440 is refused with VS_ERR_RANGE."""
    vshed, L = _lib()
    H, W, R = 300, 300, 9
    n = 37439
    assert L.vs_site_workspace(n, R) <= 1 << 20 < L.vs_site_workspace(n + 1, R)
    bm, cand = _case(41, H, W, R, n)
    ws = torch.empty(L.vs_site_workspace(n, R), dtype=torch.uint8, device="cuda")
    want = _run(L, L.vs_site, bm, cand, H, W, R, 300, 0.0, ws)
    for _ in range(2):
        _same(_run(L, L.vs_site_noalloc, bm, cand, H, W, R, 300, 0.0), want)
    big = torch.cat([cand, cand[:1]])
    bm2 = torch.cat([bm, bm[:1]])
    dummy = torch.zeros(400, dtype=torch.int64, device="cuda")
    rc = L.vs_site_noalloc(_p(bm2), _p(big), n + 1, H, W, R, 10, 0.0, _p(dummy), _p(dummy), _p(dummy),
                           _p(dummy), None)
    assert rc == vshed.VS_ERR_RANGE
