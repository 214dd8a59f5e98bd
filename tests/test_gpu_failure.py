"""Failure paths on the GPU, without faulting or hanging it: bounded waits
that are made to run out report VS_ERR_TIMEOUT to the host, and the context
and the next call are unaffected."""
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


def test_lazy_grid_barrier_timeout_is_reported(V, O):
    """One CTA of the whole-GPU lazy greedy skips its first grid-barrier
    arrival (test tuning value, waits limited to 2000 polls): the other CTAs'
    waits run out, every CTA leaves, and the call reports VS_ERR_TIMEOUT in
    *n_chosen.  The same call afterwards gives the oracle's observers."""
    H, W, R = 260, 240, 40
    z = T.spectral_fbm(H, W, 0.8, 61, 0, 600).numpy()
    rng = np.random.default_rng(61)
    cand = rng.choice(H * W, 400, replace=False).astype(np.int64)
    bm, _ = O.viewshed(z, R, 10, 10, cand, threads=8)
    tb = torch.as_tensor(bm.view(np.int32)).cuda()
    tc = torch.as_tensor(cand).cuda()
    V.tune_set(V.VS_TUNE_SITE_LAZY, R, 1)
    try:
        V.tune_set(V.VS_TUNE_SITE_BARRIER_TEST, R, 2000)
        try:
            _, _, _, nch = V.site(tb, tc, H, W, R, 50, sync=False)
            torch.cuda.synchronize()
        finally:
            V.tune_set(V.VS_TUNE_SITE_BARRIER_TEST, R, 0)
        assert int(nch.item()) == V.VS_ERR_TIMEOUT
        ch, gn, C = O.site(bm, cand, H, W, R, 50)
        gch, ggn, gC, t = V.site(tb, tc, H, W, R, 50)
    finally:
        V.tune_set(V.VS_TUNE_SITE_LAZY, R, 0)
    assert t == len(ch)
    assert gch.cpu().numpy().tolist() == ch.tolist()
    assert ggn.cpu().numpy().tolist() == gn.tolist()
    assert (gC.cpu().numpy().view(np.uint32) == C).all()
