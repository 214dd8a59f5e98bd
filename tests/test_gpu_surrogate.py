"""Learned proposal end to end on small terrains: exact labels from the
viewshed kernel, a short training run whose loss falls, and the network's
error against the exact index compared with the sampled-vix estimate."""
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


@pytest.mark.parametrize("H,W,R,wide", [(260, 240, 30, 0), (97, 300, 100, 0), (260, 240, 30, 1),
                                         (700, 650, 300, 0)])
def test_exact_labels_match_oracle(V, O, H, W, R, wide):
    """vs_exact_vix (labels of the learned proposal) bit for bit against the
    oracle's exact visibility index: interior, edge and corner posts, a grid
    narrower than the ROI, the banded large-ROI path (forced at R = 30, and
    R = 300 beyond shared memory), posts outside the grid."""
    from paper_2006_16783_gb300 import surrogate as S
    z = T.spectral_fbm(H, W, 0.8, 17 + R, 0, 800).numpy()
    g = V.Grid.from_tensor(torch.as_tensor(z), "cuda")
    posts = S.sample_posts(H, W, 300, 0, 5, "cuda")
    edge = torch.tensor([0, W - 1, (H - 1) * W, H * W - 1, W // 2, (H // 2) * W, -3, H * W],
                        dtype=torch.int64, device="cuda")
    posts = torch.cat([posts, edge])
    if wide:
        V.tune_set(V.VS_TUNE_VIEWSHED_WIDE, R, 1)
    try:
        lab = S.exact_vix(g, posts, R, 10, 10, chunk=128).cpu().numpy()
    finally:
        V.tune_set(V.VS_TUNE_VIEWSHED_WIDE, R, 0)
    want = O.exact_vix(z, R, 10, 10, posts.cpu().numpy(), threads=8)
    assert lab.view(np.uint32).tolist() == want.view(np.uint32).tolist()
    assert lab[-2] == -1.0 and lab[-1] == -1.0


@pytest.mark.slow
def test_training_reduces_loss_and_beats_sampling(V):
    from paper_2006_16783_gb300 import surrogate as S
    H, W, R = 1024, 1024, 50
    data = []
    for seed in (3000, 3001):
        z = T.spectral_fbm(H, W, 0.8, seed, 0, 1000, device="cuda")
        g = V.Grid(z.contiguous())
        posts = S.sample_posts(H, W, 30000, 32, seed, "cuda")
        data.append((g, posts, S.exact_vix(g, posts, R, 10, 10)))
    zt = T.spectral_fbm(H, W, 0.8, 3100, 0, 1000, device="cuda")
    gt = V.Grid(zt.contiguous())
    pt = S.sample_posts(H, W, 20000, 32, 9, "cuda")
    lt = S.exact_vix(gt, pt, R, 10, 10)
    tr = S.Trainer(S.init_master(0), batch=256, lr=2e-3)
    base = float((tr.predict(gt, pt) - lt).abs().mean())
    tr.fit(data, epochs=3, seed=1)
    mae = float((tr.predict(gt, pt) - lt).abs().mean())
    sampled = float((S.sampled_vix_fraction(gt, pt, R, 10, 10, 10, 77) - lt).abs().mean())
    print("held-out MAE: untrained %.4f, trained %.4f, sampled vix (S=10) %.4f" % (base, mae, sampled))
    assert mae < 0.7 * base
    assert mae < sampled
