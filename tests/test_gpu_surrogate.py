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
    # patch step 2: the 65 x 65 input spans +-64 posts, the whole R = 50 ROI
    tr = S.Trainer(S.init_master(0), batch=256, lr=2e-3, patch_step=2)
    base = float((tr.predict(gt, pt) - lt).abs().mean())
    tr.fit(data, epochs=6, seed=1)
    mae = float((tr.predict(gt, pt) - lt).abs().mean())
    sampled = float((S.sampled_vix_fraction(gt, pt, R, 10, 10, 10, 77) - lt).abs().mean())
    print("held-out MAE: untrained %.4f, trained %.4f, sampled vix (S=10) %.4f" % (base, mae, sampled))
    assert mae < 0.7 * base
    assert mae < sampled


def test_backward_is_deterministic(V):
    """No floating-point atomics in the backward: the same batch gives
    bit-identical gradients and loss on every call."""
    from paper_2006_16783_gb300 import surrogate as S
    H = W = 260
    z = T.spectral_fbm(H, W, 0.8, 8, 0, 900)
    g = V.Grid.from_tensor(z, "cuda")
    posts = S.sample_posts(H, W, 300, 0, 2, "cuda")
    labels = torch.rand(posts.numel(), device="cuda")
    master = S.init_master(1)
    packed = V.cnn_pack(master)
    save = torch.empty(posts.numel() * V.cnn_save_bytes(), dtype=torch.uint8, device="cuda")
    V.cnn_forward(g, posts, packed, save=save, patch_step=2)
    outs = []
    for _ in range(3):
        gr = torch.zeros_like(master)
        loss = torch.zeros(1, device="cuda")
        V.cnn_backward(save, labels, master, gr, loss)
        outs.append((gr, loss))
    for gr, loss in outs[1:]:
        assert torch.equal(gr, outs[0][0]) and torch.equal(loss, outs[0][1])


def test_trainer_checkpoint_resume_bit_identical(V, tmp_path):
    """Three epochs in one run, and one epoch + checkpoint to a file + a new
    trainer loaded from it + the remaining two: identical weights, Adam
    moments and step."""
    from paper_2006_16783_gb300 import surrogate as S
    H = W = 300
    z = T.spectral_fbm(H, W, 0.8, 12, 0, 900)
    g = V.Grid.from_tensor(z, "cuda")
    posts = S.sample_posts(H, W, 2000, 32, 4, "cuda")
    labels = S.exact_vix(g, posts, 30, 10, 10)
    data = [(g, posts, labels)]
    a = S.Trainer(S.init_master(0), batch=256, lr=2e-3, patch_step=2)
    a.fit(data, epochs=3, seed=7)
    b = S.Trainer(S.init_master(0), batch=256, lr=2e-3, patch_step=2)
    b.fit(data, epochs=1, seed=7)
    path = str(tmp_path / "trainer.pt")
    b.save_checkpoint(path)
    c = S.Trainer.load_checkpoint(path)
    assert c.epochs_done == 1 and c.step == b.step
    c.fit(data, epochs=3, seed=7, first_epoch=c.epochs_done)
    assert c.step == a.step
    assert torch.equal(c.master, a.master)
    assert torch.equal(c.m, a.m) and torch.equal(c.v, a.v)
