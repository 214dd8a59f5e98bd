"""The learned proposal's tensor-core forward pass against the numpy oracle
(fp64 products on the same bf16-rounded inputs and weights)."""
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


def _params(seed):
    from oracle import cnn_oracle as C
    p = C.init_params(seed)
    rng = np.random.default_rng(seed + 100)
    for l in range(5):
        p["b%d" % l] = rng.normal(0, 0.05, 32)
    p["fb"] = np.array([0.1])
    return p


def test_cnn_forward_matches_oracle(V):
    from oracle import cnn_oracle as C
    H, W = 150, 170
    z = T.spectral_fbm(H, W, 0.8, 77, 0, 1500).numpy()
    g = V.Grid.from_tensor(torch.as_tensor(z), "cuda")
    p = _params(3)
    master = torch.as_tensor(C.flatten_params(p)).cuda()
    packed = V.cnn_pack(master)
    pts = [(75, 85), (0, 0), (H - 1, W - 1), (5, 160), (140, 3), (40, 100), (100, 40), (64, 64)]
    cen = torch.tensor([y * W + x for y, x in pts], dtype=torch.int64, device="cuda")
    save = torch.zeros(len(pts) * V.cnn_save_bytes(), dtype=torch.uint8, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    y = V.cnn_forward(g, cen, packed, save=save, status=status).cpu().numpy()
    assert int(status.item()) == 0
    x0 = np.stack([C.normalize_patch(C.extract_patch(z, cy, cx)) for cy, cx in pts])
    want, (cache, a5, gg, logit) = C.forward(p, x0, keep=True)
    assert np.all(np.abs(y - want) < 5e-3), (y, want)
    _check_saved_layers(C, p, z, pts, 1, save.cpu().numpy().reshape(len(pts), -1), y)


# save record of one patch (bytes): a1..a5 bf16 [y][x][32], head fp32 (g[32],
# logit, y), then x0 bf16 [65][65]
_SIZES = [33, 17, 9, 5, 5]
_OFFS = np.cumsum([0] + [n * n * 64 for n in _SIZES]).tolist()
_HEAD = _OFFS[5]
_X0 = (_HEAD + 34 * 4 + 127) // 128 * 128


def _bf16_bits(raw):
    return (raw.copy().view(np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def _within_rounding(C, got, exact, bound, relu):
    """got (the kernel's bf16 value) lies between the bf16 roundings of the
    ends of [exact - bound, exact + bound] (rounding is monotone): equal to
    the correctly rounded exact value unless the interval holds a rounding
    boundary, and then one of its two neighbours."""
    f = (lambda v: C.bf16(np.maximum(v, 0.0))) if relu else C.bf16
    lo, hi = f(exact - bound), f(exact + bound)
    ok = (lo <= got) & (got <= hi)
    return ok


def _check_saved_layers(C, p, z, pts, step, sv, y_out):
    """Element by element, every saved activation of every patch against the
    fp64 oracle fed with the kernel's own input to that layer: the kernel
    accumulates bf16 x bf16 products (exact in fp32) in FP32, so its
    pre-activation differs from the fp64 one by at most
    (K + 2) * 2^-23 * (sum of |terms|); an element may differ from the
    correctly rounded fp64 result only where that interval holds a bf16
    rounding boundary (or the ReLU's 0), and then only by that one step."""
    n = len(pts)
    x0 = _bf16_bits(sv[:, _X0:_X0 + 65 * 65 * 2]).reshape(n, 65, 65)
    zp = np.stack([C.extract_patch(z, cy, cx, step) for cy, cx in pts]).astype(np.float64)
    ex = C.normalize_patch(zp)
    mean = np.abs(zp.mean(axis=(1, 2), keepdims=True))
    bnd = 2.0 ** -20 * (np.abs(zp) + mean) / 1000.0
    bad = ~_within_rounding(C, x0, ex, bnd, relu=False)
    assert not bad.any(), ("x0", int(bad.sum()))
    a = x0[:, None]
    for l in range(5):
        m = _SIZES[l]
        got = _bf16_bits(sv[:, _OFFS[l]:_OFFS[l] + m * m * 64]).reshape(n, m, m, 32)
        pre = C.layer_pre(p, l, a)
        K = 9 * C.LAYERS[l][0]
        bound = (K + 2) * 2.0 ** -23 * C.layer_pre(p, l, a, absolute=True)
        bad = ~_within_rounding(C, got, pre, bound, relu=True)
        assert not bad.any(), (l, int(bad.sum()), np.argwhere(bad)[:3].tolist())
        a = got.transpose(0, 3, 1, 2)
    head = sv[:, _HEAD:_HEAD + 34 * 4].copy().view(np.float32).astype(np.float64)
    g = a.mean(axis=(2, 3))
    assert np.all(np.abs(head[:, :32] - g) <= 1e-6 * (1 + np.abs(g)))
    logit = g @ p["fw"] + p["fb"][0]
    yy = 1.0 / (1.0 + np.exp(-logit))
    assert np.all(np.abs(head[:, 33] - yy) <= 1e-5), np.abs(head[:, 33] - yy).max()
    assert np.array_equal(head[:, 33].astype(np.float32), np.asarray(y_out, np.float32))


def test_cnn_lattice_matches_centres(V):
    from oracle import cnn_oracle as C
    H, W, s = 90, 130, 16
    z = T.spectral_fbm(H, W, 0.8, 5, 0, 800).numpy()
    g = V.Grid.from_tensor(torch.as_tensor(z), "cuda")
    master = torch.as_tensor(C.flatten_params(_params(8))).cuda()
    packed = V.cnn_pack(master)
    lat = V.cnn_score_lattice(g, s, packed).cpu().numpy()
    Hs, Ws = lat.shape
    cen = torch.tensor([(i * s) * W + j * s for i in range(Hs) for j in range(Ws)], dtype=torch.int64,
                       device="cuda")
    y = V.cnn_forward(g, cen, packed).cpu().numpy().reshape(Hs, Ws)
    assert np.array_equal(lat, y)


def test_cnn_forward_many_patches_per_cta(V):
    """1200 patches (several per CTA on any GB300, so every CTA reuses its
    planes, tensor memory and barriers across patches), interior and edge
    centres mixed, against the oracle on every patch."""
    from oracle import cnn_oracle as C
    H, W = 400, 420
    z = T.spectral_fbm(H, W, 0.8, 33, 0, 2500).numpy()
    g = V.Grid.from_tensor(torch.as_tensor(z), "cuda")
    p = _params(9)
    packed = V.cnn_pack(torch.as_tensor(C.flatten_params(p)).cuda())
    rng = np.random.default_rng(12)
    n = 1200
    cy = rng.integers(0, H, n)
    cx = rng.integers(0, W, n)
    cy[::5] = rng.integers(32, H - 33, len(cy[::5]))  # plenty of staged (interior) patches
    cen = torch.as_tensor(cy * W + cx).cuda()
    y = V.cnn_forward(g, cen, packed).cpu().numpy()
    x0 = np.stack([C.normalize_patch(C.extract_patch(z, int(a), int(b))) for a, b in zip(cy, cx)])
    want = C.forward(p, x0)
    err = np.abs(y - want)
    assert err.max() < 5e-3, (err.max(), int(err.argmax()))
    # the same patches in another order and launch size give the same scores
    perm = rng.permutation(n)[:700]
    y2 = V.cnn_forward(g, cen[torch.as_tensor(perm).cuda()].contiguous(), packed).cpu().numpy()
    assert np.array_equal(y2, y[perm])


@pytest.mark.parametrize("step,chunks", [(1, 5), (3, 7)])
def test_cnn_lattice_rows_and_streamed(V, step, chunks):
    """Row bands of the lattice equal the full lattice's rows; scoring while
    the terrain streams in from pinned host memory gives the same map and
    leaves the whole terrain on the device."""
    from oracle import cnn_oracle as C
    from paper_2006_16783_gb300 import surrogate as S
    H, W, s = 700, 650, 16
    z = T.spectral_fbm(H, W, 0.8, 44, 0, 2000).numpy()
    g = V.Grid.from_tensor(torch.as_tensor(z), "cuda")
    packed = V.cnn_pack(torch.as_tensor(C.flatten_params(_params(4))).cuda())
    full = V.cnn_score_lattice(g, s, packed, patch_step=step)
    Hs = full.shape[0]
    part = torch.full_like(full, -1.0)
    for r0, r1 in [(0, 7), (7, 8), (8, Hs)]:
        V.cnn_score_lattice_rows(g, s, packed, r0, r1 - r0, part[r0:r1], patch_step=step)
    assert torch.equal(part, full)
    host = g.storage.cpu().pin_memory()
    g2 = V.Grid(torch.zeros_like(g.storage), W)
    out = torch.full_like(full, -1.0)
    S.score_lattice_streamed(g2, host, s, packed, out, patch_step=step, chunks=chunks)
    torch.cuda.synchronize()
    assert torch.equal(out, full)
    assert torch.equal(g2.storage, g.storage)
    with pytest.raises(V.VsError):
        V.cnn_score_lattice_rows(g, s, packed, Hs - 1, 2, part, patch_step=step)


@pytest.mark.parametrize("step", [2, 3])
def test_cnn_strided_patches(V, step):
    """patch_step > 1 (every step-th post, clamped at the edges; these patches
    skip the TMA staging): forward against the oracle, lattice against the
    per-centre launch."""
    from oracle import cnn_oracle as C
    H, W, s = 260, 300, 16
    z = T.spectral_fbm(H, W, 0.8, 21, 0, 1500).numpy()
    g = V.Grid.from_tensor(torch.as_tensor(z), "cuda")
    p = _params(5)
    packed = V.cnn_pack(torch.as_tensor(C.flatten_params(p)).cuda())
    pts = [(130, 150), (0, 0), (H - 1, W - 1), (97, 97), (5, 290), (200, 40)]
    rng = np.random.default_rng(step)
    pts += [(int(a), int(b)) for a, b in zip(rng.integers(0, H, 40), rng.integers(0, W, 40))]
    cen = torch.tensor([y * W + x for y, x in pts], dtype=torch.int64, device="cuda")
    save = torch.zeros(len(pts) * V.cnn_save_bytes(), dtype=torch.uint8, device="cuda")
    y = V.cnn_forward(g, cen, packed, patch_step=step, save=save).cpu().numpy()
    x0 = np.stack([C.normalize_patch(C.extract_patch(z, cy, cx, step)) for cy, cx in pts])
    want = C.forward(p, x0)
    assert np.all(np.abs(y - want) < 5e-3), (y, want)
    _check_saved_layers(C, p, z, pts, step, save.cpu().numpy().reshape(len(pts), -1), y)
    lat = V.cnn_score_lattice(g, s, packed, patch_step=step).cpu().numpy()
    Hs, Ws = lat.shape
    cen = torch.tensor([(i * s) * W + j * s for i in range(Hs) for j in range(Ws)], dtype=torch.int64,
                       device="cuda")
    assert np.array_equal(lat, V.cnn_forward(g, cen, packed, patch_step=step).cpu().numpy().reshape(Hs, Ws))
    with pytest.raises(V.VsError):
        V.cnn_forward(g, cen, packed, patch_step=0)


@pytest.mark.parametrize("B,seed", [(12, 4), (37, 5)])
def test_cnn_backward_matches_oracle(V, B, seed):
    """Gradients of the batch L1 loss, element by element, against the
    oracle's fp64 backward on the same bf16-rounded operands: every element
    within 1e-2 of its value plus 2^-6 of the sum of the absolute values of
    the terms it adds up -- room for pre-activation gradients whose bf16
    rounding goes the other way after FP32 accumulation (one bf16 step,
    2^-8, per term and layer), not for a wrong tap, channel or patch."""
    from oracle import cnn_oracle as C
    H, W = 200, 210
    z = T.spectral_fbm(H, W, 0.8, 91, 0, 1200).numpy()
    g = V.Grid.from_tensor(torch.as_tensor(z), "cuda")
    p = _params(11)
    rng = np.random.default_rng(seed)
    pts = [(int(a), int(b)) for a, b in zip(rng.integers(0, H, B), rng.integers(0, W, B))]
    pts[:3] = [(0, 0), (H - 1, W - 1), (100, 0)]
    labels = rng.random(len(pts)).astype(np.float32)
    master = torch.as_tensor(C.flatten_params(p)).cuda()
    packed = V.cnn_pack(master)
    cen = torch.tensor([y * W + x for y, x in pts], dtype=torch.int64, device="cuda")
    save = torch.zeros(len(pts) * V.cnn_save_bytes(), dtype=torch.uint8, device="cuda")
    V.cnn_forward(g, cen, packed, save=save)
    grads = torch.zeros_like(master)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    V.cnn_backward(save, torch.as_tensor(labels).cuda(), master, grads, loss)
    gg = C.unflatten_params(grads.cpu().numpy())
    x0 = np.stack([C.normalize_patch(C.extract_patch(z, cy, cx)) for cy, cx in pts])
    want_loss, want, scale = C.loss_and_grads(p, x0, labels.astype(np.float64), scale=True)
    assert abs(loss.item() / len(pts) - want_loss) < 5e-3
    for k in want:
        a, b, sc = gg[k].ravel(), want[k].ravel(), scale[k].ravel()
        bad = np.abs(a - b) > 1e-2 * np.abs(b) + 2.0 ** -6 * sc
        assert not bad.any(), (k, int(bad.sum()), np.flatnonzero(bad)[:5].tolist(),
                               a[bad][:5].tolist(), b[bad][:5].tolist())


def test_cnn_adam_step(V):
    from oracle import cnn_oracle as C
    n = V.cnn_param_count()
    rng = np.random.default_rng(0)
    w = rng.normal(size=n).astype(np.float32)
    gr = rng.normal(size=n).astype(np.float32)
    tw, tg = torch.as_tensor(w).cuda(), torch.as_tensor(gr).cuda()
    m, v = torch.zeros_like(tw), torch.zeros_like(tw)
    for step in (1, 2):
        tg.copy_(torch.as_tensor(gr))
        V.cnn_adam(tw, tg, m, v, step, lr=1e-2)
    pw = {"a": w.astype(np.float64)}
    st = {}
    for step in (1, 2):
        C.adam_step(pw, {"a": gr.astype(np.float64)}, st, lr=1e-2)
    assert np.allclose(tw.cpu().numpy(), pw["a"], atol=1e-5)
    assert float(tg.abs().max()) == 0.0


@pytest.mark.parametrize("n", [1, 2, 3, 4, 151, 152, 153, 304, 305, 459, 611])
def test_cnn_forward_any_patch_count(V, n):
    """The forward keeps two patches in flight per CTA, with a ring of three
    pooling buffers and per-patch barrier phases, so launches of 1 .. 4
    patches per CTA (and CTAs with one patch fewer than others) exercise its
    start and drain.  Every score, and every saved activation, equals the
    same patch's in one large launch bit for bit (a patch's result does not
    depend on its neighbours)."""
    H, W = 300, 280
    z = T.spectral_fbm(H, W, 0.8, 57, 0, 1800).numpy()
    g = V.Grid.from_tensor(torch.as_tensor(z), "cuda")
    from oracle import cnn_oracle as C
    packed = V.cnn_pack(torch.as_tensor(C.flatten_params(_params(3))).cuda())
    rng = np.random.default_rng(1000 + n)
    big = 900
    cy = rng.integers(0, H, big)
    cx = rng.integers(0, W, big)
    cy[::3] = rng.integers(32, H - 33, len(cy[::3]))  # TMA-staged and gathered windows mixed
    cen = torch.as_tensor(cy * W + cx).cuda()
    sb = V.cnn_save_bytes()
    save = torch.zeros(big * sb, dtype=torch.uint8, device="cuda")
    y = V.cnn_forward(g, cen, packed, save=save)
    pick = torch.as_tensor(rng.choice(big, n, replace=False)).cuda()
    save_n = torch.zeros(n * sb, dtype=torch.uint8, device="cuda")
    y_n = V.cnn_forward(g, cen[pick].contiguous(), packed, save=save_n)
    assert torch.equal(y_n, y[pick])
    assert torch.equal(save_n.view(n, sb), save.view(big, sb)[pick])
    # and without a save record (the inference path)
    assert torch.equal(V.cnn_forward(g, cen[pick].contiguous(), packed), y[pick])
