"""Pins of the CNN oracle: shapes, a direct-loop convolution, bf16 rounding,
and finite-difference gradients (rounding switched off).  CPU only."""
import numpy as np
import pytest

from oracle import cnn_oracle as C


def test_shapes_and_flops():
    n = C.PATCH
    sizes = []
    for ci, co, s in C.LAYERS:
        n = C.out_size(n, s)
        sizes.append(n)
    assert sizes == [33, 17, 9, 5, 5]
    assert C.flops_per_patch() == 2 * (33 * 33 * 32 * 9 + 17 * 17 * 32 * 288 + 81 * 32 * 288
                                       + 25 * 32 * 288 + 25 * 32 * 288) + 64


def test_bf16_rounding():
    # exactly representable values stay, ties go to even, 1 + 2^-8 rounds to 1
    v = np.array([1.0, -2.5, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 3.0e38, 0.0])
    r = C.bf16(v)
    assert r[0] == 1.0 and r[1] == -2.5 and r[2] == 1.0 and r[3] == 1 + 2 ** -6 and r[5] == 0.0
    x = np.random.default_rng(0).normal(size=1000)
    assert np.all(np.abs(C.bf16(x) - x) <= np.abs(x) * 2 ** -8)


def _direct_conv(x, w, b, s):
    B, Ci, H, W = x.shape
    Co = w.shape[0]
    Ho, Wo = C.out_size(H, s), C.out_size(W, s)
    out = np.zeros((B, Ho, Wo, Co))
    for bb in range(B):
        for oy in range(Ho):
            for ox in range(Wo):
                for ky in range(3):
                    for kx in range(3):
                        iy, ix = oy * s + ky - 1, ox * s + kx - 1
                        if 0 <= iy < H and 0 <= ix < W:
                            out[bb, oy, ox] += w[:, :, ky, kx] @ x[bb, :, iy, ix]
    return out + b


@pytest.mark.parametrize("s", [1, 2])
def test_im2col_matches_direct_loop(s):
    rng = np.random.default_rng(s)
    x = rng.normal(size=(2, 3, 7, 9))
    w = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    got = C._im2col(x, s) @ w.reshape(4, 27).T + b
    assert np.allclose(got, _direct_conv(x, w, b, s))


def test_gradients_by_finite_differences():
    C.ROUND = False
    try:
        rng = np.random.default_rng(1)
        p = C.init_params(3)
        for k in p:
            if k.startswith("b") or k == "fb":
                p[k] = rng.normal(0, 0.1, p[k].shape)
        x = rng.normal(0, 0.3, (3, 65, 65))
        lab = np.array([0.2, 0.5, 0.9])
        loss, g = C.loss_and_grads(p, x, lab)
        eps = 1e-6
        for k, idx in [("w0", (3, 0, 1, 2)), ("w1", (5, 7, 0, 0)), ("w2", (1, 30, 2, 1)),
                       ("w3", (31, 2, 1, 1)), ("w4", (0, 0, 2, 2)), ("b1", (4,)), ("b4", (9,)),
                       ("fw", (6,)), ("fb", (0,))]:
            q = {kk: vv.copy() for kk, vv in p.items()}
            q[k][idx] += eps
            lp = np.abs(C.forward(q, x) - lab).mean()
            q[k][idx] -= 2 * eps
            lm = np.abs(C.forward(q, x) - lab).mean()
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - g[k][idx]) <= 1e-6 + 1e-4 * abs(fd), (k, fd, g[k][idx])
    finally:
        C.ROUND = True


def test_adam_moves_against_gradient():
    p = {"a": np.array([1.0, -1.0])}
    st = {}
    C.adam_step(p, {"a": np.array([0.5, -0.5])}, st, lr=0.1)
    assert np.allclose(p["a"], [0.9, -0.9])


def test_extract_patch_slices_and_clamps():
    """Inside the grid a patch is the plain (strided) slice; at the edges each
    coordinate is clamped on its own (brute loop on a small grid)."""
    rng = np.random.default_rng(3)
    z = rng.integers(-500, 3000, (300, 280)).astype(np.int16)
    assert np.array_equal(C.extract_patch(z, 150, 140), z[118:183, 108:173])
    assert np.array_equal(C.extract_patch(z, 150, 140, step=3), z[54:247:3, 44:237:3])
    for cy, cx, s in [(0, 0, 1), (299, 5, 2), (10, 279, 3), (150, 140, 5)]:
        p = C.extract_patch(z, cy, cx, step=s)
        for r in range(65):
            for c in range(65):
                y = min(max(cy + (r - 32) * s, 0), 299)
                x = min(max(cx + (c - 32) * s, 0), 279)
                assert p[r, c] == z[y, x]


@pytest.mark.parametrize("l", [0, 1, 4])
def test_layer_pre_matches_direct_loop(l):
    """layer_pre (the per-layer check of the tensor-core forward) against the
    direct 7-loop convolution with bf16-rounded weights; absolute=True against
    the same loop on absolute values."""
    rng = np.random.default_rng(10 + l)
    p = C.init_params(l)
    p["b%d" % l] = rng.normal(0, 0.1, 32)
    ci, co, s = C.LAYERS[l]
    x = C.bf16(rng.normal(size=(2, ci, 9, 8)))
    w = C.bf16(p["w%d" % l])
    assert np.allclose(C.layer_pre(p, l, x), _direct_conv(x, w, p["b%d" % l], s), rtol=0, atol=1e-12)
    got = C.layer_pre(p, l, x, absolute=True)
    want = _direct_conv(np.abs(x), np.abs(w), np.abs(p["b%d" % l]), s)
    assert np.allclose(got, want, rtol=0, atol=1e-12)
