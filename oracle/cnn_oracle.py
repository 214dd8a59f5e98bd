"""Plain numpy oracle of the learned candidate proposal (test infrastructure).

The paper's Vix stage only ranks posts (Sec. "The multiple transmitter siting
process", Vix: "extreme accuracy ... is not required"); the learned proposal
replaces that ranking by a small CNN that maps a 65 x 65 elevation patch to a
predicted visibility index.  The paper fixes no network, so the architecture
is this project's choice (stated here and in the CUDA kernels' header):

    x0 = bf16((z - mean(z_patch)) / 1000)                         65 x 65 x 1
    conv1 3x3 stride 2 pad 1, 1 -> 32, bias, ReLU, bf16          33 x 33 x 32
    conv2 3x3 stride 2 pad 1, 32 -> 32, bias, ReLU, bf16         17 x 17 x 32
    conv3 3x3 stride 2 pad 1, 32 -> 32, bias, ReLU, bf16          9 x  9 x 32
    conv4 3x3 stride 2 pad 1, 32 -> 32, bias, ReLU, bf16          5 x  5 x 32
    conv5 3x3 stride 1 pad 1, 32 -> 32, bias, ReLU, bf16          5 x  5 x 32
    global average pool (fp32) -> fc 32 -> 1 (+ bias) -> sigmoid
    loss = mean |y - label| (L1)

Weights enter every product as bf16; products accumulate in high precision
here (fp64) and in fp32 on the GPU.  The backward pass rounds the gradient of
each conv's pre-activation to bf16 before it meets weights or activations,
as the tensor-core kernels do.  Only the tests and the benchmark's CPU leg use
this module.
"""
import numpy as np

PATCH = 65
CH = 32
# (cin, cout, stride) of the five 3x3 convolutions
LAYERS = [(1, 32, 2), (32, 32, 2), (32, 32, 2), (32, 32, 2), (32, 32, 1)]


ROUND = True   # tests switch it off to check the gradients by finite differences


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    if not ROUND:
        return np.asarray(a, dtype=np.float64)
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (r.astype(np.uint32)).view(np.float32).astype(np.float64)


def out_size(n, stride):
    return (n + 2 - 3) // stride + 1


def normalize_patch(z_patch):
    """(z - mean) / 1000 with the mean over the patch; float64 before rounding."""
    z = np.asarray(z_patch, dtype=np.float64)
    return (z - z.mean(axis=(-2, -1), keepdims=True)) / 1000.0


def init_params(seed=0):
    """He-normal weights (fan-in 9*cin), zero biases; fc small."""
    rng = np.random.default_rng(seed)
    p = {}
    for l, (ci, co, s) in enumerate(LAYERS):
        p["w%d" % l] = rng.normal(0.0, np.sqrt(2.0 / (9 * ci)), (co, ci, 3, 3))
        p["b%d" % l] = np.zeros(co)
    p["fw"] = rng.normal(0.0, np.sqrt(1.0 / CH), CH)
    p["fb"] = np.zeros(1)
    return p


def _im2col(x, stride):
    """x: (B, C, H, W) -> (B, Ho, Wo, C*9) with zero padding 1, tap order
    (c, ky, kx) matching weight layout (co, ci, ky, kx)."""
    B, C, H, W = x.shape
    Ho, Wo = out_size(H, stride), out_size(W, stride)
    xp = np.zeros((B, C, H + 2, W + 2))
    xp[:, :, 1:-1, 1:-1] = x
    cols = np.empty((B, Ho, Wo, C, 3, 3))
    for ky in range(3):
        for kx in range(3):
            cols[:, :, :, :, ky, kx] = xp[:, :, ky:ky + stride * Ho:stride, kx:kx + stride * Wo:stride].transpose(0, 2, 3, 1)
    return cols.reshape(B, Ho, Wo, C * 9)


def _col2im(dcols, shape, stride):
    B, C, H, W = shape
    Ho, Wo = dcols.shape[1], dcols.shape[2]
    d = dcols.reshape(B, Ho, Wo, C, 3, 3)
    dxp = np.zeros((B, C, H + 2, W + 2))
    for ky in range(3):
        for kx in range(3):
            dxp[:, :, ky:ky + stride * Ho:stride, kx:kx + stride * Wo:stride] += d[:, :, :, :, ky, kx].transpose(0, 3, 1, 2)
    return dxp[:, :, 1:-1, 1:-1]


def forward(params, x0, keep=False):
    """x0: (B, 65, 65) normalized patches (rounded to bf16 here).  Returns
    y (B,) and, with keep=True, the cache needed by backward."""
    a = bf16(x0)[:, None, :, :]
    cache = []
    for l, (ci, co, s) in enumerate(LAYERS):
        cols = _im2col(a, s)
        w = bf16(params["w%d" % l]).reshape(co, ci * 9)
        pre = cols @ w.T + params["b%d" % l]              # (B, Ho, Wo, co)
        out = bf16(np.maximum(pre, 0.0))
        cache.append((a, cols, pre))
        a = out.transpose(0, 3, 1, 2)
    g = a.mean(axis=(2, 3))                               # (B, 32)
    logit = g @ params["fw"] + params["fb"][0]
    y = 1.0 / (1.0 + np.exp(-logit))
    if keep:
        return y, (cache, a, g, logit)
    return y


def layer_pre(params, l, a, absolute=False):
    """Pre-activation of conv layer l (0-based) on input a (B, cin, H, W):
    (B, Ho, Wo, 32) in fp64 from the bf16-rounded weights, plus the bias.
    With absolute=True: the sum of the absolute values of the same terms
    (|w| |a| over the taps, + |bias|), the scale of any rounding error of a
    lower-precision accumulation of that sum."""
    ci, co, s = LAYERS[l]
    cols = _im2col(np.asarray(a, dtype=np.float64), s)
    w = bf16(params["w%d" % l]).reshape(co, ci * 9)
    if absolute:
        return np.abs(cols) @ np.abs(w).T + np.abs(params["b%d" % l])
    return cols @ w.T + params["b%d" % l]


def loss_and_grads(params, x0, label, scale=False):
    """L1 loss and gradients of every parameter (dict like params).  With
    scale=True also, per gradient element, the sum of the absolute values of
    the terms it adds up (the scale of the rounding error of a lower-precision
    evaluation of the same sums)."""
    B = x0.shape[0]
    y, (cache, a5, g, logit) = forward(params, x0, keep=True)
    loss = np.abs(y - label).mean()
    dlogit = np.sign(y - label) * y * (1.0 - y) / B
    grads = {"fw": g.T @ dlogit, "fb": np.array([dlogit.sum()])}
    sc = {"fw": np.abs(g).T @ np.abs(dlogit), "fb": np.array([np.abs(dlogit).sum()])}
    dg = dlogit[:, None] * params["fw"][None, :]           # (B, 32)
    Ho, Wo = a5.shape[2], a5.shape[3]
    da = np.broadcast_to(dg[:, :, None, None] / (Ho * Wo), a5.shape).copy()
    for l in range(len(LAYERS) - 1, -1, -1):
        ci, co, s = LAYERS[l]
        a_in, cols, pre = cache[l]
        dz = bf16(da.transpose(0, 2, 3, 1) * (pre > 0))     # (B, Ho, Wo, co)
        grads["w%d" % l] = np.einsum("bhwk,bhwo->ok", cols, dz).reshape(co, ci, 3, 3)
        grads["b%d" % l] = dz.sum(axis=(0, 1, 2))
        if scale:
            sc["w%d" % l] = np.einsum("bhwk,bhwo->ok", np.abs(cols), np.abs(dz)).reshape(co, ci, 3, 3)
            sc["b%d" % l] = np.abs(dz).sum(axis=(0, 1, 2))
        if l > 0:
            w = bf16(params["w%d" % l]).reshape(co, ci * 9)
            dcols = dz @ w                                  # (B, Ho, Wo, ci*9)
            da = _col2im(dcols, a_in.shape, s)
    if scale:
        return loss, grads, sc
    return loss, grads


def adam_step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015) on fp64 copies of the master weights."""
    t = state.get("t", 0) + 1
    state["t"] = t
    for k in params:
        m = state.setdefault("m" + k, np.zeros_like(params[k]))
        v = state.setdefault("v" + k, np.zeros_like(params[k]))
        m[...] = b1 * m + (1 - b1) * grads[k]
        v[...] = b2 * v + (1 - b2) * grads[k] ** 2
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
    return params


def flops_per_patch():
    n, tot = PATCH, 0
    for ci, co, s in LAYERS:
        n = out_size(n, s)
        tot += 2 * n * n * co * ci * 9
    return tot + 2 * CH


def extract_patch(z, cy, cx, step=1):
    """65 x 65 elevations centred on post (cx, cy), every ``step``-th post;
    rows and columns outside the grid take the nearest edge post."""
    H, W = z.shape
    ys = np.clip(cy + step * np.arange(-32, 33), 0, H - 1)
    xs = np.clip(cx + step * np.arange(-32, 33), 0, W - 1)
    return np.asarray(z)[np.ix_(ys, xs)]


def flatten_params(p):
    """The library's flat fp32 parameter vector: w_l, b_l for l = 0..4, fc w, fc b."""
    parts = []
    for l in range(len(LAYERS)):
        parts += [p["w%d" % l].ravel(), p["b%d" % l].ravel()]
    parts += [p["fw"].ravel(), p["fb"].ravel()]
    return np.concatenate(parts).astype(np.float32)


def unflatten_params(v):
    v = np.asarray(v, dtype=np.float64)
    p, o = {}, 0
    for l, (ci, co, s) in enumerate(LAYERS):
        n = co * ci * 9
        p["w%d" % l] = v[o:o + n].reshape(co, ci, 3, 3)
        o += n
        p["b%d" % l] = v[o:o + co].copy()
        o += co
    p["fw"] = v[o:o + CH].copy()
    p["fb"] = v[o + CH:o + CH + 1].copy()
    return p
