"""Python binding of libvshed.so (ctypes over the C ABI in include/vshed.h).

Argument marshalling only: every step of the siting path runs in the CUDA
kernels of the library.  Tensors must be CUDA tensors on the current device;
the calls are enqueued on torch's current stream.  There is no CPU fallback:
if the library is missing or a call fails, an exception is raised.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvshed.so")
_lib = None

VS_OK, VS_ERR_ARG, VS_ERR_RANGE, VS_ERR_WS, VS_ERR_CUDA, VS_ERR_TIMEOUT, VS_ERR_DEVICE = 0, -1, -2, -3, -4, -5, -6


class VsError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__("%s failed: %s (%d)" % (fn, lib().vs_strerror(code).decode(), code))
        self.code = code


class vs_grid(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int32), ("W", ctypes.c_int32), ("pitch", ctypes.c_int64),
                ("z", ctypes.c_void_p)]


class vs_viewshed_job(ctypes.Structure):
    _fields_ = [("g", vs_grid), ("R", ctypes.c_int32), ("ht", ctypes.c_int32), ("hr", ctypes.c_int32),
                ("cand", ctypes.c_void_p), ("n", ctypes.c_int64), ("bm_out", ctypes.c_void_p),
                ("area_out", ctypes.c_void_p)]


class vs_site_job(ctypes.Structure):
    _fields_ = [("bm", ctypes.c_void_p), ("cand", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("H", ctypes.c_int32), ("W", ctypes.c_int32), ("R", ctypes.c_int32),
                ("n_obs", ctypes.c_int32), ("coverage_target", ctypes.c_double),
                ("chosen", ctypes.c_void_p), ("gains", ctypes.c_void_p), ("cum", ctypes.c_void_p),
                ("n_chosen", ctypes.c_void_p)]


class vs_vix_job(ctypes.Structure):
    _fields_ = [("g", vs_grid), ("R", ctypes.c_int32), ("ht", ctypes.c_int32), ("hr", ctypes.c_int32),
                ("S", ctypes.c_int32), ("seed", ctypes.c_uint64), ("vix_out", ctypes.c_void_p)]


class vs_findmax_job(ctypes.Structure):
    _fields_ = [("vix", ctypes.c_void_p), ("H", ctypes.c_int32), ("W", ctypes.c_int32),
                ("block", ctypes.c_int32), ("k", ctypes.c_int32), ("cand_out", ctypes.c_void_p),
                ("cap", ctypes.c_int64)]


class vs_site_options(ctypes.Structure):
    _fields_ = [("terrain", vs_grid), ("ht", ctypes.c_int32), ("weight", ctypes.c_void_p)]


(VS_TUNE_VIEWSHED_THREADS, VS_TUNE_VIX_TILE, VS_TUNE_SITE_CLUSTER, VS_TUNE_VIEWSHED_WIDE,
 VS_TUNE_SITE_LAZY, VS_TUNE_SITE_MULTI, VS_TUNE_SITE_BARRIER_TEST) = 0, 1, 2, 3, 4, 5, 6

# name -> (restype, argtypes); the exported symbols of include/vshed.h
P, i32, i64, u64, f64, sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                             ctypes.c_double, ctypes.c_size_t)
SIGNATURES = {
    "vs_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "vs_version": (ctypes.c_int, []),
    "vs_launch_count": (u64, []),
    "vs_selftest_wait_timeout": (ctypes.c_int, [P, ctypes.c_uint32, P]),
    "vs_tune_set": (ctypes.c_int, [i32, i32, i32]),
    "vs_tune_get": (ctypes.c_int, [i32, i32]),
    "vs_viewshed_batch_workspace": (sz, [i32]),
    "vs_viewshed_batch": (ctypes.c_int, [P, i32, P, sz, P]),
    "vs_site_batch_workspace": (sz, [P, i32]),
    "vs_site_batch": (ctypes.c_int, [P, i32, P, sz, P]),
    "vs_vix": (ctypes.c_int, [vs_grid, i32, i32, i32, i32, u64, P, P]),
    "vs_vix_count": (ctypes.c_int, [vs_grid, i32, i32, i32, i32, u64, P, P, P]),
    "vs_vix_workspace": (sz, [i32, i32, i32, i32]),
    "vs_vix_ws": (ctypes.c_int, [vs_grid, i32, i32, i32, i32, u64, P, P, P, sz, P]),
    "vs_findmax_count": (i64, [i32, i32, i32, i32, i32]),
    "vs_findmax": (ctypes.c_int, [P, i32, i32, i32, i32, P, i64, P]),
    "vs_findmax_f32": (ctypes.c_int, [P, i32, i32, i32, i32, i32, P, i64, P]),
    "vs_bitmap_words": (i64, [i32]),
    "vs_viewshed_workspace": (sz, [i32, i32, i32, i64]),
    "vs_viewshed": (ctypes.c_int, [vs_grid, i32, i32, i32, P, i64, P, P, P, sz, P]),
    "vs_viewshed_r3_workspace": (sz, [i32, i32]),
    "vs_viewshed_r3": (ctypes.c_int, [vs_grid, i32, i32, i32, P, i64, P, P, P, sz, P]),
    "vs_exact_vix_workspace": (sz, [i32, i32, i32, i64]),
    "vs_exact_vix": (ctypes.c_int, [vs_grid, i32, i32, i32, P, i64, P, P, sz, P]),
    "vs_vix_batch_workspace": (sz, [i32]),
    "vs_vix_batch": (ctypes.c_int, [P, i32, P, sz, P]),
    "vs_findmax_batch": (ctypes.c_int, [P, i32, P]),
    "vs_site_shard_workspace": (sz, [i32]),
    "vs_site_shard_step": (ctypes.c_int, [P, P, i64, i32, i32, i32, P, P, P, i64, i64, P, P, sz, P]),
    "vs_site_workspace": (sz, [i64, i32]),
    "vs_site": (ctypes.c_int, [P, P, i64, i32, i32, i32, i32, f64, P, P, P, P, P, sz, P]),
    "vs_site_gains": (ctypes.c_int, [P, P, i64, i32, i32, i32, P, P, P]),
    "vs_site_ex_workspace": (sz, [i64, i32]),
    "vs_site_ex": (ctypes.c_int, [P, P, i64, i32, i32, i32, i32, f64, ctypes.POINTER(vs_site_options), P, P, P, P,
                                  P, sz, P]),
    "vs_site_noalloc": (ctypes.c_int, [P, P, i64, i32, i32, i32, i32, f64, P, P, P, P, P]),
    "vs_cnn_param_count": (ctypes.c_int, []),
    "vs_cnn_packed_bytes": (sz, []),
    "vs_cnn_save_bytes": (sz, []),
    "vs_cnn_pack": (ctypes.c_int, [P, P, P]),
    "vs_cnn_forward": (ctypes.c_int, [vs_grid, P, i64, i32, P, P, P, P, P]),
    "vs_cnn_score_lattice": (ctypes.c_int, [vs_grid, i32, i32, P, P, P, P]),
    "vs_cnn_score_lattice_rows": (ctypes.c_int, [vs_grid, i32, i32, i32, i32, P, P, P, P]),
    "vs_cnn_backward_workspace": (sz, [i64]),
    "vs_cnn_backward": (ctypes.c_int, [P, P, i64, P, P, P, P, sz, P]),
    "vs_cnn_adam": (ctypes.c_int, [P, P, P, P, i64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                   ctypes.c_float, P]),
}


def lib():
    """Load libvshed.so (built by ``__graft_entry__.build()`` or
    ``python -m paper_2006_16783_gb300._build``); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libvshed.so not found at %s: build it first "
                              "(python -c 'import __graft_entry__ as g; g.build()')" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(fn, rc):
    if rc != VS_OK:
        raise VsError(fn, rc)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _need_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("libvshed works on CUDA tensors only (got a %s tensor)" % t.device)


# ------------------------------------------------------------------ terrain
class Grid:
    """A device-resident int16 terrain: ``storage`` is an (H, pitch) int16
    CUDA tensor whose first W columns are the terrain (pitch % 8 == 0)."""

    def __init__(self, storage, W=None):
        _need_cuda(storage)
        assert storage.dtype == torch.int16 and storage.dim() == 2 and storage.is_contiguous()
        self.storage = storage
        self.H = storage.shape[0]
        self.pitch = storage.shape[1]
        self.W = self.pitch if W is None else int(W)

    @classmethod
    def from_tensor(cls, z, device="cuda"):
        """Copy an (H, W) int16 tensor into pitched device storage."""
        H, W = z.shape
        pitch = (W + 7) // 8 * 8
        st = torch.zeros((H, pitch), dtype=torch.int16, device=device)
        st[:, :W] = z.to(device)
        return cls(st, W)

    def c(self):
        return vs_grid(self.H, self.W, self.pitch, self.storage.data_ptr())


# ------------------------------------------------------------------ stages
def vix_workspace(H, W, R, S):
    """Workspace bytes of vs_vix_ws (0 when the staged kernels cover R)."""
    return lib().vs_vix_workspace(H, W, R, S)


def vix(g, R, ht, hr, S, seed, out=None, ws=None):
    """Sampled visibility-index counts (uint8, H x W).  For ROIs beyond the
    staged kernels the transposed terrain goes in ``ws`` (a uint8 device
    buffer of at least vix_workspace() bytes, allocated when missing)."""
    return _vix(g, R, ht, hr, S, seed, None, out, ws)


def vix_count(g, R, ht, hr, S, seed, steps, out=None, ws=None):
    """vs_vix that also adds the number of LOS crossings it evaluated to the
    device uint64 counter ``steps`` (an int64 CUDA tensor of one element)."""
    _need_cuda(steps)
    return _vix(g, R, ht, hr, S, seed, steps, out, ws)


def _vix(g, R, ht, hr, S, seed, steps, out, ws):
    if out is None:
        out = torch.empty((g.H, g.W), dtype=torch.uint8, device=g.storage.device)
    _need_cuda(out)
    sd = ctypes.c_uint64(seed & (2**64 - 1))
    wsb = lib().vs_vix_workspace(g.H, g.W, R, S)
    if wsb == 0 and steps is None:
        _check("vs_vix", lib().vs_vix(g.c(), R, ht, hr, S, sd, _ptr(out), _stream()))
    elif wsb == 0:
        _check("vs_vix_count", lib().vs_vix_count(g.c(), R, ht, hr, S, sd, _ptr(out), _ptr(steps), _stream()))
    else:
        if ws is None or ws.numel() < wsb:
            ws = torch.empty(wsb, dtype=torch.uint8, device=out.device)
        _check("vs_vix_ws", lib().vs_vix_ws(g.c(), R, ht, hr, S, sd, _ptr(out), _ptr(steps), _ptr(ws), wsb,
                                            _stream()))
    return out


def findmax_count(H, W, stride, block, k):
    n = lib().vs_findmax_count(H, W, stride, block, k)
    if n < 0:
        raise VsError("vs_findmax_count", n)
    return n


def findmax(v, block, k, out=None):
    """Top-k posts per block of a uint8 H x W map -> int64 post indices."""
    _need_cuda(v)
    H, W = v.shape
    n = findmax_count(H, W, 1, block, k)
    if out is None:
        out = torch.empty(n, dtype=torch.int64, device=v.device)
    _check("vs_findmax", lib().vs_findmax(_ptr(v), H, W, block, k, _ptr(out), out.numel(), _stream()))
    return out[:n]


def findmax_f32(score, H, W, stride, block, k, out=None):
    """Top-k posts per block of a float score lattice of the given stride."""
    _need_cuda(score)
    assert score.dtype == torch.float32 and score.is_contiguous()
    n = findmax_count(H, W, stride, block, k)
    if out is None:
        out = torch.empty(n, dtype=torch.int64, device=score.device)
    _check("vs_findmax_f32", lib().vs_findmax_f32(_ptr(score), H, W, stride, block, k, _ptr(out),
                                                  out.numel(), _stream()))
    return out[:n]


def bitmap_words(R):
    return lib().vs_bitmap_words(R)


def words_per_row(R):
    return (2 * R) // 32 + 2


def viewshed_workspace(H, W, R, n):
    """Workspace bytes of vs_viewshed (0 when the ROI window fits in shared
    memory, else the transposed terrain the banded kernel reads)."""
    return lib().vs_viewshed_workspace(H, W, R, n)


def viewshed(g, R, ht, hr, cand, bm=None, area=None, ws=None):
    """Viewshed bitmaps uint32 [n, 2R+1, P_R] and areas int32 [n].  ws: an
    optional uint8 device buffer of at least viewshed_workspace() bytes, to
    reuse across calls."""
    _need_cuda(cand)
    cand = cand.contiguous()
    n = cand.numel()
    if bm is None:
        bm = torch.empty((n, 2 * R + 1, words_per_row(R)), dtype=torch.int32, device=cand.device)
    if area is None:
        area = torch.empty(n, dtype=torch.int32, device=cand.device)
    wsb = lib().vs_viewshed_workspace(g.H, g.W, R, n)
    if wsb and (ws is None or ws.numel() < wsb):
        ws = torch.empty(wsb, dtype=torch.uint8, device=cand.device)
    _check("vs_viewshed", lib().vs_viewshed(g.c(), R, ht, hr, _ptr(cand), n, _ptr(bm), _ptr(area),
                                            _ptr(ws), wsb, _stream()))
    return bm, area


def viewshed_r3(g, R, ht, hr, cand, bm=None, area=None, ws=None):
    """Exact per-cell viewshed (every disc cell its own LOS); same layout as
    viewshed().  ws: optional uint8 device buffer for the transposed terrain
    (allocated when missing)."""
    _need_cuda(cand)
    cand = cand.contiguous()
    n = cand.numel()
    if bm is None:
        bm = torch.empty((n, 2 * R + 1, words_per_row(R)), dtype=torch.int32, device=cand.device)
    if area is None:
        area = torch.empty(n, dtype=torch.int32, device=cand.device)
    wsb = lib().vs_viewshed_r3_workspace(g.H, g.W)
    if ws is None or ws.numel() < wsb:
        ws = torch.empty(wsb, dtype=torch.uint8, device=cand.device)
    _check("vs_viewshed_r3", lib().vs_viewshed_r3(g.c(), R, ht, hr, _ptr(cand), n, _ptr(bm), _ptr(area),
                                                  _ptr(ws), wsb, _stream()))
    return bm, area


def exact_vix(g, R, ht, hr, posts, out=None, ws=None):
    """Exact visibility index of each post (float32; -1 outside the grid):
    viewshed area over the ROI's receivers inside the grid.  ws: optional
    uint8 device buffer of at least vs_exact_vix_workspace bytes."""
    _need_cuda(posts)
    posts = posts.contiguous()
    n = posts.numel()
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=posts.device)
    wsb = lib().vs_exact_vix_workspace(g.H, g.W, R, n)
    if ws is None or ws.numel() < wsb:
        ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=posts.device)
    _check("vs_exact_vix", lib().vs_exact_vix(g.c(), R, ht, hr, _ptr(posts), n, _ptr(out), _ptr(ws), wsb,
                                              _stream()))
    return out


def site_shard_step(bm, cand, H, W, R, gains, cum, win_bm, win_post, win_local, best_key, ws):
    """One greedy step on this rank's share of the candidates (vs_site_shard_step):
    apply the broadcast winner (win_post < 0: none) and write the rank's best
    key into best_key (uint64 as int64, one element)."""
    _need_cuda(cand, gains, cum, best_key, ws)
    n = cand.numel()
    _check("vs_site_shard_step", lib().vs_site_shard_step(
        _ptr(bm) if n else None, _ptr(cand) if n else None, n, H, W, R, _ptr(gains) if n else None, _ptr(cum),
        _ptr(win_bm) if win_bm is not None else None, int(win_post), int(win_local), _ptr(best_key), _ptr(ws),
        ws.numel(), _stream()))


def site_ex(bm, cand, H, W, R, n_obs, target=0.0, grid=None, ht=0, weight=None, cum=None, sync=True):
    """vs_site with the intervisibility constraint (grid: the terrain the
    bitmaps were computed on; transmitters after the first must see one
    chosen earlier, antennas at z + ht) and / or uint8 receiver weights
    (H x W device tensor).  Same returns as site()."""
    _need_cuda(bm, cand)
    dev = cand.device
    n = cand.numel()
    if cum is None:
        cum = torch.zeros((H, (W + 31) // 32), dtype=torch.int32, device=dev)
    chosen = torch.empty(max(n_obs, 1), dtype=torch.int64, device=dev)
    gains = torch.empty(max(n_obs, 1), dtype=torch.int64, device=dev)
    nch = torch.zeros(1, dtype=torch.int32, device=dev)
    wsb = lib().vs_site_ex_workspace(n, R)
    ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=dev)
    opt = vs_site_options(grid.c() if grid is not None else vs_grid(0, 0, 0, 0), ht,
                          weight.data_ptr() if weight is not None else None)
    if weight is not None:
        _need_cuda(weight)
        assert weight.dtype == torch.uint8 and weight.shape == (H, W) and weight.is_contiguous()
    _check("vs_site_ex", lib().vs_site_ex(_ptr(bm), _ptr(cand), n, H, W, R, n_obs, float(target),
                                          ctypes.byref(opt), _ptr(chosen), _ptr(gains), _ptr(cum), _ptr(nch),
                                          _ptr(ws), wsb, _stream()))
    if not sync:
        return chosen, gains, cum, nch
    t = int(nch.item())
    if t < 0:
        raise VsError("vs_site_ex", t)
    return chosen[:t], gains[:t], cum, t


def site_workspace(n, R):
    return lib().vs_site_workspace(n, R)


def site(bm, cand, H, W, R, n_obs, target=0.0, cum=None, ws=None, sync=True):
    """Greedy siting.  Returns (chosen int64, gains int64, cum int32 [H, ceil(W/32)],
    n_chosen); with sync=True the lists are cut to n_chosen (a host sync)."""
    _need_cuda(bm, cand)
    dev = cand.device
    n = cand.numel()
    if cum is None:
        cum = torch.zeros((H, (W + 31) // 32), dtype=torch.int32, device=dev)
    chosen = torch.empty(max(n_obs, 1), dtype=torch.int64, device=dev)
    gains = torch.empty(max(n_obs, 1), dtype=torch.int64, device=dev)
    nch = torch.zeros(1, dtype=torch.int32, device=dev)
    wsb = site_workspace(n, R)
    if ws is None or ws.numel() < wsb:
        ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=dev)
    _check("vs_site", lib().vs_site(_ptr(bm), _ptr(cand.contiguous()), n, H, W, R, n_obs, float(target),
                                    _ptr(chosen), _ptr(gains), _ptr(cum), _ptr(nch), _ptr(ws), wsb,
                                    _stream()))
    if sync:
        t = int(nch.item())
        return chosen[:t], gains[:t], cum, t
    return chosen, gains, cum, nch


def site_gains(bm, cand, H, W, R, cum, out=None):
    """Dense gain pass: popcount(V_c AND NOT cum) for every candidate (uint32 as int32)."""
    _need_cuda(bm, cand, cum)
    n = cand.numel()
    if out is None:
        out = torch.empty(n, dtype=torch.int32, device=cand.device)
    _check("vs_site_gains", lib().vs_site_gains(_ptr(bm), _ptr(cand), n, H, W, R, _ptr(cum), _ptr(out),
                                                _stream()))
    return out


# ------------------------------------------------------------------ learned proposal
def cnn_param_count():
    return lib().vs_cnn_param_count()


def cnn_pack(master, packed=None):
    """fp32 master parameters (CUDA, cnn_param_count() values) -> packed operands."""
    _need_cuda(master)
    assert master.dtype == torch.float32 and master.numel() == cnn_param_count()
    if packed is None:
        packed = torch.empty(lib().vs_cnn_packed_bytes(), dtype=torch.uint8, device=master.device)
    _check("vs_cnn_pack", lib().vs_cnn_pack(_ptr(master), _ptr(packed), _stream()))
    return packed


def cnn_forward(g, centers, packed, out=None, save=None, status=None, patch_step=1):
    """Predicted visibility index of the patches centred on ``centers``."""
    _need_cuda(centers, packed)
    n = centers.numel()
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=centers.device)
    _check("vs_cnn_forward", lib().vs_cnn_forward(g.c(), _ptr(centers), n, patch_step, _ptr(packed),
                                                  _ptr(out), _ptr(save), _ptr(status), _stream()))
    return out


def cnn_save_bytes():
    return lib().vs_cnn_save_bytes()


def cnn_score_lattice_rows(g, stride, packed, row0, nrows, out, status=None, patch_step=1):
    """Lattice rows row0 .. row0+nrows-1 into out[nrows][ceil(W/stride)] (a view
    of the full score map is fine)."""
    Ws = (g.W + stride - 1) // stride
    if out.dtype != torch.float32 or not out.is_contiguous() or out.numel() < nrows * Ws:
        raise ValueError("out must be contiguous float32 with nrows*ceil(W/stride) elements")
    _check("vs_cnn_score_lattice_rows",
           lib().vs_cnn_score_lattice_rows(g.c(), stride, patch_step, row0, nrows, _ptr(packed), _ptr(out),
                                           _ptr(status), _stream()))
    return out


def cnn_score_lattice(g, stride, packed, out=None, status=None, patch_step=1):
    """Scores on the lattice of posts (i*stride, j*stride): [ceil(H/s), ceil(W/s)]."""
    Hs, Ws = (g.H + stride - 1) // stride, (g.W + stride - 1) // stride
    if out is None:
        out = torch.empty((Hs, Ws), dtype=torch.float32, device=g.storage.device)
    _check("vs_cnn_score_lattice", lib().vs_cnn_score_lattice(g.c(), stride, patch_step, _ptr(packed),
                                                              _ptr(out), _ptr(status), _stream()))
    return out


def cnn_backward(save, labels, master, grads, loss_sum, ws=None):
    """Accumulate the batch's gradients (see vs_cnn_backward)."""
    _need_cuda(save, labels, master, grads, loss_sum)
    B = labels.numel()
    wsb = lib().vs_cnn_backward_workspace(B)
    if ws is None or ws.numel() < wsb:
        ws = torch.empty(wsb, dtype=torch.uint8, device=labels.device)
    _check("vs_cnn_backward", lib().vs_cnn_backward(_ptr(save), _ptr(labels), B, _ptr(master), _ptr(grads),
                                                    _ptr(loss_sum), _ptr(ws), wsb, _stream()))
    return ws


def cnn_adam(master, grads, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    _need_cuda(master, grads, m, v)
    _check("vs_cnn_adam", lib().vs_cnn_adam(_ptr(master), _ptr(grads), _ptr(m), _ptr(v), step, lr, beta1,
                                            beta2, eps, _stream()))


# ------------------------------------------------------------------ batching and tuning
def launch_count():
    """Kernel launches the library has issued in this process."""
    return int(lib().vs_launch_count())


def tune_set(op, R, value):
    _check("vs_tune_set", lib().vs_tune_set(op, R, value))


def tune_get(op, R):
    return lib().vs_tune_get(op, R)


def vix_batch(jobs, ws):
    """jobs: list of dicts (g, R, ht, hr, S, seed, out) -> one persistent launch."""
    arr = (vs_vix_job * len(jobs))()
    for i, j in enumerate(jobs):
        _need_cuda(j["out"])
        arr[i].g = j["g"].c()
        arr[i].R, arr[i].ht, arr[i].hr, arr[i].S = j["R"], j["ht"], j["hr"], j["S"]
        arr[i].seed = j["seed"] % (1 << 64)
        arr[i].vix_out = j["out"].data_ptr()
    _check("vs_vix_batch", lib().vs_vix_batch(ctypes.cast(arr, ctypes.c_void_p), len(jobs), _ptr(ws),
                                              ws.numel(), _stream()))


def findmax_batch(jobs):
    """jobs: list of dicts (vix (H x W uint8), block, k, out) -> one launch."""
    arr = (vs_findmax_job * len(jobs))()
    for i, j in enumerate(jobs):
        _need_cuda(j["vix"], j["out"])
        H, W = j["vix"].shape
        arr[i].vix = j["vix"].data_ptr()
        arr[i].H, arr[i].W, arr[i].block, arr[i].k = H, W, j["block"], j["k"]
        arr[i].cand_out = j["out"].data_ptr()
        arr[i].cap = j["out"].numel()
    _check("vs_findmax_batch", lib().vs_findmax_batch(ctypes.cast(arr, ctypes.c_void_p), len(jobs), _stream()))


def viewshed_batch(jobs, ws):
    """jobs: list of dicts (g, R, ht, hr, cand, bm, area) -> one persistent launch."""
    arr = (vs_viewshed_job * len(jobs))()
    for i, j in enumerate(jobs):
        _need_cuda(j["cand"], j["bm"], j["area"])
        arr[i].g = j["g"].c()
        arr[i].R, arr[i].ht, arr[i].hr = j["R"], j["ht"], j["hr"]
        arr[i].cand = j["cand"].data_ptr()
        arr[i].n = j["cand"].numel()
        arr[i].bm_out = j["bm"].data_ptr()
        arr[i].area_out = j["area"].data_ptr()
    _check("vs_viewshed_batch", lib().vs_viewshed_batch(ctypes.cast(arr, ctypes.c_void_p), len(jobs),
                                                        _ptr(ws), ws.numel(), _stream()))


def site_jobs(jobs):
    arr = (vs_site_job * len(jobs))()
    for i, j in enumerate(jobs):
        arr[i].bm = j["bm"].data_ptr()
        arr[i].cand = j["cand"].data_ptr()
        arr[i].n = j["cand"].numel()
        arr[i].H, arr[i].W, arr[i].R, arr[i].n_obs = j["H"], j["W"], j["R"], j["n_obs"]
        arr[i].coverage_target = float(j.get("target", 0.0))
        arr[i].chosen = j["chosen"].data_ptr()
        arr[i].gains = j["gains"].data_ptr()
        arr[i].cum = j["cum"].data_ptr()
        arr[i].n_chosen = j["n_chosen"].data_ptr()
    return arr


def site_batch_workspace(jobs):
    arr = site_jobs(jobs)
    return lib().vs_site_batch_workspace(ctypes.cast(arr, ctypes.c_void_p), len(jobs))


def site_batch(jobs, ws):
    arr = site_jobs(jobs)
    _check("vs_site_batch", lib().vs_site_batch(ctypes.cast(arr, ctypes.c_void_p), len(jobs), _ptr(ws),
                                                ws.numel(), _stream()))


def selftest_wait_timeout(polls=4096):
    """Runs a kernel whose bounded wait must give up; returns the status it wrote."""
    st = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    _check("vs_selftest_wait_timeout", lib().vs_selftest_wait_timeout(_ptr(st), polls, _stream()))
    torch.cuda.synchronize()
    return int(st.item())
