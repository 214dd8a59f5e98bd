"""Python face of the CPU oracle (test infrastructure only).

The oracle is ``vshed_oracle.c`` compiled with the host C compiler into
``liboracle.so`` beside this file.  Only the tests, ``__graft_entry__.smoke``
and the benchmark's CPU-baseline leg may import this module; the CUDA library
never links or calls it.  Every function takes and returns numpy arrays.

Each wrapper restates which step of the paper (Franklin, Magalhaes & Li,
arXiv 2006.16783, Sec. "The multiple transmitter siting process") it follows;
the arithmetic itself lives in the C file.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vshed_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force=False):
    """Compile the oracle with gcc (plain -O2, no target-specific flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    L = ctypes.CDLL(_LIB)
    P = ctypes.c_void_p
    i32, i64, u64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    sig = {
        "or_disc_count": (i64, [i32]),
        "or_offsets": (i64, [i32, P, P]),
        "or_splitmix64_mix": (u64, [u64]),
        "or_splitmix64_nth": (u64, [u64, u64]),
        "or_los": (ctypes.c_int, [P, i32, i32, i64, i32, i32, i32, i32, i32, i32]),
        "or_vix": (ctypes.c_int, [P, i32, i32, i64, i32, i32, i32, i32, u64, P, i32]),
        "or_vix_posts": (ctypes.c_int, [P, i32, i32, i64, i32, i32, i32, i32, u64, P, i64, P]),
        "or_findmax": (i64, [P, i32, i32, i32, i32, P, i64]),
        "or_findmax_f32": (i64, [P, i32, i32, i32, i32, i32, P, i64]),
        "or_bitmap_words": (i64, [i32]),
        "or_viewshed": (ctypes.c_int, [P, i32, i32, i64, i32, i32, i32, P, i64, P, P, i32]),
        "or_viewshed_brute": (ctypes.c_int, [P, i32, i32, i64, i32, i32, i32, i64, P]),
        "or_exact_vix": (ctypes.c_int, [P, i32, i32, i64, i32, i32, i32, P, i64, P, i32]),
        "or_site_plain": (i32, [P, P, i64, i32, i32, i32, i32, f64, P, P, P]),
        "or_site_lazy": (i32, [P, P, i64, i32, i32, i32, i32, f64, P, P, P]),
        "or_coverage_need": (i64, [f64, i32, i32]),
        "or_cum_popcount": (i64, [P, i32, i32]),
        "or_cum_rebuild": (None, [P, P, i64, i32, i32, i32, P]),
        "or_intervisible": (ctypes.c_int, [P, i32, i32, i64, i32, i32, i64, i64]),
        "or_site_ex": (i32, [P, P, i64, i32, i32, i32, i32, f64, P, i64, i32, P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


def _grid(z):
    z = np.ascontiguousarray(z, dtype=np.int16)
    assert z.ndim == 2
    return z, z.shape[0], z.shape[1], z.shape[1]


# ---------------------------------------------------------------- helpers
def disc_count(R):
    """|{(dx,dy): dx^2+dy^2 <= R^2}|."""
    return _load().or_disc_count(R)


def offsets(R):
    """OFF_R: disc(R) minus the origin, ordered by dy then dx (Vix stage)."""
    n = _load().or_offsets(R, None, None)
    dx = np.zeros(n, np.int32)
    dy = np.zeros(n, np.int32)
    _load().or_offsets(R, _p(dx), _p(dy))
    return dx, dy


def splitmix64_nth(seed, i):
    """i-th (0-based) output of SplitMix64 seeded with ``seed``."""
    return _load().or_splitmix64_nth(seed & (2**64 - 1), i & (2**64 - 1))


def bitmap_words(R):
    """Words of one viewshed bitmap: (2R+1) * (floor(2R/32) + 2)."""
    return _load().or_bitmap_words(R)


def words_per_row(R):
    return (2 * R) // 32 + 2


def cum_words_per_row(W):
    return (W + 31) // 32


# ---------------------------------------------------------------- LOS / vix
def los(z, ox, oy, tx, ty, ht, hr):
    """Line of sight O->T with linear interpolation between posts (Sec.
    "Terrain visibility"); True iff T (at z+hr) is visible from O (at z+ht)."""
    z, H, W, pitch = _grid(z)
    return bool(_load().or_los(_p(z), H, W, pitch, ox, oy, tx, ty, ht, hr))


def vix(z, R, ht, hr, S, seed, threads=1):
    """Sampled visibility index count per post, uint8 H x W (Vix stage)."""
    z, H, W, pitch = _grid(z)
    out = np.zeros((H, W), np.uint8)
    rc = _load().or_vix(_p(z), H, W, pitch, R, ht, hr, S, seed & (2**64 - 1), _p(out), threads)
    if rc != 0:
        raise ValueError("or_vix: bad arguments")
    return out


def vix_posts(z, R, ht, hr, S, seed, posts, W=None):
    """Vix counts of the listed posts only.  ``z`` may be pitched: pass the
    logical width W when z has padding columns."""
    z = np.ascontiguousarray(z, dtype=np.int16)
    H, pitch = z.shape
    W = pitch if W is None else W
    posts = np.ascontiguousarray(posts, dtype=np.int64)
    out = np.zeros(posts.shape[0], np.uint8)
    rc = _load().or_vix_posts(_p(z), H, W, pitch, R, ht, hr, S, seed & (2**64 - 1), _p(posts),
                              posts.shape[0], _p(out))
    if rc != 0:
        raise ValueError("or_vix_posts: bad arguments")
    return out


# ---------------------------------------------------------------- findmax
def findmax(v, b, k):
    """Top-k posts per b x b block by (count desc, post index asc), ordered by
    block row-major then rank (Findmax stage).  Returns int64 post indices."""
    v = np.ascontiguousarray(v, dtype=np.uint8)
    H, W = v.shape
    n = _load().or_findmax(_p(v), H, W, b, k, None, 0)
    out = np.zeros(max(n, 1), np.int64)
    _load().or_findmax(_p(v), H, W, b, k, _p(out), n)
    return out[:n]


def findmax_f32(score, H, W, stride, b, k):
    """Findmax over a float score lattice of the given stride (the learned
    proposal's predicted map).  score has shape (ceil(H/stride), ceil(W/stride))."""
    score = np.ascontiguousarray(score, dtype=np.float32)
    assert score.shape == ((H + stride - 1) // stride, (W + stride - 1) // stride)
    n = _load().or_findmax_f32(_p(score), H, W, stride, b, k, None, 0)
    out = np.zeros(max(n, 1), np.int64)
    _load().or_findmax_f32(_p(score), H, W, stride, b, k, _p(out), n)
    return out[:n]


# ---------------------------------------------------------------- viewshed
def viewshed(z, R, ht, hr, cand, threads=1):
    """Ray-sweep viewshed bitmaps (Viewshed stage): returns
    (uint32 [n, 2R+1, P_R], int32 area[n])."""
    z, H, W, pitch = _grid(z)
    cand = np.ascontiguousarray(cand, dtype=np.int64)
    n = cand.shape[0]
    bm = np.zeros((n, 2 * R + 1, words_per_row(R)), np.uint32)
    area = np.zeros(n, np.int32)
    rc = _load().or_viewshed(_p(z), H, W, pitch, R, ht, hr, _p(cand), n, _p(bm), _p(area), threads)
    if rc != 0:
        raise ValueError("or_viewshed: bad arguments (%d)" % rc)
    return bm, area


def exact_vix(z, R, ht, hr, posts, threads=1):
    """Exact visibility index of each post (Sec. "Definitions"): its
    viewshed's area over the ROI's lattice points inside the grid (float32;
    -1 for a post outside the grid)."""
    z, H, W, pitch = _grid(z)
    posts = np.ascontiguousarray(posts, dtype=np.int64)
    out = np.zeros(posts.shape[0], np.float32)
    rc = _load().or_exact_vix(_p(z), H, W, pitch, R, ht, hr, _p(posts), posts.shape[0], _p(out), threads)
    if rc != 0:
        raise ValueError("or_exact_vix: bad arguments (%d)" % rc)
    return out


def viewshed_brute(z, R, ht, hr, p):
    """Per-cell LOS viewshed of one observer (definition read literally)."""
    z, H, W, pitch = _grid(z)
    bm = np.zeros((2 * R + 1, words_per_row(R)), np.uint32)
    _load().or_viewshed_brute(_p(z), H, W, pitch, R, ht, hr, int(p), _p(bm))
    return bm


def bitmap_to_window(bm, R, cx, W=None):
    """Expand one bitmap into a bool (2R+1) x (2R+1) window centred on the
    observer (column cx-R+i, row cy-R+j).  Helper for tests."""
    PR = words_per_row(R)
    gw0 = (cx - R) // 32
    bits = np.unpackbits(bm.reshape(2 * R + 1, PR).view(np.uint8), axis=1, bitorder="little")
    col0 = (cx - R) - 32 * gw0
    return bits[:, col0:col0 + 2 * R + 1].astype(bool)


# ---------------------------------------------------------------- site
def site(bm, cand, H, W, R, n_obs, target=0.0, cum=None, lazy=True):
    """Greedy siting (Site stage).  Returns (chosen int64[t], gains int64[t],
    cum uint32 [H, ceil(W/32)]).  ``cum`` (optional) is the starting
    cumulative viewshed; it is copied, not modified."""
    bm = np.ascontiguousarray(bm, dtype=np.uint32)
    cand = np.ascontiguousarray(cand, dtype=np.int64)
    n = cand.shape[0]
    C = np.zeros((H, cum_words_per_row(W)), np.uint32) if cum is None else np.array(cum, np.uint32, copy=True)
    chosen = np.zeros(max(n_obs, 1), np.int64)
    gains = np.zeros(max(n_obs, 1), np.int64)
    fn = _load().or_site_lazy if lazy else _load().or_site_plain
    t = fn(_p(bm), _p(cand), n, H, W, R, n_obs, float(target), _p(chosen), _p(gains), _p(C))
    return chosen[:t].copy(), gains[:t].copy(), C


def coverage_need(target, H, W):
    return _load().or_coverage_need(float(target), H, W)


def cum_popcount(cum, H, W):
    cum = np.ascontiguousarray(cum, dtype=np.uint32)
    return _load().or_cum_popcount(_p(cum), H, W)


def cum_rebuild(bm, cand, H, W, R):
    """Cumulative viewshed of a list of observers (OR of their bitmaps)."""
    bm = np.ascontiguousarray(bm, dtype=np.uint32)
    cand = np.ascontiguousarray(cand, dtype=np.int64)
    C = np.zeros((H, cum_words_per_row(W)), np.uint32)
    _load().or_cum_rebuild(_p(bm), _p(cand), cand.shape[0], H, W, R, _p(C))
    return C


# ---------------------------------------------------------------- site with constraints
def intervisible(z, R, ht, pa, pb):
    """Posts pa and pb within the ROI and the line between their antenna tops
    (both z + ht) clear of the terrain."""
    z, H, W, pitch = _grid(z)
    return bool(_load().or_intervisible(_p(z), H, W, pitch, R, ht, int(pa), int(pb)))


def site_ex(bm, cand, H, W, R, n_obs, target=0.0, z=None, ht=0, weight=None, cum=None):
    """Plain greedy with the optional intervisibility constraint (terrain z
    given: every transmitter after the first intervisible with one already
    chosen) and optional uint8 receiver weights (H x W).  Returns (chosen,
    gains, cum)."""
    bm = np.ascontiguousarray(bm, dtype=np.uint32)
    cand = np.ascontiguousarray(cand, dtype=np.int64)
    n = cand.shape[0]
    cum = np.zeros((H, cum_words_per_row(W)), np.uint32) if cum is None else np.array(cum, dtype=np.uint32)
    chosen = np.zeros(max(n_obs, 1), np.int64)
    gains = np.zeros(max(n_obs, 1), np.int64)
    zp, pitch = None, 0
    if z is not None:
        zp, _, _, pitch = _grid(z)
    wt = None if weight is None else np.ascontiguousarray(weight, dtype=np.uint8)
    t = _load().or_site_ex(_p(bm), _p(cand), n, H, W, R, n_obs, float(target),
                           _p(zp) if zp is not None else None, pitch, ht,
                           _p(wt) if wt is not None else None, _p(chosen), _p(gains), _p(cum))
    return chosen[:t], gains[:t], cum
