"""The C-ABI library: it loads without a GPU, exports every symbol that
include/vshed.h declares, and its host-side argument checks and size queries
answer without touching a device.  CPU only (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2006_16783_gb300 import _build
    _build.build()
    from paper_2006_16783_gb300 import vshed
    return vshed.lib()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(vs_[a-z0-9_]+)\s*\(", src))
    return names


def test_every_declared_symbol_exported(L):
    names = _declared()
    assert {"vs_vix", "vs_findmax", "vs_viewshed", "vs_site"} <= names
    for n in sorted(names):
        assert hasattr(L, n), n


def test_binding_covers_header():
    from paper_2006_16783_gb300 import vshed
    assert _declared() <= set(vshed.SIGNATURES)


def test_size_queries(L):
    from oracle import oracle as O
    for R in (1, 2, 7, 50, 100, 200, 250, 1000):
        assert L.vs_bitmap_words(R) == O.bitmap_words(R)
    assert L.vs_bitmap_words(0) < 0
    # Findmax counts: DEM1000's 100 x 100 blocks of 20 (Table t:1000) and the
    # workloads' 1600 / 8192 / 40000 candidates
    assert L.vs_findmax_count(1000, 1000, 1, 10, 20) == 200000
    assert L.vs_findmax_count(1000, 1000, 1, 25, 1) == 1600
    assert L.vs_findmax_count(16384, 16384, 1, 256, 2) == 8192
    assert L.vs_findmax_count(46400, 46400, 1, 464, 4) == 40000
    # a partial edge block with fewer posts than k contributes all of them
    # 5 x 7 posts in 3 x 3 blocks hold 9, 9, 3 / 6, 6, 2 posts
    assert L.vs_findmax_count(5, 7, 1, 3, 5) == 5 + 5 + 3 + 5 + 5 + 2
    # stride-4 lattice {0,4,8}^2 in 8 x 8 blocks: 4, 2 / 2, 1 lattice posts
    assert L.vs_findmax_count(10, 10, 4, 8, 2) == 2 + 2 + 2 + 1
    assert L.vs_site_workspace(40000, 100) >= 40000 * 4
    # the paper's US-West run (Sec. "Experiments"): 139 x 139 blocks of 20 potential
    # transmitters, 386,420 in all, for R = 1000 (block side 334 ~ R/3); R = 2000:
    # 70 x 70 blocks, 98,000
    assert L.vs_findmax_count(46400, 46400, 1, 334, 20) == 386420
    assert L.vs_findmax_count(46400, 46400, 1, 667, 20) == 98000


def test_argument_errors_need_no_device(L):
    from paper_2006_16783_gb300 import vshed
    g = vshed.vs_grid(10, 10, 16, 0)       # null terrain
    assert L.vs_vix(g, 5, 1, 1, 10, 1, None, None) == vshed.VS_ERR_ARG
    g = vshed.vs_grid(10, 10, 12, 4096)    # pitch not a multiple of 8
    assert L.vs_vix(g, 5, 1, 1, 10, 1, ctypes.c_void_p(4096), None) == vshed.VS_ERR_ARG
    g = vshed.vs_grid(10, 10, 16, 4096)
    assert L.vs_vix(g, 0, 1, 1, 10, 1, ctypes.c_void_p(4096), None) == vshed.VS_ERR_RANGE
    assert L.vs_vix(g, 5, 1, 1, 256, 1, ctypes.c_void_p(4096), None) == vshed.VS_ERR_RANGE
    assert L.vs_viewshed(g, 5, 1, 1, None, 3, None, None, None, 0, None) == vshed.VS_ERR_ARG
    assert L.vs_findmax(None, 10, 10, 2, 1, None, 0, None) == vshed.VS_ERR_ARG
    assert L.vs_site(None, ctypes.c_void_p(8), 1, 10, 10, 2, 1, 0.0, ctypes.c_void_p(8),
                     ctypes.c_void_p(8), ctypes.c_void_p(8), ctypes.c_void_p(8), None, 0,
                     None) == vshed.VS_ERR_ARG
    assert L.vs_site(ctypes.c_void_p(8), ctypes.c_void_p(8), 1, 10, 10, 2, 1, 0.0, ctypes.c_void_p(8),
                     ctypes.c_void_p(8), ctypes.c_void_p(8), ctypes.c_void_p(8), None, 0,
                     None) == vshed.VS_ERR_WS
    assert L.vs_strerror(-3) == b"workspace missing or too small"


def test_binding_refuses_cpu_tensors():
    import torch
    import paper_2006_16783_gb300 as V
    with pytest.raises(ValueError):
        V.findmax(torch.zeros((4, 4), dtype=torch.uint8), 2, 1)


def test_large_roi_size_queries(L):
    """Workspaces of the large-ROI paths: none while the staged kernels cover
    R, pair arrays (8 bytes per post) beyond; tuning values checked."""
    from paper_2006_16783_gb300 import vshed
    assert L.vs_viewshed_workspace(1000, 1000, 100, 10) == 0
    assert L.vs_viewshed_workspace(1000, 1000, 280, 10) == 0
    assert L.vs_viewshed_workspace(1000, 1200, 1000, 10) >= 8 * 1000 * 1200
    assert L.vs_vix_workspace(1000, 1000, 100, 10) == 0
    assert L.vs_vix_workspace(1000, 1200, 1000, 10) >= 8 * 1000 * 1200
    assert L.vs_viewshed_r3_workspace(300, 400) >= 8 * 300 * 400
    assert L.vs_site_ex_workspace(1000, 100) > L.vs_site_workspace(1000, 100)
    # forcing the large-ROI kernels at a small R makes them need the workspace
    assert L.vs_tune_set(vshed.VS_TUNE_VIEWSHED_WIDE, 50, 1) == 0
    try:
        assert L.vs_viewshed_workspace(500, 500, 50, 10) > 0
    finally:
        L.vs_tune_set(vshed.VS_TUNE_VIEWSHED_WIDE, 50, 0)
    assert L.vs_viewshed_workspace(500, 500, 50, 10) == 0
    assert L.vs_tune_set(vshed.VS_TUNE_VIEWSHED_WIDE, 50, 2) == vshed.VS_ERR_RANGE
    assert L.vs_tune_set(vshed.VS_TUNE_SITE_LAZY, 50, 3) == vshed.VS_ERR_RANGE
    assert L.vs_tune_set(vshed.VS_TUNE_VIX_TILE, 50, 4) == vshed.VS_ERR_RANGE
    assert L.vs_tune_set(vshed.VS_TUNE_SITE_MULTI, 50, 2) == vshed.VS_ERR_RANGE
    assert L.vs_tune_set(vshed.VS_TUNE_SITE_BARRIER_TEST, 50, (1 << 20) + 1) == vshed.VS_ERR_RANGE
    assert L.vs_tune_set(7, 50, 0) == vshed.VS_ERR_RANGE


def test_large_roi_argument_errors_need_no_device(L):
    from paper_2006_16783_gb300 import vshed
    g = vshed.vs_grid(300, 320, 320, 4096)
    d = ctypes.c_void_p(4096)
    # banded viewshed: workspace missing
    assert L.vs_viewshed(g, 400, 10, 10, d, 3, d, d, None, 0, None) == vshed.VS_ERR_WS
    # heights out of range, R out of range
    assert L.vs_viewshed(g, 400, 200001, 10, d, 3, d, d, None, 0, None) == vshed.VS_ERR_RANGE
    assert L.vs_viewshed_r3(g, 0, 10, 10, d, 3, d, d, None, 0, None) == vshed.VS_ERR_RANGE
    assert L.vs_viewshed_r3(g, 5, 10, 10, None, 3, d, d, None, 0, None) == vshed.VS_ERR_ARG
    # site with options: terrain of another size, workspace missing, weights too
    # wide for 32-bit gains
    opt = vshed.vs_site_options(vshed.vs_grid(100, 100, 104, 4096), 10, None)
    assert L.vs_site_ex(d, d, 3, 300, 320, 20, 5, 0.0, ctypes.byref(opt), d, d, d, d, d, 1 << 20,
                        None) == vshed.VS_ERR_ARG
    opt = vshed.vs_site_options(g, 10, None)
    assert L.vs_site_ex(d, d, 3, 300, 320, 20, 5, 0.0, ctypes.byref(opt), d, d, d, d, None, 0,
                        None) == vshed.VS_ERR_WS
    opt = vshed.vs_site_options(vshed.vs_grid(0, 0, 0, 0), 0, 4096)
    assert L.vs_site_ex(d, d, 3, 300, 320, 2100, 5, 0.0, ctypes.byref(opt), d, d, d, d, d, 1 << 30,
                        None) == vshed.VS_ERR_RANGE


def test_site_noalloc_limit(L):
    """vs_site_noalloc's static scratch (VS_SITE_NOALLOC_MAX_BYTES = 1 MiB)
    holds the workspace of up to 37,439 candidates at any R; one more needs
    more than the array and is refused before anything runs."""
    for R in (1, 9, 40, 100, 1000):
        assert L.vs_site_workspace(37439, R) <= 1 << 20 < L.vs_site_workspace(37440, R)
    from paper_2006_16783_gb300 import vshed
    dummy = ctypes.c_void_p(256)
    rc = L.vs_site_noalloc(dummy, dummy, 37440, 300, 300, 9, 10, 0.0, dummy, dummy, dummy, dummy, None)
    assert rc == vshed.VS_ERR_RANGE


def test_exact_vix_queries_need_no_device(L):
    from paper_2006_16783_gb300 import vshed
    assert L.vs_exact_vix_workspace(1000, 1000, 100, 500) >= 4 * 500
    assert L.vs_exact_vix_workspace(1000, 1200, 1000, 10) >= 8 * 1000 * 1200 + 10 * 4 * 2001 * 64
    assert L.vs_exact_vix_workspace(1000, 1000, 0, 10) == 0
    g = vshed.vs_grid(100, 100, 104, None)
    dummy = ctypes.c_void_p(256)
    assert L.vs_exact_vix(g, 10, 10, 10, dummy, 5, dummy, dummy, 1 << 20, None) == vshed.VS_ERR_ARG
    g = vshed.vs_grid(100, 100, 104, dummy)
    assert L.vs_exact_vix(g, 0, 10, 10, dummy, 5, dummy, dummy, 1 << 20, None) == vshed.VS_ERR_RANGE
    assert L.vs_exact_vix(g, 10, 10, 10, dummy, 5, dummy, None, 0, None) == vshed.VS_ERR_WS
