"""GB300 (sm_103a) observer-siting hot path: vix, findmax, viewshed and site
kernels behind the C ABI of include/vshed.h, with a thin ctypes binding."""
from .vshed import (Grid, VsError, bitmap_words, findmax, findmax_count, findmax_f32, lib,
                    site, site_gains, site_workspace, viewshed, vix, vix_count, words_per_row)

__all__ = ["Grid", "VsError", "bitmap_words", "findmax", "findmax_count", "findmax_f32", "lib",
           "site", "site_gains", "site_workspace", "viewshed", "vix", "vix_count", "words_per_row"]
