"""Pins for the CPU oracle against facts fixed by the paper and by mathematics
(hand-worked examples, closed forms, invariants, brute force, the published
SplitMix64 test vector).  CPU only."""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from synth import terrain as T

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([int(t) for t in line.split()])
    return rows


# ------------------------------------------------------------------ RNG
def test_splitmix64_published_vector(O):
    # SplitMix64 (Steele, Lea & Flood 2014) seeded with 1234567: the first five
    # outputs published with the reference implementation.
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423,
            4593380528125082431, 16408922859458223821]
    assert [O.splitmix64_nth(1234567, i) for i in range(5)] == want


# ------------------------------------------------------------------ disc / offsets
@pytest.mark.parametrize("R", [1, 2, 3, 7, 30, 50, 100, 150, 200, 250])
def test_disc_count_row_formula(O, R):
    # |disc(R)| = sum over rows dy of (2*isqrt(R^2 - dy^2) + 1)
    want = sum(2 * math.isqrt(R * R - dy * dy) + 1 for dy in range(-R, R + 1))
    assert O.disc_count(R) == want


def test_disc_counts_quoted():
    # the lattice-point counts quoted for the workloads (R = 50..250)
    from oracle import oracle as O
    assert [O.disc_count(r) for r in (50, 100, 150, 200, 250)] == [7845, 31417, 70681, 125629, 196321]


@pytest.mark.parametrize("R", [1, 5, 30])
def test_offset_table(O, R):
    dx, dy = O.offsets(R)
    assert len(dx) == O.disc_count(R) - 1
    pairs = list(zip(dy.tolist(), dx.tolist()))
    assert pairs == sorted(pairs) and len(set(pairs)) == len(pairs)
    assert (0, 0) not in pairs
    assert all(a * a + b * b <= R * R for b, a in pairs)


# ------------------------------------------------------------------ LOS
def test_los_golden_5x5(O):
    rows = _read_golden("los_5x5.txt")
    H, W = rows[0]
    z = np.array(rows[1:1 + H], np.int16)
    for ox, oy, tx, ty, ht, hr, vis in rows[1 + H:]:
        assert O.los(z, ox, oy, tx, ty, ht, hr) == bool(vis), (ox, oy, tx, ty, ht, hr)


def test_los_flat_all_visible(O):
    z = np.full((21, 23), 77, np.int16)
    for (tx, ty) in itertools.product(range(23), range(21)):
        for ht, hr in [(0, 0), (10, 0), (0, 10), (3, 7)]:
            assert O.los(z, 11, 10, tx, ty, ht, hr)


@pytest.mark.parametrize("direction", [(1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (1, -1), (-1, -1)])
def test_los_spike_closed_form(O, direction):
    # Flat ground at 0, one spike of height S at step j on an axis or diagonal
    # LOS (the crossing is exactly at the post, f = 0), target at step D.
    # Eye at ht, target at hr.  Blocked exactly when the spike's slope exceeds
    # the target's: (S - ht)/j > (hr - ht)/D  <=>  (S - ht)*D > (hr - ht)*j.
    sx, sy = direction
    N = 25
    o = 12
    for D in range(2, 12):
        for j in range(1, D):
            for S_h in (0, 3, 9, 40):
                for ht, hr in [(0, 0), (5, 5), (10, 2), (1, 30)]:
                    z = np.zeros((N, N), np.int16)
                    z[o + sy * j, o + sx * j] = S_h
                    want = not ((S_h - ht) * D > (hr - ht) * j)
                    got = O.los(z, o, o, o + sx * D, o + sy * D, ht, hr)
                    assert got == want, (D, j, S_h, ht, hr)


def _los_rational(z, ox, oy, tx, ty, ht, hr):
    """Independent geometric restatement with exact rationals: walk the
    segment, at every crossing of a grid line perpendicular to the major axis
    interpolate the terrain linearly between the two straddling posts and
    compare elevation angles (as slope = rise / horizontal distance)."""
    H, W = z.shape
    if not (0 <= tx < W and 0 <= ty < H):
        return False
    dx, dy = tx - ox, ty - oy
    D = max(abs(dx), abs(dy))
    if D == 0:
        return True
    e = Fraction(int(z[oy, ox]) + ht)
    length = Fraction(1)  # common factor of all horizontal distances: cancels
    target = (Fraction(int(z[ty, tx]) + hr) - e) / (D * length)
    for j in range(1, D):
        t = Fraction(j, D)
        px, py = ox + dx * t, oy + dy * t
        if abs(dx) >= abs(dy):
            px = int(px)                          # on a column exactly
            y0 = math.floor(py)
            w = py - y0
            h = int(z[y0, px]) * (1 - w) + (int(z[y0 + 1, px]) * w if w else 0)
        else:
            py = int(py)                          # on a row exactly
            x0 = math.floor(px)
            w = px - x0
            h = int(z[py, x0]) * (1 - w) + (int(z[py, x0 + 1]) * w if w else 0)
        if (Fraction(h) - e) / (j * length) > target:
            return False
    return True


def test_los_matches_rational_geometry(O):
    rng = np.random.default_rng(5)
    for trial in range(12):
        N = 17
        z = rng.integers(0, 12 if trial % 2 else 300, (N, N)).astype(np.int16)
        ht, hr = int(rng.integers(0, 6)), int(rng.integers(0, 6))
        ox, oy = int(rng.integers(0, N)), int(rng.integers(0, N))
        for tx in range(N):
            for ty in range(N):
                assert O.los(z, ox, oy, tx, ty, ht, hr) == _los_rational(z, ox, oy, tx, ty, ht, hr)


def test_los_target_outside_grid(O):
    z = np.zeros((8, 8), np.int16)
    assert not O.los(z, 0, 0, -1, 0, 10, 10)
    assert not O.los(z, 7, 7, 8, 7, 10, 10)


# ------------------------------------------------------------------ vix
def test_vix_flat_interior_counts_S(O):
    R, S = 6, 10
    z = np.full((40, 40), 500, np.int16)
    v = O.vix(z, R, 10, 10, S, seed=99)
    assert (v[R:-R, R:-R] == S).all()          # every sample inside the grid, all visible
    assert (v <= S).all()
    assert v[0, 0] < S                           # a corner loses samples that fall off the grid


def test_vix_sample_definition(O):
    # count(p) == number of visible LOS among the S SplitMix64-chosen offsets
    R, S, seed = 5, 7, 12345
    rng = np.random.default_rng(2)
    z = rng.integers(0, 40, (24, 21)).astype(np.int16)
    v = O.vix(z, R, 3, 2, S, seed)
    dx, dy = O.offsets(R)
    NR = len(dx)
    H, W = z.shape
    for p in [0, 5, 100, 250, H * W - 1]:
        x, y = p % W, p // W
        c = 0
        for s in range(S):
            u = O.splitmix64_nth(seed, p * S + s)
            idx = ((u >> 32) * NR) >> 32
            c += O.los(z, x, y, x + int(dx[idx]), y + int(dy[idx]), 3, 2)
        assert v[y, x] == c


GAMMA = 0x9E3779B97F4A7C15


def test_vix_sample_mapping_golden(O):
    """Each of the five hand-worked rows of tests/golden/vix_samples_R5.txt
    (published SplitMix64 output -> top 32 bits -> offset index -> offset)
    fixes which receiver a sample tests: on flat terrain (everything visible)
    lowering that one receiver post hides the sample, so a single-sample vix
    drops from 1 to 0; with all five samples of one post, the count is five
    minus the lowered receivers among them."""
    rows = _read_golden("vix_samples_R5.txt")
    R, H, W, cx, cy = 5, 15, 15, 7, 7
    p = cy * W + cx
    dx_t, dy_t = O.offsets(R)
    assert len(dx_t) == 80
    for m, u, hi, NR, idx, dx, dy in rows:
        assert O.splitmix64_nth(1234567, m) == u and u >> 32 == hi and NR == len(dx_t)
        assert (int(dx_t[idx]), int(dy_t[idx])) == (dx, dy)
        seed1 = (1234567 + GAMMA * (m - p)) % 2 ** 64      # S = 1: sample 0 of post p is output m
        z = np.zeros((H, W), np.int16)
        assert O.vix(z, R, 0, 0, 1, seed1)[cy, cx] == 1
        z[cy + dy, cx + dx] = -100
        assert O.vix(z, R, 0, 0, 1, seed1)[cy, cx] == 0
    seed5 = (1234567 - GAMMA * (p * 5)) % 2 ** 64           # S = 5: samples 0..4 are outputs 0..4
    for hidden in ([0, 2], [1, 3, 4], [4], []):
        z = np.zeros((H, W), np.int16)
        for m in hidden:
            _, _, _, _, _, dx, dy = rows[m]
            z[cy + dy, cx + dx] = -100
        assert O.vix(z, R, 0, 0, 5, seed5)[cy, cx] == 5 - len(hidden)


def test_vix_threads_agree(O):
    z = T.spectral_fbm(48, 40, 0.8, 3).numpy()
    a = O.vix(z, 8, 10, 10, 10, 1)
    b = O.vix(z, 8, 10, 10, 10, 1, threads=3)
    assert (a == b).all()


# ------------------------------------------------------------------ findmax
def _findmax_brute(v, b, k):
    H, W = v.shape
    out = []
    for by in range(0, H, b):
        for bx in range(0, W, b):
            items = []
            for y in range(by, min(H, by + b)):
                for x in range(bx, min(W, bx + b)):
                    items.append((-int(v[y, x]), y * W + x))
            items.sort()
            out += [p for _, p in items[:k]]
    return np.array(out, np.int64)


@pytest.mark.parametrize("H,W,b,k", [(30, 30, 5, 2), (31, 17, 8, 3), (10, 10, 3, 20), (7, 9, 25, 1)])
def test_findmax_brute(O, H, W, b, k):
    rng = np.random.default_rng(H * W + k)
    v = rng.integers(0, 4, (H, W)).astype(np.uint8)   # many ties
    assert (O.findmax(v, b, k) == _findmax_brute(v, b, k)).all()


@pytest.mark.parametrize("rows,cols,b,k,want", [
    (1000, 1000, 10, 20, 200000),     # DEM1000: 100 x 100 blocks, 20 per block (Table t:1000)
    (1000, 1000, 25, 1, 1600),        # the small synthetic workload
])
def test_findmax_count_formula(O, rows, cols, b, k, want):
    v = np.zeros((rows, cols), np.uint8)
    assert len(O.findmax(v, b, k)) == want


def test_findmax_paper_counts_arithmetic():
    # Tables t:useast and t:uswest: total potential transmitters = blocks^2 * 20
    for nb, want in [(193, 744980), (96, 184320), (139, 386420), (70, 98000)]:
        assert nb * nb * 20 == want


def test_findmax_f32_stride(O):
    rng = np.random.default_rng(0)
    H, W, s = 37, 45, 4
    sc = rng.random(((H + s - 1) // s, (W + s - 1) // s)).astype(np.float32)
    sc[2, 3] = sc[2, 4]                                   # a tie
    got = O.findmax_f32(sc, H, W, s, 10, 2)
    # brute force in post coordinates
    out = []
    for by in range(0, H, 10):
        for bx in range(0, W, 10):
            items = []
            for i in range(sc.shape[0]):
                for j in range(sc.shape[1]):
                    y, x = i * s, j * s
                    if by <= y < by + 10 and bx <= x < bx + 10:
                        items.append((-float(sc[i, j]), y * W + x))
            items.sort()
            out += [p for _, p in items[:2]]
    assert got.tolist() == out


def _f32(bits):
    return np.array([bits], np.uint32).view(np.float32)[0]


def test_findmax_f32_total_order(O):
    """Float scores rank by the IEEE-754 totalOrder predicate (IEEE 754-2008
    Sec. 5.10): -NaN < -inf < negative numbers < -0 < +0 < positive numbers
    < +inf < +NaN.  So +0 beats -0 although they compare equal (a numeric
    tie would go to the lower post), a positive NaN beats +inf and a
    negative NaN loses to -inf."""
    pnan, nnan = _f32(0x7FC00000), _f32(0xFFC00000)
    vals = np.array([[-0.0, 0.0, pnan, nnan, np.inf, -np.inf, 1.5, -1.5]], np.float32)
    got = O.findmax_f32(vals, 1, 8, 1, 8, 8).tolist()
    assert got == [2, 4, 6, 1, 0, 7, 5, 3]
    assert O.findmax_f32(vals[:, :2].copy(), 1, 2, 1, 2, 1).tolist() == [1]
    same = np.array([[0.0, 0.0, -0.0, -0.0]], np.float32)  # equal keys: lower post first
    assert O.findmax_f32(same, 1, 4, 1, 4, 4).tolist() == [0, 1, 2, 3]
    neg = np.array([[nnan, -np.inf]], np.float32)
    assert O.findmax_f32(neg, 1, 2, 1, 2, 1).tolist() == [1]


# ------------------------------------------------------------------ viewshed
def _window(O, bm, R, p, W):
    return O.bitmap_to_window(bm, R, p % W)


def _disc_grid_mask(R, p, H, W):
    cx, cy = p % W, p // W
    m = np.zeros((2 * R + 1, 2 * R + 1), bool)
    for j in range(2 * R + 1):
        for i in range(2 * R + 1):
            dx, dy = i - R, j - R
            x, y = cx + dx, cy + dy
            m[j, i] = dx * dx + dy * dy <= R * R and 0 <= x < W and 0 <= y < H
    return m


def test_viewshed_golden_5x5(O):
    rows = _read_golden("viewshed_5x5_R2.txt")
    z = np.zeros((5, 5), np.int16)
    z[2, 3] = 5
    i = 0
    while i < len(rows):
        ht, hr = rows[i]
        want = np.array(rows[i + 1:i + 6], bool)
        bm, area = O.viewshed(z, 2, ht, hr, np.array([12]))
        got = _window(O, bm[0], 2, 12, 5)
        assert (got == want).all(), (ht, hr, got.astype(int))
        assert area[0] == want.sum()
        i += 6


@pytest.mark.parametrize("R", [1, 2, 3, 7, 12])
def test_viewshed_flat_is_disc(O, R):
    H, W = 29, 37
    z = np.full((H, W), 123, np.int16)
    cand = np.array([14 * W + 18, 0, W - 1, (H - 1) * W, H * W - 1, 3 * W + 30, 20 * W + 2], np.int64)
    bm, area = O.viewshed(z, R, 10, 10, cand)
    for c, p in enumerate(cand):
        m = _disc_grid_mask(R, int(p), H, W)
        assert (_window(O, bm[c], R, int(p), W) == m).all(), (R, p)
        assert area[c] == m.sum()


def test_viewshed_flat_bits_outside_window_zero(O):
    R, H, W = 9, 30, 70
    z = np.zeros((H, W), np.int16)
    for p in [15 * W + 33, 15 * W + 9, 15 * W + 40]:
        bm, area = O.viewshed(z, R, 1, 1, np.array([p]))
        total = sum(bin(int(w)).count("1") for w in bm[0].ravel())
        assert total == area[0] == _disc_grid_mask(R, p, H, W).sum()


@pytest.mark.parametrize("c", [1, 4, 10, 18])
def test_viewshed_cone_apex_sees_all(O, c):
    # apex of z = top - round(c*dist): visible everywhere once hr >= c/2 + 1
    R = 14
    N = 2 * R + 5
    z = T.cone(N, N, N // 2, N // 2, 3000, c).numpy()
    p = (N // 2) * N + N // 2
    hr = 10
    assert hr >= c / 2 + 1
    bm, area = O.viewshed(z, R, 10, hr, np.array([p]))
    assert area[0] == O.disc_count(R)


def test_viewshed_spike_wedge(O):
    # A very tall spike on flat ground hides every cell deep inside its
    # angular wedge (half-width 0.5 post at the spike) and nothing outside
    # the doubled wedge.
    R, N = 20, 45
    o = N // 2
    z = np.zeros((N, N), np.int16)
    d = 5
    z[o, o + d] = 30000
    p = o * N + o
    bm, _ = O.viewshed(z, R, 10, 10, np.array([p]))
    win = _window(O, bm[0], R, p, N)
    for j in range(2 * R + 1):
        for i in range(2 * R + 1):
            dx, dy = i - R, j - R
            if dx * dx + dy * dy > R * R or dx <= d:
                continue
            # lateral offset of the cell's ray at the spike column
            lat = abs(dy) * d / dx
            if lat < 0.5 * 0.9 and dx > d + 1:
                assert not win[j, i], (dx, dy)
            if lat > 1.0 + 1e-9:
                assert win[j, i], (dx, dy)


@pytest.mark.parametrize("R", [11, 12, 16])
def test_viewshed_dihedral_symmetry(O, R):
    # even R makes half-way roundings occur; rounding them away from zero is
    # what keeps the sweep symmetric under every mirror
    z = T.spectral_fbm(41, 41, 0.8, 11, 0, 200).numpy()
    N = 41
    p = 20 * N + 20
    base = _window(O, O.viewshed(z, R, 5, 5, np.array([p]))[0][0], R, p, N)
    # transpose
    zt = np.ascontiguousarray(z.T)
    wt = _window(O, O.viewshed(zt, R, 5, 5, np.array([p]))[0][0], R, p, N)
    assert (wt == base.T).all()
    # mirror in x
    zm = np.ascontiguousarray(z[:, ::-1])
    wm = _window(O, O.viewshed(zm, R, 5, 5, np.array([p]))[0][0], R, p, N)
    assert (wm == base[:, ::-1]).all()
    # mirror in y
    zy = np.ascontiguousarray(z[::-1, :])
    wy = _window(O, O.viewshed(zy, R, 5, 5, np.array([p]))[0][0], R, p, N)
    assert (wy == base[::-1, :]).all()


def test_viewshed_contains_los_on_exact_ray_posts(O):
    # every post lying exactly on some ray (f = 0 at that step) that the LOS
    # definition calls visible is set in the bitmap
    R = 10
    rng = np.random.default_rng(4)
    z = rng.integers(0, 60, (31, 33)).astype(np.int16)
    H, W = z.shape
    for p in [15 * W + 16, 2 * W + 3, 28 * W + 30]:
        win = _window(O, O.viewshed(z, R, 8, 3, np.array([p]))[0][0], R, p, W)
        cx, cy = p % W, p // W
        for ex, ey in [(e1, e2) for e1 in range(-R, R + 1) for e2 in range(-R, R + 1)
                       if max(abs(e1), abs(e2)) == R]:
            xm = abs(ex) >= abs(ey)
            dmin = ey if xm else ex
            smaj = (1 if (ex if xm else ey) > 0 else -1)
            for k in range(1, R + 1):
                if (k * dmin) % R:
                    continue
                m = k * dmin // R
                dx, dy = (smaj * k, m) if xm else (m, smaj * k)
                if dx * dx + dy * dy > R * R or not (0 <= cx + dx < W and 0 <= cy + dy < H):
                    break
                if O.los(z, cx, cy, cx + dx, cy + dy, 8, 3):
                    assert win[R + dy, R + dx], (p, dx, dy)


def test_viewshed_brute_force_agreement(O):
    # the ray sweep approximates the per-cell definition; report and bound it
    R = 15
    z = T.spectral_fbm(64, 64, 0.8, 21, 0, 300).numpy()
    agree = tot = 0
    for p in [32 * 64 + 32, 10 * 64 + 50, 50 * 64 + 12]:
        a = _window(O, O.viewshed(z, R, 10, 10, np.array([p]))[0][0], R, p, 64)
        b = _window(O, O.viewshed_brute(z, R, 10, 10, p), R, p, 64)
        m = _disc_grid_mask(R, p, 64, 64)
        agree += (a == b)[m].sum()
        tot += m.sum()
    assert agree / tot > 0.9


def test_viewshed_threads_agree(O):
    z = T.spectral_fbm(50, 60, 0.8, 8, 0, 500).numpy()
    cand = np.arange(0, 3000, 97, dtype=np.int64)
    a = O.viewshed(z, 9, 10, 10, cand)
    b = O.viewshed(z, 9, 10, 10, cand, threads=4)
    assert (a[0] == b[0]).all() and (a[1] == b[1]).all()


# ------------------------------------------------------------------ site
def _site_inputs(O, seed=1, H=60, W=70, R=8, ncand=40, zr=200):
    z = T.spectral_fbm(H, W, 0.8, seed, 0, zr).numpy()
    rng = np.random.default_rng(seed)
    cand = np.sort(rng.choice(H * W, ncand, replace=False)).astype(np.int64)
    rng.shuffle(cand)
    bm, area = O.viewshed(z, R, 10, 10, cand)
    return z, cand, bm, area


def test_site_lazy_equals_plain(O):
    for seed in range(4):
        z, cand, bm, area = _site_inputs(O, seed)
        H, W = z.shape
        a = O.site(bm, cand, H, W, 8, 30, lazy=True)
        b = O.site(bm, cand, H, W, 8, 30, lazy=False)
        assert (a[0] == b[0]).all() and (a[1] == b[1]).all() and (a[2] == b[2]).all()


def test_site_invariants(O):
    z, cand, bm, area = _site_inputs(O, 7)
    H, W = z.shape
    chosen, gains, C = O.site(bm, cand, H, W, 8, 40)
    assert (np.diff(gains) <= 0).all()                     # greedy gains never grow
    assert gains.sum() == O.cum_popcount(C, H, W)          # gains add up to the coverage
    assert len(set(chosen.tolist())) == len(chosen)
    # first pick is the largest viewshed, ties to the lowest post index
    best = max(range(len(cand)), key=lambda c: (area[c], -cand[c]))
    assert chosen[0] == cand[best]
    # coverage after t observers is monotone and equals the OR of their bitmaps
    idx = {int(p): c for c, p in enumerate(cand)}
    prev = 0
    for t in range(1, len(chosen) + 1):
        sel = [idx[int(p)] for p in chosen[:t]]
        cov = O.cum_popcount(O.cum_rebuild(bm[sel], cand[sel], H, W, 8), H, W)
        assert cov == gains[:t].sum() and cov >= prev
        prev = cov


def test_site_stops_when_nothing_left(O):
    z, cand, bm, area = _site_inputs(O, 3, ncand=6)
    H, W = z.shape
    chosen, gains, C = O.site(bm, cand, H, W, 8, 100)
    assert len(chosen) <= 6 and (gains > 0).all()


def test_site_coverage_target(O):
    z, cand, bm, area = _site_inputs(O, 2, ncand=60)
    H, W = z.shape
    full = O.site(bm, cand, H, W, 8, 60)
    cov = np.cumsum(full[1])
    target = 0.5 * cov[-1] / (H * W)
    need = O.coverage_need(target, H, W)
    chosen, gains, C = O.site(bm, cand, H, W, 8, 60, target=target)
    t = int(np.searchsorted(cov, need) + 1)               # first t with coverage >= need
    assert len(chosen) == t and (chosen == full[0][:t]).all()


def test_site_resume_bit_identical(O):
    z, cand, bm, area = _site_inputs(O, 9)
    H, W = z.shape
    full = O.site(bm, cand, H, W, 8, 25)
    first = O.site(bm, cand, H, W, 8, 10)
    rest = O.site(bm, cand, H, W, 8, 15, cum=first[2])
    assert (np.concatenate([first[0], rest[0]]) == full[0]).all()
    assert (np.concatenate([first[1], rest[1]]) == full[1]).all()
    assert (rest[2] == full[2]).all()


def test_site_greedy_bound_vs_optimum(O):
    # sanity: greedy reaches >= (1 - 1/e) of the best k-subset on a tiny case
    z, cand, bm, area = _site_inputs(O, 4, H=30, W=30, R=6, ncand=9)
    H, W = z.shape
    k = 3
    chosen, gains, C = O.site(bm, cand, H, W, 6, k)
    best = 0
    for sub in itertools.combinations(range(len(cand)), k):
        s = list(sub)
        best = max(best, O.cum_popcount(O.cum_rebuild(bm[s], cand[s], H, W, 6), H, W))
    assert gains.sum() >= (1 - 1 / math.e) * best


# ------------------------------------------------------------------ exact visibility index
def _disc_rows_in_grid(R, x, y, H, W):
    """|disc(R) around (x, y) inside the grid| by rows: each row dy holds the
    columns x - h .. x + h, h = isqrt(R^2 - dy^2), clipped to the grid."""
    n = 0
    for dy in range(-R, R + 1):
        if 0 <= y + dy < H:
            h = math.isqrt(R * R - dy * dy)
            n += max(0, min(W - 1, x + h) - max(0, x - h) + 1)
    return n


def test_exact_vix_flat_is_one(O):
    # flat terrain: every receiver of the ROI inside the grid is visible (for
    # these radii every ray that leaves the grid has reached its last
    # in-grid cell: the viewshed is disc x grid, as pinned above); and a
    # window inside the grid at any R
    z = np.full((37, 45), 120, np.int16)
    H, W = z.shape
    posts = np.array([0, W - 1, (H - 1) * W, H * W - 1, 18 * W + 22, 3 * W + 40], np.int64)
    for R in (2, 7, 12):
        assert (O.exact_vix(z, R, 10, 10, posts) == 1.0).all()
    z = np.full((90, 95), -7, np.int16)
    assert (O.exact_vix(z, 40, 10, 10, np.array([45 * 95 + 47], np.int64)) == 1.0).all()


@pytest.mark.parametrize("R", [2, 5, 13, 40])
def test_exact_vix_walled_observer(O, R):
    """An observer walled in by its eight neighbours (1000 above a flat floor)
    sees itself and the walls only: every ray's first step is visible, the
    interpolated wall then hides every later step.  Visibility index = the
    in-grid cells of its 3 x 3 block over the ROI's receivers in the grid."""
    H, W = 31, 26
    for (x, y) in [(12, 15), (0, 0), (25, 30), (0, 14), (11, 0), (25, 7)]:
        z = np.zeros((H, W), np.int16)
        seen = 0
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if 0 <= x + dx < W and 0 <= y + dy < H:
                    seen += 1
                    if dx or dy:
                        z[y + dy, x + dx] = 1000
        got = O.exact_vix(z, R, 10, 10, np.array([y * W + x], np.int64))[0]
        want = np.float32(seen / _disc_rows_in_grid(R, x, y, H, W))
        assert got == want, (x, y, got, want)


def test_exact_vix_outside_grid(O):
    z = np.zeros((10, 10), np.int16)
    assert O.exact_vix(z, 3, 10, 10, np.array([-1, 100, 5], np.int64)).tolist() == [-1.0, -1.0, 1.0]
