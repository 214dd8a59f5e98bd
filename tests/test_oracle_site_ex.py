"""Pins of the oracle's constrained site step (intervisible transmitters,
weighted receivers; Sec. "Prior art" names both extensions): reductions to
the pinned plain greedy, symmetry and blocking of the intervisibility test,
a hand-built terrain where a wall decides the second transmitter, and
weighted gains recounted cell by cell.  CPU only."""
import numpy as np
import pytest

from synth import terrain as T


@pytest.fixture(scope="module")
def case(O):
    H, W, R = 90, 110, 14
    z = T.spectral_fbm(H, W, 0.8, 21, 0, 600).numpy()
    rng = np.random.default_rng(4)
    cand = rng.choice(H * W, 120, replace=False).astype(np.int64)
    bm, _ = O.viewshed(z, R, 10, 10, cand)
    return z, H, W, R, cand, bm


def test_site_ex_without_options_is_plain_greedy(O, case):
    z, H, W, R, cand, bm = case
    for target in (0.0, 0.4):
        ch, gn, C = O.site(bm, cand, H, W, R, 60, target, lazy=False)
        ch2, gn2, C2 = O.site_ex(bm, cand, H, W, R, 60, target)
        assert ch.tolist() == ch2.tolist() and gn.tolist() == gn2.tolist() and (C == C2).all()


def test_unit_weights_are_the_unweighted_greedy(O, case):
    z, H, W, R, cand, bm = case
    ch, gn, C = O.site_ex(bm, cand, H, W, R, 50)
    ch2, gn2, C2 = O.site_ex(bm, cand, H, W, R, 50, weight=np.ones((H, W), np.uint8))
    assert ch.tolist() == ch2.tolist() and gn.tolist() == gn2.tolist() and (C == C2).all()


def test_intervisibility_symmetric_and_in_range(O, case):
    z, H, W, R, cand, bm = case
    rng = np.random.default_rng(8)
    for _ in range(300):
        a, b = rng.choice(cand, 2)
        v = O.intervisible(z, R, 10, a, b)
        assert v == O.intervisible(z, R, 10, b, a)
        ax, ay, bx, by = a % W, a // W, b % W, b // W
        if (ax - bx) ** 2 + (ay - by) ** 2 > R * R:
            assert not v
    flat = np.full((40, 40), 7, np.int16)
    assert O.intervisible(flat, 10, 0, 5 * 40 + 5, 11 * 40 + 13)        # distance 10
    assert not O.intervisible(flat, 10, 0, 5 * 40 + 5, 12 * 40 + 13)    # distance > 10


def _wall_case(O):
    """Flat ground with a tall wall at column 20: transmitters on the two
    sides cannot see each other; a candidate on the right covers more of
    the right half than anything on the left covers anew."""
    H, W, R = 9, 42, 40
    z = np.zeros((H, W), np.int16)
    z[:, 20] = 1000
    A, B, C = 4 * W + 5, 4 * W + 35, 4 * W + 12
    cand = np.array([A, B, C], np.int64)
    bm, area = O.viewshed(z, R, 10, 0, cand)
    return z, H, W, R, cand, bm, area


def test_wall_decides_the_second_transmitter(O):
    z, H, W, R, cand, bm, area = _wall_case(O)
    A, B, C = cand
    assert not O.intervisible(z, R, 10, A, B) and O.intervisible(z, R, 10, A, C)
    assert not O.intervisible(z, R, 10, B, C)
    # B sees the whole right side (9 rows x 21 columns + its wall face); A and
    # C see the left side, the wall column and nothing behind it
    assert area.tolist() == [189, 198, 189]
    # unconstrained: B, then the left side through A (lower post than C)
    ch, gn, _ = O.site_ex(bm, cand, H, W, R, 3)
    assert ch.tolist() == [B, A] and gn.tolist() == [198, 180]
    # constrained: nothing behind the wall qualifies after B
    chc, gnc, _ = O.site_ex(bm, cand, H, W, R, 3, z=z, ht=10)
    assert chc.tolist() == [B] and gnc.tolist() == [198]


def test_weighted_gains_recounted(O, case):
    z, H, W, R, cand, bm = case
    rng = np.random.default_rng(12)
    wt = rng.integers(0, 256, (H, W)).astype(np.uint8)
    wt[:, : W // 2] = 0                                   # the left half counts for nothing
    ch, gn, C = O.site_ex(bm, cand, H, W, R, 30, weight=wt)
    covered = np.zeros((H, W), bool)
    idx = {int(p): i for i, p in enumerate(cand)}
    for p, g in zip(ch.tolist(), gn.tolist()):
        i = idx[p]
        win = O.bitmap_to_window(bm[i], R, p % W)
        cx, cy = p % W, p // W
        vis = np.zeros((H, W), bool)
        for r in range(2 * R + 1):
            y = cy - R + r
            if 0 <= y < H:
                for j in range(2 * R + 1):
                    x = cx - R + j
                    if 0 <= x < W and win[r, j]:
                        vis[y, x] = True
        new = vis & ~covered
        assert g == int(wt[new].astype(np.int64).sum())
        covered |= vis
        assert p % W >= W // 2 - R                         # nothing to gain far in the left half
    # weighted coverage stop: target of the total weight
    tot = int(wt.astype(np.int64).sum())
    ch2, gn2, _ = O.site_ex(bm, cand, H, W, R, 1000, target=0.5, weight=wt)
    assert sum(gn2.tolist()[:-1]) < np.ceil(0.5 * tot) <= sum(gn2.tolist()) or len(gn2) == 0 or \
        sum(gn2.tolist()) < np.ceil(0.5 * tot)
