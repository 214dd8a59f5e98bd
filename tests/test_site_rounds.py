"""The rule behind the leader cluster's multi-winner rounds, checked on the CPU
against the oracle's one-step-at-a-time greedy (Sec. "The multiple transmitter
siting process", Site).

After a round's refresh every gain is exact.  The round takes candidates in
decreasing key order (gain, then lowest post) and accepts each while its post
lies more than 2R (Chebyshev) from every post accepted earlier in the round.
Such a candidate's window misses the round's earlier windows, so its gain is
unchanged by them, and no other gain can have grown.  So each accepted
candidate is the next sequential argmax with the gain it had at the round's
start.  The accepted windows are disjoint, so each candidate's refresh is the
sum of popcount(V_c AND V_w AND NOT C) over the round's winners w.  The
kernel relies on both facts; the band compaction that overlaps the picks
relies on one more: a winner is never within 2R of another winner of the same
round.  CPU only."""
import numpy as np
import pytest

from synth import terrain as T


def _masks(O, bm, cand, H, W, R):
    """Each candidate's viewshed as a boolean H x W mask."""
    out = []
    for c, p in enumerate(cand):
        cy, cx = divmod(int(p), W)
        win = O.bitmap_to_window(bm[c], R, cx, W)
        m = np.zeros((H, W), bool)
        y0, x0 = cy - R, cx - R
        ya, yb = max(0, y0), min(H, cy + R + 1)
        xa, xb = max(0, x0), min(W, cx + R + 1)
        m[ya:yb, xa:xb] = win[ya - y0:yb - y0, xa - x0:xb - x0]
        out.append(m)
    return out


def _round_greedy(ms, cand, W, R, n_obs, sep):
    """Rounds of several winners each: keys in decreasing order while every
    post is more than ``sep`` from the round's earlier posts.  Returns the
    observers, their gains, the round sizes and whether every refresh equalled
    the sum of the round winners' overlaps with the uncovered cells."""
    cov = np.zeros_like(ms[0])
    taken = set()
    chosen, gains, sizes = [], [], []
    refresh_ok = True
    g = [int(m.sum()) for m in ms]
    while len(chosen) < n_obs:
        order = sorted(range(len(ms)), key=lambda c: (-g[c], int(cand[c])))
        rnd, posts = [], []
        for c in order:
            if c in taken or g[c] == 0 or len(chosen) + len(rnd) >= n_obs:
                break
            cy, cx = divmod(int(cand[c]), W)
            if any(max(abs(cx - wx), abs(cy - wy)) <= sep for wx, wy in posts):
                break
            rnd.append(c)
            posts.append((cx, cy))
        if not rnd:
            break
        old = cov.copy()
        for c in rnd:
            chosen.append(int(cand[c]))
            gains.append(g[c])
            taken.add(c)
            cov |= ms[c]
        # the refresh as the workers compute it, against the exact new gains
        for c, m in enumerate(ms):
            exact = 0 if c in taken else int((m & ~cov).sum())
            if c not in taken:
                lowered = g[c] - sum(int((m & ms[w] & ~old).sum()) for w in rnd)
                refresh_ok &= lowered == exact
            g[c] = exact
        sizes.append(len(rnd))
    return np.array(chosen, np.int64), np.array(gains, np.int64), sizes, refresh_ok


def _case(O, seed, H=100, W=110, R=8, ncand=60):
    z = T.spectral_fbm(H, W, 0.8, seed, 0, 200).numpy()
    rng = np.random.default_rng(seed)
    cand = rng.choice(H * W, ncand, replace=False).astype(np.int64)
    bm, _ = O.viewshed(z, R, 10, 10, cand)
    return cand, bm


@pytest.mark.parametrize("seed", [3, 4, 5, 6])
def test_rounds_reproduce_the_sequential_greedy(O, seed):
    H, W, R, n_obs = 100, 110, 8, 40
    cand, bm = _case(O, seed)
    want_ch, want_gn, _ = O.site(bm, cand, H, W, R, n_obs)
    ch, gn, sizes, refresh_ok = _round_greedy(_masks(O, bm, cand, H, W, R), cand, W, R, n_obs, 2 * R)
    assert ch.tolist() == want_ch.tolist()
    assert gn.tolist() == want_gn.tolist()
    assert refresh_ok
    # not vacuous: rounds of several winners occur
    assert max(sizes) >= 3 and len(sizes) < len(ch)


def test_a_smaller_separation_breaks_the_rule(O):
    """Windows of posts within 2R overlap: accepting them in one round gives
    stale gains, and the sequence leaves the sequential greedy's."""
    H, W, R, n_obs = 100, 110, 8, 40
    differs = False
    for seed in [3, 4, 5, 6]:
        cand, bm = _case(O, seed)
        want_ch, want_gn, _ = O.site(bm, cand, H, W, R, n_obs)
        ch, gn, _, _ = _round_greedy(_masks(O, bm, cand, H, W, R), cand, W, R, n_obs, R)
        differs |= ch.tolist() != want_ch.tolist() or gn.tolist() != want_gn.tolist()
    assert differs
