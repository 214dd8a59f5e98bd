/*
 * vshed_oracle.c -- plain, slow, obviously-correct CPU oracle for the
 * observer-siting hot path of Franklin, Magalhaes & Li, "Siting thousands of
 * radio transmitter towers on terrains with billions of points"
 * (arXiv 2006.16783).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links or calls this
 * file; only the tests, the smoke check and the benchmark's CPU-baseline leg
 * do.  It shares no code, header or table with the CUDA library.
 *
 * Every quantity is an integer: elevations are int16 posts one unit apart,
 * heights are integers, interpolated heights are kept as numerators over the
 * common denominator D, and slopes are compared by 64-bit cross
 * multiplication.  The paper leaves rounding and tie rules open; the readings
 * taken here are listed next to each function.
 *
 * Layouts (shared with the CUDA library only by documentation):
 *   terrain    z[y*pitch + x], int16, 0 <= x < W, 0 <= y < H
 *   post index p = y*W + x
 *   viewshed   uint32 bm[(2R+1)][P_R], P_R = floor(2R/32) + 2; row r is
 *              global row cy-R+r, word w covers global columns
 *              32*(floor((cx-R)/32)+w) .. +31, bit b = column 32*gw+b.
 *   cumulative uint32 cum[H][ceil(W/32)], same bit convention.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

/* ------------------------------------------------------------------ */
/* small integer helpers                                               */
/* ------------------------------------------------------------------ */

static int64_t floordiv64(int64_t a, int64_t b) /* b > 0 */
{
    int64_t q = a / b;
    if ((a % b) != 0 && (a < 0)) q -= 1;
    return q;
}

static int64_t iabs64(int64_t a) { return a < 0 ? -a : a; }

static int in_grid(int H, int W, int64_t x, int64_t y)
{
    return x >= 0 && x < W && y >= 0 && y < H;
}

static int popc32(uint32_t v)
{
    int c = 0;
    while (v) { v &= v - 1; c++; }
    return c;
}

/* ------------------------------------------------------------------ */
/* Disc of radius R and its offset table (Vix stage, Sec. "The multiple */
/* transmitter siting process": receivers drawn uniformly within a      */
/* circle of radius ROI; realised as uniform over lattice points).      */
/* ------------------------------------------------------------------ */

/* number of lattice points (dx,dy) with dx^2+dy^2 <= R^2 */
int64_t or_disc_count(int32_t R)
{
    int64_t n = 0;
    for (int64_t dy = -R; dy <= R; dy++)
        for (int64_t dx = -R; dx <= R; dx++)
            if (dx * dx + dy * dy <= (int64_t)R * R) n++;
    return n;
}

/* Offset table OFF_R = disc(R) minus the origin, ordered by dy ascending,
 * then dx ascending.  Writes N_R entries into dx[], dy[] (may be NULL to only
 * count) and returns N_R. */
int64_t or_offsets(int32_t R, int32_t *dx, int32_t *dy)
{
    int64_t n = 0;
    for (int64_t y = -R; y <= R; y++)
        for (int64_t x = -R; x <= R; x++) {
            if (x * x + y * y > (int64_t)R * R) continue;
            if (x == 0 && y == 0) continue;
            if (dx) dx[n] = (int32_t)x;
            if (dy) dy[n] = (int32_t)y;
            n++;
        }
    return n;
}

/* SplitMix64 output function (Steele, Lea & Flood 2014): the mix applied to a
 * state value that has already been advanced by the golden-ratio increment. */
uint64_t or_splitmix64_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* The i-th (0-based) output of a SplitMix64 generator seeded with seed. */
uint64_t or_splitmix64_nth(uint64_t seed, uint64_t i)
{
    uint64_t state = seed + 0x9E3779B97F4A7C15ULL * (i + 1);
    return or_splitmix64_mix(state);
}

/* ------------------------------------------------------------------ */
/* Line of sight (Sec. "Definitions": LOS; Sec. "Terrain visibility":  */
/* linear interpolation between adjacent posts).                        */
/*                                                                      */
/* Eye E = z[O] + ht, target height z[T] + hr.  D = max(|dx|,|dy|);     */
/* the major axis is x when |dx| >= |dy|.  For j = 1..D-1 the LOS      */
/* crosses the line major = j at minor = j*dmin/D, between posts y0 and */
/* y0+1 with y0 = floor(j*dmin/D) and weight f/D, f = j*dmin - y0*D.   */
/* The terrain there is Zn_j/D with Zn_j = z[p0]*(D-f) + z[p1]*f.       */
/* T is visible iff its slope is >= every crossing's slope:            */
/*     (z[T] + hr - E) * D * j  >=  (Zn_j - E*D) * D     for all j     */
/* (a grazing line does not intersect the terrain, so ties are          */
/* visible).  A target outside the grid is reported not visible.        */
/* ------------------------------------------------------------------ */
int or_los(const int16_t *z, int32_t H, int32_t W, int64_t pitch,
           int32_t ox, int32_t oy, int32_t tx, int32_t ty,
           int32_t ht, int32_t hr)
{
    if (!in_grid(H, W, ox, oy)) return 0;
    if (!in_grid(H, W, tx, ty)) return 0;
    int64_t dx = (int64_t)tx - ox, dy = (int64_t)ty - oy;
    int64_t D = iabs64(dx) > iabs64(dy) ? iabs64(dx) : iabs64(dy);
    if (D == 0) return 1;
    int xmajor = iabs64(dx) >= iabs64(dy);
    int64_t smaj = xmajor ? (dx > 0 ? 1 : -1) : (dy > 0 ? 1 : -1);
    int64_t dmin = xmajor ? dy : dx;
    int64_t E = (int64_t)z[(int64_t)oy * pitch + ox] + ht;
    int64_t tn = ((int64_t)z[(int64_t)ty * pitch + tx] + hr - E) * D;
    for (int64_t j = 1; j <= D - 1; j++) {
        int64_t n = j * dmin;
        int64_t y0 = floordiv64(n, D);
        int64_t f = n - y0 * D;
        int64_t x0, yy0, x1, yy1;
        if (xmajor) {
            x0 = ox + smaj * j; yy0 = oy + y0;
            x1 = x0;            yy1 = yy0 + 1;
        } else {
            yy0 = oy + smaj * j; x0 = ox + y0;
            yy1 = yy0;           x1 = x0 + 1;
        }
        int64_t Zn = (int64_t)z[yy0 * pitch + x0] * (D - f);
        if (f > 0) Zn += (int64_t)z[yy1 * pitch + x1] * f;
        if (tn * j < (Zn - E * D) * D) return 0;
    }
    return 1;
}

/* ------------------------------------------------------------------ */
/* Vix stage (Sec. "The multiple transmitter siting process", Vix):     */
/* for every post, S receivers drawn uniformly in the ROI circle, each  */
/* LOS-tested; the output is the count of visible ones (0..S).          */
/* Sample s of post p uses the (p*S+s)-th SplitMix64 output u of seed;  */
/* the offset index is ((u>>32) * N_R) >> 32 into OFF_R.                */
/* ------------------------------------------------------------------ */
typedef struct {
    const int16_t *z; int32_t H, W; int64_t pitch;
    int32_t R, ht, hr, S; uint64_t seed;
    const int32_t *odx, *ody; int64_t NR;
    uint8_t *out; int64_t p_begin, p_end;
} vix_job;

static void vix_range(const vix_job *J)
{
    for (int64_t p = J->p_begin; p < J->p_end; p++) {
        int32_t x = (int32_t)(p % J->W), y = (int32_t)(p / J->W);
        int cnt = 0;
        for (int32_t s = 0; s < J->S; s++) {
            uint64_t u = or_splitmix64_nth(J->seed, (uint64_t)p * (uint64_t)J->S + (uint64_t)s);
            uint64_t idx = ((u >> 32) * (uint64_t)J->NR) >> 32;
            int32_t tx = x + J->odx[idx], ty = y + J->ody[idx];
            cnt += or_los(J->z, J->H, J->W, J->pitch, x, y, tx, ty, J->ht, J->hr);
        }
        J->out[p] = (uint8_t)cnt;
    }
}

static void *vix_thread(void *a) { vix_range((const vix_job *)a); return NULL; }

/* out[H*W]; threads >= 1 splits the posts into contiguous ranges (the
 * result does not depend on the split). Returns 0, or -1 on bad arguments. */
int or_vix(const int16_t *z, int32_t H, int32_t W, int64_t pitch,
           int32_t R, int32_t ht, int32_t hr, int32_t S, uint64_t seed,
           uint8_t *out, int32_t threads)
{
    if (H < 0 || W < 0 || R < 1 || S < 0 || S > 255 || pitch < W) return -1;
    int64_t NR = or_offsets(R, NULL, NULL);
    int32_t *odx = (int32_t *)malloc(sizeof(int32_t) * (size_t)NR);
    int32_t *ody = (int32_t *)malloc(sizeof(int32_t) * (size_t)NR);
    or_offsets(R, odx, ody);
    int64_t n = (int64_t)H * W;
    if (threads < 1) threads = 1;
    vix_job *jobs = (vix_job *)calloc((size_t)threads, sizeof(vix_job));
    pthread_t *tid = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    for (int t = 0; t < threads; t++) {
        vix_job J = { z, H, W, pitch, R, ht, hr, S, seed, odx, ody, NR, out,
                      n * t / threads, n * (t + 1) / threads };
        jobs[t] = J;
    }
    for (int t = 1; t < threads; t++) pthread_create(&tid[t], NULL, vix_thread, &jobs[t]);
    vix_range(&jobs[0]);
    for (int t = 1; t < threads; t++) pthread_join(tid[t], NULL);
    free(jobs); free(tid); free(odx); free(ody);
    return 0;
}

/* Vix counts of a list of posts only (same definition as or_vix; for
 * spot checks of grids too large for the full oracle). */
int or_vix_posts(const int16_t *z, int32_t H, int32_t W, int64_t pitch,
                 int32_t R, int32_t ht, int32_t hr, int32_t S, uint64_t seed,
                 const int64_t *posts, int64_t n, uint8_t *out)
{
    if (H < 0 || W < 0 || R < 1 || S < 0 || S > 255 || pitch < W) return -1;
    int64_t NR = or_offsets(R, NULL, NULL);
    int32_t *odx = (int32_t *)malloc(sizeof(int32_t) * (size_t)NR);
    int32_t *ody = (int32_t *)malloc(sizeof(int32_t) * (size_t)NR);
    or_offsets(R, odx, ody);
    for (int64_t i = 0; i < n; i++) {
        int64_t p = posts[i];
        int32_t x = (int32_t)(p % W), y = (int32_t)(p / W);
        int cnt = 0;
        for (int32_t s = 0; s < S; s++) {
            uint64_t u = or_splitmix64_nth(seed, (uint64_t)p * (uint64_t)S + (uint64_t)s);
            uint64_t idx = ((u >> 32) * (uint64_t)NR) >> 32;
            cnt += or_los(z, H, W, pitch, x, y, x + odx[idx], y + ody[idx], ht, hr);
        }
        out[i] = (uint8_t)cnt;
    }
    free(odx); free(ody);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Findmax stage (Sec. "The multiple transmitter siting process",      */
/* Findmax): partition the terrain into b x b blocks (edge blocks may   */
/* be partial) and keep the top k posts of each block by               */
/* (value descending, post index ascending).  Output is ordered by      */
/* block (row-major over blocks), then by rank.                         */
/* ------------------------------------------------------------------ */

/* a total order on float values: larger key == larger value; NaNs with the
 * sign bit clear sort above +inf, negative ones below -inf */
static uint32_t f32_order_key(float v)
{
    uint32_t u; memcpy(&u, &v, 4);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

static int64_t findmax_generic(const uint8_t *v8, const float *vf, int64_t ld,
                               int32_t H, int32_t W, int32_t stride,
                               int32_t b, int32_t k, int64_t *out, int64_t cap)
{
    /* the value grid has Hs x Ws cells; cell (i,j) is post (i*stride, j*stride) */
    int32_t Hs = (H + stride - 1) / stride, Ws = (W + stride - 1) / stride;
    int32_t nby = (H + b - 1) / b, nbx = (W + b - 1) / b;
    int64_t total = 0;
    uint64_t *keys = NULL; int64_t keycap = 0;
    for (int32_t by = 0; by < nby; by++)
        for (int32_t bx = 0; bx < nbx; bx++) {
            int64_t m = 0;
            /* collect every value cell whose post lies inside this block:
             * cells i with by*b <= i*stride < (by+1)*b */
            int64_t i0 = ((int64_t)by * b + stride - 1) / stride;
            int64_t i1 = ((int64_t)(by + 1) * b + stride - 1) / stride;
            int64_t j0 = ((int64_t)bx * b + stride - 1) / stride;
            int64_t j1 = ((int64_t)(bx + 1) * b + stride - 1) / stride;
            if (i1 > Hs) i1 = Hs;
            if (j1 > Ws) j1 = Ws;
            for (int64_t i = i0; i < i1; i++) {
                int64_t y = i * stride;
                for (int64_t j = j0; j < j1; j++) {
                    int64_t x = j * stride;
                    if (m == keycap) {
                        keycap = keycap ? keycap * 2 : 1024;
                        keys = (uint64_t *)realloc(keys, sizeof(uint64_t) * (size_t)keycap);
                    }
                    uint32_t hi = v8 ? (uint32_t)v8[(int64_t)i * ld + j]
                                     : f32_order_key(vf[(int64_t)i * ld + j]);
                    uint32_t p = (uint32_t)(y * W + x);
                    keys[m++] = ((uint64_t)hi << 32) | (uint64_t)(0xFFFFFFFFu - p);
                }
            }
            /* k passes of "take the largest remaining key": plain selection */
            for (int32_t r = 0; r < k && r < m; r++) {
                int64_t best = r;
                for (int64_t q = r + 1; q < m; q++) if (keys[q] > keys[best]) best = q;
                uint64_t t = keys[r]; keys[r] = keys[best]; keys[best] = t;
                if (total < cap) out[total] = (int64_t)(0xFFFFFFFFu - (uint32_t)(keys[r] & 0xFFFFFFFFu));
                total++;
            }
        }
    free(keys);
    return total;
}

/* u8 visibility counts, one per post; returns the number of candidates
 * (which may exceed cap; only the first cap are written). */
int64_t or_findmax(const uint8_t *vix, int32_t H, int32_t W, int32_t b, int32_t k,
                   int64_t *out, int64_t cap)
{
    if (H < 0 || W < 0 || b < 1 || k < 1) return -1;
    return findmax_generic(vix, NULL, W, H, W, 1, b, k, out, cap);
}

/* float scores on a proposal lattice of the given stride: score[i*Ws+j]
 * belongs to post (i*stride, j*stride), Ws = ceil(W/stride). */
int64_t or_findmax_f32(const float *score, int32_t H, int32_t W, int32_t stride,
                       int32_t b, int32_t k, int64_t *out, int64_t cap)
{
    if (H < 0 || W < 0 || b < 1 || k < 1 || stride < 1) return -1;
    int32_t Ws = (W + stride - 1) / stride;
    return findmax_generic(NULL, score, Ws, H, W, stride, b, k, out, cap);
}

/* ------------------------------------------------------------------ */
/* Viewshed stage (Sec. "The multiple transmitter siting process",     */
/* Viewshed): rays from the observer to every cell of the square ring  */
/* max(|dx|,|dy|) = R (8R rays; the paper's "circle" is read as this    */
/* ring, cut at the disc, so that every disc cell is touched), walked  */
/* outward while keeping the highest horizon slope seen so far.        */
/*                                                                      */
/* Ray to ring cell (ex,ey): major axis x when |ex| >= |ey|, D = R.     */
/* At step k = 1..R the minor numerator is n = k*dmin; the cell visited */
/* is C_k = (major k, minor round(n/R)) with ties rounded away from     */
/* zero.  The ray stops when C_k leaves the grid or the disc            */
/* k^2 + rnd^2 > R^2.  C_k is visible on this ray iff there is no       */
/* horizon yet or (z[C_k] + hr - E) * R * k_h >= H_num * k.  Then the   */
/* horizon is offered the interpolated crossing at step k              */
/* (Zn_k - E*R, k), which replaces (H_num, k_h) when steeper; when the   */
/* crossing straddles a post outside the grid (f > 0) the ray stops    */
/* after its test.  A cell's bit is the OR over every ray that visits   */
/* it; the observer's own cell is always visible.                       */
/* ------------------------------------------------------------------ */
int64_t or_bitmap_words(int32_t R)
{
    return (int64_t)(2 * R + 1) * (int64_t)((2 * R) / 32 + 2);
}

static void set_bit(uint32_t *bm, int32_t R, int64_t cx, int64_t cy, int64_t x, int64_t y)
{
    int64_t PR = (2 * R) / 32 + 2;
    int64_t gw0 = floordiv64(cx - R, 32);
    int64_t row = y - (cy - R);
    int64_t w = floordiv64(x, 32) - gw0;
    int64_t bit = x - 32 * floordiv64(x, 32);
    bm[row * PR + w] |= (uint32_t)1u << bit;
}

static void viewshed_one(const int16_t *z, int32_t H, int32_t W, int64_t pitch,
                         int32_t R, int32_t ht, int32_t hr, int64_t p,
                         uint32_t *bm, int32_t *area)
{
    int64_t words = or_bitmap_words(R);
    memset(bm, 0, sizeof(uint32_t) * (size_t)words);
    int64_t ox = p % W, oy = p / W;
    int64_t E = (int64_t)z[oy * pitch + ox] + ht;
    int64_t D = R;
    for (int64_t ey = -R; ey <= R; ey++)
        for (int64_t ex = -R; ex <= R; ex++) {
            if (iabs64(ex) != R && iabs64(ey) != R) continue; /* ring cells only */
            int xmajor = iabs64(ex) >= iabs64(ey);
            int64_t smaj = xmajor ? (ex > 0 ? 1 : -1) : (ey > 0 ? 1 : -1);
            int64_t dmin = xmajor ? ey : ex;
            int have_h = 0; int64_t Hn = 0, Hk = 0;
            for (int64_t k = 1; k <= R; k++) {
                int64_t n = k * dmin;
                int64_t y0 = floordiv64(n, D);
                int64_t f = n - y0 * D;
                int64_t rnd = n >= 0 ? (2 * n + D) / (2 * D) : -((2 * (-n) + D) / (2 * D));
                int64_t cx_, cy_, x0, yy0, x1, yy1;
                if (xmajor) {
                    cx_ = ox + smaj * k; cy_ = oy + rnd;
                    x0 = cx_; yy0 = oy + y0; x1 = x0; yy1 = yy0 + 1;
                } else {
                    cy_ = oy + smaj * k; cx_ = ox + rnd;
                    yy0 = cy_; x0 = ox + y0; yy1 = yy0; x1 = x0 + 1;
                }
                if (!in_grid(H, W, cx_, cy_)) break;
                if (k * k + rnd * rnd > (int64_t)R * R) break;
                int64_t zc = z[cy_ * pitch + cx_];
                int vis = !have_h || (zc + hr - E) * D * Hk >= Hn * k;
                if (vis) set_bit(bm, R, ox, oy, cx_, cy_);
                if (f > 0 && (!in_grid(H, W, x0, yy0) || !in_grid(H, W, x1, yy1))) break;
                int64_t Zn = (int64_t)z[yy0 * pitch + x0] * (D - f);
                if (f > 0) Zn += (int64_t)z[yy1 * pitch + x1] * f;
                int64_t num = Zn - E * D;
                if (!have_h || num * Hk > Hn * k) { Hn = num; Hk = k; have_h = 1; }
            }
        }
    set_bit(bm, R, ox, oy, ox, oy);
    int32_t a = 0;
    for (int64_t w = 0; w < words; w++) a += popc32(bm[w]);
    *area = a;
}

typedef struct {
    const int16_t *z; int32_t H, W; int64_t pitch; int32_t R, ht, hr;
    const int64_t *cand; uint32_t *bm; int32_t *area; int64_t c_begin, c_end;
} vs_job;

static void *vs_thread(void *a)
{
    const vs_job *J = (const vs_job *)a;
    int64_t words = or_bitmap_words(J->R);
    for (int64_t c = J->c_begin; c < J->c_end; c++)
        viewshed_one(J->z, J->H, J->W, J->pitch, J->R, J->ht, J->hr, J->cand[c],
                     J->bm + c * words, J->area + c);
    return NULL;
}

int or_viewshed(const int16_t *z, int32_t H, int32_t W, int64_t pitch,
                int32_t R, int32_t ht, int32_t hr, const int64_t *cand, int64_t n,
                uint32_t *bm, int32_t *area, int32_t threads)
{
    if (H < 1 || W < 1 || R < 1 || pitch < W || n < 0) return -1;
    for (int64_t c = 0; c < n; c++)
        if (cand[c] < 0 || cand[c] >= (int64_t)H * W) return -2;
    if (threads < 1) threads = 1;
    vs_job *jobs = (vs_job *)calloc((size_t)threads, sizeof(vs_job));
    pthread_t *tid = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    for (int t = 0; t < threads; t++) {
        vs_job J = { z, H, W, pitch, R, ht, hr, cand, bm, area,
                     n * t / threads, n * (t + 1) / threads };
        jobs[t] = J;
    }
    for (int t = 1; t < threads; t++) pthread_create(&tid[t], NULL, vs_thread, &jobs[t]);
    vs_thread(&jobs[0]);
    for (int t = 1; t < threads; t++) pthread_join(tid[t], NULL);
    free(jobs); free(tid);
    return 0;
}

/* Brute-force viewshed: every cell of disc(R) inside the grid gets its own
 * LOS test (the Sec. "Definitions" viewshed read literally).  Same layout. */
int or_viewshed_brute(const int16_t *z, int32_t H, int32_t W, int64_t pitch,
                      int32_t R, int32_t ht, int32_t hr, int64_t p, uint32_t *bm)
{
    int64_t words = or_bitmap_words(R);
    memset(bm, 0, sizeof(uint32_t) * (size_t)words);
    int64_t ox = p % W, oy = p / W;
    for (int64_t dy = -R; dy <= R; dy++)
        for (int64_t dx = -R; dx <= R; dx++) {
            if (dx * dx + dy * dy > (int64_t)R * R) continue;
            int64_t x = ox + dx, y = oy + dy;
            if (!in_grid(H, W, x, y)) continue;
            if (or_los(z, H, W, pitch, (int32_t)ox, (int32_t)oy, (int32_t)x, (int32_t)y, ht, hr))
                set_bit(bm, R, ox, oy, x, y);
        }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Exact visibility index (Sec. "Definitions": the visibility index of */
/* a transmitter is the fraction of the receivers within its ROI that  */
/* it sees, i.e. the normalised area of its viewshed).  Numerator: the */
/* area of the post's ray-sweep viewshed (or_viewshed).  Denominator:  */
/* the receivers of the ROI, the lattice points (dx,dy) with           */
/* dx^2+dy^2 <= R^2 whose post lies inside the grid, counted one by    */
/* one.  out[i] = the quotient in double, rounded to float; a post     */
/* outside the grid gives -1.                                          */
/* ------------------------------------------------------------------ */
int or_exact_vix(const int16_t *z, int32_t H, int32_t W, int64_t pitch,
                 int32_t R, int32_t ht, int32_t hr, const int64_t *posts, int64_t n,
                 float *out, int32_t threads)
{
    if (H < 1 || W < 1 || R < 1 || pitch < W || n < 0) return -1;
    int64_t words = or_bitmap_words(R);
    int64_t chunk = 256;
    uint32_t *bm = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(words * chunk));
    int32_t *area = (int32_t *)malloc(sizeof(int32_t) * (size_t)chunk);
    int64_t *valid = (int64_t *)malloc(sizeof(int64_t) * (size_t)chunk);
    for (int64_t i0 = 0; i0 < n; i0 += chunk) {
        int64_t m = n - i0 < chunk ? n - i0 : chunk, nv = 0;
        for (int64_t i = 0; i < m; i++) {
            int64_t p = posts[i0 + i];
            if (p >= 0 && p < (int64_t)H * W) valid[nv++] = p;
        }
        memset(bm, 0, sizeof(uint32_t) * (size_t)(words * chunk));
        or_viewshed(z, H, W, pitch, R, ht, hr, valid, nv, bm, area, threads);
        int64_t v = 0;
        for (int64_t i = 0; i < m; i++) {
            int64_t p = posts[i0 + i];
            if (p < 0 || p >= (int64_t)H * W) { out[i0 + i] = -1.0f; continue; }
            int64_t ox = p % W, oy = p / W, den = 0;
            for (int64_t dy = -R; dy <= R; dy++)
                for (int64_t dx = -R; dx <= R; dx++)
                    if (dx * dx + dy * dy <= (int64_t)R * R && in_grid(H, W, ox + dx, oy + dy)) den++;
            out[i0 + i] = (float)((double)area[v++] / (double)den);
        }
    }
    free(bm); free(area); free(valid);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Site stage (Sec. "The multiple transmitter siting process", Site):  */
/* greedy; each step adds the candidate whose viewshed grows the        */
/* cumulative viewshed C the most: gain_c = popcount(V_c AND NOT C),    */
/* ties to the lowest post index.  Stop when the best gain is 0, when   */
/* n_obs observers are chosen, or when coverage popcount(C) reaches    */
/* need = ceil(target*H*W) (target <= 0 disables).  C |= V_winner.      */
/* ------------------------------------------------------------------ */
static int64_t cum_words_per_row(int32_t W) { return ((int64_t)W + 31) / 32; }

static int64_t gain_of(const uint32_t *V, int64_t p, int32_t H, int32_t W, int32_t R,
                       const uint32_t *cum)
{
    int64_t PR = (2 * R) / 32 + 2, WW = cum_words_per_row(W);
    int64_t cx = p % W, cy = p / W, gw0 = floordiv64(cx - R, 32);
    int64_t g = 0;
    for (int64_t r = 0; r < 2 * R + 1; r++) {
        int64_t y = cy - R + r;
        if (y < 0 || y >= H) continue;
        for (int64_t w = 0; w < PR; w++) {
            int64_t gw = gw0 + w;
            if (gw < 0 || gw >= WW) continue;
            g += popc32(V[r * PR + w] & ~cum[y * WW + gw]);
        }
    }
    return g;
}

static void or_into(const uint32_t *V, int64_t p, int32_t H, int32_t W, int32_t R, uint32_t *cum)
{
    int64_t PR = (2 * R) / 32 + 2, WW = cum_words_per_row(W);
    int64_t cx = p % W, cy = p / W, gw0 = floordiv64(cx - R, 32);
    for (int64_t r = 0; r < 2 * R + 1; r++) {
        int64_t y = cy - R + r;
        if (y < 0 || y >= H) continue;
        for (int64_t w = 0; w < PR; w++) {
            int64_t gw = gw0 + w;
            if (gw < 0 || gw >= WW) continue;
            cum[y * WW + gw] |= V[r * PR + w];
        }
    }
}

int64_t or_coverage_need(double target, int32_t H, int32_t W)
{
    if (!(target > 0.0)) return -1;
    double need = target * (double)H * (double)W;
    int64_t n = (int64_t)need;
    if ((double)n < need) n += 1;
    return n;
}

static int64_t cum_popcount(const uint32_t *cum, int32_t H, int32_t W)
{
    int64_t WW = cum_words_per_row(W), c = 0;
    for (int64_t i = 0; i < (int64_t)H * WW; i++) c += popc32(cum[i]);
    return c;
}

/* Plain greedy: every step re-evaluates every candidate.  cum is in/out and
 * holds the starting cumulative viewshed (all zero for a fresh run).
 * Returns the number of observers chosen. */
int32_t or_site_plain(const uint32_t *bm, const int64_t *cand, int64_t n,
                      int32_t H, int32_t W, int32_t R, int32_t n_obs, double target,
                      int64_t *chosen, int64_t *gains, uint32_t *cum)
{
    int64_t words = or_bitmap_words(R), need = or_coverage_need(target, H, W);
    int64_t covered = cum_popcount(cum, H, W);
    int32_t t = 0;
    for (; t < n_obs; t++) {
        if (need >= 0 && covered >= need) break;
        int64_t best = -1, bestg = -1;
        for (int64_t c = 0; c < n; c++) {
            int64_t g = gain_of(bm + c * words, cand[c], H, W, R, cum);
            if (g > bestg || (g == bestg && cand[c] < cand[best])) { best = c; bestg = g; }
        }
        if (best < 0 || bestg <= 0) break;
        chosen[t] = cand[best]; gains[t] = bestg;
        or_into(bm + best * words, cand[best], H, W, R, cum);
        covered += bestg;
    }
    return t;
}

/* Lazy greedy (the paper's optimisation: a candidate's gain can only shrink
 * as C grows, so an old gain is an upper bound).  A max-heap is keyed by
 * (bound, -post index); the top is re-evaluated and accepted when its fresh
 * key is still >= the next key, which makes it the exact lexicographic
 * argmax, so the result equals or_site_plain bit for bit. */
typedef struct { int64_t bound; int64_t p; int64_t c; } heap_ent;

static int ent_gt(const heap_ent *a, const heap_ent *b)
{
    if (a->bound != b->bound) return a->bound > b->bound;
    if (a->p != b->p) return a->p < b->p;
    return a->c < b->c;
}

static void heap_down(heap_ent *h, int64_t m, int64_t i)
{
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, t = i;
        if (l < m && ent_gt(&h[l], &h[t])) t = l;
        if (r < m && ent_gt(&h[r], &h[t])) t = r;
        if (t == i) return;
        heap_ent tmp = h[i]; h[i] = h[t]; h[t] = tmp; i = t;
    }
}

int32_t or_site_lazy(const uint32_t *bm, const int64_t *cand, int64_t n,
                     int32_t H, int32_t W, int32_t R, int32_t n_obs, double target,
                     int64_t *chosen, int64_t *gains, uint32_t *cum)
{
    int64_t words = or_bitmap_words(R), need = or_coverage_need(target, H, W);
    int64_t covered = cum_popcount(cum, H, W);
    heap_ent *h = (heap_ent *)malloc(sizeof(heap_ent) * (size_t)(n > 0 ? n : 1));
    int64_t m = n;
    for (int64_t c = 0; c < n; c++) {
        h[c].bound = gain_of(bm + c * words, cand[c], H, W, R, cum);
        h[c].p = cand[c]; h[c].c = c;
    }
    for (int64_t i = m / 2 - 1; i >= 0; i--) heap_down(h, m, i);
    int32_t t = 0;
    while (t < n_obs && m > 0) {
        if (need >= 0 && covered >= need) break;
        heap_ent top = h[0];
        top.bound = gain_of(bm + top.c * words, top.p, H, W, R, cum);
        /* compare the fresh key with the best remaining bound */
        h[0] = h[m - 1]; m--;
        heap_down(h, m, 0);
        if (m == 0 || !ent_gt(&h[0], &top)) {
            if (top.bound <= 0) break;
            chosen[t] = top.p; gains[t] = top.bound; t++;
            or_into(bm + top.c * words, top.p, H, W, R, cum);
            covered += top.bound;
            /* the chosen candidate now has gain 0; it stays out of the heap */
        } else {
            /* stale: re-insert with its fresh bound */
            int64_t i = m++;
            h[i] = top;
            while (i > 0) {
                int64_t par = (i - 1) / 2;
                if (!ent_gt(&h[i], &h[par])) break;
                heap_ent tmp = h[i]; h[i] = h[par]; h[par] = tmp; i = par;
            }
        }
    }
    free(h);
    return t;
}

int64_t or_cum_popcount(const uint32_t *cum, int32_t H, int32_t W)
{
    return cum_popcount(cum, H, W);
}

/* C |= V for a list of already-chosen candidates: rebuilds a cumulative
 * viewshed from a saved observer list (checkpoint / resume). */
void or_cum_rebuild(const uint32_t *bm, const int64_t *cand, int64_t n, int32_t H, int32_t W,
                    int32_t R, uint32_t *cum)
{
    int64_t words = or_bitmap_words(R);
    for (int64_t c = 0; c < n; c++) or_into(bm + c * words, cand[c], H, W, R, cum);
}

/* ------------------------------------------------------------------ */
/* Site with the constraints of Sec. "Prior art" (receivers of a given */
/* quality; intervisibility, where transmitters must be visible from   */
/* other transmitters).  Readings taken here:                          */
/*  - intervisible(a, b): the two posts are within the ROI             */
/*    (dx^2 + dy^2 <= R^2) and the line between the two antenna tops,  */
/*    both at z + ht, clears the terrain (the or_los test with the     */
/*    receiver height set to ht; the test is symmetric in a and b);    */
/*  - with the constraint, the first transmitter of the call is free   */
/*    and every later one must be intervisible with one already chosen */
/*    in this call;                                                    */
/*  - weighted receivers: post (x, y) weighs weight[y*W + x] (uint8),  */
/*    the gain of a candidate is the weight of the posts it newly      */
/*    covers, the coverage stop compares the covered weight with       */
/*    ceil(target * total weight).                                    */
/* Plain greedy: every step re-evaluates every eligible candidate;     */
/* ties as in or_site_plain (largest gain, lowest post, lowest index). */
/* z == NULL: no intervisibility constraint; weight == NULL: unit      */
/* weights (then this is or_site_plain).                               */
/* ------------------------------------------------------------------ */
static int64_t wgain_of(const uint32_t *V, int64_t p, int32_t H, int32_t W, int32_t R,
                        const uint32_t *cum, const uint8_t *weight)
{
    int64_t PR = (2 * R) / 32 + 2, WW = cum_words_per_row(W);
    int64_t cx = p % W, cy = p / W, gw0 = floordiv64(cx - R, 32);
    int64_t g = 0;
    for (int64_t r = 0; r < 2 * R + 1; r++) {
        int64_t y = cy - R + r;
        if (y < 0 || y >= H) continue;
        for (int64_t w = 0; w < PR; w++) {
            int64_t gw = gw0 + w;
            if (gw < 0 || gw >= WW) continue;
            uint32_t d = V[r * PR + w] & ~cum[y * WW + gw];
            for (int b = 0; b < 32; b++)
                if ((d >> b) & 1u) g += weight ? weight[y * W + 32 * gw + b] : 1;
        }
    }
    return g;
}

static int64_t wcovered(const uint32_t *cum, int32_t H, int32_t W, const uint8_t *weight)
{
    int64_t WW = cum_words_per_row(W), c = 0;
    for (int64_t y = 0; y < H; y++)
        for (int64_t gw = 0; gw < WW; gw++)
            for (int b = 0; b < 32; b++)
                if ((cum[y * WW + gw] >> b) & 1u) c += weight ? weight[y * W + 32 * gw + b] : 1;
    return c;
}

int or_intervisible(const int16_t *z, int32_t H, int32_t W, int64_t pitch, int32_t R, int32_t ht,
                    int64_t pa, int64_t pb)
{
    if (pa < 0 || pb < 0 || pa >= (int64_t)H * W || pb >= (int64_t)H * W) return 0;
    int64_t ax = pa % W, ay = pa / W, bx = pb % W, by = pb / W;
    int64_t dx = bx - ax, dy = by - ay;
    if (dx * dx + dy * dy > (int64_t)R * R) return 0;
    return or_los(z, H, W, pitch, (int32_t)ax, (int32_t)ay, (int32_t)bx, (int32_t)by, ht, ht);
}

int32_t or_site_ex(const uint32_t *bm, const int64_t *cand, int64_t n, int32_t H, int32_t W, int32_t R,
                   int32_t n_obs, double target, const int16_t *z, int64_t pitch, int32_t ht,
                   const uint8_t *weight, int64_t *chosen, int64_t *gains, uint32_t *cum)
{
    int64_t words = or_bitmap_words(R);
    int64_t total = weight ? 0 : (int64_t)H * W;
    if (weight)
        for (int64_t i = 0; i < (int64_t)H * W; i++) total += weight[i];
    int64_t need = -1;
    if (target > 0.0) {
        double nd = target * (double)total;
        need = (int64_t)nd;
        if ((double)need < nd) need += 1;
    }
    int64_t covered = wcovered(cum, H, W, weight);
    uint8_t *elig = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    int32_t t = 0;
    for (; t < n_obs; t++) {
        if (need >= 0 && covered >= need) break;
        int64_t best = -1, bestg = -1;
        for (int64_t c = 0; c < n; c++) {
            if (cand[c] < 0 || cand[c] >= (int64_t)H * W) continue;
            if (z && t > 0 && !elig[c]) continue;
            int64_t g = wgain_of(bm + c * words, cand[c], H, W, R, cum, weight);
            if (g > bestg || (g == bestg && cand[c] < cand[best])) { best = c; bestg = g; }
        }
        if (best < 0 || bestg <= 0) break;
        chosen[t] = cand[best]; gains[t] = bestg;
        or_into(bm + best * words, cand[best], H, W, R, cum);
        covered += bestg;
        if (z)
            for (int64_t c = 0; c < n; c++)
                if (c != best && or_intervisible(z, H, W, pitch, R, ht, cand[best], cand[c])) elig[c] = 1;
    }
    free(elig);
    return t;
}
