// viewshed.cu -- Viewshed stage (Sec. "The multiple transmitter siting
// process", Viewshed): one CTA per candidate observer.
//
// The observer's ROI window (int16 posts) is staged into shared memory by TMA
// (cp.async.bulk.tensor, tensor map view [H][pitch/8][8]); the CTA's threads
// then walk the 8R rays to the square ring max(|dx|,|dy|) = R, keeping each
// ray's running horizon (the steepest interpolated crossing so far) as an
// exact rational (numerator over step), and OR visible cells into a
// shared-memory bitmap (the output's layout with an odd row pitch, so that
// rays on rows four apart do not share a bank).  A step reads two posts --
// the two the line passes between, one of which is the cell tested -- at a
// running window address.  When the window does
// not fit in shared memory it is processed in halves (rays by the sign of the
// ring cell's dy) or quadrants (signs of dx and dy); every ray stays inside
// its half / quadrant, so each pass stages only that part.  When not even a
// quadrant fits (R above ~280), k_viewshed_wide walks the rays in bands of
// steps against the terrain in global memory (see there).
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "vs_common.cuh"

namespace vs {

struct VsParams {
    int H, W, R, ht, hr;
    const int64_t *cand;
    int64_t n;
    uint32_t *bm;
    int32_t *area;
    int PR, words;
    int nsplit;               // 1, 2 (halves by sign of ey) or 4 (quadrants)
    int WG;                   // window width in 8-element groups
    int box_rows, nbox;       // TMA boxes per pass
};

// ring cell of ray rho in [0, 8R), walking the ring so that neighbouring rays
// have neighbouring ids
__device__ __forceinline__ void ring_cell(int rho, int R, int &ex, int &ey) {
    int side = rho / (2 * R), o = rho - side * 2 * R;
    if (side == 0) { ex = R;          ey = -R + 1 + o; }
    else if (side == 1) { ey = R;     ex = R - 1 - o; }
    else if (side == 2) { ex = -R;    ey = R - 1 - o; }
    else { ey = -R;                   ex = -R + 1 + o; }
}

// Steps of a ray to ring cell (R, e) (or its rotations) inside the disc: the
// largest k <= R with k^2 + rnd(k)^2 <= R^2, rnd(k) = k*e/R rounded half away
// from zero.  The left side only grows with k, so a binary search finds it.
__device__ __forceinline__ int disc_steps(int R, int e) {
    const int ae = abs(e);
    int lo = 0, hi = R;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int r = (2 * mid * ae + R) / (2 * R);
        if (mid * mid + r * r <= R * R) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Everything one viewshed needs, for the single-terrain and the batched
// launches alike (the tensor map must stay in parameter space).
struct VsJob {
    CUtensorMap map;          // [H][pitch/8][8] view of the terrain, box 8 x WG x box_rows
    int H, W, R, ht, hr;
    int nsplit, WG, box_rows, nbox, PR, words, wide;
    const int64_t *cand;
    long long n, item0;       // candidates; first item of this job in a batch
    uint32_t *bm;
    int32_t *area;
};

// One candidate: stage the window (per sector), walk the rays of the sector,
// OR visible cells into the shared bitmap, write bitmap and area.  `phase` is
// the parity of the CTA's window barrier, carried across candidates.  Returns
// true when a window copy did not land within two bounded waits: the barrier
// can then no longer be trusted and the CTA must take no further candidate.
template <typename T>
__device__ bool vs_candidate(const CUtensorMap *tmap, const VsJob &J, long long c, unsigned char *smem,
                             uint64_t *bar, uint32_t &phase, int *s_fail, int *red) {
    const int R = J.R, PR = J.PR;
    const int PRs = PR | 1;  // odd row pitch of the shared bitmap: rays on nearby rows hit other banks
    const int WW = J.WG * 8;
    int16_t *win = (int16_t *)smem;
    const int win_elems = J.nbox * J.box_rows * WW;
    uint32_t *bms = (uint32_t *)(smem + ((win_elems * 2 + 127) & ~127));
    const int tid = threadIdx.x;
    const int64_t p = J.cand[c];
    uint32_t *out = J.bm ? J.bm + c * (int64_t)J.words : nullptr;  // NULL: areas only
    if (p < 0 || p >= (int64_t)J.H * J.W) {  // invalid candidate: empty bitmap, area -1
        if (out)
            for (int i = tid; i < J.words; i += blockDim.x) out[i] = 0;
        if (tid == 0) J.area[c] = -1;
        return false;
    }
    const int cx = (int)(p % J.W), cy = (int)(p / J.W);
    const int gw0 = floordiv(cx - R, 32);
    // the whole window inside the grid: no ray meets the grid edge, so a ray
    // ends only at the disc, after a step count found once per ray
    const bool interior = cx >= R && cx <= J.W - 1 - R && cy >= R && cy <= J.H - 1 - R;
    if (tid == 0) *s_fail = 0;
    for (int i = tid; i < (2 * R + 1) * PRs; i += blockDim.x) bms[i] = 0;
    __syncthreads();

    const int nsec = J.nsplit;
    for (int sec = 0; sec < nsec; ++sec) {
        // ---- this pass's window
        int row_lo = cy - R, col_lo = cx - R;
        if (nsec == 2) row_lo = (sec == 0) ? cy - R : cy;
        if (nsec == 4) {
            col_lo = (sec & 1) ? cx : cx - R;
            row_lo = (sec & 2) ? cy : cy - R;
        }
        const int wx0 = floordiv(col_lo, 8) * 8;
        const int wy0 = row_lo;
        if (tid == 0) {
            fence_proxy_async_smem();
            const uint32_t bytes = (uint32_t)(J.nbox * J.box_rows * WW * 2);
            mbar_arrive_expect_tx(bar, bytes);
            for (int b = 0; b < J.nbox; ++b)
                tma_load_3d(win + (size_t)b * J.box_rows * WW, tmap, 0, wx0 / 8, wy0 + b * J.box_rows, bar);
        }
        if (!mbar_wait(bar, phase)) *s_fail = 1;
        __syncthreads();
        if (*s_fail) {
            // give the copy in flight a second bounded chance to land, then
            // report the candidate as timed out; when that wait gives up too,
            // the barrier's phase may still complete later, so the CTA must not
            // reuse it (s_fail = 2: the caller stops taking candidates)
            const bool ok2 = mbar_wait(bar, phase);
            __syncthreads();
            if (tid == 0 && !ok2) *s_fail = 2;
            __syncthreads();
            phase ^= 1u;
            break;
        }
        phase ^= 1u;
        const int eye = (int)win[(cy - wy0) * WW + (cx - wx0)] + J.ht;

        // ---- rays of this sector
        for (int rho = tid; rho < 8 * R; rho += blockDim.x) {
            int ex, ey;
            ring_cell(rho, R, ex, ey);
            int s = 0;
            if (nsec == 2) s = ey > 0;
            if (nsec == 4) s = (ex > 0) + 2 * (ey > 0);
            if (s != sec) continue;
            const bool xmaj = abs(ex) >= abs(ey);
            const int smaj = xmaj ? (ex > 0 ? 1 : -1) : (ey > 0 ? 1 : -1);
            const int dmin = xmaj ? ey : ex;
            const int q = floordiv(dmin, R);
            const int rr = dmin - q * R;
            const int thr = dmin >= 0 ? R : R + 1;
            const int omaj = xmaj ? cx : cy, omin = xmaj ? cy : cx;
            const int minor_lim = xmaj ? J.H : J.W;
            // a0: window address of the post (major omaj + smaj*k, minor omin + y0),
            // the first of the two posts the line passes between at step k; the
            // cell tested at step k is that post or the next one along the minor
            // axis (amin further)
            const int amin = xmaj ? WW : 1;
            const int astep = (xmaj ? smaj : smaj * WW) + q * amin;
            int a0 = xmaj ? (omin - wy0) * WW + (omaj - wx0) : (omaj - wy0) * WW + (omin - wx0);
            const T eyeR = (T)eye * R;
            const int hre = J.hr - eye;
            int f = 0, y0 = 0, gmaj = omaj, k2 = 0;
            T Hn = 0;
            int Hk = 0;
            if (interior) {
                const int kmax = disc_steps(R, dmin);
                // bitmap word of the cell: row and column advance with k and rnd
                const int rowk = xmaj ? 0 : smaj * PRs, rowr = xmaj ? PRs : 0;
                const int wbase = R * PRs - gw0;
                for (int k = 1; k <= kmax; ++k) {
                    f += rr;
                    y0 += q;
                    a0 += astep;
                    if (f >= R) { f -= R; y0 += 1; a0 += amin; }
                    const int rb = (2 * f >= thr) ? 1 : 0;  // round half away from zero
                    const int rnd = y0 + rb;
                    gmaj += smaj;
                    const int zc = win[a0 + (rb ? amin : 0)];
                    const int zo = f > 0 ? (int)win[a0 + (rb ? 0 : amin)] : zc;
                    const bool vis = (Hk == 0) || ((T)(zc + hre) * R * Hk >= Hn * k);
                    if (vis) {
                        const int gx = xmaj ? gmaj : omin + rnd;
                        atomicOr(&bms[wbase + k * rowk + rnd * rowr + (gx >> 5)], 1u << (gx & 31));
                    }
                    const int z0 = rb ? zo : zc, z1 = rb ? zc : zo;
                    const T num = (T)z0 * (R - f) + (T)z1 * f - eyeR;
                    if (Hk == 0 || num * Hk > Hn * k) { Hn = num; Hk = k; }
                }
                continue;
            }
            for (int k = 1; k <= R; ++k) {
                f += rr;
                y0 += q;
                a0 += astep;
                if (f >= R) { f -= R; y0 += 1; a0 += amin; }
                const int rb = (2 * f >= thr) ? 1 : 0;  // round half away from zero
                const int rnd = y0 + rb;
                gmaj += smaj;
                k2 += 2 * k - 1;
                const int gmin = omin + rnd;
                const int gx = xmaj ? gmaj : gmin, gy = xmaj ? gmin : gmaj;
                if ((unsigned)gx >= (unsigned)J.W || (unsigned)gy >= (unsigned)J.H) break;
                if (k2 + rnd * rnd > R * R) break;
                // the straddling posts: the tested cell and, off a post, the
                // other one (inside the staged window even where it leaves the
                // grid), both loads issued before the test
                const int zc = win[a0 + (rb ? amin : 0)];
                const int zo = f > 0 ? (int)win[a0 + (rb ? 0 : amin)] : zc;
                const bool vis = (Hk == 0) || ((T)(zc + hre) * R * Hk >= Hn * k);
                if (vis) atomicOr(&bms[(gy - cy + R) * PRs + ((gx >> 5) - gw0)], 1u << (gx & 31));
                const int m0 = omin + y0;
                if (f > 0 && (m0 < 0 || m0 + 1 >= minor_lim)) break;
                const int z0 = rb ? zo : zc, z1 = rb ? zc : zo;
                const T num = (T)z0 * (R - f) + (T)z1 * f - eyeR;
                if (Hk == 0 || num * Hk > Hn * k) { Hn = num; Hk = k; }
            }
        }
        __syncthreads();  // every read of this window done before the next pass overwrites it
    }

    const bool fail = *s_fail != 0;
    const bool dead = *s_fail == 2;
    if (tid == 0 && !fail) atomicOr(&bms[R * PRs + ((cx >> 5) - gw0)], 1u << (cx & 31));
    __syncthreads();
    int cnt = 0;
    for (int i = tid; i < J.words; i += blockDim.x) {
        const int r = i / PR;
        const uint32_t w = fail ? 0u : bms[r * PRs + (i - r * PR)];
        if (out) out[i] = w;
        cnt += __popc(w);
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((tid & 31) == 0) red[tid >> 5] = cnt;
    __syncthreads();
    if (tid == 0) {
        int a = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += red[w];
        J.area[c] = fail ? VS_ERR_TIMEOUT : a;
    }
    __syncthreads();  // red[] and the bitmap are reused by the next candidate
    return dead;
}

__device__ __forceinline__ unsigned char *vs_smem_base(unsigned char *raw) {
    // TMA destinations must be 128-byte aligned: round the base up (the host
    // reserves 128 spare bytes)
    return raw + ((128u - (smem_u32(raw) & 127u)) & 127u);
}

// one CTA per candidate of one terrain
__global__ void __launch_bounds__(512) k_viewshed(const __grid_constant__ VsJob J) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = vs_smem_base(smem_raw);
    __shared__ uint64_t bar;
    __shared__ int red[32];
    __shared__ int s_fail;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    uint32_t phase = 0;
    if (J.wide) vs_candidate<long long>(&J.map, J, blockIdx.x, smem, &bar, phase, &s_fail, red);
    else vs_candidate<int>(&J.map, J, blockIdx.x, smem, &bar, phase, &s_fail, red);
}

// Batched viewsheds of many terrains in one persistent launch: items
// (job, candidate) are numbered job by job (jobs ordered by decreasing R, so
// the costly ones start first) and pulled from a global counter.
constexpr int kVsMaxJobs = 64;
struct VsBatch {
    VsJob job[kVsMaxJobs];
    int njobs;
    long long total;
    unsigned long long *counter;
};

__global__ void __launch_bounds__(512) k_viewshed_batch(const __grid_constant__ VsBatch B) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = vs_smem_base(smem_raw);
    __shared__ uint64_t bar;
    __shared__ int red[32];
    __shared__ int s_fail;
    __shared__ long long s_item;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    uint32_t phase = 0;
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(B.counter, 1ull);
        __syncthreads();
        const long long it = s_item;
        __syncthreads();
        if (it >= B.total) break;
        int j = 0;
        while (j + 1 < B.njobs && B.job[j + 1].item0 <= it) ++j;
        const VsJob &J = B.job[j];
        const bool dead = J.wide ? vs_candidate<long long>(&J.map, J, it - J.item0, smem, &bar, phase, &s_fail, red)
                                 : vs_candidate<int>(&J.map, J, it - J.item0, smem, &bar, phase, &s_fail, red);
        if (dead) break;  // a copy may still land in this CTA's window: take no more items
    }
}

// ------------------------------------------------------------------ wide ROI
// When the ROI window does not fit in shared memory (R above ~280 posts; the
// paper's own runs use R = 500 .. 2000) one CTA per candidate walks the rays
// of each side of the ring side by side, one ray per thread, in bands of
// steps.  The terrain is read through the L1/L2 caches instead of a staged
// window, from two arrays that pair every post with its neighbour along a
// ray's minor axis (one 32-bit load per step); the east / west one is
// transposed, so that neighbouring rays -- neighbouring threads -- read
// neighbouring words, as the north / south one is in terrain order.  Each band's visible cells collect in a shared-memory tile
// that is then ORed into the candidate's bitmap in global memory.  East / west:
// every window row x 4 words (128 columns), neighbouring rays on neighbouring
// rows.  North / south: 32 window rows stored by column -- one word per column,
// bit i = row i of the band -- so that neighbouring rays, which share a row,
// set bits of neighbouring words rather than the same word; the merge turns
// each 32 x 32 block back into row words with a warp-shuffle bit transpose.  The arithmetic is that of vs_candidate: the same cells, the
// same rounding and the same horizon test, so the bitmaps are identical.
// Values stay in 32 bits with 64-bit products, exact for every accepted input:
// |z*R + (hr - eye)*R| <= (65535 + 2*100000)*4096 < 2^31 and the interpolated
// numerator |z0*(R-f) + z1*f - eye*R| < 2^31 for R <= 4096.
constexpr int kWideThreads = 512;  // two CTAs per SM: one's band barriers overlap the other's rays
constexpr int kWideTW = 4;    // east / west tile: words per window row
constexpr int kWideTP = 5;    // its row pitch, odd: neighbouring rows in other banks
constexpr int kWideBN = 32;   // north / south tile: window rows per band (bits of a column word)

struct VsWide {
    const int16_t *z;
    long long pitch;
    // each post with its neighbour along a ray's minor axis, one 32-bit load:
    // pe[x*H + y] = z(x, y) | z(x, y+1) << 16 (east / west rays, transposed so
    // that neighbouring rays read neighbouring words), pn[y*W + x] = z(x, y) |
    // z(x+1, y) << 16 (north / south rays); a half past the grid edge is 0
    const uint32_t *pe, *pn;
    int H, W, R, ht, hr, PR, words;
    const int64_t *cand;
    long long n;
    uint32_t *bm;
    int32_t *area;
};

// the pair arrays of k_viewshed_wide, one 32 x 32 block of posts per CTA: pn
// row by row, pe through a shared-memory transpose (both coalesced)
__global__ void __launch_bounds__(256) k_vs_pairs(const int16_t *__restrict__ z, long long pitch, int H, int W,
                                                  uint32_t *__restrict__ pe, uint32_t *__restrict__ pn) {
    __shared__ uint32_t t[32][33];
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int j = ty; j < 32; j += 8) {
        const int y = y0 + j, x = x0 + tx;
        if (y < H && x < W) {
            const uint32_t z0 = (uint16_t)z[(long long)y * pitch + x];
            const uint32_t zx = x + 1 < W ? (uint16_t)z[(long long)y * pitch + x + 1] : 0u;
            const uint32_t zy = y + 1 < H ? (uint16_t)z[(long long)(y + 1) * pitch + x] : 0u;
            pn[(long long)y * W + x] = z0 | (zx << 16);
            t[j][tx] = z0 | (zy << 16);
        }
    }
    __syncthreads();
    for (int j = ty; j < 32; j += 8) {
        const int x = x0 + j, y = y0 + tx;
        if (x < W && y < H) pe[(long long)x * H + y] = t[tx][j];
    }
}

// 32 x 32 bit transpose across a warp: lane l holds row l of a bit matrix
// (bit i = column i) and gets column l (bit i = row i); five rounds of block
// swaps between lanes l and l ^ j
__device__ __forceinline__ uint32_t warp_bit_transpose(uint32_t a) {
    const int lane = threadIdx.x & 31;
    uint32_t m = 0x0000FFFFu;
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) {
        const uint32_t o = __shfl_xor_sync(0xffffffffu, a, j);
        a = (lane & j) ? ((a & ~m) | ((o >> j) & m)) : ((a & m) | ((o << j) & ~m));
        m ^= m << (j >> 1);
    }
    return a;
}

__global__ void __launch_bounds__(kWideThreads, 2) k_viewshed_wide(const VsWide P) {
    extern __shared__ __align__(16) uint32_t tile[];
    __shared__ int red[32];
    const int tid = threadIdx.x, nt = blockDim.x;
    const long long c = blockIdx.x;
    const int R = P.R, PR = P.PR;
    const int64_t p = P.cand[c];
    uint32_t *out = P.bm + c * (long long)P.words;
    for (int i = tid; i < P.words; i += nt) out[i] = 0u;
    if (p < 0 || p >= (int64_t)P.H * P.W) {  // invalid candidate: empty bitmap, area -1
        if (tid == 0) P.area[c] = -1;
        return;
    }
    const int cx = (int)(p % P.W), cy = (int)(p / P.W);
    const int gw0 = floordiv(cx - R, 32);
    const int eye = (int)P.z[(long long)cy * P.pitch + cx] + P.ht;
    const int eyeR = eye * R;
    const int hreR = (P.hr - eye) * R;
    // the whole window inside the grid: rays end only at the disc
    const bool interior = cx >= R && cx <= P.W - 1 - R && cy >= R && cy <= P.H - 1 - R;

    for (int side = 0; side < 4; ++side) {  // east, west, north, south
        const bool xmaj = side < 2;
        const int smaj = (side & 1) ? -1 : 1;
        // ring cells (smaj*R, e) for x-major sides (corners included), (e, smaj*R)
        // with |e| < R for y-major ones
        const int elo = xmaj ? -R : -R + 1, ehi = -elo;
        const int omaj = xmaj ? cx : cy, omin = xmaj ? cy : cx;
        const int major_lim = xmaj ? P.W : P.H, minor_lim = xmaj ? P.H : P.W;
        const uint32_t *base = xmaj ? P.pe + (long long)cx * P.H + cy : P.pn + (long long)cy * P.W + cx;
        const int pm = xmaj ? P.H : P.W;
        for (int ea = elo; ea <= ehi; ea += nt) {
            const int eb = min(ehi, ea + nt - 1);
            const int e = ea + tid;  // this thread's ray
            bool alive = e <= eb;
            const int q = floordiv(e, R);
            const int rr = e - q * R;
            const int thr = e >= 0 ? R : R + 1;
            const int astep = smaj * pm + q;
            // a0: offset from the observer's post of the post (major omaj +
            // smaj*k, minor omin + y0); the cell tested is that post or the
            // next one along the minor axis (offset 1 in both arrays)
            int f = 0, y0 = 0, a0 = 0, Hn = 0, Hk = 0;
            const int kmax = (interior && alive) ? disc_steps(R, e) : R;
            // window rows an east / west pass can touch, word columns of a
            // north / south one (|rnd| <= |e| along every ray)
            const int rlo = R + min(0, ea), rhi = R + max(0, eb);
            const int wlo = ((omin + min(0, ea)) >> 5) - gw0, whi = ((omin + max(0, eb)) >> 5) - gw0;
            for (int b = 0;; ++b) {
                int klo, khi, bw0 = 0;
                if (xmaj) {
                    if (smaj > 0) {
                        bw0 = ((cx + 1) >> 5) + kWideTW * b;
                        klo = max(1, 32 * bw0 - cx);
                        khi = min(R, 32 * (bw0 + kWideTW) - 1 - cx);
                    } else {
                        const int bhi = floordiv(cx - 1, 32) - kWideTW * b;
                        bw0 = bhi - kWideTW + 1;
                        klo = max(1, cx - (32 * bhi + 31));
                        khi = min(R, cx - 32 * bw0);
                    }
                } else {
                    klo = 1 + kWideBN * b;
                    khi = min(R, kWideBN * (b + 1));
                }
                if (klo > R) break;
                // also orders the previous band's merge before this clear
                if (!__syncthreads_or(alive ? 1 : 0)) break;
                const int nrow = khi - klo + 1;
                if (xmaj) {
                    for (int i = tid; i < (rhi - rlo + 1) * kWideTW; i += nt)
                        tile[(rlo + i / kWideTW) * kWideTP + (i % kWideTW)] = 0u;
                } else {
                    for (int i = 32 * wlo + tid; i < 32 * (whi + 1); i += nt) tile[i] = 0u;
                }
                __syncthreads();
                if (alive && interior) {
                    const int kend = min(khi, kmax);
                    for (int k = klo; k <= kend; ++k) {
                        f += rr;
                        y0 += q;
                        a0 += astep;
                        if (f >= R) { f -= R; y0 += 1; a0 += 1; }
                        const int rb = (2 * f >= thr) ? 1 : 0;
                        const int rnd = y0 + rb;
                        // both straddling posts in one load (inside the grid here)
                        const uint32_t pr = __ldg(base + a0);
                        const int lo = (int16_t)(pr & 0xFFFFu), hi = (int16_t)(pr >> 16);
                        const int zc = rb ? hi : lo, zo = rb ? lo : hi;
                        const bool vis = (Hk == 0) || ((long long)(zc * R + hreR) * Hk >= (long long)Hn * k);
                        if (vis) {
                            if (xmaj) {
                                const int gmaj = omaj + smaj * k;
                                atomicOr(&tile[(rnd + R) * kWideTP + ((gmaj >> 5) - bw0)], 1u << (gmaj & 31));
                            } else {
                                atomicOr(&tile[omin + rnd - 32 * gw0], 1u << (k - klo));
                            }
                        }
                        const int z0 = rb ? zo : zc, z1 = rb ? zc : zo;
                        const int num = z0 * (R - f) + z1 * f - eyeR;
                        if (Hk == 0 || (long long)num * Hk > (long long)Hn * k) { Hn = num; Hk = k; }
                    }
                    alive = kmax > khi;
                } else if (alive) {
                    for (int k = klo; k <= khi; ++k) {
                        f += rr;
                        y0 += q;
                        a0 += astep;
                        if (f >= R) { f -= R; y0 += 1; a0 += 1; }
                        const int rb = (2 * f >= thr) ? 1 : 0;  // round half away from zero
                        const int rnd = y0 + rb;
                        const int gmaj = omaj + smaj * k, gmin = omin + rnd;
                        if ((unsigned)gmaj >= (unsigned)major_lim || (unsigned)gmin >= (unsigned)minor_lim ||
                            k * k + rnd * rnd > R * R) {
                            alive = false;
                            break;
                        }
                        // both straddling posts in one load from the pair of the
                        // first one; when that post lies outside the grid (the ray
                        // stops after this test) the pair of the tested cell
                        const int m0 = omin + y0;
                        const bool stop = f > 0 && (m0 < 0 || m0 + 1 >= minor_lim);
                        const bool up = rb && !stop;  // tested cell = upper half
                        const uint32_t pr = __ldg(base + a0 + ((rb && stop) ? 1 : 0));
                        const int lo = (int16_t)(pr & 0xFFFFu), hi = (int16_t)(pr >> 16);
                        const int zc = up ? hi : lo, zo = up ? lo : hi;
                        const bool vis = (Hk == 0) || ((long long)(zc * R + hreR) * Hk >= (long long)Hn * k);
                        if (vis) {
                            if (xmaj)
                                atomicOr(&tile[(rnd + R) * kWideTP + ((gmaj >> 5) - bw0)], 1u << (gmaj & 31));
                            else
                                atomicOr(&tile[gmin - 32 * gw0], 1u << (k - klo));
                        }
                        if (stop) {
                            alive = false;
                            break;
                        }
                        const int z0 = rb ? zo : zc, z1 = rb ? zc : zo;
                        const int num = z0 * (R - f) + z1 * f - eyeR;
                        if (Hk == 0 || (long long)num * Hk > (long long)Hn * k) { Hn = num; Hk = k; }
                    }
                }
                __syncthreads();
                // OR the band into the bitmap; one thread per word, read-modify-write
                if (xmaj) {
                    for (int i = tid; i < (rhi - rlo + 1) * kWideTW; i += nt) {
                        const int r = rlo + i / kWideTW, j = i % kWideTW;
                        const uint32_t t = tile[r * kWideTP + j];
                        const int w = bw0 + j - gw0;
                        if (t && w >= 0 && w < PR) out[(long long)r * PR + w] |= t;
                    }
                } else {
                    // warp per word column: transpose its 32 x 32 block, lane i
                    // holds window row klo + i
                    const int lane = tid & 31;
                    for (int w = wlo + (tid >> 5); w <= whi; w += nt >> 5) {
                        const uint32_t t = warp_bit_transpose(tile[32 * w + lane]);
                        if (t && lane < nrow) out[(long long)(R + smaj * (klo + lane)) * PR + w] |= t;
                    }
                }
            }
        }
    }
    __syncthreads();  // every merge done before the observer's word is touched
    if (tid == 0) out[(long long)R * PR + ((cx >> 5) - gw0)] |= 1u << (cx & 31);
    __syncthreads();
    int cnt = 0;
    for (int i = tid; i < P.words; i += nt) cnt += __popc(out[i]);
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((tid & 31) == 0) red[tid >> 5] = cnt;
    __syncthreads();
    if (tid == 0) {
        int a = 0;
        for (int w = 0; w < (nt >> 5); ++w) a += red[w];
        P.area[c] = a;
    }
}

static size_t wide_smem_bytes(int R) {
    const size_t ew = (size_t)(2 * R + 1) * kWideTP;
    const size_t ns = (size_t)32 * words_per_row(R);
    return std::max(ew, ns) * 4;
}

// shared-memory bytes for a split choice
static size_t vs_smem_bytes(int R, int nsplit, int *WG, int *box_rows, int *nbox) {
    int rows = (nsplit == 1) ? 2 * R + 1 : R + 1;
    int cols = (nsplit == 4) ? R + 1 : 2 * R + 1;
    int wg = (cols + 7 + 7) / 8;  // room for rounding the left edge down to 8
    int nb = (rows + 255) / 256;
    int br = ((rows + nb - 1) / nb + 7) / 8 * 8;
    if (br > 256) { nb += 1; br = ((rows + nb - 1) / nb + 7) / 8 * 8; }
    *WG = wg; *box_rows = br; *nbox = nb;
    size_t win = (size_t)nb * br * wg * 8 * 2;
    win = (win + 127) & ~(size_t)127;
    size_t words = (size_t)(2 * R + 1) * (words_per_row(R) | 1);  // odd row pitch in shared memory
    return win + ((words + 31) & ~(size_t)31) * 4 + 64 + 128;
}

static int vs_pick_split(int R, int *nsplit, int *WG, int *box_rows, int *nbox, size_t *smem) {
    // prefer two resident CTAs per SM, else the largest window that fits
    const size_t two = 110 * 1024, one = 225 * 1024;
    for (size_t lim : {two, one})
        for (int ns : {1, 2, 4}) {
            size_t b = vs_smem_bytes(R, ns, WG, box_rows, nbox);
            if (*WG <= 256 && b <= lim) { *nsplit = ns; *smem = b; return VS_OK; }
        }
    return VS_ERR_RANGE;
}

}  // namespace vs

using namespace vs;

// R whose window does not fit in shared memory (or forced by the tuning
// table) takes the banded kernel, which needs the pair arrays
static bool vs_wide(int R) {
    if (tune_get(VS_TUNE_VIEWSHED_WIDE, R, 0) == 1) return true;
    int ns = 0, wg = 0, br = 0, nb = 0;
    size_t sm = 0;
    return vs_pick_split(R, &ns, &wg, &br, &nb, &sm) != VS_OK;
}
// the two pair arrays of the banded kernel: 4 bytes per post each
static size_t vs_pairs_bytes(int H, int W) { return (size_t)H * (size_t)W * 8 + 512; }

extern "C" size_t vs_viewshed_workspace(int32_t H, int32_t W, int32_t R, int64_t n) {
    (void)n;
    if (H < 1 || W < 1 || H > kMaxH || W > kMaxH || R < 1 || R > kMaxR || !vs_wide(R)) return 0;
    return vs_pairs_bytes(H, W);
}

static int vs_viewshed_wide(const vs_grid &g, int32_t R, int32_t ht, int32_t hr, const int64_t *cand,
                            int64_t n, uint32_t *bm_out, int32_t *area_out, void *ws, size_t ws_bytes,
                            cudaStream_t s, bool pairs_ready = false) {
    int rc = check_grid(g);
    if (rc) return rc;
    if (ht < -100000 || ht > 100000 || hr < -100000 || hr > 100000) return VS_ERR_RANGE;
    if (n < 0 || n > 0x7fffffffll) return VS_ERR_RANGE;
    if (n > 0 && (!cand || !bm_out || !area_out)) return VS_ERR_ARG;
    // window offsets of the ray walk are 32-bit
    if ((long long)R * ((long long)std::max(g.H, g.W) + 1) >= (1ll << 31)) return VS_ERR_RANGE;
    const size_t need = vs_viewshed_workspace(g.H, g.W, R, n);
    if (n == 0) return VS_OK;
    if (!ws || ws_bytes < need) return VS_ERR_WS;
    if ((rc = check_device())) return rc;
    uint32_t *pe = (uint32_t *)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    uint32_t *pn = (uint32_t *)(((uintptr_t)(pe + (size_t)g.H * g.W) + 255) & ~(uintptr_t)255);
    if (!pairs_ready) {
        const dim3 tg((unsigned)((g.W + 31) / 32), (unsigned)((g.H + 31) / 32));
        k_vs_pairs<<<tg, 256, 0, s>>>(g.z, g.pitch, g.H, g.W, pe, pn);
        vs::note_launch();
        VS_CUDA_TRY(cudaGetLastError());
    }
    VsWide P;
    P.z = g.z; P.pitch = g.pitch; P.pe = pe; P.pn = pn;
    P.H = g.H; P.W = g.W; P.R = R; P.ht = ht; P.hr = hr;
    P.PR = words_per_row(R);
    P.words = (2 * R + 1) * P.PR;
    P.cand = cand; P.n = n; P.bm = bm_out; P.area = area_out;
    const size_t smem = wide_smem_bytes(R);
    VS_CUDA_TRY(cudaFuncSetAttribute(k_viewshed_wide, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_viewshed_wide<<<(unsigned)n, kWideThreads, smem, s>>>(P);
    vs::note_launch();
    VS_CUDA_TRY(cudaGetLastError());
    return VS_OK;
}

// untuned CTA size: 512 threads (the autotuner's choice for R = 50..250 on
// GB300), fewer when the ring has fewer rays
static int default_threads(int R) {
    return 8 * R >= 512 ? 512 : (8 * R >= 256 ? 256 : 128);
}

static int vs_make_job(const vs_grid &g, int32_t R, int32_t ht, int32_t hr, const int64_t *cand,
                       int64_t n, uint32_t *bm_out, int32_t *area_out, VsJob *J, size_t *smem,
                       bool areas_only = false) {
    int rc = check_grid(g);
    if (rc) return rc;
    if (R < 1 || R > kMaxR) return VS_ERR_RANGE;
    if (ht < -100000 || ht > 100000 || hr < -100000 || hr > 100000) return VS_ERR_RANGE;
    if (n < 0 || n > 0x7fffffffll) return VS_ERR_RANGE;
    if (n > 0 && (!cand || (!bm_out && !areas_only) || !area_out)) return VS_ERR_ARG;
    memset(J, 0, sizeof(*J));
    J->H = g.H; J->W = g.W; J->R = R; J->ht = ht; J->hr = hr;
    J->cand = cand; J->n = n; J->bm = bm_out; J->area = area_out;
    J->PR = words_per_row(R);
    J->words = (2 * R + 1) * J->PR;
    if ((rc = vs_pick_split(R, &J->nsplit, &J->WG, &J->box_rows, &J->nbox, smem))) return rc;
    GridMap gm;
    if ((rc = make_grid_map(&gm, g, J->WG, J->box_rows))) return rc;
    J->map = gm.map;
    // 32-bit products are exact when (z range + |ht| + |hr|) * R^2 < 2^31
    const long long bound = (65535ll + std::abs(ht) + std::abs(hr)) * (long long)R * R;
    J->wide = bound >= (1ll << 31);
    return VS_OK;
}

extern "C" int vs_viewshed(vs_grid g, int32_t R, int32_t ht, int32_t hr, const int64_t *cand,
                           int64_t n, uint32_t *bm_out, int32_t *area_out, void *ws,
                           size_t ws_bytes, vs_stream_t st) {
    if (R < 1 || R > kMaxR) return VS_ERR_RANGE;
    if (vs_wide(R)) return vs_viewshed_wide(g, R, ht, hr, cand, n, bm_out, area_out, ws, ws_bytes, (cudaStream_t)st);
    VsJob J;
    size_t smem = 0;
    int rc = vs_make_job(g, R, ht, hr, cand, n, bm_out, area_out, &J, &smem);
    if (rc) return rc;
    if (n == 0) return VS_OK;
    if ((rc = check_device())) return rc;
    VS_CUDA_TRY(cudaFuncSetAttribute(k_viewshed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int threads = tune_get(VS_TUNE_VIEWSHED_THREADS, R, default_threads(R));
    k_viewshed<<<(unsigned)n, threads, smem, (cudaStream_t)st>>>(J);
    vs::note_launch();
    VS_CUDA_TRY(cudaGetLastError());
    return VS_OK;
}

extern "C" size_t vs_viewshed_batch_workspace(int32_t n_jobs) {
    (void)n_jobs;
    return 256;
}

extern "C" int vs_viewshed_batch(const vs_viewshed_job *jobs, int32_t n_jobs, void *ws, size_t ws_bytes,
                                 vs_stream_t st) {
    if (n_jobs < 0 || n_jobs > kVsMaxJobs) return VS_ERR_RANGE;
    if (n_jobs == 0) return VS_OK;
    if (!jobs) return VS_ERR_ARG;
    if (!ws || ws_bytes < vs_viewshed_batch_workspace(n_jobs)) return VS_ERR_WS;
    int rc = check_device();
    if (rc) return rc;
    // largest ROI first: the longest items start early, the short ones fill the tail
    int order[kVsMaxJobs];
    for (int i = 0; i < n_jobs; ++i) order[i] = i;
    std::stable_sort(order, order + n_jobs, [&](int a, int b) { return jobs[a].R > jobs[b].R; });
    static VsBatch B;  // large (16 KB): built on the host, copied into the launch's parameters
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    memset(&B, 0, sizeof(B));
    size_t smem = 0;
    long long total = 0;
    int nj = 0;
    for (int i = 0; i < n_jobs; ++i) {
        const vs_viewshed_job &q = jobs[order[i]];
        size_t sm = 0;
        if ((rc = vs_make_job(q.g, q.R, q.ht, q.hr, q.cand, q.n, q.bm_out, q.area_out, &B.job[nj], &sm)))
            return rc;
        if (q.n == 0) continue;
        B.job[nj].item0 = total;
        total += q.n;
        smem = std::max(smem, sm);
        ++nj;
    }
    if (total == 0) return VS_OK;
    B.njobs = nj;
    B.total = total;
    B.counter = (unsigned long long *)ws;
    cudaStream_t s = (cudaStream_t)st;
    VS_CUDA_TRY(cudaMemsetAsync(ws, 0, 8, s));
    VS_CUDA_TRY(cudaFuncSetAttribute(k_viewshed_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, sms = 0, per = 0;
    VS_CUDA_TRY(cudaGetDevice(&dev));
    VS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // one CTA size for the launch: the tuned size of the largest ROI
    const int threads = tune_get(VS_TUNE_VIEWSHED_THREADS, B.job[0].R, default_threads(B.job[0].R));
    VS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_viewshed_batch, threads, smem));
    const long long grid = std::min<long long>(total, (long long)sms * std::max(per, 1));
    k_viewshed_batch<<<(unsigned)grid, threads, smem, s>>>(B);
    vs::note_launch();
    VS_CUDA_TRY(cudaGetLastError());
    return VS_OK;
}

// ------------------------------------------------------------------ exact visibility index
// The label of the learned proposal (Sec. "Definitions": the visibility index
// is the fraction of the receivers within the ROI that the transmitter sees).
// Numerator: the viewshed's area (areas-only viewshed launch for windows that
// fit in shared memory; the banded kernel, in chunks through a bitmap buffer,
// for large ROIs).  Denominator: the lattice points of disc(R) whose post is
// inside the grid, summed by rows (isqrt of R^2 - dy^2, clipped to the grid).
namespace vs {
// out[i] = area[i] / den(post i), the quotient of two integers rounded once to
// float (divided in double, then rounded to float: with 53 >= 2*24 + 2
// significand bits the second rounding cannot differ from a direct one); a
// negative area (post outside the grid, timed-out wait) is passed through
__global__ void k_exact_vix(const int64_t *__restrict__ posts, int64_t n, int H, int W, int R,
                            const int32_t *__restrict__ area, float *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int a = area[i];
    if (a < 0) {
        out[i] = (float)a;
        return;
    }
    const int64_t p = posts[i];
    const int cx = (int)(p % W), cy = (int)(p / W);
    long long den = 0;
    const int y0 = max(-R, -cy), y1 = min(R, H - 1 - cy);
    for (int dy = y0; dy <= y1; ++dy) {
        const int h = isqrt_exact(R * R - dy * dy);
        den += min(W - 1, cx + h) - max(0, cx - h) + 1;
    }
    out[i] = __double2float_rn(__ddiv_rn((double)a, (double)den));
}
}  // namespace vs

static constexpr size_t kLabelBitmapBytes = (size_t)1 << 30;  // bitmap chunk of the banded path

static inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// candidates per banded chunk: bitmaps within kLabelBitmapBytes
static int64_t label_chunk(int32_t R, int64_t n) {
    const int64_t words = (int64_t)(2 * R + 1) * words_per_row(R);
    return std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)(kLabelBitmapBytes / (4 * (size_t)words))));
}

extern "C" size_t vs_exact_vix_workspace(int32_t H, int32_t W, int32_t R, int64_t n) {
    if (H < 1 || W < 1 || H > kMaxH || W > kMaxH || R < 1 || R > kMaxR || n < 0) return 0;
    size_t b = al256((size_t)n * 4) + 256;
    if (vs_wide(R)) {
        const int64_t words = (int64_t)(2 * R + 1) * words_per_row(R);
        b += al256(vs_pairs_bytes(H, W)) + al256((size_t)label_chunk(R, n) * words * 4);
    }
    return b;
}

extern "C" int vs_exact_vix(vs_grid g, int32_t R, int32_t ht, int32_t hr, const int64_t *posts, int64_t n,
                            float *out, void *ws, size_t ws_bytes, vs_stream_t st) {
    if (R < 1 || R > kMaxR) return VS_ERR_RANGE;
    int rc = check_grid(g);
    if (rc) return rc;
    if (ht < -100000 || ht > 100000 || hr < -100000 || hr > 100000) return VS_ERR_RANGE;
    if (n < 0 || n > 0x7fffffffll) return VS_ERR_RANGE;
    if (n == 0) return VS_OK;
    if (!posts || !out) return VS_ERR_ARG;
    if (!ws || ws_bytes < vs_exact_vix_workspace(g.H, g.W, R, n)) return VS_ERR_WS;
    if ((rc = check_device())) return rc;
    cudaStream_t s = (cudaStream_t)st;
    char *w = (char *)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    int32_t *area = (int32_t *)w;
    w += al256((size_t)n * 4);
    if (vs_wide(R)) {
        const size_t pb = al256(vs_pairs_bytes(g.H, g.W));
        uint32_t *bm = (uint32_t *)(w + pb);
        const int64_t chunk = label_chunk(R, n);
        for (int64_t i = 0; i < n; i += chunk) {
            const int64_t m = std::min(chunk, n - i);
            if ((rc = vs_viewshed_wide(g, R, ht, hr, posts + i, m, bm, area + i, w, pb, s, i > 0))) return rc;
        }
    } else {
        VsJob J;
        size_t smem = 0;
        if ((rc = vs_make_job(g, R, ht, hr, posts, n, nullptr, area, &J, &smem, true))) return rc;
        VS_CUDA_TRY(cudaFuncSetAttribute(k_viewshed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const int threads = tune_get(VS_TUNE_VIEWSHED_THREADS, R, default_threads(R));
        k_viewshed<<<(unsigned)n, threads, smem, s>>>(J);
        vs::note_launch();
        VS_CUDA_TRY(cudaGetLastError());
    }
    k_exact_vix<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(posts, n, g.H, g.W, R, area, out);
    vs::note_launch();
    VS_CUDA_TRY(cudaGetLastError());
    return VS_OK;
}
