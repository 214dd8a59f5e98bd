// vix.cu -- Vix stage (Sec. "The multiple transmitter siting process", Vix):
// approximate visibility index of every post from S random lines of sight.
//
// One CTA owns a TX x TY tile of posts.  The tile plus an R-post halo is
// staged into shared memory with TMA; every LOS of the tile's posts then
// reads only shared memory.  Receivers are drawn by a counter-based generator
// (SplitMix64 of the sample number), so no random state is stored and the
// samples of a post do not depend on the launch shape.  When the halo window
// is too large for shared memory the samples are processed in passes by the
// sign of dy (halves) or of dx and dy (quadrants); a LOS never leaves the
// bounding box of its two end posts, so each pass stages only that part.
#include <algorithm>
#include <cstdlib>

#include <mutex>
#include <cstring>
#include "vs_common.cuh"

namespace vs {

constexpr int kVixThreads = 1024;
constexpr int kVixMaxPPT = 4;  // posts per thread

struct VixParams {
    int H, W, R, ht, hr, S;
    uint64_t seed;
    uint8_t *out;
    int NR;                // |disc(R)| - 1
    int nsplit;            // 1, 2 (by sign of dy) or 4 (signs of dx, dy)
    int TX, TY;            // tile of posts per CTA
    int WG;                // window width in 8-element groups
    int box_rows, nbox;    // TMA boxes per pass
    unsigned long long *steps;  // optional: crossings evaluated (accumulated)
};

__device__ __forceinline__ uint64_t splitmix64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <bool COUNT>
__global__ void __launch_bounds__(kVixThreads, 1) k_vix(const __grid_constant__ CUtensorMap tmap,
                                                        const VixParams P) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    const int R = P.R, TX = P.TX, TY = P.TY;
    const int WW = P.WG * 8;
    int16_t *win = (int16_t *)smem;
    const int win_elems = P.nbox * P.box_rows * WW;
    int *rowstart = (int *)(smem + ((win_elems * 2 + 127) & ~127));  // 2R+2 entries
    int *hwtab = rowstart + (2 * R + 2);                                 // 2R+1 entries
    uint64_t *bar = (uint64_t *)(hwtab + ((2 * R + 1 + 1) & ~1));
    __shared__ int warp_tot[32];
    __shared__ int s_fail;

    const int tid = threadIdx.x;
    const int tx0 = blockIdx.x * TX, ty0 = blockIdx.y * TY;

    if (tid == 0) {
        mbar_init(bar, 1);
        s_fail = 0;
    }

    // ---- row table of the offset list OFF_R (rows dy = -R..R, dx ascending,
    // origin removed): rowstart[i] = entries in rows before dy = i - R
    {
        const int nrow = 2 * R + 1;
        const int chunk = (nrow + kVixThreads - 1) / kVixThreads;
        const int i0 = tid * chunk, i1 = min(nrow, i0 + chunk);
        int local = 0;
        for (int i = i0; i < i1; ++i) {
            const int dy = i - R;
            const int hw = isqrt_exact(R * R - dy * dy);
            hwtab[i] = hw;
            local += 2 * hw + 1 - (dy == 0 ? 1 : 0);
        }
        int incl = local;
        const int lane = tid & 31, wid = tid >> 5;
        for (int o = 1; o < 32; o <<= 1) {
            int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) warp_tot[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int t = warp_tot[lane];
            for (int o = 1; o < 32; o <<= 1) {
                int v = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += v;
            }
            warp_tot[lane] = t;  // inclusive over warps
        }
        __syncthreads();
        int run = incl - local + (wid > 0 ? warp_tot[wid - 1] : 0);
        if (tid == 0) rowstart[0] = 0;
        for (int i = i0; i < i1; ++i) {
            const int dy = i - R;
            run += 2 * hwtab[i] + 1 - (dy == 0 ? 1 : 0);
            rowstart[i + 1] = run;
        }
    }
    __syncthreads();

    int cnt[kVixMaxPPT];
#pragma unroll
    for (int j = 0; j < kVixMaxPPT; ++j) cnt[j] = 0;
    const int nposts = TX * TY;
    const uint64_t GOLD = 0x9E3779B97F4A7C15ull;
    unsigned long long nsteps = 0;

    for (int sec = 0; sec < P.nsplit; ++sec) {
        int col_lo = tx0 - R, row_lo = ty0 - R;
        if (P.nsplit == 2) row_lo = (sec == 0) ? ty0 - R : ty0;
        if (P.nsplit == 4) {
            col_lo = (sec & 1) ? tx0 : tx0 - R;
            row_lo = (sec & 2) ? ty0 : ty0 - R;
        }
        const int wx0 = floordiv(col_lo, 8) * 8;
        const int wy0 = row_lo;
        if (tid == 0) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, (uint32_t)(win_elems * 2));
            for (int b = 0; b < P.nbox; ++b)
                tma_load_3d(win + (size_t)b * P.box_rows * WW, &tmap, 0, wx0 / 8,
                            wy0 + b * P.box_rows, bar);
        }
        if (!mbar_wait(bar, (uint32_t)(sec & 1))) s_fail = 1;
        __syncthreads();
        if (s_fail) {
            mbar_wait(bar, (uint32_t)(sec & 1));
            break;
        }

#pragma unroll
        for (int j = 0; j < kVixMaxPPT; ++j) {
            const int i = tid + j * kVixThreads;
            if (i >= nposts) break;
            const int gx = tx0 + i % TX, gy = ty0 + i / TX;
            if (gx >= P.W || gy >= P.H) continue;
            const int a0 = (gy - wy0) * WW + (gx - wx0);
            const int E = (int)win[a0] + P.ht;
            const uint64_t p = (uint64_t)gy * (uint64_t)P.W + (uint64_t)gx;
            uint64_t state = P.seed + GOLD * (p * (uint64_t)P.S + 1ull);
            for (int s = 0; s < P.S; ++s, state += GOLD) {
                const uint64_t u = splitmix64_mix(state);
                const unsigned idx = __umulhi((unsigned)(u >> 32), (unsigned)P.NR);
                // row of OFF_R holding entry idx
                int lo = 0, hi = 2 * R;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if ((unsigned)rowstart[mid] <= idx) lo = mid; else hi = mid - 1;
                }
                const int dy = lo - R;
                int dx = -hwtab[lo] + (int)(idx - (unsigned)rowstart[lo]);
                if (dy == 0 && dx >= 0) dx += 1;
                int s_of = 0;
                if (P.nsplit == 2) s_of = dy > 0;
                if (P.nsplit == 4) s_of = (dx > 0) + 2 * (dy > 0);
                if (s_of != sec) continue;
                if ((unsigned)(gx + dx) >= (unsigned)P.W || (unsigned)(gy + dy) >= (unsigned)P.H)
                    continue;  // receiver off the terrain: not visible
                // ---- line of sight (Sec. "Terrain visibility")
                const int adx = abs(dx), ady = abs(dy);
                const bool xmaj = adx >= ady;
                const int D = xmaj ? adx : ady;
                const int dmin = xmaj ? dy : dx;
                const int ms = xmaj ? (dx > 0 ? 1 : -1) : (dy > 0 ? WW : -WW);
                const int ns = xmaj ? WW : 1;
                const int q = floordiv(dmin, D);
                const int r = dmin - q * D;
                const int step = ms + q * ns;
                const int tsl = (int)win[a0 + dx + dy * WW] + P.hr - E;
                int f = 0, a = a0, lhs = 0;
                bool vis = true;
                for (int jj = 1; jj < D; ++jj) {
                    f += r;
                    a += step;
                    if (f >= D) { f -= D; a += ns; }
                    lhs += tsl;
                    const int z0 = win[a];
                    const int z1 = win[f ? a + ns : a];
                    const int rhs = (z0 - E) * D + (z1 - z0) * f;
                    if (lhs < rhs) { vis = false; if (COUNT) nsteps += jj; break; }
                }
                if (COUNT && vis) nsteps += D - 1;
                cnt[j] += vis ? 1 : 0;
            }
        }
        __syncthreads();
    }

#pragma unroll
    for (int j = 0; j < kVixMaxPPT; ++j) {
        const int i = tid + j * kVixThreads;
        if (i >= nposts) break;
        const int gx = tx0 + i % TX, gy = ty0 + i / TX;
        if (gx >= P.W || gy >= P.H) continue;
        // a timed-out window load is reported as 0xFF (above any valid count)
        P.out[(size_t)gy * P.W + gx] = s_fail ? (uint8_t)0xFF : (uint8_t)cnt[j];
    }
    if (COUNT) {
        for (int o = 16; o > 0; o >>= 1) nsteps += __shfl_xor_sync(0xffffffffu, nsteps, o);
        if ((tid & 31) == 0 && nsteps) atomicAdd(P.steps, nsteps);
    }
}

// ------------------------------------------------------------------ length-sorted variant
// The same computation with the lines of sight of a CTA ordered by length
// before they are walked.  A warp walks 32 consecutive lines of the sorted
// list, so its lanes have (nearly) the same number of crossings and little
// time is lost waiting for the longest lane; the per-line set-up is paid
// once per line instead of once per crossing.  Lines are described by a
// packed 32-bit item (post in tile: 11 bits, dx+R and dy+R: 10 bits each),
// so this variant serves R <= 511 and tiles of at most 2048 posts.
constexpr int kVixSB = 10;  // samples per post in one sorted batch

struct Vix2Params {
    VixParams b;
    int lgTX;          // log2(TX)
    int sb;            // samples per batch
};

__device__ __forceinline__ void vix_offset(uint64_t state, unsigned NR, int R, const int *rowstart,
                                           const int *hwtab, int &dx, int &dy) {
    const uint64_t u = splitmix64_mix(state);
    const unsigned idx = __umulhi((unsigned)(u >> 32), NR);
    int lo = 0, hi = 2 * R;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((unsigned)rowstart[mid] <= idx) lo = mid; else hi = mid - 1;
    }
    dy = lo - R;
    dx = -hwtab[lo] + (int)(idx - (unsigned)rowstart[lo]);
    if (dy == 0 && dx >= 0) dx += 1;
}

// one tile of posts (left column tx0, top row ty0) of one terrain; the CTA's
// mbarrier and its phase parity are carried across tiles.  Returns true when a
// window copy did not land within two bounded waits (the barrier can then no
// longer be trusted: the CTA must take no further tile).
template <bool COUNT>
__device__ bool vix2_tile(const CUtensorMap *tmapp, const Vix2Params &Q, int tx0, int ty0, unsigned char *smem,
                          uint64_t *bar, uint32_t &phase, int *warp_tot, int *s_failp) {
    const VixParams &P = Q.b;
    int &s_fail = *s_failp;
    const int R = P.R, TX = P.TX, TY = P.TY, lgTX = Q.lgTX;
    const int WW = P.WG * 8;
    const int nposts = TX * TY;
    int16_t *win = (int16_t *)smem;
    const int win_elems = P.nbox * P.box_rows * WW;
    uint32_t *items = (uint32_t *)(smem + ((win_elems * 2 + 127) & ~127));
    int *cnt = (int *)(items + nposts * Q.sb);
    int *hist = cnt + nposts;                      // R + 2 entries
    int *rowstart = hist + ((R + 2 + 3) & ~3);      // 2R + 2 entries
    int *hwtab = rowstart + (2 * R + 2);            // 2R + 1 entries

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) s_fail = 0;
    for (int i = tid; i < nposts; i += blockDim.x) cnt[i] = 0;
    // ---- row table of OFF_R (as in k_vix)
    {
        const int nrow = 2 * R + 1;
        const int chunk = (nrow + kVixThreads - 1) / kVixThreads;
        const int i0 = tid * chunk, i1 = min(nrow, i0 + chunk);
        int local = 0;
        for (int i = i0; i < i1; ++i) {
            const int dy = i - R;
            const int hw = isqrt_exact(R * R - dy * dy);
            hwtab[i] = hw;
            local += 2 * hw + 1 - (dy == 0 ? 1 : 0);
        }
        int incl = local;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) warp_tot[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int t = warp_tot[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += v;
            }
            warp_tot[lane] = t;
        }
        __syncthreads();
        int run = incl - local + (wid > 0 ? warp_tot[wid - 1] : 0);
        if (tid == 0) rowstart[0] = 0;
        for (int i = i0; i < i1; ++i) {
            run += 2 * hwtab[i] + 1 - (i == R ? 1 : 0);
            rowstart[i + 1] = run;
        }
    }
    __syncthreads();
    const uint64_t GOLD = 0x9E3779B97F4A7C15ull;
    const unsigned NR = (unsigned)P.NR;
    unsigned long long nsteps = 0;

    for (int sec = 0; sec < P.nsplit; ++sec) {
        int col_lo = tx0 - R, row_lo = ty0 - R;
        if (P.nsplit == 2) row_lo = (sec == 0) ? ty0 - R : ty0;
        if (P.nsplit == 4) {
            col_lo = (sec & 1) ? tx0 : tx0 - R;
            row_lo = (sec & 2) ? ty0 : ty0 - R;
        }
        const int wx0 = floordiv(col_lo, 8) * 8;
        const int wy0 = row_lo;
        if (tid == 0) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, (uint32_t)(win_elems * 2));
            for (int b = 0; b < P.nbox; ++b)
                tma_load_3d(win + (size_t)b * P.box_rows * WW, tmapp, 0, wx0 / 8,
                            wy0 + b * P.box_rows, bar);
        }
        if (!mbar_wait(bar, phase & 1u)) s_fail = 1;
        __syncthreads();
        if (s_fail) {
            const bool ok2 = mbar_wait(bar, phase & 1u);
            __syncthreads();
            if (tid == 0 && !ok2) s_fail = 2;
            __syncthreads();
            phase ^= 1u;
            break;
        }
        phase ^= 1u;
        for (int s0 = 0; s0 < P.S; s0 += Q.sb) {
            const int nb = min(Q.sb, P.S - s0);
            // ---- pass A: how many lines of each length
            for (int i = tid; i < R + 2; i += blockDim.x) hist[i] = 0;
            __syncthreads();
            for (int pp = tid; pp < nposts; pp += blockDim.x) {
                const int gx = tx0 + (pp & (TX - 1)), gy = ty0 + (pp >> lgTX);
                const bool in = gx < P.W && gy < P.H;
                const uint64_t p = (uint64_t)gy * (uint64_t)P.W + (uint64_t)gx;
                uint64_t state = P.seed + GOLD * (p * (uint64_t)P.S + (uint64_t)s0 + 1ull);
                for (int s = 0; s < nb; ++s, state += GOLD) {
                    int dx, dy;
                    vix_offset(state, NR, R, rowstart, hwtab, dx, dy);
                    int s_of = 0;
                    if (P.nsplit == 2) s_of = dy > 0;
                    if (P.nsplit == 4) s_of = (dx > 0) + 2 * (dy > 0);
                    const bool ok = in && s_of == sec && (unsigned)(gx + dx) < (unsigned)P.W &&
                                    (unsigned)(gy + dy) < (unsigned)P.H;
                    const int D = max(abs(dx), abs(dy));
                    const unsigned m = __match_any_sync(__activemask(), ok ? D : -1);
                    if (ok && lane == __ffs(m) - 1) atomicAdd(&hist[D], __popc(m));
                }
            }
            __syncthreads();
            // ---- exclusive scan of the histogram (warp 0); hist[R+1] = total
            if (wid == 0) {
                const int nbin = R + 2;
                const int per = (nbin + 31) / 32;
                const int b0 = lane * per, b1 = min(nbin, b0 + per);
                int loc = 0;
                for (int i = b0; i < b1; ++i) loc += hist[i];
                int incl = loc;
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v;
                }
                int run = incl - loc;
                for (int i = b0; i < b1; ++i) {
                    const int v = hist[i];
                    hist[i] = run;
                    run += v;
                }
            }
            __syncthreads();
            const int total = hist[R + 1];
            __syncthreads();
            // ---- pass B: the same lines again, scattered into length order
            for (int pp = tid; pp < nposts; pp += blockDim.x) {
                const int gx = tx0 + (pp & (TX - 1)), gy = ty0 + (pp >> lgTX);
                const bool in = gx < P.W && gy < P.H;
                const uint64_t p = (uint64_t)gy * (uint64_t)P.W + (uint64_t)gx;
                uint64_t state = P.seed + GOLD * (p * (uint64_t)P.S + (uint64_t)s0 + 1ull);
                for (int s = 0; s < nb; ++s, state += GOLD) {
                    int dx, dy;
                    vix_offset(state, NR, R, rowstart, hwtab, dx, dy);
                    int s_of = 0;
                    if (P.nsplit == 2) s_of = dy > 0;
                    if (P.nsplit == 4) s_of = (dx > 0) + 2 * (dy > 0);
                    const bool ok = in && s_of == sec && (unsigned)(gx + dx) < (unsigned)P.W &&
                                    (unsigned)(gy + dy) < (unsigned)P.H;
                    const int D = max(abs(dx), abs(dy));
                    const unsigned m = __match_any_sync(__activemask(), ok ? D : -1);
                    int base = 0;
                    if (ok && lane == __ffs(m) - 1) base = atomicAdd(&hist[D], __popc(m));
                    base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
                    if (ok)
                        items[base + __popc(m & ((1u << lane) - 1u))] =
                            (uint32_t)pp | ((uint32_t)(dx + R) << 11) | ((uint32_t)(dy + R) << 21);
                }
            }
            __syncthreads();
            // ---- pass C: walk the lines, 32 of (nearly) equal length per warp step
            for (int i = wid * 32 + lane; i - lane < total; i += blockDim.x) {
                if (i >= total) continue;
                const uint32_t it = items[i];
                const int pp = (int)(it & 2047u);
                const int dx = (int)((it >> 11) & 1023u) - R, dy = (int)(it >> 21) - R;
                const int gx = tx0 + (pp & (TX - 1)), gy = ty0 + (pp >> lgTX);
                const int a0 = (gy - wy0) * WW + (gx - wx0);
                const int E = (int)win[a0] + P.ht;
                const int adx = abs(dx), ady = abs(dy);
                const bool xmaj = adx >= ady;
                const int D = xmaj ? adx : ady;
                const int dmin = xmaj ? dy : dx;
                const int ms = xmaj ? (dx > 0 ? 1 : -1) : (dy > 0 ? WW : -WW);
                const int ns = xmaj ? WW : 1;
                const int q = floordiv(dmin, D);
                const int r = dmin - q * D;
                const int step = ms + q * ns;
                const int tsl = (int)win[a0 + dx + dy * WW] + P.hr - E;
                const int16_t *w1 = win + ns;
                // blocked at crossing j iff z0*(D-f) + z1*f > E*D + tsl*j
                int a = a0, f = 0, thr = E * D;
                bool vis = true;
                int done = 0;
                const int nstep = D - 1;
                if (nstep & 1) {
                    f += r; a += step; thr += tsl;
                    if (f >= D) { f -= D; a += ns; }
                    vis = (int)win[a] * (D - f) + (int)w1[a] * f <= thr;
                    done = 1;
                }
                for (int k = nstep >> 1; vis && k > 0; --k) {
                    f += r; a += step; thr += tsl;
                    if (f >= D) { f -= D; a += ns; }
                    const int v1 = (int)win[a] * (D - f) + (int)w1[a] * f;
                    const int t1 = thr;
                    f += r; a += step; thr += tsl;
                    if (f >= D) { f -= D; a += ns; }
                    const int v2 = (int)win[a] * (D - f) + (int)w1[a] * f;
                    if (COUNT) done += (v1 > t1) ? 1 : 2;
                    vis = (v1 <= t1) & (v2 <= thr);
                }
                if (COUNT) nsteps += done;
                if (vis) atomicAdd(&cnt[pp], 1);
            }
            __syncthreads();
        }
    }

    for (int pp = tid; pp < nposts; pp += blockDim.x) {
        const int gx = tx0 + (pp & (TX - 1)), gy = ty0 + (pp >> lgTX);
        if (gx >= P.W || gy >= P.H) continue;
        P.out[(size_t)gy * P.W + gx] = s_fail ? (uint8_t)0xFF : (uint8_t)cnt[pp];
    }
    if (COUNT) {
        for (int o = 16; o > 0; o >>= 1) nsteps += __shfl_xor_sync(0xffffffffu, nsteps, o);
        if (lane == 0 && nsteps) atomicAdd(P.steps, nsteps);
    }
    const bool dead = s_fail == 2;
    __syncthreads();  // shared memory is reused by the CTA's next tile
    return dead;
}

template <bool COUNT>
__global__ void __launch_bounds__(kVixThreads, 1) k_vix2(const __grid_constant__ CUtensorMap tmap,
                                                         const Vix2Params Q) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    __shared__ uint64_t bar;
    __shared__ int warp_tot[32];
    __shared__ int s_fail;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    uint32_t phase = 0;
    vix2_tile<COUNT>(&tmap, Q, blockIdx.x * Q.b.TX, blockIdx.y * Q.b.TY, smem, &bar, phase, warp_tot, &s_fail);
}

// Batched vix of many terrains in one persistent launch: items (job, tile)
// are numbered job by job (jobs ordered by decreasing R, so the costly ones
// start first) and pulled from a global counter; each job's TMA descriptor
// and parameters sit in the launch's parameters.
constexpr int kVixMaxJobs = 64;
struct Vix2Job {
    CUtensorMap map;
    Vix2Params Q;
    int tiles_x;
    long long item0;
};
struct Vix2Batch {
    Vix2Job job[kVixMaxJobs];
    int njobs;
    long long total;
    unsigned long long *counter;
};
__global__ void __launch_bounds__(kVixThreads, 1) k_vix2_batch(const __grid_constant__ Vix2Batch B) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    __shared__ uint64_t bar;
    __shared__ int warp_tot[32];
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
        const Vix2Job &J = B.job[j];
        const long long t = it - J.item0;
        const int tx = (int)(t % J.tiles_x), ty = (int)(t / J.tiles_x);
        if (vix2_tile<false>(&J.map, J.Q, tx * J.Q.b.TX, ty * J.Q.b.TY, smem, &bar, phase, warp_tot, &s_fail))
            break;  // a copy may still land in this CTA's window: take no more items
    }
}


// ------------------------------------------------------------------ wide ROI
// For ROIs whose halo window does not fit in shared memory (R above ~280; the
// paper's own runs use R = 500 .. 2000), a warp walks one line of sight at a
// time, 32 consecutive crossings per instruction (lane l takes crossing
// j0 + l), against the terrain in global memory, and a warp vote ends the
// line at its first blocked crossing.  With a workspace the walk reads both
// posts of a crossing with one load from pair arrays laid out so that a
// warp's loads are contiguous (warp_los_pair); without one, x-major lines
// read terrain rows and y-major lines the terrain with a row stride.  Each lane
// draws the samples of its own post (the same generator and offset table as
// k_vix); the warp then walks its 32 posts' lines one after another.  The
// test is k_vix's: visible iff j*(z_T + hr - E) >= (z0 - E)*D + (z1 - z0)*f
// at every crossing j = 1 .. D-1, in 32-bit integers.
struct VixWide {
    const int16_t *z;
    long long pitch;
    const uint32_t *py, *px;  // pair arrays of warp_los_pair, or null
    int H, W, R, ht, hr, S, NR;
    uint64_t seed;
    uint8_t *out;
    unsigned long long *steps;
};

// row table of OFF_R (rows dy = -R..R, dx ascending, origin removed):
// hwtab[i] = half-width of row dy = i - R, rowstart[i] = entries before it
__device__ void vix_tables(int R, int *rowstart, int *hwtab, int *warp_tot) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nt = blockDim.x;
    const int nrow = 2 * R + 1;
    const int chunk = (nrow + nt - 1) / nt;
    const int i0 = tid * chunk, i1 = min(nrow, i0 + chunk);
    int local = 0;
    for (int i = i0; i < i1; ++i) {
        const int dy = i - R;
        const int hw = isqrt_exact(R * R - dy * dy);
        hwtab[i] = hw;
        local += 2 * hw + 1 - (dy == 0 ? 1 : 0);
    }
    int incl = local;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int t = lane < (nt >> 5) ? warp_tot[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += v;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    int run = incl - local + (wid > 0 ? warp_tot[wid - 1] : 0);
    if (tid == 0) rowstart[0] = 0;
    for (int i = i0; i < i1; ++i) {
        run += 2 * hwtab[i] + 1 - (i == R ? 1 : 0);
        rowstart[i + 1] = run;
    }
    __syncthreads();
}

// One line of sight from post (ox, oy) with eye E to the post (ox+dx, oy+dy),
// walked by the whole warp: lane l takes crossings j0 + l, two chunks of 32
// per trip (the second chunk's loads in flight before the first chunk's vote).
// ts = z_T + hr - E.  Visible iff j*ts >= (z0 - E)*D + (z1 - z0)*f at every
// crossing j = 1 .. D-1 (Sec. "Terrain visibility": the LOS against the
// terrain interpolated linearly between the two posts it passes between).
// x-major lines read terrain rows, y-major lines the transposed terrain when
// given (else the terrain with a row stride).  Every lane returns the same
// result; with COUNT, nsteps grows by the crossings evaluated (the first
// blocked one, else D - 1), identically in every lane.
template <bool COUNT>
__device__ __forceinline__ bool warp_los(const int16_t *z, long long pitch, const int16_t *zt, long long pitcht,
                                         int ox, int oy, int E, int dx, int dy, int ts,
                                         unsigned long long &nsteps) {
    const int lane = threadIdx.x & 31;
    const int adx = abs(dx), ady = abs(dy);
    const bool xmaj = adx >= ady;
    const int D = xmaj ? adx : ady;
    const int dmin = xmaj ? dy : dx;
    const int sg = xmaj ? (dx > 0 ? 1 : -1) : (dy > 0 ? 1 : -1);
    // strides along the major (ms) and minor (ns) axes of the array read
    const int16_t *bp;
    int ms, ns;
    if (xmaj) { bp = z + (long long)oy * pitch + ox; ms = 1; ns = (int)pitch; }
    else if (zt) { bp = zt + (long long)ox * pitcht + oy; ms = 1; ns = (int)pitcht; }
    else { bp = z + (long long)oy * pitch + ox; ms = (int)pitch; ns = 1; }
    // this lane's first crossing j = 1 + lane
    int j = 1 + lane;
    const int yq = floordiv(j * dmin, D);
    int f = j * dmin - yq * D;
    int off = j * sg * ms + yq * ns;
    const int q32 = floordiv(32 * dmin, D), r32 = 32 * dmin - q32 * D;
    const int step32 = 32 * sg * ms + q32 * ns;
    int lhs = j * ts;
    for (int j0 = 1; j0 < D; j0 += 64) {
        int fb = f + r32, offb = off + step32;
        if (fb >= D) { fb -= D; offb += ns; }
        int z0a = 0, z1a = 0, z0b = 0, z1b = 0;
        if (j < D) {
            z0a = __ldg(bp + off);
            z1a = f ? (int)__ldg(bp + off + ns) : z0a;
        }
        if (j + 32 < D) {
            z0b = __ldg(bp + offb);
            z1b = fb ? (int)__ldg(bp + offb + ns) : z0b;
        }
        const bool ba = j < D && lhs < (z0a - E) * D + (z1a - z0a) * f;
        const bool bb = j + 32 < D && lhs + 32 * ts < (z0b - E) * D + (z1b - z0b) * fb;
        const unsigned va = __ballot_sync(0xffffffffu, ba);
        const unsigned vb = __ballot_sync(0xffffffffu, bb);
        if (va | vb) {
            if (COUNT) nsteps += (unsigned long long)(va ? j0 + __ffs(va) - 1 : j0 + 32 + __ffs(vb) - 1);
            return false;
        }
        j += 64;
        lhs += 64 * ts;
        off = offb + step32;
        f = fb + r32;
        if (f >= D) { f -= D; off += ns; }
    }
    if (COUNT && D > 1) nsteps += (unsigned long long)(D - 1);
    return true;
}

// The same line walk reading both posts of a crossing with one 32-bit load:
// Py[y*W + x] = z(x, y) | z(x, y+1) << 16 for x-major lines (consecutive
// crossings = consecutive x, so a warp's loads are contiguous) and
// Px[x*H + y] = z(x, y) | z(x+1, y) << 16, transposed, for y-major ones.  Half
// the loads and half the cache lines of warp_los (the walk is bound by L1
// traffic).  The upper half of a pair past the grid edge is never used: a
// crossing between two posts has both inside the line's bounding box.
template <bool COUNT>
__device__ __forceinline__ bool warp_los_pair(const uint32_t *Py, const uint32_t *Px, int H, int W, int ox, int oy,
                                              int E, int dx, int dy, int ts, unsigned long long &nsteps) {
    const int lane = threadIdx.x & 31;
    const int adx = abs(dx), ady = abs(dy);
    const bool xmaj = adx >= ady;
    const int D = xmaj ? adx : ady;
    const int dmin = xmaj ? dy : dx;
    const int sg = xmaj ? (dx > 0 ? 1 : -1) : (dy > 0 ? 1 : -1);
    // element (major m, minor n) of the pair array: x-major Py[n][m], y-major Px[m][n]
    const uint32_t *bp = xmaj ? Py + (long long)oy * W + ox : Px + (long long)ox * H + oy;
    const int ns = xmaj ? W : H;  // stride along the minor axis
    int j = 1 + lane;
    const int yq = floordiv(j * dmin, D);
    int f = j * dmin - yq * D;
    long long off = (long long)j * sg + (long long)yq * ns;
    const int q32 = floordiv(32 * dmin, D), r32 = 32 * dmin - q32 * D;
    const long long step32 = 32ll * sg + (long long)q32 * ns;
    int lhs = j * ts;
    for (int j0 = 1; j0 < D; j0 += 64) {
        int fb = f + r32;
        long long offb = off + step32;
        if (fb >= D) { fb -= D; offb += ns; }
        uint32_t pa = 0, pb = 0;
        if (j < D) pa = __ldg(bp + off);
        if (j + 32 < D) pb = __ldg(bp + offb);
        const int z0a = (int16_t)(pa & 0xFFFFu), z1a = f ? (int)(int16_t)(pa >> 16) : z0a;
        const int z0b = (int16_t)(pb & 0xFFFFu), z1b = fb ? (int)(int16_t)(pb >> 16) : z0b;
        const bool ba = j < D && lhs < (z0a - E) * D + (z1a - z0a) * f;
        const bool bb = j + 32 < D && lhs + 32 * ts < (z0b - E) * D + (z1b - z0b) * fb;
        const unsigned va = __ballot_sync(0xffffffffu, ba);
        const unsigned vb = __ballot_sync(0xffffffffu, bb);
        if (va | vb) {
            if (COUNT) nsteps += (unsigned long long)(va ? j0 + __ffs(va) - 1 : j0 + 32 + __ffs(vb) - 1);
            return false;
        }
        j += 64;
        lhs += 64 * ts;
        off = offb + step32;
        f = fb + r32;
        if (f >= D) { f -= D; off += ns; }
    }
    if (COUNT && D > 1) nsteps += (unsigned long long)(D - 1);
    return true;
}

// the pair arrays of warp_los_pair, one 32 x 32 block of posts per CTA: Py
// written row by row, Px through a shared-memory transpose (both coalesced)
__global__ void __launch_bounds__(256) k_pairs_i16(const int16_t *__restrict__ z, long long pitch, int H, int W,
                                                   uint32_t *__restrict__ Py, uint32_t *__restrict__ Px) {
    __shared__ uint32_t t[32][33];
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int j = ty; j < 32; j += 8) {
        const int y = y0 + j, x = x0 + tx;
        if (y < H && x < W) {
            const uint32_t z0 = (uint16_t)z[(long long)y * pitch + x];
            const uint32_t zy = y + 1 < H ? (uint16_t)z[(long long)(y + 1) * pitch + x] : 0u;
            const uint32_t zx = x + 1 < W ? (uint16_t)z[(long long)y * pitch + x + 1] : 0u;
            Py[(long long)y * W + x] = z0 | (zy << 16);
            t[j][tx] = z0 | (zx << 16);
        }
    }
    __syncthreads();
    for (int j = ty; j < 32; j += 8) {
        const int x = x0 + j, y = y0 + tx;
        if (x < W && y < H) Px[(long long)x * H + y] = t[tx][j];
    }
}

// 512 threads = 16 warps = a 32 x 16 tile of posts; three CTAs per SM (48 warps)
// to hide the cache latency of the line walks
constexpr int kVixWideThreads = 512;
constexpr int kVixStrip = 16;  // tiles per strip of the visiting order

template <bool COUNT>
__global__ void __launch_bounds__(kVixWideThreads, 3) k_vix_wide(const VixWide P) {
    extern __shared__ int vix_tab[];
    __shared__ int warp_tot[32];
    const int R = P.R;
    int *rowstart = vix_tab;            // 2R + 2 entries
    int *hwtab = vix_tab + 2 * R + 2;   // 2R + 1 entries
    vix_tables(R, rowstart, hwtab, warp_tot);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    // tiles visited in vertical strips of kVixStrip tiles, so that the CTAs
    // resident at a time cover a compact block of posts whose lines (and the
    // terrain around it) stay in L2, rather than a long band of rows
    const int ntx = (P.W + 31) / 32, nty = (P.H + kVixWideThreads / 32 - 1) / (kVixWideThreads / 32);
    const int b = blockIdx.x, strip = b / (kVixStrip * nty);
    const int sw = min(kVixStrip, ntx - strip * kVixStrip), idx = b - strip * kVixStrip * nty;
    const int tyb = idx / sw, txb = strip * kVixStrip + (idx - tyb * sw);
    const int x0 = txb * 32, y = tyb * (kVixWideThreads / 32) + wid;
    const int x = x0 + lane;
    if (y >= P.H) return;  // whole warp: no block barrier follows
    const bool mine = x < P.W;
    const int16_t *zrow = P.z + (long long)y * P.pitch;
    const int E = mine ? (int)zrow[x] + P.ht : 0;
    const uint64_t GOLD = 0x9E3779B97F4A7C15ull;
    const uint64_t p = (uint64_t)y * (uint64_t)P.W + (uint64_t)x;
    uint64_t state = P.seed + GOLD * (p * (uint64_t)P.S + 1ull);
    int cnt = 0;
    unsigned long long nsteps = 0;
    for (int s = 0; s < P.S; ++s, state += GOLD) {
        int dx = 0, dy = 0, tsl = 0;
        bool valid = false;
        if (mine) {
            vix_offset(state, (unsigned)P.NR, R, rowstart, hwtab, dx, dy);
            valid = (unsigned)(x + dx) < (unsigned)P.W && (unsigned)(y + dy) < (unsigned)P.H;
            if (valid) tsl = (int)__ldg(P.z + (long long)(y + dy) * P.pitch + (x + dx)) + P.hr - E;
        }
        unsigned todo = __ballot_sync(0xffffffffu, valid);
        unsigned visbits = 0;
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int ldx = __shfl_sync(0xffffffffu, dx, src), ldy = __shfl_sync(0xffffffffu, dy, src);
            const int lE = __shfl_sync(0xffffffffu, E, src), lts = __shfl_sync(0xffffffffu, tsl, src);
            const bool vis = P.py ? warp_los_pair<COUNT>(P.py, P.px, P.H, P.W, x0 + src, y, lE, ldx, ldy, lts, nsteps)
                                  : warp_los<COUNT>(P.z, P.pitch, nullptr, 0, x0 + src, y, lE, ldx, ldy, lts, nsteps);
            if (vis) visbits |= 1u << src;
        }
        cnt += (visbits >> lane) & 1u;
    }
    if (mine) P.out[(size_t)y * P.W + x] = (uint8_t)cnt;
    if (COUNT && lane == 0 && nsteps) atomicAdd(P.steps, nsteps);  // every lane counted the same lines
}

// ------------------------------------------------------------------ exact per-cell viewshed (R3)
// Every cell of the ROI disc inside the grid gets its own line of sight from
// the observer (warp_los: the vix test, target height z + hr) -- the viewshed
// as defined in Sec. "Definitions", of which the ray sweep of vs_viewshed
// (R2-style, Sec. "The multiple transmitter siting process", Viewshed) is an
// approximation.  CTA per candidate; a warp takes one bitmap word at a time --
// 32 cells of one row, one line each, walked by the whole warp in turn -- and
// the ballot of their results is the word.  Output layout as vs_viewshed.
struct VsR3 {
    const int16_t *z;
    long long pitch;
    const uint32_t *py, *px;  // pair arrays of warp_los_pair, or null
    int H, W, R, ht, hr, PR, words;
    const int64_t *cand;
    long long n;
    uint32_t *bm;
    int32_t *area;
};

constexpr int kR3Threads = 512;

__global__ void __launch_bounds__(kR3Threads) k_viewshed_r3(const VsR3 P) {
    __shared__ int red[32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    const long long c = blockIdx.x;
    const int R = P.R, PR = P.PR;
    const int64_t p = P.cand[c];
    uint32_t *out = P.bm + c * (long long)P.words;
    if (p < 0 || p >= (int64_t)P.H * P.W) {  // invalid candidate: empty bitmap, area -1
        for (int i = tid; i < P.words; i += blockDim.x) out[i] = 0u;
        if (tid == 0) P.area[c] = -1;
        return;
    }
    const int cx = (int)(p % P.W), cy = (int)(p / P.W);
    const int gw0 = floordiv(cx - R, 32);
    const int E = (int)P.z[(long long)cy * P.pitch + cx] + P.ht;
    int cnt = 0;
    unsigned long long unused = 0;
    for (int item = wid; item < P.words; item += nw) {
        const int r = item / PR, w = item - r * PR;
        const int dy = r - R, y = cy + dy;
        const int col = 32 * (gw0 + w) + lane, dx = col - cx;
        const bool in = (unsigned)y < (unsigned)P.H && (unsigned)col < (unsigned)P.W && dx * dx + dy * dy <= R * R;
        const bool self = dx == 0 && dy == 0;
        int ts = 0;
        if (in && !self) ts = (int)__ldg(P.z + (long long)y * P.pitch + col) + P.hr - E;
        unsigned todo = __ballot_sync(0xffffffffu, in && !self);
        unsigned bits = __ballot_sync(0xffffffffu, in && self);  // the observer's own cell
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int ldx = __shfl_sync(0xffffffffu, dx, src), lts = __shfl_sync(0xffffffffu, ts, src);
            const bool v = P.py ? warp_los_pair<false>(P.py, P.px, P.H, P.W, cx, cy, E, ldx, dy, lts, unused)
                                : warp_los<false>(P.z, P.pitch, nullptr, 0, cx, cy, E, ldx, dy, lts, unused);
            if (v) bits |= 1u << src;
        }
        if (lane == 0) {
            out[item] = bits;
            cnt += __popc(bits);
        }
    }
    if (lane == 0) red[wid] = cnt;
    __syncthreads();
    if (tid == 0) {
        int a = 0;
        for (int i = 0; i < nw; ++i) a += red[i];
        P.area[c] = a;
    }
}

static size_t vix2_smem_bytes(int R, int nsplit, int TX, int TY, int sb, int *WG, int *box_rows,
                              int *nbox) {
    // one spare row below and column to the right: the second straddling post
    // of a crossing is read even when its weight is zero
    const int rows = ((nsplit == 1) ? TY + 2 * R : TY + R) + 1;
    const int cols = ((nsplit == 4) ? TX + R : TX + 2 * R) + 1;
    const int wg = (cols + 7 + 7) / 8;
    int nb = (rows + 255) / 256;
    int br = ((rows + nb - 1) / nb + 7) / 8 * 8;
    if (br > 256) { nb += 1; br = ((rows + nb - 1) / nb + 7) / 8 * 8; }
    *WG = wg; *box_rows = br; *nbox = nb;
    size_t win = ((size_t)nb * br * wg * 8 * 2 + 127) & ~(size_t)127;
    return win + (size_t)TX * TY * sb * 4 + (size_t)TX * TY * 4 + (size_t)((R + 2 + 3) & ~3) * 4 +
           (size_t)(2 * R + 2) * 4 + (size_t)(2 * R + 2) * 4 + 16 + 128;
}

static size_t vix_smem_bytes(int R, int nsplit, int TX, int TY, int *WG, int *box_rows,
                             int *nbox) {
    const int rows = (nsplit == 1) ? TY + 2 * R : TY + R;
    const int cols = (nsplit == 4) ? TX + R : TX + 2 * R;
    const int wg = (cols + 7 + 7) / 8;
    int nb = (rows + 255) / 256;
    int br = ((rows + nb - 1) / nb + 7) / 8 * 8;
    if (br > 256) { nb += 1; br = ((rows + nb - 1) / nb + 7) / 8 * 8; }
    *WG = wg; *box_rows = br; *nbox = nb;
    size_t win = ((size_t)nb * br * wg * 8 * 2 + 127) & ~(size_t)127;
    return win + (size_t)(2 * R + 2) * 4 + (size_t)(2 * R + 2) * 4 + 16 + 128;
}

}  // namespace vs

using namespace vs;

// the staged kernels cover R when one of their windows fits in shared memory
static bool vix_staged_fits(int R, int S) {
    const int sb = std::max(std::min(S, kVixSB), 1);
    int WG, br, nb;
    for (int ns : {1, 2, 4})
        for (int t : {64, 32}) {
            if (R <= 511) {
                const size_t b = vix2_smem_bytes(R, ns, t, 32, sb, &WG, &br, &nb);
                if (WG <= 256 && b <= (size_t)225 * 1024) return true;
            }
            const size_t b = vix_smem_bytes(R, ns, t, 32, &WG, &br, &nb);
            if (WG <= 256 && b <= (size_t)225 * 1024) return true;
        }
    return false;
}

static bool vix_wide(int R, int S) {
    return tune_get(VS_TUNE_VIX_TILE, R, 0) == 3 || !vix_staged_fits(R, S);
}

// the two pair arrays of warp_los_pair: 4 bytes per post each
static size_t pairs_bytes(int H, int W) { return (size_t)H * (size_t)W * 8 + 512; }

// build the pair arrays in the workspace when it is large enough
static bool pairs_make(const vs_grid &g, void *ws, size_t ws_bytes, cudaStream_t s, uint32_t **py, uint32_t **px) {
    *py = *px = nullptr;
    if (!ws || ws_bytes < pairs_bytes(g.H, g.W)) return true;
    uint32_t *a = (uint32_t *)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    uint32_t *b = (uint32_t *)(((uintptr_t)(a + (size_t)g.H * g.W) + 255) & ~(uintptr_t)255);
    const dim3 tg((unsigned)((g.W + 31) / 32), (unsigned)((g.H + 31) / 32));
    k_pairs_i16<<<tg, 256, 0, s>>>(g.z, g.pitch, g.H, g.W, a, b);
    vs::note_launch();
    if (cudaGetLastError() != cudaSuccess) return false;
    *py = a;
    *px = b;
    return true;
}

static int vix_launch_wide(const vs_grid &g, int32_t R, int32_t ht, int32_t hr, int32_t S, uint64_t seed,
                           uint8_t *vix_out, unsigned long long *steps, void *ws, size_t ws_bytes,
                           cudaStream_t s, int NR) {
    uint32_t *py, *px;
    // without the pair arrays, offsets along a line (up to crossing D + 95,
    // D <= 1.42 R) in the plain layout are 32-bit
    if ((!ws || ws_bytes < pairs_bytes(g.H, g.W)) && (long long)(3 * R + 128) * g.pitch >= (1ll << 31))
        return VS_ERR_RANGE;
    if (!pairs_make(g, ws, ws_bytes, s, &py, &px)) return VS_ERR_CUDA;
    VixWide P;
    P.z = g.z; P.pitch = g.pitch; P.py = py; P.px = px;
    P.H = g.H; P.W = g.W; P.R = R; P.ht = ht; P.hr = hr; P.S = S; P.NR = NR;
    P.seed = seed; P.out = vix_out; P.steps = steps;
    const size_t smem = (size_t)(4 * R + 3) * 4;
    const int rows = kVixWideThreads / 32;
    const dim3 grid((unsigned)(((g.W + 31) / 32) * ((g.H + rows - 1) / rows)));  // one tile per CTA
    if (steps) {
        VS_CUDA_TRY(cudaFuncSetAttribute(k_vix_wide<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_vix_wide<true><<<grid, kVixWideThreads, smem, s>>>(P);
        vs::note_launch();
    } else {
        VS_CUDA_TRY(cudaFuncSetAttribute(k_vix_wide<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_vix_wide<false><<<grid, kVixWideThreads, smem, s>>>(P);
        vs::note_launch();
    }
    VS_CUDA_TRY(cudaGetLastError());
    return VS_OK;
}

// the parameters common to the vix kernels; NR = |disc(R)| - 1
static void vix_params(const vs_grid &g, int32_t R, int32_t ht, int32_t hr, int32_t S, uint64_t seed,
                       uint8_t *vix_out, VixParams *P) {
    memset(P, 0, sizeof(*P));
    P->H = g.H; P->W = g.W; P->R = R; P->ht = ht; P->hr = hr; P->S = S; P->seed = seed; P->out = vix_out;
    long long nr = 0;
    for (int dy = -R; dy <= R; ++dy) {
        long long v = (long long)R * R - (long long)dy * dy, s = (long long)std::sqrt((double)v);
        while (s * s > v) --s;
        while ((s + 1) * (s + 1) <= v) ++s;
        nr += 2 * s + 1;
    }
    P->NR = (int)(nr - 1);
}

// tile, passes and sample batch of the length-sorted kernel for P's R and S:
// the largest tile whose staged window fits, fewest passes first; false when
// none fits in shared memory
static bool vix2_pick(const VixParams &P, unsigned long long *steps, Vix2Params *Q, size_t *smem) {
    const int R = P.R;
    const int pref = tune_get(VS_TUNE_VIX_TILE, R, 0);
    const int tiles2[2][2] = {{pref == 2 ? 32 : 64, 32}, {32, 32}};
    const int sb = std::min(P.S, kVixSB);
    for (int ns : {1, 2, 4}) {
        for (auto &t : tiles2) {
            int WG, br, nb;
            const size_t b = vix2_smem_bytes(R, ns, t[0], t[1], std::max(sb, 1), &WG, &br, &nb);
            if (WG > 256 || b > (size_t)225 * 1024) continue;
            Q->b = P;
            Q->b.nsplit = ns; Q->b.TX = t[0]; Q->b.TY = t[1]; Q->b.WG = WG; Q->b.box_rows = br;
            Q->b.nbox = nb; Q->b.steps = steps;
            Q->lgTX = (t[0] == 64) ? 6 : 5;
            Q->sb = std::max(sb, 1);
            *smem = b;
            return true;
        }
    }
    return false;
}

static int vix_launch(vs_grid g, int32_t R, int32_t ht, int32_t hr, int32_t S, uint64_t seed,
                      uint8_t *vix_out, unsigned long long *steps, void *ws, size_t ws_bytes,
                      vs_stream_t st) {
    int rc = check_grid(g);
    if (rc) return rc;
    if (!vix_out) return VS_ERR_ARG;
    if (R < 1 || R > kMaxR || S < 0 || S > 255) return VS_ERR_RANGE;
    if (ht < -100000 || ht > 100000 || hr < -100000 || hr > 100000) return VS_ERR_RANGE;
    if ((rc = check_device())) return rc;

    VixParams P;
    vix_params(g, R, ht, hr, S, seed, vix_out, &P);

    if (vix_wide(R, S))
        return vix_launch_wide(g, R, ht, hr, S, seed, vix_out, steps, ws, ws_bytes, (cudaStream_t)st, P.NR);

    // length-sorted variant when the packed line items can describe R
    Vix2Params Q;
    size_t b = 0;
    if (R <= 511 && vix2_pick(P, steps, &Q, &b)) {
        GridMap gm;
        if ((rc = make_grid_map(&gm, g, Q.b.WG, Q.b.box_rows))) return rc;
        dim3 grid((g.W + Q.b.TX - 1) / Q.b.TX, (g.H + Q.b.TY - 1) / Q.b.TY);
        if (steps) {
            VS_CUDA_TRY(cudaFuncSetAttribute(k_vix2<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b));
            k_vix2<true><<<grid, kVixThreads, b, (cudaStream_t)st>>>(gm.map, Q);
            vs::note_launch();
        } else {
            VS_CUDA_TRY(cudaFuncSetAttribute(k_vix2<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b));
            k_vix2<false><<<grid, kVixThreads, b, (cudaStream_t)st>>>(gm.map, Q);
            vs::note_launch();
        }
        VS_CUDA_TRY(cudaGetLastError());
        return VS_OK;
    }

    // tile / split choice: the largest tile whose staged window fits, fewest
    // passes first (each pass re-draws the samples and re-stages a window)
    size_t smem = 0;
    bool found = false;
    const int tiles[2][2] = {{64, 32}, {32, 32}};
    for (int ns : {1, 2, 4}) {
        for (auto &t : tiles) {
            int WG, br, nb;
            size_t b = vix_smem_bytes(R, ns, t[0], t[1], &WG, &br, &nb);
            if (WG <= 256 && b <= (size_t)225 * 1024) {
                P.nsplit = ns; P.TX = t[0]; P.TY = t[1]; P.WG = WG; P.box_rows = br;
                P.nbox = nb; smem = b; found = true;
                break;
            }
        }
        if (found) break;
    }
    if (!found) return VS_ERR_RANGE;
    GridMap gm;
    if ((rc = make_grid_map(&gm, g, P.WG, P.box_rows))) return rc;
    P.steps = steps;
    dim3 grid((g.W + P.TX - 1) / P.TX, (g.H + P.TY - 1) / P.TY);
    if (steps) {
        VS_CUDA_TRY(cudaFuncSetAttribute(k_vix<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_vix<true><<<grid, kVixThreads, smem, (cudaStream_t)st>>>(gm.map, P);
        vs::note_launch();
    } else {
        VS_CUDA_TRY(cudaFuncSetAttribute(k_vix<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_vix<false><<<grid, kVixThreads, smem, (cudaStream_t)st>>>(gm.map, P);
        vs::note_launch();
    }
    VS_CUDA_TRY(cudaGetLastError());
    return VS_OK;
}

extern "C" int vs_vix(vs_grid g, int32_t R, int32_t ht, int32_t hr, int32_t S, uint64_t seed,
                      uint8_t *vix_out, vs_stream_t st) {
    return vix_launch(g, R, ht, hr, S, seed, vix_out, nullptr, nullptr, 0, st);
}

extern "C" int vs_vix_count(vs_grid g, int32_t R, int32_t ht, int32_t hr, int32_t S, uint64_t seed,
                            uint8_t *vix_out, uint64_t *los_steps, vs_stream_t st) {
    if (!los_steps) return VS_ERR_ARG;
    return vix_launch(g, R, ht, hr, S, seed, vix_out, (unsigned long long *)los_steps, nullptr, 0, st);
}

extern "C" size_t vs_vix_workspace(int32_t H, int32_t W, int32_t R, int32_t S) {
    if (H < 1 || W < 1 || H > kMaxH || W > kMaxH || R < 1 || R > kMaxR || S < 0 || S > 255) return 0;
    if (!vix_wide(R, S)) return 0;
    return pairs_bytes(H, W);
}

extern "C" int vs_vix_ws(vs_grid g, int32_t R, int32_t ht, int32_t hr, int32_t S, uint64_t seed,
                         uint8_t *vix_out, uint64_t *los_steps, void *ws, size_t ws_bytes, vs_stream_t st) {
    return vix_launch(g, R, ht, hr, S, seed, vix_out, (unsigned long long *)los_steps, ws, ws_bytes, st);
}

extern "C" size_t vs_viewshed_r3_workspace(int32_t H, int32_t W) {
    if (H < 1 || W < 1 || H > kMaxH || W > kMaxH) return 0;
    return pairs_bytes(H, W);
}

extern "C" int vs_viewshed_r3(vs_grid g, int32_t R, int32_t ht, int32_t hr, const int64_t *cand, int64_t n,
                              uint32_t *bm_out, int32_t *area_out, void *ws, size_t ws_bytes, vs_stream_t st) {
    int rc = check_grid(g);
    if (rc) return rc;
    if (R < 1 || R > kMaxR) return VS_ERR_RANGE;
    if (ht < -100000 || ht > 100000 || hr < -100000 || hr > 100000) return VS_ERR_RANGE;
    if (n < 0 || n > 0x7fffffffll) return VS_ERR_RANGE;
    if (n > 0 && (!cand || !bm_out || !area_out)) return VS_ERR_ARG;
    const bool pairs = ws && ws_bytes >= pairs_bytes(g.H, g.W);
    if (!pairs && (long long)(3 * R + 128) * g.pitch >= (1ll << 31)) return VS_ERR_RANGE;
    if (n == 0) return VS_OK;
    if ((rc = check_device())) return rc;
    cudaStream_t s = (cudaStream_t)st;
    VsR3 P;
    P.z = g.z; P.pitch = g.pitch; P.py = nullptr; P.px = nullptr;
    P.H = g.H; P.W = g.W; P.R = R; P.ht = ht; P.hr = hr;
    P.PR = (2 * R) / 32 + 2;
    P.words = (2 * R + 1) * P.PR;
    P.cand = cand; P.n = n; P.bm = bm_out; P.area = area_out;
    if (pairs) {
        uint32_t *py, *px;
        if (!pairs_make(g, ws, ws_bytes, s, &py, &px) || !py) return VS_ERR_CUDA;
        P.py = py;
        P.px = px;
    }
    k_viewshed_r3<<<(unsigned)n, kR3Threads, 0, s>>>(P);
    vs::note_launch();
    VS_CUDA_TRY(cudaGetLastError());
    return VS_OK;
}

extern "C" size_t vs_vix_batch_workspace(int32_t n_jobs) {
    (void)n_jobs;
    return 256;
}

extern "C" int vs_vix_batch(const vs_vix_job *jobs, int32_t n_jobs, void *ws, size_t ws_bytes, vs_stream_t st) {
    if (n_jobs < 0 || n_jobs > kVixMaxJobs) return VS_ERR_RANGE;
    if (n_jobs == 0) return VS_OK;
    if (!jobs) return VS_ERR_ARG;
    if (!ws || ws_bytes < vs_vix_batch_workspace(n_jobs)) return VS_ERR_WS;
    int rc = check_device();
    if (rc) return rc;
    // largest ROI first: the longest items start early, the short ones fill the tail
    int order[kVixMaxJobs];
    for (int i = 0; i < n_jobs; ++i) order[i] = i;
    std::stable_sort(order, order + n_jobs, [&](int a, int b) { return jobs[a].R > jobs[b].R; });
    static Vix2Batch B;  // large: built on the host, copied into the launch's parameters
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    memset(&B, 0, sizeof(B));
    size_t smem = 0;
    long long total = 0;
    int nj = 0;
    for (int i = 0; i < n_jobs; ++i) {
        const vs_vix_job &q = jobs[order[i]];
        if ((rc = check_grid(q.g))) return rc;
        if (!q.vix_out) return VS_ERR_ARG;
        if (q.R < 1 || q.R > 511 || q.S < 0 || q.S > 255) return VS_ERR_RANGE;
        if (q.ht < -100000 || q.ht > 100000 || q.hr < -100000 || q.hr > 100000) return VS_ERR_RANGE;
        VixParams P;
        vix_params(q.g, q.R, q.ht, q.hr, q.S, q.seed, q.vix_out, &P);
        Vix2Job &J = B.job[nj];
        size_t b = 0;
        if (!vix2_pick(P, nullptr, &J.Q, &b)) return VS_ERR_RANGE;  // window beyond shared memory
        GridMap gm;
        if ((rc = make_grid_map(&gm, q.g, J.Q.b.WG, J.Q.b.box_rows))) return rc;
        J.map = gm.map;
        J.tiles_x = (q.g.W + J.Q.b.TX - 1) / J.Q.b.TX;
        const long long tiles = (long long)J.tiles_x * ((q.g.H + J.Q.b.TY - 1) / J.Q.b.TY);
        J.item0 = total;
        total += tiles;
        smem = std::max(smem, b);
        ++nj;
    }
    B.njobs = nj;
    B.total = total;
    B.counter = (unsigned long long *)ws;
    cudaStream_t s = (cudaStream_t)st;
    VS_CUDA_TRY(cudaMemsetAsync(ws, 0, 8, s));
    VS_CUDA_TRY(cudaFuncSetAttribute(k_vix2_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, sms = 0, per = 0;
    VS_CUDA_TRY(cudaGetDevice(&dev));
    VS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    VS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_vix2_batch, kVixThreads, smem));
    const long long grid = std::min<long long>(total, (long long)sms * std::max(per, 1));
    k_vix2_batch<<<(unsigned)grid, kVixThreads, smem, s>>>(B);
    vs::note_launch();
    VS_CUDA_TRY(cudaGetLastError());
    return VS_OK;
}
