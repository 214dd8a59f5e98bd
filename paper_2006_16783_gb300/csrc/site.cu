// site.cu -- Site stage (Sec. "The multiple transmitter siting process",
// Site): greedy union of viewsheds with AND-NOT / popcount gains and OR
// updates of the cumulative viewshed.
//
// 1. k_site_gains: one streaming pass over every bitmap computing
//    gain_c = popcount(V_c AND NOT C) (HBM bound).
// 2. k_site_loop: one persistent thread-block cluster runs all greedy steps.
//    Candidate c lives in CTA (c mod Q), slot c / Q, of the cluster's shared
//    memory (gain, post index, packed x/y).  Each step:
//      a. every CTA reduces its slots to the key (gain << 32 | ~p) -- largest
//         gain, then lowest post index -- and writes it into every CTA's
//         shared memory (DSMEM); cluster barrier; all CTAs reduce the Q keys;
//      b. the CTA owning absolute row y (y mod Q) ORs the winner's row into C
//         and broadcasts delta = V_win AND NOT C_old for that row to every
//         CTA; cluster barrier;
//      c. each CTA lowers the gain of its candidates whose window overlaps the
//         winner's by popcount(V_c AND delta) over the overlap.  This is exact:
//         gain_c(C | V_win) = gain_c(C) - popcount(V_c AND delta).
//    Only candidates within Chebyshev distance 2R of the winner can change,
//    which is the paper's observation that old gains stay valid upper bounds,
//    applied exactly.
#include <algorithm>
#include <cooperative_groups.h>
#include <cstring>
#include <mutex>

#include "vs_common.cuh"

namespace cg = cooperative_groups;

namespace vs {

constexpr int kSiteThreads = 1024;
constexpr int kGainThreads = 256;

// ------------------------------------------------------------------ dense gain pass
// one warp computes candidate c's gain
__device__ __forceinline__ void site_gain_warp(const uint32_t *__restrict__ bm, const int64_t *__restrict__ cand,
                                               int64_t n, int H, int W, int R, const uint32_t *__restrict__ cum,
                                               uint32_t *__restrict__ gains, int64_t c) {
    const int lane = threadIdx.x & 31;
    if (c >= n) return;
    const int64_t p = cand[c];
    if (p < 0 || p >= (int64_t)H * W) {
        if (lane == 0) gains[c] = 0;
        return;
    }
    const int PR = words_per_row(R), WWc = (W + 31) >> 5;
    const int cx = (int)(p % W), cy = (int)(p / W);
    const int gw0 = floordiv(cx - R, 32);
    const uint32_t *V = bm + c * (int64_t)(2 * R + 1) * PR;
    unsigned sum = 0;
    const int words = (2 * R + 1) * PR;
    if ((PR & 3) == 0 && (((uintptr_t)V) & 15) == 0) {
        // rows of whole 16-byte vectors: a lane reads 4 words of one row per
        // load, four vectors in flight; the C words beside them one by one
        const int q4 = PR >> 2, nvec = words >> 2;
        const uint4 *V4 = (const uint4 *)V;
#pragma unroll 4
        for (int i = lane; i < nvec; i += 32) {
            const uint4 v = __ldg(V4 + i);
            const int r = i / q4, w = 4 * (i - r * q4);
            const int y = cy - R + r;
            if (y < 0 || y >= H) continue;
            const uint32_t *Cr = cum + (int64_t)y * WWc + gw0 + w;
            const int g = gw0 + w;
            const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (g + j >= 0 && g + j < WWc) sum += __popc(vv[j] & ~__ldg(Cr + j));
        }
    } else if (PR <= 32) {
        // lanes cover rpi whole rows per iteration
        const int rpi = 32 / PR;
        const int roff = lane / PR, w = lane - roff * PR;
        const int gw = gw0 + w;
        const bool col_ok = lane < rpi * PR && gw >= 0 && gw < WWc;
        const int nrow = 2 * R + 1;
#pragma unroll 4
        for (int r = roff; r < nrow; r += rpi) {
            if (lane >= rpi * PR) break;
            const int y = cy - R + r;
            uint32_t v = __ldg(V + r * PR + w);
            if (col_ok && y >= 0 && y < H) v &= ~__ldg(cum + (int64_t)y * WWc + gw);
            else v = 0;
            sum += __popc(v);
        }
    } else {
        for (int r = 0; r < 2 * R + 1; ++r) {
            const int y = cy - R + r;
            if (y < 0 || y >= H) continue;
            for (int w = lane; w < PR; w += 32) {
                const int gw = gw0 + w;
                if (gw < 0 || gw >= WWc) continue;
                sum += __popc(V[r * PR + w] & ~cum[(int64_t)y * WWc + gw]);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) gains[c] = sum;
}

__global__ void __launch_bounds__(kGainThreads) k_site_gains(const uint32_t *__restrict__ bm,
                                                             const int64_t *__restrict__ cand,
                                                             int64_t n, int H, int W, int R,
                                                             const uint32_t *__restrict__ cum,
                                                             uint32_t *__restrict__ gains) {
    site_gain_warp(bm, cand, n, H, W, R, cum, gains,
                   (int64_t)blockIdx.x * (kGainThreads / 32) + (threadIdx.x >> 5));
}

__global__ void k_cum_popcount(const uint32_t *__restrict__ cum, int64_t nwords,
                               unsigned long long *out) {
    unsigned long long s = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nwords;
         i += (int64_t)gridDim.x * blockDim.x)
        s += __popc(cum[i]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

// ------------------------------------------------------------------ greedy loop
struct SiteParams {
    const uint32_t *bm;
    const int64_t *cand;
    int64_t n;
    int H, W, R, PR, words, WWc;
    int n_obs;
    long long need;  // coverage threshold, -1 = off
    int64_t *chosen, *gains;
    uint32_t *cum;
    int32_t *n_chosen;
    const uint32_t *gain0;
    const unsigned long long *covered0;
    int slots;  // slots per CTA
};

struct KeyIdx {
    uint64_t key;
    int c;
};

__device__ __forceinline__ bool ki_better(uint64_t ka, int ca, uint64_t kb, int cb) {
    return ka > kb || (ka == kb && ca < cb);
}

__global__ void __launch_bounds__(kSiteThreads, 1) k_site_loop(const SiteParams P) {
    cg::cluster_group cl = cg::this_cluster();
    const int Q = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int R = P.R, PR = P.PR, W = P.W, H = P.H, WWc = P.WWc;

    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *s_gain = (uint32_t *)smem;
    uint32_t *s_p = s_gain + P.slots;
    uint32_t *s_xy = s_p + P.slots;
    int *s_list = (int *)(s_xy + P.slots);
    uint32_t *s_delta = (uint32_t *)(s_list + P.slots);
    __shared__ uint64_t s_keys[16];
    __shared__ int s_kc[16];
    __shared__ uint64_t s_rk[32];
    __shared__ int s_rc[32];
    __shared__ int s_nlist;

    for (int i = tid; i < P.slots; i += blockDim.x) {
        const int64_t c = rank + (int64_t)i * Q;
        uint32_t g = 0, pp = 0, xy = 0;
        if (c < P.n) {
            const int64_t p = P.cand[c];
            if (p >= 0 && p < (int64_t)H * W) {
                g = P.gain0[c];
                pp = (uint32_t)p;
                xy = (uint32_t)(p % W) | ((uint32_t)(p / W) << 16);
            }
        }
        s_gain[i] = g;
        s_p[i] = pp;
        s_xy[i] = xy;
    }
    long long covered = (P.need >= 0) ? (long long)*P.covered0 : 0;
    cl.sync();

    int t = 0;
    for (; t < P.n_obs; ++t) {
        if (P.need >= 0 && covered >= P.need) break;
        // ---- a. local then cluster-wide argmax
        uint64_t bk = 0;
        int bc = 0x7fffffff;
        for (int i = tid; i < P.slots; i += blockDim.x) {
            const uint32_t g = s_gain[i];
            if (!g) continue;
            const uint64_t k = ((uint64_t)g << 32) | (uint64_t)(0xFFFFFFFFu - s_p[i]);
            const int c = rank + i * Q;
            if (ki_better(k, c, bk, bc)) { bk = k; bc = c; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const uint64_t k2 = __shfl_xor_sync(0xffffffffu, bk, o);
            const int c2 = __shfl_xor_sync(0xffffffffu, bc, o);
            if (ki_better(k2, c2, bk, bc)) { bk = k2; bc = c2; }
        }
        if (lane == 0) { s_rk[wid] = bk; s_rc[wid] = bc; }
        if (tid == 0) s_nlist = 0;
        __syncthreads();
        if (wid == 0) {
            bk = (lane < (int)(blockDim.x >> 5)) ? s_rk[lane] : 0;
            bc = (lane < (int)(blockDim.x >> 5)) ? s_rc[lane] : 0x7fffffff;
            for (int o = 16; o > 0; o >>= 1) {
                const uint64_t k2 = __shfl_xor_sync(0xffffffffu, bk, o);
                const int c2 = __shfl_xor_sync(0xffffffffu, bc, o);
                if (ki_better(k2, c2, bk, bc)) { bk = k2; bc = c2; }
            }
            if (lane < Q) {
                *cl.map_shared_rank(&s_keys[rank], lane) = bk;
                *cl.map_shared_rank(&s_kc[rank], lane) = bc;
            }
        }
        cl.sync();
        uint64_t gk = s_keys[0];
        int gc = s_kc[0];
        for (int q = 1; q < Q; ++q)
            if (ki_better(s_keys[q], s_kc[q], gk, gc)) { gk = s_keys[q]; gc = s_kc[q]; }
        const uint32_t g = (uint32_t)(gk >> 32);
        if (g == 0) break;
        const uint32_t wp = 0xFFFFFFFFu - (uint32_t)(gk & 0xFFFFFFFFu);
        if (rank == 0 && tid == 0) {
            P.chosen[t] = (int64_t)wp;
            P.gains[t] = (int64_t)g;
        }
        covered += g;
        const int wx = (int)(wp % (uint32_t)W), wy = (int)(wp / (uint32_t)W);
        const int wgw0 = floordiv(wx - R, 32);
        const uint32_t *Vw = P.bm + (int64_t)gc * P.words;

        // ---- b. rows of the winner window owned by this CTA: update C, broadcast delta
        const int nrow = 2 * R + 1;
        const int ylo = wy - R;
        int r0 = ((rank - ylo) % Q + Q) % Q;  // first window row with (ylo + r) mod Q == rank
        for (int e = tid; ; e += blockDim.x) {
            const int rr = e / PR, w = e - (e / PR) * PR;
            const int r = r0 + rr * Q;
            if (r >= nrow) break;
            const int y = ylo + r, gw = wgw0 + w;
            uint32_t d = 0;
            if (y >= 0 && y < H && gw >= 0 && gw < WWc) {
                const uint32_t v = __ldg(Vw + r * PR + w);
                if (v) {
                    uint32_t *cp = P.cum + (int64_t)y * WWc + gw;
                    const uint32_t old = *cp;
                    d = v & ~old;
                    if (d) *cp = old | v;
                }
            }
            for (int q = 0; q < Q; ++q) *cl.map_shared_rank(&s_delta[r * PR + w], q) = d;
        }
        cl.sync();

        // ---- c. lower the gains of overlapping candidates
        for (int i = tid; i < P.slots; i += blockDim.x) {
            if (!s_gain[i]) continue;
            const int cx = (int)(s_xy[i] & 0xFFFFu), cy = (int)(s_xy[i] >> 16);
            if (abs(cx - wx) <= 2 * R && abs(cy - wy) <= 2 * R) s_list[atomicAdd(&s_nlist, 1)] = i;
        }
        __syncthreads();
        const int nl = s_nlist;
        for (int l = wid; l < nl; l += (blockDim.x >> 5)) {
            const int i = s_list[l];
            const int cx = (int)(s_xy[i] & 0xFFFFu), cy = (int)(s_xy[i] >> 16);
            const int cgw0 = floordiv(cx - R, 32);
            const int ya = max(max(cy, wy) - R, 0), yb = min(min(cy, wy) + R, H - 1);
            const int ga = max(max(cgw0, wgw0), 0), gb = min(min(cgw0, wgw0) + PR - 1, WWc - 1);
            unsigned sum = 0;
            if (ya <= yb && ga <= gb) {
                const int nw = gb - ga + 1;
                const int tot = (yb - ya + 1) * nw;
                const uint32_t *Vc = P.bm + (int64_t)(rank + (int64_t)i * Q) * P.words;
                for (int e = lane; e < tot; e += 32) {
                    const int dy = e / nw, gw = ga + (e - dy * nw);
                    const int y = ya + dy;
                    const uint32_t dl = s_delta[(y - wy + R) * PR + (gw - wgw0)];
                    if (dl) sum += __popc(__ldg(Vc + (y - cy + R) * PR + (gw - cgw0)) & dl);
                }
            }
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            if (lane == 0) s_gain[i] -= sum;
        }
        __syncthreads();
    }
    if (rank == 0 && tid == 0) *P.n_chosen = t;
    cl.sync();  // no CTA leaves while another may still address its shared memory
}

// ------------------------------------------------------------------ single-CTA greedy loop
// For candidate counts whose gains fit in one CTA's shared memory.  Slots are
// the candidates sorted by post index, so "largest gain, then lowest post
// index" is "largest (gain, -slot)": the argmax needs no post indices.  Each
// thread owns a contiguous run of slots and caches its best key; only runs
// whose gains changed are rescanned.  Per greedy step there are three rounds
// of memory latency: the winner's metadata, then its bitmap / C window / the
// band of candidates within 2R rows, then the overlapping candidates' words.

// slot of every candidate: rank by (post index, candidate index); invalid
// posts sort last
// ---- slot order: candidates sorted by (post, candidate index); an invalid
// post sorts as 0xFFFFFFFF.  Keys (post << 32 | candidate) are sorted in
// chunks of 1024 in shared memory (bitonic network); a key's rank is its
// position in its chunk plus, for every other chunk, the number of smaller
// keys there (binary search); candidates are then scattered to their ranks.
constexpr int kRankChunk = 1024;

__device__ __forceinline__ uint64_t slot_key(const int64_t *cand, int64_t c, int64_t HW) {
    const int64_t p = cand[c];
    const uint32_t pc = (p >= 0 && p < HW) ? (uint32_t)p : 0xFFFFFFFFu;
    return ((uint64_t)pc << 32) | (uint64_t)(uint32_t)c;
}

// sorted chunks into keys[]; rank[c] = position of candidate c in its chunk
__device__ __forceinline__ void rank_chunk(const int64_t *__restrict__ cand, int64_t n, int64_t HW,
                                           uint64_t *__restrict__ keys, uint32_t *__restrict__ rank, int64_t blk,
                                           uint64_t *sk) {
    const int t = threadIdx.x;
    const int64_t c = blk * kRankChunk + t;
    sk[t] = (c < n) ? slot_key(cand, c, HW) : ~0ull;
    __syncthreads();
    for (int size = 2; size <= kRankChunk; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const int j = t ^ stride;
            if (j > t) {
                const uint64_t a = sk[t], b = sk[j];
                const bool up = (t & size) == 0;
                if ((a > b) == up) {
                    sk[t] = b;
                    sk[j] = a;
                }
            }
            __syncthreads();
        }
    if (c < n) {
        const uint64_t k = sk[t];  // padding (~0) sorts after every real key
        keys[blk * kRankChunk + t] = k;
        rank[(uint32_t)k] = (uint32_t)t;
    }
    __syncthreads();  // sk is reused by the CTA's next chunk
}

__global__ void __launch_bounds__(kRankChunk) k_rank_chunks(const int64_t *__restrict__ cand, int64_t n, int64_t HW,
                                                           uint64_t *__restrict__ keys, uint32_t *__restrict__ rank) {
    __shared__ uint64_t sk[kRankChunk];
    rank_chunk(cand, n, HW, keys, rank, blockIdx.x, sk);
}

// rank[c] += number of keys of chunk blockIdx.y below candidate c's key, for
// the keys of chunk blockIdx.x
__device__ __forceinline__ void rank_cross(const uint64_t *__restrict__ keys, int64_t n, uint32_t *__restrict__ rank,
                                           int64_t bx, int64_t by, uint64_t *sk) {
    if (bx == by) return;
    const int t = threadIdx.x;
    const int64_t b0 = by * kRankChunk, a0 = bx * kRankChunk;
    const int mb = (int)min((int64_t)kRankChunk, n - b0);
    if (t < mb) sk[t] = keys[b0 + t];
    __syncthreads();
    if (a0 + t < n) {
        const uint64_t k = keys[a0 + t];
        int lo = 0, hi = mb;  // first key of chunk y not below k
        while (lo < hi) {
            const int m = (lo + hi) >> 1;
            if (sk[m] < k) lo = m + 1; else hi = m;
        }
        if (lo) atomicAdd(&rank[(uint32_t)k], (uint32_t)lo);
    }
    __syncthreads();  // sk is reused by the CTA's next pair of chunks
}

__global__ void __launch_bounds__(kRankChunk) k_rank_cross(const uint64_t *__restrict__ keys, int64_t n,
                                                          uint32_t *__restrict__ rank) {
    __shared__ uint64_t sk[kRankChunk];
    rank_cross(keys, n, rank, blockIdx.x, blockIdx.y, sk);
}

__global__ void k_rank_scatter(const uint32_t *__restrict__ rank, int64_t n, uint32_t *__restrict__ sorig) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) sorig[rank[c]] = (uint32_t)c;
}

__global__ void k_rank_posts(const int64_t *__restrict__ cand, const uint32_t *__restrict__ sorig, int64_t n,
                             int64_t HW, uint32_t *__restrict__ sp) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) sp[i] = (uint32_t)(slot_key(cand, sorig[i], HW) >> 32);
}

// for every slot, the slot range holding the candidates within 2R rows
__device__ __forceinline__ void site_band(const uint32_t *__restrict__ sp, int64_t n, int W, int R,
                                          uint32_t *__restrict__ slo, uint32_t *__restrict__ shi, int64_t i) {
    if (i >= n) return;
    const uint32_t p = sp[i];
    if (p == 0xFFFFFFFFu) { slo[i] = (uint32_t)i; shi[i] = (uint32_t)i; return; }
    const int64_t y = p / (uint32_t)W;
    const uint64_t a = (uint64_t)max((int64_t)0, y - 2 * R) * (uint64_t)W;
    const uint64_t b = (uint64_t)(y + 2 * R + 1) * (uint64_t)W;
    int64_t lo = 0, hi = n;  // first slot with sp >= a
    while (lo < hi) { const int64_t m = (lo + hi) >> 1; if ((uint64_t)sp[m] < a) lo = m + 1; else hi = m; }
    const int64_t L = lo;
    lo = L; hi = n;          // first slot with sp >= b
    while (lo < hi) { const int64_t m = (lo + hi) >> 1; if ((uint64_t)sp[m] < b) lo = m + 1; else hi = m; }
    slo[i] = (uint32_t)L;
    shi[i] = (uint32_t)lo;
}

__global__ void k_site_bands(const uint32_t *__restrict__ sp, int64_t n, int W, int R,
                             uint32_t *__restrict__ slo, uint32_t *__restrict__ shi) {
    site_band(sp, n, W, R, slo, shi, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

struct Site1Params {
    const uint32_t *bm;
    int n;
    int H, W, R, PR, words, WWc;
    int n_obs;
    long long need;
    int64_t *chosen, *gains;
    uint32_t *cum;
    int32_t *n_chosen;
    const uint32_t *gain0;   // candidate order
    const uint32_t *sp, *sorig, *slo, *shi;  // slot order
    const unsigned long long *covered0;
    int vec_rows;            // bitmap rows are whole 16-byte vectors (PR % 4 == 0, bm 16-byte aligned)
    uint32_t *gbuf;          // gains in global memory (jobs whose gains exceed shared memory), or null
};

__device__ __forceinline__ uint64_t u64max(uint64_t a, uint64_t b) { return a > b ? a : b; }

// inclusive prefix sum over the lanes of a warp
__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// One greedy step per iteration, the whole block on it.  Per step: the block
// argmax of the cached gains; the winner's window, where the newly covered
// bits (delta = V_win AND NOT C) are found and C is updated; the winner's
// band (slots within 2R rows) compacted to the other candidates whose window
// meets the winner's; their gains lowered by popc(V_c AND delta) over the
// overlap, reading V_c only where delta is non-zero; the winner's gain set
// to zero (all of it is now covered).
// Global loads that do not depend on each other are issued together (the
// window's V and C words with the band's slot posts; the refresh's words in
// batches), and the compaction's counts and overlap prefixes come from warp
// scans, so a step costs four block barriers.  One SM's scattered loads
// (about 0.55 per cycle measured) bound the refresh.
__device__ __forceinline__ void site1_body(const Site1Params &P) {
    extern __shared__ __align__(16) unsigned char smem[];
    // the gains in shared memory, or (too many candidates for it) in global memory
    uint32_t *s_gain = P.gbuf ? P.gbuf : (uint32_t *)smem;                          // n
    uint32_t *s_delta = P.gbuf ? (uint32_t *)smem : s_gain + ((P.n + 3) & ~3);    // words
    int *s_list = (int *)(s_delta + ((P.words + 3) & ~3)); // kSiteThreads
    __shared__ uint64_t s_red[32];
    __shared__ int s_wcnt[32], s_wsum[32];
    __shared__ int s_dirty[kSiteThreads];
    __shared__ int s_pref[kSiteThreads + 1];
    __shared__ unsigned s_sum[kSiteThreads];
    __shared__ int4 s_geo[kSiteThreads];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int n = P.n, R = P.R, PR = P.PR, W = P.W, H = P.H, WWc = P.WWc;
    const int cs = (n + kSiteThreads - 1) / kSiteThreads;
    const int my0 = tid * cs, my1 = min(n, my0 + cs);

    for (int i = tid; i < n; i += blockDim.x)
        s_gain[i] = (P.sp[i] == 0xFFFFFFFFu) ? 0u : P.gain0[P.sorig[i]];
    s_dirty[tid] = 0;
    __syncthreads();
    // best cached key of this thread's slots (four independent max chains)
    auto local_best = [&]() {
        uint64_t b[4] = {0ull, 0ull, 0ull, 0ull};
        int i = my0;
        for (; i + 4 <= my1; i += 4) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t g = s_gain[i + q];
                b[q] = u64max(b[q], g ? (((uint64_t)g << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)(i + q))) : 0ull);
            }
        }
        for (; i < my1; ++i) {
            const uint32_t g = s_gain[i];
            b[0] = u64max(b[0], g ? (((uint64_t)g << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)i)) : 0ull);
        }
        return u64max(u64max(b[0], b[1]), u64max(b[2], b[3]));
    };
    uint64_t best = local_best();
    long long covered = (P.need >= 0) ? (long long)*P.covered0 : 0;

    int t = 0;
    for (; t < P.n_obs; ++t) {
        if (P.need >= 0 && covered >= P.need) break;
        // ---- block argmax of the cached keys
        uint64_t k = best;
        for (int o = 16; o > 0; o >>= 1) k = u64max(k, __shfl_xor_sync(0xffffffffu, k, o));
        if (lane == 0) s_red[wid] = k;
        __syncthreads();
        k = s_red[lane];
        for (int o = 16; o > 0; o >>= 1) k = u64max(k, __shfl_xor_sync(0xffffffffu, k, o));
        const uint32_t g = (uint32_t)(k >> 32);
        if (g == 0) break;
        const int s = (int)(0xFFFFFFFFu - (uint32_t)(k & 0xFFFFFFFFu));
        // ---- the winner's metadata
        const uint32_t wp = P.sp[s];
        const uint32_t wc = P.sorig[s];
        const int lo = (int)P.slo[s], hi = (int)P.shi[s];  // the winner's slot lies in [lo, hi)
        if (tid == 0) {
            P.chosen[t] = (int64_t)wp;
            P.gains[t] = (int64_t)g;
        }
        covered += g;
        const int wx = (int)(wp % (uint32_t)W), wy = (int)(wp / (uint32_t)W);
        const int wgw0 = floordiv(wx - R, 32);
        const uint32_t *Vw = P.bm + (int64_t)wc * P.words;
        // the band's first slot posts and bitmap indices, loaded beside the
        // window's words
        uint32_t bsp = (lo + tid < hi) ? P.sp[lo + tid] : 0u;
        uint32_t bso = (lo + tid < hi) ? P.sorig[lo + tid] : 0u;
        // ---- delta = V_win AND NOT C over the window, C |= V_win (the
        // loads of two passes are issued before either is used)
        for (int e0 = 0; e0 < P.words; e0 += 2 * kSiteThreads) {
            uint32_t v[2] = {0u, 0u}, old[2] = {0u, 0u};
            uint32_t *cp[2] = {nullptr, nullptr};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int e = e0 + h * kSiteThreads + tid;
                if (e < P.words) {
                    const int r = e / PR, w = e - r * PR;
                    const int y = wy - R + r, gw = wgw0 + w;
                    if (y >= 0 && y < H && gw >= 0 && gw < WWc) {
                        cp[h] = P.cum + (int64_t)y * WWc + gw;
                        v[h] = __ldg(Vw + e);
                        old[h] = *cp[h];
                    }
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int e = e0 + h * kSiteThreads + tid;
                if (e < P.words) {
                    const uint32_t d = cp[h] ? (v[h] & ~old[h]) : 0u;
                    if (d) *cp[h] = old[h] | v[h];
                    s_delta[e] = d;
                }
            }
        }
        // ---- band chunks: compact the other slots whose window meets the
        // winner's, with their overlap (rows x words) and its exclusive prefix
        for (int b0 = lo; b0 < hi; b0 += kSiteThreads) {
            const int i = b0 + tid;
            if (b0 != lo) {
                bsp = (i < hi) ? P.sp[i] : 0u;
                bso = (i < hi) ? P.sorig[i] : 0u;
            }
            bool aff = false;
            int ovl = 0;
            int4 geo = make_int4(0, 0, 0, 0);
            if (i < hi && i != s && s_gain[i] != 0) {
                const int cx = (int)(bsp % (uint32_t)W), cy = (int)(bsp / (uint32_t)W);
                if (abs(cx - wx) <= 2 * R) {
                    aff = true;
                    const int cgw0 = floordiv(cx - R, 32);
                    const int ya = max(max(cy, wy) - R, 0), yb = min(min(cy, wy) + R, H - 1);
                    const int ga = max(max(cgw0, wgw0), 0), gb = min(min(cgw0, wgw0) + PR - 1, WWc - 1);
                    const int nwd = (ya <= yb && ga <= gb) ? gb - ga + 1 : 0;
                    ovl = (ya <= yb && ga <= gb) ? (yb - ya + 1) * (P.vec_rows ? 1 : nwd) : 0;
                    // the overlap's first word in the delta window and in the
                    // candidate's bitmap (n * words < 2^32 on this path)
                    const int dbase = (ya - wy + R) * PR + (ga - wgw0);
                    const uint32_t vbase = bso * (uint32_t)P.words + (uint32_t)((ya - cy + R) * PR + (ga - cgw0));
                    geo = make_int4(dbase, (int)vbase, nwd, ga - cgw0);
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, aff);
            const int incl = warp_incl_scan(ovl, lane);
            if (lane == 31) {
                s_wcnt[wid] = __popc(bal);
                s_wsum[wid] = incl;
            }
            __syncthreads();  // also publishes s_delta
            // every warp scans the 32 warp totals
            const int wcn = s_wcnt[lane], wsm = s_wsum[lane];
            const int icn = warp_incl_scan(wcn, lane), ism = warp_incl_scan(wsm, lane);
            const int cnt_base = __shfl_sync(0xffffffffu, icn - wcn, wid);
            const int sum_base = __shfl_sync(0xffffffffu, ism - wsm, wid);
            const int tot = __shfl_sync(0xffffffffu, icn, 31);
            const int TT = __shfl_sync(0xffffffffu, ism, 31);
            if (aff) {
                const int li = cnt_base + __popc(bal & ((1u << lane) - 1u));
                s_list[li] = i;
                s_pref[li] = sum_base + incl - ovl;
                s_geo[li] = geo;
                s_sum[li] = 0;
            }
            if (tid == 0) s_pref[tot] = TT;
            __syncthreads();
            if (P.vec_rows) {
                // ---- refresh by overlap rows: row e (over all listed
                // candidates) on thread e mod 1024; its delta words come from
                // shared memory first, and only a row with new coverage reads
                // its candidate's bitmap row, as PR/4 16-byte loads
                for (int e = tid; e < TT; e += kSiteThreads) {
                    int l = 0, h2 = tot - 1;  // last l with s_pref[l] <= e
                    while (l < h2) {
                        const int m = (l + h2 + 1) >> 1;
                        if (s_pref[m] <= e) l = m; else h2 = m - 1;
                    }
                    const int4 gq = s_geo[l];
                    const int r = e - s_pref[l], nwd = gq.z, c0 = gq.w;  // overlap words c0 .. c0+nwd-1 of the row
                    const uint32_t *dl = s_delta + gq.x + r * PR;
                    uint32_t any = 0u;
                    for (int j = 0; j < nwd; ++j) any |= dl[j];
                    if (!any) continue;
                    const uint4 *vr = (const uint4 *)(P.bm + (uint32_t)gq.y - (uint32_t)c0 + (uint32_t)(r * PR));
                    unsigned sum = 0;
                    for (int q4 = 0; q4 < PR / 4; ++q4) {
                        const uint4 v = __ldg(vr + q4);
                        const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                        for (int t = 0; t < 4; ++t) {
                            const int j = 4 * q4 + t - c0;
                            if (j >= 0 && j < nwd) sum += __popc(vv[t] & dl[j]);
                        }
                    }
                    if (sum) atomicAdd(&s_sum[l], sum);
                }
            } else {
                // ---- every thread takes an equal run of the overlap words of all
                // listed candidates; within one candidate's overlap it walks rows
                // and words with running indices, loading eight words at a time
                // and reading V_c only where delta is non-zero
                const int per = (TT + kSiteThreads - 1) / kSiteThreads;
                const int e0 = tid * per, e1 = min(TT, e0 + per);
                if (e0 < e1) {
                    int l = 0, hi2 = tot - 1;  // last l with s_pref[l] <= e0
                    while (l < hi2) {
                        const int m = (l + hi2 + 1) >> 1;
                        if (s_pref[m] <= e0) l = m; else hi2 = m - 1;
                    }
                    int e = e0;
                    while (e < e1) {
                        const int pl = s_pref[l], pn = s_pref[l + 1];
                        if (e >= pn) {  // empty overlaps are skipped
                            ++l;
                            continue;
                        }
                        const int4 gq = s_geo[l];
                        const int nwd = gq.z, skip = PR - nwd;
                        const int u = e - pl, dy = u / nwd;
                        int dw = u - dy * nwd;
                        int di = gq.x + dy * PR + dw;
                        const uint32_t *vp = P.bm + (uint32_t)gq.y + (uint32_t)(dy * PR + dw);
                        const int send = min(e1, pn);
                        unsigned sum = 0;
                        for (; e < send; e += 8) {
                            uint32_t v[8];
    #pragma unroll
                            for (int q = 0; q < 8; ++q) {
                                v[q] = 0u;
                                if (e + q < send) {
                                    const uint32_t dl = s_delta[di];
                                    if (dl) v[q] = __ldg(vp) & dl;
                                    ++dw;
                                    ++di;
                                    ++vp;
                                    if (dw == nwd) {
                                        dw = 0;
                                        di += skip;
                                        vp += skip;
                                    }
                                }
                            }
    #pragma unroll
                            for (int q = 0; q < 8; ++q) sum += __popc(v[q]);
                        }
                        e = send;
                        if (sum) atomicAdd(&s_sum[l], sum);
                        ++l;
                    }
                }
            }
            __syncthreads();
            for (int q = tid; q < tot; q += kSiteThreads) {
                const int ci = s_list[q];
                s_gain[ci] -= s_sum[q];
                s_dirty[ci / cs] = 1;
            }
            if (tid == 0 && b0 == lo) {  // the winner covers all of its own gain
                s_gain[s] = 0;
                s_dirty[s / cs] = 1;
            }
            __syncthreads();
        }
        // the band held at least the winner, so the chunk loop ran and its
        // barriers order these gain reads after every update of this step
        if (s_dirty[tid]) {
            s_dirty[tid] = 0;
            best = local_best();
        }
    }
    if (tid == 0) *P.n_chosen = t;
}

__global__ void __launch_bounds__(kSiteThreads, 1) k_site_loop1(const Site1Params P) { site1_body(P); }

// ------------------------------------------------------------------ leader cluster
// The same greedy steps on a thread-block cluster of Q CTAs: the leader (rank
// 0) keeps every gain in its shared memory and takes the sequential part of a
// step (argmax, winner metadata, band compaction); the memory-heavy part --
// the winner's window (V and C words, C updated) and the refresh of the
// affected candidates' overlap rows -- is split by window row, row r on the
// CTA of rank r mod Q, so Q SMs issue its loads.  A step is one or more
// rounds (one per 1024-slot chunk of the winner's band):
//   leader: [new step: stop test, argmax, metadata]; compaction of the chunk;
//           header + list written into every CTA's shared memory
//   cluster barrier A; every CTA reads the same stop flag
//   all:    [new step: its window rows -> local delta rows, C updated];
//           its refresh rows -> partial sums added into the leader's s_sum
//   cluster barrier B
//   leader: gains lowered; [last chunk: winner's gain 0, owners rescan]
// Every CTA passes both barriers the same number of times.  Requires bitmap
// rows that are whole 16-byte vectors (PR % 4 == 0).
struct SiteQHeader {
    int stop, first, last, tot;
    int wx, wy, wgw0, pad;
};

__global__ void __launch_bounds__(kSiteThreads, 1) k_site_loopq(const Site1Params P) {
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank(), Q = (int)cl.num_blocks();
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *s_gain = (uint32_t *)smem;                 // n (leader)
    uint32_t *s_dloc = s_gain + ((P.n + 3) & ~3);        // this CTA's delta rows
    __shared__ SiteQHeader s_hdr;
    __shared__ int4 s_geo[kSiteThreads];                 // per listed candidate (broadcast)
    __shared__ unsigned s_sum[kSiteThreads];             // leader: summed partial refreshes
    __shared__ unsigned s_part[kSiteThreads];            // this CTA's partial refreshes
    __shared__ int s_cpref[kSiteThreads + 1];            // this CTA's row prefix over the list
    __shared__ int s_list[kSiteThreads];                 // leader: slots of the list
    __shared__ int s_dirty[kSiteThreads];                // leader
    __shared__ uint64_t s_red[32];
    __shared__ int s_wa[32], s_wb[32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int n = P.n, R = P.R, PR = P.PR, W = P.W, H = P.H, WWc = P.WWc;
    const int cs = (n + kSiteThreads - 1) / kSiteThreads;
    const int my0 = tid * cs, my1 = min(n, my0 + cs);
    const int nrow_loc = (2 * R + 1 - rank + Q - 1) / Q;  // window rows r = rank + Q*i of this CTA

    if (rank == 0) {
        for (int i = tid; i < n; i += kSiteThreads)
            s_gain[i] = (P.sp[i] == 0xFFFFFFFFu) ? 0u : P.gain0[P.sorig[i]];
        s_dirty[tid] = 0;
    }
    __syncthreads();
    auto local_best = [&]() {
        uint64_t b[4] = {0ull, 0ull, 0ull, 0ull};
        int i = my0;
        for (; i + 4 <= my1; i += 4) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t g = s_gain[i + q];
                b[q] = u64max(b[q], g ? (((uint64_t)g << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)(i + q))) : 0ull);
            }
        }
        for (; i < my1; ++i) {
            const uint32_t g = s_gain[i];
            b[0] = u64max(b[0], g ? (((uint64_t)g << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)i)) : 0ull);
        }
        return u64max(u64max(b[0], b[1]), u64max(b[2], b[3]));
    };
    uint64_t best = (rank == 0) ? local_best() : 0ull;
    long long covered = (rank == 0 && P.need >= 0) ? (long long)*P.covered0 : 0;
    int t = 0;               // leader: steps done
    int s = -1, lo = 0, hi = 0, b0 = 0;
    uint32_t wc = 0u;
    bool in_step = false;    // leader: a step's band is being processed
    cl.sync();

    for (;;) {
        // ================================================ leader: the round's work list
        if (rank == 0) {
            bool stop = false, first = false;
            if (!in_step) {
                stop = t >= P.n_obs || (P.need >= 0 && covered >= P.need);
                uint64_t k = 0ull;
                if (!stop) {
                    k = best;
                    for (int o = 16; o > 0; o >>= 1) k = u64max(k, __shfl_xor_sync(0xffffffffu, k, o));
                    if (lane == 0) s_red[wid] = k;
                    __syncthreads();
                    k = s_red[lane];
                    for (int o = 16; o > 0; o >>= 1) k = u64max(k, __shfl_xor_sync(0xffffffffu, k, o));
                    if ((uint32_t)(k >> 32) == 0u) stop = true;
                }
                if (!stop) {
                    const uint32_t g = (uint32_t)(k >> 32);
                    s = (int)(0xFFFFFFFFu - (uint32_t)(k & 0xFFFFFFFFu));
                    const uint32_t wp = P.sp[s];
                    wc = P.sorig[s];
                    lo = (int)P.slo[s];
                    hi = (int)P.shi[s];  // the winner's slot lies in [lo, hi)
                    if (tid == 0) {
                        P.chosen[t] = (int64_t)wp;
                        P.gains[t] = (int64_t)g;
                        s_hdr.wx = (int)(wp % (uint32_t)W);
                        s_hdr.wy = (int)(wp / (uint32_t)W);
                        s_hdr.wgw0 = floordiv((int)(wp % (uint32_t)W) - R, 32);
                    }
                    covered += g;
                    b0 = lo;
                    first = true;
                    in_step = true;
                }
            }
            int tot = 0;
            bool last = true;
            if (!stop) {
                __syncthreads();  // s_hdr geometry of a new step
                const int wx = s_hdr.wx, wy = s_hdr.wy, wgw0 = s_hdr.wgw0;
                const int i = b0 + tid;
                bool aff = false;
                int4 geo = make_int4(0, 0, 0, 0);
                if (i < hi && i != s && s_gain[i] != 0) {
                    const uint32_t bsp = P.sp[i];
                    const int cx = (int)(bsp % (uint32_t)W), cy = (int)(bsp / (uint32_t)W);
                    if (abs(cx - wx) <= 2 * R) {
                        const int cgw0 = floordiv(cx - R, 32);
                        const int ya = max(max(cy, wy) - R, 0), yb = min(min(cy, wy) + R, H - 1);
                        const int ga = max(max(cgw0, wgw0), 0), gb = min(min(cgw0, wgw0) + PR - 1, WWc - 1);
                        if (ya <= yb && ga <= gb) {
                            aff = true;
                            const int ra = ya - (wy - R), rb = yb - (wy - R);
                            const uint32_t vrow0 = P.sorig[i] * (uint32_t)P.words + (uint32_t)((ya - cy + R) * PR);
                            geo = make_int4(ra | (rb << 16), (gb - ga + 1) | ((ga - cgw0) << 10) | ((ga - wgw0) << 20),
                                            (int)vrow0, 0);
                        }
                    }
                }
                const unsigned bal = __ballot_sync(0xffffffffu, aff);
                if (lane == 0) s_wa[wid] = __popc(bal);
                __syncthreads();
                const int wcn = s_wa[lane];
                int icn = wcn;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int u = __shfl_up_sync(0xffffffffu, icn, o);
                    if (lane >= o) icn += u;
                }
                const int base = __shfl_sync(0xffffffffu, icn - wcn, wid);
                tot = __shfl_sync(0xffffffffu, icn, 31);
                last = b0 + kSiteThreads >= hi;
                if (aff) {
                    const int li = base + __popc(bal & ((1u << lane) - 1u));
                    s_list[li] = i;
                    s_sum[li] = 0u;
                    for (int q = 0; q < Q; ++q) *cl.map_shared_rank(&s_geo[li], q) = geo;
                }
            }
            if (tid < Q) {
                SiteQHeader h;
                h.stop = stop ? 1 : 0;
                h.first = first ? 1 : 0;
                h.last = last ? 1 : 0;
                h.tot = tot;
                h.wx = s_hdr.wx;
                h.wy = s_hdr.wy;
                h.wgw0 = s_hdr.wgw0;
                h.pad = (int)wc;
                *cl.map_shared_rank(&s_hdr, tid) = h;
            }
        }
        cl.sync();  // A: the round's header and list are in every CTA
        const SiteQHeader h = s_hdr;
        if (h.stop) break;
        const int wy = h.wy, wgw0 = h.wgw0, tot = h.tot;
        // ================================================ all: this CTA's rows
        // ---- its refresh rows: per listed candidate, the overlap rows r with
        // r = rank (mod Q), as an exclusive prefix over the list
        if (tid < tot) s_part[tid] = 0u;
        int cnt = 0;
        if (tid < tot) {
            const int ra = s_geo[tid].x & 0xFFFF, rb = s_geo[tid].x >> 16;
            const int r0 = ra + ((rank - ra) % Q + Q) % Q;
            cnt = (r0 <= rb) ? (rb - r0) / Q + 1 : 0;
        }
        int inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += u;
        }
        if (lane == 31) s_wb[wid] = inc;
        __syncthreads();
        {
            const int wv = s_wb[lane];
            int iw = wv;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, iw, o);
                if (lane >= o) iw += u;
            }
            const int wbase = __shfl_sync(0xffffffffu, iw - wv, wid);
            const int rows_all = __shfl_sync(0xffffffffu, iw, 31);
            if (tid < tot) s_cpref[tid] = wbase + inc - cnt;
            if (tid == 0) s_cpref[tot] = rows_all;
        }
        __syncthreads();
        const int TT = s_cpref[tot];
        // row item e of this CTA: its candidate, window row and bitmap row
        auto row_item = [&](int e, int &l, int &r, const uint4 *&vr) {
            l = 0;
            int h2 = tot - 1;  // last l with s_cpref[l] <= e
            while (l < h2) {
                const int m = (l + h2 + 1) >> 1;
                if (s_cpref[m] <= e) l = m; else h2 = m - 1;
            }
            const int4 gq = s_geo[l];
            const int ra = gq.x & 0xFFFF;
            r = ra + ((rank - ra) % Q + Q) % Q + Q * (e - s_cpref[l]);
            vr = (const uint4 *)(P.bm + (uint32_t)gq.z + (uint32_t)((r - ra) * PR));
        };
        // the first refresh row of this thread is loaded now, beside the
        // window's words (the loads do not depend on the new coverage)
        constexpr int kPreVec = 4;  // rows of up to 16 words
        const bool pre = tid < TT && PR / 4 <= kPreVec;
        uint4 pv[kPreVec];
        int pl = 0, pr = 0;
        if (pre) {
            const uint4 *vr;
            row_item(tid, pl, pr, vr);
#pragma unroll
            for (int q4 = 0; q4 < kPreVec; ++q4)
                if (q4 < PR / 4) pv[q4] = __ldg(vr + q4);
        }
        // ---- its window rows (first round of a step): delta rows, C updated
        if (h.first) {
            const uint32_t *Vw = P.bm + (int64_t)(uint32_t)h.pad * P.words;
            for (int e = tid; e < nrow_loc * PR; e += kSiteThreads) {
                const int il = e / PR, w = e - il * PR;
                const int r = rank + Q * il;
                const int y = wy - R + r, gw = wgw0 + w;
                uint32_t d = 0u;
                if (y >= 0 && y < H && gw >= 0 && gw < WWc) {
                    uint32_t *cp = P.cum + (int64_t)y * WWc + gw;
                    const uint32_t v = __ldg(Vw + r * PR + w);
                    const uint32_t old = *cp;
                    d = v & ~old;
                    if (d) *cp = old | v;
                }
                s_dloc[e] = d;
            }
        }
        __syncthreads();  // publishes s_dloc and the zeroed s_part
        // ---- refresh: popc(V_c AND delta) over each row's overlap words
        auto popc_words = [&](const uint4 &v, int q4, const uint32_t *dl, int c0, int nwd) {
            const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
            unsigned sum = 0;
#pragma unroll
            for (int t4 = 0; t4 < 4; ++t4) {
                const int j = 4 * q4 + t4 - c0;
                if (j >= 0 && j < nwd) sum += __popc(vv[t4] & dl[j]);
            }
            return sum;
        };
        if (pre) {
            const int4 gq = s_geo[pl];
            const int nwd = gq.y & 0x3FF, c0 = (gq.y >> 10) & 0x3FF, dw0 = gq.y >> 20;
            const uint32_t *dl = s_dloc + ((pr - rank) / Q) * PR + dw0;
            unsigned sum = 0;
#pragma unroll
            for (int q4 = 0; q4 < kPreVec; ++q4)
                if (q4 < PR / 4) sum += popc_words(pv[q4], q4, dl, c0, nwd);
            if (sum) atomicAdd(&s_part[pl], sum);
        }
        for (int e = tid + (pre ? kSiteThreads : 0); e < TT; e += kSiteThreads) {
            int l, r;
            const uint4 *vr;
            row_item(e, l, r, vr);
            const int4 gq = s_geo[l];
            const int nwd = gq.y & 0x3FF, c0 = (gq.y >> 10) & 0x3FF, dw0 = gq.y >> 20;
            const uint32_t *dl = s_dloc + ((r - rank) / Q) * PR + dw0;
            unsigned sum = 0;
            for (int q4 = 0; q4 < PR / 4; ++q4) sum += popc_words(__ldg(vr + q4), q4, dl, c0, nwd);
            if (sum) atomicAdd(&s_part[l], sum);
        }
        __syncthreads();
        if (tid < tot && s_part[tid]) atomicAdd(cl.map_shared_rank(&s_sum[tid], 0), s_part[tid]);
        cl.sync();  // B: every partial refresh is in the leader's s_sum
        // ================================================ leader: lower the gains
        if (rank == 0) {
            for (int q = tid; q < tot; q += kSiteThreads) {
                const int ci = s_list[q];
                s_gain[ci] -= s_sum[q];
                s_dirty[ci / cs] = 1;
            }
            if (h.last) {
                if (tid == 0) {
                    s_gain[s] = 0u;
                    s_dirty[s / cs] = 1;
                }
                in_step = false;
                ++t;
            } else {
                b0 += kSiteThreads;
            }
            __syncthreads();
            if (h.last && s_dirty[tid]) {
                s_dirty[tid] = 0;
                best = local_best();
            }
        }
    }
    if (rank == 0 && tid == 0) *P.n_chosen = t;
    cl.sync();  // no CTA leaves while another may still address its shared memory
}

// ------------------------------------------------------------------ multi-winner leader cluster
// Several greedy steps per round, with results identical to one step at a
// time.  After a round's refresh every cached gain is exact.  The leader then
// takes candidates in decreasing key order (gain, then lowest slot) and
// accepts each while it lies more than 2R (Chebyshev distance of the posts)
// from every candidate already accepted in this round, stopping at the first
// that does not (or at n_obs, the coverage stop, a zero gain, or the round's
// capacity).  Every accepted candidate is exactly the next sequential argmax:
// its window is disjoint from the windows accepted before it in the round,
// so its gain is unchanged by them (Sec. "The multiple transmitter siting
// process", Site: a gain can only shrink as coverage grows, so no other
// candidate can have risen above it), and every other key can only have
// fallen.  The accepted windows are disjoint, so their newly covered bits
// (deltas) are disjoint too and the refreshes they cause add up.
//
// Roles: the leader (rank 0) holds the gains; each of its threads caches the
// two best keys of its run of slots and their posts, so warp 0 picks the
// round's winners with no block barrier (the owner of a winner promotes its
// second key; a run whose second key is used up is rescanned by the warp).
// While warp 0 picks, groups of the leader's other warps take each winner as
// soon as it is accepted and compact its band (slots within 2R rows) into a
// list of (candidate, winner) pairs whose windows meet.  A list holds at most
// kMultiList pairs; a round whose pairs do not fit compacts its bands again
// after the picks, in band order, over as many lists as they need.  The
// workers (ranks 1..Q-1) own window rows r = rank-1 (mod Q-1): on a round's
// first list they compute every winner's delta rows and OR the winners into C
// (atomically: two disjoint windows can share a boundary word of C), then
// every list adds popc(V_c AND delta) over its overlap rows into the leader's
// sums, which the leader subtracts from the gains.
constexpr int kMultiList = 1024;   // (candidate, winner) pairs per list
constexpr int kMultiMaxL = 64;     // winners per round
constexpr int kMultiItems = 8;     // band slots per leader thread and pass
constexpr int kCompactG = 4;       // warps that compact one winner's band during the picks
constexpr long kMultiSpin = 1L << 22;  // polls of a compacting warp for the next winner (~0.2 s)

struct SiteMParams {
    Site1Params b;
    int Lmax;     // winners per round: <= kMultiMaxL and the workers' delta rows
    int nrow;     // window rows per worker: ceil((2R+1) / (Q-1))
    unsigned long long *stats;  // rounds, lists, rescans of used-up runs (spare workspace bytes)
};

struct SiteMHeader {
    int stop, first, last, tot, L, pad0, pad1, pad2;
};

__device__ __forceinline__ uint64_t slot_key(uint32_t g, int i) {
    return g ? (((uint64_t)g << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)i)) : 0ull;
}
__device__ __forceinline__ int key_slot(uint64_t k) { return (int)(0xFFFFFFFFu - (uint32_t)(k & 0xFFFFFFFFu)); }

__global__ void __launch_bounds__(kSiteThreads, 1) k_site_multi(const SiteMParams M) {
    const Site1Params &P = M.b;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank(), Q = (int)cl.num_blocks(), Qw = Q - 1;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int n = P.n, R = P.R, PR = P.PR, W = P.W, H = P.H, WWc = P.WWc;
    const int cs = (n + kSiteThreads - 1) / kSiteThreads;
    const int my0 = min(n, tid * cs), my1 = min(n, my0 + cs);
    const int nrow = M.nrow;
    extern __shared__ __align__(16) unsigned char smem[];
    // leader: gains, then the list's slots and sums
    uint32_t *s_gain = (uint32_t *)smem;
    int *s_list = (int *)(s_gain + ((n + 3) & ~3));
    unsigned *s_sum = (unsigned *)(s_list + kMultiList);
    // worker: delta rows of every winner, list row prefix, partial sums
    uint32_t *s_dloc = (uint32_t *)smem;
    int *s_cpref = (int *)(s_dloc + (size_t)M.Lmax * nrow * PR);
    unsigned *s_part = (unsigned *)(s_cpref + kMultiList + 4);
    __shared__ SiteMHeader s_hdr;
    __shared__ int4 s_win[kMultiMaxL];      // per winner: wx, wy, wgw0, bitmap index (broadcast)
    __shared__ int4 s_geo[kMultiList];      // per pair (broadcast)
    // leader selection state
    __shared__ uint64_t s_tkey[kSiteThreads], s_tkey2[kSiteThreads];
    __shared__ uint32_t s_tpost[kSiteThreads], s_tpost2[kSiteThreads];
    __shared__ unsigned char s_t2ok[kSiteThreads], s_dirty[kSiteThreads];
    __shared__ uint64_t s_wkey[32];
    __shared__ int s_wslot[kMultiMaxL], s_wx[kMultiMaxL], s_wy[kMultiMaxL];
    __shared__ uint32_t s_wpost[kMultiMaxL], s_wgain[kMultiMaxL];
    __shared__ int s_blo[kMultiMaxL], s_bpref[kMultiMaxL + 1];
    __shared__ int s_wa[32], s_wb[32];
    __shared__ int s_nL, s_cut;
    // the round's winners as warp 0 accepts them (count, then a final flag),
    // the pairs that warps 1..31 compact from their bands meanwhile, and
    // whether those pairs overflowed a list or a wait gave up
    __shared__ int s_nacc, s_seldone, s_ntot, s_ovf, s_err;

    const uint32_t *sp = P.sp;
    if (rank == 0) {
        for (int i = tid; i < n; i += kSiteThreads)
            s_gain[i] = (sp[i] == 0xFFFFFFFFu) ? 0u : P.gain0[P.sorig[i]];
        s_dirty[tid] = 1;
    }
    if (tid == 0) s_err = 0;
    __syncthreads();
    long long covered = (rank == 0 && P.need >= 0) ? (long long)*P.covered0 : 0;
    int t = 0, L = 0, cursor = 0, NI = 0;
    bool in_round = false, first = false;
    unsigned long long n_rounds = 0, n_lists = 0, n_rescans = 0;  // leader thread 0's counts
    cl.sync();

    for (;;) {
        // ================================================ leader
        if (rank == 0) {
            bool stop = false;
            if (!in_round) {
                // ---- the two best keys of every dirty run and their posts
                if (s_dirty[tid]) {
                    s_dirty[tid] = 0;
                    uint64_t a1 = 0ull, a2 = 0ull, c1 = 0ull, c2 = 0ull;  // two chains
                    int i = my0;
                    for (; i + 2 <= my1; i += 2) {
                        const uint64_t ka = slot_key(s_gain[i], i), kb = slot_key(s_gain[i + 1], i + 1);
                        if (ka > a1) { a2 = a1; a1 = ka; } else if (ka > a2) a2 = ka;
                        if (kb > c1) { c2 = c1; c1 = kb; } else if (kb > c2) c2 = kb;
                    }
                    if (i < my1) {
                        const uint64_t ka = slot_key(s_gain[i], i);
                        if (ka > a1) { a2 = a1; a1 = ka; } else if (ka > a2) a2 = ka;
                    }
                    const uint64_t b1 = u64max(a1, c1);
                    const uint64_t b2 = u64max(a1 > c1 ? a2 : c2, a1 > c1 ? c1 : a1);
                    const uint32_t p1 = b1 ? sp[key_slot(b1)] : 0u;
                    const uint32_t p2 = b2 ? sp[key_slot(b2)] : 0u;
                    s_tkey[tid] = b1;
                    s_tkey2[tid] = b2;
                    s_tpost[tid] = p1;
                    s_tpost2[tid] = p2;
                    s_t2ok[tid] = 1;
                }
                __syncthreads();
                {
                    uint64_t k = s_tkey[tid];
                    for (int o = 16; o > 0; o >>= 1) k = u64max(k, __shfl_xor_sync(0xffffffffu, k, o));
                    if (lane == 0) s_wkey[wid] = k;
                }
                if (tid == 0) {
                    s_nacc = 0;
                    s_seldone = 0;
                    s_ntot = 0;
                    s_ovf = 0;
                }
                __syncthreads();
                // ---- warp 0 picks the round's winners.  Lane j holds warp j's best
                // key as (gain, ~slot) and the coordinates of winners j and j + 32;
                // the 64-bit max is two 32-bit warp reductions (gain, then ~slot
                // among the lanes holding that gain).
                if (wid == 0) {
                    const uint64_t k0 = s_wkey[lane];
                    uint32_t khi = (uint32_t)(k0 >> 32), klo = (uint32_t)k0;
                    int ax = 0, ay = 0, bx = 0, by = 0;
                    int nl = 0;
                    for (;;) {
                        if (t + nl >= P.n_obs || nl >= M.Lmax) break;
                        if (P.need >= 0 && covered >= P.need) break;
                        const uint32_t g = __reduce_max_sync(0xffffffffu, khi);
                        if (g == 0u) break;
                        const uint32_t lo = __reduce_max_sync(0xffffffffu, khi == g ? klo : 0u);
                        const int slot = (int)(0xFFFFFFFFu - lo);
                        const int own = slot / cs;
                        const uint32_t post = s_tpost[own];
                        const int x = (int)(post % (uint32_t)W), y = (int)(post / (uint32_t)W);
                        const bool conf = (lane < nl && abs(x - ax) <= 2 * R && abs(y - ay) <= 2 * R) ||
                                          (lane + 32 < nl && abs(x - bx) <= 2 * R && abs(y - by) <= 2 * R);
                        if (__any_sync(0xffffffffu, conf)) break;
                        if (lane == (nl & 31)) {
                            if (nl < 32) { ax = x; ay = y; } else { bx = x; by = y; }
                        }
                        const bool t2 = s_t2ok[own] != 0;
                        __syncwarp();  // every lane has read the owner's state before lane 0 changes it
                        if (lane == 0) {
                            s_wslot[nl] = slot;
                            s_wpost[nl] = post;
                            s_wgain[nl] = g;
                            s_wx[nl] = x;
                            s_wy[nl] = y;
                            s_gain[slot] = 0u;
                            if (t2) {  // the owner's second key becomes its best
                                s_tkey[own] = s_tkey2[own];
                                s_tpost[own] = s_tpost2[own];
                                s_t2ok[own] = 0;
                            }
                            __threadfence_block();  // the winner (and its zero gain) before its count
                            *(volatile int *)&s_nacc = nl + 1;
                        }
                        ++nl;
                        covered += g;
                        __syncwarp();
                        if (!t2) {  // its run is rescanned (its second key was used up)
                            if (lane == 0) ++n_rescans;
                            const int r0 = min(n, own * cs), r1 = min(n, r0 + cs);
                            uint64_t bk = 0ull;
                            for (int i = r0 + lane; i < r1; i += 32) bk = u64max(bk, slot_key(s_gain[i], i));
                            const uint32_t bh = __reduce_max_sync(0xffffffffu, (uint32_t)(bk >> 32));
                            const uint32_t bl = __reduce_max_sync(0xffffffffu, (uint32_t)(bk >> 32) == bh ? (uint32_t)bk : 0u);
                            if (lane == 0) {
                                const uint64_t kb = ((uint64_t)bh << 32) | bl;
                                s_tkey[own] = kb;
                                s_tpost[own] = kb ? sp[key_slot(kb)] : 0u;
                            }
                            __syncwarp();
                        }
                        // the owner warp's best key
                        const int ow = own >> 5;
                        const uint64_t kk = s_tkey[(ow << 5) + lane];
                        const uint32_t hh = __reduce_max_sync(0xffffffffu, (uint32_t)(kk >> 32));
                        const uint32_t ll = __reduce_max_sync(0xffffffffu, (uint32_t)(kk >> 32) == hh ? (uint32_t)kk : 0u);
                        if (lane == ow) { khi = hh; klo = ll; }
                    }
                    if (lane == 0) {
                        s_nL = nl;
                        __threadfence_block();
                        *(volatile int *)&s_seldone = 1;
                    }
                } else {
                    // ---- meanwhile groups of kCompactG warps (of warps 1..31) take
                    // winner j = group (mod groups) as soon as it is accepted: its
                    // metadata and geometry (into every worker), its band size,
                    // and the band slots whose windows meet its window appended
                    // to the list, the band split over the group's warps.  The list's
                    // order is free: each pair's refresh is added into its own
                    // sum.  A later winner of the round is more than 2R from
                    // every earlier one, so it is never a pair of theirs, and an
                    // accepted winner's gain is 0 before its count is published.
                    constexpr int kGroups = 31 / kCompactG;
                    const int grp = (wid - 1) / kCompactG, part = (wid - 1) % kCompactG;
                    for (int j = grp; grp < kGroups && j < kMultiMaxL; j += kGroups) {
                        int ready = 0;
                        if (lane == 0) {  // lane 0 polls; the warp follows its answer
                            for (long it = 0;; ++it) {
                                if (*(volatile int *)&s_nacc > j) { ready = 1; break; }
                                if (*(volatile int *)&s_seldone) {
                                    ready = *(volatile int *)&s_nacc > j;
                                    break;
                                }
                                if (it > kMultiSpin) {
                                    s_err = 1;
                                    break;
                                }
                                __nanosleep(32);
                            }
                            __threadfence_block();
                        }
                        __syncwarp();
                        if (!__shfl_sync(0xffffffffu, ready, 0)) break;
                        const int slot = s_wslot[j], wx = s_wx[j], wy = s_wy[j];
                        const int lo = (int)P.slo[slot], hi = (int)P.shi[slot];
                        const int wgw0 = floordiv(wx - R, 32);
                        const int4 wv = make_int4(wx, wy, wgw0, (int)P.sorig[slot]);
                        if (part == 0) {
                            if (lane == 0) {
                                s_win[j] = wv;
                                s_blo[j] = lo;
                                s_bpref[j] = hi - lo;
                            }
                            if (lane >= 1 && lane < Q) *cl.map_shared_rank(&s_win[j], lane) = wv;
                        }
                        for (int i0 = lo + 32 * part; i0 < hi; i0 += 32 * kCompactG * kMultiItems) {
                            uint32_t ip[kMultiItems], io[kMultiItems];
                            bool gz[kMultiItems];
#pragma unroll
                            for (int q = 0; q < kMultiItems; ++q) {
                                const int i = i0 + 32 * kCompactG * q + lane;
                                gz[q] = i >= hi || s_gain[i] == 0u;
                                ip[q] = i < hi ? sp[i] : 0u;
                                io[q] = i < hi ? P.sorig[i] : 0u;
                            }
#pragma unroll
                            for (int q = 0; q < kMultiItems; ++q) {
                                const int i = i0 + 32 * kCompactG * q + lane;
                                int4 geo = make_int4(0, 0, 0, 0);
                                bool aff = false;
                                if (!gz[q]) {
                                    const int cx = (int)(ip[q] % (uint32_t)W), cy = (int)(ip[q] / (uint32_t)W);
                                    if (abs(cx - wx) <= 2 * R && abs(cy - wy) <= 2 * R) {
                                        const int cgw0 = floordiv(cx - R, 32);
                                        const int ya = max(max(cy, wy) - R, 0), yb = min(min(cy, wy) + R, H - 1);
                                        const int ga = max(max(cgw0, wgw0), 0), gb = min(min(cgw0, wgw0) + PR - 1, WWc - 1);
                                        if (ya <= yb && ga <= gb) {
                                            aff = true;
                                            const int ra = ya - (wy - R), rb = yb - (wy - R);
                                            const uint32_t vrow0 = io[q] * (uint32_t)P.words + (uint32_t)((ya - cy + R) * PR);
                                            geo = make_int4(ra | (rb << 16),
                                                            (gb - ga + 1) | ((ga - cgw0) << 10) | ((ga - wgw0) << 20),
                                                            (int)vrow0, j);
                                        }
                                    }
                                }
                                const unsigned am = __ballot_sync(0xffffffffu, aff);
                                if (am) {
                                    int base = 0;
                                    if (lane == 0) base = atomicAdd(&s_ntot, __popc(am));
                                    base = __shfl_sync(0xffffffffu, base, 0);
                                    if (aff) {
                                        const int li = base + __popc(am & ((1u << lane) - 1u));
                                        if (li < kMultiList) {
                                            s_list[li] = i;
                                            s_sum[li] = 0u;
                                            for (int r = 1; r < Q; ++r) *cl.map_shared_rank(&s_geo[li], r) = geo;
                                        } else {
                                            s_ovf = 1;
                                        }
                                    }
                                }
                            }
                        }
                    }
                }
                __syncthreads();
                L = s_nL;
                if (L == 0 || s_err) {
                    stop = true;
                } else if (!s_ovf) {
                    // every pair is in one list
                    NI = 0;
                    cursor = 0;
                    in_round = true;
                    first = true;
                    ++n_rounds;
                } else {
                    // too many pairs for one list: the bands are compacted again
                    // below, in band order, over as many lists as they need
                    if (wid == 0) {  // exclusive prefix of the band sizes (L <= 64)
                        const int a = lane < L ? s_bpref[lane] : 0;
                        const int b = lane + 32 < L ? s_bpref[lane + 32] : 0;
                        const int ia = warp_incl_scan(a, lane);
                        const int ta = __shfl_sync(0xffffffffu, ia, 31);
                        const int ib = warp_incl_scan(b, lane) + ta;
                        __syncwarp();
                        if (lane < L) s_bpref[lane] = ia - a;
                        if (lane + 32 < L) s_bpref[lane + 32] = ib - b;
                        if (lane == 31) s_bpref[L] = ib;
                    }
                    __syncthreads();
                    NI = s_bpref[L];
                    cursor = 0;
                    in_round = true;
                    first = true;
                    ++n_rounds;
                }
            }
            // ---- compaction of band slots [cursor, NI) into the list
            int tot = 0;
            if (!stop && NI == 0) tot = min(s_ntot, kMultiList);  // the list compacted during the picks
            if (!stop) {
                while (cursor < NI && tot < kMultiList) {
                    const int chunk = min(NI - cursor, kMultiItems * kSiteThreads);
                    const int per = (chunk + kSiteThreads - 1) / kSiteThreads;
                    const int e0 = cursor + tid * per, e1 = min(cursor + chunk, e0 + per);
                    uint32_t ip[kMultiItems], io[kMultiItems];
                    int jfirst = 0;
                    if (e0 < e1) {  // winner of the first item: last j with s_bpref[j] <= e0
                        int hi2 = L - 1;
                        while (jfirst < hi2) {
                            const int m = (jfirst + hi2 + 1) >> 1;
                            if (s_bpref[m] <= e0) jfirst = m; else hi2 = m - 1;
                        }
                    }
                    {
                        int j = jfirst;
#pragma unroll
                        for (int q = 0; q < kMultiItems; ++q) {
                            const int e = e0 + q;
                            ip[q] = 0xFFFFFFFFu;
                            io[q] = 0u;
                            if (e < e1) {
                                while (s_bpref[j + 1] <= e) ++j;
                                const int i = s_blo[j] + (e - s_bpref[j]);
                                if (s_gain[i] != 0u) {
                                    ip[q] = sp[i];
                                    io[q] = P.sorig[i];
                                }
                            }
                        }
                    }
                    // pass 1: which items' windows meet their winner's
                    unsigned affm = 0u;
                    {
                        int j = jfirst;
#pragma unroll
                        for (int q = 0; q < kMultiItems; ++q) {
                            const int e = e0 + q;
                            if (e < e1) {
                                while (s_bpref[j + 1] <= e) ++j;
                                if (ip[q] != 0xFFFFFFFFu) {
                                    const int4 wv = s_win[j];
                                    const int cx = (int)(ip[q] % (uint32_t)W), cy = (int)(ip[q] / (uint32_t)W);
                                    if (abs(cx - wv.x) <= 2 * R && abs(cy - wv.y) <= 2 * R) {
                                        const int cgw0 = floordiv(cx - R, 32);
                                        const int ya = max(max(cy, wv.y) - R, 0), yb = min(min(cy, wv.y) + R, H - 1);
                                        const int ga = max(max(cgw0, wv.z), 0), gb = min(min(cgw0, wv.z) + PR - 1, WWc - 1);
                                        if (ya <= yb && ga <= gb) affm |= 1u << q;
                                    }
                                }
                            }
                        }
                    }
                    const int cnt = __popc(affm);
                    // block exclusive scan of the counts
                    const int inc = warp_incl_scan(cnt, lane);
                    if (lane == 31) s_wa[wid] = inc;
                    if (tid == 0) s_cut = 0x7fffffff;
                    __syncthreads();
                    const int wv = s_wa[lane];
                    const int iw = warp_incl_scan(wv, lane);
                    const int base = tot + __shfl_sync(0xffffffffu, iw - wv, wid) + inc - cnt;
                    const int T = __shfl_sync(0xffffffffu, iw, 31);
                    // pass 2: the affected items' pairs, in item order
                    int li = base;
                    if (affm) {
                        int j = jfirst;
#pragma unroll
                        for (int q = 0; q < kMultiItems; ++q) {
                            const int e = e0 + q;
                            if (e < e1) while (s_bpref[j + 1] <= e) ++j;
                            if (affm & (1u << q)) {
                                if (li < kMultiList) {
                                    const int4 wv = s_win[j];
                                    const int wy = wv.y, wgw0 = wv.z;
                                    const int cx = (int)(ip[q] % (uint32_t)W), cy = (int)(ip[q] / (uint32_t)W);
                                    const int cgw0 = floordiv(cx - R, 32);
                                    const int ya = max(max(cy, wy) - R, 0), yb = min(min(cy, wy) + R, H - 1);
                                    const int ga = max(max(cgw0, wgw0), 0), gb = min(min(cgw0, wgw0) + PR - 1, WWc - 1);
                                    const int ra = ya - (wy - R), rb = yb - (wy - R);
                                    const uint32_t vrow0 = io[q] * (uint32_t)P.words + (uint32_t)((ya - cy + R) * PR);
                                    const int4 geo = make_int4(ra | (rb << 16),
                                                               (gb - ga + 1) | ((ga - cgw0) << 10) | ((ga - wgw0) << 20),
                                                               (int)vrow0, j);
                                    s_list[li] = s_blo[j] + (e - s_bpref[j]);
                                    s_sum[li] = 0u;
                                    for (int r = 1; r < Q; ++r) *cl.map_shared_rank(&s_geo[li], r) = geo;
                                } else {
                                    atomicMin(&s_cut, e);
                                }
                                ++li;
                            }
                        }
                    }
                    __syncthreads();
                    if (tot + T > kMultiList) {
                        cursor = s_cut;  // the first slot whose pair did not fit
                        tot = kMultiList;
                    } else {
                        cursor += chunk;
                        tot += T;
                    }
                    __syncthreads();  // s_cut and s_wa are reused by the next pass
                }
            }
            if (!stop) ++n_lists;
            if (tid < Q) {
                SiteMHeader h;
                h.stop = stop ? 1 : 0;
                h.first = first ? 1 : 0;
                h.last = (cursor >= NI) ? 1 : 0;
                h.tot = tot;
                h.L = L;
                h.pad0 = h.pad1 = h.pad2 = 0;
                *cl.map_shared_rank(&s_hdr, tid) = h;
            }
        }
        cl.sync();  // A: header, winners and list are in every CTA
        const SiteMHeader h = s_hdr;
        if (h.stop) break;
        // ================================================ workers
        if (rank > 0) {
            const int wr = rank - 1, tot = h.tot, Lr = h.L;
            int cnt = 0;
            if (tid < tot) {
                const int ra = s_geo[tid].x & 0xFFFF, rb = s_geo[tid].x >> 16;
                const int r0 = ra + ((wr - ra) % Qw + Qw) % Qw;
                cnt = (r0 <= rb) ? (rb - r0) / Qw + 1 : 0;
                s_part[tid] = 0u;
            }
            const int inc = warp_incl_scan(cnt, lane);
            if (lane == 31) s_wb[wid] = inc;
            __syncthreads();
            {
                const int wv = s_wb[lane];
                const int iw = warp_incl_scan(wv, lane);
                const int wbase = __shfl_sync(0xffffffffu, iw - wv, wid);
                const int rows_all = __shfl_sync(0xffffffffu, iw, 31);
                if (tid < tot) s_cpref[tid] = wbase + inc - cnt;
                if (tid == 0) s_cpref[tot] = rows_all;
            }
            __syncthreads();  // s_cpref and the zeroed s_part
            const int TT = s_cpref[tot];
            // row item e of this worker: its pair, window row and bitmap row
            auto row_item = [&](int e, int &l, int &r, const uint4 *&vr) {
                l = 0;
                int h2 = tot - 1;  // last l with s_cpref[l] <= e
                while (l < h2) {
                    const int m = (l + h2 + 1) >> 1;
                    if (s_cpref[m] <= e) l = m; else h2 = m - 1;
                }
                const int4 gq = s_geo[l];
                const int ra = gq.x & 0xFFFF;
                r = ra + ((wr - ra) % Qw + Qw) % Qw + Qw * (e - s_cpref[l]);
                vr = (const uint4 *)(P.bm + (uint32_t)gq.z + (uint32_t)((r - ra) * PR));
            };
            // the first refresh row of each thread is loaded beside the window's
            // words (only the popcounts need the new coverage)
            constexpr int kPreVec = 2;  // rows of up to 8 words (R = 100: 8)
            const bool pre = tid < TT && PR / 4 <= kPreVec;
            uint4 pv[kPreVec];
            int pl = 0, prr = 0;
            if (pre) {
                const uint4 *vr;
                row_item(tid, pl, prr, vr);
#pragma unroll
                for (int q4 = 0; q4 < kPreVec; ++q4)
                    if (q4 < PR / 4) pv[q4] = __ldg(vr + q4);
            }
            // ---- this worker's window rows of every winner (a round's first list)
            if (h.first) {
                const int per_w = nrow * PR;
                for (int e = tid; e < Lr * per_w; e += kSiteThreads) {
                    const int j = e / per_w, rem = e - j * per_w;
                    const int il = rem / PR, w = rem - il * PR;
                    const int r = wr + Qw * il;
                    const int4 wv = s_win[j];
                    uint32_t d = 0u;
                    if (r <= 2 * R) {
                        const int y = wv.y - R + r, gw = wv.z + w;
                        if (y >= 0 && y < H && gw >= 0 && gw < WWc) {
                            uint32_t *cp = P.cum + (int64_t)y * WWc + gw;
                            const uint32_t v = __ldg(P.bm + (int64_t)(uint32_t)wv.w * P.words + r * PR + w);
                            const uint32_t old = *cp;
                            d = v & ~old;
                            if (d) atomicOr(cp, v);
                        }
                    }
                    s_dloc[e] = d;
                }
            }
            __syncthreads();  // s_dloc published
            // popc(V_c AND delta) over the overlap words of one refresh row
            auto row_sum = [&](const uint32_t *dl, int c0, int nwd, int q4, const uint4 &v) {
                const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
                unsigned sum = 0;
#pragma unroll
                for (int t4 = 0; t4 < 4; ++t4) {
                    const int jw = 4 * q4 + t4 - c0;
                    if (jw >= 0 && jw < nwd) sum += __popc(vv[t4] & dl[jw]);
                }
                return sum;
            };
            auto row_delta = [&](int l, int r, int &c0, int &nwd) {
                const int4 gq = s_geo[l];
                nwd = gq.y & 0x3FF;
                c0 = (gq.y >> 10) & 0x3FF;
                const int dw0 = gq.y >> 20;
                return s_dloc + ((size_t)gq.w * nrow + (r - wr) / Qw) * PR + dw0;
            };
            if (pre) {
                int c0, nwd;
                const uint32_t *dl = row_delta(pl, prr, c0, nwd);
                unsigned sum = 0;
#pragma unroll
                for (int q4 = 0; q4 < kPreVec; ++q4)
                    if (q4 < PR / 4) sum += row_sum(dl, c0, nwd, q4, pv[q4]);
                if (sum) atomicAdd(&s_part[pl], sum);
            }
            for (int e = tid + (pre ? kSiteThreads : 0); e < TT; e += kSiteThreads) {
                int l, r, c0, nwd;
                const uint4 *vr;
                row_item(e, l, r, vr);
                const uint32_t *dl = row_delta(l, r, c0, nwd);
                uint32_t any = 0u;
                for (int jw = 0; jw < nwd; ++jw) any |= dl[jw];
                if (!any) continue;
                unsigned sum = 0;
                for (int q4 = 0; q4 < PR / 4; ++q4) sum += row_sum(dl, c0, nwd, q4, __ldg(vr + q4));
                if (sum) atomicAdd(&s_part[l], sum);
            }
            __syncthreads();
            if (tid < tot && s_part[tid]) atomicAdd(cl.map_shared_rank(&s_sum[tid], 0), s_part[tid]);
        }
        cl.sync();  // B: every partial refresh is in the leader's sums
        // ================================================ leader: lower the gains
        if (rank == 0) {
            for (int q = tid; q < h.tot; q += kSiteThreads) {
                const unsigned d = s_sum[q];
                if (d) {
                    const int ci = s_list[q];
                    atomicSub(&s_gain[ci], d);
                    s_dirty[ci / cs] = 1;
                }
            }
            first = false;
            if (h.last) {
                if (tid < L) {
                    P.chosen[t + tid] = (int64_t)s_wpost[tid];
                    P.gains[t + tid] = (int64_t)s_wgain[tid];
                    s_dirty[s_wslot[tid] / cs] = 1;
                }
                t += L;
                in_round = false;
            }
            __syncthreads();
        }
    }
    if (rank == 0 && tid == 0) {
        *P.n_chosen = s_err ? VS_ERR_TIMEOUT : t;
        M.stats[0] = n_rounds;
        M.stats[1] = n_lists;
        M.stats[2] = n_rescans;
    }
    cl.sync();  // no CTA leaves while another may still address its shared memory
}

// many independent greedy loops (one per terrain) in one launch: CTA j runs job j
constexpr int kSiteMaxJobs = 64;
struct Site1Batch {
    Site1Params job[kSiteMaxJobs];
};
__global__ void __launch_bounds__(kSiteThreads, 1) k_site_loop1_batch(const __grid_constant__ Site1Batch B) {
    site1_body(B.job[blockIdx.x]);
}

// The preparation of many greedy problems in six launches, one per step for
// every job (a job's blocks of a step follow the previous job's): 0 dense
// gains (and the coverage count zeroed), 1 slot-order chunks (and the
// coverage count of the starting cumulative viewshed), 2 cross-chunk ranks,
// 3 scatter to slots, 4 slot posts, 5 bands.  Each step's body is the one the
// single-problem launches use.
constexpr int kPrepPhases = 6;
constexpr int kCovBlocks = 16;
struct PrepJob {
    const uint32_t *bm;
    const int64_t *cand;
    int64_t n;
    int H, W, R, count_cov;
    const uint32_t *cum;
    uint32_t *g0, *sp, *sorig, *slo, *shi;
    unsigned long long *cov;
    int64_t nch;
    long long blk0[kPrepPhases];
};
struct PrepBatch {
    PrepJob job[kSiteMaxJobs];
    int njobs;
};
__global__ void __launch_bounds__(kRankChunk) k_site_prep_batch(const __grid_constant__ PrepBatch B, int phase) {
    __shared__ uint64_t sk[kRankChunk];
    int j = 0;
    while (j + 1 < B.njobs && B.job[j + 1].blk0[phase] <= (long long)blockIdx.x) ++j;
    const PrepJob &J = B.job[j];
    const int64_t b = (int64_t)blockIdx.x - J.blk0[phase];
    const int64_t HW = (int64_t)J.H * J.W;
    if (phase == 0) {
        if (b == 0 && threadIdx.x == 0 && J.count_cov) *J.cov = 0ull;
        site_gain_warp(J.bm, J.cand, J.n, J.H, J.W, J.R, J.cum, J.g0, b * (blockDim.x / 32) + (threadIdx.x >> 5));
    } else if (phase == 1) {
        if (b < J.nch) {
            rank_chunk(J.cand, J.n, HW, (uint64_t *)J.slo, J.sp, b, sk);
        } else if (J.count_cov) {  // popcount of the starting cumulative viewshed
            const int64_t nw = (int64_t)J.H * ((J.W + 31) / 32);
            unsigned long long v = 0;
            for (int64_t i = (b - J.nch) * blockDim.x + threadIdx.x; i < nw; i += (int64_t)kCovBlocks * blockDim.x)
                v += __popc(J.cum[i]);
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if ((threadIdx.x & 31) == 0 && v) atomicAdd(J.cov, v);
        }
    } else if (phase == 2) {
        rank_cross((const uint64_t *)J.slo, J.n, J.sp, b % J.nch, b / J.nch, sk);
    } else {
        const int64_t i = b * blockDim.x + threadIdx.x;
        if (i < J.n) {
            if (phase == 3) J.sorig[J.sp[i]] = (uint32_t)i;
            else if (phase == 4) J.sp[i] = (uint32_t)(slot_key(J.cand, J.sorig[i], HW) >> 32);
        }
        if (phase == 5) site_band(J.sp, J.n, J.W, J.R, J.slo, J.shi, i);
    }
}

// ------------------------------------------------------------------ lazy greedy
// For calls whose gains or windows do not fit in one cluster's shared memory
// (the paper's own regime: R = 1000, ~386,000 candidates, 512 KB bitmaps),
// one CTA runs the paper's lazy evaluation (Sec. "The multiple transmitter
// siting process", Site: a candidate cannot gain more later than it gains
// now).  Gains live in global memory as upper bounds with a flag saying that
// the bound is exact for the current C.  A table of per-block maxima of the
// keys (bound, lowest post, lowest index) sits in shared memory.  Each round
// takes the table's best candidate: when its bound is exact it is the true
// argmax -- every other bound is at least its candidate's gain -- and is
// accepted; otherwise its gain is evaluated over its window and the round
// repeats.  Accepting ORs the winner's window into C and clears the flag of
// every candidate whose window can meet the winner's (Chebyshev distance of
// the posts <= 2R), found through a grid of cells of side >= 2R that buckets
// the candidates, so a bound stays exact as long as nothing near it changes.
struct LazyParams {
    const uint32_t *bm;
    const int64_t *cand;
    int n, H, W, R, PR, words, WWc;
    int n_obs;
    long long need;
    int64_t *chosen, *gains;
    uint32_t *cum;
    int32_t *n_chosen;
    uint32_t *g;             // [n] gain bounds (initialised with the exact gains)
    uint8_t *fresh;          // [n] 1 = bound exact for the current C
    int bs, nb;              // candidates per block of the maxima table, blocks
    const uint32_t *cstart;  // [ncell + 1] first item of each cell
    const uint32_t *citems;  // candidate indices grouped by cell
    int cs, ncx, ncy;        // cell side (>= 2R), cells per row / column
    const unsigned long long *covered0;
    // options of vs_site_ex (k_site_lazy_grid only)
    const int16_t *z;        // terrain for the intervisibility constraint, or null
    long long zpitch;
    int ht;                  // antenna height above the post (both ends)
    uint8_t *elig;           // [n] intervisible with a transmitter chosen in this call
    const uint8_t *weight;   // receiver weights H x W (pitch W), or null = 1 each
    const unsigned long long *wsum;  // [2]: total weight, weight already covered
    double target;           // weighted coverage stop (<= 0: off)
    // failure-path test (VS_TUNE_SITE_BARRIER_TEST): CTA 1 skips its arrival at
    // the first grid barrier, and every barrier wait gives up after bar_polls
    // polls (0 = the library's default limit)
    int bar_skip;
    unsigned bar_polls;
};

__global__ void k_lazy_count(const int64_t *__restrict__ cand, int n, int H, int W, int cs, int ncx,
                             uint32_t *__restrict__ counts) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int64_t p = cand[c];
    if (p < 0 || p >= (int64_t)H * W) return;
    const int x = (int)(p % W), y = (int)(p / W);
    atomicAdd(&counts[(y / cs) * ncx + x / cs], 1u);
}

// exclusive scan of the cell counts (one CTA), copied to the scatter cursors
// (counts and cursor may be the same array: each entry is read and written by one thread)
__global__ void __launch_bounds__(1024) k_lazy_scan(const uint32_t *counts, int ncell, uint32_t *cstart,
                                                    uint32_t *cursor) {
    __shared__ uint32_t s_w[32];
    __shared__ uint32_t s_carry;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < ncell; base += 1024) {
        const int i = base + tid;
        const uint32_t v = i < ncell ? counts[i] : 0u;
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += u;
        }
        if (lane == 31) s_w[wid] = x;
        __syncthreads();
        if (wid == 0) {
            uint32_t y = s_w[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, y, o);
                if (lane >= o) y += u;
            }
            s_w[lane] = y;
        }
        __syncthreads();
        const uint32_t excl = s_carry + (wid ? s_w[wid - 1] : 0u) + x - v;
        if (i < ncell) { cstart[i] = excl; cursor[i] = excl; }
        __syncthreads();
        if (tid == 1023) s_carry = excl + v;
        __syncthreads();
    }
    if (tid == 0) cstart[ncell] = s_carry;
}

__global__ void k_lazy_scatter(const int64_t *__restrict__ cand, int n, int H, int W, int cs, int ncx,
                               uint32_t *__restrict__ cursor, uint32_t *__restrict__ citems) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int64_t p = cand[c];
    if (p < 0 || p >= (int64_t)H * W) return;
    const int x = (int)(p % W), y = (int)(p / W);
    citems[atomicAdd(&cursor[(y / cs) * ncx + x / cs], 1u)] = (uint32_t)c;
}

__device__ __forceinline__ uint64_t lazy_key(uint32_t g, int64_t p) {
    return ((uint64_t)g << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)p);
}

// block-wide argmax of (key, index): larger key, then lower index
__device__ __forceinline__ void lazy_block_best(uint64_t &k, int &c, uint64_t *s_k, int *s_c) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t k2 = __shfl_xor_sync(0xffffffffu, k, o);
        const int c2 = __shfl_xor_sync(0xffffffffu, c, o);
        if (ki_better(k2, c2, k, c)) { k = k2; c = c2; }
    }
    if (lane == 0) { s_k[wid] = k; s_c[wid] = c; }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        k = lane < nw ? s_k[lane] : 0ull;
        c = lane < nw ? s_c[lane] : 0x7fffffff;
        for (int o = 16; o > 0; o >>= 1) {
            const uint64_t k2 = __shfl_xor_sync(0xffffffffu, k, o);
            const int c2 = __shfl_xor_sync(0xffffffffu, c, o);
            if (ki_better(k2, c2, k, c)) { k = k2; c = c2; }
        }
        if (lane == 0) { s_k[32] = k; s_c[32] = c; }
    }
    __syncthreads();
    k = s_k[32];
    c = s_c[32];
    __syncthreads();  // s_k / s_c reused by the next call
}

// this thread's share of popcount(V_c AND NOT C) over c's window clipped to
// the grid; with commit, C |= V_c.  The clipped window is walked as one flat
// range of (row, word) pairs, eight pairs per thread in flight.
template <bool WEIGHTS = false>
__device__ __forceinline__ unsigned lazy_window(const LazyParams &P, int c, int64_t p, bool commit,
                                                int part = 0, int nparts = 1) {
    constexpr int U = 8;
    const int R = P.R, PR = P.PR, WWc = P.WWc;
    const int cx = (int)(p % P.W), cy = (int)(p / P.W);
    const int gw0 = floordiv(cx - R, 32);
    const int r_lo = max(0, R - cy), r_hi = min(2 * R, P.H - 1 - cy + R);
    const int w_lo = max(0, -gw0), w_hi = min(PR - 1, WWc - 1 - gw0);
    const int nr = r_hi - r_lo + 1, nw = w_hi - w_lo + 1;
    const int total = nr * nw;
    const uint32_t *V = P.bm + (long long)c * P.words + (long long)r_lo * PR + w_lo;
    uint32_t *C = P.cum + (long long)(cy - R + r_lo) * WWc + (gw0 + w_lo);
    const int nt = blockDim.x;
    const int dr = nt / nw, dw = nt - dr * nw;
    // this part of the flat range: [i_begin, i_end)
    const int i_begin = (int)((long long)total * part / nparts);
    const int i_end = (int)((long long)total * (part + 1) / nparts);
    const int i0 = i_begin + threadIdx.x;
    int r = i0 / nw, w = i0 - r * nw;
    unsigned sum = 0;
    for (int i = i0; i < i_end; i += U * nt) {
        uint32_t v[U], cw[U];
        int off[U];
        int rr = r, ww = w;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            off[u] = -1;
            if (i + u * nt < i_end) {
                off[u] = rr * WWc + ww;
                v[u] = __ldg(V + rr * PR + ww);
                cw[u] = __ldcg(C + off[u]);  // L2: other CTAs of k_site_lazy_grid update C
            }
            ww += dw;
            rr += dr;
            if (ww >= nw) { ww -= nw; rr += 1; }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (off[u] < 0) continue;
            uint32_t d = v[u] & ~cw[u];
            if (commit && d) C[off[u]] = cw[u] | v[u];
            if (!WEIGHTS || !P.weight) {
                sum += __popc(d);
            } else {  // receiver weights of the newly covered posts
                const int row = off[u] / WWc, col32 = off[u] - row * WWc;
                const uint8_t *wr = P.weight + (long long)(cy - R + r_lo + row) * P.W + 32 * (gw0 + w_lo + col32);
                while (d) {
                    const int b = __ffs(d) - 1;
                    d &= d - 1;
                    sum += wr[b];
                }
            }
        }
        r = rr;
        w = ww;
    }
    return sum;
}

__device__ __forceinline__ unsigned lazy_block_sum(unsigned s, unsigned *s_u) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) s_u[wid] = s;
    __syncthreads();
    unsigned t = 0;
    for (int j = 0; j < (int)(blockDim.x >> 5); ++j) t += s_u[j];
    __syncthreads();
    return t;
}

// recompute the table entry of block b from the gains in global memory
__device__ __forceinline__ void lazy_refresh_block(const LazyParams &P, int b, uint64_t *bkey, int *bidx,
                                                   uint64_t *s_k, int *s_c) {
    uint64_t k = 0;
    int c = 0x7fffffff;
    const int e = min(P.n, (b + 1) * P.bs);
    for (int i = b * P.bs + threadIdx.x; i < e; i += blockDim.x) {
        const uint64_t ki = lazy_key(P.g[i], P.cand[i]);
        if (ki_better(ki, i, k, c)) { k = ki; c = i; }
    }
    lazy_block_best(k, c, s_k, s_c);
    if (threadIdx.x == 0) { bkey[b] = k; bidx[b] = c; }
    __syncthreads();
}

__global__ void __launch_bounds__(kSiteThreads, 1) k_site_lazy(const LazyParams P) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *bkey = (uint64_t *)smem;
    int *bidx = (int *)(bkey + P.nb);
    __shared__ uint64_t s_k[33];
    __shared__ int s_c[33];
    __shared__ unsigned s_u[32];
    __shared__ long long s_p;
    __shared__ int s_fresh;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

    // the table: warp per block
    for (int b = wid; b < P.nb; b += (int)(blockDim.x >> 5)) {
        uint64_t k = 0;
        int c = 0x7fffffff;
        const int e = min(P.n, (b + 1) * P.bs);
        for (int i = b * P.bs + lane; i < e; i += 32) {
            const uint64_t ki = lazy_key(P.g[i], P.cand[i]);
            if (ki_better(ki, i, k, c)) { k = ki; c = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const uint64_t k2 = __shfl_xor_sync(0xffffffffu, k, o);
            const int c2 = __shfl_xor_sync(0xffffffffu, c, o);
            if (ki_better(k2, c2, k, c)) { k = k2; c = c2; }
        }
        if (lane == 0) { bkey[b] = k; bidx[b] = c; }
    }
    __syncthreads();

    long long covered = P.need >= 0 ? (long long)*P.covered0 : 0;
    int t = 0;
    // between two acceptances each candidate is evaluated at most once, so the
    // rounds are bounded; the guard only stops a loop that broke that rule
    const long long max_rounds = (long long)P.n * ((long long)P.n_obs + 1) + 2ll * P.n_obs + 16;
    long long rounds = 0;
    while (t < P.n_obs && ++rounds <= max_rounds) {
        if (P.need >= 0 && covered >= P.need) break;
        uint64_t k = 0;
        int c = 0x7fffffff;
        for (int b = tid; b < P.nb; b += blockDim.x)
            if (ki_better(bkey[b], bidx[b], k, c)) { k = bkey[b]; c = bidx[b]; }
        lazy_block_best(k, c, s_k, s_c);
        if ((k >> 32) == 0) break;  // best gain 0: nothing left to cover
        if (tid == 0) { s_p = P.cand[c]; s_fresh = P.fresh[c]; }
        __syncthreads();
        const int64_t p = s_p;
        const int fresh = s_fresh;
        if (!fresh) {  // a stale bound: evaluate the gain and search again
            const unsigned gnew = lazy_block_sum(lazy_window(P, c, p, false), s_u);
            if (tid == 0) { P.g[c] = gnew; P.fresh[c] = 1; }
            __syncthreads();
            lazy_refresh_block(P, c / P.bs, bkey, bidx, s_k, s_c);
            continue;
        }
        const uint32_t gw = (uint32_t)(k >> 32);
        if (tid == 0) {
            P.chosen[t] = p;
            P.gains[t] = gw;
            P.g[c] = 0;  // all of its viewshed is covered now
        }
        lazy_window(P, c, p, true);
        covered += gw;
        __syncthreads();
        lazy_refresh_block(P, c / P.bs, bkey, bidx, s_k, s_c);
        // bounds that may have changed: candidates within Chebyshev distance 2R
        const int cx = (int)(p % P.W), cy = (int)(p / P.W), R2 = 2 * P.R;
        const int x0 = max(0, cx - R2) / P.cs, x1 = min(P.W - 1, cx + R2) / P.cs;
        const int y0 = max(0, cy - R2) / P.cs, y1 = min(P.H - 1, cy + R2) / P.cs;
        for (int yc = y0; yc <= y1; ++yc)
            for (int xc = x0; xc <= x1; ++xc) {
                const int cell = yc * P.ncx + xc;
                const uint32_t e = P.cstart[cell + 1];
                for (uint32_t j = P.cstart[cell] + tid; j < e; j += blockDim.x) {
                    const int c2 = (int)P.citems[j];
                    const int64_t p2 = P.cand[c2];
                    const int x2 = (int)(p2 % P.W), y2 = (int)(p2 / P.W);
                    if (c2 != c && abs(x2 - cx) <= R2 && abs(y2 - cy) <= R2) P.fresh[c2] = 0;
                }
            }
        __syncthreads();
        ++t;
    }
    if (tid == 0) *P.n_chosen = t;
}

// The lazy greedy on the whole GPU: one cooperative launch, one CTA per SM,
// each CTA owning a slice of the candidates.  A step is a fixed sequence of
// phases separated by grid barriers:
//   A  F = the largest key among exact (fresh) gains;
//   B  every stale candidate whose bound key is >= F goes on a work list --
//      only those can beat F, so after B..C the best key is an exact gain;
//   C  the CTAs evaluate the work list, one window per CTA at a time;
//   D  the largest key (bound, lowest post) and then the lowest index holding
//      it (duplicate posts) -- the winner, exactly the sequential argmax;
//   E  C |= V_winner (the window split over the CTAs), the winner's gain set
//      to 0, stale flags for the candidates within Chebyshev distance 2R.
// Arrays other CTAs write during the launch (gains, flags, work list, C) are
// read through L2 (ld.global.cg), never from a stale L1 line.
// Keys and counters of a step live in slots indexed by the step's parity; CTA
// 0 clears the other parity's slots during E.  Barrier waits are bounded: a
// wait that gives up raises an error flag every CTA checks after each
// barrier, and the call reports VS_ERR_TIMEOUT in *n_chosen.
struct LazyCtl {
    unsigned long long F[2];     // largest fresh key
    unsigned long long best[2];  // largest key after the evaluations
    unsigned widx[2];            // 0xFFFFFFFF - lowest index holding best
    unsigned nwork[2];           // work-list length
    unsigned next[2];            // work-list cursor
    unsigned bar_count;
    unsigned bar_gen;
    int err;
};
static_assert(sizeof(LazyCtl) <= 256, "control block fits its workspace slot");

// grid barrier (all CTAs of a cooperative launch); false when a wait gave up
__device__ __forceinline__ bool lazy_grid_sync(LazyCtl *ctl, unsigned &gen, int skip = 0, unsigned polls = 0) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        const unsigned g0 = gen;
        const uint32_t limit = polls ? polls : kWaitPolls;
        const bool arrive = !(skip && blockIdx.x == 1 && g0 == 0);
        if (arrive && atomicAdd(&ctl->bar_count, 1u) == gridDim.x - 1) {
            atomicExch(&ctl->bar_count, 0u);
            __threadfence();
            atomicAdd(&ctl->bar_gen, 1u);
        } else {
            uint32_t i = 0;
            while (*(volatile unsigned *)&ctl->bar_gen == g0) {
                if (++i > limit || *(volatile int *)&ctl->err) {
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        gen = g0 + 1;
        if (!ok) atomicExch(&ctl->err, 1);
        s_ok = ok && !*(volatile int *)&ctl->err;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long v, unsigned long long *s_red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v = u64max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) s_red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < (int)(blockDim.x >> 5) ? s_red[lane] : 0ull;
        for (int o = 16; o > 0; o >>= 1) v = u64max(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) s_red[32] = v;
    }
    __syncthreads();
    v = s_red[32];
    __syncthreads();
    return v;
}

// Transmitters a and b intervisible: the line between the antenna tops (both
// z + ht) clears the terrain interpolated between the two posts it passes
// between at every crossing -- the vix line-of-sight test with the receiver
// height set to ht (Sec. "Terrain visibility"; symmetric in a and b).  One
// thread walks the line; 32-bit values (|j * dz| < 2^31 for R <= 4096).
__device__ __forceinline__ bool tx_intervisible(const int16_t *z, long long pitch, int ax, int ay, int bx, int by,
                                                int ht) {
    const int dx = bx - ax, dy = by - ay;
    const int adx = abs(dx), ady = abs(dy);
    const bool xmaj = adx >= ady;
    const int D = xmaj ? adx : ady;
    if (D <= 1) return true;
    const int E = (int)z[(long long)ay * pitch + ax] + ht;
    const int ts = (int)z[(long long)by * pitch + bx] + ht - E;
    const int dmin = xmaj ? dy : dx;
    const int q = floordiv(dmin, D), rr = dmin - q * D;
    const long long ms = xmaj ? (dx > 0 ? 1 : -1) : (dy > 0 ? pitch : -pitch);
    const long long ns = xmaj ? pitch : 1;
    const int16_t *a = z + (long long)ay * pitch + ax;
    int f = 0;
    for (int j = 1; j < D; ++j) {
        f += rr;
        a += ms + q * ns;
        if (f >= D) { f -= D; a += ns; }
        const int z0 = a[0];
        const int z1 = f ? (int)a[ns] : z0;
        if (j * ts < (z0 - E) * D + (z1 - z0) * f) return false;
    }
    return true;
}

template <bool OPT>  // OPT: the options of vs_site_ex (eligibility, weights) are compiled in
__global__ void __launch_bounds__(kSiteThreads, 1) k_site_lazy_grid(const LazyParams P, LazyCtl *ctl,
                                                                   uint32_t *work) {
    __shared__ unsigned long long s_red[33];
    __shared__ unsigned s_u[32];
    __shared__ int s_item;
    const int tid = threadIdx.x, G = gridDim.x, b = blockIdx.x;
    const int lo = (int)((long long)P.n * b / G), hi = (int)((long long)P.n * (b + 1) / G);
    unsigned gen = 0;
    long long need = P.need;
    long long covered = need >= 0 ? (long long)*P.covered0 : 0;
    if (OPT && P.weight) {  // weighted coverage: the stop compares covered weight
        covered = (long long)P.wsum[1];
        need = -1;
        if (P.target > 0.0) {
            const double nd = P.target * (double)P.wsum[0];
            need = (long long)nd;
            if ((double)need < nd) need += 1;
        }
    }
    const bool con = OPT && P.z != nullptr;
    int t = 0;
    bool ok = true;
    for (; t < P.n_obs; ++t) {
        if (need >= 0 && covered >= need) break;
        const int par = t & 1;
        const bool free_pick = !con || t == 0;  // the first transmitter of the call is free
        // A: largest fresh key
        unsigned long long k = 0;
        for (int c = lo + tid; c < hi; c += blockDim.x)
            if ((free_pick || __ldcg(P.elig + c)) && __ldcg(P.fresh + c))
                k = u64max(k, lazy_key(__ldcg(P.g + c), P.cand[c]));
        k = block_max_u64(k, s_red);
        if (tid == 0 && k) atomicMax(&ctl->F[par], k);
        if (!(ok = lazy_grid_sync(ctl, gen, P.bar_skip, P.bar_polls))) break;
        const unsigned long long F = *(volatile unsigned long long *)&ctl->F[par];
        // B: stale bounds that may beat F
        for (int c = lo + tid; c < hi; c += blockDim.x)
            if ((free_pick || __ldcg(P.elig + c)) && !__ldcg(P.fresh + c) && lazy_key(__ldcg(P.g + c), P.cand[c]) >= F)
                work[atomicAdd(&ctl->nwork[par], 1u)] = (uint32_t)c;
        if (!(ok = lazy_grid_sync(ctl, gen, P.bar_skip, P.bar_polls))) break;
        const unsigned m = *(volatile unsigned *)&ctl->nwork[par];
        // C: evaluate them, one window per CTA at a time
        for (;;) {
            if (tid == 0) s_item = (int)atomicAdd(&ctl->next[par], 1u);
            __syncthreads();
            const int it = s_item;
            __syncthreads();
            if ((unsigned)it >= m) break;
            const int c = (int)__ldcg(work + it);
            const int64_t pc = P.cand[c];
            // a post outside the grid covers nothing (its bound may be the
            // unknown all-ones of weighted gains)
            const bool valid = pc >= 0 && pc < (int64_t)P.H * P.W;
            const unsigned gnew = valid ? lazy_block_sum(lazy_window<OPT>(P, c, pc, false), s_u) : 0u;
            if (tid == 0) { P.g[c] = gnew; P.fresh[c] = 1; }
        }
        if (!(ok = lazy_grid_sync(ctl, gen, P.bar_skip, P.bar_polls))) break;
        // D: the largest key, then the lowest index holding it
        k = 0;
        for (int c = lo + tid; c < hi; c += blockDim.x)
            if (free_pick || __ldcg(P.elig + c)) k = u64max(k, lazy_key(__ldcg(P.g + c), P.cand[c]));
        k = block_max_u64(k, s_red);
        if (tid == 0 && k) atomicMax(&ctl->best[par], k);
        if (!(ok = lazy_grid_sync(ctl, gen, P.bar_skip, P.bar_polls))) break;
        const unsigned long long best = *(volatile unsigned long long *)&ctl->best[par];
        if ((best >> 32) == 0) break;  // best gain 0 (or no eligible candidate): nothing left to cover
        for (int c = lo + tid; c < hi; c += blockDim.x)
            if ((free_pick || __ldcg(P.elig + c)) && lazy_key(__ldcg(P.g + c), P.cand[c]) == best) atomicMax(&ctl->widx[par], 0xFFFFFFFFu - (unsigned)c);
        if (!(ok = lazy_grid_sync(ctl, gen, P.bar_skip, P.bar_polls))) break;
        const int w = (int)(0xFFFFFFFFu - *(volatile unsigned *)&ctl->widx[par]);
        const int64_t pw = P.cand[w];
        const uint32_t gw = (uint32_t)(best >> 32);
        // E: accept
        lazy_window<OPT>(P, w, pw, true, b, G);
        const int cx = (int)(pw % P.W), cy = (int)(pw / P.W), R2 = 2 * P.R;
        const int x0 = max(0, cx - R2) / P.cs, x1 = min(P.W - 1, cx + R2) / P.cs;
        const int y0 = max(0, cy - R2) / P.cs, y1 = min(P.H - 1, cy + R2) / P.cs;
        const int gt = b * blockDim.x + tid, gs = G * blockDim.x;
        for (int yc = y0; yc <= y1; ++yc)
            for (int xc = x0; xc <= x1; ++xc) {
                const int cell = yc * P.ncx + xc;
                const uint32_t e = P.cstart[cell + 1];
                for (uint32_t j = P.cstart[cell] + gt; j < e; j += gs) {
                    const int c2 = (int)P.citems[j];
                    const int64_t p2 = P.cand[c2];
                    const int xx = (int)(p2 % P.W), yy = (int)(p2 / P.W);
                    if (c2 != w && abs(xx - cx) <= R2 && abs(yy - cy) <= R2) P.fresh[c2] = 0;
                    // intervisible with the new transmitter: eligible from now on
                    if (con && c2 != w && (xx - cx) * (xx - cx) + (yy - cy) * (yy - cy) <= P.R * P.R &&
                        tx_intervisible(P.z, P.zpitch, cx, cy, xx, yy, P.ht))
                        P.elig[c2] = 1;
                }
            }
        if (b == 0 && tid == 0) {
            P.chosen[t] = pw;
            P.gains[t] = gw;
            P.g[w] = 0;  // all of its viewshed is covered now
            const int q = par ^ 1;
            ctl->F[q] = 0; ctl->best[q] = 0; ctl->widx[q] = 0; ctl->nwork[q] = 0; ctl->next[q] = 0;
        }
        covered += gw;
        if (!(ok = lazy_grid_sync(ctl, gen, P.bar_skip, P.bar_polls))) break;
    }
    if (b == 0 && tid == 0) *P.n_chosen = ok ? t : VS_ERR_TIMEOUT;
}

static size_t site_smem_bytes(int slots, int words) {
    return (size_t)slots * 16 + (size_t)words * 4 + 16;
}

// largest cluster size (16, 8, ..., 1) that can be co-resident with this smem
static int pick_cluster(size_t smem) {
    for (int q : {16, 8, 4, 2, 1}) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(q);
        cfg.blockDim = dim3(kSiteThreads);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = q;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclus = 0;
        if (cudaOccupancyMaxActiveClusters(&nclus, k_site_loop, &cfg) == cudaSuccess && nclus >= 1)
            return q;
        cudaGetLastError();
    }
    return 0;
}

}  // namespace vs

using namespace vs;

static inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// cells of the lazy greedy's bucket grid: at most max(64, min(n, 65536))
static int64_t lazy_cell_cap(int64_t n) { return std::max<int64_t>(64, std::min<int64_t>(n, 65536)); }

extern "C" size_t vs_site_workspace(int64_t n, int32_t R) {
    (void)R;
    if (n < 0) return 0;
    // gains, sorted posts, order, band bounds (the lazy greedy: bounds, flags,
    // items by cell), plus the lazy greedy's cell starts and cursors
    return 5 * align256((size_t)n * 4) + 2 * align256((size_t)(lazy_cell_cap(n) + 1) * 4) + 256;
}

// lazy greedy: bucket the candidates and launch the loop
// the options of vs_site_ex, resolved on the host
struct LazyOpts {
    const int16_t *z;
    long long zpitch;
    int ht;
    const uint8_t *weight;
    double target;
    uint8_t *elig;
    unsigned long long *wsum;
};

static int site_lazy(const uint32_t *bm, const int64_t *cand, int64_t n, int32_t H, int32_t W, int32_t R,
                     int32_t n_obs, long long need, int64_t *chosen, int64_t *gains, uint32_t *cum,
                     int32_t *n_chosen, uint32_t *g0, void *ws, const unsigned long long *cov, cudaStream_t s,
                     const LazyOpts *opt = nullptr) {
    if (n >= (1ll << 31) - 1) return VS_ERR_RANGE;
    const size_t a4 = align256((size_t)n * 4);
    uint8_t *fresh = (uint8_t *)((char *)ws + a4);
    uint32_t *citems = (uint32_t *)((char *)ws + 2 * a4);
    const int64_t cap = lazy_cell_cap(n);
    // after the coverage counter (ws + 5 * a4, 8 of 256 bytes)
    uint32_t *cstart = (uint32_t *)((char *)ws + 5 * a4 + 256);
    uint32_t *cursor = (uint32_t *)((char *)cstart + align256((size_t)(cap + 1) * 4));
    // cell side: 2R, doubled until the grid has at most cap cells
    long long cs = 2ll * R;
    while (((H + cs - 1) / cs) * ((W + cs - 1) / cs) > cap) cs *= 2;
    const int ncx = (int)((W + cs - 1) / cs), ncy = (int)((H + cs - 1) / cs);
    const int ncell = ncx * ncy;
    // table blocks: at most 16384 entries (12 bytes each) in shared memory
    int bs = 256;
    while ((n + bs - 1) / bs > 16384) bs *= 2;
    const int nb = (int)((n + bs - 1) / bs);
    if (opt && opt->weight) {
        // weighted gains: every bound starts unknown (all ones) and stale, so
        // the first step evaluates every candidate
        VS_CUDA_TRY(cudaMemsetAsync(fresh, 0, (size_t)n, s));
        VS_CUDA_TRY(cudaMemsetAsync(g0, 0xFF, (size_t)n * 4, s));
    } else {
        VS_CUDA_TRY(cudaMemsetAsync(fresh, 1, (size_t)n, s));
    }
    VS_CUDA_TRY(cudaMemsetAsync(cursor, 0, (size_t)ncell * 4, s));
    const unsigned gb = (unsigned)((n + 255) / 256);
    k_lazy_count<<<gb, 256, 0, s>>>(cand, (int)n, H, W, (int)cs, ncx, cursor);
    vs::note_launch();
    VS_CUDA_TRY(cudaGetLastError());
    // counts -> starts, and the cursors (in place) for the scatter
    k_lazy_scan<<<1, 1024, 0, s>>>(cursor, ncell, cstart, cursor);
    vs::note_launch();
    VS_CUDA_TRY(cudaGetLastError());
    k_lazy_scatter<<<gb, 256, 0, s>>>(cand, (int)n, H, W, (int)cs, ncx, cursor, citems);
    vs::note_launch();
    VS_CUDA_TRY(cudaGetLastError());
    LazyParams L;
    L.bm = bm; L.cand = cand; L.n = (int)n; L.H = H; L.W = W; L.R = R;
    L.PR = words_per_row(R); L.words = (2 * R + 1) * L.PR; L.WWc = (W + 31) / 32;
    L.n_obs = n_obs; L.need = need; L.chosen = chosen; L.gains = gains; L.cum = cum; L.n_chosen = n_chosen;
    L.g = g0; L.fresh = fresh; L.bs = bs; L.nb = nb; L.cstart = cstart; L.citems = citems;
    L.cs = (int)cs; L.ncx = ncx; L.ncy = ncy; L.covered0 = cov;
    L.z = opt ? opt->z : nullptr;
    L.zpitch = opt ? opt->zpitch : 0;
    L.ht = opt ? opt->ht : 0;
    L.elig = opt ? opt->elig : nullptr;
    L.weight = opt ? opt->weight : nullptr;
    L.wsum = opt ? opt->wsum : nullptr;
    L.target = opt ? opt->target : 0.0;
    {
        const int bt = tune_get(VS_TUNE_SITE_BARRIER_TEST, R, 0);
        L.bar_skip = bt > 0 ? 1 : 0;
        L.bar_polls = bt > 0 ? (unsigned)bt : 0u;
    }
    if (opt || tune_get(VS_TUNE_SITE_LAZY, R, 0) != 2) {
        // the whole GPU: one CTA per SM in one cooperative launch
        int dev = 0, sms = 0, per = 0, coop = 0;
        VS_CUDA_TRY(cudaGetDevice(&dev));
        VS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        VS_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        const void *kern = opt ? (const void *)k_site_lazy_grid<true> : (const void *)k_site_lazy_grid<false>;
        VS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kSiteThreads, 0));
        if (coop && per >= 1 && sms >= 1) {
            LazyCtl *ctl = (LazyCtl *)((char *)ws + 4 * a4);
            uint32_t *work = (uint32_t *)((char *)ws + 3 * a4);
            VS_CUDA_TRY(cudaMemsetAsync(ctl, 0, sizeof(LazyCtl), s));
            void *args[] = {(void *)&L, (void *)&ctl, (void *)&work};
            VS_CUDA_TRY(cudaLaunchCooperativeKernel(kern, dim3((unsigned)sms), dim3(kSiteThreads), args, 0, s));
            vs::note_launch();
            return VS_OK;
        }
        if (opt) return VS_ERR_DEVICE;  // the options run on the grid kernel only
    }
    const size_t smem = (size_t)nb * 12 + 16;
    VS_CUDA_TRY(cudaFuncSetAttribute(k_site_lazy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_site_lazy<<<1, kSiteThreads, smem, s>>>(L);
    vs::note_launch();
    VS_CUDA_TRY(cudaGetLastError());
    return VS_OK;
}

extern "C" int vs_site_gains(const uint32_t *bm, const int64_t *cand, int64_t n, int32_t H,
                             int32_t W, int32_t R, const uint32_t *cum, uint32_t *gains_out,
                             vs_stream_t st) {
    if (n < 0) return VS_ERR_RANGE;
    if (n == 0) return VS_OK;
    if (!bm || !cand || !cum || !gains_out) return VS_ERR_ARG;
    if (H < 1 || W < 1 || R < 1 || R > kMaxR || (long long)H * W >= (1ll << 32) - 1) return VS_ERR_RANGE;
    int rc = check_device();
    if (rc) return rc;
    const int per = kGainThreads / 32;
    k_site_gains<<<(unsigned)((n + per - 1) / per), kGainThreads, 0, (cudaStream_t)st>>>(
        bm, cand, n, H, W, R, cum, gains_out);
    vs::note_launch();
    VS_CUDA_TRY(cudaGetLastError());
    return VS_OK;
}

static size_t site1_smem_bytes(int64_t n, int words) {
    return (size_t)((n + 3) & ~3) * 4 + (size_t)((words + 3) & ~3) * 4 + (size_t)kSiteThreads * 4;
}
static bool site1_fits(int64_t n, int words) {  // + ~33 KB of static shared memory
    return n < (1 << 30) && site1_smem_bytes(n, words) <= (size_t)kSmemLimit - 40 * 1024;
}

// leader cluster: the leader's gains plus a CTA's window rows of delta
static size_t siteq_smem_bytes(int64_t n, int R, int PR, int q) {
    const int rows = (2 * R + 1 + q - 1) / q;
    return (size_t)((n + 3) & ~3) * 4 + (size_t)rows * PR * 4 + 16;
}
static bool siteq_fits(size_t smem) {  // + ~37 KB of static shared memory
    return smem <= (size_t)kSmemLimit - 40 * 1024;
}
static bool siteq_launchable(size_t smem, int q) {
    if (cudaFuncSetAttribute(k_site_loopq, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(k_site_loopq, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(q);
    cfg.blockDim = dim3(kSiteThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = q;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclus = 0;
    if (cudaOccupancyMaxActiveClusters(&nclus, k_site_loopq, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return nclus >= 1;
}

// multi-winner leader cluster of q CTAs (q - 1 workers): VS_OK when launched,
// a negative code on a CUDA error, 1 when the call does not fit it
static int launch_site_multi(const Site1Params &Q1, int q, unsigned long long *stats, cudaStream_t s) {
    if (q < 2 || q > 16) return 1;
    const int nrow = (2 * Q1.R + 1 + (q - 1) - 1) / (q - 1);
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_site_multi) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    const long long budget = (long long)kSmemLimit - (long long)fa.sharedSizeBytes - 256;
    const long long lead = (long long)((Q1.n + 3) & ~3) * 4 + (long long)kMultiList * 8;
    const long long per = (long long)nrow * Q1.PR * 4;
    const long long fixed = (long long)(kMultiList + 4) * 4 + (long long)kMultiList * 4;
    if (lead > budget || per <= 0 || budget - fixed < per) return 1;
    const int Lmax = (int)std::min<long long>(kMultiMaxL, (budget - fixed) / per);
    const size_t dyn = (size_t)std::max(lead, fixed + (long long)Lmax * per);
    if (cudaFuncSetAttribute(k_site_multi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess ||
        cudaFuncSetAttribute(k_site_multi, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(q);
    cfg.blockDim = dim3(kSiteThreads);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = q;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclus = 0;
    if (cudaOccupancyMaxActiveClusters(&nclus, k_site_multi, &cfg) != cudaSuccess || nclus < 1) {
        cudaGetLastError();
        return 1;
    }
    SiteMParams M;
    M.b = Q1;
    M.Lmax = Lmax;
    M.nrow = nrow;
    M.stats = stats;
    VS_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_site_multi, M));
    vs::note_launch();
    return VS_OK;
}

static int site_impl(const uint32_t *bm, const int64_t *cand, int64_t n, int32_t H, int32_t W,
                     int32_t R, int32_t n_obs, double coverage_target, int64_t *chosen,
                     int64_t *gains, uint32_t *cum, int32_t *n_chosen, void *ws,
                     size_t ws_bytes, vs_stream_t st, Site1Params *job_out, size_t *smem_out) {
    if (n < 0 || n_obs < 0) return VS_ERR_RANGE;
    if (!cum || !n_chosen || (n > 0 && (!bm || !cand)) || (n_obs > 0 && (!chosen || !gains)))
        return VS_ERR_ARG;
    if (H < 1 || W < 1 || H > 65535 || W > 65535 || R < 1 || R > kMaxR) return VS_ERR_RANGE;
    if (ws_bytes < vs_site_workspace(n, R) || !ws) return VS_ERR_WS;
    int rc = check_device();
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)st;

    SiteParams P;
    P.bm = bm; P.cand = cand; P.n = n; P.H = H; P.W = W; P.R = R;
    P.PR = words_per_row(R); P.words = (2 * R + 1) * P.PR; P.WWc = (W + 31) / 32;
    P.n_obs = n_obs;
    P.chosen = chosen; P.gains = gains; P.cum = cum; P.n_chosen = n_chosen;
    const size_t a4 = align256((size_t)n * 4);
    uint32_t *g0 = (uint32_t *)ws;
    uint32_t *sp = (uint32_t *)((char *)ws + a4);
    uint32_t *sorig = (uint32_t *)((char *)ws + 2 * a4);
    uint32_t *slo = (uint32_t *)((char *)ws + 3 * a4);
    uint32_t *shi = (uint32_t *)((char *)ws + 4 * a4);
    unsigned long long *cov = (unsigned long long *)((char *)ws + 5 * a4);
    P.gain0 = g0;
    P.covered0 = cov;
    P.need = -1;
    if (coverage_target > 0.0) {
        const double need = coverage_target * (double)H * (double)W;
        long long nn = (long long)need;
        if ((double)nn < need) nn += 1;
        P.need = nn;
        VS_CUDA_TRY(cudaMemsetAsync(cov, 0, 8, s));
        const int64_t nw = (int64_t)H * P.WWc;
        k_cum_popcount<<<4 * 152, 256, 0, s>>>(cum, nw, cov);
        vs::note_launch();
        VS_CUDA_TRY(cudaGetLastError());
    }
    if (n > 0 && (rc = vs_site_gains(bm, cand, n, H, W, R, cum, g0, st))) return rc;
    if (!job_out && n > 0 && tune_get(VS_TUNE_SITE_LAZY, R, 0) == 1)
        return site_lazy(bm, cand, n, H, W, R, n_obs, P.need, chosen, gains, cum, n_chosen, g0, ws, cov, s);

    // one CTA, or a leader cluster, when every gain fits in one CTA's shared
    // memory; the tuning table picks the cluster size (0 = 8 CTAs, 1 = one CTA)
    const int qtune = job_out ? 1 : tune_get(VS_TUNE_SITE_CLUSTER, R, 0);
    const size_t smem1 = site1_smem_bytes(n, P.words);
    if (n > 0 && site1_fits(n, P.words)) {
        {   // slot order (sp doubles as the rank array, slo..shi as the key buffer)
            const unsigned nch = (unsigned)((n + kRankChunk - 1) / kRankChunk);
            uint64_t *keys = (uint64_t *)slo;
            k_rank_chunks<<<nch, kRankChunk, 0, s>>>(cand, n, (int64_t)H * W, keys, sp);
            vs::note_launch();
            VS_CUDA_TRY(cudaGetLastError());
            if (nch > 1) {
                k_rank_cross<<<dim3(nch, nch), kRankChunk, 0, s>>>(keys, n, sp);
                vs::note_launch();
                VS_CUDA_TRY(cudaGetLastError());
            }
            k_rank_scatter<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(sp, n, sorig);
            vs::note_launch();
            VS_CUDA_TRY(cudaGetLastError());
            k_rank_posts<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(cand, sorig, n, (int64_t)H * W, sp);
            vs::note_launch();
            VS_CUDA_TRY(cudaGetLastError());
        }
        k_site_bands<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(sp, n, W, R, slo, shi);
        vs::note_launch();
        VS_CUDA_TRY(cudaGetLastError());
        Site1Params Q1;
        Q1.bm = bm; Q1.n = (int)n; Q1.H = H; Q1.W = W; Q1.R = R; Q1.PR = P.PR; Q1.words = P.words;
        Q1.WWc = P.WWc; Q1.n_obs = n_obs; Q1.need = P.need; Q1.chosen = chosen; Q1.gains = gains;
        Q1.cum = cum; Q1.n_chosen = n_chosen; Q1.gain0 = g0; Q1.sp = sp; Q1.sorig = sorig;
        Q1.slo = slo; Q1.shi = shi; Q1.covered0 = cov;
        Q1.vec_rows = (P.PR % 4 == 0 && ((uintptr_t)bm & 15) == 0) ? 1 : 0;
        Q1.gbuf = nullptr;
        if (job_out) {  // batched call: the caller launches the loop
            *job_out = Q1;
            *smem_out = smem1;
            return VS_OK;
        }
        // leader cluster: bitmap rows must be whole 16-byte vectors
        const int qc = (qtune == 0) ? 8 : qtune;
        if (qc >= 2 && Q1.vec_rows && tune_get(VS_TUNE_SITE_MULTI, R, 0) != 1 &&
            (uint64_t)n * (uint64_t)P.words < (1ull << 32)) {
            // three counters of the loop in the workspace's spare bytes, after
            // the coverage count (diagnostics, read by nothing in the library).
            // Untuned, a 16-CTA cluster is tried first: more workers shorten a
            // round's refresh (14.1 ms against 14.8 ms for 4096 steps over
            // 40,000 candidates at R = 100); where it cannot be scheduled, 8.
            int mrc = 1;
            if (qtune == 0) mrc = launch_site_multi(Q1, 16, cov + 1, s);
            if (mrc > 0) mrc = launch_site_multi(Q1, qc, cov + 1, s);
            if (mrc <= 0) return mrc;  // launched, or a CUDA error; > 0: does not fit
        }
        if (qc >= 2 && Q1.vec_rows && (uintptr_t)cum % 16 == 0) {
            const size_t smemq = siteq_smem_bytes(n, R, P.PR, qc);
            if (siteq_fits(smemq) && siteq_launchable(smemq, qc)) {
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3(qc);
                cfg.blockDim = dim3(kSiteThreads);
                cfg.dynamicSmemBytes = smemq;
                cfg.stream = s;
                cudaLaunchAttribute at[1];
                at[0].id = cudaLaunchAttributeClusterDimension;
                at[0].val.clusterDim.x = qc;
                at[0].val.clusterDim.y = 1;
                at[0].val.clusterDim.z = 1;
                cfg.attrs = at;
                cfg.numAttrs = 1;
                VS_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_site_loopq, Q1));
                vs::note_launch();
                return VS_OK;
            }
        }
        VS_CUDA_TRY(cudaFuncSetAttribute(k_site_loop1, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem1));
        k_site_loop1<<<1, kSiteThreads, smem1, s>>>(Q1);
        vs::note_launch();
        VS_CUDA_TRY(cudaGetLastError());
        return VS_OK;
    }
    if (job_out) return VS_ERR_RANGE;  // too many candidates for one CTA: not batchable

    // choose the cluster: largest Q whose slots fit in shared memory
    int Q = 0, slots = 0;
    size_t smem = 0;
    VS_CUDA_TRY(cudaFuncSetAttribute(k_site_loop, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    for (int q : {16, 8, 4, 2, 1}) {
        const int sl = (int)std::max<int64_t>(1, (n + q - 1) / q);
        const size_t b = site_smem_bytes(sl, P.words);
        if (b > (size_t)kSmemLimit - 2048) continue;
        VS_CUDA_TRY(cudaFuncSetAttribute(k_site_loop, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b));
        const int qq = pick_cluster(b);
        if (qq >= q) { Q = q; slots = sl; smem = b; break; }
    }
    if (Q == 0)  // neither the gains nor the windows fit: the lazy greedy
        return site_lazy(bm, cand, n, H, W, R, n_obs, P.need, chosen, gains, cum, n_chosen, g0, ws, cov, s);
    P.slots = slots;

    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(Q);
    cfg.blockDim = dim3(kSiteThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = Q;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    VS_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_site_loop, P));
    vs::note_launch();
    return VS_OK;
}

extern "C" int vs_site(const uint32_t *bm, const int64_t *cand, int64_t n, int32_t H, int32_t W,
                       int32_t R, int32_t n_obs, double coverage_target, int64_t *chosen,
                       int64_t *gains, uint32_t *cum, int32_t *n_chosen, void *ws,
                       size_t ws_bytes, vs_stream_t st) {
    return site_impl(bm, cand, n, H, W, R, n_obs, coverage_target, chosen, gains, cum, n_chosen, ws,
                     ws_bytes, st, nullptr, nullptr);
}

// out[0] += total receiver weight, out[1] += weight of the posts set in cum
__global__ void k_weight_sums(const uint32_t *__restrict__ cum, const uint8_t *__restrict__ weight, int H, int W,
                              unsigned long long *out) {
    const int WWc = (W + 31) / 32;
    const long long nw = (long long)H * WWc, np = (long long)H * W;
    unsigned long long tot = 0, cov = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += (long long)gridDim.x * blockDim.x)
        tot += weight[i];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += (long long)gridDim.x * blockDim.x) {
        uint32_t u = cum[i];
        const long long y = i / WWc, gw = i - y * WWc;
        while (u) {
            const int b = __ffs(u) - 1;
            u &= u - 1;
            if (32 * gw + b < W) cov += weight[y * W + 32 * gw + b];
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        tot += __shfl_xor_sync(0xffffffffu, tot, o);
        cov += __shfl_xor_sync(0xffffffffu, cov, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (tot) atomicAdd(&out[0], tot);
        if (cov) atomicAdd(&out[1], cov);
    }
}

extern "C" size_t vs_site_ex_workspace(int64_t n, int32_t R) {
    if (n < 0) return 0;
    return vs_site_workspace(n, R) + align256((size_t)n) + 256;  // + eligibility flags, weight sums
}

extern "C" int vs_site_ex(const uint32_t *bm, const int64_t *cand, int64_t n, int32_t H, int32_t W, int32_t R,
                          int32_t n_obs, double coverage_target, const vs_site_options *opt, int64_t *chosen,
                          int64_t *gains, uint32_t *cum, int32_t *n_chosen, void *ws, size_t ws_bytes,
                          vs_stream_t st) {
    const bool con = opt && opt->terrain.z;
    const bool wtd = opt && opt->weight;
    if (!con && !wtd)
        return vs_site(bm, cand, n, H, W, R, n_obs, coverage_target, chosen, gains, cum, n_chosen, ws, ws_bytes, st);
    if (n < 0 || n_obs < 0) return VS_ERR_RANGE;
    if (!cum || !n_chosen || (n > 0 && (!bm || !cand)) || (n_obs > 0 && (!chosen || !gains))) return VS_ERR_ARG;
    if (H < 1 || W < 1 || H > 65535 || W > 65535 || R < 1 || R > kMaxR) return VS_ERR_RANGE;
    if (n >= (1ll << 31) - 1) return VS_ERR_RANGE;
    if (con) {
        int rc = check_grid(opt->terrain);
        if (rc) return rc;
        if (opt->terrain.H != H || opt->terrain.W != W) return VS_ERR_ARG;
        if (opt->ht < -100000 || opt->ht > 100000) return VS_ERR_RANGE;
    }
    if (wtd && (long long)(2 * R + 1) * (2 * R + 1) * 255 >= (1ll << 32)) return VS_ERR_RANGE;  // 32-bit gains
    if (!ws || ws_bytes < vs_site_ex_workspace(n, R)) return VS_ERR_WS;
    int rc = check_device();
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)st;
    if (n == 0) {
        VS_CUDA_TRY(cudaMemsetAsync(n_chosen, 0, 4, s));
        return VS_OK;
    }
    const size_t a4 = align256((size_t)n * 4);
    uint32_t *g0 = (uint32_t *)ws;
    unsigned long long *cov = (unsigned long long *)((char *)ws + 5 * a4);
    const size_t base = vs_site_workspace(n, R);
    LazyOpts o;
    o.z = con ? opt->terrain.z : nullptr;
    o.zpitch = con ? opt->terrain.pitch : 0;
    o.ht = con ? opt->ht : 0;
    o.weight = wtd ? opt->weight : nullptr;
    o.target = coverage_target;
    o.elig = (uint8_t *)((char *)ws + base);
    o.wsum = (unsigned long long *)((char *)ws + base + align256((size_t)n));
    VS_CUDA_TRY(cudaMemsetAsync(o.elig, 0, (size_t)n, s));
    long long need = -1;
    if (wtd) {
        VS_CUDA_TRY(cudaMemsetAsync(o.wsum, 0, 16, s));
        k_weight_sums<<<4 * 152, 256, 0, s>>>(cum, o.weight, H, W, o.wsum);
        vs::note_launch();
        VS_CUDA_TRY(cudaGetLastError());
    } else {
        if (coverage_target > 0.0) {
            const double nd = coverage_target * (double)H * (double)W;
            need = (long long)nd;
            if ((double)need < nd) need += 1;
            VS_CUDA_TRY(cudaMemsetAsync(cov, 0, 8, s));
            k_cum_popcount<<<4 * 152, 256, 0, s>>>(cum, (int64_t)H * ((W + 31) / 32), cov);
            vs::note_launch();
            VS_CUDA_TRY(cudaGetLastError());
        }
        if ((rc = vs_site_gains(bm, cand, n, H, W, R, cum, g0, st))) return rc;
    }
    return site_lazy(bm, cand, n, H, W, R, n_obs, need, chosen, gains, cum, n_chosen, g0, ws, cov, s, &o);
}

// a batch job whose gains do not fit one CTA's shared memory keeps them in
// global memory, after its workspace
static bool site_batch_global(int64_t n, int R) {
    return n > 0 && !site1_fits(n, (2 * R + 1) * words_per_row(R));
}

extern "C" size_t vs_site_batch_workspace(const vs_site_job *jobs, int32_t n_jobs) {
    if (!jobs || n_jobs < 0) return 0;
    size_t t = 0;
    for (int i = 0; i < n_jobs; ++i) {
        t += align256(vs_site_workspace(jobs[i].n, jobs[i].R));
        if (site_batch_global(jobs[i].n, jobs[i].R)) t += align256((size_t)jobs[i].n * 4);
    }
    return t + 256;
}

extern "C" int vs_site_batch(const vs_site_job *jobs, int32_t n_jobs, void *ws, size_t ws_bytes,
                             vs_stream_t st) {
    if (n_jobs < 0 || n_jobs > kSiteMaxJobs) return VS_ERR_RANGE;
    if (n_jobs == 0) return VS_OK;
    if (!jobs) return VS_ERR_ARG;
    if (!ws || ws_bytes < vs_site_batch_workspace(jobs, n_jobs)) return VS_ERR_WS;
    int rc = check_device();
    if (rc) return rc;
    static Site1Batch B;
    static PrepBatch PB;
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    memset(&B, 0, sizeof(B));
    memset(&PB, 0, sizeof(PB));
    size_t smem = 0, off = 0;
    long long nblk[kPrepPhases] = {0, 0, 0, 0, 0, 0};
    for (int i = 0; i < n_jobs; ++i) {
        const vs_site_job &q = jobs[i];
        const int64_t n = q.n;
        if (n < 0 || q.n_obs < 0) return VS_ERR_RANGE;
        if (!q.cum || !q.n_chosen || (n > 0 && (!q.bm || !q.cand)) || (q.n_obs > 0 && (!q.chosen || !q.gains)))
            return VS_ERR_ARG;
        if (q.H < 1 || q.W < 1 || q.H > 65535 || q.W > 65535 || q.R < 1 || q.R > kMaxR) return VS_ERR_RANGE;
        if (n >= (1 << 30)) return VS_ERR_RANGE;
        char *wsj = (char *)ws + off;
        const size_t a4 = align256((size_t)n * 4);
        off += align256(vs_site_workspace(n, q.R));
        const bool global = site_batch_global(n, q.R);
        uint32_t *gbuf = nullptr;
        if (global) {
            gbuf = (uint32_t *)((char *)ws + off);
            off += align256((size_t)n * 4);
        }
        Site1Params &Q1 = B.job[i];
        const int PR = words_per_row(q.R), words = (2 * q.R + 1) * PR;
        Q1.bm = q.bm; Q1.n = (int)n; Q1.H = q.H; Q1.W = q.W; Q1.R = q.R; Q1.PR = PR; Q1.words = words;
        Q1.WWc = (q.W + 31) / 32; Q1.n_obs = q.n_obs; Q1.chosen = q.chosen; Q1.gains = q.gains;
        Q1.cum = q.cum; Q1.n_chosen = q.n_chosen;
        Q1.gain0 = (uint32_t *)wsj;
        Q1.sp = (uint32_t *)(wsj + a4);
        Q1.sorig = (uint32_t *)(wsj + 2 * a4);
        Q1.slo = (uint32_t *)(wsj + 3 * a4);
        Q1.shi = (uint32_t *)(wsj + 4 * a4);
        Q1.covered0 = (unsigned long long *)(wsj + 5 * a4);
        Q1.need = -1;
        if (q.coverage_target > 0.0) {
            const double need = q.coverage_target * (double)q.H * (double)q.W;
            long long nn = (long long)need;
            if ((double)nn < need) nn += 1;
            Q1.need = nn;
        }
        Q1.vec_rows = (PR % 4 == 0 && ((uintptr_t)q.bm & 15) == 0) ? 1 : 0;
        Q1.gbuf = gbuf;
        smem = std::max(smem, global ? site1_smem_bytes(0, words) : site1_smem_bytes(n, words));
        PrepJob &J = PB.job[i];
        J.bm = q.bm; J.cand = q.cand; J.n = n; J.H = q.H; J.W = q.W; J.R = q.R;
        J.count_cov = Q1.need >= 0 ? 1 : 0;
        J.cum = q.cum; J.g0 = (uint32_t *)Q1.gain0; J.sp = (uint32_t *)Q1.sp; J.sorig = (uint32_t *)Q1.sorig;
        J.slo = (uint32_t *)Q1.slo; J.shi = (uint32_t *)Q1.shi;
        J.cov = (unsigned long long *)Q1.covered0;
        J.nch = (n + kRankChunk - 1) / kRankChunk;
        const long long cnt[kPrepPhases] = {(n + 7) / 8, J.nch + (J.count_cov ? kCovBlocks : 0),
                                             J.nch > 1 ? J.nch * J.nch : 0, (n + 1023) / 1024, (n + 1023) / 1024,
                                             (n + 1023) / 1024};
        for (int ph = 0; ph < kPrepPhases; ++ph) {
            J.blk0[ph] = nblk[ph];
            nblk[ph] += cnt[ph];
        }
    }
    PB.njobs = n_jobs;
    cudaStream_t s = (cudaStream_t)st;
    // phases 0 (a warp per candidate, 8 per block) and 3..5 (one thread per
    // candidate) use 256 or 1024 threads; 1 and 2 one 1024-key chunk per block
    const int threads[kPrepPhases] = {256, 1024, 1024, 1024, 1024, 1024};
    // every step is launched (one idle block when no job has work in it), so
    // that the number of launches does not depend on the jobs
    for (int ph = 0; ph < kPrepPhases; ++ph) {
        if (nblk[ph] > 0x7fffffffll) return VS_ERR_RANGE;
        k_site_prep_batch<<<(unsigned)std::max(nblk[ph], 1ll), threads[ph], 0, s>>>(PB, ph);
        vs::note_launch();
        VS_CUDA_TRY(cudaGetLastError());
    }
    VS_CUDA_TRY(cudaFuncSetAttribute(k_site_loop1_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    k_site_loop1_batch<<<n_jobs, kSiteThreads, smem, s>>>(B);
    vs::note_launch();
    VS_CUDA_TRY(cudaGetLastError());
    return VS_OK;
}

// ------------------------------------------------------------------ vs_site without allocation
// A variant of vs_site for callers that cannot allocate device memory: its
// scratch lives in this file-scope device array instead of a caller-provided
// workspace.  Every GPU that loads the library holds the array until exit.
namespace {
constexpr size_t kSiteNoAllocBytes = 1u << 20;  // VS_SITE_NOALLOC_MAX_BYTES in vshed.h
static __device__ __align__(256) unsigned char g_site_scratch[kSiteNoAllocBytes];

// The array's device address is only valid in the context it was looked up
// in: a caller's cudaDeviceReset destroys the primary context, and the array
// may sit elsewhere in the next one.  So the cached address is tagged with the
// context's process-unique ID (cuCtxGetId) and looked up again when it changes.
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);
struct ScratchSlot {
    unsigned long long ctx_id;
    void *ptr;
};
std::mutex g_scratch_mu;
ScratchSlot g_scratch[64];  // per device ordinal

// ID of the calling thread's current context; false when none is current or
// the driver does not offer the query
bool current_ctx_id(unsigned long long *id) {
    static CtxGetCurrentFn get_cur = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) ==
                cudaSuccess && qa == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) ==
                cudaSuccess && qb == cudaDriverEntryPointSuccess) {
            get_cur = (CtxGetCurrentFn)a;
            get_id = (CtxGetIdFn)b;
        }
    });
    if (!get_cur || !get_id) return false;
    CUcontext ctx = nullptr;
    if (get_cur(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return get_id(ctx, id) == CUDA_SUCCESS;
}
}  // namespace

extern "C" int vs_site_noalloc(const uint32_t *bm, const int64_t *cand, int64_t n, int32_t H,
                               int32_t W, int32_t R, int32_t n_obs, double coverage_target,
                               int64_t *chosen, int64_t *gains, uint32_t *cum,
                               int32_t *n_chosen, vs_stream_t st) {
    if (n < 0 || R < 1 || R > kMaxR) return VS_ERR_RANGE;
    const size_t need = vs_site_workspace(n, R);
    if (need > kSiteNoAllocBytes) return VS_ERR_RANGE;  // too many candidates for the array
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return VS_ERR_DEVICE;
    void *scratch = nullptr;
    {
        // set-up per device (and again per context), with that device current:
        // the host-side name of the array is not a device address, so ask the
        // runtime for it
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        unsigned long long id = 0;
        const bool have_id = current_ctx_id(&id);
        ScratchSlot &sl = g_scratch[dev];
        if (!sl.ptr || (have_id && id != sl.ctx_id)) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_site_scratch) != cudaSuccess || !p) return VS_ERR_CUDA;
            unsigned long long id2 = 0;
            sl.ptr = p;
            sl.ctx_id = current_ctx_id(&id2) ? id2 : 0;  // the lookup made the context current
        }
        scratch = sl.ptr;
    }
    return vs_site(bm, cand, n, H, W, R, n_obs, coverage_target, chosen, gains, cum, n_chosen,
                   scratch, kSiteNoAllocBytes, st);
}
