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
#include <mutex>

#include "vs_common.cuh"

namespace cg = cooperative_groups;

namespace vs {

constexpr int kSiteThreads = 1024;
constexpr int kGainThreads = 256;

// ------------------------------------------------------------------ dense gain pass
__global__ void __launch_bounds__(kGainThreads) k_site_gains(const uint32_t *__restrict__ bm,
                                                             const int64_t *__restrict__ cand,
                                                             int64_t n, int H, int W, int R,
                                                             const uint32_t *__restrict__ cum,
                                                             uint32_t *__restrict__ gains) {
    const int lane = threadIdx.x & 31;
    const int64_t c = (int64_t)blockIdx.x * (kGainThreads / 32) + (threadIdx.x >> 5);
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
    if (PR <= 32) {
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

extern "C" size_t vs_site_workspace(int64_t n, int32_t R) {
    (void)R;
    if (n < 0) return 0;
    return align256((size_t)n * 4) + 256;
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
    VS_CUDA_TRY(cudaGetLastError());
    return VS_OK;
}

extern "C" int vs_site(const uint32_t *bm, const int64_t *cand, int64_t n, int32_t H, int32_t W,
                       int32_t R, int32_t n_obs, double coverage_target, int64_t *chosen,
                       int64_t *gains, uint32_t *cum, int32_t *n_chosen, void *ws,
                       size_t ws_bytes, vs_stream_t st) {
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
    uint32_t *g0 = (uint32_t *)ws;
    unsigned long long *cov = (unsigned long long *)((char *)ws + align256((size_t)n * 4));
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
        VS_CUDA_TRY(cudaGetLastError());
    }
    if (n > 0 && (rc = vs_site_gains(bm, cand, n, H, W, R, cum, g0, st))) return rc;

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
    if (Q == 0) return VS_ERR_RANGE;
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
    return VS_OK;
}

// ------------------------------------------------------------------ vs_site without allocation
// A variant of vs_site for callers that cannot allocate device memory: its
// scratch lives in this file-scope device array instead of a caller-provided
// workspace.  Every GPU that loads the library holds the array until exit.
namespace {
constexpr size_t kSiteNoAllocBytes = 1u << 20;  // VS_SITE_NOALLOC_MAX_BYTES in vshed.h
static __device__ __align__(256) unsigned char g_site_scratch[kSiteNoAllocBytes];
std::mutex g_scratch_mu;
void *g_scratch_ptr[64];  // device address of g_site_scratch, per device ordinal
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
        // one-time set-up per device, with that device current: the host-side
        // name of the array is not a device address, so ask the runtime for it
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_site_scratch) != cudaSuccess || !p) return VS_ERR_CUDA;
            g_scratch_ptr[dev] = p;
        }
        scratch = g_scratch_ptr[dev];
    }
    return vs_site(bm, cand, n, H, W, R, n_obs, coverage_target, chosen, gains, cum, n_chosen,
                   scratch, kSiteNoAllocBytes, st);
}
