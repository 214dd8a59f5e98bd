// site_shard.cu -- the greedy site step with the candidates split over
// several ranks (Sec. "The multiple transmitter siting process", Site; the
// candidates of the paper's parallel Site loop divided between processes).
//
// Every rank holds its own candidates' bitmaps and exact gains and a full copy
// of the cumulative viewshed C.  A step: each rank's best key
// (gain << 32) | (0xFFFFFFFF - post) -> the largest over the ranks (an
// all-reduce of one 8-byte value, done by the caller) -> the winner's bitmap,
// broadcast by the rank that owns it -> vs_site_shard_step on every rank ORs
// it into C and lowers the gains of the rank's candidates whose window meets
// the winner's by popcount(V_c AND delta), delta = V_win AND NOT C before the
// update; the same launch returns the rank's new best key.  The winner is the
// sequential greedy's, ties included (posts are unique across ranks; equal
// posts on one rank are told apart by the lowest candidate index, which the
// owner resolves).
#include <algorithm>

#include "vs_common.cuh"

namespace vs {
namespace shard {

constexpr int kThreads = 256;

// delta = V_win AND NOT C over the winner's window (clipped to the grid), then
// C |= V_win; the rank's best key is reset for the refresh launch
__global__ void k_shard_window(const uint32_t *__restrict__ win_bm, int64_t win_post, int H, int W, int R,
                               uint32_t *__restrict__ cum, uint32_t *__restrict__ delta,
                               unsigned long long *__restrict__ best_key) {
    const int PR = words_per_row(R), words = (2 * R + 1) * PR, WWc = (W + 31) >> 5;
    if (blockIdx.x == 0 && threadIdx.x == 0) *best_key = 0ull;
    if (win_post < 0) return;
    const int wx = (int)(win_post % W), wy = (int)(win_post / W), gw0 = floordiv(wx - R, 32);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < words; e += gridDim.x * blockDim.x) {
        const int r = e / PR, w = e - r * PR, y = wy - R + r, gw = gw0 + w;
        uint32_t d = 0u;
        if (y >= 0 && y < H && gw >= 0 && gw < WWc) {
            uint32_t *cp = cum + (int64_t)y * WWc + gw;
            const uint32_t v = win_bm[e], old = *cp;
            d = v & ~old;
            if (d) *cp = old | v;
        }
        delta[e] = d;
    }
}

// per local candidate: lower its gain by what the winner newly covers inside
// its window (the winner's own candidate, on the rank that owns it, drops to
// 0), then the block's largest key into *best_key
__global__ void __launch_bounds__(kThreads) k_shard_refresh(const uint32_t *__restrict__ bm,
                                                            const int64_t *__restrict__ cand, int64_t n, int H,
                                                            int W, int R, uint32_t *__restrict__ gains,
                                                            const uint32_t *__restrict__ delta, int64_t win_post,
                                                            int64_t win_local,
                                                            unsigned long long *__restrict__ best_key) {
    __shared__ unsigned long long s_red[kThreads / 32];
    const int PR = words_per_row(R), WWc = (W + 31) >> 5;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long key = 0ull;
    if (c < n) {
        const int64_t p = cand[c];
        uint32_t g = gains[c];
        if (p >= 0 && p < (int64_t)H * W && g != 0u) {
            const int cx = (int)(p % W), cy = (int)(p / W);
            if (c == win_local) {
                g = 0u;
            } else if (win_post >= 0) {
                const int wx = (int)(win_post % W), wy = (int)(win_post / W);
                if (abs(cx - wx) <= 2 * R && abs(cy - wy) <= 2 * R) {
                    const int wgw0 = floordiv(wx - R, 32), cgw0 = floordiv(cx - R, 32);
                    const int ya = max(max(cy, wy) - R, 0), yb = min(min(cy, wy) + R, H - 1);
                    const int ga = max(max(cgw0, wgw0), 0), gb = min(min(cgw0, wgw0) + PR - 1, WWc - 1);
                    const uint32_t *V = bm + c * (int64_t)(2 * R + 1) * PR;
                    unsigned sum = 0;
                    for (int y = ya; y <= yb; ++y)
                        for (int gw = ga; gw <= gb; ++gw) {
                            const uint32_t d = delta[(y - wy + R) * PR + (gw - wgw0)];
                            if (d) sum += __popc(V[(y - cy + R) * PR + (gw - cgw0)] & d);
                        }
                    g -= sum;
                }
            }
            gains[c] = g;
            if (g) key = ((unsigned long long)g << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)p);
        } else if (c == win_local) {
            gains[c] = 0u;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
        key = k2 > key ? k2 : key;
    }
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = key;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long b = 0ull;
        for (int w = 0; w < kThreads / 32; ++w) b = s_red[w] > b ? s_red[w] : b;
        if (b) atomicMax(best_key, b);
    }
}

}  // namespace shard
}  // namespace vs

using namespace vs;

extern "C" size_t vs_site_shard_workspace(int32_t R) {
    if (R < 1 || R > kMaxR) return 0;
    return (size_t)(2 * R + 1) * words_per_row(R) * 4 + 256;
}

extern "C" int vs_site_shard_step(const uint32_t *bm, const int64_t *cand, int64_t n, int32_t H, int32_t W,
                                  int32_t R, uint32_t *gains, uint32_t *cum, const uint32_t *win_bm,
                                  int64_t win_post, int64_t win_local, uint64_t *best_key, void *ws,
                                  size_t ws_bytes, vs_stream_t st) {
    if (n < 0 || R < 1 || R > kMaxR) return VS_ERR_RANGE;
    if (H < 1 || W < 1 || H > 65535 || W > 65535) return VS_ERR_RANGE;
    if (!cum || !best_key || (n > 0 && (!bm || !cand || !gains))) return VS_ERR_ARG;
    if (win_post >= (int64_t)H * W || win_local >= n) return VS_ERR_RANGE;
    if (win_post >= 0 && !win_bm) return VS_ERR_ARG;
    if (!ws || ws_bytes < vs_site_shard_workspace(R)) return VS_ERR_WS;
    int rc = check_device();
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)st;
    uint32_t *delta = (uint32_t *)(((uintptr_t)ws + 15) & ~(uintptr_t)15);
    unsigned long long *bk = (unsigned long long *)best_key;
    const int words = (2 * R + 1) * words_per_row(R);
    shard::k_shard_window<<<(unsigned)std::min(64, (words + 255) / 256), 256, 0, s>>>(win_bm, win_post, H, W, R, cum,
                                                                                     delta, bk);
    vs::note_launch();
    VS_CUDA_TRY(cudaGetLastError());
    if (n > 0) {
        shard::k_shard_refresh<<<(unsigned)((n + shard::kThreads - 1) / shard::kThreads), shard::kThreads, 0, s>>>(
            bm, cand, n, H, W, R, gains, delta, win_post, win_local, bk);
        vs::note_launch();
        VS_CUDA_TRY(cudaGetLastError());
    }
    return VS_OK;
}
