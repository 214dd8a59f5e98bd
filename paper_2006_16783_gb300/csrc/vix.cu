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

static int vix_launch(vs_grid g, int32_t R, int32_t ht, int32_t hr, int32_t S, uint64_t seed,
                      uint8_t *vix_out, unsigned long long *steps, vs_stream_t st) {
    int rc = check_grid(g);
    if (rc) return rc;
    if (!vix_out) return VS_ERR_ARG;
    if (R < 1 || R > kMaxR || S < 0 || S > 255) return VS_ERR_RANGE;
    if (ht < -100000 || ht > 100000 || hr < -100000 || hr > 100000) return VS_ERR_RANGE;
    if ((rc = check_device())) return rc;

    VixParams P;
    P.H = g.H; P.W = g.W; P.R = R; P.ht = ht; P.hr = hr; P.S = S; P.seed = seed; P.out = vix_out;
    long long nr = 0;
    for (int dy = -R; dy <= R; ++dy) {
        long long v = (long long)R * R - (long long)dy * dy, s = (long long)std::sqrt((double)v);
        while (s * s > v) --s;
        while ((s + 1) * (s + 1) <= v) ++s;
        nr += 2 * s + 1;
    }
    P.NR = (int)(nr - 1);

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
    } else {
        VS_CUDA_TRY(cudaFuncSetAttribute(k_vix<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_vix<false><<<grid, kVixThreads, smem, (cudaStream_t)st>>>(gm.map, P);
    }
    VS_CUDA_TRY(cudaGetLastError());
    return VS_OK;
}

extern "C" int vs_vix(vs_grid g, int32_t R, int32_t ht, int32_t hr, int32_t S, uint64_t seed,
                      uint8_t *vix_out, vs_stream_t st) {
    return vix_launch(g, R, ht, hr, S, seed, vix_out, nullptr, st);
}

extern "C" int vs_vix_count(vs_grid g, int32_t R, int32_t ht, int32_t hr, int32_t S, uint64_t seed,
                            uint8_t *vix_out, uint64_t *los_steps, vs_stream_t st) {
    if (!los_steps) return VS_ERR_ARG;
    return vix_launch(g, R, ht, hr, S, seed, vix_out, (unsigned long long *)los_steps, st);
}
