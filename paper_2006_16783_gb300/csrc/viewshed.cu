// viewshed.cu -- Viewshed stage (Sec. "The multiple transmitter siting
// process", Viewshed): one CTA per candidate observer.
//
// The observer's ROI window (int16 posts) is staged into shared memory by TMA
// (cp.async.bulk.tensor, tensor map view [H][pitch/8][8]); the CTA's threads
// then walk the 8R rays to the square ring max(|dx|,|dy|) = R, keeping each
// ray's running horizon (the steepest interpolated crossing so far) as an
// exact rational (numerator over step), and OR visible cells into a
// shared-memory bitmap laid out exactly like the output.  When the window does
// not fit in shared memory it is processed in halves (rays by the sign of the
// ring cell's dy) or quadrants (signs of dx and dy); every ray stays inside
// its half / quadrant, so each pass stages only that part.
#include <algorithm>
#include <cstdlib>

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

template <typename T>
__global__ void __launch_bounds__(256) k_viewshed(const __grid_constant__ CUtensorMap tmap,
                                                  const VsParams P) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // TMA destinations must be 128-byte aligned: round the base up (the host
    // reserves 128 spare bytes)
    unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    const int R = P.R, PR = P.PR;
    const int WW = P.WG * 8;
    int16_t *win = (int16_t *)smem;
    const int win_elems = P.nbox * P.box_rows * WW;
    uint32_t *bms = (uint32_t *)(smem + ((win_elems * 2 + 127) & ~127));
    uint64_t *bar = (uint64_t *)(bms + ((P.words + 31) & ~31));
    __shared__ int red[8];
    __shared__ int s_fail;

    const int tid = threadIdx.x;
    const int64_t c = blockIdx.x;
    const int64_t p = P.cand[c];
    uint32_t *out = P.bm + c * (int64_t)P.words;
    if (p < 0 || p >= (int64_t)P.H * P.W) {  // invalid candidate: empty bitmap, area -1
        for (int i = tid; i < P.words; i += blockDim.x) out[i] = 0;
        if (tid == 0) P.area[c] = -1;
        return;
    }
    const int cx = (int)(p % P.W), cy = (int)(p / P.W);
    const int gw0 = floordiv(cx - R, 32);

    if (tid == 0) {
        mbar_init(bar, 1);
        s_fail = 0;
    }
    for (int i = tid; i < P.words; i += blockDim.x) bms[i] = 0;
    __syncthreads();

    const int nsec = P.nsplit;
    int eye = 0;
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
            const uint32_t bytes = (uint32_t)(P.nbox * P.box_rows * WW * 2);
            mbar_arrive_expect_tx(bar, bytes);
            for (int b = 0; b < P.nbox; ++b)
                tma_load_3d(win + (size_t)b * P.box_rows * WW, &tmap, 0, wx0 / 8,
                            wy0 + b * P.box_rows, bar);
        }
        if (!mbar_wait(bar, (uint32_t)(sec & 1))) s_fail = 1;
        __syncthreads();
        if (s_fail) {
            // give the copy in flight a second bounded chance to land before the
            // CTA leaves, then report the candidate as timed out
            mbar_wait(bar, (uint32_t)(sec & 1));
            break;
        }
        eye = (int)win[(cy - wy0) * WW + (cx - wx0)] + P.ht;

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
            const int minor_lim = xmaj ? P.H : P.W;
            const int minor_step = xmaj ? WW : 1;
            int f = 0, y0 = 0;
            T Hn = 0;
            int Hk = 0;
            for (int k = 1; k <= R; ++k) {
                f += rr;
                y0 += q;
                if (f >= R) { f -= R; y0 += 1; }
                const int rnd = y0 + (2 * f >= thr ? 1 : 0);
                const int gmaj = omaj + smaj * k;
                const int gmin = omin + rnd;
                const int gx = xmaj ? gmaj : gmin, gy = xmaj ? gmin : gmaj;
                if ((unsigned)gx >= (unsigned)P.W || (unsigned)gy >= (unsigned)P.H) break;
                if (k * k + rnd * rnd > R * R) break;
                const int zc = win[(gy - wy0) * WW + (gx - wx0)];
                const bool vis = (Hk == 0) || ((T)(zc + P.hr - eye) * R * Hk >= Hn * k);
                if (vis)
                    atomicOr(&bms[(gy - cy + R) * PR + ((gx >> 5) - gw0)], 1u << (gx & 31));
                const int m0 = omin + y0;
                if (f > 0 && (m0 < 0 || m0 + 1 >= minor_lim)) break;
                const int a0 = xmaj ? (m0 - wy0) * WW + (gmaj - wx0) : (gmaj - wy0) * WW + (m0 - wx0);
                const int z0 = win[a0];
                const int z1 = win[a0 + (f > 0 ? minor_step : 0)];
                const T num = (T)z0 * (R - f) + (T)z1 * f - (T)eye * R;
                if (Hk == 0 || num * Hk > Hn * k) { Hn = num; Hk = k; }
            }
        }
        __syncthreads();  // every read of this window done before the next pass overwrites it
    }

    if (tid == 0 && !s_fail) atomicOr(&bms[R * PR + ((cx >> 5) - gw0)], 1u << (cx & 31));
    __syncthreads();
    int cnt = 0;
    for (int i = tid; i < P.words; i += blockDim.x) {
        uint32_t w = s_fail ? 0u : bms[i];
        out[i] = w;
        cnt += __popc(w);
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((tid & 31) == 0) red[tid >> 5] = cnt;
    __syncthreads();
    if (tid == 0) {
        int a = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += red[w];
        P.area[c] = s_fail ? VS_ERR_TIMEOUT : a;
    }
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
    size_t words = (size_t)(2 * R + 1) * words_per_row(R);
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

extern "C" size_t vs_viewshed_workspace(int32_t R, int64_t n) {
    (void)R; (void)n;
    return 0;
}

extern "C" int vs_viewshed(vs_grid g, int32_t R, int32_t ht, int32_t hr, const int64_t *cand,
                           int64_t n, uint32_t *bm_out, int32_t *area_out, void *ws,
                           size_t ws_bytes, vs_stream_t st) {
    (void)ws; (void)ws_bytes;
    int rc = check_grid(g);
    if (rc) return rc;
    if (R < 1 || R > kMaxR) return VS_ERR_RANGE;
    if (ht < -100000 || ht > 100000 || hr < -100000 || hr > 100000) return VS_ERR_RANGE;
    if (n < 0 || n > 0x7fffffffll) return VS_ERR_RANGE;
    if (n == 0) return VS_OK;
    if (!cand || !bm_out || !area_out) return VS_ERR_ARG;
    if ((rc = check_device())) return rc;

    VsParams P;
    P.H = g.H; P.W = g.W; P.R = R; P.ht = ht; P.hr = hr;
    P.cand = cand; P.n = n; P.bm = bm_out; P.area = area_out;
    P.PR = words_per_row(R);
    P.words = (2 * R + 1) * P.PR;
    size_t smem = 0;
    if ((rc = vs_pick_split(R, &P.nsplit, &P.WG, &P.box_rows, &P.nbox, &smem))) return rc;
    GridMap gm;
    if ((rc = make_grid_map(&gm, g, P.WG, P.box_rows))) return rc;

    // 32-bit products are exact when (z range + |ht| + |hr|) * R^2 < 2^31
    const long long bound = (65535ll + std::abs(ht) + std::abs(hr)) * (long long)R * R;
    cudaStream_t s = (cudaStream_t)st;
    if (bound < (1ll << 31)) {
        VS_CUDA_TRY(cudaFuncSetAttribute(k_viewshed<int>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
        k_viewshed<int><<<(unsigned)n, 256, smem, s>>>(gm.map, P);
    } else {
        VS_CUDA_TRY(cudaFuncSetAttribute(k_viewshed<long long>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_viewshed<long long><<<(unsigned)n, 256, smem, s>>>(gm.map, P);
    }
    VS_CUDA_TRY(cudaGetLastError());
    return VS_OK;
}
