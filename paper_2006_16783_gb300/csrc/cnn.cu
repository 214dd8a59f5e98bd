// cnn.cu -- learned candidate proposal: a 5-layer CNN that maps a 65x65
// elevation patch to a predicted visibility index (the Vix stage's ranking
// replaced by a learned one; the paper's Vix stage only ranks posts,
// Sec. "The multiple transmitter siting process", Vix).
//
// Network (fixed by this library; the paper specifies none):
//   x0 = bf16((z - mean(patch)) / 1000)                           65x65x1
//   conv1 3x3 s2 p1 1->32, bias, ReLU, bf16                      33x33x32
//   conv2 3x3 s2 p1 32->32                                       17x17x32
//   conv3 3x3 s2 p1 32->32                                        9x 9x32
//   conv4 3x3 s2 p1 32->32                                        5x 5x32
//   conv5 3x3 s1 p1 32->32                                        5x 5x32
//   global average pool -> fc 32->1 -> sigmoid
//
// Forward kernel: one persistent 128-thread CTA per SM works through patches
// entirely in shared memory.  Every convolution is an implicit GEMM on the
// 5th-generation tensor cores: tcgen05.mma kind::f16 (BF16 x BF16 -> FP32),
// M = 128 output pixels, N = 32 channels, K = 16 per instruction, the FP32
// accumulator in tensor memory (32 columns), read back with tcgen05.ld by
// the four warps (one TMEM lane quarter each) for the bias + ReLU + BF16
// epilogue.  Operands are read straight from shared memory through matrix
// descriptors (no swizzle, K-major 8x16-byte core matrices):
//   * A stride-2 layer's input is stored as four parity planes (even/odd row
//     x even/odd column) in blocks of 8 channels, each plane with a zero
//     border row/column and a row pitch of (output width + 1) pixels.  For
//     output pixel m = y*pitch + x, tap (ky,kx) reads plane
//     (ky != 1, kx != 1) at m + (ky != 0)*pitch + (kx != 0): every tap of a
//     128-pixel tile is one contiguous run of 16-byte rows, i.e. a plain
//     descriptor (leading offset = next 8-channel block, stride offset =
//     next 8 pixels).  The one junk column per row is discarded.
//   * The stride-1 last layer uses one plane with a border on all sides.
//   * The 1-channel first layer uses an explicit im2col tile (K = 9 taps
//     padded to 16).
#include <algorithm>

#include <cuda_bf16.h>

#include "vs_common.cuh"

namespace vs {
namespace cnn {

constexpr int kThreads = 512;  // 16 warps: 4 TMEM lane quarters x 4 channel blocks
constexpr int kPatch = 65;

// ---- master parameter layout (fp32): w_l [32][cin][3][3], b_l [32], fw [32], fb
constexpr int kNParams = 288 + 32 + 4 * (9216 + 32) + 33;
__host__ __device__ constexpr int off_w(int l) { return l == 0 ? 0 : 320 + (l - 1) * 9248; }
__host__ __device__ constexpr int off_b(int l) { return l == 0 ? 288 : 320 + (l - 1) * 9248 + 9216; }
constexpr int kOffFw = 320 + 4 * 9248;

// ---- packed layout (bytes): B operands (bf16), biases (fp32), fc (fp32)
constexpr int kB1Bytes = 1024;                 // 32 x 16
constexpr int kBlBytes = 9 * 2 * 1024;         // per 32->32 layer: 9 taps x 2 K-steps
constexpr int kPkB1 = 0;
__host__ __device__ constexpr int pk_bl(int l) { return kB1Bytes + (l - 1) * kBlBytes; }  // l = 1..4
constexpr int kPkBias = kB1Bytes + 4 * kBlBytes;  // 5 x 32 floats
constexpr int kPkFc = kPkBias + 5 * 32 * 4;       // 32 + 1 floats (padded to 36)
constexpr int kPackedBytes = kPkFc + 36 * 4;

// ---- activations saved for the backward pass, per patch (bytes)
constexpr int kA1 = 33 * 33 * 32 * 2, kA2 = 17 * 17 * 32 * 2, kA3 = 9 * 9 * 32 * 2,
              kA4 = 5 * 5 * 32 * 2, kA5 = 5 * 5 * 32 * 2;
constexpr int kSvA1 = 0, kSvA2 = kSvA1 + kA1, kSvA3 = kSvA2 + kA2, kSvA4 = kSvA3 + kA3,
              kSvA5 = kSvA4 + kA4, kSvHead = kSvA5 + kA5;  // head: g[32], logit, y (fp32)
constexpr int kSaveBytes = ((kSvHead + 34 * 4) + 127) & ~127;
constexpr int kSvInput = kSaveBytes;                       // x0: 65x65 bf16
constexpr int kSaveBytesTotal = kSaveBytes + ((kPatch * kPatch * 2 + 127) & ~127);

// ---- shared-memory plan of the forward kernel (bytes, 128-aligned)
constexpr int kPln2 = 18 * 18, kPln3 = 10 * 10, kPln4 = 6 * 6, kPln5 = 7 * 7;
constexpr int kSmW = 0;
constexpr int kSmP2 = ((kSmW + kPackedBytes) + 127) & ~127;
constexpr int kP2Bytes = (16 * kPln2 + 96) * 16;
constexpr int kSmU = ((kSmP2 + kP2Bytes) + 127) & ~127;  // A1 im2col, later P3/P4/P5
constexpr int kA1Bytes = 1152 * 32;
constexpr int kP3Off = 0, kP3Bytes = (16 * kPln3 + 40) * 16;
constexpr int kP4Off = kP3Off + kP3Bytes, kP4Bytes = (16 * kPln4 + 104) * 16;
constexpr int kP5Off = kP4Off + kP4Bytes, kP5Bytes = (4 * kPln5 + 100) * 16;
constexpr int kUBytes = (kP5Off + kP5Bytes) > kA1Bytes ? (kP5Off + kP5Bytes) : kA1Bytes;
constexpr int kSmPatch = ((kSmU + kUBytes) + 127) & ~127;   // 67x67 bf16, zero border
constexpr int kPatchBytes = ((67 * 67 * 2) + 127) & ~127;
constexpr int kSmGap = kSmPatch + kPatchBytes;              // 25 x 32 floats
constexpr int kSmStage = ((kSmGap + 25 * 32 * 4) + 127) & ~127;  // TMA-staged patch
constexpr int kStageW = 72;                                  // 65 columns + 8-alignment slack
constexpr int kStageBytes = ((kPatch * kStageW * 2) + 127) & ~127;
constexpr int kSmEnd = kSmStage + kStageBytes;
constexpr int kSmemBytes = kSmEnd + 128;                    // + base alignment slack

// instruction descriptor: kind::f16, A = B = BF16, D = F32, K-major A and B,
// N = 32, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) |
                            ((128u >> 4) << 24);

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void umma(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dt),
        "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 8 consecutive FP32 accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}

__device__ __forceinline__ float bf16_round(float v) {
    return __bfloat162float(__float2bfloat16_rn(v));
}

// ------------------------------------------------------------------ packing
// fp32 master parameters -> bf16 B operands in the K-major core-matrix
// layout ([n/8][k/8][n%8][k%8], 8x8 bf16 = 128 B per core matrix), fp32
// biases and fc.
__global__ void k_cnn_pack(const float *__restrict__ master, unsigned char *__restrict__ packed) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthr = gridDim.x * blockDim.x;
    __nv_bfloat16 *B1 = (__nv_bfloat16 *)(packed + kPkB1);
    for (int e = tid; e < 32 * 16; e += nthr) {
        const int n = e / 16, k = e % 16;
        const float w = (k < 9) ? master[off_w(0) + n * 9 + k] : 0.f;
        B1[((n / 8) * 2 + k / 8) * 64 + (n % 8) * 8 + (k % 8)] = __float2bfloat16_rn(w);
    }
    for (int e = tid; e < 4 * 9 * 2 * 32 * 16; e += nthr) {
        const int l = 1 + e / (9 * 2 * 512);
        const int rem = e % (9 * 2 * 512);
        const int t = rem / 1024, ks = (rem / 512) % 2, nk = rem % 512;
        const int n = nk / 16, k = nk % 16;
        const int cin = ks * 16 + k, ky = t / 3, kx = t % 3;
        const float w = master[off_w(l) + ((n * 32 + cin) * 3 + ky) * 3 + kx];
        __nv_bfloat16 *Bl = (__nv_bfloat16 *)(packed + pk_bl(l) + (t * 2 + ks) * 1024);
        Bl[((n / 8) * 2 + k / 8) * 64 + (n % 8) * 8 + (k % 8)] = __float2bfloat16_rn(w);
    }
    float *bias = (float *)(packed + kPkBias);
    for (int e = tid; e < 5 * 32; e += nthr) bias[e] = master[off_b(e / 32) + e % 32];
    float *fc = (float *)(packed + kPkFc);
    for (int e = tid; e < 33; e += nthr) fc[e] = master[kOffFw + e];
}

// ------------------------------------------------------------------ forward
// A patch whose 65x65 window lies inside the grid is staged by one TMA tile
// load (72 x 65 posts, the left edge rounded down to 8), prefetched while the
// previous patch runs through the convolutions; windows that cross the grid
// edge are gathered with clamped loads.
struct FwdParams {
    const int16_t *z;
    int H, W;
    long long pitch;
    const int64_t *centers;  // patch centres (post index) or null for the lattice
    long long n;             // number of patches
    int stride, Ws;          // lattice mode: patch i at post ((i / Ws)*stride, (i % Ws)*stride)
    int step;                // patch element (r, c) is post (cy + (r-32)*step, cx + (c-32)*step)
    const unsigned char *packed;
    float *out;              // n predicted visibility indices
    unsigned char *save;     // optional: activations for the backward pass
    int *status;             // optional: set to VS_ERR_TIMEOUT if an MMA wait gave up
};

// Implicit-GEMM tiles run in two halves so that the tensor core works on
// tile t+1 while the CUDA cores run the epilogue of tile t: issue_tile
// (after every input of the tile is in shared memory) puts `nmma` MMAs into
// TMEM accumulator buffer `buf` (32 columns each) and commits them to
// bar[buf]; finish_tile waits for them and reads this thread's row.
template <typename F>
__device__ __forceinline__ void issue_tile(uint64_t *bar, uint32_t tmem, int buf, int nmma, F &&mma_desc) {
    if (threadIdx.x == 0) {
        tc_fence_after();
        for (int i = 0; i < nmma; ++i) {
            uint64_t ad, bd;
            mma_desc(i, ad, bd);
            umma(tmem + (uint32_t)(buf * 32), ad, bd, i > 0 ? 1u : 0u);
        }
        umma_commit(&bar[buf]);
    }
}

__device__ __forceinline__ bool finish_tile(uint64_t *bar, uint32_t *phase, uint32_t tmem, int buf,
                                            float *acc) {
    const bool ok = mbar_wait(&bar[buf], phase[buf]);
    phase[buf] ^= 1u;
    tc_fence_after();
    // warp w reads TMEM lane quarter (w & 3) -- rows 32(w & 3) .. +31 -- and
    // the 8 columns of channel block (w >> 2)
    const int warp = threadIdx.x >> 5;
    tmem_ld8(tmem + (uint32_t)(buf * 32 + 8 * (warp >> 2)) + ((uint32_t)((warp & 3) * 32) << 16), acc);
    tc_fence_before();
    return ok;
}

// inputs written by every thread become visible to the tensor core
__device__ __forceinline__ void publish_smem() {
    fence_proxy_async_smem();
    __syncthreads();
}


// epilogue of one output row: bias + ReLU, rounded to bf16, 32 channels as
// 16 packed words
// one 8-channel block of one output row: bias + ReLU, rounded to bf16
__device__ __forceinline__ uint4 relu_pack8(const float *acc, const float *bias) {
    uint32_t w[4];
#pragma unroll
    for (int c = 0; c < 4; ++c)
        w[c] = pack_bf16x2(fmaxf(acc[2 * c] + bias[2 * c], 0.f), fmaxf(acc[2 * c + 1] + bias[2 * c + 1], 0.f));
    return make_uint4(w[0], w[1], w[2], w[3]);
}

__device__ __forceinline__ long long patch_centre(const FwdParams &P, long long pi) {
    if (P.centers) return P.centers[pi];
    return (pi / P.Ws) * (long long)P.stride * P.W + (pi % P.Ws) * (long long)P.stride;
}

// staged by TMA: contiguous patches (step 1) whose window lies inside the grid
__device__ __forceinline__ bool patch_inside(const FwdParams &P, long long cpost) {
    const int cy = (int)(cpost / P.W), cx = (int)(cpost % P.W);
    return P.step == 1 && cy >= 32 && cy + 32 < P.H && cx >= 32 && cx + 32 < P.W;
}

__global__ void __launch_bounds__(kThreads, 1) k_cnn_forward(const __grid_constant__ CUtensorMap tmap,
                                                             const FwdParams P) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *sm = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    __shared__ uint64_t bar[2];
    __shared__ uint64_t pbar;
    __shared__ uint32_t s_tmem;
    __shared__ int s_red[kThreads / 32];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    unsigned char *Wp = sm + kSmW;
    unsigned char *P2 = sm + kSmP2;
    unsigned char *U = sm + kSmU;
    unsigned char *P3 = U + kP3Off, *P4 = U + kP4Off, *P5 = U + kP5Off;
    __nv_bfloat16 *pb = (__nv_bfloat16 *)(sm + kSmPatch);
    float *gap = (float *)(sm + kSmGap);
    int16_t *raw = (int16_t *)U;  // the patch's posts, before im2col reuses U
    int16_t *stage = (int16_t *)(sm + kSmStage);

    // ---- one-time set-up: weights, zeroed planes, barriers, tensor memory
    for (int i = tid; i < kPackedBytes / 16; i += kThreads)
        ((uint4 *)Wp)[i] = ((const uint4 *)P.packed)[i];
    for (int i = tid; i < kP2Bytes / 16; i += kThreads) ((uint4 *)P2)[i] = make_uint4(0, 0, 0, 0);
    for (int i = tid; i < kPatchBytes / 16; i += kThreads) ((uint4 *)pb)[i] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init(&pbar, 1);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(
                         smem_u32(&s_tmem))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    uint32_t phase[2] = {0u, 0u};
    uint32_t pphase = 0u;
    // stage the first patch
    auto stage_patch = [&](long long pi) {
        const long long cp = patch_centre(P, pi);
        const int cy = (int)(cp / P.W), cx = (int)(cp % P.W);
        const int x0 = floordiv(cx - 32, 8) * 8;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&pbar, (uint32_t)(kPatch * kStageW * 2));
        tma_load_3d(stage, &tmap, 0, x0 / 8, cy - 32, &pbar);
    };
    if (tid == 0 && blockIdx.x < P.n && patch_inside(P, patch_centre(P, blockIdx.x))) stage_patch(blockIdx.x);
    bool ok = true;
    const float *bias = (const float *)(Wp + kPkBias);
    const float *fc = (const float *)(Wp + kPkFc);
    const uint32_t sW = smem_u32(Wp), sP2 = smem_u32(P2), sU = smem_u32(U);
    const uint32_t sP3 = sU + kP3Off, sP4 = sU + kP4Off, sP5 = sU + kP5Off;

    // tap t, K-step ks of a 32->32 layer reading stride-2 parity planes
    auto plane_desc = [&](uint32_t base, int pln, int pitch, int m0, int l, int i, uint64_t &ad, uint64_t &bd) {
        const int t = i >> 1, ks = i & 1, ky = t / 3, kx = t % 3;
        const int plane = ((ky != 1) << 1) | (kx != 1);
        const int shift = (ky != 0 ? pitch : 0) + (kx != 0 ? 1 : 0);
        ad = sdesc(base + ((2 * ks * 4 + plane) * pln + m0 + shift) * 16, 4 * pln * 16, 128);
        bd = sdesc(sW + pk_bl(l) + (t * 2 + ks) * 1024, 128, 256);
    };

    for (long long pi = blockIdx.x; pi < P.n; pi += gridDim.x) {
        // ---- patch: the staged tile, or a clamped gather at the grid edge
        const long long cpost = patch_centre(P, pi);
        const int cy = (int)(cpost / P.W), cx = (int)(cpost % P.W);
        int sum = 0;
        if (patch_inside(P, cpost)) {
            if (!mbar_wait(&pbar, pphase)) ok = false;
            pphase ^= 1u;
            const int off = (cx - 32) - floordiv(cx - 32, 8) * 8;
            for (int e = tid; e < kPatch * kPatch; e += kThreads) {
                const int16_t v = stage[(e / kPatch) * kStageW + off + e % kPatch];
                raw[e] = v;
                sum += v;
            }
        } else {
            for (int e = tid; e < kPatch * kPatch; e += kThreads) {
                const int r = min(max(cy + (e / kPatch - 32) * P.step, 0), P.H - 1);
                const int c = min(max(cx + (e % kPatch - 32) * P.step, 0), P.W - 1);
                const int16_t v = P.z[(long long)r * P.pitch + c];
                raw[e] = v;
                sum += v;
            }
        }
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) s_red[warp] = sum;
        __syncthreads();
        int tot = 0;
#pragma unroll
        for (int q = 0; q < kThreads / 32; ++q) tot += s_red[q];
        const float mean = (float)tot / (float)(kPatch * kPatch);
        unsigned char *sv = P.save ? P.save + pi * (long long)kSaveBytesTotal : nullptr;
        for (int e = tid; e < kPatch * kPatch; e += kThreads) {
            const __nv_bfloat16 x = __float2bfloat16_rn(((float)raw[e] - mean) / 1000.0f);
            pb[(e / kPatch + 1) * 67 + (e % kPatch + 1)] = x;
            if (sv) ((__nv_bfloat16 *)(sv + kSvInput))[e] = x;
        }
        __syncthreads();
        // the staging tile is free: prefetch the next patch during the convolutions
        {
            const long long nx = pi + gridDim.x;
            if (tid == 0 && nx < P.n && patch_inside(P, patch_centre(P, nx))) stage_patch(nx);
        }

        // ---- conv1: explicit im2col (1152 rows x 16 K), 9 M-tiles of one MMA each
        for (int m = tid; m < 1152; m += kThreads) {
            const int y = m / 34, x = m % 34;
            uint32_t w[8];
            if (y < 33 && x < 33) {
                __nv_bfloat16 t[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) t[k] = __float2bfloat16_rn(0.f);
#pragma unroll
                for (int k = 0; k < 9; ++k) t[k] = pb[(2 * y + k / 3) * 67 + (2 * x + k % 3)];
#pragma unroll
                for (int k = 0; k < 8; ++k) w[k] = *(uint32_t *)&t[2 * k];
            } else {
#pragma unroll
                for (int k = 0; k < 8; ++k) w[k] = 0;
            }
            unsigned char *row = U + (m / 8) * 256 + (m % 8) * 16;
            *(uint4 *)row = make_uint4(w[0], w[1], w[2], w[3]);
            *(uint4 *)(row + 128) = make_uint4(w[4], w[5], w[6], w[7]);
        }
        publish_smem();
        float acc[8];
        const int row = 32 * (warp & 3) + lane;  // accumulator row (TMEM lane) of this thread
        const int cb = warp >> 2;                // its 8-channel block
        auto l1 = [&](int mt) {
            return [=](int, uint64_t &ad, uint64_t &bd) {
                ad = sdesc(sU + mt * 4096, 128, 256);
                bd = sdesc(sW + kPkB1, 128, 256);
            };
        };
        issue_tile(bar, tmem, 0, 1, l1(0));
        for (int mt = 0; mt < 9; ++mt) {
            if (mt + 1 < 9) issue_tile(bar, tmem, (mt + 1) & 1, 1, l1(mt + 1));
            ok &= finish_tile(bar, phase, tmem, mt & 1, acc);
            const int m = mt * 128 + row, y = m / 34, x = m % 34;
            if (y < 33 && x < 33) {
                const uint4 v = relu_pack8(acc, bias + 8 * cb);
                const int plane = ((y & 1) << 1) | (x & 1);
                const int pix = ((y >> 1) + 1) * 18 + (x >> 1) + 1;
                *(uint4 *)(P2 + (((long long)cb * 4 + plane) * kPln2 + pix) * 16) = v;
                if (sv) *(uint4 *)(sv + kSvA1 + (y * 33 + x) * 64 + cb * 16) = v;
            }
            __syncthreads();  // this buffer's tcgen05.ld done before it is reissued
        }
        // A1 is dead: clear the region that now holds the next layers' planes
        for (int i = tid; i < kUBytes / 16; i += kThreads) ((uint4 *)U)[i] = make_uint4(0, 0, 0, 0);
        publish_smem();

        // ---- conv2: 3 tiles, input P2 (pitch 18, plane 324), output P3 (pitch 10)
        auto l2 = [&](int mt) {
            return [=](int i, uint64_t &ad, uint64_t &bd) { plane_desc(sP2, kPln2, 18, mt * 128, 1, i, ad, bd); };
        };
        issue_tile(bar, tmem, 0, 18, l2(0));
        for (int mt = 0; mt < 3; ++mt) {
            if (mt + 1 < 3) issue_tile(bar, tmem, (mt + 1) & 1, 18, l2(mt + 1));
            ok &= finish_tile(bar, phase, tmem, mt & 1, acc);
            const int m = mt * 128 + row, y = m / 18, x = m % 18;
            if (y < 17 && x < 17) {
                const uint4 v = relu_pack8(acc, bias + 32 + 8 * cb);
                const int plane = ((y & 1) << 1) | (x & 1);
                const int pix = ((y >> 1) + 1) * 10 + (x >> 1) + 1;
                *(uint4 *)(P3 + (((long long)cb * 4 + plane) * kPln3 + pix) * 16) = v;
                if (sv) *(uint4 *)(sv + kSvA2 + (y * 17 + x) * 64 + cb * 16) = v;
            }
            __syncthreads();
        }
        publish_smem();
        // ---- conv3: 1 tile, input P3 (pitch 10, plane 100), output P4 (pitch 6)
        issue_tile(bar, tmem, 0, 18, [&](int i, uint64_t &ad, uint64_t &bd) { plane_desc(sP3, kPln3, 10, 0, 2, i, ad, bd); });
        ok &= finish_tile(bar, phase, tmem, 0, acc);
        {
            const int y = row / 10, x = row % 10;
            if (y < 9 && x < 9) {
                const uint4 v = relu_pack8(acc, bias + 64 + 8 * cb);
                const int plane = ((y & 1) << 1) | (x & 1);
                const int pix = ((y >> 1) + 1) * 6 + (x >> 1) + 1;
                *(uint4 *)(P4 + (((long long)cb * 4 + plane) * kPln4 + pix) * 16) = v;
                if (sv) *(uint4 *)(sv + kSvA3 + (y * 9 + x) * 64 + cb * 16) = v;
            }
        }
        publish_smem();
        // ---- conv4: 1 tile, input P4 (pitch 6, plane 36), output P5 (stride-1 plane, pitch 7)
        issue_tile(bar, tmem, 1, 18, [&](int i, uint64_t &ad, uint64_t &bd) { plane_desc(sP4, kPln4, 6, 0, 3, i, ad, bd); });
        ok &= finish_tile(bar, phase, tmem, 1, acc);
        {
            const int y = row / 6, x = row % 6;
            if (y < 5 && x < 5) {
                const uint4 v = relu_pack8(acc, bias + 96 + 8 * cb);
                const int pix = (y + 1) * 7 + (x + 1);
                *(uint4 *)(P5 + ((long long)cb * kPln5 + pix) * 16) = v;
                if (sv) *(uint4 *)(sv + kSvA4 + (y * 5 + x) * 64 + cb * 16) = v;
            }
        }
        publish_smem();
        // ---- conv5 (stride 1): 1 tile, input P5 (pitch 7, plane 49) -> pooling buffer
        issue_tile(bar, tmem, 0, 18, [&](int i, uint64_t &ad, uint64_t &bd) {
            const int t = i >> 1, ks = i & 1, ky = t / 3, kx = t % 3;
            ad = sdesc(sP5 + ((2 * ks) * kPln5 + ky * 7 + kx) * 16, kPln5 * 16, 128);
            bd = sdesc(sW + pk_bl(4) + (t * 2 + ks) * 1024, 128, 256);
        });
        ok &= finish_tile(bar, phase, tmem, 0, acc);
        {
            const int y = row / 7, x = row % 7;
            if (y < 5 && x < 5) {
                const uint4 v = relu_pack8(acc, bias + 128 + 8 * cb);
                const __nv_bfloat16 *h = (const __nv_bfloat16 *)&v;
#pragma unroll
                for (int c = 0; c < 8; ++c) gap[(y * 5 + x) * 32 + 8 * cb + c] = __bfloat162float(h[c]);
                if (sv) *(uint4 *)(sv + kSvA5 + (y * 5 + x) * 64 + cb * 16) = v;
            }
        }
        __syncthreads();
        // ---- global average pool, fc, sigmoid (fixed summation order)
        if (tid < 32) {
            float g = 0.f;
            for (int r = 0; r < 25; ++r) g += gap[r * 32 + tid];
            g *= (1.0f / 25.0f);
            float t = g * fc[tid];
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (tid == 0) {
                const float logit = t + fc[32];
                const float yv = 1.0f / (1.0f + expf(-logit));
                P.out[pi] = yv;
                if (sv) {
                    float *hd = (float *)(sv + kSvHead);
                    hd[32] = logit;
                    hd[33] = yv;
                }
            }
            if (sv) ((float *)(sv + kSvHead))[tid] = g;
        }
        // a timed-out tensor-core wait stops the CTA (uniformly) after this patch
        if (!__syncthreads_and(ok)) break;
    }
    if (!ok && P.status && threadIdx.x == 0) atomicExch(P.status, VS_ERR_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem) : "memory");
}

// ------------------------------------------------------------------ training
// Backward pass, layer by layer over a batch (the forward kernel saved every
// activation).  Each CTA keeps its partial weight gradient in shared memory
// over the patches it owns and adds it to the global gradient once, so the
// global atomics do not scale with the batch.  Products take bf16-valued
// operands (saved activations, bf16-rounded weights, bf16-rounded
// pre-activation gradients) and accumulate in FP32 on the CUDA cores.
constexpr int kBwdThreads = 256;

struct LayerGeo {
    int Hin, Win, Cin, Hout, Wout, stride;
    int sv_in, sv_out;  // byte offsets of the layer's input / output in a save record
};

__host__ __device__ inline LayerGeo layer_geo(int l) {
    const int hin[5] = {65, 33, 17, 9, 5}, hout[5] = {33, 17, 9, 5, 5};
    const int svin[5] = {kSvInput, kSvA1, kSvA2, kSvA3, kSvA4};
    const int svout[5] = {kSvA1, kSvA2, kSvA3, kSvA4, kSvA5};
    LayerGeo g;
    g.Hin = g.Win = hin[l];
    g.Cin = l == 0 ? 1 : 32;
    g.Hout = g.Wout = hout[l];
    g.stride = l == 4 ? 1 : 2;
    g.sv_in = svin[l];
    g.sv_out = svout[l];
    return g;
}

// dL/dlogit = sign(y - label) * y (1 - y) / B (L1 loss through the sigmoid);
// fc gradients; dL/da5 = dL/dg / 25 on every pooled pixel.  One warp per patch.
__global__ void k_cnn_head_bwd(const unsigned char *__restrict__ save, const float *__restrict__ labels,
                               long long B, float inv_batch, const float *__restrict__ master,
                               float *__restrict__ grads, float *__restrict__ da5,
                               float *__restrict__ loss_sum) {
    const long long b = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int c = threadIdx.x & 31;
    if (b >= B) return;
    const float *hd = (const float *)(save + b * (long long)kSaveBytesTotal + kSvHead);
    const float y = hd[33], lab = labels[b];
    const float sgn = (y > lab) ? 1.f : ((y < lab) ? -1.f : 0.f);
    const float dlogit = sgn * y * (1.f - y) * inv_batch;
    atomicAdd(&grads[kOffFw + c], dlogit * hd[c]);
    if (c == 0) {
        atomicAdd(&grads[kOffFw + 32], dlogit);
        atomicAdd(loss_sum, fabsf(y - lab));
    }
    const float d = dlogit * master[kOffFw + c] * (1.0f / 25.0f);
    for (int pix = 0; pix < 25; ++pix) da5[(b * 25 + pix) * 32 + c] = d;
}

__global__ void __launch_bounds__(kBwdThreads) k_cnn_conv_bwd(const unsigned char *__restrict__ save,
                                                              long long B, int l,
                                                              const float *__restrict__ da_out,
                                                              const float *__restrict__ master,
                                                              float *__restrict__ grads,
                                                              float *__restrict__ da_in) {
    extern __shared__ __align__(16) unsigned char smb[];
    const LayerGeo G = layer_geo(l);
    const int nW = 32 * G.Cin * 9;
    const int nin = G.Hin * G.Win * G.Cin, nout = G.Hout * G.Wout * 32;
    float *Wr = (float *)smb;                         // nW, bf16-rounded weights
    float *dW = Wr + nW;                              // nW partial gradient
    float *db = dW + nW;                              // 32
    __nv_bfloat16 *ain = (__nv_bfloat16 *)(db + 32);  // nin
    __nv_bfloat16 *dz = ain + ((nin + 7) & ~7);       // nout
    const int tid = threadIdx.x;
    for (int i = tid; i < nW; i += blockDim.x) {
        Wr[i] = bf16_round(master[off_w(l) + i]);
        dW[i] = 0.f;
    }
    if (tid < 32) db[tid] = 0.f;
    __syncthreads();
    const int s = G.stride;
    for (long long b = blockIdx.x; b < B; b += gridDim.x) {
        const unsigned char *rec = save + b * (long long)kSaveBytesTotal;
        const __nv_bfloat16 *gin = (const __nv_bfloat16 *)(rec + G.sv_in);
        const __nv_bfloat16 *gout = (const __nv_bfloat16 *)(rec + G.sv_out);
        for (int i = tid; i < nin; i += blockDim.x) ain[i] = gin[i];
        for (int i = tid; i < nout; i += blockDim.x) {
            const float a = __bfloat162float(gout[i]);
            dz[i] = __float2bfloat16_rn(a > 0.f ? da_out[b * nout + i] : 0.f);
        }
        __syncthreads();
        if (tid < 32) {
            float t = 0.f;
            for (int p = 0; p < G.Hout * G.Wout; ++p) t += __bfloat162float(dz[p * 32 + tid]);
            db[tid] += t;
        }
        // weight gradient: dW[cout][cin][ky][kx] += sum over output pixels
        for (int o = tid; o < nW; o += blockDim.x) {
            const int cout = o / (G.Cin * 9), rem = o - cout * (G.Cin * 9);
            const int cin = rem / 9, tap = rem - cin * 9, ky = tap / 3, kx = tap - ky * 3;
            float acc = 0.f;
            for (int y = 0; y < G.Hout; ++y) {
                const int iy = s * y + ky - 1;
                if (iy < 0 || iy >= G.Hin) continue;
                for (int x = 0; x < G.Wout; ++x) {
                    const int ix = s * x + kx - 1;
                    if (ix < 0 || ix >= G.Win) continue;
                    acc += __bfloat162float(dz[(y * G.Wout + x) * 32 + cout]) *
                           __bfloat162float(ain[(iy * G.Win + ix) * G.Cin + cin]);
                }
            }
            dW[o] += acc;
        }
        // input gradient (not needed below the first layer)
        if (da_in) {
            for (int e = tid; e < nin; e += blockDim.x) {
                const int ipix = e / G.Cin, cin = e - ipix * G.Cin;
                const int iy = ipix / G.Win, ix = ipix - iy * G.Win;
                float acc = 0.f;
                for (int ky = 0; ky < 3; ++ky) {
                    const int ty = iy + 1 - ky;
                    if (ty < 0 || ty % s) continue;
                    const int y = ty / s;
                    if (y >= G.Hout) continue;
                    for (int kx = 0; kx < 3; ++kx) {
                        const int tx = ix + 1 - kx;
                        if (tx < 0 || tx % s) continue;
                        const int x = tx / s;
                        if (x >= G.Wout) continue;
                        const __nv_bfloat16 *dzp = dz + (y * G.Wout + x) * 32;
                        const float *wp = Wr + cin * 9 + ky * 3 + kx;
#pragma unroll 8
                        for (int co = 0; co < 32; ++co) acc += __bfloat162float(dzp[co]) * wp[co * G.Cin * 9];
                    }
                }
                da_in[b * nin + e] = acc;
            }
        }
        __syncthreads();
    }
    for (int i = tid; i < nW; i += blockDim.x) atomicAdd(&grads[off_w(l) + i], dW[i]);
    if (tid < 32) atomicAdd(&grads[off_b(l) + tid], db[tid]);
}

__host__ __device__ inline size_t conv_bwd_smem(int l) {
    const LayerGeo G = layer_geo(l);
    const int nW = 32 * G.Cin * 9, nin = G.Hin * G.Win * G.Cin, nout = G.Hout * G.Wout * 32;
    return (size_t)(2 * nW + 32) * 4 + (size_t)((nin + 7) & ~7) * 2 + (size_t)nout * 2 + 16;
}

// Adam (Kingma & Ba 2015) on the fp32 master weights; clears the gradients.
__global__ void k_cnn_adam(float *__restrict__ w, float *__restrict__ g, float *__restrict__ m,
                           float *__restrict__ v, int n, float lr, float b1, float b2, float eps,
                           float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    g[i] = 0.f;
}

}  // namespace cnn
}  // namespace vs

using namespace vs;

extern "C" int vs_cnn_param_count(void) { return cnn::kNParams; }
extern "C" size_t vs_cnn_packed_bytes(void) { return (size_t)cnn::kPackedBytes; }
extern "C" size_t vs_cnn_save_bytes(void) { return (size_t)cnn::kSaveBytesTotal; }

extern "C" int vs_cnn_pack(const float *master, void *packed, vs_stream_t st) {
    if (!master || !packed || ((uintptr_t)packed & 15)) return VS_ERR_ARG;
    int rc = check_device();
    if (rc) return rc;
    cnn::k_cnn_pack<<<64, 256, 0, (cudaStream_t)st>>>(master, (unsigned char *)packed);
    VS_CUDA_TRY(cudaGetLastError());
    return VS_OK;
}

static int cnn_forward_launch(vs_grid g, const int64_t *centers, int64_t n, int32_t stride,
                              int32_t patch_step, const void *packed, float *out, void *save,
                              int32_t *status, vs_stream_t st) {
    if (patch_step < 1 || patch_step > 64) return VS_ERR_RANGE;
    int rc = check_grid(g);
    if (rc) return rc;
    if (!packed || !out || ((uintptr_t)packed & 15) || (save && ((uintptr_t)save & 15)))
        return VS_ERR_ARG;
    if (n < 0) return VS_ERR_RANGE;
    if (n == 0) return VS_OK;
    if ((rc = check_device())) return rc;
    cnn::FwdParams P;
    P.z = g.z; P.H = g.H; P.W = g.W; P.pitch = g.pitch;
    P.centers = centers; P.n = n; P.stride = stride; P.step = patch_step;
    P.Ws = stride > 0 ? (g.W + stride - 1) / stride : 1;
    P.packed = (const unsigned char *)packed; P.out = out;
    P.save = (unsigned char *)save; P.status = status;
    int dev = 0, sms = 0;
    VS_CUDA_TRY(cudaGetDevice(&dev));
    VS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    VS_CUDA_TRY(cudaFuncSetAttribute(cnn::k_cnn_forward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     cnn::kSmemBytes));
    const long long grid = std::min<long long>(n, (long long)sms);
    GridMap gm;  // 72 x 65 post tiles for the staged patches
    if ((rc = make_grid_map(&gm, g, cnn::kStageW / 8, cnn::kPatch))) return rc;
    cnn::k_cnn_forward<<<(unsigned)grid, cnn::kThreads, cnn::kSmemBytes, (cudaStream_t)st>>>(gm.map, P);
    VS_CUDA_TRY(cudaGetLastError());
    return VS_OK;
}

extern "C" int vs_cnn_forward(vs_grid g, const int64_t *centers, int64_t n, int32_t patch_step,
                              const void *packed, float *out, void *save, int32_t *status,
                              vs_stream_t st) {
    if (!centers && n > 0) return VS_ERR_ARG;
    return cnn_forward_launch(g, centers, n, 0, patch_step, packed, out, save, status, st);
}

extern "C" int vs_cnn_score_lattice(vs_grid g, int32_t stride, int32_t patch_step, const void *packed,
                                    float *score_out, int32_t *status, vs_stream_t st) {
    if (stride < 1) return VS_ERR_RANGE;
    if (g.H < 1 || g.W < 1) return VS_ERR_RANGE;
    const int64_t Hs = (g.H + stride - 1) / stride, Ws = (g.W + stride - 1) / stride;
    return cnn_forward_launch(g, nullptr, Hs * Ws, stride, patch_step, packed, score_out, nullptr,
                              status, st);
}

// per patch: dL/da of layers 5, 4, 3, 2, 1 (fp32)
static size_t cnn_da_floats(int l) {  // gradient w.r.t. the output of layer l
    const int h[5] = {33, 17, 9, 5, 5};
    return (size_t)h[l] * h[l] * 32;
}

extern "C" size_t vs_cnn_backward_workspace(int64_t B) {
    if (B < 0) return 0;
    size_t per = 0;
    for (int l = 0; l < 5; ++l) per += cnn_da_floats(l);
    return (size_t)B * per * 4 + 256;
}

extern "C" int vs_cnn_backward(const void *save, const float *labels, int64_t B, const float *master,
                               float *grads, float *loss_sum, void *ws, size_t ws_bytes,
                               vs_stream_t st) {
    if (!save || !labels || !master || !grads || !loss_sum || ((uintptr_t)save & 15)) return VS_ERR_ARG;
    if (B < 1) return VS_ERR_RANGE;
    if (!ws || ws_bytes < vs_cnn_backward_workspace(B)) return VS_ERR_WS;
    int rc = check_device();
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)st;
    float *da[5];
    float *p = (float *)ws;
    for (int l = 0; l < 5; ++l) { da[l] = p; p += (size_t)B * cnn_da_floats(l); }
    const unsigned char *sv = (const unsigned char *)save;
    cnn::k_cnn_head_bwd<<<(unsigned)((B * 32 + 255) / 256), 256, 0, s>>>(sv, labels, B, 1.0f / (float)B,
                                                                          master, grads, da[4], loss_sum);
    VS_CUDA_TRY(cudaGetLastError());
    int dev = 0, sms = 0;
    VS_CUDA_TRY(cudaGetDevice(&dev));
    VS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    for (int l = 4; l >= 0; --l) {
        const size_t smem = cnn::conv_bwd_smem(l);
        VS_CUDA_TRY(cudaFuncSetAttribute(cnn::k_cnn_conv_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const unsigned grid = (unsigned)std::min<long long>(B, (long long)sms);
        cnn::k_cnn_conv_bwd<<<grid, cnn::kBwdThreads, smem, s>>>(sv, B, l, da[l], master, grads,
                                                                  l > 0 ? da[l - 1] : nullptr);
        VS_CUDA_TRY(cudaGetLastError());
    }
    return VS_OK;
}

extern "C" int vs_cnn_adam(float *master, float *grads, float *m, float *v, int64_t step, float lr,
                           float beta1, float beta2, float eps, vs_stream_t st) {
    if (!master || !grads || !m || !v) return VS_ERR_ARG;
    if (step < 1 || !(lr > 0.f)) return VS_ERR_RANGE;
    int rc = check_device();
    if (rc) return rc;
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    const int n = cnn::kNParams;
    cnn::k_cnn_adam<<<(n + 255) / 256, 256, 0, (cudaStream_t)st>>>(master, grads, m, v, n, lr, beta1,
                                                                   beta2, eps, c1, c2);
    VS_CUDA_TRY(cudaGetLastError());
    return VS_OK;
}
