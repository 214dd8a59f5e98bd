// cnn_bwd.cu -- training backward pass of the learned candidate proposal
// (the network of cnn.cu) on the 5th-generation tensor cores.
//
// Every contraction of the backward pass is a GEMM with BF16 operands and
// FP32 accumulation in tensor memory:
//   weight gradient of conv l (l = 0..4):
//     dW_l[cout][cin][tap] = sum over patches b and output pixels p of
//                            dz_l[b,p][cout] * a_in[b, pixel(p, tap)][cin]
//     = D[m = tap*cin + cin'][n = cout], K = (b, p): A = im2col of the saved
//     input activations, transposed; B = dz_l, transposed.
//   data gradient of conv l (l = 1..4), the input of layer l:
//     da_{l-1}[b,q][cin] = sum over taps and cout of
//                          dz_l[b, out(q, tap)][cout] * W_l[cout][cin][tap]
//     = D[m = (b, q)][n = cin], K = (tap, cout): A = the dz values each input
//     pixel receives, per tap (im2col of the transposed convolution); B = W_l
//     rounded to bf16, transposed.
// with dz_l = bf16(da_l * [a_l > 0]) the pre-activation gradient rounded to
// bf16 (the ReLU's derivative through the saved bf16 output).  The operands
// are written to global memory by small kernels, already in the tensor
// cores' K-major core-matrix layout (8 rows x 16 bytes per core matrix), and
// one GEMM kernel streams them through shared memory with bulk copies.  The
// head (pool, fc, sigmoid, L1 loss) runs on CUDA cores.
#include <algorithm>

#include <cuda_bf16.h>

#include "cnn_layout.cuh"
#include "vs_common.cuh"

namespace vs {
namespace cnnb {

using namespace vs::cnn;

// ------------------------------------------------------------------ GEMM
// D[M][32] = sum_k A[m][k] B[n][k], bf16 x bf16 -> fp32.
// A: tiles of 128 rows x 64 K (16 KB) ordered [m-tile][k-chunk]; B: tiles of
// 32 rows x 64 K (4 KB) ordered [k-chunk].  Inside a tile, core matrix
// (row group g, K group j) holds rows 8g..8g+7, K 8j..8j+7 as 8 rows of 16
// bytes at byte (g*8 + j) * 128: K-adjacent core matrices are 128 bytes
// apart, row-adjacent ones 1024.
constexpr int kGemmStages = 4;
constexpr int kTileA = 128 * 64 * 2, kTileB = 32 * 64 * 2;
constexpr int kGemmThreads = 192;  // warps 0..3 epilogue, 4 copies, 5 MMA

// element (r, k) of a tile with rows of 64 K values, as a byte offset
__host__ __device__ __forceinline__ uint32_t tile_off(int r, int k) {
    return (uint32_t)((((r >> 3) * 8 + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

// instruction descriptor: kind::f16, A = B = BF16, D = F32, K-major, N = 32, M = 128
constexpr uint32_t kIdescG = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint64_t sdesc_g(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// where D[m][n] goes: mode 0 (weight gradient, split over K) stores the
// split's partial sum at out[(split * mvalid + m) * 32 + n] for m < mvalid
// (k_wgrad_reduce adds the splits in a fixed order); mode 1 (data gradient)
// stores out[m * 32 + n] for m < mvalid.  a_rows: rows of each A tile held in memory and copied (128, or
// 16 for the first layer's 9 taps: the MMA still computes 128 rows, those it
// reads from whatever the shared buffer holds only reach discarded outputs).
struct GemmArgs {
    const unsigned char *A, *B;
    int mtiles, kchunks, ksplit;
    int a_rows;
    float *out;
    long long mvalid;
    int cin, mode;
    int *status;
};

__global__ void __launch_bounds__(kGemmThreads, 1) k_tc_gemm(const GemmArgs G) {
    extern __shared__ __align__(1024) unsigned char smg[];
    unsigned char *sA = (unsigned char *)(((uintptr_t)smg + 1023) & ~(uintptr_t)1023);
    unsigned char *sB = sA + kGemmStages * kTileA;
    __shared__ uint64_t full[kGemmStages], empty[kGemmStages], done;
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int mt = blockIdx.x % G.mtiles, ks = blockIdx.x / G.mtiles;
    const int c0 = (int)((long long)ks * G.kchunks / G.ksplit);
    const int c1 = (int)((long long)(ks + 1) * G.kchunks / G.ksplit);
    const int nc = c1 - c0;
    if (tid == 0) {
        for (int s = 0; s < kGemmStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        s_fail = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(&s_tmem))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    if (warp == 4) {
        // ---- copies: stage s is reused once the MMAs that read it committed
        if (lane == 0) {
            for (int i = 0; i < nc; ++i) {
                const int s = i % kGemmStages;
                if (i >= kGemmStages && !mbar_wait(&empty[s], (uint32_t)(((i / kGemmStages) - 1) & 1))) {
                    s_fail = 1;
                    break;
                }
                if (s_fail) break;
                const uint32_t abytes = (uint32_t)G.a_rows * 128u;
                mbar_arrive_expect_tx(&full[s], abytes + (uint32_t)kTileB);
                const int c = c0 + i;
                bulk_g2s(sA + s * kTileA, G.A + ((size_t)mt * G.kchunks + c) * abytes, abytes, &full[s]);
                bulk_g2s(sB + s * kTileB, G.B + (size_t)c * kTileB, kTileB, &full[s]);
            }
        }
    } else if (warp == 5) {
        // ---- MMA issue: four K = 16 steps per 64-wide chunk
        if (lane == 0) {
            bool ok = true;
            for (int i = 0; i < nc; ++i) {
                const int s = i % kGemmStages;
                if (!mbar_wait(&full[s], (uint32_t)((i / kGemmStages) & 1))) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint64_t da = sdesc_g(smem_u32(sA + s * kTileA), 128, 1024);
                const uint64_t db = sdesc_g(smem_u32(sB + s * kTileB), 128, 1024);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint32_t acc = (i > 0 || kk > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                        "l"(da + (uint64_t)(kk * 16)), "l"(db + (uint64_t)(kk * 16)), "r"(kIdescG), "r"(acc));
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&empty[s]))
                             : "memory");
            }
            if (!ok) s_fail = 1;
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&done))
                         : "memory");
        }
    } else {
        // ---- epilogue: thread = accumulator row (TMEM lane), 32 columns
        const bool ok = mbar_wait(&done, 0u);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int r = warp * 32 + lane;
        const long long m = (long long)mt * 128 + r;
        uint32_t v[32];
        const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%32];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%33];\n\t"
            "tcgen05.wait::ld.sync.aligned;"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
              "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
              "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(ta), "r"(ta + 16u)
            : "memory");
        if (nc > 0 && m < G.mvalid) {
            // a wait that gave up leaves NaN in the outputs, so that the
            // failure shows in the gradients instead of passing silently
            const bool good = ok && !s_fail;
            const long long row = G.mode == 0 ? (long long)ks * G.mvalid + m : m;
            float4 *o = (float4 *)(G.out + row * 32);
#pragma unroll
            for (int q = 0; q < 8; ++q)
                o[q] = good ? make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                                          __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]))
                            : make_float4(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000),
                                          __int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
        }
        if ((!ok || s_fail) && G.status && tid == 0) atomicExch(G.status, VS_ERR_TIMEOUT);
    }
    // no copy may still be landing when the CTA leaves: wait for every stage
    // whose copy was issued (bounded), then release tensor memory
    if (warp == 4 && lane == 0 && s_fail) {
        for (int s = 0; s < kGemmStages && s < nc; ++s) mbar_wait(&full[s], 0u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem) : "memory");
}

// ------------------------------------------------------------------ head
// dL/dlogit = sign(y - label) * y (1 - y) / B (L1 loss through the sigmoid)
// and |y - label| per patch into hd2[b] (k_head_reduce sums them, and the fc
// gradients, in patch order); dL/da5 = dL/dg / 25 on every pooled pixel.
// One warp per patch.
__global__ void k_head_bwd(const unsigned char *__restrict__ save, const float *__restrict__ labels,
                           long long B, float inv_batch, const float *__restrict__ master,
                           float2 *__restrict__ hd2, float *__restrict__ da5) {
    const long long b = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int c = threadIdx.x & 31;
    if (b >= B) return;
    const float *hd = (const float *)(save + b * (long long)kSaveBytesTotal + kSvHead);
    const float y = hd[33], lab = labels[b];
    const float sgn = (y > lab) ? 1.f : ((y < lab) ? -1.f : 0.f);
    const float dlogit = sgn * y * (1.f - y) * inv_batch;
    if (c == 0) hd2[b] = make_float2(dlogit, fabsf(y - lab));
    const float d = dlogit * master[kOffFw + c] * (1.0f / 25.0f);
    for (int pix = 0; pix < 25; ++pix) da5[(b * 25 + pix) * 32 + c] = d;
}

// fc gradients (sum over patches of dlogit * pooled features, and of dlogit)
// and the loss sum, each added in patch order by one thread
__global__ void k_head_reduce(const unsigned char *__restrict__ save, const float2 *__restrict__ hd2, long long B,
                              float *__restrict__ grads, float *__restrict__ loss_sum) {
    const int c = threadIdx.x;
    float acc = 0.f;
    for (long long b = 0; b < B; ++b) {
        const float2 h = hd2[b];
        if (c < 32) acc += h.x * ((const float *)(save + b * (long long)kSaveBytesTotal + kSvHead))[c];
        else if (c == 32) acc += h.x;
        else acc += h.y;
    }
    if (c < 33) grads[kOffFw + c] += acc;
    else if (c == 33) *loss_sum += acc;
}

// out[map(i)] += sum over r < nrows of part[r * n + i], in row order:
// mode 0, the weight gradient of a layer (i = m * 32 + n, m = tap * cin + c
// -> w[n][c][tap]); mode 1, the bias (i = channel)
__global__ void k_ordered_sum(const float *__restrict__ part, int nrows, int n, int mode, int cin,
                              float *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float acc = 0.f;
    for (int r = 0; r < nrows; ++r) acc += part[(long long)r * n + i];
    if (mode == 0) {
        const int m = i >> 5, nn = i & 31, tap = m / cin, c = m - tap * cin;
        out[(nn * cin + c) * 9 + tap] += acc;
    } else {
        out[i] += acc;
    }
}

// ------------------------------------------------------------------ dz
// dz = bf16(da * [a > 0]) for every (patch, output pixel) k and channel:
// written as the weight-gradient GEMM's B operand (rows = channel, K = k,
// tiles of 64 K; the K tail zero) and, for the layers whose data gradient is
// needed (l >= 1), plain ([k][32] bf16); the bias gradient is the sum of dz
// over k.  Thread = (k, group of 8 channels).
constexpr int kDzThreads = 256;
__global__ void __launch_bounds__(kDzThreads) k_bwd_dz(const unsigned char *__restrict__ save, long long B,
                                                       int l, const float *__restrict__ da,
                                                       __nv_bfloat16 *__restrict__ dz_plain,
                                                       unsigned char *__restrict__ dzT, long long kpad,
                                                       float *__restrict__ bias_part) {
    __shared__ float s_acc[kDzThreads][9];
    const LayerGeo G = layer_geo(l);
    const int P = G.Hout * G.Wout;
    const long long K = B * P;
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int j = threadIdx.x & 3;
    for (long long k = ((long long)blockIdx.x * kDzThreads + threadIdx.x) >> 2; k < kpad;
         k += ((long long)gridDim.x * kDzThreads) >> 2) {
        __align__(16) __nv_bfloat16 d8[8];
        if (k < K) {
            const long long b = k / P;
            const int p = (int)(k - b * P);
            const uint4 a4 = *(const uint4 *)(save + b * (long long)kSaveBytesTotal + G.sv_out + (p * 32 + 8 * j) * 2);
            const __nv_bfloat16 *a8 = (const __nv_bfloat16 *)&a4;
            const float4 g0 = *(const float4 *)(da + k * 32 + 8 * j);
            const float4 g1 = *(const float4 *)(da + k * 32 + 8 * j + 4);
            const float g[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                d8[i] = __float2bfloat16_rn(__bfloat162float(a8[i]) > 0.f ? g[i] : 0.f);
                acc[i] += __bfloat162float(d8[i]);
            }
            if (dz_plain) *(uint4 *)(dz_plain + k * 32 + 8 * j) = *(const uint4 *)d8;
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) d8[i] = __float2bfloat16_rn(0.f);
        }
        if (dzT) {
            unsigned char *tile = dzT + (k >> 6) * (long long)kTileB;
#pragma unroll
            for (int i = 0; i < 8; ++i) *(__nv_bfloat16 *)(tile + tile_off(8 * j + i, (int)(k & 63))) = d8[i];
        }
    }
    // the block's partial bias gradient, summed over its threads in a fixed order
#pragma unroll
    for (int i = 0; i < 8; ++i) s_acc[threadIdx.x][i] = acc[i];
    __syncthreads();
    if (threadIdx.x < 32) {
        const int jj = threadIdx.x >> 3, ii = threadIdx.x & 7;
        float t = 0.f;
        for (int q = jj; q < kDzThreads; q += 4) t += s_acc[q][ii];
        bias_part[blockIdx.x * 32 + threadIdx.x] = t;
    }
}

// ------------------------------------------------------------------ im2col^T of a layer's input
// A operand of the weight-gradient GEMM of layer l: row m = tap * cin + c,
// K = k = (patch, output pixel): a_in[b][s*y + ky - 1][s*x + kx - 1][c], zero
// outside the input and in the K tail.  cin = 32: a warp = the 32 channels of
// one group of 8 consecutive k, tap by tap (its 32 rows of a tap are
// consecutive, so each store fills whole core matrices); cin = 1 (the first
// layer): a thread = (group of 8 k, row r < 16), rows 9..15 zero.  Rows 288..383
// of the third tile of a 32-channel layer reach only discarded outputs and
// are not written.
__global__ void __launch_bounds__(256) k_bwd_acolT(const unsigned char *__restrict__ save, long long B, int l,
                                                   unsigned char *__restrict__ A, int kchunks, int a_rows) {
    const LayerGeo G = layer_geo(l);
    const uint32_t P = (uint32_t)(G.Hout * G.Wout), Wo = (uint32_t)G.Wout;
    const int s = G.stride;
    const uint32_t K = (uint32_t)(B * P);
    const uint32_t ngroups = (uint32_t)kchunks * 8u;
    const uint32_t abytes = (uint32_t)a_rows * 128u;
    const bool wide = G.Cin == 32;
    const uint32_t total = ngroups * (wide ? 32u : 16u);
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const uint32_t kg = wide ? t >> 5 : t >> 4;
        const int c = wide ? (int)(t & 31) : 0;
        const int r16 = (int)(t & 15);
        const int ntap = wide ? 9 : 1;
        for (int ti = 0; ti < ntap; ++ti) {
            const int tap = wide ? ti : r16;
            const int m = wide ? tap * 32 + c : r16;
            __align__(16) __nv_bfloat16 v8[8];
            const int ky = tap / 3, kx = tap - ky * 3;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const uint32_t k = kg * 8u + (uint32_t)i;
                float v = 0.f;
                if (tap < 9 && k < K) {
                    const uint32_t b = k / P, p = k - b * P, y = p / Wo, x = p - y * Wo;
                    const int iy = s * (int)y + ky - 1, ix = s * (int)x + kx - 1;
                    if (iy >= 0 && iy < G.Hin && ix >= 0 && ix < G.Win)
                        v = __bfloat162float(*(const __nv_bfloat16 *)(save + (size_t)b * kSaveBytesTotal + G.sv_in +
                                                                      (size_t)((iy * G.Win + ix) * G.Cin + c) * 2));
                }
                v8[i] = __float2bfloat16_rn(v);
            }
            const uint32_t kc = kg >> 3;
            unsigned char *tile = A + ((size_t)(m >> 7) * kchunks + kc) * abytes;
            *(uint4 *)(tile + tile_off(m & 127, (int)((kg & 7) * 8))) = *(const uint4 *)v8;
        }
    }
}

// ------------------------------------------------------------------ im2col of the transposed convolution
// A operand of the data-gradient GEMM of layer l >= 1: row m = (b, q) over
// the layer's input pixels q = iy*Win + ix, K = tap*32 + cout (288, padded to
// 320 with zeros): dz_l[b][y][x][cout] where s*y + ky - 1 = iy and
// s*x + kx - 1 = ix, zero where no output pixel reaches q through that tap.
// Thread = (row m, 8 channels of one tap); a warp's rows are consecutive.
__global__ void __launch_bounds__(256) k_bwd_dzcol(const __nv_bfloat16 *__restrict__ dz, long long B, int l,
                                                   unsigned char *__restrict__ A, long long mtiles) {
    const LayerGeo G = layer_geo(l);
    const int Q = G.Hin * G.Win, s = G.stride;
    const long long rows = mtiles * 128;
    const long long total = rows * 40;  // 40 groups of 8 K per row (320)
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long m = t % rows;
        const int kg = (int)(t / rows);
        uint4 v = make_uint4(0, 0, 0, 0);
        const int tap = kg >> 2, cg = kg & 3;
        if (tap < 9 && m < B * Q) {
            const long long b = m / Q;
            const int q = (int)(m - b * Q), iy = q / G.Win, ix = q - iy * G.Win;
            const int ky = tap / 3, kx = tap - ky * 3;
            const int ty = iy + 1 - ky, tx = ix + 1 - kx;
            if (ty >= 0 && tx >= 0 && ty % s == 0 && tx % s == 0) {
                const int y = ty / s, x = tx / s;
                if (y < G.Hout && x < G.Wout)
                    v = *(const uint4 *)(dz + ((b * G.Hout + y) * G.Wout + x) * 32 + cg * 8);
            }
        }
        unsigned char *tile = A + ((m >> 7) * 5 + (kg >> 3)) * (long long)kTileA;
        *(uint4 *)(tile + tile_off((int)(m & 127), (kg & 7) * 8)) = v;
    }
}

// B operand of the data-gradient GEMM: row n = cin, K = tap*32 + cout:
// bf16(W_l[cout][cin][tap]) for layers 1..4 (tiles at WT + (l-1) * 5 * 4 KB)
__global__ void k_bwd_wT(const float *__restrict__ master, unsigned char *__restrict__ WT) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;  // 4 layers x 32 x 320
    if (e >= 4 * 32 * 320) return;
    const int l = 1 + e / (32 * 320), rem = e % (32 * 320), n = rem / 320, kk = rem % 320;
    float w = 0.f;
    if (kk < 288) {
        const int tap = kk / 32, cout = kk % 32;
        w = master[off_w(l) + (cout * 32 + n) * 9 + tap];
    }
    unsigned char *tile = WT + ((l - 1) * 5 + kk / 64) * kTileB;
    *(__nv_bfloat16 *)(tile + tile_off(n, kk & 63)) = __float2bfloat16_rn(w);
}

}  // namespace cnnb
}  // namespace vs

using namespace vs;

namespace {

constexpr int kDzGrid = 1024;     // blocks of k_bwd_dz (rows of its bias partials)
constexpr int kMaxKSplit = 256;   // splits of a weight-gradient GEMM

struct BwdLayout {
    long long B;
    size_t off_hd2, off_bpart, off_wpart;
    long long kc[5];       // weight-gradient K chunks of 64 per layer (l >= 1)
    long long mt_col[5];   // data-gradient row tiles of 128 per layer (l >= 1)
    size_t off_da[5], off_dz[5], off_dzT[5], off_wT, off_scratch, total;
};

inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

BwdLayout bwd_layout(long long B) {
    BwdLayout L;
    L.B = B;
    size_t o = 0;
    for (int l = 0; l < 5; ++l) {
        const cnn::LayerGeo G = cnn::layer_geo(l);
        const long long P = (long long)G.Hout * G.Wout, Q = (long long)G.Hin * G.Win;
        L.kc[l] = (B * P + 63) / 64;
        L.mt_col[l] = (B * Q + 127) / 128;
        L.off_da[l] = o;  o += al256((size_t)(B * P) * 32 * 4);
        L.off_dz[l] = o;  o += al256((size_t)(B * P) * 32 * 2);
        L.off_dzT[l] = o; o += al256((size_t)L.kc[l] * cnnb::kTileB);
    }
    L.off_wT = o;
    o += al256((size_t)4 * 5 * cnnb::kTileB);
    L.off_hd2 = o;
    o += al256((size_t)B * 8);
    L.off_bpart = o;
    o += al256((size_t)kDzGrid * 32 * 4);
    L.off_wpart = o;
    o += al256((size_t)kMaxKSplit * 288 * 32 * 4);
    // the A operands of one layer at a time: im2col^T (3 row tiles) and the
    // transposed convolution's im2col (5 K chunks per row tile)
    size_t scratch = al256((size_t)L.kc[0] * 16 * 128);  // the first layer: 16-row A tiles
    for (int l = 1; l < 5; ++l)
        scratch = std::max(scratch, al256((size_t)3 * L.kc[l] * cnnb::kTileA) +
                                        al256((size_t)L.mt_col[l] * 5 * cnnb::kTileA));
    L.off_scratch = o;
    o += scratch;
    L.total = o + 256;
    return L;
}

int launch_gemm(const cnnb::GemmArgs &G, int sms, cudaStream_t s) {
    const size_t smem = (size_t)cnnb::kGemmStages * (cnnb::kTileA + cnnb::kTileB) + 1024;
    VS_CUDA_TRY(cudaFuncSetAttribute(cnnb::k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    (void)sms;
    cnnb::k_tc_gemm<<<(unsigned)(G.mtiles * G.ksplit), cnnb::kGemmThreads, smem, s>>>(G);
    vs::note_launch();
    VS_CUDA_TRY(cudaGetLastError());
    return VS_OK;
}

}  // namespace

extern "C" size_t vs_cnn_backward_workspace(int64_t B) {
    if (B < 1 || B > (1ll << 24)) return 0;
    return bwd_layout(B).total;
}

extern "C" int vs_cnn_backward(const void *save, const float *labels, int64_t B, const float *master,
                               float *grads, float *loss_sum, void *ws, size_t ws_bytes,
                               vs_stream_t st) {
    if (!save || !labels || !master || !grads || !loss_sum || ((uintptr_t)save & 15)) return VS_ERR_ARG;
    if (B < 1 || B > (1ll << 24)) return VS_ERR_RANGE;
    const BwdLayout L = bwd_layout(B);
    if (!ws || ws_bytes < L.total) return VS_ERR_WS;
    int rc = check_device();
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)st;
    int dev = 0, sms = 0;
    VS_CUDA_TRY(cudaGetDevice(&dev));
    VS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    unsigned char *w = (unsigned char *)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    const unsigned char *sv = (const unsigned char *)save;
    auto da = [&](int l) { return (float *)(w + L.off_da[l]); };
    auto dz = [&](int l) { return (__nv_bfloat16 *)(w + L.off_dz[l]); };
    unsigned char *wT = w + L.off_wT;
    // head: loss, fc gradients, dL/da5
    float2 *hd2 = (float2 *)(w + L.off_hd2);
    float *bpart = (float *)(w + L.off_bpart), *wpart = (float *)(w + L.off_wpart);
    cnnb::k_head_bwd<<<(unsigned)((B * 32 + 255) / 256), 256, 0, s>>>(sv, labels, B, 1.0f / (float)B, master, hd2,
                                                                       da(4));
    vs::note_launch();
    VS_CUDA_TRY(cudaGetLastError());
    cnnb::k_head_reduce<<<1, 34, 0, s>>>(sv, hd2, B, grads, loss_sum);
    vs::note_launch();
    VS_CUDA_TRY(cudaGetLastError());
    cnnb::k_bwd_wT<<<(4 * 32 * 320 + 255) / 256, 256, 0, s>>>(master, wT);
    vs::note_launch();
    VS_CUDA_TRY(cudaGetLastError());
    const unsigned grid_el = (unsigned)std::min(4 * sms, kDzGrid);
    for (int l = 4; l >= 0; --l) {
        const cnn::LayerGeo G = cnn::layer_geo(l);
        const int a_rows = l == 0 ? 16 : 128, mtiles = l == 0 ? 1 : 3;
        cnnb::k_bwd_dz<<<grid_el, cnnb::kDzThreads, 0, s>>>(sv, B, l, da(l), l >= 1 ? dz(l) : nullptr,
                                                             w + L.off_dzT[l], L.kc[l] * 64, bpart);
        vs::note_launch();
        VS_CUDA_TRY(cudaGetLastError());
        cnnb::k_ordered_sum<<<1, 32, 0, s>>>(bpart, (int)grid_el, 32, 1, 1, grads + cnn::off_b(l));
        vs::note_launch();
        VS_CUDA_TRY(cudaGetLastError());
        unsigned char *acolT = w + L.off_scratch;
        // weight gradient: D[tap * cin + c][cout], K = (patch, output pixel), split over K
        cnnb::k_bwd_acolT<<<grid_el, 256, 0, s>>>(sv, B, l, acolT, (int)L.kc[l], a_rows);
        vs::note_launch();
        VS_CUDA_TRY(cudaGetLastError());
        cnnb::GemmArgs gw;
        gw.A = acolT;
        gw.B = w + L.off_dzT[l];
        gw.mtiles = mtiles;
        gw.kchunks = (int)L.kc[l];
        gw.ksplit = (int)std::max<long long>(
            1, std::min<long long>(std::min<long long>(L.kc[l], kMaxKSplit), (2LL * sms + mtiles - 1) / mtiles));
        gw.a_rows = a_rows;
        gw.out = wpart;
        gw.mvalid = 9 * G.Cin;
        gw.cin = G.Cin;
        gw.mode = 0;
        gw.status = nullptr;
        if ((rc = launch_gemm(gw, sms, s))) return rc;
        const int nw = 9 * G.Cin * 32;
        cnnb::k_ordered_sum<<<(nw + 255) / 256, 256, 0, s>>>(wpart, gw.ksplit, nw, 0, G.Cin, grads + cnn::off_w(l));
        vs::note_launch();
        VS_CUDA_TRY(cudaGetLastError());
        if (l == 0) break;
        // data gradient of the layer's input: D[(patch, input pixel)][cin], K = (tap, cout)
        unsigned char *dzcol = acolT + al256((size_t)3 * L.kc[l] * cnnb::kTileA);
        cnnb::k_bwd_dzcol<<<grid_el, 256, 0, s>>>(dz(l), B, l, dzcol, L.mt_col[l]);
        vs::note_launch();
        VS_CUDA_TRY(cudaGetLastError());
        cnnb::GemmArgs gd;
        gd.A = dzcol;
        gd.B = wT + (size_t)(l - 1) * 5 * cnnb::kTileB;
        gd.mtiles = (int)L.mt_col[l];
        gd.kchunks = 5;
        gd.ksplit = 1;
        gd.a_rows = 128;
        gd.out = da(l - 1);
        gd.mvalid = B * (long long)G.Hin * G.Win;
        gd.cin = 32;
        gd.mode = 1;
        gd.status = nullptr;
        if ((rc = launch_gemm(gd, sms, s))) return rc;
    }
    return VS_OK;
}
