// cnn.cu -- learned candidate proposal: a 5-layer CNN that maps a 65x65
// elevation patch to a predicted visibility index (the Vix stage's ranking
// replaced by a learned one; the paper's Vix stage only ranks posts,
// Sec. "The multiple transmitter siting process", Vix).
//
// Network (fixed by this library; the paper specifies none):
//   x0 = bf16((z - mean(patch)) / 1000)                           65x65x1
//        (fp32: the integer sum / 4225, then a multiply by fp32(0.001))
//   conv1 3x3 s2 p1 1->32, bias, ReLU, bf16                      33x33x32
//   conv2 3x3 s2 p1 32->32                                       17x17x32
//   conv3 3x3 s2 p1 32->32                                        9x 9x32
//   conv4 3x3 s2 p1 32->32                                        5x 5x32
//   conv5 3x3 s1 p1 32->32                                        5x 5x32
//   global average pool -> fc 32->1 -> sigmoid
//
// Forward kernel: one persistent 512-thread CTA per SM works through patches
// entirely in shared memory, its warps split into roles (epilogue, front end,
// MMA issue; see the role table below) that hand work to each other through
// mbarriers.  Every convolution is an implicit GEMM on the 5th-generation
// tensor cores: tcgen05.mma kind::f16 (BF16 x BF16 -> FP32), M = 128 output
// pixels, N = 32 channels, K = 16 per instruction, the FP32 accumulator in
// tensor memory (32 columns per tile), read back with tcgen05.ld for the
// bias + ReLU + BF16 epilogue.  Operands are read straight from shared
// memory through matrix descriptors (no swizzle, K-major 8x16-byte core
// matrices):
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
// At N = 32 an MMA costs a fixed ~46 cycles whatever N <= 64 (measured), so
// the 117 MMAs of a patch bound the kernel at ~6K cycles per patch and SM;
// the rest of a patch's chain is epilogue and hand-off latency.
#include <algorithm>

#include <cuda_bf16.h>

#include "vs_common.cuh"
#include "cnn_layout.cuh"

namespace vs {
namespace cnn {

constexpr int kThreads = 512;  // 16 warps
// ---- packed layout (bytes): B operands (bf16), biases (fp32), fc (fp32)
constexpr int kB1Bytes = 1024;                 // 32 x 16
constexpr int kBlBytes = 9 * 2 * 1024;         // per 32->32 layer: 9 taps x 2 K-steps
constexpr int kPkB1 = 0;
__host__ __device__ constexpr int pk_bl(int l) { return kB1Bytes + (l - 1) * kBlBytes; }  // l = 1..4
constexpr int kPkBias = kB1Bytes + 4 * kBlBytes;  // 5 x 32 floats
constexpr int kPkFc = kPkBias + 5 * 32 * 4;       // 32 + 1 floats (padded to 36)
constexpr int kPackedBytes = kPkFc + 36 * 4;


// ---- shared-memory plan of the forward kernel (bytes, 128-aligned)
constexpr int kPln2 = 18 * 18, kPln3 = 10 * 10, kPln4 = 6 * 6, kPln5 = 7 * 7;
constexpr int kSmW = 0;
constexpr int kSmP2 = ((kSmW + kPackedBytes) + 127) & ~127;
constexpr int kP2Bytes = (16 * kPln2 + 96) * 16;
constexpr int kSmU = ((kSmP2 + kP2Bytes) + 127) & ~127;  // conv1 im2col tile
constexpr int kA1Bytes = 1152 * 32;
constexpr int kUBytes = kA1Bytes;
// conv3..5 inputs reuse the start of the conv2 input region (dead once every
// conv2 MMA has completed)
constexpr int kP3Off = 0, kP3Bytes = (16 * kPln3 + 40) * 16;
constexpr int kP4Off = kP3Off + kP3Bytes, kP4Bytes = (16 * kPln4 + 104) * 16;
constexpr int kP5Off = kP4Off + kP4Bytes, kP5Bytes = (4 * kPln5 + 100) * 16;
constexpr int kP345Bytes = kP5Off + kP5Bytes;
static_assert(kP345Bytes <= kP2Bytes, "conv3..5 planes must fit in the conv2 input region");
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
    int stride, Ws;          // lattice mode: patch i at post ((row0 + i / Ws)*stride, (i % Ws)*stride)
    int row0;                // lattice mode: first lattice row of this launch
    int step;                // patch element (r, c) is post (cy + (r-32)*step, cx + (c-32)*step)
    const unsigned char *packed;
    float *out;              // n predicted visibility indices
    unsigned char *save;     // optional: activations for the backward pass
    int *status;             // optional: set to VS_ERR_TIMEOUT if an MMA wait gave up
};

// one 8-channel block of one accumulator row: bias + ReLU, rounded to bf16
// (packed fp32 pair adds, then one relu-converting pack per channel pair)
__device__ __forceinline__ void add_f32x2(float &a0, float &a1, float b0, float b1) {
    asm("{\n\t.reg .b64 x, y;\n\tmov.b64 x, {%0, %1};\n\tmov.b64 y, {%2, %3};\n\t"
        "add.rn.f32x2 x, x, y;\n\tmov.b64 {%0, %1}, x;\n\t}"
        : "+f"(a0), "+f"(a1)
        : "f"(b0), "f"(b1));
}
__device__ __forceinline__ uint32_t relu_bf16x2(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}
__device__ __forceinline__ uint4 relu_pack8(float *acc, const float *bias) {
    uint32_t w[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        add_f32x2(acc[2 * c], acc[2 * c + 1], bias[2 * c], bias[2 * c + 1]);
        w[c] = relu_bf16x2(acc[2 * c], acc[2 * c + 1]);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// centre (row, column) of patch pi; posts and patch indices are below 2^32
// (the host checks H*W), so 32-bit unsigned arithmetic suffices
__device__ __forceinline__ void patch_rc(const FwdParams &P, long long pi, int &cy, int &cx) {
    if (P.centers) {
        const uint32_t c = (uint32_t)P.centers[pi];
        const uint32_t y = c / (uint32_t)P.W;
        cy = (int)y;
        cx = (int)(c - y * (uint32_t)P.W);
    } else {
        const uint32_t iy = (uint32_t)pi / (uint32_t)P.Ws;
        cy = ((int)iy + P.row0) * P.stride;
        cx = (int)((uint32_t)pi - iy * (uint32_t)P.Ws) * P.stride;
    }
}

// staged by TMA: contiguous patches (step 1) whose window lies inside the grid
__device__ __forceinline__ bool patch_inside(const FwdParams &P, int cy, int cx) {
    return P.step == 1 && cy >= 32 && cy + 32 < P.H && cx >= 32 && cx + 32 < P.W;
}

// ---- warp roles of the forward kernel (16 warps)
//   warps 0..7   epilogue: TMEM -> bias + ReLU + bf16 -> the next layer's
//                planes, and the pooling buffer (thread: one accumulator row,
//                16 channels)
//   warps 8..14  front: a later patch's posts, mean, normalisation and
//                im2col, and the head (pool, fc, sigmoid) of an earlier one
//   warp 15      MMA issue (one lane)
// so the front end and the head run beside the chain conv1 epilogue -> conv2
// -> epilogue -> conv3 -> ... -> conv5 epilogue, which alternates between the
// tensor core and the epilogue warps.
constexpr int kEpiWarps = 8, kFrontWarps = 7, kMmaWarp = kEpiWarps + kFrontWarps;
constexpr int kEpiThreads = kEpiWarps * 32, kFrontThreads = kFrontWarps * 32;
static_assert((kMmaWarp + 1) * 32 == kThreads, "role split must cover the CTA");
constexpr int kPerFront = (kPatch * kPatch + kFrontThreads - 1) / kFrontThreads;  // posts per front thread
constexpr int kRowsFront = (1152 + kFrontThreads - 1) / kFrontThreads;           // im2col rows per front thread

// Tensor memory: every accumulator tile of a patch has its own 32 columns
// (conv1 tiles 0..8, conv2 tiles 0..2, conv3, conv4, conv5: 15 x 32 = 480 of
// the 512 columns).
constexpr int kTmemCols = 512;
constexpr int kColL2 = 9 * 32, kColL3 = 12 * 32, kColL4 = 13 * 32, kColL5 = 14 * 32;
// mbarriers, each completing once per patch:
//   tcgen05.commit   conv1 tiles in groups of three, conv2 tiles, conv3, conv4, conv5
//   front -> MMA     im2col tile written (every front thread arrives)
//   epilogue -> MMA  conv1 accumulators read; conv1 tiles 0..5 written (all
//                    that conv2's first tile reads); every conv2 input plane
//                    written; conv3, conv4, conv5 input planes written
//   epilogue -> front  pooling buffer written (every epilogue thread arrives)
//   front -> epilogue  pooling buffer read (one head warp arrives)
enum {
    kBarC1 = 0, kBarC2 = 3, kBarC3 = 6, kBarC4 = 7, kBarC5 = 8,
    kBarURdy = 9, kBarC1Free = 10, kBarP2a = 11, kBarP2 = 12, kBarP3 = 13, kBarP4 = 14, kBarP5 = 15,
    kBarGap = 16, kBarGapFree = 17,
    kNBar = 18
};
__host__ __device__ constexpr uint32_t bar_count(int b) {
    return b == kBarURdy ? kFrontThreads : b == kBarGapFree ? 32 : b >= kBarC1Free ? kEpiThreads : 1;
}

__device__ __forceinline__ void group_sync(int id, int n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
// OR over a group of warps (named barrier with a predicate reduction): the
// same answer in every thread of the group
__device__ __forceinline__ bool group_any(int id, int n, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "barrier.red.or.pred q, %2, %3, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(n)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// non-suspending bounded wait (the MMA lane wakes as soon as the phase flips)
__device__ __forceinline__ bool mbar_wait_spin(uint64_t *bar, uint32_t parity) {
    const uint32_t addr = smem_u32(bar);
    for (uint32_t i = 0; i < kWaitPolls; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
// 16 consecutive FP32 accumulator columns of this thread's TMEM lane, for one
// or three tiles, with one wait
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld16x3(uint32_t t0, uint32_t t1, uint32_t t2, float (*v)[16]) {
    uint32_t r[48];
#define VS_R16(o) "=r"(r[o + 0]), "=r"(r[o + 1]), "=r"(r[o + 2]), "=r"(r[o + 3]), "=r"(r[o + 4]), \
    "=r"(r[o + 5]), "=r"(r[o + 6]), "=r"(r[o + 7]), "=r"(r[o + 8]), "=r"(r[o + 9]), "=r"(r[o + 10]), \
    "=r"(r[o + 11]), "=r"(r[o + 12]), "=r"(r[o + 13]), "=r"(r[o + 14]), "=r"(r[o + 15])
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%48];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%49];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47}, [%50];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : VS_R16(0), VS_R16(16), VS_R16(32)
        : "r"(t0), "r"(t1), "r"(t2)
        : "memory");
#undef VS_R16
#pragma unroll
    for (int i = 0; i < 48; ++i) v[i / 16][i % 16] = __uint_as_float(r[i]);
}
// tensor-core MMA with a compile-time accumulate flag
template <int ACC>
__device__ __forceinline__ void umma_c(uint32_t dt, uint64_t ad, uint64_t bd) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dt),
        "l"(ad), "l"(bd), "r"(kIdesc), "n"(ACC));
}

// The conv3..5 input planes overwrite the start of the conv2 input planes
// (kP345Bytes / 16 = 2616 sixteen-byte cells).  Cells no epilogue writes --
// borders, the extra row/column of odd parity planes, tails -- must read as
// zero, so each layer switch clears exactly those: p345_unwritten(u) for the
// conv3..5 planes, p2_unwritten(u) for the conv2 planes.  They are disjoint
// from the cells the epilogues write, so clearing needs no ordering against
// the epilogue stores.
__device__ __forceinline__ bool planes_written(int cell, int pitch, int rows_even, int pb) {
    const int r = cell / pitch, c = cell - r * pitch;
    const int py = (pb >> 1) & 1, px = pb & 1;  // parity plane of plane block pb
    return r >= 1 && r <= rows_even - py && c >= 1 && c <= rows_even - px;
}
__device__ __forceinline__ bool p345_unwritten(int u) {
    if (u < 16 * kPln3) return !planes_written(u % kPln3, 10, 9, u / kPln3);
    u -= kP3Bytes / 16;
    if (u < 0) return true;
    if (u < 16 * kPln4) return !planes_written(u % kPln4, 6, 5, u / kPln4);
    u -= kP4Bytes / 16;
    if (u < 0) return true;
    if (u < 4 * kPln5) {
        const int c = u % kPln5, r = c / 7, x = c % 7;
        return !(r >= 1 && r <= 5 && x >= 1 && x <= 5);
    }
    return true;
}
__device__ __forceinline__ bool p2_unwritten(int u) { return !planes_written(u % kPln2, 18, 17, u / kPln2); }
constexpr int kP345Cells = kP345Bytes / 16;

__global__ void __launch_bounds__(kThreads, 1) k_cnn_forward(const __grid_constant__ CUtensorMap tmap,
                                                             const FwdParams P) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *sm = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    __shared__ uint64_t bar[kNBar];
    __shared__ uint64_t pbar;
    __shared__ uint32_t s_tmem;
    __shared__ int s_red[kFrontWarps];
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    unsigned char *Wp = sm + kSmW;
    unsigned char *X = sm + kSmP2;  // conv2 input planes, then conv3..5 input planes
    unsigned char *U = sm + kSmU;
    __nv_bfloat16 *pb = (__nv_bfloat16 *)(sm + kSmPatch);
    float *gap = (float *)(sm + kSmGap);
    int16_t *stage = (int16_t *)(sm + kSmStage);

    // ---- one-time set-up: weights, zeroed planes, barriers, tensor memory
    for (int i = tid; i < kPackedBytes / 16; i += kThreads)
        ((uint4 *)Wp)[i] = ((const uint4 *)P.packed)[i];
    for (int i = tid; i < kP2Bytes / 16; i += kThreads) ((uint4 *)X)[i] = make_uint4(0, 0, 0, 0);
    for (int i = tid; i < kPatchBytes / 16; i += kThreads) ((uint4 *)pb)[i] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        for (int b = 0; b < kNBar; ++b) mbar_init(&bar[b], bar_count(b));
        mbar_init(&pbar, 1);
        s_abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)), "n"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const long long nk = (P.n - blockIdx.x + gridDim.x - 1) / gridDim.x;  // patches of this CTA
    volatile int *abort_flag = &s_abort;

    if (warp < kEpiWarps) {
        // ================================================================ epilogue
        const int row = 32 * (warp & 3) + lane;  // accumulator row (TMEM lane)
        const int half = warp >> 2;              // channels 16*half .. +15 (blocks 2h, 2h+1)
        const uint32_t tq = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(16 * half);
        unsigned char *P3 = X + kP3Off, *P4 = X + kP4Off, *P5 = X + kP5Off;
        const float *bias = (const float *)(Wp + kPkBias);
        // destinations (16-byte units) of this thread's rows for channel block
        // 2*half; block 2*half+1 is one plane set further; -1: junk row
        int d1[9], d2[3], d3, d4, d5;
#pragma unroll
        for (int mt = 0; mt < 9; ++mt) {
            const int m = mt * 128 + row, y = m / 34, x = m % 34;
            d1[mt] = (y < 33 && x < 33)
                         ? (2 * half * 4 + (((y & 1) << 1) | (x & 1))) * kPln2 + ((y >> 1) + 1) * 18 + (x >> 1) + 1
                         : -1;
        }
#pragma unroll
        for (int mt = 0; mt < 3; ++mt) {
            const int m = mt * 128 + row, y = m / 18, x = m % 18;
            d2[mt] = (y < 17 && x < 17)
                         ? (2 * half * 4 + (((y & 1) << 1) | (x & 1))) * kPln3 + ((y >> 1) + 1) * 10 + (x >> 1) + 1
                         : -1;
        }
        {
            int y = row / 10, x = row % 10;
            d3 = (y < 9 && x < 9)
                     ? (2 * half * 4 + (((y & 1) << 1) | (x & 1))) * kPln4 + ((y >> 1) + 1) * 6 + (x >> 1) + 1
                     : -1;
            y = row / 6; x = row % 6;
            d4 = (y < 5 && x < 5) ? 2 * half * kPln5 + (y + 1) * 7 + (x + 1) : -1;
            y = row / 7; x = row % 7;
            d5 = (y < 5 && x < 5) ? y * 5 + x : -1;
        }
        auto load_bias = [&](int l, float *b) {
#pragma unroll
            for (int c = 0; c < 16; ++c) b[c] = bias[32 * l + 16 * half + c];
        };
        auto put2 = [&](unsigned char *base, int d, int next, uint4 lo, uint4 hi) {
            *(uint4 *)(base + (long long)d * 16) = lo;
            *(uint4 *)(base + (long long)(d + next) * 16) = hi;
        };
        auto save2 = [&](unsigned char *sv, int off, int pix, uint4 lo, uint4 hi) {
            unsigned char *o = sv + off + pix * 64 + half * 32;
            *(uint4 *)o = lo;
            *(uint4 *)(o + 16) = hi;
        };
        // this thread's cells u = tid + 256 i of the overlapped region that a
        // layer switch clears (bit i)
        constexpr int kCellIters = (kP345Cells + kEpiThreads - 1) / kEpiThreads;
        uint32_t clr345 = 0u, clr2 = 0u;
#pragma unroll
        for (int i = 0; i < kCellIters; ++i) {
            const int u = tid + i * kEpiThreads;
            if (u < kP345Cells) {
                clr345 |= (uint32_t)p345_unwritten(u) << i;
                clr2 |= (uint32_t)p2_unwritten(u) << i;
            }
        }
        auto clear_cells = [&](uint32_t mask) {
#pragma unroll
            for (int i = 0; i < kCellIters; ++i)
                if ((mask >> i) & 1u) ((uint4 *)X)[tid + i * kEpiThreads] = make_uint4(0, 0, 0, 0);
        };
        bool ok = true;
        float bl[16], acc[16];
        for (long long k = 0; k < nk; ++k) {
            // a timed-out wait anywhere stops every epilogue thread here, together
            if (group_any(1, kEpiThreads, !ok || *abort_flag)) {
                ok = false;
                break;
            }
            const uint32_t ph = (uint32_t)(k & 1);
            const long long pi = blockIdx.x + k * gridDim.x;
            unsigned char *sv = P.save ? P.save + pi * (long long)kSaveBytesTotal : nullptr;
            // ---- conv1 epilogue -> conv2 input planes, three tiles per wait
            load_bias(0, bl);
#pragma unroll
            for (int g = 0; g < 3; ++g) {
                ok &= mbar_wait(&bar[kBarC1 + g], ph);
                tc_fence_after();
                float a3[3][16];
                tmem_ld16x3(tq + (uint32_t)(96 * g), tq + (uint32_t)(96 * g + 32), tq + (uint32_t)(96 * g + 64), a3);
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const int mt = 3 * g + i;
                    if (d1[mt] >= 0) {
                        const uint4 lo = relu_pack8(a3[i], bl), hi = relu_pack8(a3[i] + 8, bl + 8);
                        put2(X, d1[mt], 4 * kPln2, lo, hi);
                        if (sv) {
                            const int m = mt * 128 + row;
                            save2(sv, kSvA1, (m / 34) * 33 + m % 34, lo, hi);
                        }
                    }
                }
                if (g == 1) {
                    // tiles 0..5 hold every input row that conv2's first tile reads
                    fence_proxy_async_smem();
                    mbar_arrive(&bar[kBarP2a]);
                }
            }
            tc_fence_before();
            mbar_arrive(&bar[kBarC1Free]);
            fence_proxy_async_smem();
            mbar_arrive(&bar[kBarP2]);
            // ---- conv2 epilogue: all three tiles read, then the region is
            // refilled with the conv3 input planes
            load_bias(1, bl);
            uint4 o2[3][2];
#pragma unroll
            for (int mt = 0; mt < 3; ++mt) {
                ok &= mbar_wait(&bar[kBarC2 + mt], ph);
                tc_fence_after();
                tmem_ld16(tq + (uint32_t)(kColL2 + 32 * mt), acc);
                o2[mt][0] = relu_pack8(acc, bl);
                o2[mt][1] = relu_pack8(acc + 8, bl + 8);
            }
            clear_cells(clr345);  // conv2 has completed: its input is dead
#pragma unroll
            for (int mt = 0; mt < 3; ++mt) {
                if (d2[mt] >= 0) {
                    put2(P3, d2[mt], 4 * kPln3, o2[mt][0], o2[mt][1]);
                    if (sv) {
                        const int m = mt * 128 + row;
                        save2(sv, kSvA2, (m / 18) * 17 + m % 18, o2[mt][0], o2[mt][1]);
                    }
                }
            }
            tc_fence_before();
            fence_proxy_async_smem();
            mbar_arrive(&bar[kBarP3]);
            // ---- conv3 epilogue -> conv4 input planes
            load_bias(2, bl);
            ok &= mbar_wait(&bar[kBarC3], ph);
            tc_fence_after();
            tmem_ld16(tq + (uint32_t)kColL3, acc);
            if (d3 >= 0) {
                const uint4 lo = relu_pack8(acc, bl), hi = relu_pack8(acc + 8, bl + 8);
                put2(P4, d3, 4 * kPln4, lo, hi);
                if (sv) save2(sv, kSvA3, (row / 10) * 9 + row % 10, lo, hi);
            }
            tc_fence_before();
            fence_proxy_async_smem();
            mbar_arrive(&bar[kBarP4]);
            // ---- conv4 epilogue -> conv5 input plane (stride 1)
            load_bias(3, bl);
            ok &= mbar_wait(&bar[kBarC4], ph);
            tc_fence_after();
            tmem_ld16(tq + (uint32_t)kColL4, acc);
            if (d4 >= 0) {
                const uint4 lo = relu_pack8(acc, bl), hi = relu_pack8(acc + 8, bl + 8);
                put2(P5, d4, kPln5, lo, hi);
                if (sv) save2(sv, kSvA4, (row / 6) * 5 + row % 6, lo, hi);
            }
            tc_fence_before();
            fence_proxy_async_smem();
            mbar_arrive(&bar[kBarP5]);
            // ---- conv5 epilogue -> pooling buffer (once the head has read
            // the previous patch's)
            load_bias(4, bl);
            ok &= mbar_wait(&bar[kBarC5], ph);
            tc_fence_after();
            tmem_ld16(tq + (uint32_t)kColL5, acc);
            tc_fence_before();
            if (k > 0) ok &= mbar_wait(&bar[kBarGapFree], ph ^ 1u);
            if (d5 >= 0) {
                const uint4 lo = relu_pack8(acc, bl), hi = relu_pack8(acc + 8, bl + 8);
                const __nv_bfloat16 *h0 = (const __nv_bfloat16 *)&lo, *h1 = (const __nv_bfloat16 *)&hi;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    gap[d5 * 32 + 16 * half + c] = __bfloat162float(h0[c]);
                    gap[d5 * 32 + 16 * half + 8 + c] = __bfloat162float(h1[c]);
                }
                if (sv) save2(sv, kSvA5, d5, lo, hi);
            }
            mbar_arrive(&bar[kBarGap]);
            clear_cells(clr2);  // conv5 has completed: the conv3..5 planes are dead
        }
        if (!ok) *abort_flag = 1;
        if (!ok && P.status && tid == 0) atomicExch(P.status, VS_ERR_TIMEOUT);
    } else if (warp < kMmaWarp) {
        // ================================================================ front
        const int ft = tid - kEpiThreads, fw = warp - kEpiWarps;
        const float *fc = (const float *)(Wp + kPkFc);
        auto stage_patch = [&](int cy, int cx) {
            const int x0 = floordiv(cx - 32, 8) * 8;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&pbar, (uint32_t)(kPatch * kStageW * 2));
            tma_load_3d(stage, &tmap, 0, x0 / 8, cy - 32, &pbar);
        };
        bool ok = true;
        uint32_t pphase = 0u;
        bool pending = false;  // a TMA load of a patch is in flight
        if (ft == 0 && nk > 0) {
            int y, x;
            patch_rc(P, blockIdx.x, y, x);
            if (patch_inside(P, y, x)) stage_patch(y, x);
        }
        // iteration k: front end of patch k (k < nk), head of patch k - 2
        for (long long k = 0; k < nk + 2; ++k) {
            if (group_any(2, kFrontThreads, !ok || *abort_flag)) {
                ok = false;
                break;
            }
            const long long pi = blockIdx.x + k * gridDim.x;
            if (k < nk) {
                int cy, cx;
                patch_rc(P, pi, cy, cx);
                int16_t pv[kPerFront];
                if (patch_inside(P, cy, cx)) {
                    ok &= mbar_wait(&pbar, pphase);
                    pphase ^= 1u;
                    const int off = (cx - 32) - floordiv(cx - 32, 8) * 8;
#pragma unroll
                    for (int j = 0; j < kPerFront; ++j) {
                        const int e = ft + j * kFrontThreads, r = e / kPatch, c = e - r * kPatch;
                        pv[j] = (e < kPatch * kPatch) ? stage[r * kStageW + off + c] : (int16_t)0;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < kPerFront; ++j) {
                        const int e = ft + j * kFrontThreads, r = e / kPatch, c = e - r * kPatch;
                        const int gy = min(max(cy + (r - 32) * P.step, 0), P.H - 1);
                        const int gx = min(max(cx + (c - 32) * P.step, 0), P.W - 1);
                        pv[j] = (e < kPatch * kPatch) ? P.z[(long long)gy * P.pitch + gx] : (int16_t)0;
                    }
                }
                int sum = 0;
#pragma unroll
                for (int j = 0; j < kPerFront; ++j) sum += pv[j];
                for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
                if (lane == 0) s_red[fw] = sum;
                group_sync(2, kFrontThreads);
                // the staging tile has been read: prefetch the next patch
                pending = false;
                if (k + 1 < nk) {
                    int y, x;
                    patch_rc(P, pi + gridDim.x, y, x);
                    if (patch_inside(P, y, x)) {
                        pending = true;
                        if (ft == 0) stage_patch(y, x);
                    }
                }
                int tot = 0;
#pragma unroll
                for (int q = 0; q < kFrontWarps; ++q) tot += s_red[q];
                const float mean = (float)tot / (float)(kPatch * kPatch);
                unsigned char *sv = P.save ? P.save + pi * (long long)kSaveBytesTotal : nullptr;
#pragma unroll
                for (int j = 0; j < kPerFront; ++j) {
                    const int e = ft + j * kFrontThreads, r = e / kPatch, c = e - r * kPatch;
                    if (e < kPatch * kPatch) {
                        const __nv_bfloat16 x = __float2bfloat16_rn(((float)pv[j] - mean) * 1.0e-3f);
                        pb[(r + 1) * 67 + (c + 1)] = x;
                        if (sv) ((__nv_bfloat16 *)(sv + kSvInput))[e] = x;
                    }
                }
            }
            // ---- head of patch k - 2: global average pool, fc, sigmoid
            // (fixed summation order), by the first front warp
            if (k >= 2 && fw == 0) {
                const long long ph2 = k - 2;
                bool w = mbar_wait(&bar[kBarGap], (uint32_t)(ph2 & 1));
                float gv[25];
#pragma unroll
                for (int r = 0; r < 25; ++r) gv[r] = gap[r * 32 + lane];
                __syncwarp();
                mbar_arrive(&bar[kBarGapFree]);
                float g = 0.f;
#pragma unroll
                for (int r = 0; r < 25; ++r) g += gv[r];
                g *= (1.0f / 25.0f);
                float t = g * fc[lane];
                for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
                const long long p2 = blockIdx.x + ph2 * gridDim.x;
                unsigned char *sv = P.save ? P.save + p2 * (long long)kSaveBytesTotal : nullptr;
                if (lane == 0) {
                    const float logit = t + fc[32];
                    const float yv = 1.0f / (1.0f + expf(-logit));
                    P.out[p2] = yv;
                    if (sv) {
                        float *hd = (float *)(sv + kSvHead);
                        hd[32] = logit;
                        hd[33] = yv;
                    }
                }
                if (sv) ((float *)(sv + kSvHead))[lane] = g;
                ok &= w;
            }
            if (k < nk) {
                group_sync(2, kFrontThreads);
                // im2col of this patch once the previous patch's conv1 has read U
                if (k > 0) ok &= mbar_wait(&bar[kBarC1 + 2], (uint32_t)((k - 1) & 1));
#pragma unroll
                for (int j0 = 0; j0 < kRowsFront; j0 += 3) {
                    uint32_t w[3][5];
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const int m = ft + (j0 + j) * kFrontThreads, y = m / 34, x = m % 34;
                        const unsigned short *src = (const unsigned short *)pb + (2 * y) * 67 + 2 * x;
                        const bool live = m < 1152 && y < 33 && x < 33;
                        uint32_t t[9];
#pragma unroll
                        for (int q = 0; q < 9; ++q) t[q] = live ? (uint32_t)src[(q / 3) * 67 + (q % 3)] : 0u;
#pragma unroll
                        for (int q = 0; q < 4; ++q) w[j][q] = t[2 * q] | (t[2 * q + 1] << 16);
                        w[j][4] = t[8];
                    }
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const int m = ft + (j0 + j) * kFrontThreads;
                        if (m < 1152) {
                            unsigned char *dst = U + (m / 8) * 256 + (m % 8) * 16;
                            *(uint4 *)dst = make_uint4(w[j][0], w[j][1], w[j][2], w[j][3]);
                            *(uint4 *)(dst + 128) = make_uint4(w[j][4], 0u, 0u, 0u);
                        }
                    }
                }
                fence_proxy_async_smem();
                mbar_arrive(&bar[kBarURdy]);
            }
        }
        // leave no TMA load in flight
        if (pending && ft == 0) mbar_wait(&pbar, pphase);
        if (!ok) *abort_flag = 1;
        if (!ok && P.status && ft == 0) atomicExch(P.status, VS_ERR_TIMEOUT);
    } else {
        // ================================================================ MMA issue
        const uint32_t sW = smem_u32(Wp), sX = smem_u32(X), sU = smem_u32(U);
        // descriptor bases; an operand at byte offset o from a base adds o >> 4
        // to the address field (shared addresses stay below 2^18 bytes)
        const uint64_t dB = sdesc(sW, 128, 256);
        const uint64_t dA1 = sdesc(sU, 128, 256);
        const uint64_t dA2 = sdesc(sX, 4 * kPln2 * 16, 128);
        const uint64_t dA3 = sdesc(sX + kP3Off, 4 * kPln3 * 16, 128);
        const uint64_t dA4 = sdesc(sX + kP4Off, 4 * kPln4 * 16, 128);
        const uint64_t dA5 = sdesc(sX + kP5Off, kPln5 * 16, 128);
        bool ok = true;
        int last = -1;  // barrier of the last commit, for the exit wait
        uint32_t last_ph = 0u;
        auto wait_all = [&](int b, uint32_t ph) {
            bool r = true;
            if (lane == 0) r = mbar_wait_spin(&bar[b], ph);
            r = __shfl_sync(0xffffffffu, (int)r, 0) != 0;
            tc_fence_after();
            return r;
        };
        // a 32->32 layer's tile: 9 taps x 2 K-steps reading stride-2 parity planes
        auto conv_tile = [&](uint64_t dA, int pln, int pitch, int m0, int l, uint32_t col) {
#pragma unroll
            for (int i = 0; i < 18; ++i) {
                const int t = i >> 1, ks = i & 1, ky = t / 3, kx = t % 3;
                const int plane = ((ky != 1) << 1) | (kx != 1);
                const int shift = (ky != 0 ? pitch : 0) + (kx != 0 ? 1 : 0);
                const uint64_t ad = dA + (uint64_t)((2 * ks * 4 + plane) * pln + m0 + shift);
                const uint64_t bd = dB + (uint64_t)((pk_bl(l) + (t * 2 + ks) * 1024) >> 4);
                if (i == 0) umma_c<0>(tmem + col, ad, bd);
                else umma_c<1>(tmem + col, ad, bd);
            }
        };
        for (long long k = 0; k < nk; ++k) {
            if (__any_sync(0xffffffffu, !ok || *abort_flag)) break;
            const uint32_t ph = (uint32_t)(k & 1);
            // ---- conv1: the im2col tile is written and the previous patch's
            // conv1 accumulators have been read
            ok &= wait_all(kBarURdy, ph);
            if (k > 0) ok &= wait_all(kBarC1Free, ph ^ 1u);
            if (lane == 0) {
#pragma unroll
                for (int mt = 0; mt < 9; ++mt) {
                    umma_c<0>(tmem + (uint32_t)(32 * mt), dA1 + (uint64_t)(mt * 256), dB + (uint64_t)(kPkB1 >> 4));
                    if (mt % 3 == 2) umma_commit(&bar[kBarC1 + mt / 3]);
                }
            }
            __syncwarp();
            // ---- conv2: 3 tiles, input pitch 18; the first needs conv1 tiles 0..5
            ok &= wait_all(kBarP2a, ph);
            if (lane == 0) {
                conv_tile(dA2, kPln2, 18, 0, 1, (uint32_t)kColL2);
                umma_commit(&bar[kBarC2]);
            }
            __syncwarp();
            ok &= wait_all(kBarP2, ph);
            if (lane == 0) {
                for (int mt = 1; mt < 3; ++mt) {
                    conv_tile(dA2, kPln2, 18, mt * 128, 1, (uint32_t)(kColL2 + 32 * mt));
                    umma_commit(&bar[kBarC2 + mt]);
                }
            }
            __syncwarp();
            // ---- conv3: 1 tile, input pitch 10
            ok &= wait_all(kBarP3, ph);
            if (lane == 0) {
                conv_tile(dA3, kPln3, 10, 0, 2, (uint32_t)kColL3);
                umma_commit(&bar[kBarC3]);
            }
            __syncwarp();
            // ---- conv4: 1 tile, input pitch 6
            ok &= wait_all(kBarP4, ph);
            if (lane == 0) {
                conv_tile(dA4, kPln4, 6, 0, 3, (uint32_t)kColL4);
                umma_commit(&bar[kBarC4]);
            }
            __syncwarp();
            // ---- conv5 (stride 1): 1 tile, input pitch 7, one plane with a full border
            ok &= wait_all(kBarP5, ph);
            if (lane == 0) {
#pragma unroll
                for (int i = 0; i < 18; ++i) {
                    const int t = i >> 1, ks = i & 1, ky = t / 3, kx = t % 3;
                    const uint64_t ad = dA5 + (uint64_t)((2 * ks) * kPln5 + ky * 7 + kx);
                    const uint64_t bd = dB + (uint64_t)((pk_bl(4) + (t * 2 + ks) * 1024) >> 4);
                    if (i == 0) umma_c<0>(tmem + (uint32_t)kColL5, ad, bd);
                    else umma_c<1>(tmem + (uint32_t)kColL5, ad, bd);
                }
                umma_commit(&bar[kBarC5]);
            }
            __syncwarp();
            last = kBarC5;
            last_ph = ph;
        }
        // leave no MMA in flight
        if (last >= 0) wait_all(last, last_ph);
        if (!ok) *abort_flag = 1;
        if (!ok && P.status && lane == 0) atomicExch(P.status, VS_ERR_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(kTmemCols)
                     : "memory");
}

// ------------------------------------------------------------------ training
// Backward pass, layer by layer over a batch (the forward kernel saved every
// activation).  Each CTA keeps its partial weight gradient in shared memory
// over the patches it owns and adds it to the global gradient once, so the
// global atomics do not scale with the batch.  Products take bf16-valued
// operands (saved activations, bf16-rounded weights, bf16-rounded

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
    vs::note_launch();
    VS_CUDA_TRY(cudaGetLastError());
    return VS_OK;
}

static int cnn_forward_launch(vs_grid g, const int64_t *centers, int64_t n, int32_t stride,
                              int32_t row0, int32_t patch_step, const void *packed, float *out,
                              void *save, int32_t *status, vs_stream_t st) {
    if (patch_step < 1 || patch_step > 64) return VS_ERR_RANGE;
    int rc = check_grid(g);
    if (rc) return rc;
    if ((long long)g.H * g.W > 0xFFFFFFFFll) return VS_ERR_RANGE;  // posts are 32-bit in the kernel
    if (!packed || !out || ((uintptr_t)packed & 15) || (save && ((uintptr_t)save & 15)))
        return VS_ERR_ARG;
    if (n < 0) return VS_ERR_RANGE;
    if (n == 0) return VS_OK;
    if ((rc = check_device())) return rc;
    cnn::FwdParams P;
    P.z = g.z; P.H = g.H; P.W = g.W; P.pitch = g.pitch;
    P.centers = centers; P.n = n; P.stride = stride; P.step = patch_step; P.row0 = row0;
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
    vs::note_launch();
    VS_CUDA_TRY(cudaGetLastError());
    return VS_OK;
}

extern "C" int vs_cnn_forward(vs_grid g, const int64_t *centers, int64_t n, int32_t patch_step,
                              const void *packed, float *out, void *save, int32_t *status,
                              vs_stream_t st) {
    if (!centers && n > 0) return VS_ERR_ARG;
    return cnn_forward_launch(g, centers, n, 0, 0, patch_step, packed, out, save, status, st);
}

extern "C" int vs_cnn_score_lattice(vs_grid g, int32_t stride, int32_t patch_step, const void *packed,
                                    float *score_out, int32_t *status, vs_stream_t st) {
    if (stride < 1) return VS_ERR_RANGE;
    if (g.H < 1 || g.W < 1) return VS_ERR_RANGE;
    const int64_t Hs = (g.H + stride - 1) / stride, Ws = (g.W + stride - 1) / stride;
    return cnn_forward_launch(g, nullptr, Hs * Ws, stride, 0, patch_step, packed, score_out, nullptr,
                              status, st);
}

extern "C" int vs_cnn_score_lattice_rows(vs_grid g, int32_t stride, int32_t patch_step, int32_t row0,
                                         int32_t nrows, const void *packed, float *score_out,
                                         int32_t *status, vs_stream_t st) {
    if (stride < 1) return VS_ERR_RANGE;
    if (g.H < 1 || g.W < 1) return VS_ERR_RANGE;
    const int64_t Hs = (g.H + stride - 1) / stride, Ws = (g.W + stride - 1) / stride;
    if (row0 < 0 || nrows < 0 || (int64_t)row0 + nrows > Hs) return VS_ERR_RANGE;
    return cnn_forward_launch(g, nullptr, (int64_t)nrows * Ws, stride, row0, patch_step, packed, score_out,
                              nullptr, status, st);
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
    vs::note_launch();
    VS_CUDA_TRY(cudaGetLastError());
    return VS_OK;
}
