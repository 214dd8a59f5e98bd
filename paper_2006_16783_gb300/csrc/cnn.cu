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
// entirely on chip, its warps split into roles (conv1 group, conv2..5 group,
// front end, MMA issue; see the role table below) that hand work to each
// other through mbarriers, with two patches in flight: the conv1 group and
// the conv1/conv2 MMAs of patch k+1 run beside the conv3..5 chain of patch k,
// whose MMAs the conv2..5 group issues itself (two MMA issuers share the
// tensor core).
// Every convolution is an implicit GEMM on the 5th-generation tensor cores:
// tcgen05.mma kind::f16 (BF16 x BF16 -> FP32), M = 128 output pixels,
// N = 32 channels, K = 16 per instruction, the FP32 accumulator in tensor
// memory (32 columns per tile), read back with tcgen05.ld for the bias +
// ReLU + BF16 epilogue.  Operands:
//   * A stride-2 layer's input is stored in shared memory as four parity
//     planes (even/odd row x even/odd column) in blocks of 8 channels, each
//     plane with a zero border row/column and a row pitch of (output width
//     + 1) pixels.  For output pixel m = y*pitch + x, tap (ky,kx) reads plane
//     (ky != 1, kx != 1) at m + (ky != 0)*pitch + (kx != 0): every tap of a
//     128-pixel tile is one contiguous run of 16-byte rows, i.e. a plain
//     matrix descriptor (no swizzle, K-major 8x16-byte core matrices; leading
//     offset = next 8-channel block, stride offset = next 8 pixels).  The one
//     junk column per row is discarded.
//   * The stride-1 last layer uses one plane with a border on all sides.
//   * The 1-channel first layer takes A from tensor memory: the conv1 group
//     writes each output pixel's 9 taps (K padded to 16) into its TMEM lane
//     with tcgen05.st, so the im2col tile needs no shared memory.
//   * B (the weights) always comes from shared memory.
// At N = 32 an MMA with A in shared memory costs ~46 cycles whatever N <= 64
// (measured): it is bound by the shared-memory operand reads, so the 108
// MMAs of conv2..5 bound the kernel at ~5K cycles per patch and SM; the rest
// of a patch's time is the epilogue / hand-off latency of the conv3..5 chain,
// which the second patch in flight overlaps.
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
constexpr int kSmP2 = ((kSmW + kPackedBytes) + 127) & ~127;  // conv2 input planes
constexpr int kP2Bytes = (16 * kPln2 + 96) * 16;
// conv3..5 input planes, each followed by the cells that the last taps'
// descriptors run over (read as zero, never written)
constexpr int kSmP345 = ((kSmP2 + kP2Bytes) + 127) & ~127;
constexpr int kP3Off = 0, kP3Bytes = (16 * kPln3 + 40) * 16;
constexpr int kP4Off = kP3Off + kP3Bytes, kP4Bytes = (16 * kPln4 + 104) * 16;
constexpr int kP5Off = kP4Off + kP4Bytes, kP5Bytes = (4 * kPln5 + 100) * 16;
constexpr int kP345Bytes = kP5Off + kP5Bytes;
// the normalised patch, bf16 with a zero border, rows of kPbPitch = 66 elements: row r + 1 holds x0[r][0..64]
// at 1..65, and its right border is the next row's left border (both zero).  An even pitch of 33 words
// keeps the conv1 operand's loads free of bank conflicts where a warp's pixels wrap to the next output row.
constexpr int kPbPitch = 66;
constexpr int kSmPatch = ((kSmP345 + kP345Bytes) + 127) & ~127;
constexpr int kPatchBytes = (((67 * kPbPitch + 1) * 2) + 127) & ~127;
constexpr int kNGap = 3;  // pooling buffers (ring), each [32 channels][25 pixels] fp32
constexpr int kGapBytes = 25 * 32 * 4;
constexpr int kSmGap = kSmPatch + kPatchBytes;
constexpr int kSmStage = ((kSmGap + kNGap * kGapBytes) + 127) & ~127;  // TMA-staged patch
constexpr int kStageW = 72;                                   // 65 columns + 8-alignment slack
constexpr int kStageBytes = ((kPatch * kStageW * 2) + 127) & ~127;
constexpr int kSmEnd = kSmStage + kStageBytes;
constexpr int kSmemBytes = kSmEnd + 128;                     // + base alignment slack
static_assert(kSmemBytes + 512 <= kSmemLimit, "forward plan exceeds shared memory");

// instruction descriptors: kind::f16, A = B = BF16, D = F32, K-major A and
// B, N = 32, M = 128 or 64.  An M = 64 tile's row r lands in TMEM lane
// 32 * (r / 16) + r % 16 (lanes 0..15 of each quarter).
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) |
                            ((128u >> 4) << 24);
constexpr uint32_t kIdesc64 = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) |
                              ((64u >> 4) << 24);

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
//   warps 0..3   conv1 group: patch k's conv1 operand (im2col: 9 taps of an
//                output pixel into its TMEM lane) and conv1 epilogue (TMEM ->
//                bias + ReLU + bf16 -> conv2 input planes); thread: one
//                accumulator row, 32 channels
//   warps 4..7   conv2..5 group: the conv2 epilogue, then conv3, conv4 and
//                conv5 (their MMAs issued by one thread of the group once
//                the group has written the layer's input) and epilogues
//                (-> conv3, conv4, conv5 input planes, pooling buffer);
//                thread: one accumulator row, 32 channels
//   warps 8..14  front: a later patch's posts, mean and normalisation, and
//                the head (pool, fc, sigmoid) of an earlier one
//   warp 15      MMA issue (one lane): conv1 and conv2 of each patch, so
//                that they run beside the conv3..5 chain of the patch before
constexpr int kAWarps = 4, kBWarps = 4, kFrontWarps = 7;
constexpr int kBWarp0 = kAWarps, kFrontWarp0 = kAWarps + kBWarps, kMmaWarp = kFrontWarp0 + kFrontWarps;
constexpr int kAThreads = kAWarps * 32, kBThreads = kBWarps * 32, kFrontThreads = kFrontWarps * 32;
constexpr int kRowsFront = (kPatch + kFrontWarps - 1) / kFrontWarps;  // window rows per front warp
static_assert((kMmaWarp + 1) * 32 == kThreads, "role split must cover the CTA");
static_assert(kAWarps == 4 && kBWarps == 4, "TMEM lane quarters: warp w reads lanes 32*(w%4)..+31");

// Tensor memory (512 columns): conv1 tiles 0..8, conv2 tiles 0..2 and one
// tile that conv3, conv4 and conv5 take in turn (32 FP32 columns each), and
// the conv1 A operand (8 columns of bf16 pairs per tile).
constexpr int kTmemCols = 512;
constexpr int kColL2 = 9 * 32, kColL345 = 12 * 32, kColA1 = 13 * 32;
static_assert(kColA1 + 9 * 8 <= kTmemCols, "tensor memory plan");
// mbarriers, each completing once per patch (the pooling ring: once per
// kNGap patches):
//   tcgen05.commit     conv1 tiles in groups of three, conv2 tiles, conv3,
//                      conv4, conv5
//   conv1 group ->     conv1 operand written (MMA); conv1 accumulators read
//                      (MMA); conv1 tiles 0..5 written, i.e. every input row
//                      conv2's first tile reads (MMA); every conv2 input plane
//                      written (MMA); patch buffer read (front)
//   conv2..5 group ->  conv2 accumulators read (MMA); pooling buffer
//                      written (head)
//   front ->           normalised patch written (conv1 group)
//   head ->            pooling buffer read (conv2..5 group)
enum {
    kBarC1 = 0, kBarC2 = 3, kBarC3 = 6, kBarC4 = 7, kBarC5 = 8,
    kBarARdy = 9, kBarC1Free = 10, kBarP2a = 11, kBarP2 = 12, kBarPbFree = 13,
    kBarC2Free = 14,
    kBarGapFull = 15, kBarGapFree = kBarGapFull + kNGap, kBarPbRdy = kBarGapFree + kNGap,
    kNBar = kBarPbRdy + 1
};
// (arrivals: one per warp of the producing group, after a __syncwarp)
__host__ __device__ constexpr uint32_t bar_count(int b) {
    return b < kBarARdy ? 1u
           : b <= kBarPbFree ? (uint32_t)kAWarps
           : b < kBarGapFree ? (uint32_t)kBWarps
           : b < kBarPbRdy ? 1u
                           : (uint32_t)kFrontWarps;
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
// One arrival for the whole warp, after every lane's earlier writes and
// fences (the warp barrier orders them before lane 0's release).
__device__ __forceinline__ void warp_arrive(uint64_t *bar) {
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(bar);
}
// Lane 0 waits (bounded) and the warp continues together: the warp barrier
// orders lane 0's acquire before every lane's later reads (and, after a
// tcgen05.fence::after_thread_sync, before its tensor-memory loads).
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity) {
    int ok = 1;
    if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity) ? 1 : 0;
    __syncwarp();
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}
// one non-blocking look: has the barrier completed the phase of this parity?
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// 16 or 32 consecutive FP32 accumulator columns of this thread's TMEM lane,
// with one wait
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
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
    uint32_t r[32];
#define VS_R16(o) "=r"(r[o + 0]), "=r"(r[o + 1]), "=r"(r[o + 2]), "=r"(r[o + 3]), "=r"(r[o + 4]), \
    "=r"(r[o + 5]), "=r"(r[o + 6]), "=r"(r[o + 7]), "=r"(r[o + 8]), "=r"(r[o + 9]), "=r"(r[o + 10]), \
    "=r"(r[o + 11]), "=r"(r[o + 12]), "=r"(r[o + 13]), "=r"(r[o + 14]), "=r"(r[o + 15])
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : VS_R16(0), VS_R16(16)
        : "r"(taddr)
        : "memory");
#undef VS_R16
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
// 8 consecutive 32-bit columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t *w) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
                 "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// tensor-core MMA, A from shared memory; acc = 0 overwrites the accumulator
__device__ __forceinline__ void umma_s(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dt),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
// A 32->32 stride-2 layer's tile: 9 taps x 2 K-steps reading parity planes
// (descriptor bases dA, dB; an operand at byte offset o from a base adds o >> 4
// to the address field -- shared addresses stay below 2^18 bytes)
__device__ __forceinline__ void conv_tile(uint32_t dt, uint64_t dA, uint64_t dB, int pln, int pitch, int m0, int l,
                                          uint32_t idesc) {
#pragma unroll
    for (int i = 0; i < 18; ++i) {
        const int t = i >> 1, ks = i & 1, ky = t / 3, kx = t - 3 * ky;
        const int plane = ((ky != 1) << 1) | (kx != 1);
        const int shift = (ky != 0 ? pitch : 0) + (kx != 0 ? 1 : 0);
        const uint64_t ad = dA + (uint64_t)((2 * ks * 4 + plane) * pln + m0 + shift);
        const uint64_t bd = dB + (uint64_t)((pk_bl(l) + (t * 2 + ks) * 1024) >> 4);
        umma_s(dt, ad, bd, idesc, (uint32_t)i);
    }
}
// conv5 (stride 1): one plane with a full border, input pitch 7
__device__ __forceinline__ void conv5_tile(uint32_t dt, uint64_t dA5, uint64_t dB, uint32_t idesc) {
#pragma unroll
    for (int i = 0; i < 18; ++i) {
        const int t = i >> 1, ks = i & 1, ky = t / 3, kx = t - 3 * ky;
        const uint64_t ad = dA5 + (uint64_t)((2 * ks) * kPln5 + ky * 7 + kx);
        const uint64_t bd = dB + (uint64_t)((pk_bl(4) + (t * 2 + ks) * 1024) >> 4);
        umma_s(dt, ad, bd, idesc, (uint32_t)i);
    }
}
// tensor-core MMA, A from tensor memory (lane m = row m, K in bf16 pairs),
// overwriting the accumulator
__device__ __forceinline__ void umma_t0(uint32_t dt, uint32_t at, uint64_t bd) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(dt),
        "r"(at), "l"(bd), "r"(kIdesc), "n"(0));
}

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
    unsigned char *X2 = sm + kSmP2;      // conv2 input planes
    unsigned char *X345 = sm + kSmP345;  // conv3, conv4, conv5 input planes
    __nv_bfloat16 *pb = (__nv_bfloat16 *)(sm + kSmPatch);
    float *gap = (float *)(sm + kSmGap);
    int16_t *stage = (int16_t *)(sm + kSmStage);

    // ---- one-time set-up: weights; zeroed planes and patch buffer (their
    // borders are never written); barriers; tensor memory
    for (int i = tid; i < kPackedBytes / 16; i += kThreads)
        ((uint4 *)Wp)[i] = ((const uint4 *)P.packed)[i];
    for (int i = tid; i < (kSmGap - kSmP2) / 16; i += kThreads) ((uint4 *)X2)[i] = make_uint4(0, 0, 0, 0);
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

    if (warp < kBWarp0) {
        // ================================================================ conv1 group
        const int row = 32 * warp + lane;                          // TMEM lane
        const uint32_t tl = tmem + ((uint32_t)(32 * warp) << 16);  // this warp's lane quarter
        float b1[32];  // conv1 bias, held for the whole launch
#pragma unroll
        for (int c = 0; c < 32; c += 4) {
            const float4 v = *(const float4 *)(Wp + kPkBias + 4 * c);
            b1[c] = v.x;
            b1[c + 1] = v.y;
            b1[c + 2] = v.z;
            b1[c + 3] = v.w;
        }
        const unsigned short *pbu = (const unsigned short *)pb;
        bool ok = true;
        for (long long k = 0; k < nk; ++k) {
            // a timed-out wait anywhere stops every thread of the group here, together
            if (group_any(1, kAThreads, !ok || *abort_flag)) {
                ok = false;
                break;
            }
            const uint32_t ph = (uint32_t)(k & 1);
            const long long pi = blockIdx.x + k * gridDim.x;
            unsigned char *sv = P.save ? P.save + pi * (long long)kSaveBytesTotal : nullptr;
            // ---- conv1 operand: output pixel m = 34 y + x takes at K = 3 ky + kx
            // the input x0[2y - 1 + ky][2x - 1 + kx] (the patch buffer has a
            // zero border: x0[r][c] is pb[(r + 1) * kPbPitch + c + 1]).  The conv1
            // MMAs of patch k - 1, which read these columns, have completed:
            // this group waited for them before its epilogue.
            ok &= warp_wait(&bar[kBarPbRdy], ph);
            tc_fence_after();
#pragma unroll 1
            for (int mt = 0; mt < 9; ++mt) {
                const int m = mt * 128 + row, y = m / 34, x = m - 34 * y;
                const bool live = y < 33 && x < 33;
                const unsigned short *src = pbu + (2 * y) * kPbPitch + 2 * x;
                uint32_t t[9];
#pragma unroll
                for (int q = 0; q < 9; ++q) t[q] = live ? (uint32_t)src[(q / 3) * kPbPitch + (q % 3)] : 0u;
                uint32_t w[8];
#pragma unroll
                for (int q = 0; q < 4; ++q) w[q] = t[2 * q] | (t[2 * q + 1] << 16);
                w[4] = t[8];
                w[5] = w[6] = w[7] = 0u;
                tmem_st8(tl + (uint32_t)(kColA1 + 8 * mt), w);
            }
            tmem_wait_st();
            tc_fence_before();
            warp_arrive(&bar[kBarARdy]);
            if (lane == 0) mbar_arrive(&bar[kBarPbFree]);
            // ---- conv1 epilogue -> conv2 input planes, three tiles per
            // commit.  Group g writes plane rows 1..6, 6..12, 12..17; conv2
            // tile t of the previous patch reads (for its valid pixels) plane
            // rows 0..8, 7..15, 14..17, so group g waits for tile g of patch
            // k - 1 (commits complete in order).
#pragma unroll 1
            for (int g = 0; g < 3; ++g) {
                if (k > 0) ok &= warp_wait(&bar[kBarC2 + g], ph ^ 1u);
                ok &= warp_wait(&bar[kBarC1 + g], ph);
                tc_fence_after();
#pragma unroll 1
                for (int mt = 3 * g; mt < 3 * g + 3; ++mt) {
                    float a[32];
                    tmem_ld32(tl + (uint32_t)(32 * mt), a);
                    // conv2 input cell (16-byte unit, channel block 0; block cb
                    // is 4 cb planes further) of this thread's row; none for a
                    // junk column or padding row
                    const int m = mt * 128 + row, y = m / 34, x = m - 34 * y;
                    if (y < 33 && x < 33) {
                        const int d = (((y & 1) << 1) | (x & 1)) * kPln2 + ((y >> 1) + 1) * 18 + (x >> 1) + 1;
#pragma unroll
                        for (int cb = 0; cb < 4; ++cb) {
                            const uint4 v = relu_pack8(a + 8 * cb, b1 + 8 * cb);
                            *(uint4 *)(X2 + (long long)(d + cb * 4 * kPln2) * 16) = v;
                            if (sv) *(uint4 *)(sv + kSvA1 + (y * 33 + x) * 64 + cb * 16) = v;
                        }
                    }
                }
                if (g == 1) {
                    // tiles 0..5 hold every input row that conv2's first tile reads
                    fence_proxy_async_smem();
                    warp_arrive(&bar[kBarP2a]);
                }
            }
            tc_fence_before();
            fence_proxy_async_smem();
            warp_arrive(&bar[kBarC1Free]);
            if (lane == 0) mbar_arrive(&bar[kBarP2]);
        }
        if (!ok) *abort_flag = 1;
        if (!ok && P.status && tid == 0) atomicExch(P.status, VS_ERR_TIMEOUT);
    } else if (warp < kFrontWarp0) {
        // ================================================================ conv2..5 group
        const int wb = warp - kBWarp0;           // lane quarter
        const int row = 32 * wb + lane;          // accumulator row (TMEM lane)
        const uint32_t tq = tmem + ((uint32_t)(32 * wb) << 16);
        unsigned char *P3 = X345 + kP3Off, *P4 = X345 + kP4Off, *P5 = X345 + kP5Off;
        const float *bias = (const float *)(Wp + kPkBias);
        // destinations (16-byte units) of this thread's rows for channel
        // block 0 (block cb is 4 * cb planes further for the parity-plane
        // layouts, cb planes for conv5's); -1: junk row.  Rows of the M = 64
        // tiles (conv2 tile 2, conv4, conv5) are 16 * quarter + lane, held by
        // lanes 0..15.
        const int row64 = lane < 16 ? 16 * wb + lane : 64;
        int d3, d4, d5;
        {
            int y = row / 10, x = row % 10;
            d3 = (y < 9 && x < 9) ? (((y & 1) << 1) | (x & 1)) * kPln4 + ((y >> 1) + 1) * 6 + (x >> 1) + 1 : -1;
            y = row64 / 6; x = row64 % 6;
            d4 = (y < 5 && x < 5) ? (y + 1) * 7 + (x + 1) : -1;
            y = row64 / 7; x = row64 % 7;
            d5 = (y < 5 && x < 5) ? y * 5 + x : -1;
        }
        auto load_bias = [&](int l, float *b) {
#pragma unroll
            for (int c = 0; c < 32; c += 4) {
                const float4 v = *(const float4 *)(bias + 32 * l + c);
                b[c] = v.x;
                b[c + 1] = v.y;
                b[c + 2] = v.z;
                b[c + 3] = v.w;
            }
        };
        // bias + ReLU + bf16 of one accumulator row (32 channels) into four
        // 16-byte blocks at base + (d + cb * next) * 16, and the save record
        auto put4 = [&](unsigned char *base, int d, int next, const float *a, const float *bl, unsigned char *sv,
                        int off, int pix) {
#pragma unroll
            for (int cb = 0; cb < 4; ++cb) {
                const uint4 v = relu_pack8(const_cast<float *>(a) + 8 * cb, bl + 8 * cb);
                *(uint4 *)(base + (long long)(d + cb * next) * 16) = v;
                if (sv) *(uint4 *)(sv + off + pix * 64 + cb * 16) = v;
            }
        };
        // conv3, conv4 and conv5 are issued by one thread of this group once
        // the whole group has written their input (named barrier 2): the
        // chain conv3 -> epilogue -> conv4 -> ... stays inside the group
        const bool issuer = wb == 0 && lane == 0;
        const uint64_t dB = sdesc(smem_u32(Wp), 128, 256);
        const uint64_t dA3 = sdesc(smem_u32(P3), 4 * kPln3 * 16, 128);
        const uint64_t dA4 = sdesc(smem_u32(P4), 4 * kPln4 * 16, 128);
        const uint64_t dA5 = sdesc(smem_u32(P5), kPln5 * 16, 128);
        const uint32_t t345 = tmem + (uint32_t)kColL345;
        int last = -1;  // the issuer's last commit and its parity, for the exit wait
        uint32_t last_ph = 0u;
        bool ok = true;
        float bl[32], acc[32];
        for (long long k = 0; k < nk; ++k) {
            if (group_any(2, kBThreads, !ok || *abort_flag)) {
                ok = false;
                break;
            }
            const uint32_t ph = (uint32_t)(k & 1);
            const long long pi = blockIdx.x + k * gridDim.x;
            unsigned char *sv = P.save ? P.save + pi * (long long)kSaveBytesTotal : nullptr;
            // ---- conv2 epilogue -> conv3 input planes (which conv3 of
            // patch k - 1 has read: this group waited for it below), tile by
            // tile; after the last read the accumulators are free for the
            // next patch's conv2
            load_bias(1, bl);
#pragma unroll 1
            for (int mt = 0; mt < 3; ++mt) {
                ok &= warp_wait(&bar[kBarC2 + mt], ph);
                tc_fence_after();
                tmem_ld32(tq + (uint32_t)(kColL2 + 32 * mt), acc);
                if (mt == 2) {
                    tc_fence_before();
                    warp_arrive(&bar[kBarC2Free]);
                }
                const int m = mt < 2 ? mt * 128 + row : 256 + row64, y = m / 18, x = m - 18 * y;
                if (y < 17 && x < 17)
                    put4(P3, (((y & 1) << 1) | (x & 1)) * kPln3 + ((y >> 1) + 1) * 10 + (x >> 1) + 1, 4 * kPln3, acc,
                         bl, sv, kSvA2, y * 17 + x);
            }
            fence_proxy_async_smem();
            group_sync(2, kBThreads);  // conv3's input is written; conv5 of patch k-1 was read
            if (issuer) {
                tc_fence_after();
                conv_tile(t345, dA3, dB, kPln3, 10, 0, 2, kIdesc);
                umma_commit(&bar[kBarC3]);
                last = kBarC3;
                last_ph = ph;
            }
            // ---- conv3 epilogue -> conv4 input planes (the shared conv3..5
            // accumulator is free once read)
            load_bias(2, bl);
            ok &= warp_wait(&bar[kBarC3], ph);
            tc_fence_after();
            tmem_ld32(tq + (uint32_t)kColL345, acc);
            tc_fence_before();
            if (d3 >= 0) put4(P4, d3, 4 * kPln4, acc, bl, sv, kSvA3, (row / 10) * 9 + row % 10);
            fence_proxy_async_smem();
            group_sync(2, kBThreads);
            if (issuer) {
                tc_fence_after();
                conv_tile(t345, dA4, dB, kPln4, 6, 0, 3, kIdesc64);
                umma_commit(&bar[kBarC4]);
                last = kBarC4;
            }
            // ---- conv4 epilogue -> conv5 input plane (stride 1)
            load_bias(3, bl);
            ok &= warp_wait(&bar[kBarC4], ph);
            tc_fence_after();
            tmem_ld32(tq + (uint32_t)kColL345, acc);
            tc_fence_before();
            if (d4 >= 0) put4(P5, d4, kPln5, acc, bl, sv, kSvA4, (row64 / 6) * 5 + row64 % 6);
            fence_proxy_async_smem();
            group_sync(2, kBThreads);
            if (issuer) {
                tc_fence_after();
                conv5_tile(t345, dA5, dB, kIdesc64);
                umma_commit(&bar[kBarC5]);
                last = kBarC5;
            }
            // ---- conv5 epilogue -> pooling buffer k % kNGap, once the head
            // has read patch k - kNGap's
            load_bias(4, bl);
            ok &= warp_wait(&bar[kBarC5], ph);
            tc_fence_after();
            tmem_ld32(tq + (uint32_t)kColL345, acc);
            tc_fence_before();
            const int gb = (int)(k % kNGap);
            if (k >= kNGap) ok &= warp_wait(&bar[kBarGapFree + gb], (uint32_t)(((k - kNGap) / kNGap) & 1));
            float *gp = gap + gb * (kGapBytes / 4);
            if (d5 >= 0) {
#pragma unroll
                for (int cb = 0; cb < 4; ++cb) {
                    const uint4 v = relu_pack8(acc + 8 * cb, bl + 8 * cb);
                    const __nv_bfloat16 *h = (const __nv_bfloat16 *)&v;
#pragma unroll
                    for (int c = 0; c < 8; ++c) gp[(8 * cb + c) * 25 + d5] = __bfloat162float(h[c]);
                    if (sv) *(uint4 *)(sv + kSvA5 + d5 * 64 + cb * 16) = v;
                }
            }
            warp_arrive(&bar[kBarGapFull + gb]);
        }
        // leave no MMA in flight: the issuer's last commit completes after its earlier MMAs
        if (issuer && last >= 0) mbar_wait(&bar[last], last_ph);
        if (!ok) *abort_flag = 1;
        if (!ok && P.status && issuer) atomicExch(P.status, VS_ERR_TIMEOUT);
    } else if (warp < kMmaWarp) {
        // ================================================================ front
        const int ft = tid - kFrontWarp0 * 32, fw = warp - kFrontWarp0;
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
        if (nk > 0) {
            int y, x;
            patch_rc(P, blockIdx.x, y, x);
            if (patch_inside(P, y, x)) {
                pending = true;
                if (ft == 0) stage_patch(y, x);
            }
        }
        // iteration k: front end of patch k (k < nk), head of patch k - kNGap
        for (long long k = 0; k < nk + kNGap; ++k) {
            if (group_any(3, kFrontThreads, !ok || *abort_flag)) {
                ok = false;
                break;
            }
            const long long pi = blockIdx.x + k * gridDim.x;
            if (k < nk) {
                int cy, cx;
                patch_rc(P, pi, cy, cx);
                // thread (fw, lane) holds, in registers, rows fw + 7 i of the
                // 65 x 65 window at columns lane, lane + 32 (and 64 for lane 0)
                int16_t v[kRowsFront][3];
                if (patch_inside(P, cy, cx)) {
                    ok &= warp_wait(&pbar, pphase);
                    pphase ^= 1u;
                    pending = false;
                    const int off = (cx - 32) - floordiv(cx - 32, 8) * 8;
#pragma unroll
                    for (int i = 0; i < kRowsFront; ++i) {
                        const int16_t *row = stage + min(fw + kFrontWarps * i, kPatch - 1) * kStageW + off;
                        v[i][0] = row[lane];
                        v[i][1] = row[lane + 32];
                        v[i][2] = row[lane == 0 ? 64 : 0];
                    }
                } else {
                    // a window across the grid edge (or a strided one):
                    // clamped loads, all in flight together
                    const int gx0 = min(max(cx + (lane - 32) * P.step, 0), P.W - 1);
                    const int gx1 = min(max(cx + lane * P.step, 0), P.W - 1);
                    const int gx2 = min(max(cx + 32 * P.step, 0), P.W - 1);
#pragma unroll
                    for (int i = 0; i < kRowsFront; ++i) {
                        const int r = min(fw + kFrontWarps * i, kPatch - 1);
                        const int gy = min(max(cy + (r - 32) * P.step, 0), P.H - 1);
                        const int16_t *row = P.z + (long long)gy * P.pitch;
                        v[i][0] = row[gx0];
                        v[i][1] = row[gx1];
                        v[i][2] = row[gx2];
                    }
                }
                int sum = 0;
#pragma unroll
                for (int i = 0; i < kRowsFront; ++i)
                    if (fw + kFrontWarps * i < kPatch) sum += v[i][0] + v[i][1] + (lane == 0 ? v[i][2] : 0);
                for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
                if (lane == 0) s_red[fw] = sum;
                // every front thread has read the staging tile: prefetch the next patch
                group_sync(3, kFrontThreads);
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
                // the conv1 group has read patch k - 1 from the patch buffer
                if (k > 0) ok &= warp_wait(&bar[kBarPbFree], (uint32_t)((k - 1) & 1));
                unsigned char *sv = P.save ? P.save + pi * (long long)kSaveBytesTotal : nullptr;
                __nv_bfloat16 *x0s = sv ? (__nv_bfloat16 *)(sv + kSvInput) : nullptr;
#pragma unroll
                for (int i = 0; i < kRowsFront; ++i) {
                    const int r = fw + kFrontWarps * i;
                    if (r < kPatch) {
                        __nv_bfloat16 *dst = pb + (r + 1) * kPbPitch + 1;
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            const int c = lane + 32 * q;
                            if (q < 2 || lane == 0) {
                                const __nv_bfloat16 x = __float2bfloat16_rn(((float)v[i][q] - mean) * 1.0e-3f);
                                dst[c] = x;
                                if (x0s) x0s[r * kPatch + c] = x;
                            }
                        }
                    }
                }
                warp_arrive(&bar[kBarPbRdy]);
            }
            // ---- head of patch k - kNGap: global average pool, fc, sigmoid
            // (fixed summation order), by the first front warp
            if (k >= kNGap && fw == 0) {
                const long long hk = k - kNGap;
                const int gb = (int)(hk % kNGap);
                bool w = warp_wait(&bar[kBarGapFull + gb], (uint32_t)((hk / kNGap) & 1));
                const float *gp = gap + gb * (kGapBytes / 4);
                float gv[25];
#pragma unroll
                for (int r = 0; r < 25; ++r) gv[r] = gp[lane * 25 + r];
                warp_arrive(&bar[kBarGapFree + gb]);
                float g = 0.f;
#pragma unroll
                for (int r = 0; r < 25; ++r) g += gv[r];
                g *= (1.0f / 25.0f);
                float t = g * fc[lane];
                for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
                const long long p2 = blockIdx.x + hk * gridDim.x;
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
        }
        // leave no TMA load in flight
        if (pending && ft == 0) mbar_wait(&pbar, pphase);
        if (!ok) *abort_flag = 1;
        if (!ok && P.status && ft == 0) atomicExch(P.status, VS_ERR_TIMEOUT);
    } else {
        // ================================================================ MMA issue
        // conv1 (9 tiles, A from tensor memory) and conv2 (tile 0 once conv1
        // tiles 0..5 are written, tiles 1 and 2 once all are) of each patch
        if (lane == 0) {
            const uint64_t dB = sdesc(smem_u32(Wp), 128, 256);
            const uint64_t dA2 = sdesc(smem_u32(X2), 4 * kPln2 * 16, 128);
            bool ok = true;
            int last = -1;  // barrier of the last commit and its parity, for the exit wait
            uint32_t last_ph = 0u;
            auto wait = [&](int b, uint32_t ph, bool stop_on_abort = true) {
                uint32_t i = 0;
                while (!mbar_test(&bar[b], ph)) {
                    if (++i >= kWaitPolls || (stop_on_abort && (i & 1023u) == 0 && *abort_flag)) return false;
                }
                return true;
            };
            for (long long k = 0; k < nk && ok; ++k) {
                const uint32_t ph = (uint32_t)(k & 1);
                // conv1: its operand is written and the previous patch's
                // conv1 accumulators have been read
                ok = wait(kBarARdy, ph) && (k == 0 || wait(kBarC1Free, ph ^ 1u));
                if (!ok) break;
                tc_fence_after();
#pragma unroll
                for (int mt = 0; mt < 9; ++mt) {
                    umma_t0(tmem + (uint32_t)(32 * mt), tmem + (uint32_t)(kColA1 + 8 * mt), dB + (uint64_t)(kPkB1 >> 4));
                    if (mt % 3 == 2) umma_commit(&bar[kBarC1 + mt / 3]);
                }
                last = kBarC1 + 2;
                last_ph = ph;
                // conv2 tile 0: conv1 tiles 0..5 are in the planes and the
                // previous patch's conv2 accumulators have been read
                ok = wait(kBarP2a, ph) && (k == 0 || wait(kBarC2Free, ph ^ 1u));
                if (!ok) break;
                tc_fence_after();
                conv_tile(tmem + (uint32_t)kColL2, dA2, dB, kPln2, 18, 0, 1, kIdesc);
                umma_commit(&bar[kBarC2]);
                last = kBarC2;
                // conv2 tiles 1 and 2 (tile 2 holds output pixels 256..305: M = 64)
                ok = wait(kBarP2, ph);
                if (!ok) break;
                tc_fence_after();
                conv_tile(tmem + (uint32_t)(kColL2 + 32), dA2, dB, kPln2, 18, 128, 1, kIdesc);
                umma_commit(&bar[kBarC2 + 1]);
                conv_tile(tmem + (uint32_t)(kColL2 + 64), dA2, dB, kPln2, 18, 256, 1, kIdesc64);
                umma_commit(&bar[kBarC2 + 2]);
                last = kBarC2 + 2;
            }
            // leave no MMA in flight: the last commit completes after every earlier MMA
            if (last >= 0) wait(last, last_ph, false);
            if (!ok) {
                *abort_flag = 1;
                if (P.status) atomicExch(P.status, VS_ERR_TIMEOUT);
            }
        }
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(kTmemCols)
                     : "memory");
}

// ------------------------------------------------------------------ training
// The backward kernels are in cnn_bwd.cu; the optimiser step is here.

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
