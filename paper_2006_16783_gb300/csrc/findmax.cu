// findmax.cu -- Findmax stage (Sec. "The multiple transmitter siting
// process", Findmax): top-k posts of every block, ties to the lower index.
//
// One CTA per block.  Each post becomes a 64-bit key (value << 32 | ~p), so
// "larger key" is exactly "larger value, then lower post index" and keys are
// unique.  Round r takes the block-wide maximum over keys below the key
// chosen in round r-1; the first round streams the block from HBM and later
// rounds hit L2.  The CTA's output position is the sum of
// min(k, block size) over the blocks before it, computed in parallel.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "vs_common.cuh"

namespace vs {

constexpr int kFmThreads = 256;

__device__ __forceinline__ uint32_t value_key(uint8_t v) { return v; }
__device__ __forceinline__ uint32_t value_key(float v) {
    const uint32_t u = __float_as_uint(v);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ long long llmin(long long a, long long b) { return a < b ? a : b; }

__device__ __forceinline__ long long lattice_count(long long lo, long long hi, long long s) {
    if (hi <= lo) return 0;
    return (hi + s - 1) / s - (lo + s - 1) / s;
}

__device__ __forceinline__ uint64_t block_max_u64(uint64_t v, uint64_t *red) {
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    v = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// block blk (row-major over blocks) of one map; the CTA's threads all take part
constexpr int kFmCols = 2048, kFmRows = 2048;  // block-count tables of the output offset

template <typename V>
__device__ __forceinline__ void findmax_block(const V *val, int H, int W, int stride, int Ws, int b, int k,
                                              int nbx, int blk, int64_t *out, uint64_t *red,
                                              long long *s_offp, int *s_nx, int *s_ny) {
    long long &s_off = *s_offp;
    const int by = blk / nbx, bx = blk - (blk / nbx) * nbx;
    const long long i0 = ((long long)by * b + stride - 1) / stride;
    const long long i1 = llmin(((long long)(by + 1) * b + stride - 1) / stride,
                                             (H + stride - 1) / stride);
    const long long j0 = ((long long)bx * b + stride - 1) / stride;
    const long long j1 = llmin(((long long)(bx + 1) * b + stride - 1) / stride, Ws);
    const long long m = (i1 - i0) * (j1 - j0);

    // output offset: sum of min(k, size) over the blocks before this one.
    // Block (qy, qx) holds ny(qy) * nx(qx) lattice posts; with the row and
    // column counts in shared memory each thread sums one block column over
    // the rows before this one (plus this row's columns left of this block),
    // one multiply and min per term.  Grids of more block rows or columns
    // than the tables hold take a term per block instead.
    {
        long long acc = 0;
        if (nbx <= kFmCols && by < kFmRows) {
            for (int q = threadIdx.x; q < nbx; q += blockDim.x)
                s_nx[q] = (int)lattice_count((long long)q * b, llmin(W, (long long)(q + 1) * b), stride);
            for (int q = threadIdx.x; q <= by; q += blockDim.x)
                s_ny[q] = (int)lattice_count((long long)q * b, llmin(H, (long long)(q + 1) * b), stride);
            __syncthreads();
            for (int qx = threadIdx.x; qx < nbx; qx += blockDim.x) {
                const long long nx = s_nx[qx];
                long long a = 0;
                for (int qy = 0; qy < by; ++qy) a += llmin(k, (long long)s_ny[qy] * nx);
                if (qx < bx) a += llmin(k, (long long)s_ny[by] * nx);
                acc += a;
            }
        } else {
            for (int q = threadIdx.x; q < blk; q += blockDim.x) {
                const int qy = q / nbx, qx = q - (q / nbx) * nbx;
                const long long ny = lattice_count((long long)qy * b, llmin(H, (long long)(qy + 1) * b), stride);
                const long long nx = lattice_count((long long)qx * b, llmin(W, (long long)(qx + 1) * b), stride);
                acc += llmin(k, ny * nx);
            }
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (uint64_t)acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long t = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += (long long)red[w];
            s_off = t;
        }
        __syncthreads();
    }
    const long long off = s_off;

    uint64_t bound = ~0ull;
    const int rounds = (int)llmin(k, m);
    for (int r = 0; r < rounds; ++r) {
        uint64_t best = 0;
        const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (long long i = i0 + (threadIdx.x >> 5); i < i1; i += nw) {
            const V *row = val + i * Ws;
            const uint32_t prow = (uint32_t)(i * stride * (long long)W);
            for (int j = (int)j0 + lane; j < (int)j1; j += 32) {
                const uint32_t p = prow + (uint32_t)(j * stride);
                const uint64_t key = ((uint64_t)value_key(row[j]) << 32) | (uint64_t)(0xFFFFFFFFu - p);
                if (key < bound && key > best) best = key;
            }
        }
        best = block_max_u64(best, red);
        if (threadIdx.x == 0) out[off + r] = (int64_t)(0xFFFFFFFFu - (uint32_t)(best & 0xFFFFFFFFu));
        bound = best;
    }
    __syncthreads();  // red and s_off are reused by the CTA's next block
}

template <typename V>
__global__ void __launch_bounds__(kFmThreads) k_findmax(const V *val, int H, int W, int stride,
                                                        int Ws, int b, int k, int nbx,
                                                        int64_t *out) {
    __shared__ uint64_t red[32];
    __shared__ long long s_off;
    __shared__ int s_nx[kFmCols], s_ny[kFmRows];
    findmax_block<V>(val, H, W, stride, Ws, b, k, nbx, (int)blockIdx.x, out, red, &s_off, s_nx, s_ny);
}

// Many uint8 maps in one launch: the blocks of every job are numbered job by
// job and CTA i takes block i.
constexpr int kFmMaxJobs = 64;
struct FmJob {
    const uint8_t *val;
    int H, W, b, k, nbx;
    int64_t *out;
    long long blk0;  // first CTA of the job
};
struct FmBatch {
    FmJob job[kFmMaxJobs];
    int njobs;
};
__global__ void __launch_bounds__(kFmThreads) k_findmax_batch(const __grid_constant__ FmBatch B) {
    __shared__ uint64_t red[32];
    __shared__ long long s_off;
    __shared__ int s_nx[kFmCols], s_ny[kFmRows];
    int j = 0;
    while (j + 1 < B.njobs && B.job[j + 1].blk0 <= (long long)blockIdx.x) ++j;
    const FmJob &J = B.job[j];
    findmax_block<uint8_t>(J.val, J.H, J.W, 1, J.W, J.b, J.k, J.nbx, (int)(blockIdx.x - J.blk0), J.out, red, &s_off,
                           s_nx, s_ny);
}

// Single pass for uint8 maps and k <= KM: every thread keeps its own KM
// largest keys in registers while it streams its rows (4 posts per load);
// the block's top k are then taken from the threads' lists, k rounds of a
// block-wide maximum over the list heads.  Any key in the block's top k is
// in its thread's top k, so the result equals the multi-round kernel's.
template <int KM>
__global__ void __launch_bounds__(kFmThreads) k_findmax_u8(const uint8_t *__restrict__ val, int H,
                                                           int W, int b, int k, int nbx,
                                                           const long long *__restrict__ unused,
                                                           int64_t *out) {
    (void)unused;
    __shared__ uint64_t red[32];
    __shared__ long long s_off;
    const int by = blockIdx.x / nbx, bx = blockIdx.x - (blockIdx.x / nbx) * nbx;
    const int y0 = by * b, y1 = min(H, (by + 1) * b);
    const int x0 = bx * b, x1 = min(W, (bx + 1) * b);
    {
        // output offset: every block before this one gives min(k, its size)
        long long acc = 0;
        for (int q = threadIdx.x; q < (int)blockIdx.x; q += blockDim.x) {
            const int qy = q / nbx, qx = q - (q / nbx) * nbx;
            const long long ny = min(H, (qy + 1) * b) - qy * b, nx = min(W, (qx + 1) * b) - qx * b;
            acc += llmin(k, ny * nx);
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (uint64_t)acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long t = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += (long long)red[w];
            s_off = t;
        }
        __syncthreads();
    }
    uint64_t lst[KM];
#pragma unroll
    for (int i = 0; i < KM; ++i) lst[i] = 0;
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int y = y0 + (threadIdx.x >> 5); y < y1; y += nw) {
        const uint32_t prow = (uint32_t)y * (uint32_t)W;
        const uint32_t a = prow + (uint32_t)x0, e = prow + (uint32_t)x1;  // byte range [a, e)
        const uint32_t w0 = a >> 2, w1 = (e + 3) >> 2;
        const uint32_t *words = (const uint32_t *)val;
        for (uint32_t wi = w0 + lane; wi < w1; wi += 32) {
            const uint32_t v4 = __ldg(words + wi);
            // A thread meets its posts in increasing index order, so once its
            // list is full a post can enter only with a value above the
            // list's smallest (an equal value has a higher index, a smaller
            // key): a word whose largest byte is not above it is skipped.
            const uint32_t vmax = __vmaxu4(v4, __vmaxu4(v4 >> 8, v4 >> 16)) & 0xFFu;
            const uint32_t vmax4 = vmax > ((v4 >> 24) & 0xFFu) ? vmax : ((v4 >> 24) & 0xFFu);
            if (lst[KM - 1] != 0 && vmax4 <= (uint32_t)(lst[KM - 1] >> 32)) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t p = wi * 4 + j;
                if (p < a || p >= e) continue;
                const uint64_t key = ((uint64_t)((v4 >> (8 * j)) & 0xFFu) << 32) | (uint64_t)(0xFFFFFFFFu - p);
                if (key > lst[KM - 1]) {
                    lst[KM - 1] = key;
#pragma unroll
                    for (int i = KM - 1; i > 0; --i)
                        if (lst[i] > lst[i - 1]) { const uint64_t t = lst[i]; lst[i] = lst[i - 1]; lst[i - 1] = t; }
                }
            }
        }
    }
    const long long m = (long long)(y1 - y0) * (x1 - x0);
    const int rounds = (int)llmin(k, m);
    for (int r = 0; r < rounds; ++r) {
        const uint64_t best = block_max_u64(lst[0], red);
        if (lst[0] == best) {  // keys are unique: exactly one thread pops
#pragma unroll
            for (int i = 0; i < KM - 1; ++i) lst[i] = lst[i + 1];
            lst[KM - 1] = 0;
        }
        if (threadIdx.x == 0) out[s_off + r] = (int64_t)(0xFFFFFFFFu - (uint32_t)(best & 0xFFFFFFFFu));
    }
}

}  // namespace vs

using namespace vs;

template <typename V>
static int findmax_launch(const V *val, int32_t H, int32_t W, int32_t stride, int32_t block,
                          int32_t k, int64_t *cand_out, int64_t cap, vs_stream_t st) {
    if (!val || !cand_out) return VS_ERR_ARG;
    if (H < 1 || W < 1 || stride < 1 || block < 1 || k < 1) return VS_ERR_RANGE;
    if ((long long)H * W >= (1ll << 32) - 1) return VS_ERR_RANGE;
    const int64_t need = vs_findmax_count(H, W, stride, block, k);
    if (need < 0) return (int)need;
    if (cap < need) return VS_ERR_RANGE;
    const long long nby = (H + (long long)block - 1) / block, nbx = (W + (long long)block - 1) / block;
    if (nby * nbx > 0x7fffffffll) return VS_ERR_RANGE;
    int rc = check_device();
    if (rc) return rc;
    const int Ws = (W + stride - 1) / stride;
    // 4-post loads need a 4-byte aligned map whose size is a multiple of 4
    // (the last word must not run past the caller's buffer)
    if (sizeof(V) == 1 && stride == 1 && k <= 8 && (((uintptr_t)val) & 3) == 0 &&
        ((long long)H * W) % 4 == 0) {
        if (k <= 4) {
            k_findmax_u8<4><<<(unsigned)(nby * nbx), kFmThreads, 0, (cudaStream_t)st>>>(
                (const uint8_t *)val, H, W, block, k, (int)nbx, nullptr, cand_out);
            vs::note_launch();
        } else {
            k_findmax_u8<8><<<(unsigned)(nby * nbx), kFmThreads, 0, (cudaStream_t)st>>>(
                (const uint8_t *)val, H, W, block, k, (int)nbx, nullptr, cand_out);
            vs::note_launch();
        }
        VS_CUDA_TRY(cudaGetLastError());
        return VS_OK;
    }
    k_findmax<V><<<(unsigned)(nby * nbx), kFmThreads, 0, (cudaStream_t)st>>>(
        val, H, W, stride, Ws, block, k, (int)nbx, cand_out);
    vs::note_launch();
    VS_CUDA_TRY(cudaGetLastError());
    return VS_OK;
}

extern "C" int vs_findmax(const uint8_t *vix, int32_t H, int32_t W, int32_t block, int32_t k,
                          int64_t *cand_out, int64_t cap, vs_stream_t st) {
    return findmax_launch<uint8_t>(vix, H, W, 1, block, k, cand_out, cap, st);
}

extern "C" int vs_findmax_f32(const float *score, int32_t H, int32_t W, int32_t stride,
                              int32_t block, int32_t k, int64_t *cand_out, int64_t cap,
                              vs_stream_t st) {
    return findmax_launch<float>(score, H, W, stride, block, k, cand_out, cap, st);
}

extern "C" int vs_findmax_batch(const vs_findmax_job *jobs, int32_t n_jobs, vs_stream_t st) {
    if (n_jobs < 0 || n_jobs > kFmMaxJobs) return VS_ERR_RANGE;
    if (n_jobs == 0) return VS_OK;
    if (!jobs) return VS_ERR_ARG;
    static FmBatch B;  // built on the host, copied into the launch's parameters
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    memset(&B, 0, sizeof(B));
    long long total = 0;
    int nj = 0;
    for (int i = 0; i < n_jobs; ++i) {
        const vs_findmax_job &q = jobs[i];
        if (!q.vix || !q.cand_out) return VS_ERR_ARG;
        if (q.H < 1 || q.W < 1 || q.block < 1 || q.k < 1) return VS_ERR_RANGE;
        if ((long long)q.H * q.W >= (1ll << 32) - 1) return VS_ERR_RANGE;
        const int64_t need = vs_findmax_count(q.H, q.W, 1, q.block, q.k);
        if (need < 0) return (int)need;
        if (q.cap < need) return VS_ERR_RANGE;
        const long long nby = (q.H + (long long)q.block - 1) / q.block, nbx = (q.W + (long long)q.block - 1) / q.block;
        FmJob &J = B.job[nj++];
        J.val = q.vix; J.H = q.H; J.W = q.W; J.b = q.block; J.k = q.k; J.nbx = (int)nbx; J.out = q.cand_out;
        J.blk0 = total;
        total += nby * nbx;
    }
    if (total > 0x7fffffffll) return VS_ERR_RANGE;
    B.njobs = nj;
    int rc = check_device();
    if (rc) return rc;
    k_findmax_batch<<<(unsigned)total, kFmThreads, 0, (cudaStream_t)st>>>(B);
    vs::note_launch();
    VS_CUDA_TRY(cudaGetLastError());
    return VS_OK;
}
