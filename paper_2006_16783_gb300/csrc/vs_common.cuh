// vs_common.cuh -- shared device/host helpers of libvshed (sm_103a).
//
// TMA staging of int16 terrain windows, bounded mbarrier waits, small integer
// helpers and launch/argument checking used by every kernel file.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/vshed.h"

namespace vs {

// ------------------------------------------------------------------ limits
constexpr int kMaxR = 4096;
constexpr int kMaxH = 100000;
constexpr int kSmemLimit = 227 * 1024;     // opt-in dynamic shared memory per CTA on sm_103
// a bounded mbarrier wait gives up after this many polls (each try_wait
// suspends for a while in hardware; the limit is far above any real latency)
constexpr uint32_t kWaitPolls = 1u << 24;

// ------------------------------------------------------------------ integer helpers
__host__ __device__ __forceinline__ int floordiv(int a, int b) {  // b > 0
    int q = a / b;
    return (q * b > a) ? q - 1 : q;
}
__host__ __device__ __forceinline__ long long floordiv64(long long a, long long b) {
    long long q = a / b;
    return (q * b > a) ? q - 1 : q;
}
__host__ __device__ __forceinline__ int words_per_row(int R) { return (2 * R) / 32 + 2; }

// exact floor(sqrt(v)) for 0 <= v < 2^31
__device__ __forceinline__ int isqrt_exact(int v) {
    int s = (int)sqrtf((float)v);
    while (s > 0 && s * s > v) --s;
    while ((s + 1) * (s + 1) <= v) ++s;
    return s;
}

// ------------------------------------------------------------------ mbarrier + TMA (inline PTX)
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// Wait until the barrier completes the given phase parity.  Returns false if
// the wait gave up after kWaitPolls polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t polls = kWaitPolls) {
    uint32_t addr = smem_u32(bar);
    for (uint32_t i = 0; i < polls; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 3-D tiled TMA load (tensor map of an int16 grid viewed as
// [H][pitch/8][8]): box lands row-major in shared memory.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int c0, int c1,
                                            int c2, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

// ------------------------------------------------------------------ host side
// Window of an int16 grid described for TMA: the grid is viewed as
// [H][pitch/8][8] so that one box of (8, wg, rows) elements fills a
// row-major shared-memory window of 8*wg columns and `rows` rows.
struct GridMap {
    CUtensorMap map;
};

// Build the tensor map; box = 8 x wg x rows (wg <= 256, rows <= 256).
int make_grid_map(GridMap *gm, const vs_grid &g, int wg, int rows);

// launch-shape table filled by vs_tune_set (the autotuner); tune_get returns
// the stored value for (op, R) or `fallback`
int tune_get(int op, int R, int fallback);

// counts the kernel launches the library issues (vs_launch_count)
void note_launch();

// argument checks shared by several entry points
int check_grid(const vs_grid &g);
int check_device();  // current device is sm_103 (cached per device)

#define VS_CUDA_TRY(expr)                       \
    do {                                        \
        cudaError_t e_ = (expr);                \
        if (e_ != cudaSuccess) return VS_ERR_CUDA; \
    } while (0)

}  // namespace vs
