// vs_api.cu -- host-side helpers of the C ABI: error strings, argument
// checks, the TMA tensor-map builder and the size queries.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <string.h>

#include "vs_common.cuh"

namespace vs {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

int make_grid_map(GridMap *gm, const vs_grid &g, int wg, int rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return VS_ERR_CUDA;
    if (wg < 1 || wg > 256 || rows < 1 || rows > 256) return VS_ERR_RANGE;
    cuuint64_t dims[3] = {8, (cuuint64_t)(g.pitch / 8), (cuuint64_t)g.H};
    cuuint64_t strides[2] = {16, (cuuint64_t)g.pitch * 2};
    cuuint32_t box[3] = {8, (cuuint32_t)wg, (cuuint32_t)rows};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(&gm->map, CU_TENSOR_MAP_DATA_TYPE_UINT16 /* bit copy of int16 */, 3, (void *)g.z, dims, strides, box,
                    estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? VS_OK : VS_ERR_CUDA;
}

// (op, R) -> value; R <= kMaxR, ops 0..6
constexpr int kTuneOps = 7;
static int g_tune[kTuneOps][kMaxR + 1];
static std::mutex g_tune_mu;

int tune_get(int op, int R, int fallback) {
    if (op < 0 || op >= kTuneOps || R < 1 || R > kMaxR) return fallback;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const int v = g_tune[op][R];
    return v > 0 ? v : fallback;
}

static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1ull, std::memory_order_relaxed); }

int check_grid(const vs_grid &g) {
    if (!g.z) return VS_ERR_ARG;
    if (g.H < 1 || g.W < 1 || g.H > kMaxH || g.W > kMaxH) return VS_ERR_RANGE;
    if ((long long)g.H * g.W >= (1ll << 32) - 1) return VS_ERR_RANGE;
    if (g.pitch < g.W || (g.pitch % 8) != 0) return VS_ERR_ARG;
    if (((uintptr_t)g.z & 15) != 0) return VS_ERR_ARG;
    return VS_OK;
}

int check_device() {
    static int ok_dev[64];  // 0 unknown, 1 ok, -1 bad
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return VS_ERR_DEVICE;
    if (dev < 0 || dev >= 64) return VS_ERR_DEVICE;
    if (ok_dev[dev] == 0) {
        int major = 0, minor = 0;
        if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess)
            return VS_ERR_DEVICE;
        ok_dev[dev] = (major == 10 && minor == 3) ? 1 : -1;
    }
    return ok_dev[dev] == 1 ? VS_OK : VS_ERR_DEVICE;
}

}  // namespace vs

extern "C" {

const char *vs_strerror(int code) {
    switch (code) {
        case VS_OK: return "ok";
        case VS_ERR_ARG: return "invalid argument (null pointer, size, alignment or pitch)";
        case VS_ERR_RANGE: return "parameter outside its supported range";
        case VS_ERR_WS: return "workspace missing or too small";
        case VS_ERR_CUDA: return "CUDA runtime error";
        case VS_ERR_TIMEOUT: return "bounded device wait timed out";
        case VS_ERR_DEVICE: return "no usable sm_103 device";
        default: return "unknown status";
    }
}

int vs_version(void) { return 100; }

uint64_t vs_launch_count(void) { return (uint64_t)vs::g_launches.load(std::memory_order_relaxed); }

int vs_tune_set(int32_t op, int32_t R, int32_t value) {
    if (op < 0 || op >= vs::kTuneOps || R < 1 || R > vs::kMaxR) return VS_ERR_RANGE;
    if (op == VS_TUNE_VIEWSHED_THREADS && value != 0 && value != 128 && value != 256 && value != 512)
        return VS_ERR_RANGE;
    if (op == VS_TUNE_VIX_TILE && (value < 0 || value > 3)) return VS_ERR_RANGE;
    if (op == VS_TUNE_SITE_CLUSTER && value != 0 && value != 1 && value != 2 && value != 4 && value != 8 &&
        value != 16)
        return VS_ERR_RANGE;
    if (op == VS_TUNE_VIEWSHED_WIDE && value != 0 && value != 1) return VS_ERR_RANGE;
    if (op == VS_TUNE_SITE_LAZY && (value < 0 || value > 2)) return VS_ERR_RANGE;
    if (op == VS_TUNE_SITE_MULTI && value != 0 && value != 1) return VS_ERR_RANGE;
    if (op == VS_TUNE_SITE_BARRIER_TEST && (value < 0 || value > (1 << 20))) return VS_ERR_RANGE;
    std::lock_guard<std::mutex> lk(vs::g_tune_mu);
    vs::g_tune[op][R] = value;
    return VS_OK;
}

int vs_tune_get(int32_t op, int32_t R) { return vs::tune_get(op, R, 0); }

int64_t vs_bitmap_words(int32_t R) {
    if (R < 1 || R > vs::kMaxR) return VS_ERR_RANGE;
    return (int64_t)(2 * R + 1) * vs::words_per_row(R);
}

// number of lattice points i >= 0 with lo <= i*stride < hi
static inline int64_t lattice_count(int64_t lo, int64_t hi, int64_t stride) {
    if (hi <= lo) return 0;
    int64_t a = (lo + stride - 1) / stride, b = (hi + stride - 1) / stride;
    return b - a;
}

int64_t vs_findmax_count(int32_t H, int32_t W, int32_t stride, int32_t block, int32_t k) {
    if (H < 1 || W < 1 || stride < 1 || block < 1 || k < 1) return VS_ERR_RANGE;
    int64_t nby = (H + (int64_t)block - 1) / block, nbx = (W + (int64_t)block - 1) / block;
    int64_t total = 0;
    for (int64_t by = 0; by < nby; ++by) {
        int64_t ny = lattice_count(by * block, std::min<int64_t>(H, (by + 1) * block), stride);
        for (int64_t bx = 0; bx < nbx; ++bx) {
            int64_t nx = lattice_count(bx * block, std::min<int64_t>(W, (bx + 1) * block), stride);
            total += std::min<int64_t>(k, ny * nx);
        }
    }
    return total;
}

}  // extern "C"

// ------------------------------------------------------------------ bounded-wait self-test
// A barrier that expects one arrival nobody makes: the bounded wait gives up
// and the kernel reports VS_ERR_TIMEOUT through `status`, leaving the
// context usable.  The same wait routine guards every TMA and tensor-core
// completion in the library.
__global__ void k_selftest_wait(int32_t *status, uint32_t polls) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) vs::mbar_init(&bar, 1);
    __syncthreads();
    const bool ok = vs::mbar_wait(&bar, 0, polls);
    if (threadIdx.x == 0) *status = ok ? VS_OK : VS_ERR_TIMEOUT;
}

extern "C" int vs_selftest_wait_timeout(int32_t *status, uint32_t polls, vs_stream_t st) {
    if (!status || polls == 0 || polls > (1u << 24)) return VS_ERR_ARG;
    int rc = vs::check_device();
    if (rc) return rc;
    k_selftest_wait<<<1, 32, 0, (cudaStream_t)st>>>(status, polls);
    vs::note_launch();
    VS_CUDA_TRY(cudaGetLastError());
    return VS_OK;
}
