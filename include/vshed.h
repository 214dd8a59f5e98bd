/*
 * vshed.h -- C ABI of the GB300 (sm_103a) observer-siting library libvshed.so.
 *
 * The library implements the data-parallel hot path of the multiple
 * transmitter siting process of Franklin, Magalhaes & Li, "Siting thousands of
 * radio transmitter towers on terrains with billions of points"
 * (arXiv 2006.16783), Sec. "The multiple transmitter siting process":
 *   Vix      -> vs_vix          sampled visibility index of every post
 *   Findmax  -> vs_findmax      per-block top-k candidate transmitters
 *   Viewshed -> vs_viewshed     ray-sweep viewshed bitmap of every candidate
 *   Site     -> vs_site         greedy union of viewsheds
 * plus the learned-proposal and batched entry points that sit beside them.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Terrain: int16 elevations z[y*pitch + x], 0 <= x < W, 0 <= y < H, posts
 *    one unit apart (Sec. "Terrain visibility": z_ij, i = x, j = y).  The
 *    pitch is in elements and must be a multiple of 8 (16 bytes) and >= W;
 *    the base pointer must be 16-byte aligned.  Columns W..pitch-1 are never
 *    interpreted as terrain.
 *  - Post index p = y*W + x (int64 in the API).  H*W must be < 2^32.
 *  - Heights ht (transmitter) and hr (receiver) are integers in the same unit
 *    as z (Sec. "Definitions"); |ht|, |hr| <= 100000.  The ROI R is a
 *    horizontal radius in posts, 1 <= R <= 4096 (Sec. "Definitions": ROI).
 *  - All pointers to arrays are DEVICE pointers unless stated otherwise; the
 *    caller owns every buffer.  No entry point allocates device memory; calls
 *    that need scratch take a caller-provided workspace whose size is given by
 *    the matching *_workspace() query.
 *  - Every call is asynchronous on the given stream (NULL = legacy default
 *    stream) and performs no host-device synchronisation unless stated.
 *  - Return value: VS_OK (0) or a negative VS_ERR_* code.  Argument errors are
 *    detected on the host before anything is launched; nothing is written then.
 *  - Bitmaps are uint32 words; bit b of a word that covers global columns
 *    32*g .. 32*g+31 is column 32*g + b.
 */
#ifndef VSHED_H
#define VSHED_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *vs_stream_t; /* identical to cudaStream_t */

enum {
    VS_OK = 0,
    VS_ERR_ARG = -1,     /* null pointer, negative size, bad alignment / pitch */
    VS_ERR_RANGE = -2,   /* a parameter outside its documented range           */
    VS_ERR_WS = -3,      /* workspace missing or smaller than *_workspace()     */
    VS_ERR_CUDA = -4,    /* a CUDA runtime call or launch failed                */
    VS_ERR_TIMEOUT = -5, /* a bounded device wait gave up (reported on device)  */
    VS_ERR_DEVICE = -6   /* no usable sm_100-family device                      */
};

/* Read-only view of a device-resident terrain. */
typedef struct {
    int32_t H, W;       /* rows, columns (>= 1)                          */
    int64_t pitch;      /* row pitch in elements, multiple of 8, >= W    */
    const int16_t *z;   /* device pointer, 16-byte aligned               */
} vs_grid;

/* Human-readable name of a status code (static string, never NULL). */
const char *vs_strerror(int code);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int vs_version(void);

/* Number of kernel launches the library has issued in this process (counted
 * on the host as each launch is made; replays of a captured CUDA graph launch
 * without passing through the library and are not counted). */
uint64_t vs_launch_count(void);

/* Launch-shape table used by the kernels, filled by an autotuner (the
 * library's Python autotune module times the candidates and stores the
 * fastest).  The results of every call are independent of these settings.
 *   VS_TUNE_VIEWSHED_THREADS: threads per viewshed CTA = rays walked at once
 *     per candidate ("ray bundle"), 128 / 256 / 512 (0 = default: 512, or
 *     fewer when the ring has fewer than 512 rays)
 *   VS_TUNE_VIX_TILE: vix post tile, 1 = 64x32, 2 = 32x32 (0 = default: the
 *     largest tile whose window fits), 3 = the warp-per-line kernel that reads
 *     the terrain in global memory (the path every R takes whose halo window
 *     does not fit in shared memory, R above ~280)
 *   VS_TUNE_SITE_CLUSTER: the greedy site loop of vs_site when every gain
 *     fits in one CTA's shared memory: 0 = default (when bitmap rows are
 *     whole 16-byte vectors, i.e. (2R/32 + 2) % 4 == 0, the multi-winner
 *     leader cluster of 16 CTAs, or of 8 where 16 cannot be scheduled, and
 *     the single-winner one of 8 CTAs where neither fits; else one CTA),
 *     1 = one CTA, 2 / 4 / 8 / 16 = a leader cluster of that
 *     many CTAs (the leader keeps the gains and picks each winner, the window
 *     and refresh loads are split over the cluster's SMs).  R is the call's R.
 *     vs_site_batch always uses one CTA per job.
 *   VS_TUNE_VIEWSHED_WIDE: 1 = vs_viewshed walks the rays in bands of steps
 *     against the terrain in global memory (the path every R takes whose
 *     window does not fit in shared memory, R above ~280) even when the
 *     window would fit; 0 = default.
 *   VS_TUNE_SITE_LAZY: vs_site runs the lazy greedy (the path of calls whose
 *     gains or windows do not fit in one cluster's shared memory) even when
 *     another loop would fit: 1 = on the whole GPU (one cooperative launch,
 *     the lazy path's default), 2 = in one CTA; 0 = default.
 *   VS_TUNE_SITE_MULTI: the leader cluster's rounds of several greedy steps
 *     (the candidates taken in key order while each lies more than 2R from
 *     every other winner of the round; same results as one step at a time):
 *     0 = default (on whenever the leader cluster runs and the gains fit),
 *     1 = off (one step per round).
 *   VS_TUNE_SITE_BARRIER_TEST: a test of the failure path, not a launch
 *     shape: v > 0 (up to 2^20) makes one CTA of the whole-GPU lazy greedy
 *     skip its arrival at the first grid barrier and every barrier wait give
 *     up after v polls, so that the call reports VS_ERR_TIMEOUT in *n_chosen
 *     (the GPU and the next call are unaffected); 0 = off. */
enum {
    VS_TUNE_VIEWSHED_THREADS = 0,
    VS_TUNE_VIX_TILE = 1,
    VS_TUNE_SITE_CLUSTER = 2,
    VS_TUNE_VIEWSHED_WIDE = 3,
    VS_TUNE_SITE_LAZY = 4,
    VS_TUNE_SITE_MULTI = 5,
    VS_TUNE_SITE_BARRIER_TEST = 6
};
int vs_tune_set(int32_t op, int32_t R, int32_t value);
int vs_tune_get(int32_t op, int32_t R);

/* ------------------------------------------------------------------------
 * Vix (Sec. "The multiple transmitter siting process", Vix; LOS as in
 * Sec. "Definitions" and "Terrain visibility").
 *
 * For every post p and sample s < S, the receiver offset is
 *   u   = SplitMix64 output number p*S+s of a generator seeded with seed
 *         (state seed + 0x9E3779B97F4A7C15*(p*S+s+1), then the SplitMix64 mix)
 *   idx = ((u >> 32) * N_R) >> 32
 *   off = OFF_R[idx], OFF_R = {(dx,dy): dx^2+dy^2 <= R^2} minus (0,0), ordered
 *         by dy ascending then dx ascending, N_R = |OFF_R|.
 * The sample counts when the target lies inside the grid and the line of
 * sight from (x, y, z+ht) to (x+dx, y+dy, z'+hr) clears the terrain linearly
 * interpolated between the two posts it passes between, with grazing lines
 * visible.  vix_out[p] (uint8, H*W entries, row-major with pitch W) is the
 * number of counted samples, 0..S.
 *
 * Errors: VS_ERR_ARG (null pointers, pitch), VS_ERR_RANGE (R, S outside
 * 1..4096 / 0..255, heights), VS_ERR_CUDA.
 * ---------------------------------------------------------------------- */
int vs_vix(vs_grid g, int32_t R, int32_t ht, int32_t hr, int32_t S, uint64_t seed,
           uint8_t *vix_out, vs_stream_t st);

/* Large ROIs.  A tile's halo window fits in shared memory up to R ~ 280;
 * beyond that (the paper's runs use R = 500..2000, Sec. "Experiments") a warp
 * walks one line of sight at a time, 32 consecutive crossings per
 * instruction, against the terrain in global memory.  With room for them the
 * call first writes two arrays that hold every post paired with its neighbour
 * along y (row-major) and along x (transposed), so that a crossing reads both
 * of its posts with one contiguous 32-bit load: vs_vix_workspace(H, W, R, S)
 * bytes (0 when the staged kernels cover R, else 8 x H x W plus 512 bytes).
 * vs_vix_ws is vs_vix (los_steps NULL) or vs_vix_count (los_steps set) with
 * that workspace; ws may be NULL or smaller, then lines read the terrain in
 * place (same results, slower).  vs_vix and vs_vix_count are vs_vix_ws
 * without a workspace.  Without it, large R needs (3R + 128) * pitch < 2^31
 * (else VS_ERR_RANGE). */
size_t vs_vix_workspace(int32_t H, int32_t W, int32_t R, int32_t S);
int vs_vix_ws(vs_grid g, int32_t R, int32_t ht, int32_t hr, int32_t S, uint64_t seed,
              uint8_t *vix_out, uint64_t *los_steps, void *ws, size_t ws_bytes, vs_stream_t st);

/* Batched vix: up to 64 terrains (different sizes, ROIs, heights, sample
 * counts, seeds) in ONE persistent launch over (terrain, tile) items; each job
 * is exactly the arguments of one vs_vix call and gets its results.  Each
 * job's halo window must fit in shared memory (R up to ~280; else
 * VS_ERR_RANGE).  jobs is a HOST array read during the call; ws:
 * vs_vix_batch_workspace bytes (a work counter, re-initialised by every call;
 * calls that overlap on the GPU need separate workspaces). */
typedef struct {
    vs_grid g;
    int32_t R, ht, hr, S;
    uint64_t seed;
    uint8_t *vix_out;  /* H x W, device */
} vs_vix_job;
size_t vs_vix_batch_workspace(int32_t n_jobs);
int vs_vix_batch(const vs_vix_job *jobs, int32_t n_jobs, void *ws, size_t ws_bytes, vs_stream_t st);

/* vs_vix plus work accounting: *los_steps (device uint64, accumulated, not
 * cleared) grows by the number of LOS crossings evaluated -- j = 1..D-1 for a
 * visible sample, j = 1..j_block for a blocked one (the test ends at the first
 * crossing above the line).  Output identical to vs_vix. */
int vs_vix_count(vs_grid g, int32_t R, int32_t ht, int32_t hr, int32_t S, uint64_t seed,
                 uint8_t *vix_out, uint64_t *los_steps, vs_stream_t st);

/* ------------------------------------------------------------------------
 * Findmax (Sec. "The multiple transmitter siting process", Findmax).
 *
 * The grid is cut into blocks of block x block posts (edge blocks may be
 * partial).  From every block the k posts with the largest value are kept,
 * ties going to the lower post index.  cand_out receives the post indices
 * ordered by block (row-major over blocks), then by rank; a block with fewer
 * than k posts contributes all of them.
 *
 * vs_findmax_count() returns the number of candidates that a call produces
 * (computed on the host), or a negative error code.  cap is the capacity of
 * cand_out in entries and must be >= that count (else VS_ERR_RANGE).
 *
 * vs_findmax:     vix is uint8 H x W (pitch W), as written by vs_vix.
 * vs_findmax_f32: score is float on a proposal lattice of the given stride:
 *                 score[i*Ws + j] belongs to post (j*stride, i*stride),
 *                 Ws = ceil(W/stride), Hs = ceil(H/stride).  Floats are
 *                 ordered by their IEEE-754 total order.
 * ---------------------------------------------------------------------- */
int64_t vs_findmax_count(int32_t H, int32_t W, int32_t stride, int32_t block, int32_t k);
int vs_findmax(const uint8_t *vix, int32_t H, int32_t W, int32_t block, int32_t k,
               int64_t *cand_out, int64_t cap, vs_stream_t st);
int vs_findmax_f32(const float *score, int32_t H, int32_t W, int32_t stride, int32_t block,
                   int32_t k, int64_t *cand_out, int64_t cap, vs_stream_t st);

/* Batched findmax: up to 64 uint8 maps (one per terrain) in ONE launch, each
 * job exactly the arguments of one vs_findmax call and with its results.  jobs
 * is a HOST array read during the call. */
typedef struct {
    const uint8_t *vix;  /* H x W uint8 map (pitch W), device */
    int32_t H, W, block, k;
    int64_t *cand_out;   /* device, cap entries */
    int64_t cap;
} vs_findmax_job;
int vs_findmax_batch(const vs_findmax_job *jobs, int32_t n_jobs, vs_stream_t st);

/* ------------------------------------------------------------------------
 * Viewshed (Sec. "The multiple transmitter siting process", Viewshed; the
 * bitmap packing of the same paragraph, here in 32-bit words).
 *
 * For each candidate post, rays run from the observer (eye z+ht) to the 8R
 * cells of the square ring max(|dx|,|dy|) = R.  A ray to ring cell (ex,ey)
 * with major axis x when |ex| >= |ey| visits at step k = 1..R the cell
 * (major k, minor round(k*dmin/R)), ties rounded away from zero, and stops
 * when that cell leaves the grid or the disc k^2+minor^2 > R^2.  The cell is
 * visible on the ray when no horizon exists yet or its elevation angle
 * (z+hr-eye)/k is >= the horizon's; then the terrain where the ray crosses
 * the line major = k (linear interpolation between the straddling posts) is
 * offered as the new horizon, and the ray stops when one of those posts lies
 * outside the grid.  A cell's bit is the OR over the rays that visit it; the
 * observer's own cell is always set.  All comparisons are exact integer
 * cross-products.
 *
 * Output layout, per candidate c: bm_out[c*vs_bitmap_words(R) + r*P_R + w],
 * P_R = floor(2R/32)+2 words per row, rows r = 0..2R are global rows
 * cy-R+r, word w covers global columns 32*(floor((cx-R)/32)+w) .. +31.  Bits
 * outside the grid or the disc are 0.  area_out[c] = popcount of the bitmap;
 * a candidate index outside [0, H*W) yields an all-zero bitmap and area -1.
 *
 * Windows that fit in shared memory (R up to ~280 posts) are staged there by
 * TMA.  Larger ROIs -- the paper's own runs use R = 500..2000 (Sec.
 * "Experiments", Tables of the DEM1000 and US-West runs) -- walk the rays in
 * bands of steps against the terrain in global memory, read from two arrays
 * that pair every post with its neighbour along x and along y (one of them
 * transposed), which the call writes into the workspace first.  Both paths
 * give identical bitmaps.
 *
 * ws / ws_bytes: workspace of at least vs_viewshed_workspace(H, W, R, n)
 * bytes: 0 when the window fits in shared memory (ws may then be NULL), else
 * 8 x H x W plus 512 bytes for the pair arrays (17.2 GB at 46400^2).  Too
 * small: VS_ERR_WS.  With a large R, R * (max(H, W) + 1) < 2^31 (else
 * VS_ERR_RANGE).
 * ---------------------------------------------------------------------- */
int64_t vs_bitmap_words(int32_t R); /* (2R+1) * (floor(2R/32)+2) */
size_t vs_viewshed_workspace(int32_t H, int32_t W, int32_t R, int64_t n);
int vs_viewshed(vs_grid g, int32_t R, int32_t ht, int32_t hr, const int64_t *cand, int64_t n,
                uint32_t *bm_out, int32_t *area_out, void *ws, size_t ws_bytes, vs_stream_t st);

/* Exact per-cell viewshed (the "R3" of the siting literature): every cell
 * of disc(R) inside the grid gets its own line of sight from the observer,
 * tested exactly as a vix sample (Sec. "Terrain visibility": the LOS against
 * the terrain interpolated between the two posts it passes between, grazing
 * lines visible, receiver at z + hr) -- the viewshed of Sec. "Definitions"
 * read literally, against which vs_viewshed's ray sweep (R2-style) is an
 * approximation.  Same arguments, output layout and errors as vs_viewshed.
 * Costs ~0.6*pi*R^3 crossings per candidate (vs_viewshed: ~7R^2 steps): an
 * accuracy reference, not the siting path.  ws: optional, at least
 * vs_viewshed_r3_workspace(H, W) bytes for the pair arrays of vs_vix_ws;
 * NULL or smaller: the terrain is read in place, same results.  Without them
 * it needs (3R + 128) * pitch < 2^31. */
size_t vs_viewshed_r3_workspace(int32_t H, int32_t W);
int vs_viewshed_r3(vs_grid g, int32_t R, int32_t ht, int32_t hr, const int64_t *cand, int64_t n,
                   uint32_t *bm_out, int32_t *area_out, void *ws, size_t ws_bytes, vs_stream_t st);

/* Exact visibility index of each listed post (Sec. "Definitions": the
 * visibility index of a transmitter is the fraction of the receivers within
 * its ROI that it sees; here the label the learned proposal is trained on):
 *   out[i] = area of the post's vs_viewshed bitmap
 *            / |{(dx,dy): dx^2+dy^2 <= R^2, post + (dx,dy) inside the grid}|,
 * the quotient of the two integers rounded once to float (round to nearest
 * even).  posts[n]: int64 post indices (device); out[n]: float (device).  A
 * post outside the grid gives -1; a timed-out device wait gives
 * VS_ERR_TIMEOUT (as a float).  No bitmap is returned.  ws: at least
 * vs_exact_vix_workspace(H, W, R, n) bytes (4 bytes per post, plus for ROIs
 * beyond shared memory the pair arrays of vs_viewshed and a bitmap buffer of
 * at most 1 GiB through which the posts are processed in chunks).  Errors as
 * vs_viewshed. */
size_t vs_exact_vix_workspace(int32_t H, int32_t W, int32_t R, int64_t n);
int vs_exact_vix(vs_grid g, int32_t R, int32_t ht, int32_t hr, const int64_t *posts, int64_t n,
                 float *out, void *ws, size_t ws_bytes, vs_stream_t st);

/* Batched viewsheds: the candidates of up to 64 terrains (different sizes,
 * ROIs, heights) in ONE persistent launch.  jobs is a HOST array read during
 * the call; each job is exactly the arguments of one vs_viewshed call, and
 * the results are identical to those calls.  ws: vs_viewshed_batch_workspace
 * bytes (a work counter, re-initialised by every call; calls that overlap on
 * the GPU need separate workspaces). */
typedef struct {
    vs_grid g;
    int32_t R, ht, hr;
    const int64_t *cand;
    int64_t n;
    uint32_t *bm_out;
    int32_t *area_out;
} vs_viewshed_job;
size_t vs_viewshed_batch_workspace(int32_t n_jobs);
int vs_viewshed_batch(const vs_viewshed_job *jobs, int32_t n_jobs, void *ws, size_t ws_bytes,
                      vs_stream_t st);

/* ------------------------------------------------------------------------
 * Site (Sec. "The multiple transmitter siting process", Site).
 *
 * Greedy: starting from the cumulative viewshed held in cum (uint32
 * H x ceil(W/32), same bit convention; all zero for a fresh run), each step
 * picks the candidate with the largest gain popcount(V_c AND NOT cum), ties to
 * the lowest post index, appends its post index to chosen[] and its gain to
 * gains[], and ORs V_c into cum.  It stops after n_obs observers, when the
 * best gain is 0, or -- when coverage_target > 0 -- as soon as
 * popcount(cum) >= ceil(coverage_target * H * W) before a step.
 * *n_chosen (device int32) receives the number chosen, or a negative VS_ERR_*
 * code when the device reports a failure (VS_ERR_TIMEOUT: a bounded wait of
 * the lazy greedy's grid barrier, or of the leader cluster's band compaction
 * for the next winner, gave up; chosen[] and cum are then incomplete).  Calling again with the returned cum continues the same greedy
 * sequence (checkpoint / resume).
 *
 * bm, cand, n, R describe the candidates exactly as vs_viewshed wrote them.
 * chosen and gains have room for n_obs int64 entries.  Requires W, H <= 65535.
 * ws / ws_bytes: workspace of at least vs_site_workspace(n, R) bytes.
 * ---------------------------------------------------------------------- */
size_t vs_site_workspace(int64_t n, int32_t R);
int vs_site(const uint32_t *bm, const int64_t *cand, int64_t n, int32_t H, int32_t W, int32_t R,
            int32_t n_obs, double coverage_target, int64_t *chosen, int64_t *gains,
            uint32_t *cum, int32_t *n_chosen, void *ws, size_t ws_bytes, vs_stream_t st);

/* Site with the constraints the paper names as extensions (Sec. "Prior
 * art": receivers of a given quality; intervisibility, where transmitters
 * must be visible from other transmitters).  Readings:
 *   - intervisibility (terrain.z != NULL): the first transmitter of the call
 *     is free; every later one must be intervisible with one chosen earlier
 *     in the call: the posts within the ROI (dx^2 + dy^2 <= R^2) and the line
 *     between the antenna tops, both at z + ht, clearing the terrain by the
 *     vix line-of-sight test (symmetric in the two ends).  terrain is the grid
 *     the bitmaps were computed on (same H, W);
 *   - weighted receivers (weight != NULL): post (x, y) weighs weight[y*W + x]
 *     (uint8, pitch W); gains[] are the weights of the newly covered posts and
 *     the coverage stop compares covered weight with
 *     ceil(coverage_target * total weight).  Needs (2R+1)^2 * 255 < 2^32.
 * Ties as in vs_site.  opt == NULL or neither option set: exactly vs_site.
 * Otherwise the lazy greedy on the whole GPU runs (one cooperative launch;
 * VS_ERR_DEVICE without cooperative launch support).  ws: at least
 * vs_site_ex_workspace(n, R) bytes. */
typedef struct {
    vs_grid terrain;       /* z == NULL: no intervisibility constraint */
    int32_t ht;            /* antenna height above the post, both ends */
    const uint8_t *weight; /* H x W receiver weights, NULL = 1 each     */
} vs_site_options;
size_t vs_site_ex_workspace(int64_t n, int32_t R);
int vs_site_ex(const uint32_t *bm, const int64_t *cand, int64_t n, int32_t H, int32_t W, int32_t R,
               int32_t n_obs, double coverage_target, const vs_site_options *opt, int64_t *chosen,
               int64_t *gains, uint32_t *cum, int32_t *n_chosen, void *ws, size_t ws_bytes, vs_stream_t st);

/* vs_site for callers that cannot allocate device memory.  The paper has no
 * counterpart; this is a convenience of the library.
 *
 * Some callers can neither call cudaMalloc nor hand over a workspace: code
 * running inside a host application that owns every device allocation
 * through its own pool and forbids allocation calls from plug-ins, latency-
 * critical loops that cannot afford the implicit device synchronisation of
 * cudaMalloc/cudaFree, and bindings from languages that have no device
 * allocator at all.  This entry point needs nothing from them beyond the
 * inputs and outputs of vs_site: its scratch is a static device array of
 * VS_SITE_NOALLOC_MAX_BYTES inside libvshed.so, reserved on every GPU that
 * loads the library until the process exits.
 *
 *  - Same arguments, results and errors as vs_site, minus the workspace.
 *  - Limit: vs_site_workspace(n, R) must not exceed VS_SITE_NOALLOC_MAX_BYTES
 *    (1 MiB, i.e. up to 37,439 candidates, for any R); larger calls return
 *    VS_ERR_RANGE and launch nothing.
 *  - The first call on each device looks up the array's device address (a
 *    runtime query, with that device current); make that first call before
 *    any stream capture.  The address belongs to the device's current CUDA
 *    context: a call made after that context changed (e.g. after the caller's
 *    cudaDeviceReset) looks it up again, so it too should come before any
 *    stream capture.
 *  - Every call on a device shares the one array and leaves its contents
 *    behind; the call re-initialises everything it reads.  Calls whose work
 *    overlaps on the GPU (other streams, other host threads) race on the
 *    array: serialise them.
 *  - It calls no cudaMalloc, cudaFree or allocating library routine. */
#define VS_SITE_NOALLOC_MAX_BYTES (1u << 20)
int vs_site_noalloc(const uint32_t *bm, const int64_t *cand, int64_t n, int32_t H, int32_t W,
                    int32_t R, int32_t n_obs, double coverage_target, int64_t *chosen,
                    int64_t *gains, uint32_t *cum, int32_t *n_chosen, vs_stream_t st);

/* Site with the candidates split over several ranks (the paper's parallel
 * Site loop over candidates, divided between processes, one GPU each; Sec.
 * "The multiple transmitter siting process", Site).  Each rank holds its own
 * candidates (bm, cand, n as vs_viewshed wrote them), their exact gains
 * (device uint32 [n], initialised with vs_site_gains) and a full copy of the
 * cumulative viewshed cum.  One greedy step on one rank:
 *   - win_post >= 0: the step's winner, whose bitmap win_bm (device,
 *     vs_bitmap_words(R) words, vs_viewshed's layout) every rank received
 *     from the rank that owns it, is ORed into cum, and every local candidate
 *     whose window meets the winner's loses popcount(V_c AND delta), delta =
 *     win_bm AND NOT cum before the update; win_local is the winner's index
 *     among this rank's candidates (its gain becomes 0), -1 on other ranks.
 *     win_post < 0: no winner yet (the first step).
 *   - *best_key (device uint64) = the largest (gain << 32) | (0xFFFFFFFF -
 *     post) over this rank's candidates, 0 when every gain is 0.
 * The caller takes the largest key over the ranks (an all-reduce of one
 * 8-byte value); its rank finds the lowest index holding it and broadcasts
 * that bitmap.  The sequence of winners is the single-rank greedy's (posts are
 * unique across ranks).  ws: vs_site_shard_workspace(R) bytes.  Requires
 * W, H <= 65535. */
size_t vs_site_shard_workspace(int32_t R);
int vs_site_shard_step(const uint32_t *bm, const int64_t *cand, int64_t n, int32_t H, int32_t W, int32_t R,
                       uint32_t *gains, uint32_t *cum, const uint32_t *win_bm, int64_t win_post,
                       int64_t win_local, uint64_t *best_key, void *ws, size_t ws_bytes, vs_stream_t st);

/* Batched site: up to 64 independent greedy problems (one per terrain), each
 * exactly the arguments of one vs_site call minus the workspace, with the
 * same results.  The greedy loops of every job small enough for one CTA's
 * shared memory run in ONE launch (one CTA per job); other jobs run as
 * ordinary vs_site calls.  jobs is a HOST array read during the call; ws:
 * vs_site_batch_workspace(jobs, n_jobs) bytes, 256-byte aligned. */
typedef struct {
    const uint32_t *bm;
    const int64_t *cand;
    int64_t n;
    int32_t H, W, R, n_obs;
    double coverage_target;
    int64_t *chosen, *gains;
    uint32_t *cum;
    int32_t *n_chosen;
} vs_site_job;
size_t vs_site_batch_workspace(const vs_site_job *jobs, int32_t n_jobs);
int vs_site_batch(const vs_site_job *jobs, int32_t n_jobs, void *ws, size_t ws_bytes, vs_stream_t st);

/* Dense gain pass (the first step of vs_site, exposed on its own): for every
 * candidate c, gains_out[c] = popcount(V_c AND NOT cum).  One streaming pass
 * over all n bitmaps. */
int vs_site_gains(const uint32_t *bm, const int64_t *cand, int64_t n, int32_t H, int32_t W,
                  int32_t R, const uint32_t *cum, uint32_t *gains_out, vs_stream_t st);

/* ------------------------------------------------------------------------
 * Learned candidate proposal (replaces the sampled ranking of the Vix stage,
 * Sec. "The multiple transmitter siting process", Vix, whose only use is to
 * rank posts; the network itself is this library's, the paper has none).
 *
 * Network: x0 = bf16((z - mean over the 65x65 patch) / 1000); four 3x3
 * stride-2 convolutions and one 3x3 stride-1 convolution, 32 channels, bias +
 * ReLU, activations rounded to bf16; global average pool; fc 32 -> 1;
 * sigmoid.  Patches are centred on a post; element (r, c), r, c = 0..64, is
 * the post (cy + (r-32)*patch_step, cx + (c-32)*patch_step) (patch_step 1..64:
 * step 3 lets the 65x65 input span an R = 100 ROI); rows/columns outside
 * the grid are clamped to the nearest edge post.  Products are BF16 x BF16 on
 * the tensor cores (tcgen05), accumulated in FP32.
 *
 * Parameters: vs_cnn_param_count() fp32 values ("master" weights, device):
 *   w_l [32][cin][3][3] then b_l [32] for l = 0..4 (cin = 1 for l = 0, else
 *   32), then fc weights [32] and fc bias [1].
 * vs_cnn_pack converts them into the kernels' operand layout (a device
 * buffer of vs_cnn_packed_bytes(), 16-byte aligned); repack after every
 * weight update.
 *
 * vs_cnn_forward: n patches centred on posts centers[n] (int64 post indices
 * in [0, H*W)); out[n] = predicted visibility index (fp32).  Both entry
 * points need H*W < 2^32 (else VS_ERR_RANGE).  save (optional, device, n *
 * vs_cnn_save_bytes() bytes, 16-byte aligned) receives every activation for
 * vs_cnn_backward.  status (optional, device int32) is set to VS_ERR_TIMEOUT
 * if a bounded tensor-core wait gave up.
 * vs_cnn_score_lattice: one patch per lattice post (i*stride, j*stride),
 * score_out [ceil(H/stride)][ceil(W/stride)], the input of vs_findmax_f32.
 * ---------------------------------------------------------------------- */
int vs_cnn_param_count(void);
size_t vs_cnn_packed_bytes(void);
size_t vs_cnn_save_bytes(void);
int vs_cnn_pack(const float *master, void *packed, vs_stream_t st);
int vs_cnn_forward(vs_grid g, const int64_t *centers, int64_t n, int32_t patch_step,
                   const void *packed, float *out, void *save, int32_t *status, vs_stream_t st);
int vs_cnn_score_lattice(vs_grid g, int32_t stride, int32_t patch_step, const void *packed,
                         float *score_out, int32_t *status, vs_stream_t st);
/* Lattice rows row0 .. row0+nrows-1 only (0 <= row0, row0 + nrows <= ceil(H/stride)):
 * score_out [nrows][ceil(W/stride)] receives exactly the rows vs_cnn_score_lattice
 * writes there.  A patch of lattice row i reads terrain rows within 32*patch_step of
 * i*stride, so a caller streaming the terrain in by row chunks can score the rows
 * whose posts have arrived. */
int vs_cnn_score_lattice_rows(vs_grid g, int32_t stride, int32_t patch_step, int32_t row0,
                              int32_t nrows, const void *packed, float *score_out,
                              int32_t *status, vs_stream_t st);

/* Training.  vs_cnn_backward: gradients of the mean L1 loss
 * mean_b |y_b - labels[b]| over a batch of B patches whose forward pass
 * (vs_cnn_forward with `save`) wrote `save`; master must be the weights that
 * forward used.  grads (fp32, vs_cnn_param_count() values, same layout as
 * master) is ACCUMULATED; *loss_sum (device fp32) grows by the sum of
 * |y - label|.  Pre-activation gradients are rounded to bf16 before they meet
 * weights or activations; products accumulate in FP32.  ws: at least
 * vs_cnn_backward_workspace(B) bytes.
 * vs_cnn_adam: one Adam step (Kingma & Ba 2015) on master with moments m, v
 * (fp32, zero before step 1); step counts from 1; grads are cleared. */
size_t vs_cnn_backward_workspace(int64_t B);
int vs_cnn_backward(const void *save, const float *labels, int64_t B, const float *master,
                    float *grads, float *loss_sum, void *ws, size_t ws_bytes, vs_stream_t st);
int vs_cnn_adam(float *master, float *grads, float *m, float *v, int64_t step, float lr,
                float beta1, float beta2, float eps, vs_stream_t st);

/* Self-test of the failure path (no counterpart in the paper): a kernel
 * waits on a barrier that nothing completes, gives up after `polls` polls
 * (1 .. 2^24) and writes VS_ERR_TIMEOUT to *status (device int32); the
 * context stays usable.  Every TMA and tensor-core completion in the
 * library is guarded by the same bounded wait. */
int vs_selftest_wait_timeout(int32_t *status, uint32_t polls, vs_stream_t st);

#ifdef __cplusplus
}
#endif
#endif /* VSHED_H */
