/*
 * apsp.h -- C ABI of the GB300 blocked Floyd-Warshall library (libapsp.so).
 *
 * The method is the blocked all-pairs shortest-paths algorithm studied in
 * Rucci, De Giusti, Naiouf, "Blocked All-Pairs Shortest Paths Algorithm on
 * Intel Xeon Phi KNL Processor: A Case Study" (arXiv 1811.01201):
 *   - problem statement (Section 3): input an N x N distance matrix D with
 *     D[i][j] the weight of edge i -> j; output D[i][j] = shortest distance and
 *     P[i][j] = the most recently added intermediate vertex, for path
 *     reconstruction;
 *   - blocking (Section 4.1, Fig. 2-3): D split into BS x BS blocks, R = N/BS
 *     rounds, each round updating the diagonal block, then the blocks of its
 *     row and column, then all remaining blocks;
 *   - relaxation (Section 4.2): one addition and one comparison per update,
 *     here a strict '<', so ties keep the earlier intermediate.
 *
 * Conventions shared by every call:
 *   - Matrices are dense, row-major, n x n, leading dimension n, 4-byte
 *     elements: weights/distances are IEEE fp32, path entries int32.
 *   - Absent edges are +INFINITY. Weights must be >= 0 (or +INF) and not NaN;
 *     W[i][i] is ignored (the diagonal of D is forced to 0).
 *   - P[i][j] = -1 means "direct edge, i == j, or unreachable"; otherwise it is
 *     the global index of the intermediate vertex recorded by the last strict
 *     improvement of D[i][j]. The path is path(i,P[i][j]) ++ path(P[i][j],j).
 *   - Device pointers are CUDA global-memory pointers owned by the caller;
 *     `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Work is enqueued on `stream`; the call returns once it is
 *     enqueued, except where a call says it synchronises.
 *   - No call aborts the process. Every call returns an apsp_status; a sticky
 *     CUDA error is reported as APSP_ECUDA.
 *   - Results are deterministic: for the same W, n and block size they are
 *     bit-identical from run to run and between the single-graph, batched and
 *     served entry points.
 */
#ifndef APSP_H
#define APSP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  APSP_OK = 0,
  APSP_EINVAL = -1,     /* bad argument: n < 1, NULL pointer, negative or NaN weight, unsupported option */
  APSP_ENOMEM = -2,     /* device/host allocation failed, workspace too small, or over the HBM budget */
  APSP_ECUDA = -3,      /* a CUDA runtime call or kernel launch failed */
  APSP_ETIMEOUT = -4,   /* a bounded wait ran out (poll timeout, device-side spin limit) */
  APSP_EBUSY = -5,      /* resource busy: no free slot, or the result is not ready yet */
  APSP_ECANCELLED = -6, /* the job was cancelled or the server is shutting down */
  APSP_ENOTFOUND = -7   /* unknown job id */
} apsp_status;

/* Arithmetic used for the distance matrix. */
enum {
  APSP_DTYPE_AUTO = 0,  /* U16X2 when eligible (see below), else F32 */
  APSP_DTYPE_F32 = 1,   /* fp32 distances */
  APSP_DTYPE_U16X2 = 2  /* exact packed 16-bit distances, two per 32-bit lane, saturating at 65535 = INF */
};

/*
 * Per-call options. Zero-initialise and set what you need.
 *   bs:       block size BS (Section 4.1). 0 = the library default: on the
 *             fp32 path apsp_default_bs(n), on the 16-bit path 128 for
 *             n > 16384 and apsp_default_bs(n) otherwise (apsp_run_info.bs_used
 *             reports it); else 32, 64 or 128.
 *   dtype:    APSP_DTYPE_*. U16X2 is eligible only when every finite weight is
 *             an integer and either max_w * (n - 1) < 65535, so that every
 *             path length fits in 16 bits, or every off-diagonal edge is
 *             present and max_w < 65535 (then no distance ever exceeds its
 *             direct edge); it gives bit-identical D and P to F32.
 *             Requesting U16X2 for an ineligible W returns APSP_EINVAL.
 *   validate: 1 = scan W on the device for negative / NaN weights (and, for
 *             AUTO/U16X2, eligibility) before running; the call then
 *             synchronises `stream` once. 0 = trust the caller (F32 only;
 *             fully asynchronous, usable inside CUDA-graph capture).
 */
typedef struct {
  int bs;
  int dtype;
  int validate;
  int flags;       /* APSP_FLAG_* bits */
} apsp_options;

/* APSP_FLAG_TIME_PHASES: record CUDA events around every phase launch and
 * report the summed device time per phase in apsp_run_info.phase_ms; the call
 * then synchronises `stream` before returning. */
#define APSP_FLAG_TIME_PHASES 1

/* APSP_FLAG_TEST_PANEL_TIMEOUT: testing only. Every fp32 phase-3 CTA waits,
 * with a bound, for the two panel slices it requests by bulk copy; with this
 * flag it announces the slices but never copies them, so the wait expires
 * after 20 ms per CTA wave, the CTA leaves its tile untouched and sets the
 * device fault word that apsp_device_status reports. The results of such a
 * call are wrong by design; nothing faults or hangs. */
#define APSP_FLAG_TEST_PANEL_TIMEOUT 0x40000000

/* What a call actually did (optional output). */
typedef struct {
  int bs_used;       /* block size of the run; the oracle must use the same BS to match P bit-exactly */
  int dtype_used;    /* APSP_DTYPE_F32 or APSP_DTYPE_U16X2 */
  int rounds;        /* number of block rounds R = n_pad / BS */
  int n_pad;         /* working order: n rounded up to a multiple of 128 */
  int launches;      /* kernels this call launched */
  int phase_launches[3];
  float phase_ms[3]; /* with APSP_FLAG_TIME_PHASES: device ms in phases 1, 2, 3 (else 0) */
} apsp_run_info;

/*
 * Device fault word of the single-graph solver on the current device: a
 * phase-3 CTA whose bounded wait for its panel slices expired (2 s; a slice
 * normally arrives within microseconds) sets it and leaves its tile, so the
 * solve that ran it is wrong. Returns APSP_ETIMEOUT if it is set, else APSP_OK;
 * clear != 0 resets it. Reflects work that has finished: synchronise the
 * streams first. apsp_fw_host checks and clears it itself (APSP_ETIMEOUT).
 */
apsp_status apsp_device_status(int clear);

/* Library default block size of the fp32 path for order n (deterministic in n). */
int apsp_default_bs(int n);

/*
 * Block-size autotuner. The paper tuned BS by hand for its machine (Section
 * 5.2: 256 serial, 64 with 68 threads); this measures it on the current GPU:
 * a synthetic dense integer-weight graph of order n is solved once per
 * candidate BS in {32, 64, 128} after a warm-up, and *best_bs receives the
 * fastest. ms_out (optional, 3 floats) receives the timed solve of each
 * candidate. Allocates its graph with the stream-ordered allocator and
 * synchronises `stream`. The choice is advisory: pass it as apsp_options.bs.
 */
apsp_status apsp_autotune_bs(int n, int* best_bs, float* ms_out, void* stream);

/* Human-readable name of a status code (static string). */
const char* apsp_status_str(apsp_status s);

/*
 * Bytes of device workspace apsp_fw_ex needs for (n, opt): always at least
 * 256 (the input scan's counters) plus the round's packed panel slices
 * (ceil(n/128) * bs * 1072 bytes on the fp32 path, * 800 on the 16-bit path;
 * bs = opt->bs, or apsp_default_bs(n) when it is 0) and the packed diagonal
 * block (8 * bs * (bs + 4) bytes); n*n-sized working
 * matrices are added when n is not a multiple of 128 or the 16-bit path may
 * be chosen. Returns 0 on invalid arguments (apsp_fw_ex reports them).
 * The figure assumes that D and P start on 16-byte boundaries, as every
 * cudaMalloc and PyTorch allocation does: the solve runs in place in the
 * caller's D and P only then. apsp_fw_workspace_size_for gives the need for
 * the actual D and P (a misaligned one adds its padded working copy,
 * 4 * n_pad^2 bytes). apsp_fw_ex checks a caller workspace against that
 * need before it enqueues anything and returns APSP_ENOMEM if it is short.
 */
size_t apsp_fw_workspace_size(int n, const apsp_options* opt);
size_t apsp_fw_workspace_size_for(int n, const apsp_options* opt, const float* D, const int32_t* P);

/*
 * All-pairs shortest paths of one graph (Section 3; blocked per Section 4.1).
 *   W: device, n*n fp32 weights (may alias D: in-place run).
 *   D: device, n*n fp32 output distances.
 *   P: device, n*n int32 output path matrix.
 * Uses default options (bs = apsp_default_bs(n), dtype AUTO, validate 1), so
 * it synchronises `stream` once after the validation scan. Any workspace is
 * taken from the stream-ordered allocator and returned before the call ends.
 */
apsp_status apsp_fw(const float* W, float* D, int32_t* P, int n, void* stream);

/*
 * As apsp_fw with explicit options and caller-provided workspace.
 *   opt: NULL = defaults.
 *   workspace / workspace_bytes: device buffer of at least
 *     apsp_fw_workspace_size(n, opt) bytes, 256-byte aligned, or NULL/0 to let
 *     the library allocate with cudaMallocAsync on `stream`.
 *   info: optional output (may be NULL).
 */
apsp_status apsp_fw_ex(const float* W, float* D, int32_t* P, int n, const apsp_options* opt, void* workspace,
                       size_t workspace_bytes, apsp_run_info* info, void* stream);

/*
 * End-to-end call on HOST buffers: copies W (host, n*n fp32) to the device,
 * runs apsp_fw_ex, copies D and P back to host memory, and synchronises
 * `stream` before returning. W, D, P are host pointers (page-locked memory
 * gives the fastest copies). Device memory is allocated and freed inside:
 * 8*n*n bytes (W is copied into the device D and solved in place) plus the
 * workspace apsp_fw_ex would allocate; APSP_ENOMEM if that fails.
 */
apsp_status apsp_fw_host(const float* W, float* D, int32_t* P, int n, const apsp_options* opt,
                         apsp_run_info* info, void* stream);

/*
 * Many independent graphs in one persistent launch. One CTA runs the whole
 * blocked Floyd-Warshall (Section 4.1) of one graph at a time and then takes
 * the next graph from a device work queue (largest first), so thousands of
 * uneven graphs share the GPU without a launch per graph or per round.
 *   W, D, P: HOST arrays of `count` DEVICE pointers; graph g has order n[g]
 *            (host array), 1 <= n[g] <= APSP_BATCH_MAX_N, row-major with
 *            leading dimension n[g]. W[g] may alias D[g].
 *   opt:     NULL or bs 0/32 (the batched block size is 32), dtype AUTO/F32
 *            (computes in fp32), validate 0/1 (1: scan every W for negative
 *            or NaN weights first).
 *   bs_used: optional HOST array of `count` ints receiving each graph's BS.
 * Synchronises `stream` before returning. Results equal apsp_fw_ex with
 * bs = bs_used[g] (and dtype F32), bit for bit.
 */
#define APSP_BATCH_MAX_N 512
apsp_status apsp_fw_batched(const float* const* W, float* const* D, int32_t* const* P, const int* n, int count,
                            const apsp_options* opt, int* bs_used, void* stream);

/* Block size the batched kernel uses for a graph of order n (32). */
int apsp_batched_bs(int n);

/*
 * Reusable batch for repeated or graph-captured launches.
 * apsp_batch_create validates the arguments as apsp_fw_batched does, uploads
 * the descriptor table to device memory it owns, and synchronises `stream`.
 * apsp_batch_launch enqueues the whole batch on `stream` as one queue reset
 * (a memset) plus ONE persistent kernel launch; it allocates nothing and does
 * not synchronise, so it may be captured into a CUDA graph and replayed. The
 * W/D/P buffers named at creation must stay valid while launches run.
 * apsp_batch_destroy frees the table (after the caller's last launch ended).
 */
typedef struct apsp_batch apsp_batch;
apsp_status apsp_batch_create(const float* const* W, float* const* D, int32_t* const* P, const int* n, int count,
                              const apsp_options* opt, apsp_batch** out, void* stream);
apsp_status apsp_batch_launch(apsp_batch* b, void* stream);
apsp_status apsp_batch_destroy(apsp_batch* b);

/*
 * Autotuner of the batched launch (the paper tunes its block size to the
 * machine, Section 5): phase 3 of a keyed graph runs on tiles of 32 x 64,
 * 64 x 64 or 128 x 64 elements (named by their height: 32, 64, 128), laid
 * over the rows and columns outside the round's block; by default each graph
 * takes the shape whose tile grid wastes least for its n (the size rule).
 * For each size class the batch holds (n <= 64,
 * <= 128, <= 256, <= 512) it times a persistent launch over that class's
 * graphs with the size rule and with each tile height for the whole class
 * (one warm-up and two timed runs each), keeps the fastest, and later
 * apsp_batch_launch calls use it. The block size stays 32 (apsp_batched_bs);
 * the tile does not change any result.
 *   rows_out: optional HOST array of 4 ints, per class the chosen height, 0
 *             when the size rule was fastest, -1 for classes without graphs.
 * It runs the batch's solves, so W must not alias D (APSP_EINVAL otherwise);
 * it synchronises `stream` and must not run while a launch of b is in flight
 * or during stream capture. Before any autotuning every graph uses the size
 * rule.
 */
apsp_status apsp_batch_autotune(apsp_batch* b, int* rows_out, void* stream);

/* ---------------------------------------------------------------- serving */

typedef struct apsp_server apsp_server;

typedef struct {
  uint64_t submitted;   /* jobs accepted by apsp_serve_submit */
  uint64_t completed;   /* jobs whose results are ready */
  uint64_t rejected;    /* submits refused (invalid, over budget) */
  uint64_t in_flight;   /* admitted jobs not yet completed */
  uint64_t queued;      /* submitted jobs waiting for admission */
  double graphs_per_s;  /* completed / (time of last completion - time of first submit) */
  double p50_ms;        /* median submit -> result-ready latency of completed jobs */
  double p99_ms;        /* 99th percentile of the same */
  double mean_ms;
  double max_ms;
  uint64_t hbm_in_use;  /* bytes of device memory held by admitted jobs */
  uint64_t hbm_peak;    /* high-water mark of hbm_in_use */
} apsp_stats;

/*
 * Create a continuous-batching server on the current CUDA device.
 *   hbm_budget_bytes: cap on the device memory admitted jobs may hold at once
 *                     (each job holds its D, P and staging buffers).
 *   max_slots:        cap on jobs resident on the device at once (>= 1).
 * A scheduler thread admits queued jobs as budget and slots free up, packs
 * small graphs into batched launches and gives large graphs their own
 * streams, so work submitted while other work runs overlaps on the device.
 */
apsp_status apsp_serve_create(apsp_server** out, size_t hbm_budget_bytes, int max_slots);

/*
 * Queue one APSP job. W is a HOST pointer to n*n fp32 weights; it is copied
 * before the call returns. Never blocks on the GPU. *job_id receives the id.
 * Returns APSP_EINVAL for a malformed W (negative / NaN weight, n < 1) and
 * APSP_ENOMEM when the job alone could never fit in the HBM budget.
 */
apsp_status apsp_serve_submit(apsp_server* s, const float* W, int n, uint64_t* job_id);

/*
 * apsp_serve_submit with per-job options (opt NULL = as apsp_serve_submit):
 *   bs:    0 = the default, else 32, 64 or 128;
 *   dtype: AUTO (the 16-bit path where eligible), F32, or U16X2 (APSP_EINVAL
 *          for an ineligible W);
 *   flags: 0 or APSP_FLAG_TEST_PANEL_TIMEOUT (testing only: the job's
 *          bounded device waits expire, and its poll returns APSP_ETIMEOUT);
 *          other flags are rejected with APSP_EINVAL;
 *   validate: ignored (the server always checks W on the host).
 * Graphs of order <= 512 with bs 0/32, dtype AUTO/F32 and no flag join the
 * batched launches; every other job runs the single-graph path with its
 * options. A job whose device waits expired fails alone: jobs running beside
 * it are not affected.
 */
apsp_status apsp_serve_submit_ex(apsp_server* s, const float* W, int n, const apsp_options* opt, uint64_t* job_id);

/*
 * Wait up to timeout_ms (0 = don't wait, < 0 = forever) for job_id and copy
 * its result to HOST buffers D (n*n fp32) and P (n*n int32); either may be
 * NULL. On success the job is released. Returns APSP_EBUSY / APSP_ETIMEOUT
 * while it is not ready, APSP_ENOTFOUND for an unknown id. A finished job
 * that failed is released too and returns its status (APSP_ETIMEOUT when a
 * bounded device wait of its solve expired, APSP_ENOMEM or APSP_ECUDA). bs_used (may be
 * NULL) receives the block size the job ran with.
 */
apsp_status apsp_serve_poll(apsp_server* s, uint64_t job_id, float* D, int32_t* P, int* bs_used, int timeout_ms);

/* Snapshot of the server's counters and latency percentiles. */
apsp_status apsp_serve_stats(apsp_server* s, apsp_stats* out);

/* Cancel queued jobs, drain the device, join the scheduler, free everything. */
apsp_status apsp_serve_destroy(apsp_server* s);

/* ---------------------------------------------------------------- allocation-free solve */

/*
 * apsp_fw_noalloc: the single-graph solve of apsp_fw_ex without any device
 * memory allocation. The paper has no counterpart; this exists for callers
 * that cannot allocate device memory when they need a solve (a host framework
 * that owns all device memory, code that must not block on or fail in an
 * allocator mid-run, environments without the stream-ordered allocator).
 * Its workspace is one fixed array of APSP_NOALLOC_SCRATCH_BYTES in device
 * memory, part of the library and held by every GPU that loads it until the
 * process exits.
 *   W, D, P, n, opt, info, stream: as apsp_fw_ex (W, D, P device pointers the
 *     caller owns; opt NULL = defaults). APSP_FLAG_TIME_PHASES is rejected
 *     (APSP_EINVAL) because it would create CUDA events.
 *   Limit: apsp_fw_workspace_size(n, opt) must not exceed
 *     APSP_NOALLOC_SCRATCH_BYTES, else APSP_ENOMEM and nothing is enqueued.
 *     With dtype F32 that allows any n that is a multiple of 128 (up to
 *     62464 with bs = 128, whose packed panel slices are larger) and any
 *     n <= 2816 otherwise; AUTO / U16X2 allow n <= 2816, or n <= 5632 (5504
 *     with bs = 128) when n is a multiple of 128 (room for the 16-bit
 *     working matrix).
 *   The first call on a device looks up the array's device address (once per
 *   device, with that device current); make that first call before any CUDA
 *   stream capture.
 *   All calls on a device share the array: calls that overlap on the GPU race
 *   and corrupt each other. Nothing carries over between calls; each call
 *   zeroes or rewrites what it uses.
 */
#define APSP_NOALLOC_SCRATCH_BYTES (64u << 20)
apsp_status apsp_fw_noalloc(const float* W, float* D, int32_t* P, int n, const apsp_options* opt,
                            apsp_run_info* info, void* stream);

/* Size of the fixed array apsp_fw_noalloc works in (APSP_NOALLOC_SCRATCH_BYTES). */
size_t apsp_noalloc_scratch_bytes(void);

/* ---------------------------------------------------------------- path reconstruction */

/*
 * Section 3 of arXiv 1811.01201: P[i][j] is the intermediate vertex added last
 * to the path i -> j, kept for rebuilding the path; the path is
 * path(i, P[i][j]) followed by path(P[i][j], j), and P == -1 is the direct
 * edge.
 *
 * apsp_paths: batched walks of a DEVICE P, one thread per pair.
 *   P:     device, n*n int32, row-major, leading dimension n (as apsp_fw* write it).
 *   pairs: device, 2*count int32: the (i, j) pairs, i first.
 *   out:   device, count*cap int32: path t is out[t*cap .. t*cap + len[t] - 1]
 *          (i first, j last); the rest of the row is overwritten as scratch.
 *   len:   device, count int32: the vertex count of each path, or -1 exactly
 *          where apsp_path (below) returns -1 for the same P, pair and cap.
 * Vertex lists equal apsp_path's on a host copy of P. The buffers stay the
 * caller's. Asynchronous on `stream` (one kernel launch, no allocation, so it
 * may be captured into a CUDA graph).
 * Errors: APSP_EINVAL for n < 1, count < 0, cap < 1 or a null pointer with
 * count > 0 (nothing launched); APSP_ECUDA if the launch fails. count == 0
 * launches nothing.
 */
apsp_status apsp_paths(const int32_t* P, int n, const int32_t* pairs, int count, int32_t* out, int cap,
                       int32_t* len, void* stream);

/* ---------------------------------------------------------------- host helpers */

/*
 * Vertices of the shortest path i -> j encoded in a HOST copy of P (n*n int32):
 * writes i, ..., j into out (capacity cap) and returns the count, or -1 when
 * the walk is malformed, exceeds cap or n vertices, or an index is out of range.
 * Unreachable pairs (and i == j) give the single vertex i (count 1) only when
 * i == j; for i != j with P == -1 the result is the direct edge (count 2) --
 * check D[i][j] for reachability.
 */
int apsp_path(const int32_t* P, int n, int i, int j, int32_t* out, int cap);

#ifdef __cplusplus
}
#endif

#endif /* APSP_H */
