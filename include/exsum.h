/*
 * exsum.h -- C ABI of a GB300 (sm_103a) CUDA library for multidimensional
 * included and excluded sums (Xu, Fraser, Leiserson, "Multidimensional
 * Included and Excluded Sums", SIAM ACDA 2021).
 *
 * Problem (Sec. 2, Definition "Included and Excluded Sums"): for a
 * d-dimensional tensor A of shape n_1 x ... x n_d, a box size
 * k = (k_1, ..., k_d) and an associative, commutative operator (+) with
 * identity e, the INCLUDED sum at x reduces A over the box
 * [x_1, x_1+k_1) x ... x [x_d, x_d+k_d) clipped to the tensor (Sec. 2,
 * colon notation), and the EXCLUDED sum at x reduces A over every coordinate
 * outside that box (the "strong" problem of Sec. 1: no inverse is used).
 *
 * Common conventions for every entry point below
 *   Layout      Tensors are dense and row-major: dimension d (index d-1 in
 *               `shape`) is contiguous, dimension 1 is the slowest.
 *   Pointers    `in` and `out` are DEVICE pointers on the current CUDA
 *               device.  `in` is read only; `out` must not overlap `in`.
 *               The caller owns both.  `shape` and `k` are HOST arrays of
 *               `d` entries, read during the call only.
 *   Types       in dtype -> out dtype:  I32 -> I32, I64 -> I64,
 *               F32 -> F32, BF16 -> F32 (bf16 inputs are accumulated and
 *               returned in fp32).  Integer + wraps modulo 2^32 / 2^64, so
 *               integer results are exact and order-independent; max is
 *               exact.  Floating-point + accumulates in fp32 with
 *               compensated (two-sum) carries on every long reduction.
 *   Arguments   1 <= d <= EXSUM_MAX_DIMS, n_i >= 1, 1 <= k_i <= n_i
 *               (Sec. 1 requires k_i <= n_i); anything else returns
 *               EXSUM_EINVAL before any work is queued.
 *   Streams     `stream` is a cudaStream_t (NULL = legacy default stream).
 *               Work is queued asynchronously on it; nothing synchronises
 *               unless stated.  Results are ready when the stream reaches
 *               the point after the call.
 *   Errors      0 on success, a negative EXSUM_E* code otherwise.  A CUDA
 *               error is reported as EXSUM_ECUDA; exsum_last_cuda_error()
 *               returns the underlying cudaError_t of the calling thread.
 *               On error, the contents of `out` are unspecified.
 */
#ifndef EXSUM_H
#define EXSUM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EXSUM_MAX_DIMS 8

typedef enum { EXSUM_OP_ADD = 0, EXSUM_OP_MAX = 1 } exsum_op;

typedef enum { EXSUM_I32 = 0, EXSUM_I64 = 1, EXSUM_F32 = 2, EXSUM_BF16 = 3 } exsum_dtype;

enum {
    EXSUM_OK = 0,
    EXSUM_EINVAL = -1,      /* invalid argument (shape, box, dtype, op, pointer) */
    EXSUM_ENOMEM = -2,      /* workspace too small, or an allocation failed */
    EXSUM_EUNSUPPORTED = -3,/* valid request this build does not handle */
    EXSUM_ECUDA = -4,       /* a CUDA runtime call failed; see exsum_last_cuda_error */
    EXSUM_ETIMEDOUT = -5,   /* a bounded host-side wait ran out */
    EXSUM_EBUSY = -6        /* resource busy (server full, capture in progress) */
};

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int exsum_version(void);

/* Static description of a status code (never NULL). */
const char *exsum_strerror(int status);

/* The cudaError_t (as int) behind the calling thread's last EXSUM_ECUDA. */
int exsum_last_cuda_error(void);

/* Output dtype for an input dtype (BF16 -> F32, others unchanged); -1 if
 * `dtype` is not an exsum_dtype. */
int exsum_out_dtype(int dtype);

/* Bytes per element of a dtype; 0 if unknown. */
size_t exsum_dtype_size(int dtype);

/*
 * Workspace needed by exsum_included_ws (excluded == 0) or
 * exsum_excluded_ws (excluded != 0) for this problem, in bytes.  Returns 0
 * with *status = EXSUM_EINVAL for invalid arguments (status may be NULL).
 * The figure includes 256-byte alignment padding of each sub-buffer.
 */
size_t exsum_workspace_bytes(int d, const int64_t *shape, const int64_t *k, int op, int dtype,
                             int excluded, int *status);

/*
 * Included sums by BDBS (Sec. 3, "Included Sums in 1D" and "Generalizing to
 * Arbitrary Dimensions"): the k-blocked Range-Prefix-Row / Range-Suffix-Row
 * scans and Combine-Along-Row of BDBS-1D applied along dimensions d, ..., 1
 * in turn (BDBS-Along-Dim, Sec. 5).  out[x] = (+) over the clipped box at x.
 * `out` has the output dtype and the same shape; with two or more
 * dimensions whose box side exceeds 1, `out` also holds intermediates during
 * the call.  Uses a workspace that the
 * library allocates and caches per device (cudaMalloc on first use or
 * growth, outside any stream capture; a call made while `stream` is being
 * captured that would need to grow the cache returns EXSUM_EBUSY).
 */
int exsum_included(const void *in, void *out, int d, const int64_t *shape, const int64_t *k,
                   int op, int dtype, void *stream);

/*
 * Weak excluded sums (BDBS complement; Sec. 1 and Sec. 6, "BDBSC"): the total
 * of the tensor minus the included sum at each point.  This needs an inverse
 * of the operator, so only integer + is supported (dtype EXSUM_I32 or
 * EXSUM_I64; int32 and int64 + wrap modulo 2^32 and 2^64, which makes the
 * result exact and equal to the strong excluded sum).  Other dtypes return
 * EXSUM_EUNSUPPORTED.  Same arguments, ownership and workspace policy as
 * exsum_included (op is +); `out` also holds the included sums during the
 * call.  Runs on `stream` and returns without waiting.
 */
int exsum_excluded_weak(const void *in, void *out, int d, const int64_t *shape, const int64_t *k,
                        int dtype, void *stream);

/* As exsum_included, with a caller-owned DEVICE workspace of at least
 * exsum_workspace_bytes(..., excluded = 0) bytes (EXSUM_ENOMEM if smaller).
 * Allocates nothing; safe to capture in a CUDA graph. */
int exsum_included_ws(const void *in, void *out, int d, const int64_t *shape, const int64_t *k,
                      int op, int dtype, void *workspace, size_t workspace_bytes, void *stream);

/*
 * Excluded sums by the box-complement algorithm (Sec. 4, Theorem "Recursive
 * Box-complement" and Corollary "Excluded-sum Components"; Sec. 5,
 * Fig. "exsum-code").  For each x the complement of the box is split into
 * the 2d disjoint regions of the Corollary; region pair i is the prefix and
 * the suffix along dimension i of the tensor reduced over dimensions < i
 * (Prefix-Along-Dim / Suffix-Along-Dim) with included sums along the
 * dimensions > i (BDBS-Along-Dim), added in by Add-Contribution.
 * The GPU schedule applies the included sums along dimensions > i before the
 * prefix/suffix along dimension i (both reduce over product sets, so the
 * order is immaterial for a commutative operator), which needs one BDBS per
 * step instead of two; see the library's design notes.
 * Same arguments, ownership and workspace policy as exsum_included.  `out`
 * is written exactly once, by the last kernel of the call, and is not used
 * as scratch.
 */
int exsum_excluded(const void *in, void *out, int d, const int64_t *shape, const int64_t *k,
                   int op, int dtype, void *stream);

/* As exsum_excluded, with a caller-owned DEVICE workspace of at least
 * exsum_workspace_bytes(..., excluded = 1) bytes.  Allocates nothing. */
int exsum_excluded_ws(const void *in, void *out, int d, const int64_t *shape, const int64_t *k,
                      int op, int dtype, void *workspace, size_t workspace_bytes, void *stream);

/*
 * Excluded sums without any allocation.  The paper has no counterpart; this
 * entry point exists for callers that cannot allocate device memory when
 * they need the result -- a plugin inside a host framework that owns the
 * device-memory budget, a real-time loop that cannot afford cudaMalloc's
 * implicit synchronisation, a deployment whose allocations are fixed at
 * start-up.  It runs exactly the exsum_excluded pipeline on a scratch
 * buffer built into the library image: a static device array of
 * EXSUM_NOALLOC_SCRATCH_BYTES bytes that every GPU loading the library
 * holds until the process exits.  The caller still owns and passes `in` and
 * `out` (device pointers, as for exsum_excluded).
 *   - Problems whose workspace (exsum_workspace_bytes(..., excluded = 1))
 *     exceeds EXSUM_NOALLOC_SCRATCH_BYTES are rejected with EXSUM_ENOMEM
 *     before any work is queued; invalid arguments give EXSUM_EINVAL.
 *   - It calls no cudaMalloc, cudaFree or allocating library routine
 *     (keep the launch trace off, its default, when calling it).
 *   - The first call on a device looks up the device address of the buffer
 *     (cudaGetSymbolAddress, with that device current); make that first
 *     call before any stream capture on that device.  Later calls made
 *     outside a capture look it up again (cheap), so a cudaDeviceReset
 *     between calls is safe; calls inside a capture use the address of the
 *     last uncaptured call, so do not reset the device between that call
 *     and the capture.
 *   - All calls on a device share the one buffer, and a call leaves its
 *     intermediates there; the pipeline writes every scratch word before it
 *     reads it, so nothing needs clearing between calls.  Calls whose work
 *     overlaps on the GPU (different streams, or different host threads
 *     without ordering) race on the buffer; order them on one stream.
 */
#define EXSUM_NOALLOC_SCRATCH_BYTES (64u << 20)
int exsum_excluded_noalloc(const void *in, void *out, int d, const int64_t *shape, const int64_t *k,
                           int op, int dtype, void *stream);

/* Frees the library's cached per-device workspaces (synchronises the
 * device first).  Returns 0 or EXSUM_ECUDA. */
int exsum_release_cached_workspace(void);

/* Blocks of the bulk-staged final pass that gave up their bounded wait for a
 * tile's copy (about a second) and returned without writing that tile's
 * outputs, since the library was loaded, on the current device.  Never
 * expected to be non-zero; a non-zero count means the affected results are
 * wrong.  Reads device memory (synchronising with the device). */
unsigned exsum_device_timeouts(void);

/* ---------------------------------------------------------------------------
 * The paper's comparison methods on the GPU (baselines for box-complement;
 * same arguments, ownership and stream semantics as exsum_excluded).
 * ------------------------------------------------------------------------- */

/*
 * Summed-area table (Sec. 1, SAT / SATC): the inclusive prefix along every
 * dimension, then at every x the alternating sum of the table at the 2^d
 * corners of the box (inclusion-exclusion) -- the included sum, or with
 * excluded != 0 the weak excluded sum (total minus the included sum).
 * Integer + only (it needs an inverse), wrapping modulo 2^32 or 2^64, so the
 * result equals the strong excluded sum bit for bit; other dtypes give
 * EXSUM_EUNSUPPORTED.  Workspace: N elements of the dtype (cached, as for
 * exsum_excluded).
 */
int exsum_sat(const void *in, void *out, int d, const int64_t *shape, const int64_t *k, int excluded, int dtype,
              void *stream);

/*
 * Corners (App. A): the 2^d tensors T_b of (+) over the orthant below or
 * above each point in every dimension (b in {prefix, suffix}^d, from
 * 2^(d+1) - 2 inclusive scans), then out[x] = (+) of one entry of each,
 * at the box's corners shifted so that the 2^d orthants tile the complement
 * of the box exactly -- the strong excluded sum, for + and max, d = 2 or 3
 * (EXSUM_EUNSUPPORTED otherwise).  Workspace: 2^(d+1) - 2 tensors of the
 * carry type (fp32 +: compensated pairs, 8 bytes).
 */
int exsum_corners(const void *in, void *out, int d, const int64_t *shape, const int64_t *k, int op, int dtype,
                  void *stream);

/* The region of dimension `dim` that corner `corner` of exsum_corners takes
 * for d = 2 or 3: 0 below x, 1 below x + k, 2 from x on, 3 from x + k on
 * (-1 for arguments out of range).  Host only; lets a test check that the
 * regions tile the complement of the box. */
int exsum_corner_region(int d, int corner, int dim);

/*
 * Operator-cost experiment (the paper's slowed operator, Sec. 6): int64 +
 * whose every application also runs `extra` dependent steps that leave its
 * value unchanged (exsum_slow_extra sets it for the device, >= 0), through
 * box-complement's
 * row schedule (strong excluded sum), BDBS (included sum), corners (d = 2,
 * 3) or a calibration kernel applying the operator
 * EXSUM_SLOW_CALIBRATE_REPS times per element.  The slope of time against
 * `extra`, over the calibration's slope per application, is the number of
 * operator applications per element of a method.  int64 input and output,
 * arguments as for exsum_excluded.
 */
enum { EXSUM_SLOW_BOX_COMPLEMENT = 0, EXSUM_SLOW_BDBS = 1, EXSUM_SLOW_CORNERS = 2, EXSUM_SLOW_CALIBRATE = 3 };
#define EXSUM_SLOW_CALIBRATE_REPS 16
int exsum_slow_extra(int extra);
int exsum_slow_run(const void *in, void *out, int d, const int64_t *shape, const int64_t *k, int method,
                   void *stream);

/* ---------------------------------------------------------------------------
 * Batches of uneven tensors.  Not in the paper; it batches many independent
 * excluded sums (Sec. 5) so that they fill the GPU together.
 * ------------------------------------------------------------------------- */
typedef struct {
    const void *in;                  /* DEVICE input (host for EXSUM_SERVE_HOST requests) */
    void *out;                       /* DEVICE output (host for EXSUM_SERVE_HOST requests) */
    int d;                           /* dimensions, 1..EXSUM_MAX_DIMS */
    int op;                          /* exsum_op */
    int dtype;                       /* exsum_dtype of `in` */
    int64_t shape[EXSUM_MAX_DIMS];   /* first d entries used */
    int64_t k[EXSUM_MAX_DIMS];       /* first d entries used */
} exsum_desc;

typedef struct exsum_batch exsum_batch;

/*
 * Plans the excluded sums of `count` tensors as ONE CUDA graph.  Every
 * descriptor is validated as for exsum_excluded (EXSUM_EINVAL otherwise).
 * Two schedules:
 *   levels  every tensor whose excluded sum takes the row schedule with the
 *           two-dimensional lower problem (d = 3; Sec. 4) or the small d = 2
 *           path, with fp32 +, joins a level set: each pass level of all
 *           those tensors is ONE launch (per register class) whose blocks
 *           take (tensor, pass, tile) items from a device work list -- at
 *           most thirteen kernels and one memset per replay, whatever the
 *           batch size.
 *           The other tensors run on one lane beside it;
 *   lanes   the tensors are assigned to `lanes` concurrent streams --
 *           longest processing time first (order 0) or round-robin by size
 *           (order 1) -- each lane with one workspace sized for its largest
 *           tensor, every tensor with its own chain of kernels.
 * lanes > 0 picks the lanes schedule with that many streams, lanes ==
 * EXSUM_BATCH_LEVELS the level schedule with its default tuning (or the
 * one the environment variable EXSUM_LEVEL_TUNE gives as
 * "lc,interleave,tiles_per_vb,tall,persist"; see exsum_batch_schedule), and
 * lanes == 0 autotunes: candidate schedules (levels with several strided
 * chunk lengths, row-total placements, final-pass tiles per block and tile
 * heights; lanes with 1..32 streams and both orders) are captured and their
 * replays timed on the device (inputs are read and outputs written during
 * tuning), and the fastest is kept; the choice is remembered per batch
 * signature (shapes, boxes, ops, dtypes) for the process and, if the
 * environment variable EXSUM_TUNE_CACHE names a file, appended there and
 * read back by later processes.  Workspaces are allocated here with
 * cudaMalloc.  `stream` must not be capturing (EXSUM_EBUSY).  On success
 * *plan owns the graph and the workspaces until exsum_batch_destroy.
 */
#define EXSUM_BATCH_LEVELS (-1)
int exsum_batch_create(const exsum_desc *descs, int count, int lanes, void *stream,
                       exsum_batch **plan);

/* Launches the planned batch on `stream` (one cudaGraphLaunch). */
int exsum_batch_launch(exsum_batch *plan, void *stream);

/* Schedule of a plan: lanes, order, total workspace bytes, kernels per launch. */
int exsum_batch_info(const exsum_batch *plan, int *lanes, int *order, size_t *workspace_bytes,
                     int64_t *kernels);

/* The rest of the schedule (any pointer may be NULL): mode (0 lanes, 1
 * levels), tensors in the level set, and the level tuning: rows per strided
 * chunk (0: sized per tensor), row totals interleaved with the strided
 * chunks over the same rows (1) or after them (0), tiles per virtual block
 * of the bulk final pass, tall (1) or per-tensor (0) k_rowx tiles, and
 * persistent grids pulling work-list slots from a counter (1) or one block
 * per slot (0). */
int exsum_batch_schedule(const exsum_batch *plan, int *mode, int *level_tensors, int *lc, int *interleave,
                         int *tiles_per_vb, int *tall, int *persist);

/* Waits for the device, then frees the plan's graph and workspaces. */
void exsum_batch_destroy(exsum_batch *plan);

/* ---------------------------------------------------------------------------
 * Request server (continuous batching).  Not in the paper.
 * ------------------------------------------------------------------------- */
typedef struct exsum_server exsum_server;

/* In/out of a submitted request are HOST pointers: the server stages them
 * through its device memory (copy in, compute, copy out). */
#define EXSUM_SERVE_HOST 1

/*
 * Starts a server on the current device: one device arena of
 * `mem_budget_bytes` (allocated here, once) for the requests' workspaces and
 * staging buffers, `max_slots` CUDA streams (1..256) on which admitted
 * requests run concurrently, and a host worker thread.  Returns NULL on
 * invalid arguments or if the arena or streams cannot be created.
 */
exsum_server *exsum_server_create(size_t mem_budget_bytes, int max_slots);

/*
 * Queues one excluded sum (box-complement, as exsum_excluded).  Requests are
 * admitted in arrival order as soon as a slot is free and the request's
 * memory (workspace, plus input and output for EXSUM_SERVE_HOST) fits in the
 * free part of the budget; requests arriving while others run are admitted
 * as memory and slots free up, and run concurrently with them.  Device
 * pointers must stay valid, and host buffers untouched, until the request
 * completes.  Returns EXSUM_EINVAL for a malformed descriptor, EXSUM_ENOMEM
 * for a request larger than the whole budget, EXSUM_EBUSY after shutdown
 * began; otherwise *ticket identifies the request.
 */
int exsum_server_submit(exsum_server *srv, const exsum_desc *desc, int flags, uint64_t *ticket);

/*
 * As exsum_server_submit, for a request that arrives at `arrival_ns` on the
 * server's clock (exsum_server_now_ns): it is not admitted before then, and
 * its latency is measured from then.  Requests must be submitted in order of
 * arrival (they are admitted first come, first served).  Lets a load
 * generator hand the server a whole arrival schedule ahead of time.
 */
int exsum_server_submit_at(exsum_server *srv, const exsum_desc *desc, int flags,
                           int64_t arrival_ns, uint64_t *ticket);

/* The server's clock: host steady clock in nanoseconds. */
int64_t exsum_server_now_ns(void);

/*
 * Waits at most timeout_ns for a request: its status once complete,
 * EXSUM_ETIMEDOUT if still queued or running at the deadline (never blocks
 * longer), EXSUM_EINVAL for an unknown ticket.
 */
int exsum_server_wait(exsum_server *srv, uint64_t ticket, int64_t timeout_ns);

/* Server-clock times (ns) of a completed request: arrival (submission, or
 * the arrival time given to exsum_server_submit_at), admission (work queued
 * on its slot) and completion (signalled from its stream). */
int exsum_server_ticket_times(exsum_server *srv, uint64_t ticket, int64_t *submit_ns,
                              int64_t *start_ns, int64_t *done_ns);

/* Forgets a completed request (its ticket becomes unknown); EXSUM_EBUSY if
 * it has not completed. */
int exsum_server_release(exsum_server *srv, uint64_t ticket);

/* Requests completed so far, or -1 for a NULL server. */
int64_t exsum_server_completed(exsum_server *srv);

/* Stops admitting new requests, finishes every queued and running one,
 * then frees the server. */
void exsum_server_destroy(exsum_server *srv);

/*
 * Host-side fault injection for tests of the failure path (no counterpart in
 * the paper).  The next `count` requests the server admits are not launched:
 * each ends as if its launch had returned `status` (a negative EXSUM_E*
 * code), releases its memory and slot through the same stream-ordered
 * completion as a real failure, and exsum_server_wait returns `status` for
 * it.  count = 0 switches injection off.  Nothing reaches the GPU, so no
 * device fault is involved.  Returns EXSUM_EINVAL for a NULL server, a
 * negative count or a non-negative status.
 */
int exsum_server_fail_next(exsum_server *srv, int count, int status);

/*
 * Launch trace.  The paper reports time per element (Sec. 6); this breaks a
 * call's device time down by pass.  While enabled, every kernel the library
 * launches is bracketed by a pair of CUDA events recorded on the stream it
 * is launched on (inside a stream capture the pair becomes two event-record
 * nodes of the graph, re-recorded on every replay).  exsum_trace_collect
 * waits for the recorded events, writes up to `cap` records in launch order
 * -- kernel tag (see exsum_kernel_name), recursion level of box-complement
 * (0 = the input tensor), elements the pass covers, device milliseconds --
 * and returns the number of records (which may exceed cap), or EXSUM_ECUDA.
 * With clear != 0 the trace is emptied; with clear == 0 it is kept, so the
 * records of a captured graph can be read again after each replay.  Any of
 * the output arrays may be NULL.
 */
void exsum_trace_enable(int on);
int exsum_trace_collect(int *tags, int *levels, int64_t *elems, float *ms, int cap, int clear);

/* Static name of a kernel tag ("unknown" for others). */
const char *exsum_kernel_name(int tag);

/* Kernels launched by the library in this process so far. */
int64_t exsum_launch_count(void);

/* Side streams the library has created in this process so far (two per
 * caller stream on which an excluded sum first forked; diagnostics, no
 * counterpart in the paper). */
int64_t exsum_side_streams_created(void);

/*
 * Graph helpers (no counterpart in the paper).  Calls captured into a CUDA
 * graph from the caller's stream keep, per kernel node, the priority of the
 * stream it was captured on: the side branches of excluded sums run on
 * streams of the greatest priority.  A graph instantiated here honours those
 * node priorities (cudaGraphInstantiateFlagUseNodePriority), so the short
 * side-branch kernels are not queued behind the blocks of the full-tensor
 * pass they run beside; a graph instantiated without the flag runs every
 * node at the priority of the stream it is launched into.
 *
 * `graph` is a cudaGraph_t (the caller keeps ownership); *exec receives a
 * cudaGraphExec_t that the caller frees with exsum_graph_exec_destroy.
 * exsum_graph_launch launches it into `stream` (a cudaStream_t, NULL for the
 * legacy default stream) and returns without waiting.  All three return
 * EXSUM_OK, EXSUM_EINVAL for a NULL graph, exec or exec pointer, or
 * EXSUM_ECUDA (see exsum_last_cuda_error).
 */
int exsum_graph_instantiate(void *graph, void **exec);
int exsum_graph_launch(void *exec, void *stream);
int exsum_graph_exec_destroy(void *exec);

#ifdef __cplusplus
}
#endif

#endif /* EXSUM_H */
