/*
 * fsp.h -- C ABI of the GB300 library for batched evaluation of the
 * two-machine lower bound of the permutation flow-shop problem.
 *
 * Method: Melab, Chakroun, Mezmaz, Tuyttens, "A GPU-accelerated
 * Branch-and-Bound Algorithm for the Flow-Shop Scheduling Problem"
 * (arXiv:1208.3933).  Problem statement: Section II-B (n jobs visit machines
 * M_1..M_m in order, one permutation for every machine, minimise the
 * makespan).  Bound: Section II-C (Lageweg, Lenstra and Rinnooy Kan's
 * generalisation of Johnson's two-machine rule), Section II-D (tables PTM,
 * LM, JM, RM, QM, MM; Table I) and the figure "Pseudo-code implementing the
 * LB function".  Parallel model: Section III-A (the pool of sub-problems is
 * bounded on the GPU, one evaluation per sub-problem).
 *
 * Conventions for every entry point:
 *   - Jobs are numbered 0..n-1 and machines 0..m-1.
 *   - A node (sub-problem) is a scheduled prefix sigma of d distinct jobs;
 *     its unscheduled set U is every other job.  A pool of N nodes is an
 *     int16 matrix [N][n] (row-major; only the first d entries of a row are
 *     read, the rest is ignored) plus an int32 vector of depths [N].
 *   - The caller owns every buffer it passes; the library keeps no pointer
 *     to it after the call returns (or, for stream-ordered calls, after the
 *     enqueued work completes).
 *   - "device" pointers are CUDA global-memory pointers on the device that
 *     was current when the instance was created; "host" pointers are
 *     ordinary (pinned or pageable) host memory.
 *   - Every error that can be detected on the host is returned at once and
 *     nothing is enqueued.  Bad rows never fault: their bound is
 *     FSP_LB_INVALID.
 *   - Entry points are thread-safe for distinct instances; one instance may
 *     be used by several threads for stream-ordered bounding.
 */
#ifndef FSP_H
#define FSP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque instance: the processing times plus every per-instance table of
 * Section II-D, kept resident on the device for the instance's lifetime. */
typedef struct fsp_instance fsp_instance;

typedef enum fsp_status {
    FSP_OK = 0,
    FSP_EINVAL = -1,     /* a bad argument (null pointer, size out of range, wrong device) */
    FSP_ENOMEM = -2,     /* host or device allocation failed */
    FSP_ECUDA = -3,      /* a CUDA runtime call or kernel launch failed */
    FSP_EBADNODE = -4,   /* (B&B only) an internal node failed validation */
    FSP_ETIMEDOUT = -5,  /* a bounded device- or host-side wait ran out */
    FSP_ENOTFOUND = -6,  /* branch-and-bound: no schedule of makespan <= ub0 */
    FSP_EBUSY = -7       /* a server refused work (shut down or over budget) */
} fsp_status;

/* Bound written for a row whose depth is outside [0,n], whose prefix holds a
 * job outside [0,n) or holds a job twice. */
#define FSP_LB_INVALID (-1)

/* Limits of fsp_instance_create. */
#define FSP_MAX_JOBS 1024
#define FSP_MAX_MACHINES 32

/* Read-only facts about an instance (fsp_instance_query). */
typedef struct fsp_instance_info {
    int32_t n;              /* jobs */
    int32_t m;              /* machines */
    int32_t pairs;          /* machine couples k<l: m(m-1)/2 */
    int32_t compact;        /* 1: 32-bit Johnson records, 0: 128-bit records */
    int64_t device_bytes;   /* device memory held by the instance */
    int32_t device;         /* CUDA ordinal the tables live on */
    int32_t flags;          /* FSP_INSTANCE_* options given at creation */
} fsp_instance_info;

/* Launch shape of the bounding kernel.  Zero in any field means "choose":
 * the library then uses the autotuned shape for this instance and pool size
 * when one is cached, else its built-in heuristic.  Two kernels compute the
 * same bound:
 *   FSP_KERNEL_LOCKSTEP  each thread bounds K nodes, all threads of a warp
 *                        walk the same couple (suits few couples, m <= 8);
 *   FSP_KERNEL_LANES     each warp bounds 32 nodes, its lanes walk 32
 *                        different couples (suits m >= 9). */
#define FSP_KERNEL_AUTO 0
#define FSP_KERNEL_LOCKSTEP 1
#define FSP_KERNEL_LANES 2
/* Lanes kernel staging: all records resident in shared memory (warps then
 * work independently); streamed through two tile buffers, each block setting
 * up its nodes and scanning in one kernel; or split: a prep kernel sets up
 * every 32-node batch into stream-ordered scratch (from a per-device memory
 * pool the library keeps; about (n + 48 m + 64) * 4 bytes per 32 nodes, at
 * most 2^20 nodes' worth per call) and a scan kernel streams the tiles; or
 * warp: every warp streams the tiles through its own ring of buffers and the
 * warps of a block work independently; or global: no tiles, every warp reads
 * its couples' records from global memory (L2/L1) through a ring of register
 * loads, and each warp takes its own work items (a 32-node batch and a slice
 * of the couples), so a small pool can occupy every SM (32-bit records only;
 * blocks_per_sm up to 16 / warps_per_block). */
#define FSP_STAGING_AUTO 0
#define FSP_STAGING_RESIDENT 1
#define FSP_STAGING_STREAMED 2
#define FSP_STAGING_SPLIT 3
#define FSP_STAGING_WARP 4
#define FSP_STAGING_GLOBAL 5
typedef struct fsp_launch_config {
    int32_t kernel;              /* FSP_KERNEL_* */
    int32_t nodes_per_thread;    /* lockstep: K in {1,2,4,8}; lanes: nodes per warp, 32 (0 = 32) or,
                                    streamed staging with compact records, 28 or 56: one or two sets
                                    of 28 nodes (a set's flag word leaves bits 7, 15, 23 and 31
                                    unused), each Johnson record applied to every node of the warp */
    int32_t blocks_per_sm;       /* resident blocks per SM (lockstep 1 or 2; lanes: streamed staging
                                    1..8, split/warp staging 1 or 2, global staging 1..16; at most
                                    16 warps per SM) */
    int32_t pairs_per_tile;      /* lockstep: couples staged in shared memory at a time;
                                    lanes, streamed, split and global: couples per work item,
                                    rounded up to whole groups of 32 (fewer than all: a block
                                    batch is split by couples over several work items, for pools
                                    too small to occupy every SM); other stagings: all couples.
                                    0 = chosen from the pool size; the resolved value is P for
                                    all. */
    int32_t warps_per_block;     /* lanes: 1..16 warps of 32 nodes */
    int32_t positions_per_tile;  /* lanes, streamed/split/warp: Johnson positions per tile (multiple of 4) */
    int32_t staging;             /* lanes: FSP_STAGING_* */
    int32_t tail_slices;         /* lanes, streamed, every couple per work item: the block
                                    batches of the last partial wave are split into this many
                                    couple slices (at most G), so that they occupy more of the
                                    grid; 0 or 1 = none (the default; the autotuner also tries
                                    2 and 3); other stagings: 1 */
} fsp_launch_config;

/*
 * fsp_instance_create -- builds the tables of Section II-D once per instance
 * ("computed once at the beginning of the algorithm") and uploads them to the
 * current CUDA device.
 *   p    host, row-major [n][m] int32 processing times p_jk >= 0, copied;
 *   n    1 <= n <= FSP_MAX_JOBS;  m  2 <= m <= FSP_MAX_MACHINES;
 *        the sum of all p_jk must be below 2^30 (every time the bound forms
 *        then fits in int32);
 *   out  receives the new instance (NULL on failure).
 * Errors: FSP_EINVAL for a bad argument (checked before any CUDA call),
 * FSP_ENOMEM, FSP_ECUDA.
 */
fsp_status fsp_instance_create(const int32_t *p, int32_t n, int32_t m, fsp_instance **out);

/* Options of fsp_instance_create_ex.
 *   FSP_INSTANCE_RELEASE_PER_JOB  the release time of machine k (the RM row
 *     of the figure "Pseudo-code implementing the LB function", where a
 *     couple's scan starts) is read per job, as Section II-D names RM "the matrix of the
 *     earliest starting times of jobs": r_k = min over unscheduled j of
 *     est_jk, with est_j0 = C(sigma,0) and est_jk = max(C(sigma,k),
 *     est_j,k-1 + p_j,k-1); r_k = C(sigma,k) when no job is left.  It is
 *     never earlier than the default max(C(sigma,k), min_U sum_{h<k} p_jh),
 *     so the bound is at least as tight, at about n' m more operations per
 *     node.  Bounded by the couple-lanes kernels only (a node-lockstep shape
 *     is refused with FSP_EINVAL). */
#define FSP_INSTANCE_RELEASE_PER_JOB 0x1u

/* fsp_instance_create with options (flags: FSP_INSTANCE_* bits; other bits
 * give FSP_EINVAL).  fsp_instance_create(p, n, m, out) is flags = 0. */
fsp_status fsp_instance_create_ex(const int32_t *p, int32_t n, int32_t m, uint32_t flags,
                                  fsp_instance **out);

/* Frees the instance and its device tables.  NULL is a no-op.  No bounding
 * call on this instance may be in flight. */
void fsp_instance_destroy(fsp_instance *inst);

/* Fills *info.  Errors: FSP_EINVAL for a NULL argument. */
fsp_status fsp_instance_query(const fsp_instance *inst, fsp_instance_info *info);

/*
 * fsp_bound_pool -- the bounding operator of Section III-A over one pool:
 * for every node x, out_lb[x] = max over couples (k,l), k<l, of the
 * two-machine-with-lags value of the figure "Pseudo-code implementing the LB
 * function" (release times from the prefix, Johnson order filtered to U,
 * minimum latency of machine l), or FSP_LB_INVALID for a bad row.
 *   nodes   device int16 [N][n], row-major (read-only);
 *   depths  device int32 [N] (read-only);
 *   N       number of nodes, N >= 0 (0 enqueues nothing);
 *   out_lb  device int32 [N] (written);
 *   cuda_stream  a cudaStream_t, or NULL for the legacy default stream.
 * Stream-ordered: returns once the work is enqueued.
 * Errors: FSP_EINVAL (NULL pointers with N > 0, N < 0, current device is not
 * the instance's), FSP_ECUDA (launch failure).  A device-side wait that ran
 * out is reported by the next call on the instance as FSP_ETIMEDOUT.
 */
fsp_status fsp_bound_pool(const fsp_instance *inst, const int16_t *nodes, const int32_t *depths,
                          int64_t N, int32_t *out_lb, void *cuda_stream);

/* fsp_bound_pool with an explicit launch shape (cfg may be NULL = choose).
 * Errors as fsp_bound_pool, plus FSP_EINVAL for a shape that cannot run. */
fsp_status fsp_bound_pool_ex(const fsp_instance *inst, const int16_t *nodes, const int32_t *depths,
                             int64_t N, int32_t *out_lb, void *cuda_stream,
                             const fsp_launch_config *cfg);

/*
 * fsp_bound_pool_host -- the paper's accounting of one pool (Section III-A:
 * the pool is off-loaded to the device, the bounds are returned to the
 * host): copies nodes and depths from host memory, bounds them, copies the
 * bounds back, and returns when out_lb is filled.  The pool is moved in
 * chunks so that copies and bounding overlap, through device staging memory
 * from the library's stream-ordered pool (page-locked host buffers copy
 * fastest).
 *   nodes host int16 [N][n]; depths host int32 [N]; out_lb host int32 [N].
 *   cuda_stream orders the work (NULL = legacy default stream); the call
 *   synchronises with it before returning.
 * Errors as fsp_bound_pool, plus FSP_ENOMEM.
 */
fsp_status fsp_bound_pool_host(const fsp_instance *inst, const int16_t *nodes,
                               const int32_t *depths, int64_t N, int32_t *out_lb,
                               void *cuda_stream);

/*
 * fsp_branch_and_bound -- depth-first B&B (Section II-A operators, Section
 * II-B forward branching) with GPU bounding of every expanded node's
 * children as one pool (Section III-A):
 *   - UB starts at ub0 + 1 and there is no incumbent; the root is bounded;
 *   - a popped node with LB >= UB is eliminated (the paper eliminates on
 *     LB > UB; with UB = best + 1 this finds the same optimum);
 *   - a popped leaf (depth n, whose bound is its makespan) becomes the
 *     incumbent and UB := its makespan;
 *   - the children of a popped inner node are bounded together, ordered by
 *     (LB, job) ascending and pushed so the smallest is explored first;
 *     children with LB >= UB are dropped.
 *   ub0            any int32; FSP_ENOTFOUND if no schedule has makespan <= ub0;
 *   best_perm      host int16 [n] (or NULL) receives an optimal permutation;
 *   best_makespan  host (or NULL) receives its makespan;
 *   nodes_bounded  host (or NULL) receives the number of bound evaluations.
 * Synchronous; uses its own CUDA stream.
 * Errors: FSP_EINVAL, FSP_ENOMEM, FSP_ECUDA, FSP_EBADNODE, FSP_ENOTFOUND.
 */
fsp_status fsp_branch_and_bound(const fsp_instance *inst, int32_t ub0, int16_t *best_perm,
                                int32_t *best_makespan, int64_t *nodes_bounded);

/*
 * fsp_branch_and_bound_device -- the same depth-first B&B with branching and
 * elimination on the device as well (the steps on either side of the bound,
 * which the paper runs on the CPU in Section III-A).  The open nodes live in
 * a device stack; each round pops up to `expand` nodes from its top (a node
 * whose LB reached UB is eliminated), generates their children on the device
 * (one per unscheduled job, forward branching of Section II-B), bounds them
 * as one pool, takes the best leaf as the incumbent when it lowers UB, drops
 * children with LB >= UB and pushes the rest where the parents were -- the
 * children of the topmost parent on top, each parent's children in
 * decreasing (LB, job) order so the smallest is popped first.  Node rows
 * never leave the device, and the round's sizes live in device state: a
 * depth-first search with at most 16,384 child slots per round (expand * n)
 * enqueues up to 16 rounds at a time (replays of one captured round) and
 * the host reads the state once per such group (node limit, stack growth,
 * end); other searches read it once per round.
 *   ub0, best_perm, best_makespan, nodes_bounded  as fsp_branch_and_bound
 *                  (with expand = 1 the exploration order is the same, up to
 *                  when a leaf updates UB: at generation, not when popped);
 *   expand         parents per round, 0..65536 (0 = 256);
 *   selection      FSP_SELECT_DEPTH_FIRST: the parents are the top of the
 *                  stack (the paper's configurations); FSP_SELECT_BEST_FIRST:
 *                  the `expand` open nodes of smallest LB, deeper first among
 *                  equal bounds (the paper's own GPU B&B selects best-first,
 *                  Section IV), found by binning the key (LB, -depth) of the
 *                  open nodes between the root's bound and UB (4096 bins;
 *                  on a wider range a bin holds several keys) and swapped to
 *                  the top of the stack before the round; nodes of one bin
 *                  are taken by stack position, the most recently pushed
 *                  first, so the search is deterministic;
 *   node_limit     0 = none; otherwise the search stops with FSP_ETIMEDOUT
 *                  once that many bounds were evaluated, checked between
 *                  groups of rounds (nodes_bounded is still written).
 * Synchronous; uses its own CUDA stream; device memory grows with the stack
 * (at least expand * n children of n int16 jobs, plus the stack).
 * Errors: FSP_EINVAL, FSP_ENOMEM, FSP_ECUDA, FSP_EBADNODE, FSP_ENOTFOUND,
 * FSP_ETIMEDOUT.
 */
#define FSP_SELECT_DEPTH_FIRST 0
#define FSP_SELECT_BEST_FIRST 1
fsp_status fsp_branch_and_bound_device(const fsp_instance *inst, int32_t ub0, int32_t expand,
                                       int32_t selection, int64_t node_limit, int16_t *best_perm,
                                       int32_t *best_makespan, int64_t *nodes_bounded);

/*
 * fsp_autotune -- picks the launch shape for pools of N nodes of this
 * instance.  The paper notes that the best configuration depends on the
 * instance and pool size and must be found at run time by testing (Section
 * VI); this times every shape of both kernels that fits the device on the
 * given pool (the bounds are written to out_lb), requires all of them to
 * produce identical bounds, and remembers the fastest in the instance, so
 * later fsp_bound_pool calls with the same N use it.
 *   nodes, depths, out_lb  device buffers as in fsp_bound_pool, N >= 1;
 *   cache_path  NULL, or a text file: a cached entry for (device, n, m,
 *               record format, N) is used without timing, and a new result
 *               is appended;
 *   best, best_ms  (optional) the chosen shape and its time per launch in ms
 *               (-1 when it came from the cache).
 * Synchronous on cuda_stream.  Errors: FSP_EINVAL, FSP_ECUDA (a launch failed
 * or two shapes disagreed), FSP_ETIMEDOUT.
 */
fsp_status fsp_autotune(const fsp_instance *inst, const int16_t *nodes, const int32_t *depths, int64_t N,
                        int32_t *out_lb, void *cuda_stream, const char *cache_path,
                        fsp_launch_config *best, float *best_ms);

/* The launch shape fsp_bound_pool would use for N nodes (autotuned if
 * fsp_autotune ran for this N, else the built-in heuristic).
 * Errors: FSP_EINVAL, FSP_ECUDA. */
fsp_status fsp_tuned_config(const fsp_instance *inst, int64_t N, fsp_launch_config *cfg);

/* One pool of a batch: N nodes of instance `inst`, with device buffers laid
 * out as in fsp_bound_pool. */
typedef struct fsp_pool_desc {
    const fsp_instance *inst;
    const int16_t *nodes;   /* device [N][inst->n] */
    const int32_t *depths;  /* device [N] */
    int32_t *out_lb;        /* device [N] */
    int64_t N;
} fsp_pool_desc;

/* A batch plan: many pools, possibly of different instances and sizes,
 * bounded together by one persistent launch. */
typedef struct fsp_batch fsp_batch;

/*
 * fsp_batch_create -- plans the batched form of the bounding operator
 * (Section III-A applied to several pools at once): every pool is cut into
 * 32-node work items, ordered longest first, and the plan (per-pool arguments,
 * work items and a work counter) is uploaded to the current device, which
 * must be the device of every instance.
 *   pools  host array of `count` descriptors (copied; the device buffers they
 *          name must stay valid while the batch is launched);
 *   warps_per_block  1..16, or 0 to choose (16, or for a plan of fewer than
 *          16 work items per SM the fewest warps that give every item its
 *          own warp with at most one block per SM);
 *   out    receives the plan.
 * Every instance must use 32-bit Johnson records (fsp_instance_info.compact).
 * Errors: FSP_EINVAL, FSP_ENOMEM, FSP_ECUDA.
 */
fsp_status fsp_batch_create(const fsp_pool_desc *pools, int32_t count, int32_t warps_per_block,
                            fsp_batch **out);

/* fsp_batch_create with a couple split: a work item is a 32-node batch and a
 * slice of ceil(couples_per_item / 32) groups of 32 machine couples of its
 * instance (the pair split of the couple-lanes scan); a pool whose instance
 * has more groups is cut into that many slices per batch, each slice sets up
 * its nodes and scans its couples, and the slices meet in an atomic max on
 * the pool's bounds (zeroed by the launch first; an invalid row is found
 * invalid by every slice).  couples_per_item = 0: every couple in one item
 * (fsp_batch_create).  Spreads few or uneven pools over more warps.
 * Errors as fsp_batch_create (FSP_EINVAL also for couples_per_item < 0). */
fsp_status fsp_batch_create_ex(const fsp_pool_desc *pools, int32_t count, int32_t warps_per_block,
                               int32_t couples_per_item, fsp_batch **out);

/* Enqueues the whole batch on the stream as one persistent kernel (after a
 * reset of its work counter): each warp claims work items until none is
 * left.  Stream-ordered; launches of one plan must not overlap.
 * Errors: FSP_EINVAL (NULL, wrong device), FSP_ECUDA. */
fsp_status fsp_batch_launch(fsp_batch *batch, void *cuda_stream);

/* As fsp_batch_launch, through a CUDA graph (counter reset + kernel) captured
 * on the first call and replayed afterwards. */
fsp_status fsp_batch_launch_graph(fsp_batch *batch, void *cuda_stream);

/* Work items, nodes, warps per block and blocks of a plan (any may be NULL). */
fsp_status fsp_batch_query(const fsp_batch *batch, int64_t *work_items, int64_t *nodes,
                           int32_t *warps_per_block, int32_t *blocks);
/* fsp_batch_query plus the plan's couples per work item (0 = all). */
fsp_status fsp_batch_query_ex(const fsp_batch *batch, int64_t *work_items, int64_t *nodes,
                              int32_t *warps_per_block, int32_t *blocks, int32_t *couples_per_item);

/* Frees the plan; none of its launches may be in flight.  NULL is a no-op. */
void fsp_batch_destroy(fsp_batch *batch);

/*
 * fsp_batch_autotune -- picks the node tile of a batch plan (warps, hence
 * 32-node work items in flight, per block) by timing plans of the same pools
 * with 16, 12, 8, 6, 4 and 2 warps per block on the stream (one warm-up and
 * three timed launches each; shapes that do not fit are skipped).  The pools'
 * out_lb buffers are written (every shape writes the same bounds).
 *   pools, count   as fsp_batch_create (count >= 1);
 *   best_warps     receives the fastest warps_per_block, for fsp_batch_create;
 *   best_ms        (or NULL) receives its time per launch.
 * Synchronous.  Errors: FSP_EINVAL, FSP_ENOMEM, FSP_ECUDA.
 */
fsp_status fsp_batch_autotune(const fsp_pool_desc *pools, int32_t count, void *cuda_stream,
                              int32_t *best_warps, float *best_ms);

/* fsp_batch_autotune over both shapes of the plan, the node tile and the
 * pair split: first the warps per block as above (every couple in one work
 * item), then the two fastest tiles again with 32, 64, 96 and 128 couples
 * per work item (fsp_batch_create_ex); the fastest pair is returned.
 *   best_couples_per_item  (or NULL: the node tile alone is tuned) receives
 *                          0 or the couples per work item.
 * Synchronous.  Errors as fsp_batch_autotune. */
fsp_status fsp_batch_autotune_ex(const fsp_pool_desc *pools, int32_t count, void *cuda_stream,
                                 int32_t *best_warps, int32_t *best_couples_per_item, float *best_ms);

/* ---------------------------------------------------------------------
 * Bounding server: continuous batching of many clients' pools.
 * --------------------------------------------------------------------- */
typedef struct fsp_server fsp_server;
typedef struct fsp_request fsp_request;

typedef struct fsp_server_config {
    int64_t hbm_budget_bytes;  /* device arena for admitted pools (0 = 1 GiB) */
    int32_t max_batch_pools;   /* pools gathered into one launch (0 = 256) */
    int32_t slots;             /* batches in flight at once, 1..8 (0 = 2) */
    int32_t warps_per_block;   /* batched kernel shape (0 = choose) */
    int32_t reserved;
} fsp_server_config;

typedef struct fsp_server_stats {
    int64_t pools_done, nodes_done, batches;
    double mean_pools_per_batch;
    double p50_us, p99_us, mean_us;  /* submission-to-completion latency */
    double active_seconds;           /* first completed submission to last completion */
    int64_t queued, in_flight;
    int64_t arena_bytes, arena_bytes_used;
} fsp_server_stats;

/*
 * fsp_server_create -- a bounding server on the current device (the paper's
 * bounding operator, Section III-A, offered to many concurrent B&B searches
 * or other clients).  A dispatcher thread admits queued pools in arrival
 * order while their device footprint (nodes, depths, bounds) fits the
 * arena, gathers the admitted pools into one batched launch per free slot
 * (a CUDA stream), copies pools in and bounds out, and keeps admitting while
 * earlier batches run, so later arrivals overlap them on the device.
 * Instances stay resident; their tables are not copied per request.
 * Errors: FSP_EINVAL, FSP_ENOMEM, FSP_ECUDA.
 */
fsp_status fsp_server_create(const fsp_server_config *cfg, fsp_server **out);

/* Queues a pool of N nodes of `inst` (host buffers, pinned or pageable:
 * nodes [N][n], depths [N], out_lb [N]); the buffers must stay valid until
 * the request completes or is cancelled.  *req receives the request handle.
 * Errors: FSP_EINVAL; FSP_EBUSY when the server no longer accepts work or the
 * pool alone exceeds the whole arena (admission refused). */
fsp_status fsp_server_submit(fsp_server *srv, const fsp_instance *inst, const int16_t *nodes,
                             const int32_t *depths, int64_t N, int32_t *out_lb, fsp_request **req);

/* Waits up to timeout_us microseconds (negative = no limit) for the request:
 * FSP_OK when out_lb holds the bounds, FSP_ETIMEDOUT if it is still pending
 * (the handle stays valid), FSP_EBUSY if it was cancelled, or the error that
 * failed its batch. */
fsp_status fsp_request_wait(fsp_request *req, int64_t timeout_us);

/* Removes a request that is still queued (FSP_OK); admitted requests run to
 * completion (FSP_EBUSY). */
fsp_status fsp_request_cancel(fsp_request *req);

/* Drops the handle; a request still running is freed when it completes. */
void fsp_request_release(fsp_request *req);

/* Counters and latency percentiles since creation or the last reset. */
fsp_status fsp_server_get_stats(fsp_server *srv, fsp_server_stats *stats);
fsp_status fsp_server_reset_stats(fsp_server *srv);

/* Stops accepting requests (later submissions get FSP_EBUSY); queued and
 * running requests complete. */
fsp_status fsp_server_shutdown(fsp_server *srv);

/* Shuts down, waits for every admitted and queued request, frees the server
 * and every request handle it issued (released or not): no handle may be
 * used afterwards. */
void fsp_server_destroy(fsp_server *srv);

/*
 * fsp_server_search -- a depth-first B&B client of the server (Section II-A
 * operators, Section II-B branching) that expands the top `expand` nodes of
 * its stack at once and submits all their children as one pool, so that many
 * searches keep the server's batches full.  UB starts at ub0 + 1; a child
 * whose bound reaches UB is dropped; a bounded leaf (depth n) below UB
 * becomes the incumbent at once.  The optimum equals fsp_branch_and_bound's;
 * node counts differ (several nodes expanded per step).
 *   expand  nodes expanded per request (>= 1);
 *   node_limit  stop after this many bound evaluations (0 = no limit); the
 *           search then returns FSP_ETIMEDOUT with its best incumbent so far;
 *   best_perm (host int16 [n] or NULL), best_makespan, nodes_bounded (or NULL).
 * srv may be NULL: the same search then bounds each pool by its own plain
 * launch (fsp_bound_pool_host on a stream of its own), so that the served
 * and the plain forms can be compared on identical pools (the search is
 * deterministic: same ub0 and expand, same pools, same result).
 * Synchronous.  Errors: FSP_EINVAL, FSP_ENOMEM, FSP_EBUSY, FSP_EBADNODE,
 * FSP_ENOTFOUND (no schedule of makespan <= ub0), FSP_ETIMEDOUT.
 */

/* NEH constructive heuristic (Nawaz, Enscore and Ham 1983; not part of the
 * paper's method): a complete schedule whose makespan serves as ub0.
 * perm: host int16 [n] or NULL.  Errors: FSP_EINVAL. */
fsp_status fsp_neh(const fsp_instance *inst, int16_t *perm, int32_t *makespan);

/* Iterated greedy heuristic (Ruiz and Stuetzle 2007; not part of the
 * paper's method): from the NEH schedule, `iterations` rounds of removing
 * four random jobs, reinserting each at its best position and improving the
 * result by reinsertion until no move helps, accepted like simulated
 * annealing.  A tighter ub0 than NEH, so a search proves the optimum with
 * fewer nodes.  Deterministic for a given seed.
 *   iterations  >= 0 (0 = the NEH schedule);  seed  any value;
 *   perm  host int16 [n] or NULL: the best schedule found;
 *   makespan  receives its makespan (recomputed from perm: a valid upper bound).
 * Synchronous, host only.  Errors: FSP_EINVAL. */
fsp_status fsp_iterated_greedy(const fsp_instance *inst, int32_t iterations, uint64_t seed, int16_t *perm,
                               int32_t *makespan);
fsp_status fsp_server_search(fsp_server *srv, const fsp_instance *inst, int32_t ub0, int32_t expand,
                             int64_t node_limit, int16_t *best_perm, int32_t *best_makespan,
                             int64_t *nodes_bounded);

/*
 * fsp_server_solve -- one problem solved by `searchers` cooperating
 * depth-first searches over the server (the multi-search extension the paper
 * names as future work, on one GPU).  Each searcher runs fsp_server_search's
 * step on its own stack; all share one incumbent, so a schedule found by one
 * prunes every stack at once; a searcher whose stack is empty steals the
 * bottom half (the shallowest nodes) of the fullest stack.  The search ends
 * when every stack is empty and no searcher has a pool in flight.  The
 * optimum equals fsp_branch_and_bound's; node counts vary from run to run
 * (the interleaving of the searchers is not fixed).
 *   searchers  1..256 host threads; expand  nodes expanded per request;
 *   node_limit, best_perm, best_makespan, nodes_bounded  as fsp_server_search;
 *   steals     host (or NULL): number of steals.
 * Synchronous.  Errors as fsp_server_search.
 */
fsp_status fsp_server_solve(fsp_server *srv, const fsp_instance *inst, int32_t ub0, int32_t searchers,
                            int32_t expand, int64_t node_limit, int16_t *best_perm,
                            int32_t *best_makespan, int64_t *nodes_bounded, int64_t *steals);

/* Largest number of pools fsp_bound_batch_noalloc accepts in one call. */
#define FSP_NOALLOC_MAX_POOLS 64

/*
 * fsp_bound_batch_noalloc -- the batched bound of fsp_batch_create followed by
 * fsp_batch_launch, for callers that cannot allocate memory when they need a
 * bound: a process whose GPU memory is already owned by another allocator, a
 * serving loop that must not take cudaMalloc's implicit synchronisation, or
 * code running where allocation is not permitted.  The paper has no
 * counterpart; it exists for such callers only.
 *   pools  host array of `count` descriptors, 0 <= count <= FSP_NOALLOC_MAX_POOLS
 *          (more is refused with FSP_EINVAL); every instance must use 32-bit
 *          records and live on the current device;
 *   cuda_stream  orders the work (NULL = legacy default stream).
 * No device or host memory is allocated: the plan and the work counter live in
 * a fixed per-device array inside the library, sized for
 * FSP_NOALLOC_MAX_POOLS pools.  Every call reuses that array (it keeps the
 * previous call's plan; the counter is reset by each call), so two calls whose
 * work overlaps on the GPU race: order them on one stream or synchronise
 * between them.  The first call on a device looks up the array's address with
 * that device current; make that first call outside any stream capture.
 * Stream-ordered; the descriptors are consumed before the call returns.
 * Errors: FSP_EINVAL, FSP_ECUDA.
 */
fsp_status fsp_bound_batch_noalloc(const fsp_pool_desc *pools, int32_t count, void *cuda_stream);

/* Static English text for a status code (never NULL). */
const char *fsp_status_string(fsp_status s);

/* Library version as "major.minor.patch" (static string). */
const char *fsp_version(void);

/* fsp_check_wait_timeout -- self-check of the device-side bounded waits (no
 * counterpart in the paper): every wait in the bounding kernels gives up
 * after a clock64 limit, reports FSP_ETIMEDOUT and returns instead of
 * hanging.  This runs one such wait, limit_cycles long (1..2^32), on a
 * barrier phase that nothing completes; it returns FSP_ETIMEDOUT when the
 * mechanism works (the instance stays usable), FSP_EINVAL/FSP_ECUDA on a bad
 * argument or launch. */
fsp_status fsp_check_wait_timeout(const fsp_instance *inst, int64_t limit_cycles);

/* fsp_kernel_launches -- number of CUDA kernels this library has enqueued in
 * the process so far (every entry point counts its own launches; no compute
 * of the method, the paper has no counterpart).  For launch accounting around
 * a timed region. */
int64_t fsp_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* FSP_H */
