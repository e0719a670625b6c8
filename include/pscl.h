/*
 * pscl.h -- C ABI of the GB300 (sm_103a) library for the two-level sampling-based
 * clustering of "A parallel sampling based clustering" (Sastry & Netti, arXiv 1412.1947).
 *
 * The method (Algorithm 1 and §V of the paper):
 *   1. scale every attribute (Algorithm 1, step 1)             -> pscl_scale_features
 *   2. peel equal-sized subclusters around a landmark and run
 *      Lloyd's k-means on each (Algorithm 1, steps 2-5; §II)    -> pscl_subcluster
 *   3. run Lloyd's k-means on the pooled local centers (§V)    -> pscl_cluster
 *
 * Conventions shared by every entry point
 *   - Every function returns a pscl_status; none aborts.  pscl_last_error() gives a
 *     message for the calling thread's last failure.
 *   - Points are n x d, row-major (all d attributes of a point are contiguous, the
 *     paper's "row major flattening", §V), float32.  n >= 1, 1 <= d <= 1024.
 *   - Work is queued on the context's CUDA stream and runs asynchronously; the
 *     pscl_get_* calls synchronise that stream before copying results out.
 *   - The library allocates and owns all device memory it uses; caller buffers are
 *     only read (inputs) or written (outputs) and are never retained, except the
 *     device input pointer of pscl_job_create/pscl_job_load, which must stay valid
 *     until the next pscl_scale_features on that job has completed.
 *   - Calls on one job must come in the order scale -> subcluster -> cluster
 *     (PSCL_ESTATE otherwise); a job is used by one host thread at a time.
 *   - Inputs must be finite; a non-finite value makes pscl_scale_features' result
 *     undefined and is reported as PSCL_EINVAL by the next pscl_get_* call.
 */
#ifndef PSCL_H
#define PSCL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pscl_ctx pscl_ctx;
typedef struct pscl_job pscl_job;

typedef enum {
    PSCL_OK = 0,
    PSCL_EINVAL = 1,   /* bad argument (size, pointer, enum value)                    */
    PSCL_ESTATE = 2,   /* call out of order (e.g. cluster before subcluster)           */
    PSCL_ENOMEM = 3,   /* the job would exceed the context's device-memory budget      */
    PSCL_EBUSY = 4,    /* serving queue full; retry later (never blocks)               */
    PSCL_ETIMEOUT = 5, /* a bounded wait gave up                                       */
    PSCL_ECUDA = 6     /* a CUDA runtime call failed; see pscl_last_error()            */
} pscl_status;

/* Storage type of the points.  PSCL_BF16: bfloat16 bit patterns (uint16); they are widened
 * to float32 (exactly) at the start of every run and the scaled values are rounded to
 * bfloat16 (Algorithm 1 step 1 in the job's storage type), kept in float32. */
typedef enum { PSCL_F32 = 0, PSCL_BF16 = 1 } pscl_dtype;

/* Arithmetic of the Lloyd assignment step (§I's "nearest center").
 *  PSCL_PREC_FP32: direct float32 sum of (x_j - c_j)^2 on the CUDA cores.
 *  PSCL_PREC_TF32, PSCL_PREC_BF16: the -2 x.c part on the tensor cores with TF32 or
 *      BF16 inputs and float32 accumulation, every point whose best two centers are
 *      closer than the contraction's error bound re-decided by the float32 direct sum.
 *  PSCL_PREC_TF32X3, PSCL_PREC_BF16X3: the same with every operand split into a high
 *      and a low TF32 / BF16 part and the three leading products summed in one
 *      contraction (far fewer near ties to re-decide).
 *  PSCL_PREC_TC: per point set, TF32X3 where its operands fit one CTA's shared memory,
 *      else BF16X3 (the split mode that serves the shape; the result is the same).
 *  The contraction covers d in {16, 32, 64, 128} and at most 256 centers per point set
 *  whose operand tiles fit one CTA's shared memory (d = 128 only in BF16 with 16
 *  centers, d = 64 in TF32X3 only with 16); other shapes use the float32 direct sum.
 *  The near-tie bound is rigorous, so every mode assigns exactly as PSCL_PREC_FP32 does.
 *  Every mode yields the same partition into subclusters; the update step is the same
 *  exact fixed-point mean in all modes. */
typedef enum {
    PSCL_PREC_FP32 = 0,
    PSCL_PREC_TF32 = 1,
    PSCL_PREC_BF16 = 2,
    PSCL_PREC_TF32X3 = 3,
    PSCL_PREC_BF16X3 = 4,
    PSCL_PREC_TC = 5
} pscl_prec;

/* Job options (pscl_job_set_option). */
typedef enum {
    /* 1: run the local Lloyd as one launch pair per subcluster per iteration (the
     *    plain per-subcluster form) instead of batching all subclusters.  Default 0. */
    PSCL_OPT_PLAIN_LLOYD = 1,
    /* 1: keep the labels of every Lloyd iteration for pscl_get_label_trace. Default 0. */
    PSCL_OPT_TRACE_LABELS = 2,
    /* 1: every Lloyd run starts from the first k_eff members of its point set instead
     *    of the seeded shuffle (used by worked examples).  Default 0. */
    PSCL_OPT_INIT_FIRST_K = 3,
    /* 1: record the pipeline's launches into a CUDA graph on first use and replay it
     *    on later runs with the same parameters.  Default 0. */
    PSCL_OPT_GRAPH = 4,
    /* 1: time every kernel launch of later unrecorded runs with CUDA events on the
     *    context's stream (pscl_get_kernel_times).  Default 0. */
    PSCL_OPT_KERNEL_TIMING = 5,
    /* Batches only (pscl_batch_set_option): rows per work unit of the Lloyd launches,
     *    32..1024 (rounded up to a multiple of 32), 0 = the planner's default.  A tuning
     *    choice: results do not depend on it. */
    PSCL_OPT_UNIT_ROWS = 6,
    /* Rows per thread in the float32 assignment kernel: 0 = automatic (one row when no
     *    work unit of the run has more rows than the kernel's 256 threads, else up to 4
     *    rows kept in registers), 1 = one, 2 = eight for d <= 16.  Jobs and batches;
     *    results do not depend on it. */
    PSCL_OPT_ROWS_PER_THREAD = 7,
    /* Jobs only, 1: the Lloyd on the pooled local centers weighs each local center by its
     *    cluster's size (members in the last local iteration): a center moves to the
     *    size-weighted mean of its pooled points, so the second level clusters the
     *    subclusters' means as the abstract describes, each standing for its points.
     *    The local level and the final SSE over all n points are unchanged; the pooled
     *    Lloyd then runs in float32 (prec ignored) with global 64-bit sums.  Needs
     *    n < 2^31 (else PSCL_EINVAL).  Default 0 (unweighted). */
    PSCL_OPT_POOL_WEIGHTED = 8,
    /* Jobs only: rounds of the peel that one pass of landmark distances may serve, 1..32,
     *    0 = the default (32).  The landmark changes only after every remaining point holding
     *    some attribute's minimum has been taken, and until then the next round is the next
     *    N points of the same order, so one pass settles up to this many rounds at once (an
     *    epoch resolves only the rounds before the last holder of some attribute's value
     *    leaves, read off the keys).  A tuning choice: results do not depend on it. */
    PSCL_OPT_PEEL_ROUNDS = 9,
    /* Polls of every bounded device-side wait (the peel's grid barriers, the tensor-core
     *    assignment's commit waits) before it gives up and the job reports PSCL_ETIMEOUT;
     *    0 = the default (2^25 polls per barrier, about a second or two).  Jobs only. */
    PSCL_OPT_WAIT_LIMIT = 10,
    /* Test hook, jobs only: 1 = the peel's first grid barrier waits for one arrival more
     *    than the grid gives, 2 = the tensor-core assignment waits once on a barrier that
     *    nothing completes; either wait gives up after PSCL_OPT_WAIT_LIMIT polls and the
     *    job reports PSCL_ETIMEOUT.  For tests of the give-up path; default 0. */
    PSCL_OPT_TEST_STALL = 11,
    /* Jobs only: most thread blocks of the peel's cooperative launch, 0 = as many as fit
     *    (two per SM).  A smaller grid lets the peels of several jobs run side by side; a
     *    tuning choice: results do not depend on it. */
    PSCL_OPT_PEEL_GRID = 12
} pscl_option;

/* The library's kernels, for pscl_get_kernel_times. */
typedef enum {
    PSCL_K_SCALE_MINMAX = 0, /* column minima / maxima                           */
    PSCL_K_SCALE_APPLY,      /* element-wise min-max scaling                     */
    PSCL_K_PEEL,             /* all peel rounds (one persistent launch)          */
    PSCL_K_GATHER,           /* subcluster-packed copy of the points             */
    PSCL_K_LLOYD_INIT,       /* seeded initial centers                           */
    PSCL_K_LLOYD_ASSIGN,     /* nearest center + fixed-point sums                */
    PSCL_K_LLOYD_FINALIZE,   /* centers = sums / counts                          */
    PSCL_K_FINAL_SSE,        /* nearest final center and SSE of every point      */
    PSCL_K_LLOYD_SUMS,       /* after a tensor-core assignment: near ties
                                re-decided in float32, fixed-point sums          */
    PSCL_K_COUNT
} pscl_kernel;

/* Context: one device, one stream, one device-memory budget.
 *   device            CUDA device ordinal.
 *   hbm_budget_bytes  upper bound on device memory the context's jobs may hold
 *                     (0 = no bound beyond what the device has).
 *   stream            a cudaStream_t to queue work on, or NULL for a stream the
 *                     context creates (and destroys) itself.
 * Errors: PSCL_EINVAL (out is NULL, bad device), PSCL_ECUDA. */
int pscl_ctx_create(pscl_ctx **out, int device, size_t hbm_budget_bytes, void *stream);
int pscl_ctx_destroy(pscl_ctx *ctx);
/* Bytes of device memory currently held by the context's jobs. */
size_t pscl_ctx_bytes_in_use(const pscl_ctx *ctx);
/* Message of the calling thread's last failed call ("" if none). Never NULL. */
const char *pscl_last_error(void);

/* Job: one clustering problem.
 *   points            n x d row-major, float32 or bfloat16 (dtype), on the host (points_on_device = 0; copied
 *                     to the device before the call returns its status) or on the
 *                     context's device (points_on_device = 1; read later, by
 *                     pscl_scale_features, on the context's stream: their writes must
 *                     be complete or queued on that stream first -- a context created
 *                     with a NULL stream has its own non-blocking stream, which does not
 *                     wait for work on the legacy default stream).
 * Errors: PSCL_EINVAL (NULL pointer, n < 1, d outside 1..1024, dtype not PSCL_F32 / PSCL_BF16),
 *         PSCL_ENOMEM (over budget), PSCL_ECUDA. */
int pscl_job_create(pscl_ctx *ctx, const void *points, int dtype, int64_t n, int32_t d,
                    int points_on_device, pscl_job **out);
/* Replace the job's points by another n x d set (same n, d) and reset it to the state
 * right after pscl_job_create.  Buffers and recorded graphs are kept. */
int pscl_job_load(pscl_job *job, const void *points, int points_on_device);
int pscl_job_set_option(pscl_job *job, int option, int64_t value);
int pscl_job_destroy(pscl_job *job);

/* Feature scaling (Algorithm 1, step 1): per attribute j, with mn_j / mx_j the
 * minimum / maximum over all points, x'_ij = float((double(x_ij) - mn_j) * (1 / (mx_j -
 * mn_j))) computed in double; a constant attribute becomes 0.  All later steps work on
 * the scaled points. */
int pscl_scale_features(pscl_job *job);

/* Equal-sized subclustering (Algorithm 1 steps 2-5, repeated on the points left out as
 * in §II) followed by Lloyd's k-means on every subcluster (Algorithm 1 step 4, §I).
 *   N        subcluster size, >= 1.  S = ceil(n / N) subclusters; the last one holds
 *            the n - (S-1) N points left.
 *   local_k  local centers per subcluster, >= 1; a subcluster of m < local_k points gets
 *            k_eff = m centers.  P = sum of k_eff pooled centers.
 *   iters    Lloyd iterations (>= 0), exactly this many.
 *   seed     initial centers: the first k_eff entries of a Fisher-Yates shuffle of the
 *            subcluster driven by SplitMix64 keyed by (seed, stage 0, subcluster index).
 *   prec     a pscl_prec.
 * Round r: L = per-attribute minimum of the remaining points; the N remaining points
 * nearest to L by squared Euclidean distance (float64, ascending attribute order; equal
 * distances by ascending point index) form subcluster r and are removed.
 * Errors: PSCL_EINVAL, PSCL_ESTATE (not scaled yet), PSCL_ENOMEM, PSCL_ECUDA. */
int pscl_subcluster(pscl_job *job, int64_t N, int32_t local_k, int32_t iters, uint64_t seed,
                    int prec);

/* Unequal-sized subclustering (Algorithm 2) in place of pscl_subcluster: L and H are the
 * points made of every attribute's lowest and highest scaled value; the segment from L
 * to H is cut into m equal pieces whose middles are the landmarks
 *     l_i = float(L + ((i + 1/2) / m) (H - L)), i = 0..m-1   (double arithmetic);
 * every point joins its nearest landmark (squared Euclidean distance in float64 as for
 * pscl_subcluster, the lower landmark index on ties).  The groups that got points are the
 * subclusters, in landmark order, points in ascending index; then Lloyd runs on each of
 * them as in pscl_subcluster (local_k, iters, seed, prec; subcluster s = the s-th
 * non-empty group), and pscl_cluster follows as usual.  m: 1..4096.  Synchronises with
 * the device once (the group sizes plan the Lloyd launches), so it is not recorded by
 * PSCL_OPT_GRAPH.  Errors as pscl_subcluster. */
int pscl_subcluster_unequal(pscl_job *job, int32_t m, int32_t local_k, int32_t iters, uint64_t seed, int prec);

/* Final clustering of the P pooled local centers (§V) into final_k centers with Lloyd
 * (initial centers keyed by (seed, stage 1, 0)), then the nearest final center and the
 * sum of squared errors of every scaled point.
 * Errors: PSCL_EINVAL (final_k < 1 or > P), PSCL_ESTATE, PSCL_ENOMEM, PSCL_ECUDA. */
int pscl_cluster(pscl_job *job, int32_t final_k, int32_t iters, uint64_t seed, int prec);

/* The three steps in one call: pscl_scale_features, pscl_subcluster(N, local_k, iters,
 * seed, prec) and pscl_cluster(final_k, iters, seed, prec).  With PSCL_OPT_GRAPH the
 * launches are recorded into a CUDA graph on the first call and replayed by later calls
 * with the same arguments and input pointer (the input's contents may change).
 * Errors: as the three calls. */
int pscl_run(pscl_job *job, int64_t N, int32_t local_k, int32_t final_k, int32_t iters,
             uint64_t seed, int prec);

/* Wait for all queued work of the job. */
int pscl_job_sync(pscl_job *job);

/* Results (each synchronises the stream first; any pointer may be NULL to skip it).
 *   pscl_get_scaled:        out n*d float, the scaled points (original order).
 *   pscl_get_partition:     perm n (original index of the i-th point in subcluster-packed
 *                           order; subcluster s is perm[seg_off[s] .. seg_off[s+1]-1], in
 *                           ascending index), seg_off S+1, *n_seg = S.
 *   pscl_get_local_centers: centers P*d float in (subcluster, center) order, k_eff S,
 *                           counts P (members of each local center, last iteration).
 *   pscl_get_result:        centers final_k*d float, labels n (nearest final center of
 *                           every point, original order), *sse. */
int pscl_get_scaled(pscl_job *job, float *out);
int pscl_get_partition(pscl_job *job, int64_t *perm, int64_t *seg_off, int64_t *n_seg);
int pscl_get_local_centers(pscl_job *job, float *centers, int32_t *k_eff, int32_t *counts);
int pscl_get_result(pscl_job *job, float *centers, int32_t *labels, double *sse);
/* Sizes of the current plan: *n_seg = S, *n_pooled = P (after pscl_subcluster). */
int pscl_get_sizes(pscl_job *job, int64_t *n_seg, int64_t *n_pooled);
/* Labels of every Lloyd iteration (needs PSCL_OPT_TRACE_LABELS before the run).
 *   stage 0: iters*n int32, iteration-major, subcluster-packed order;
 *   stage 1: iters*P int32, the final Lloyd over the pooled centers. */
int pscl_get_label_trace(pscl_job *job, int stage, int32_t *out);
/* Launches of every kernel (PSCL_K_COUNT entries) queued by the last run, and, if
 * PSCL_OPT_KERNEL_TIMING was on for it, their summed device time in milliseconds (else
 * 0).  Either pointer may be NULL. */
int pscl_get_kernel_times(pscl_job *job, int64_t *launches, float *ms);
/* Near-tie statistics of the last run's tensor-core assignments (PSCL_PREC_TF32/BF16):
 * *rechecked rows re-decided by the float32 direct distance out of *assigned rows
 * (both 0 under PSCL_PREC_FP32).  Either pointer may be NULL. */
int pscl_get_recheck_stats(pscl_job *job, int64_t *rechecked, int64_t *assigned);
/* Statistics of the last equal-sized subclustering (Algorithm 1 steps 2-5): *epochs
 * (rounds committed together from one landmark), *passes (distance passes over the points
 * left: one per landmark change), *key_updates (of those passes, the ones that updated
 * the keys from the few attributes whose landmark value moved instead of recomputing
 * them) and *barriers (grid-wide barriers the launch passed).  PSCL_ESTATE if no such
 * subclustering ran on the job.  Pointers may be NULL. */
int pscl_get_peel_stats(pscl_job *job, int64_t *epochs, int64_t *passes, int64_t *key_updates,
                        int64_t *barriers);
/* Device time of the phases of the last run in milliseconds: [0] scale, [1] peel,
 * [2] local Lloyd (incl. init), [3] final Lloyd, [4] SSE pass. */
int pscl_get_phase_ms(pscl_job *job, float *ms5);

/* Measured float32 FMA throughput of `device` in TFLOP/s (2 flops per FMA): independent
 * FMA chains on every SM at full occupancy, timed with CUDA events, best of five after a
 * warm-up.  The peak that the float32 direct assignment (one subtract and one FMA per
 * attribute of a distance) is graded against; not part of the method.  Allocates and
 * frees a few KB of device memory; takes some tens of milliseconds.
 * Errors: PSCL_EINVAL (tflops NULL), PSCL_ECUDA. */
int pscl_measure_fp32_fma(int device, double *tflops);

/* Measurement service beside the method: the time of one grid-wide barrier of the peel's
 * own implementation (monotonic arrival counter, release on arrival, acquire while
 * polling, bounded waits) in the peel's launch shape on `device` (its block size, shared
 * memory and CTAs per SM), the best of three runs of 2000 barriers in a row, in
 * microseconds: the latency floor that the peel's barriers put under its epochs.
 * PSCL_EINVAL if us is NULL, PSCL_ECUDA on a CUDA error, PSCL_ETIMEOUT if a wait gave up. */
int pscl_measure_grid_barrier(int device, double *us);

/* Nearest center and sum of squared errors of n points, allocating nothing.
 *
 * The paper has no counterpart: this is a service for callers that cannot allocate
 * device memory (a framework whose allocator owns the device, a real-time host that
 * forbids allocation after start-up, code where an allocation would synchronise).  It
 * runs the kernel of the SSE step of pscl_cluster: labels[i] = the nearest of the k
 * centers to points[i] (float32 squared distance, lowest index on ties) and *sse = the
 * sum over points of that distance, added in double in a fixed order.
 *   points   n x d float32 row-major, device memory of the current device
 *   centers  k x d float32 row-major, device memory
 *   labels   n int32, device memory (written)
 *   sse      one double, device memory (written)
 *   stream   cudaStream_t to run on, or NULL for the default stream
 * Limits: 1 <= n <= 2^31-1, 1 <= d <= 1024, 1 <= k <= 4096; PSCL_EINVAL beyond.
 * Scratch: a fixed array of 4096 float64 partial sums plus a counter (33 KB) that every
 * device loading the library holds until exit.  Every call on a device shares it and it
 * keeps the last call's contents (the counter is cleared at the start of each call), so
 * calls whose work overlaps on the GPU race: order them on one stream or synchronise.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture.  The address is looked up again when
 * the current context is not the one it was found in (after cudaDeviceReset, say); that
 * call too must come before any capture.  Nothing is allocated or freed.
 * Errors: PSCL_EINVAL, PSCL_ECUDA (see pscl_last_error()). */
int pscl_assign_sse_noalloc(const float *points, int64_t n, int32_t d, const float *centers,
                            int32_t k, int32_t *labels, double *sse, void *stream);

/* Device bytes a job of this shape holds once pscl_run has planned it (every allocation
 * of pscl_job_create, pscl_subcluster and pscl_cluster, as counted against the budget):
 * the admission figure of the server below.  No device work. */
int pscl_job_footprint(pscl_ctx *ctx, int64_t n, int32_t d, int64_t N, int32_t local_k, int32_t final_k,
                       int32_t iters, int dtype, int points_on_device, int trace, size_t *bytes);

/* ---------------------------------------------------------------- serving
 * A request loop for whole two-level jobs (scale + pscl_subcluster + pscl_cluster) of
 * mixed shapes, with continuous batching: a native scheduler thread admits queued jobs
 * onto `slots` execution slots (one CUDA stream each) as slots and device memory free up,
 * so jobs that arrive while others run start at once and their kernels overlap on the
 * device.  Admission: a job starts when a slot is free and its pscl_job_footprint fits
 * the budget left; jobs start in arrival order, except that a later job that fits may
 * start ahead of an earlier one that does not, until that one has been passed over 32
 * times.  Each result equals the result of the same job run alone (every kernel is
 * deterministic).  The paper has no serving layer; this is the form its method takes
 * behind a service. */
typedef struct pscl_server pscl_server;
typedef struct {
    const void *points;   /* n x d float32, row-major; must stay valid until the job is done */
    int32_t on_device;    /* 1: 16-byte aligned device memory of the server's device (read in
                             place); 0: host memory, copied when the job is admitted */
    int32_t dtype;        /* PSCL_F32, or PSCL_BF16 (bfloat16 bit patterns) */
    int64_t n;
    int32_t d;
    int64_t N;            /* subcluster size */
    int32_t local_k, final_k, iters;
    uint64_t seed;
    int32_t prec;         /* pscl_prec of both Lloyd stages */
    int32_t want_labels;  /* 1: keep the n labels of the final clustering for pscl_fetch */
} pscl_job_desc;
typedef enum { PSCL_JOB_QUEUED = 0, PSCL_JOB_RUNNING = 1, PSCL_JOB_DONE = 2, PSCL_JOB_FAILED = 3 } pscl_job_state;
/* slots: 1..64 jobs on the device at once; hbm_budget_bytes: admission budget (0 = 90% of
 * the device memory free now).  The server's contexts live on ctx's device. */
int pscl_server_create(pscl_ctx *ctx, int32_t slots, size_t hbm_budget_bytes, pscl_server **out);
/* Queues a job and returns at once with its ticket.  PSCL_EINVAL for a bad shape,
 * PSCL_ENOMEM if its footprint exceeds the whole budget (it could never start), PSCL_EBUSY
 * if 2^20 jobs are already queued; never blocks on the device. */
int pscl_submit(pscl_server *s, const pscl_job_desc *desc, uint64_t *ticket);
/* The ticket's pscl_job_state. */
int pscl_poll(pscl_server *s, uint64_t ticket, int32_t *state);
/* Waits until the job is done or failed; timeout_us < 0 waits without limit, otherwise
 * PSCL_ETIMEOUT when the time is up (the job keeps going). */
int pscl_wait(pscl_server *s, uint64_t ticket, int64_t timeout_us);
/* Results of a finished job, then the ticket is released (any output may be NULL):
 * centers final_k x d float32 (scaled coordinates), labels n int32 (needs want_labels),
 * sse, times_ms[3] = {queued, admitted to done, submitted to done} on the host clock.
 * A failed job returns its error code.  PSCL_ESTATE if the job has not finished. */
int pscl_fetch(pscl_server *s, uint64_t ticket, float *centers, int32_t *labels, double *sse, double *times_ms);
/* out[8]: completed, failed, queued, running, bytes in use, peak bytes in use, most jobs
 * running at once, budget. */
int pscl_server_stats(pscl_server *s, int64_t *out);
/* Fails the queued jobs, waits for the running ones, releases everything. */
int pscl_server_destroy(pscl_server *s);

/* ---------------------------------------------------------------- uneven batches
 * Many independent clustering instances of uneven sizes, each with its own k: the
 * first-level Lloyd runs of Algorithm 1 step 4 (§II), given directly instead of produced
 * by the peel.  Every instance is min-max scaled on its own (Algorithm 1 step 1, same
 * formula as pscl_scale_features) and then clustered by Lloyd (§I) from the seeded
 * initial centers of segment = its index, stage 0 (the seeding of pscl_subcluster).
 * All instances advance together: each launch covers work units of every instance, and a
 * run is recorded once into a CUDA graph (PSCL_OPT_GRAPH, on by default for batches) and
 * replayed.  The paper has no batch of independent problems; it is the serving form of
 * its first level.
 *
 * points: sum(sizes) x d float32, row-major, instance after instance (host memory, or
 *         16-byte aligned device memory of the context's device with on_device = 1; a
 *         device buffer is read, not copied, by every run and must outlive the batch).
 * sizes, k: n_inst entries each; sizes >= 1, 1 <= k <= 4096; instance i gets
 *         k_eff = min(k[i], sizes[i]) centers.  sum(sizes) <= 2^31 - 1.
 * Errors: PSCL_EINVAL (bad argument), PSCL_ENOMEM (budget or device memory),
 *         PSCL_ECUDA.  The library owns every device allocation of the batch. */
typedef struct pscl_batch pscl_batch;
int pscl_batch_create(pscl_ctx *ctx, const void *points, int on_device, int32_t d, int32_t n_inst,
                      const int64_t *sizes, const int32_t *k, pscl_batch **out);
/* New points of the same shape for later runs (host memory is copied on the context's
 * stream; a device buffer is used in place, as for pscl_batch_create). */
int pscl_batch_load(pscl_batch *b, const void *points, int on_device);
/* Options: PSCL_OPT_TRACE_LABELS, PSCL_OPT_GRAPH, PSCL_OPT_PLAIN_LLOYD (one launch pair
 * per instance and iteration, for comparison), PSCL_OPT_UNIT_ROWS,
 * PSCL_OPT_ROWS_PER_THREAD; others return PSCL_EINVAL. */
int pscl_batch_set_option(pscl_batch *b, int option, int64_t value);
/* Autotuner: times `iters` Lloyd iterations of this batch (unrecorded, after one warm-up
 * run) for every work-unit size in {128, 256, 512, 1024} rows and the three rows-per-thread
 * settings, keeps the fastest and applies it; the choice is remembered for later batches
 * of the same (device, d, largest k, log2 of the rows, prec).  Writes the choice and
 * whether it came from that memory (any output may be NULL).  Results never depend on it. */
int pscl_batch_tune(pscl_batch *b, int32_t iters, int prec, int64_t *unit_rows, int32_t *rows_per_thread,
                    int32_t *cached);
/* Queues scale + seeded init + `iters` Lloyd iterations + per-instance SSE on the
 * context's stream and returns; prec as for pscl_subcluster. */
int pscl_batch_run(pscl_batch *b, int32_t iters, uint64_t seed, int prec);
/* Waits for the batch's queued work; PSCL_EINVAL if an input value is not finite. */
int pscl_batch_sync(pscl_batch *b);
/* Results of the last run (waits first; any output may be NULL):
 *   centers: sum(k_eff) x d float32, instance after instance, in scaled coordinates;
 *   labels:  sum(sizes) int32, the nearest final center of every point (index within its
 *            instance, lowest on ties);
 *   sse:     n_inst doubles, per instance the sum over its scaled points of the squared
 *            distance to the nearest final center. */
int pscl_batch_get(pscl_batch *b, float *centers, int32_t *labels, double *sse);
/* The scaled points, sum(sizes) x d float32. */
int pscl_batch_get_scaled(pscl_batch *b, float *out);
/* iters x sum(sizes) labels of every iteration (needs PSCL_OPT_TRACE_LABELS). */
int pscl_batch_get_label_trace(pscl_batch *b, int32_t *out);
/* Kernel launches of the last run (counted when it was queued or recorded). */
int pscl_batch_launches(pscl_batch *b, int64_t *launches);
/* Device time of the Lloyd iterations of the last unrecorded run, in milliseconds. */
int pscl_batch_lloyd_ms(pscl_batch *b, float *ms);
int pscl_batch_destroy(pscl_batch *b);

#ifdef __cplusplus
}
#endif
#endif /* PSCL_H */
