/*
 * idw.h -- C ABI of the GB300 (sm_103a) library for global Shepard
 * inverse-distance-weighted (IDW) interpolation.
 *
 * The operation (Mei & Tian, "Performance Impact of Data Layout on the
 * GPU-accelerated IDW Interpolation", Sec. 2.1, Eq. 1): for every query
 * (prediction point) q,
 *
 *     Z(q) = sum_i w_i z_i / sum_i w_i,   w_i = d(q, x_i)^(-p),
 *
 * over ALL n data points (standard, global IDW; Sec. 1 and Sec. 2.1), with p
 * an arbitrary positive real (Sec. 2.1; typically 2).  The two local forms
 * the paper names among its related work (Sec. 1) are here too: Eq. 1 over
 * the data points within a radius R (idw_interpolate_local) and over the k
 * nearest data points (idw_interpolate_knn), each with a prepared index for
 * repeated queries (idw_local_index_*), and modified Shepard weights on the
 * radius form (idw_interpolate_modified).  Every form has gradients with
 * respect to z, the data and query coordinates, and p (idw_backward,
 * idw_local_backward, idw_modified_backward, idw_knn_backward).
 *
 * Conventions shared by every entry point:
 *   - A data point is a row (x, y, z): d is the 2-D Euclidean distance in
 *     (x, y), and z is the sampled value.  Rows are contiguous, row-major,
 *     3 elements each (the paper's unaligned AoS record, Sec. 3.2); the
 *     library restages them internally.  Queries are rows (x, y).
 *   - d^(-p) is evaluated as (d^2)^(-p/2); no square root is taken.
 *   - A query whose (x, y) equals a data point's (x, y) numerically (so
 *     d = 0, where Eq. 1 is undefined) gets the z of the LOWEST such index.
 *   - NaN in a query's inputs gives NaN in its result unless an exact hit
 *     is found first; inputs are not scanned for NaN unless the handle's
 *     IDW_OPT_VALIDATE_INPUTS option is set.
 *   - Pointers named "device" are CUDA device (or managed) memory owned by
 *     the caller; they must stay valid until the work on `stream` is done.
 *     Every float array needs 4-byte alignment, every double array 8-byte.
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Compute entry points are asynchronous: they validate their
 *     arguments on the host, enqueue kernels and return.  A CUDA error that
 *     occurs later is reported by a later call or by idw_sync_status().
 *   - A handle owns a device workspace that grows on demand.  Calls on one
 *     handle must not overlap on different streams; use one handle per
 *     concurrently used stream.  Handles are not thread-safe.
 *   - Sizes: 1 <= n < 2^31 and 0 <= m < 2^31; m = 0 is a no-op.
 */
#ifndef IDW_GB300_H
#define IDW_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct idw_handle_s *idw_handle_t;

typedef enum {
    IDW_OK = 0,
    IDW_ERR_INVALID_ARG = 1,   /* null pointer, bad size, p <= 0 or non-finite p */
    IDW_ERR_ALIGNMENT = 2,     /* a pointer lacks the element alignment */
    IDW_ERR_CUDA = 3,          /* a CUDA runtime call failed (see idw_last_cuda_error) */
    IDW_ERR_NOT_FINITE_INPUT = 4, /* NaN / inf input found (only with IDW_OPT_VALIDATE_INPUTS) */
    IDW_ERR_WORKSPACE = 5,     /* device workspace could not be allocated */
    IDW_ERR_UNSUPPORTED = 6,   /* device is not sm_103 or option not supported */
    IDW_ERR_DEVICE_TIMEOUT = 7 /* a bounded wait inside a kernel gave up */
} idw_status;

typedef enum {
    /* FP32 pair arithmetic with compensated (two-sum) accumulation; the
     * per-query combine of partial sums and the division run in FP64.
     * data/queries/out are float. */
    IDW_PREC_F32_COMP = 0,
    /* Plain FP64 throughout (the comparison form). data/queries/out are
     * double. */
    IDW_PREC_F64_PLAIN = 1
} idw_precision;

/* Human-readable name of a status code (static storage). */
const char *idw_status_string(idw_status s);

/* Creates a handle bound to CUDA device `device` (made current during each
 * call).  Fails with IDW_ERR_UNSUPPORTED if the device is not compute
 * capability 10.3. */
idw_status idw_create(idw_handle_t *handle, int device);

/*
 * As idw_create, with the autotuner's JSON cache file given directly
 * (NULL: as idw_create, i.e. the IDW_AUTOTUNE_CACHE environment variable or
 * memory only).  The file is read now if it exists and rewritten after each
 * tuning; a missing or unreadable file starts an empty table.
 */
idw_status idw_create_ex(idw_handle_t *handle, int device, const char *autotune_cache);

/* Frees the handle and its workspace after synchronising the device. */
idw_status idw_destroy(idw_handle_t handle);

/* Text of the last CUDA error seen by this handle (static storage). */
const char *idw_last_cuda_error(idw_handle_t handle);

/*
 * Eq. 1 for m queries against n data points.
 *   data_xyz   : device, n x 3 (x, y, z) rows; float or double per `prec`.
 *   queries_xy : device, m x 2 (x, y) rows; same type.
 *   p          : power parameter, finite and > 0 (Sec. 2.1).
 *   out        : device, m results; float (F32_COMP) or double (F64_PLAIN).
 */
idw_status idw_interpolate(idw_handle_t handle, const void *data_xyz, int64_t n,
                           const void *queries_xy, int64_t m, double p, idw_precision prec,
                           void *out, void *stream);

/*
 * As idw_interpolate, and also saves what the adjoint needs:
 *   s0_out  : device, m doubles, nullable: the weight sum S0 = sum_i w_i
 *             (+inf at an exact hit).
 *   hit_out : device, m int32, nullable: the exact-hit index, -1 for an
 *             ordinary query, or -2 where the sums left FP32's range and the
 *             query was recomputed in FP64 (F32_COMP only).
 */
idw_status idw_interpolate_saved(idw_handle_t handle, const void *data_xyz, int64_t n,
                                 const void *queries_xy, int64_t m, double p,
                                 idw_precision prec, void *out, double *s0_out,
                                 int32_t *hit_out, void *stream);

/*
 * idw_interpolate with HOST buffers: copies the inputs to the device,
 * computes, copies the results back and synchronises `stream` before it
 * returns.  Page-locked host memory gives the fastest copies.
 */
idw_status idw_interpolate_host(idw_handle_t handle, const void *data_xyz, int64_t n,
                                const void *queries_xy, int64_t m, double p,
                                idw_precision prec, void *out, void *stream);

/*
 * `count` independent problems (Eq. 1 for each).  The arrays of pointers
 * and sizes are HOST arrays of length `count`; the pointers they hold are
 * device pointers laid out as in idw_interpolate.  IDW_PREC_F32_COMP runs
 * the batch as one persistent launch (chunks of 256 problems);
 * IDW_PREC_F64_PLAIN, the comparison form, runs one stream-ordered
 * single-problem call per instance.  Instances with m_k = 0 are skipped.
 */
idw_status idw_interpolate_batched(idw_handle_t handle, int32_t count,
                                   const void *const *data_xyz, const int64_t *n,
                                   const void *const *queries_xy, const int64_t *m, double p,
                                   idw_precision prec, void *const *out, void *stream);

/*
 * Adjoint of Eq. 1 for L = sum_j g_j Z(q_j) (F32 pair arithmetic with
 * compensated accumulation, FP64 combine).  With S0 = sum_i w_i:
 *   dL/dz_i = sum_j g_j w_ij / S0_j
 *   dL/dx_i = sum_j g_j (p / S0_j) (z_i - Z_j) w_ij (q_j - x_i) / d_ij^2
 *   dL/dq_j = -g_j (p / S0_j) sum_i (z_i - Z_j) w_ij (q_j - x_i) / d_ij^2
 *   dL/dp   = -sum_j g_j / (2 S0_j) sum_i (z_i - Z_j) w_ij ln d_ij^2
 * At an exact hit k of query j only dL/dz_k receives g_j.
 *   data_xyz, queries_xy : device float, as in idw_interpolate.
 *   Z, s0, hit           : device, m each: the outputs of
 *                          idw_interpolate_saved for the same inputs.
 *   grad_out             : device float, m: g_j.
 *   grad_z (n), grad_data_xy (n x 2), grad_query_xy (m x 2) : device float,
 *   grad_p (1) : device double; each nullable (NULL skips that gradient).
 *   The gradient buffers are overwritten, not accumulated into.
 */
idw_status idw_backward(idw_handle_t handle, const float *data_xyz, int64_t n,
                        const float *queries_xy, int64_t m, double p, const float *Z,
                        const double *s0, const int32_t *hit, const float *grad_out,
                        float *grad_z, float *grad_data_xy, float *grad_query_xy,
                        double *grad_p, void *stream);

/* Synchronises `stream`, then reports any pending CUDA error or a bounded
 * in-kernel wait that gave up (IDW_ERR_DEVICE_TIMEOUT), and clears it. */
idw_status idw_sync_status(idw_handle_t handle, void *stream);

/*
 * Host-only launch plan of the single-problem forward pass (no GPU needed).
 * The data are cut into tiles of `records_per_tile` points and the queries
 * into tiles of `queries_per_cta`; one work unit is one (query tile, data
 * tile) pair, and each of `grid` persistent CTAs sweeps one contiguous run
 * of floor(units * g / grid) .. floor(units * (g + 1) / grid) units.  A query
 * tile split across several CTAs is summed by the FP64 combine; each
 * (query tile, CTA) piece owns partial slot (query_tile + cta).
 */
typedef struct {
    int32_t queries_per_thread;
    int32_t threads_per_cta;
    int32_t queries_per_cta;
    int32_t records_per_tile;
    int64_t query_tiles;
    int64_t data_tiles;
    int64_t units;
    int32_t grid;
    int32_t max_pieces_per_query_tile;
    int64_t partial_slots;
    size_t workspace_bytes;
} idw_plan_info;

/* Fills `plan` for `sm_count` SMs holding `ctas_per_sm` CTAs each
 * (0 = the library's default for the precision). */
idw_status idw_plan_forward(int32_t sm_count, int32_t ctas_per_sm, int64_t n, int64_t m,
                            double p, idw_precision prec, idw_plan_info *plan);

/*
 * Handle options (the paper has no counterpart; these tune the sweep).
 *   IDW_OPT_AUTOTUNE            0/1 (default 0).  When 1, the first
 *       FP32-compensated call of each size class (weight form, log2 of the
 *       mean n and m and of the number of pairs) runs every compiled sweep
 *       variant on the call's stream, timed with CUDA events, and keeps the
 *       fastest for that class; calls made while the stream is being
 *       captured use the default instead.  If the environment variable
 *       IDW_AUTOTUNE_CACHE names a file when the handle is created, tuned
 *       classes are read from and written to it (JSON).
 *   IDW_OPT_SWEEP_VARIANT       -1 (default: autotuned if enabled; else, at
 *       p = 2, variant 5 for problems with fewer than 4 work units of 256
 *       points x 2048 queries per resident CTA; else 4 when its 4096-query
 *       tiles pad the queries within 1% of variant 0's; else 0) or:
 *       0: 2048 queries per CTA, 1 of 4 query pairs shares a reciprocal;
 *       1: 2048 queries per CTA, no shared reciprocal;
 *       2: 2048 queries per CTA, 1 of 4 query pairs shares a reciprocal
 *          and a second one on every other data point;
 *       3: 1024 queries per CTA, 1 of 4 query pairs shares a reciprocal;
 *       4: 4096 queries per CTA (one 512-thread CTA per SM), as variant 0;
 *       5: as variant 0 with work units of 64 data points instead of 256
 *          (p = 2 only; other p run variant 0).
 *       The persistent grid always fills the GPU, so the number of pieces
 *       each query tile is split into (the split-N factor) follows from the
 *       query-tile size and the problem sizes.
 *   IDW_OPT_FORCE_GENERAL_POWER 0/1: evaluate p = 2 through the log2/exp2
 *       form used for other p (for comparing the two forms).
 *   IDW_OPT_STAGING_LAYOUT      layout of the staged data tiles: -1 (default)
 *       picks per weight form, 1 at p = 2 and 0 otherwise (the faster of
 *       each on GB300); 0 duplicated pair records (x,x,y,y)+(z,z),
 *       24 B/point; 1 the paper's aligned AoS record (x,y,z,pad),
 *       16 B/point (Sec. 3.3); 2 SoA arrays x, y, z, 12 B/point (Sec. 2.2).
 *       Layouts 1 and 2 build the register pairs with moves.  A forced
 *       layout applies to single FP32 problems with sweep variant 0 (the
 *       layout ablation) and is ignored otherwise.  For IDW_PREC_F64_PLAIN
 *       it selects that form's staging: -1 or 0 the paper's Hybrid layout
 *       ((x,y) pairs beside z, 24 B/point, Sec. 3.5; the default), 1 aligned
 *       (x,y,z,pad) records (32 B/point), 2 SoA (24 B/point); the results
 *       are bit-identical in every layout.
 *   IDW_OPT_VALIDATE_INPUTS     0/1 (default 0).  When 1, every call that
 *                               takes this handle first scans its data,
 *                               queries (and, for idw_backward, grad_out) for
 *                               NaN or infinite values and returns
 *                               IDW_ERR_NOT_FINITE_INPUT, computing nothing,
 *                               if it finds any.  The scan's verdict is read
 *                               back, so a validating call synchronises its
 *                               stream and returns IDW_ERR_UNSUPPORTED while
 *                               the stream is being captured.  Off, inputs are
 *                               not scanned and NaN propagates (Eq. 1 is
 *                               evaluated as given).
 *   IDW_OPT_LOCAL_QUERY_ORDER   0 (default) or 1.  The local forms (radius
 *                               and k-NN, one-shot and prepared index, and
 *                               idw_knn_backward) sort the queries into the
 *                               grid's cells so that neighbouring threads
 *                               read the same data.  1 keeps the caller's
 *                               order instead, which saves that sort when
 *                               the queries already come in spatial order
 *                               (a raster of prediction points) and costs
 *                               locality when they do not.  Results are the
 *                               same either way.  idw_local_backward always
 *                               sorts (its data-side pass finds queries by
 *                               cell).
 *   IDW_OPT_DETERMINISTIC       0 (default) or 1.  idw_knn_backward adds the
 *                               data-side terms (dL/dz, dL/dx) with float
 *                               atomics, whose order, and so the last bits,
 *                               can vary between calls.  1 makes repeated
 *                               calls on the same inputs bit-identical:
 *                               neighbour rows in key order; the
 *                               (point, query) selections sorted by point
 *                               with a stable radix sort, so each point's
 *                               terms are summed in increasing query order;
 *                               dL/dp summed over queries in index order.  It
 *                               needs m k < 2^31 (else IDW_ERR_UNSUPPORTED)
 *                               and about 40 m k more workspace bytes.
 *   IDW_OPT_FMA_LOG2            0 (default) or 1.  The general-power form
 *                               (p != 2, one problem) takes log2 d^2 of one
 *                               pair in 16 from a degree-8 minimax polynomial
 *                               on the FMA pipe instead of the MUFU pipe
 *                               (error at most 1.5u absolute on [1/2, 2] and
 *                               1.5u relative elsewhere, below lg2.approx's).
 *                               It runs sweep variant 4.  Measured slower on
 *                               GB300 than the MUFU path at every fraction
 *                               from 1/16 to 1/4, so it stays off; it exists
 *                               to balance the pipes where that trade wins.
 *   IDW_OPT_KNN_SEARCH          0 (default) or 1.  The k-NN search of
 *                               idw_interpolate_knn and idw_knn_backward: 0
 *                               one thread per query, each growing its own
 *                               square of cells at its own pace; 1 the same
 *                               per-query search with the 32 lanes of a warp
 *                               kept in step (the same step and row order,
 *                               each lane's row runs walked as one stream,
 *                               heap inserts merged by the warp together).
 *                               The selection, and so the result, is the
 *                               same.  1 keeps more lanes busy but spends
 *                               as many instructions on keeping them in
 *                               step, and is slower at k >= 32 and on
 *                               clustered data.  Prepared indexes use 0.
 *   IDW_OPT_LAST_VARIANT        read-only: the variant of the last call.
 *   IDW_OPT_TUNED_CLASSES       read-only: size classes tuned so far.
 * Unknown options or out-of-range values give IDW_ERR_INVALID_ARG.
 */
typedef enum {
    IDW_OPT_AUTOTUNE = 1,
    IDW_OPT_SWEEP_VARIANT = 2,
    IDW_OPT_FORCE_GENERAL_POWER = 3,
    IDW_OPT_LAST_VARIANT = 4,
    IDW_OPT_TUNED_CLASSES = 5,
    IDW_OPT_STAGING_LAYOUT = 6,
    IDW_OPT_VALIDATE_INPUTS = 7,
    IDW_OPT_LOCAL_QUERY_ORDER = 8,
    IDW_OPT_DETERMINISTIC = 9,
    IDW_OPT_FMA_LOG2 = 10,
    IDW_OPT_KNN_SEARCH = 11
} idw_option;

idw_status idw_set_option(idw_handle_t handle, idw_option option, int64_t value);
idw_status idw_get_option(idw_handle_t handle, idw_option option, int64_t *value);

/*
 * Kernel timing (tracing).  While enabled, every forward call records a pair
 * of CUDA events around its all-pairs sweep kernel on the call's stream.
 * idw_profile_read synchronises those events, returns the summed sweep time
 * in milliseconds and the number of sweep launches, and clears the record.
 */
idw_status idw_profile_enable(idw_handle_t handle, int enable);
idw_status idw_profile_read(idw_handle_t handle, double *sweep_ms, int64_t *launches);

/*
 * Failure-detection self-test: launches one CTA that waits, through the same
 * bounded mbarrier wait the sweep kernels use, on a barrier that nothing
 * completes.  After about two seconds the wait gives up and sets the
 * handle's device error word, so the next idw_sync_status() returns
 * IDW_ERR_DEVICE_TIMEOUT while the CUDA context stays usable.
 */
idw_status idw_selftest_bounded_wait(idw_handle_t handle, void *stream);

/*
 * Diagnostic: measures the issue rate of the arithmetic pipes the forward
 * pass uses, in operations per SM per clock (from in-kernel clock counters,
 * so independent of the clock speed).  rates[0..5] receive:
 *   FFMA (fp32), FFMA2 (packed fp32x2, counted as 2 ops), MUFU rcp,
 *   MUFU lg2, MUFU ex2, DFMA (fp64).
 * Synchronous; runs for a few milliseconds on `device`.
 */
idw_status idw_measure_pipe_rates(int device, double rates[6]);

/*
 * Diagnostic: the accuracy of the three MUFU approximations in the weight
 * w = d^-p (Sec. 2.1, Eq. 1), measured exhaustively over every positive fp32
 * input of the range each is used on.  errs[0..3] receive:
 *   errs[0]  max |rcp.approx(x) x - 1| over normal x with normal 1/x;
 *   errs[1]  max |lg2.approx(x) - log2 x| over x in [1/2, 2] (absolute, in
 *            log2 units);
 *   errs[2]  max |ex2.approx(t) / 2^t - 1| over |t| in [2^-30, 126] where
 *            2^t is a normal float;
 *   errs[3]  max |lg2.approx(x) - log2 x| / |log2 x| over every other normal
 *            x (the result's own fp32 rounding included).
 * These are the constants of the FP32 form's worst-case error bound.  The
 * reference values come from the device's FP64 log2 and exp2 (the
 * reciprocal's check r x - 1 is exact in FP64).  Synchronous; about four
 * billion evaluations, well under a second on a GB300.  Errors:
 * IDW_ERR_INVALID_ARG (null errs, bad device), IDW_ERR_CUDA.
 */
idw_status idw_measure_mufu_errors(int device, double errs[4]);

/*
 * Diagnostic of a debug build (the library compiled with -DIDW_DEBUG_CHECKS,
 * e.g. paper_1402_4986_gb300.build.build(debug=True)): the kernels of the
 * local and k-nearest-neighbour forms check every gather, scatter, cell,
 * heap and output index; a failed check sets its site's bit in a device word
 * and skips the access (nothing traps).  This call writes that word for
 * `device` to *sites and clears it.  Bits: 0 cell index, 1 sorted-data
 * gather, 2 scatter position, 3 output row, 4 heap slot or data index,
 * 5 occupancy-block index, 6 hit index, 7 summed-area-table entry.  A
 * release build returns
 * IDW_ERR_UNSUPPORTED (and *sites = 0).  Synchronous.
 */
idw_status idw_debug_check_failures(int device, uint32_t *sites);

/*
 * The paper's own GPU designs, as measured baselines (not the fast path):
 *   IDW_PAPER_NAIVE : one thread per prediction point reading every data
 *                     point from global memory (Sec. 3; data read m times);
 *   IDW_PAPER_TILED : one thread per prediction point, each block staging
 *                     256 data points in shared memory at a time (Sec. 4.2;
 *                     data read m / 256 times).
 * in the paper's data layouts (Sec. 2.2, 3.2-3.5):
 *   IDW_LAYOUT_SOA    : x[n], y[n], z[n]
 *   IDW_LAYOUT_AOS    : unaligned rows (x, y, z) -- the caller's rows as they are
 *   IDW_LAYOUT_AOAS   : aligned records (x, y, z, pad) of 16 (float) or
 *                       32 (double) bytes
 *   IDW_LAYOUT_HYBRID : (x, y) pairs beside z[n] (the paper uses it for double)
 * They sum plainly (no compensation) in the precision given: data, queries
 * and out are float for IDW_PREC_F32_COMP (here: plain FP32) and double for
 * IDW_PREC_F64_PLAIN.  p = 2 is 1/d^2, other p use pow().  A query that
 * coincides with a data point takes the z of the lowest such index.  Other
 * layouts than AoS are staged into the handle's workspace first.
 * Arguments, ownership and errors as in idw_interpolate.
 */
typedef enum { IDW_PAPER_NAIVE = 0, IDW_PAPER_TILED = 1 } idw_paper_kernel;
typedef enum {
    IDW_LAYOUT_SOA = 0,
    IDW_LAYOUT_AOS = 1,
    IDW_LAYOUT_AOAS = 2,
    IDW_LAYOUT_HYBRID = 3
} idw_paper_layout;

idw_status idw_paper_interpolate(idw_handle_t handle, idw_paper_kernel kernel,
                                 idw_paper_layout layout, const void *data_xyz, int64_t n,
                                 const void *queries_xy, int64_t m, double p, idw_precision prec,
                                 void *out, void *stream);

/*
 * Allocation-free FP32-compensated interpolation.  The paper has no
 * counterpart; this exists for callers that cannot allocate device memory:
 * a host application that owns the whole device-memory budget and does not
 * let its plug-ins allocate, or a latency-critical loop that cannot afford
 * cudaMalloc/cudaFree (both synchronise the device).  Such callers cannot
 * create a handle either, because idw_create allocates, so this call takes
 * none.  It computes what idw_interpolate computes with IDW_PREC_F32_COMP,
 * with the same kernels, on the CURRENT device.
 *
 *   data_xyz, queries_xy, out : device float arrays laid out as in
 *                               idw_interpolate (caller-owned, 4-byte aligned).
 *   stream                    : cudaStream_t as void* (NULL = legacy stream).
 *
 * Scratch: instead of a workspace it uses one fixed 32 MiB device array
 * that every GPU loading the library holds until the process exits.  It
 * never calls cudaMalloc, cudaFree or any allocating routine.  A problem
 * whose scratch (about 24 bytes per data point, 4 bytes per query, plus
 * 32 KiB per query tile and per persistent CTA) exceeds the array is
 * rejected with IDW_ERR_WORKSPACE before anything is launched; on a 152-SM
 * GB300, n = m = 262144 fits.
 *
 * It plans the launch as idw_interpolate does on a handle without tuning
 * options: the same default sweep variant for the size and weight form.
 *
 * The first call on a device sets that device up (it looks up the array's
 * device address, clears its control words and waits for the clear), so make
 * that first call before any stream capture.  Every call shares the one array
 * and it keeps the last call's contents; each call clears, on its stream,
 * what its kernels need to start at zero.  Calls whose work overlaps on the
 * GPU (different streams, or concurrent host threads) race on the array:
 * order them on one stream.  A sweep whose bounded wait gives up (see
 * idw_selftest_bounded_wait) leaves that call's output invalid and sets a
 * sticky error bit in the shared control words; idw_noalloc_sync_status
 * reports and clears it.  Returns IDW_ERR_INVALID_ARG, IDW_ERR_ALIGNMENT,
 * IDW_ERR_UNSUPPORTED (not compute capability 10.3), IDW_ERR_WORKSPACE (too
 * large) or IDW_ERR_CUDA; the kernels run asynchronously after it returns.
 */
idw_status idw_interpolate_noalloc(const float *data_xyz, int64_t n, const float *queries_xy,
                                   int64_t m, double p, float *out, void *stream);

/*
 * Device-side status of the allocation-free calls on the current device (the
 * paper has no counterpart; see idw_interpolate_noalloc): waits for `stream`
 * (cudaStream_t as void*), reads the sticky error bits of the shared control
 * words, clears them, and returns IDW_ERR_DEVICE_TIMEOUT if a bounded wait
 * gave up since the last check, else IDW_OK (IDW_ERR_CUDA on a CUDA error).
 * It allocates nothing; it synchronises, so call it outside stream capture.
 */
idw_status idw_noalloc_sync_status(void *stream);

/*
 * The failure-detection self-test of idw_selftest_bounded_wait, reporting
 * into the allocation-free path's shared control words instead of a
 * handle's: after about two seconds the next idw_noalloc_sync_status
 * returns IDW_ERR_DEVICE_TIMEOUT.  Allocates nothing.
 */
idw_status idw_noalloc_selftest_bounded_wait(void *stream);

/*
 * Local (radius-limited) Shepard interpolation.  The paper computes the
 * global form of Eq. 1 and names the local form, which uses only the data
 * points near each prediction point, among the related work (Sec. 1).
 * Here Z(q) is Eq. 1 over the data points within distance `radius` of q:
 *
 *   member i of q  iff  fl32(fmaf(dy, dy, fl32(dx * dx))) < fl32(radius^2),
 *                       dx = fl32(qx - x_i), dy = fl32(qy - y_i),
 *
 * decided in FP32 on the caller's coordinates (so a point at distance R
 * exactly, or within FP32 rounding of it, is in or out as that expression
 * says).  Weights are d^-p in FP32 and summed in FP64 per query.  A query
 * that coincides with a data point takes the z of the lowest such index
 * (count -1); a query with no member gets NaN (count 0).  Data points with a
 * non-finite coordinate are ignored; a query with one gets NaN.
 *
 *   data_xyz, queries_xy, out : device float arrays as in idw_interpolate.
 *   radius                    : R > 0 (+inf gives the global form).
 *   count_out                 : NULL, or device int32[m] receiving the number
 *                               of members of each query (-1 at a hit).
 *
 * Method, all on `stream` without host synchronisation (so the call can be
 * captured into a CUDA graph): the bounding box of the data; a uniform grid
 * of cells about R/2 wide (at most 2048 per axis and one cell per two data
 * points), planned by one device thread; a counting sort of the data and of
 * the queries into the cells; then one thread per query, in cell order,
 * walks the rows of cells its disc of radius R reaches.  Weights are summed
 * as compensated FP32 pairs; a query whose sums leave FP32's range is
 * redone in FP64.  Scatter positions come from atomics, so candidates may be
 * summed in a different order from call to call: results can differ in the
 * last bit.
 * Workspace (the handle's): 16 bytes per data point, 16 per query and 16 per
 * cell, for at most min(2^22, max(1024, n/2)) cells.  Errors as in
 * idw_interpolate, plus IDW_ERR_INVALID_ARG for radius <= 0 or NaN; the
 * kernels run asynchronously after it returns.
 */
idw_status idw_interpolate_local(idw_handle_t handle, const float *data_xyz, int64_t n,
                                 const float *queries_xy, int64_t m, double p, double radius,
                                 float *out, int32_t *count_out, void *stream);

/*
 * Modified Shepard interpolation: the radius form's members (the same FP32
 * test as idw_interpolate_local) with Franke and Nielson's local weights
 *
 *     w_i = ((R - d_i) / (R d_i))^p = (1/d_i - 1/R)^p,
 *
 * which fall to 0 continuously as d_i reaches R, so Z has no jump when a
 * point crosses the radius (the plain radius form's weights d^-p do).  p = 2
 * is the classic choice.  R = +inf gives d^-p, the global form.  The base
 * 1/d - 1/R is taken from the FP32 reciprocal square root and clamped at 0;
 * hits, NaN and the FP64 pass are as in idw_interpolate_local (an FP64
 * query with no member of positive weight gets NaN).  Arguments, counts,
 * workspace, errors and the method are those of idw_interpolate_local.
 */
idw_status idw_interpolate_modified(idw_handle_t handle, const float *data_xyz, int64_t n,
                                    const float *queries_xy, int64_t m, double p, double radius,
                                    float *out, int32_t *count_out, void *stream);

/*
 * k-nearest-neighbour Shepard interpolation, the other local form of the
 * related work the paper cites (Sec. 1): Z(q) is Eq. 1 over the k finite
 * data points nearest to q.  Nearness is the key (d2, index) with
 *
 *   d2 = fl32(fmaf(dy, dy, fl32(dx * dx))),  dx = fl32(qx - x_i), dy = fl32(qy - y_i),
 *
 * ranked ascending, so exact ties go to the lower data index and the
 * selection is one definite set.  Weights are d^-p from the selected keys
 * (FP32, summed as compensated pairs; FP64 where the sums leave FP32's
 * range).  A query that coincides with a data point takes the z of the
 * lowest such index (the selection is still reported).  Fewer than k finite
 * points: all of them.  Non-finite data points are ignored; a non-finite
 * query gets NaN and selects nothing.
 *
 *   data_xyz, queries_xy, out : device float arrays as in idw_interpolate.
 *   k                         : 1 <= k <= 64.
 *   nbr_out                   : NULL, or device int32[m * k]: row j holds the
 *                               selected data indices in key order, -1 padded.
 *   kd2_out                   : NULL, or device float[m]: the k-th (largest
 *                               selected) key's d2, NaN when nothing is selected.
 *
 * Method, on `stream` without host synchronisation (graph-capturable): the
 * grid build of idw_interpolate_local with cells sized for k points at the
 * data's mean density, then one thread per query (in cell order) grows a
 * square of cells around the grid cell nearest to it, keeping the k best
 * keys in shared memory.  Band sizes come from a summed-area table of the
 * cells; once k keys are held, cells whose points provably lie beyond the
 * k-th key are skipped; the search stops once the k-th key is below a
 * conservative FP32 lower bound on the key of any point not yet seen.
 * Workspace as idw_interpolate_local.  Errors as in idw_interpolate, plus
 * IDW_ERR_INVALID_ARG for k outside [1, 64].
 */
idw_status idw_interpolate_knn(idw_handle_t handle, const float *data_xyz, int64_t n,
                               const float *queries_xy, int64_t m, double p, int32_t k,
                               float *out, int32_t *nbr_out, float *kd2_out, void *stream);

/*
 * Gradients of the local (radius) form: for L = sum_j grad_out[j] Z(q_j),
 * with Z from idw_interpolate_local at the same radius, writes
 *   grad_z[i]        = dL/dz_i                (n floats),
 *   grad_data_xy[i]  = dL/d(x_i, y_i)         (n x 2 floats),
 *   grad_query_xy[j] = dL/d(qx_j, qy_j)       (m x 2 floats),
 *   grad_p[0]        = dL/dp                  (one double).
 * Each may be NULL (not computed).  Each query's membership set (the FP32
 * test of idw_interpolate_local) is held fixed: it is piecewise constant in
 * every input, so each derivative is that of the global form (see
 * idw_backward) summed over the members.  A query with an exact hit passes
 * grad_out[j] to dL/dz of its point (the lowest coincident index) and
 * nothing else; a query without members (Z = NaN) contributes nothing, and
 * non-finite data points get zero gradients.
 *
 * Method, on `stream` without host synchronisation: the grid build of
 * idw_interpolate_local, then one thread per query (cell order) finds its
 * members and computes Z, S0, dL/dq and its share of dL/dp with weights
 * scaled by the members' smallest d^2 (FP32; FP64 where the FP32 values
 * leave their range), and one thread per data point walks the queries whose
 * disc reaches it with the same FP32 membership test and sums dL/dz and
 * dL/dx in registers (one write per point: deterministic, no atomics).
 * dL/dp is a sum of per-warp FP64 atomics, so its last bits may vary.
 * Workspace: that of idw_interpolate_local plus 40 bytes per query.
 * Errors as in idw_interpolate_local; grad_p must be 8-byte aligned.
 */
idw_status idw_local_backward(idw_handle_t handle, const float *data_xyz, int64_t n,
                              const float *queries_xy, int64_t m, double p, double radius,
                              const float *grad_out, float *grad_z, float *grad_data_xy,
                              float *grad_query_xy, double *grad_p, void *stream);

/*
 * Gradients of modified Shepard (idw_interpolate_modified): as
 * idw_local_backward, with each pair's terms those of the weights
 * w = t^p, t = 1/d - 1/R:  dw/dq = -p w (q - x) / (t d^3) = -dw/dx and
 * dw/dp = w ln t.  Members of zero weight contribute nothing.
 */
idw_status idw_modified_backward(idw_handle_t handle, const float *data_xyz, int64_t n,
                                 const float *queries_xy, int64_t m, double p, double radius,
                                 const float *grad_out, float *grad_z, float *grad_data_xy,
                                 float *grad_query_xy, double *grad_p, void *stream);

/*
 * Gradients of the k-nearest-neighbour form: as idw_local_backward, for Z
 * from idw_interpolate_knn with the same k (1 <= k <= 64).  Each query's
 * selection (its k smallest keys) is held fixed, so each derivative is the
 * global one summed over the selected points; a hit passes grad_out[j] to
 * dL/dz of the lowest coincident index, a query that selects nothing
 * contributes nothing.  Method: the search of idw_interpolate_knn with its
 * neighbour lists kept in the workspace, then one thread per query (cell
 * order) computes dL/dq and its dL/dp share and adds its data-side terms
 * with one 16-byte vector atomic per (query, neighbour) pair into a
 * per-point accumulator (their order, and so the last bits of grad_z and
 * grad_data_xy, can vary between calls).  FP64 where the FP32 values leave
 * their range.  Workspace: that of idw_interpolate_knn plus 4 (k + 2)
 * bytes per query and 16 per data point.  Errors as in idw_interpolate_knn;
 * grad_data_xy must be 8-byte aligned.
 */
idw_status idw_knn_backward(idw_handle_t handle, const float *data_xyz, int64_t n,
                            const float *queries_xy, int64_t m, double p, int32_t k,
                            const float *grad_out, float *grad_z, float *grad_data_xy,
                            float *grad_query_xy, double *grad_p, void *stream);

/*
 * Prepared index of the local forms: the data side of idw_interpolate_local
 * or idw_interpolate_knn (bounding box, grid plan, counting sort of the
 * data, and for k-NN the cell-count tables) built once, then queried by any
 * number of calls that each sort only their own queries.  Results are those
 * of the one-shot calls on the same data: the same members and neighbour
 * lists, values within the last bits (candidate order within a cell may
 * differ).
 *
 * idw_local_index_create builds an index over `data_xyz` (device float
 * n x 3, as in idw_interpolate) for exactly one form:
 *   radius > 0 and k == 0      : a radius index (cells for radius R; R may
 *                                be +inf, which gives the global form);
 *   radius == 0, 1 <= k <= 64  : a k-NN index (cells for k neighbours).
 * The index copies what it needs (sorted records; for k-NN also the data),
 * so `data_xyz` may be freed or changed once the build has run.  It owns
 * device memory on the handle's device (about 16 bytes per data point and
 * 8 per cell; k-NN adds 12 per data point, 4 per cell and 264 KB), allocated
 * here (cudaMalloc, so the call cannot be captured).  The build is enqueued
 * on `stream`: order later queries on other streams after it.  With
 * IDW_OPT_VALIDATE_INPUTS set the data are scanned first.  Errors:
 * IDW_ERR_INVALID_ARG (null handle, index or data, n outside [1, 2^31),
 * a bad radius / k combination), IDW_ERR_ALIGNMENT, IDW_ERR_WORKSPACE (the
 * allocation failed), IDW_ERR_NOT_FINITE_INPUT, IDW_ERR_CUDA.
 *
 * idw_local_index_interpolate is idw_interpolate_local on a radius index,
 * for any 0 < radius <= the build radius (a smaller radius still uses the
 * build's cells); idw_local_index_modified is idw_interpolate_modified
 * there.  idw_local_index_knn is idw_interpolate_knn on a k-NN
 * index, for any 1 <= k <= 64.  Outputs, NaN and hit rules are those of
 * the one-shot calls.  Both run on `stream` without host synchronisation
 * (graph-capturable once the handle's workspace has grown) and take the
 * handle's workspace: 16 bytes per query and 8 per cell.  The handle must be
 * on the index's device; calling the wrong form's query on an index, a
 * radius above the build radius or k outside [1, 64] gives
 * IDW_ERR_INVALID_ARG.  Several handles (one per stream) may query one
 * index at the same time: queries only read it.
 *
 * idw_local_index_destroy frees the index (cudaFree: the device is
 * synchronised first).  Destroying NULL returns IDW_ERR_INVALID_ARG.
 */
typedef struct idw_local_index_s *idw_local_index_t;

idw_status idw_local_index_create(idw_handle_t handle, const float *data_xyz, int64_t n,
                                  double radius, int32_t k, idw_local_index_t *index,
                                  void *stream);
idw_status idw_local_index_interpolate(idw_handle_t handle, idw_local_index_t index,
                                       const float *queries_xy, int64_t m, double p,
                                       double radius, float *out, int32_t *count_out,
                                       void *stream);
idw_status idw_local_index_modified(idw_handle_t handle, idw_local_index_t index,
                                    const float *queries_xy, int64_t m, double p, double radius,
                                    float *out, int32_t *count_out, void *stream);
idw_status idw_local_index_knn(idw_handle_t handle, idw_local_index_t index,
                               const float *queries_xy, int64_t m, double p, int32_t k,
                               float *out, int32_t *nbr_out, float *kd2_out, void *stream);
idw_status idw_local_index_destroy(idw_local_index_t index);

#ifdef __cplusplus
}
#endif

#endif /* IDW_GB300_H */
