/*
 * qai.h -- C ABI of libqai, GB300-native quantization-aware interpolation.
 *
 * The library implements the artifact-mitigation method of Jiao et al.,
 * "Mitigating Artifacts in Pre-quantization Based Scientific Data Compressors
 * with Quantization-aware Interpolation" (Sec. VI, Algorithm 4): given the
 * int32 pre-quantization indices q of a field (Eq. 1, q = round(x / 2 eps))
 * and the absolute error bound eps, it returns the compensated field
 * D'' = D' + C with D' = 2 q eps, in fp32. All work runs in hand-written
 * CUDA kernels for sm_103a; the host code only validates and launches.
 *
 * Conventions shared by every entry point:
 *  - Fields are dense, C order (slowest axis first), rank 1..3. Extent-1 axes
 *    are squeezed before the stencils (a 1 x ny x nx field is 2-D).
 *  - Supported extents after squeezing: rank 1: n <= 32768; rank 2 and 3:
 *    x (contiguous) <= 16383, y and z <= 4096; N = prod(dims) < 2^31.
 *    Larger shapes return QAI_ERR_SHAPE.
 *  - Pointers named d_* are device memory, h_* host memory; all of it is owned
 *    by the caller and never freed by the library. Outputs must not alias
 *    inputs or each other.
 *  - Calls are asynchronous and stream-ordered on `stream` (0 = legacy
 *    default stream). The returned status covers argument errors and launch
 *    errors; faults inside kernels surface on a later synchronisation.
 *  - On any error nothing is launched, and qai_last_error() returns a
 *    one-line description (per host thread).
 */
#ifndef QAI_H
#define QAI_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QAI_OK = 0,
    QAI_ERR_INVALID_ARG = 1,  /* NULL pointer, bad eps/eta/p/rule, small workspace */
    QAI_ERR_SHAPE = 2,        /* rank or extents outside the supported range       */
    QAI_ERR_RANGE = 3,        /* reserved                                          */
    QAI_ERR_CUDA = 4,         /* a CUDA runtime call or launch failed              */
    QAI_ERR_OOM = 5,          /* internal workspace allocation failed              */
    QAI_ERR_TIMEOUT = 6,      /* a bounded device-side wait ran out                */
    QAI_ERR_INTERNAL = 7
} qai_status;

/* Method parameters. Defaults (qai_default_params) reproduce the paper. */
typedef struct {
    double eta;              /* compensation factor at boundaries, Sec. VI step E
                                (paper: 0.9); finite, >= 0                         */
    double idw_power;        /* exponent p of the inverse-distance weights:
                                w = (1/k1^p) / (1/k1^p + 1/k2^p); paper: 1; > 0    */
    int32_t grad_threshold;  /* Algorithm 2 fast-varying test on the central
                                difference (q[+1]-q[-1])/2 >= 1, as the integer
                                |q[+1]-q[-1]| >= grad_threshold; default 2, >= 1  */
    int32_t sign_rule;       /* Algorithm 2 boundary sign: 0 = sgn of the sum of
                                (q_nb - q) over the axis neighbours (default);
                                1 = sgn(q_nb - q) of the first differing neighbour
                                in the order z-, z+, y-, y+, x-, x+                */
    int32_t b2_rule;         /* Algorithm 3 GetBoundary(S): 0 = a neighbour with
                                the same q and a different S (default);
                                1 = any neighbour with a different S               */
    uint32_t flags;          /* 0, or QAI_FLAG_OUTPUT_C, optionally with one route
                                selection bit below                                */
} qai_params;

#define QAI_FLAG_OUTPUT_C 1u  /* write the compensation C (step E) instead of D''  */

/* Route selection for rank-2 and rank-3 plain calls. These bits exist for
 * testing and measurement: every route computes the same Dist1, I1, S and
 * Dist2 where they reach the output, so the output bits do not depend on them
 * (qai_route_counts reports which route ran). At most one QAI_FLAG_EDT2_* bit.
 *  QAI_FLAG_EDT2_DENSE       the dense second EDT over the whole field (the
 *                            separable passes of Algorithm 1), no route
 *  QAI_FLAG_EDT2_HANDOVER    the route's kernels run and hand every field
 *                            over to the dense second EDT
 *  QAI_FLAG_EDT2_LIST        no shell search: every point that needs Dist2
 *                            takes the search over the listed B2 sites
 *  QAI_FLAG_EDT1_SEPARABLE   the first EDT by the separable passes alone,
 *                            without the bounded nearest-site search first */
#define QAI_FLAG_EDT2_DENSE 0x10u
#define QAI_FLAG_EDT2_HANDOVER 0x20u
#define QAI_FLAG_EDT2_LIST 0x40u
#define QAI_FLAG_EDT1_SEPARABLE 0x80u

/* Optional per-step outputs of Algorithm 4 (debug and parity checking).
 * Each pointer is a device array of N elements, or NULL to skip it.
 * Distances are squared Euclidean distances in grid units; a point that no
 * boundary reaches gets INT32_MAX. idx1 is the linear index of the nearest
 * quantization boundary point, the smallest linear index among equally near
 * ones, -1 if the field has no boundary; it needs the workspace sized with
 * QAI_WS_INDEX. */
typedef struct {
    uint8_t* b1;     /* quantization boundary map B1 (Algorithm 2)          */
    int8_t* sb;      /* boundary sign map S_B in {-1,0,1} (Algorithm 2)     */
    int32_t* dist1;  /* Dist1, squared distance to B1 (step B)              */
    int32_t* idx1;   /* I1, nearest boundary point (step B)                 */
    int8_t* s;       /* propagated sign map S (Algorithm 3)                 */
    uint8_t* b2;     /* sign-flipping boundary map B2 (Algorithm 3)         */
    int32_t* dist2;  /* Dist2, squared distance to B2 (step D)              */
} qai_debug_out;

#define QAI_WS_INDEX 1u   /* workspace_size flag: room to carry idx1          */

/* Fills *p with the paper's defaults: eta 0.9, p 1, threshold 2, rules 0. */
void qai_default_params(qai_params* p);

/* Bytes of device workspace qai_mitigate needs for this shape. flags: 0, or
 * QAI_WS_INDEX when debug idx1 output is wanted. Returns QAI_ERR_SHAPE for an
 * unsupported shape. */
qai_status qai_workspace_size(int rank, const int64_t* dims, uint32_t flags, size_t* bytes);

/* Algorithm 4 (Sec. VI, steps A-E) on a device-resident field.
 *  d_q      int32[N] pre-quantization indices (Eq. 1), device
 *  d_out    float[N] compensated field D'' = 2 q eps + C, device
 *  rank, dims  rank 1..3 and its extents, slowest first (host array)
 *  eb       absolute error bound eps > 0, finite
 *  params   NULL for the defaults
 *  d_ws, ws_bytes  device workspace of at least qai_workspace_size() bytes,
 *           256-byte aligned; d_ws = NULL makes the call allocate and free it
 *           stream-ordered (cudaMallocAsync / cudaFreeAsync)
 *  stream   CUDA stream of every launch
 *  dbg      NULL, or the per-step outputs wanted
 * Error bound: |x - D''| <= (1 + eta) eps wherever |x - 2 q eps| <= eps. */
qai_status qai_mitigate(const int32_t* d_q, float* d_out, int rank, const int64_t* dims,
                        double eb, const qai_params* params, void* d_ws, size_t ws_bytes,
                        cudaStream_t stream, const qai_debug_out* dbg);

/* How the last plain qai_mitigate call on this workspace computed the two
 * EDTs (steps B and D) of a rank-2 or rank-3 field. The first: where B1 is
 * dense, every point's nearest B1 point is a few cells away, and a bounded
 * exact search finds it (in order of distance, then linear index: the tie
 * rule of Algorithm 1's passes); the separable passes run when it cannot.
 * The second: step E needs Dist2 only at the points with S != 0 off B1
 * (elsewhere C = 0, or the weight is 1: Sec. VI-E), so a plain call finds
 * their nearest B2 site by an exact shell search, lists the B2 sites and
 * searches them all for the points the shell search leaves, and runs the
 * dense second EDT over the whole field only when one of those lists
 * overflows. Outputs are the same bits on every route.
 *  d_ws     the workspace of that call (device), after the call completed
 *  counts   host int32[6]: points with S != 0 off B1; of them, those left to
 *           the list search; B2 sites listed (0 if the list was not needed);
 *           1 if the dense second EDT ran, else 0; B1 points with S != 0
 *           (-1 if there were too many to list); 1 if the separable first
 *           EDT ran because some point had no B1 point within squared
 *           distance 8 (the first EDT's bounded search), else 0
 * Synchronises `stream`. Returns QAI_ERR_SHAPE for rank-1 fields (no such
 * route) or an unsupported shape, QAI_ERR_INVALID_ARG for NULL pointers, and
 * QAI_ERR_TIMEOUT (with the counts filled) when a bounded wait inside that
 * call's kernels ran out, so that its output is not valid. */
qai_status qai_route_counts(const void* d_ws, int rank, const int64_t* dims, int32_t* counts,
                            cudaStream_t stream);

/* Bytes of device workspace qai_mitigate_host needs: the device copies of q
 * and D'' plus qai_workspace_size(rank, dims, 0). */
qai_status qai_workspace_size_host(int rank, const int64_t* dims, size_t* bytes);

/* qai_mitigate end to end from host memory: copies h_q (int32[N], host) to the
 * device, runs Algorithm 4, and copies D'' back into h_out (float[N], host),
 * all on `stream`. Pinned host buffers make the copies asynchronous; the call
 * returns before they finish, so synchronise `stream` before reading h_out.
 * d_ws (>= qai_workspace_size_host bytes) is required. */
qai_status qai_mitigate_host(const int32_t* h_q, float* h_out, int rank, const int64_t* dims,
                             double eb, const qai_params* params, void* d_ws, size_t ws_bytes,
                             cudaStream_t stream);

/* ---- Adjoint of step E (no counterpart in the paper) ----------------------
 * With the EDT assignment held fixed (Dist1, Dist2 and S as Algorithm 4
 * computes them), D'' = D' + S w eta eps is linear in D' and eta; for a loss
 * L with G = dL/dD'':
 *   dL/dD' = G,  dL/deta = sum G S w eps,
 *   dL/dp  = sum G S eta eps w (1 - w) (ln k2 - ln k1),  w = 1/(1 + (k1/k2)^p)
 * (dw/dp = 0 where k1 = 0, k2 = 0 or no B2 exists). Every term vanishes
 * where S = 0. Stored mode keeps S, Dist1 and Dist2 from the forward (9 bytes
 * per point; for 2-D and 3-D fields Dist1 and Dist2 only where S != 0 off B1,
 * 0 elsewhere -- where S != 0 on B1, Dist1 = 0 and the weight is 1); recompute
 * mode re-runs the forward in the backward call and keeps nothing in between
 * (a plain forward for 2-D and 3-D fields, Dist2 recorded where it is
 * computed). */

/* Bytes of the saved state of the stored mode (256-byte aligned buffer). */
qai_status qai_saved_size(int rank, const int64_t* dims, size_t* bytes);

/* qai_mitigate that also fills d_saved (qai_saved_size bytes, device,
 * 256-byte aligned) with the saved state of qai_mitigate_backward (above). */
qai_status qai_mitigate_save(const int32_t* d_q, float* d_out, int rank, const int64_t* dims,
                             double eb, const qai_params* params, void* d_saved, void* d_ws,
                             size_t ws_bytes, cudaStream_t stream);

/* D' = 2 q eps (Eq. 1, the dequantized field) in fp32, computed as every
 * kernel of the library computes it: float(q) * float(2 eps), rounded once.
 *  d_q   int32[n] indices, device;  d_out  float[n], device;  n >= 0. */
qai_status qai_dequantize(const int32_t* d_q, float* d_out, int64_t n, double eb, cudaStream_t stream);

/* Algorithm 4 with the dequantized field given: d_out = d_dprime + C, C the
 * compensation of step E computed from d_q (the differentiable form, where
 * D' is an independent input: dL/dD' = dL/dD''). d_dprime is float[N],
 * device; with d_dprime = 2 q eps the result equals qai_mitigate's to one
 * fp32 rounding. d_saved: NULL, or the stored-mode saved state to fill, as
 * qai_mitigate_save. Other arguments as qai_mitigate_save. */
qai_status qai_mitigate_add(const int32_t* d_q, const float* d_dprime, float* d_out, int rank,
                            const int64_t* dims, double eb, const qai_params* params, void* d_saved,
                            void* d_ws, size_t ws_bytes, cudaStream_t stream);

/* Device workspace of qai_mitigate_backward: 32 KiB of block partial sums
 * (stored mode); with recompute != 0, the partial sums (at least 32 KiB) plus
 * the forward workspace and two more 4-byte field-sized arrays (the forward's
 * D'' and Dist2). */
qai_status qai_workspace_size_backward(int rank, const int64_t* dims, int recompute, size_t* bytes);

/* Adjoint of step E.
 *  d_q            int32[N] indices the forward ran on, device
 *  d_grad_out     float[N] G = dL/dD'', device
 *  d_grad_dprime  float[N] receives dL/dD' (= G), device, or NULL
 *  d_grad_params  double[2] receives (dL/deta, dL/dp), device
 *  eb, params     as given to the forward
 *  d_saved        the forward's saved state (stored mode), or NULL to
 *                 recompute it from d_q
 *  d_ws, ws_bytes qai_workspace_size_backward(rank, dims, d_saved == NULL)
 *                 bytes, device, 256-byte aligned
 * Sums run in fp32 with compensation, folded into FP64 in a fixed order (the
 * same result on every run of a mode; the two modes group the terms
 * differently, so they agree to rounding, not bit for bit). Asynchronous on
 * `stream` like every other call. */
qai_status qai_mitigate_backward(const int32_t* d_q, const float* d_grad_out, float* d_grad_dprime,
                                 double* d_grad_params, int rank, const int64_t* dims, double eb,
                                 const qai_params* params, const void* d_saved, void* d_ws,
                                 size_t ws_bytes, cudaStream_t stream);

/* ---- Batched form (no counterpart in the paper) ---------------------------
 * n independent fields in one call: field i is d_q[i] -> d_out[i] (device
 * buffers), rank ranks[i], extents dims[3*i .. 3*i + ranks[i]) (slowest first),
 * bound eb[i]; params are shared. Rank-2 and rank-3 fields run as persistent
 * grouped launches: each kernel of a plain qai_mitigate call's sequence runs
 * once for all of them (fields with the same tile shape share a launch; up to
 * 64 fields a launch), its resident CTAs taking (field, block) work items
 * from a device cursor in queue order; a field whose fallback flag is clear
 * adds no items to the fallback kernels. Rank-1 fields run as two grouped
 * kernels over all of them. The whole launch sequence (argument tables copied
 * in from pinned host memory, cursors and route counters cleared, the
 * grouped kernels) is captured into a CUDA graph the first time a batch is
 * seen (keyed by every pointer, extent and parameter) and replayed
 * afterwards: a repeated batch is one graph launch on `stream`. With a
 * QAI_FLAG_EDT2_* or QAI_FLAG_EDT1_SEPARABLE bit, or when `stream` is already
 * capturing (the launches are then recorded into the caller's graph), rank-2
 * and rank-3 fields run their own plain sequences on streams forked from
 * `stream`. Results equal those of n qai_mitigate calls. The queue order and
 * tile shapes (and, per field, the stream count) come from
 * qai_autotune_batched when it has seen a batch of the same shapes. */

/* Device workspace of a batch: the fields' workspaces and a header for the
 * grouped launches (argument tables, cursors, route counters). */
qai_status qai_workspace_size_batched(int n, const int32_t* ranks, const int64_t* dims, size_t* bytes);

qai_status qai_mitigate_batched(int n, const int32_t* const* d_q, float* const* d_out,
                                const int32_t* ranks, const int64_t* dims, const double* eb,
                                const qai_params* params, void* d_ws, size_t ws_bytes,
                                cudaStream_t stream);

/* Autotuner result for the fields of one rank. */
typedef struct {
    int32_t rank;             /* 1, 2 or 3 (0: no field of this rank)                 */
    int32_t fields;
    int32_t streams;          /* per-field form: streams the fields are dealt onto
                                 (rank 1: 1); grouped form: 0                          */
    int32_t order;            /* 0: fields as given, 1: largest field first           */
    float ms;                 /* time of the group's launches with this choice (the
                                 grouped form: of ranks 2 and 3 together)              */
    int32_t grouped;          /* 1: persistent grouped launches                       */
    int32_t tile_w;           /* column-pass tile width (0: the plain call's tiles)   */
    int32_t rows_per_band;    /* column-pass band height (0: the plain call's tiles)  */
    int32_t points_per_block; /* points per work item of the grid-stride kernels      */
    int32_t launches;         /* kernel launches of the grouped form per batch        */
} qai_batch_choice;

/* Times candidates on this batch itself (running its launches several times;
 * the outputs hold a correct result afterwards) and keeps the fastest for
 * later qai_mitigate_batched calls with the same shapes: for the grouped form
 * (ranks 2 and 3 together), greedily the queue order, then the points per
 * work item (2^14 .. 2^18), then the column tiles (band height x largest
 * width); for the per-field form, the stream count (1, 2, 4, 8) and field
 * order per rank. Reports them in choices[0..2] (ranks 1..3) when non-NULL.
 * Synchronises `stream`. */
qai_status qai_autotune_batched(int n, const int32_t* const* d_q, float* const* d_out,
                                const int32_t* ranks, const int64_t* dims, const double* eb,
                                const qai_params* params, void* d_ws, size_t ws_bytes,
                                cudaStream_t stream, qai_batch_choice* choices);

/* ---- Quality metrics (Sec. III-B, Eq. 3 and Eq. 4) -------------------------
 * How close a field y (D' or D'') is to the original x. Readings: both fields
 * are normalised by the range of x before SSIM (v' = (v - min x) / range x;
 * a constant x is only shifted), since Eq. 3's c1 = 1e-4 and c2 = 9e-4 assume
 * data in [0, 1]; "sample" variances and covariance divide the centred sums
 * by n - 1 (n = points of a window); on every axis (extent-1 axes dropped) a
 * window spans m = min(window, extent) points and starts at 0, stride,
 * 2 stride, ... while it fits; the field's SSIM is the mean over all windows.
 * The paper's setting is window 7, stride 2. */
typedef struct {
    double x_min, x_max; /* range of the original field */
    double mse;          /* mean of (x - y)^2 over all points */
    double psnr;         /* Eq. 4 in dB: 20 log10((x_max - x_min) / sqrt(mse));
                            +inf when mse = 0, -inf when x is constant */
    double ssim;         /* Eq. 3 averaged over the windows */
    int64_t windows;     /* number of windows */
} qai_quality_out;

/* Device workspace of qai_quality for this shape, window and stride. */
qai_status qai_workspace_size_quality(int rank, const int64_t* dims, int window, int stride,
                                      size_t* bytes);

/* PSNR and SSIM of y against x.
 *  d_x, d_y     float[N] original and reconstructed field, device, C order
 *  rank, dims   as qai_mitigate (the same shapes are accepted)
 *  window       1..11 points per axis (7 in the paper)
 *  stride       1..4 (2 in the paper)
 *  d_result     one qai_quality_out, device; written on `stream`
 *  d_ssim_map   float[windows] per-window SSIM (z, y, x order of the window
 *               starts), device, or NULL
 *  d_ws         qai_workspace_size_quality bytes, device, 256-byte aligned
 * Sums are fp32 per window and over points with compensation, FP64 across
 * windows and blocks, added in a fixed order (the same result on every run).
 * Returns QAI_ERR_INVALID_ARG for NULL inputs, a window or stride out of
 * range, or a short or misaligned workspace; QAI_ERR_SHAPE as qai_mitigate. */
qai_status qai_quality(const float* d_x, const float* d_y, int rank, const int64_t* dims, int window,
                       int stride, qai_quality_out* d_result, float* d_ssim_map, void* d_ws,
                       size_t ws_bytes, cudaStream_t stream);

/* Largest field (points, after squeezing) that qai_mitigate_static accepts. */
#define QAI_STATIC_MAX_POINTS 2097152

/* qai_mitigate for callers that cannot allocate device memory at all: code
 * running inside a host framework that owns every device allocation and
 * forbids new ones while it executes (a plugin's execute callback, for one),
 * or a latency-critical path that cannot afford cudaMalloc's implicit
 * synchronisation and has no workspace of its own to hand over. The paper has
 * no counterpart; it is a deployment convenience of this library.
 *
 * Instead of a workspace it uses one scratch array compiled into the library
 * (a 256-byte aligned __device__ array of 15 * QAI_STATIC_MAX_POINTS + 1 MiB
 * bytes, about 31 MiB). Every GPU on which the library's code is loaded holds
 * that array until the process exits.
 *
 * First call on a device: it looks up the array's device address
 * (cudaGetSymbolAddress) with that device current. Under CUDA's lazy module
 * loading (the default) that lookup loads the array's module on the device,
 * which commits the array's memory there; if that fails (out of memory, for
 * one) the call returns QAI_ERR_CUDA. So make the first call on each device
 * outside any region that must not allocate, and before any stream capture.
 * Later calls allocate nothing: no cudaMalloc, no cudaFree, no library
 * routine that allocates.
 *  d_q, d_out, rank, dims, eb, params, stream: as for qai_mitigate (the
 *          caller still passes the input and the output buffers).
 * Fields larger than QAI_STATIC_MAX_POINTS points return QAI_ERR_SHAPE before
 * any CUDA call, and so do fields whose workspace (qai_workspace_size) is
 * larger than the array; every field of at most QAI_STATIC_MAX_POINTS points
 * with an x extent (after squeezing) of 16 or more fits. Every call shares the array, which keeps the last call's
 * contents; the call's first kernel clears the few counters that must start
 * at zero, and every other slice is written before it is read. Calls whose
 * work overlaps on the GPU (two streams, or two host threads) race on the
 * array and corrupt each other's results: serialise them, for example on one
 * stream. No per-step (debug) outputs. */
qai_status qai_mitigate_static(const int32_t* d_q, float* d_out, int rank, const int64_t* dims,
                               double eb, const qai_params* params, cudaStream_t stream);

/* ---- Sharded calls (Section VII-B, distributed-memory parallelization) -----
 * A rank-2 or rank-3 field (every extent >= 2) is cut along axis 0 (z of a
 * 3-D field, y of a 2-D one) into P contiguous slabs, one per process; slab k
 * holds the planes [floor(k n0 / P), floor((k + 1) n0 / P)). The processes'
 * exchanges are host code (paper_2602_20097_gb300/sharded.py over
 * torch.distributed); these entry points are each process's device work.
 *
 *  extended slab  a slab plus the one plane on each side that a neighbour
 *                 owns (none past the field's ends): ext_dims = {planes, n1}
 *                 or {planes, n1, n2}, C order. Step A and GetBoundary(S) on
 *                 it equal the whole field's on the slab's own planes: its
 *                 first and last planes are not interior to it, and its other
 *                 planes see their true neighbours.
 *  band           every line along axis 0 through a range of `width` axis-1
 *                 indices: band_dims = {n0, width} or {n0, width, n2}, C order
 *                 (a band of a 3-D field is a z-by-width-by-nx block).
 *
 * The exact form (sequentially compliant) runs, on every process,
 * qai_shard_rows(1) on its extended slab; an all-to-all from slabs to bands;
 * qai_shard_lines(1) on its band (Dist1 and S = S_B[I1] of the whole field);
 * S back to the extended slabs; qai_shard_rows(2); an all-to-all to bands;
 * qai_shard_lines(2) (Dist2 fused with step E); D'' back to the slabs. The
 * result equals qai_mitigate's on the whole field bit for bit. The
 * approximate form (the paper's "local communication" strategy) runs both
 * qai_shard_lines on the extended slab itself, with the neighbours' S planes
 * copied into it between the two phases: the EDTs see only the slab's own
 * sites. */

/* Workspace of qai_shard_rows on an extended slab, and the bytes per point of
 * its output words (2 for rank 2, 4 for rank 3). */
qai_status qai_shard_sizes(int rank, const int64_t* ext_dims, size_t* ws_bytes, int* word_bytes);

/* Row work on an extended slab: the passes of an EDT along every axis but
 * axis 0 (Algorithm 1; x, then y for 3-D).
 *  phase 1  step A (Algorithm 2: B1 and S_B) and the first EDT's passes with
 *           the sign code of each nearest B1 point carried along; writes the
 *           equal-q neighbour map d_eqm (1 byte a point) and d_words. d_s is
 *           unused.
 *  phase 2  GetBoundary(S) (Algorithm 3: B2 from S and q) and the second
 *           EDT's passes; reads d_q, d_eqm (from phase 1 on the same slab) and
 *           d_s (S on the extended slab, int8), writes d_words.
 * d_words holds word_bytes per point (qai_shard_sizes), d_ws ws_bytes, all
 * device memory owned by the caller. QAI_ERR_SHAPE for extents beyond the
 * line limits of qai_mitigate or >= 2^31 points. */
qai_status qai_shard_rows(int phase, int rank, const int64_t* ext_dims, const int32_t* d_q,
                          const int8_t* d_s, uint8_t* d_eqm, void* d_words, void* d_ws, size_t ws_bytes,
                          const qai_params* params, cudaStream_t stream);

/* Line work on a band (or, in the approximate form, on an extended slab
 * viewed as one band): the last pass of an EDT, along axis 0.
 *  phase 1  reads the phase-1 words; writes Dist1 (int32 squared distance,
 *           INT32_MAX where the lines hold no B1 point), S (int8) and
 *           d_count (uint16 per line: its points with S != 0, saturated).
 *  phase 2  reads the phase-2 words, d_q, Dist1, S and d_count of the same
 *           band; writes D'' (float32) = 2 q eps + S w eta eps (step E).
 * band_dims: the block's extents; dims: the whole field's (they bound the
 * distances the words can carry; band_dims[a] <= dims[a]). Arrays of the block's points (d_count: one
 * entry per line), device memory owned by the caller. */
qai_status qai_shard_lines(int phase, int rank, const int64_t* band_dims, const int64_t* dims,
                           const void* d_words, const int32_t* d_q, int32_t* d_dist1, int8_t* d_s,
                           uint16_t* d_count, float* d_out, double eb, const qai_params* params,
                           cudaStream_t stream);

/* Strided device-to-device block copy for the exchanges: `height` runs of
 * `width` bytes, `src_pitch` / `dst_pitch` bytes apart (pitches >= width). */
qai_status qai_shard_copy(void* d_dst, int64_t dst_pitch, const void* d_src, int64_t src_pitch, int64_t width,
                          int64_t height, cudaStream_t stream);

/* Per-kernel timing. While enabled, every kernel the library launches is
 * bracketed by CUDA events recorded on the launch stream. qai_profile_read
 * waits for the recorded events, then reports, per kernel name, the launch
 * count, the summed device time and the algorithmic bytes (the bytes the
 * kernel must read and write: inputs and outputs, no halo re-reads), and
 * resets the counters. Returns the number of kernel names (<= cap) filled. */
typedef struct {
    char name[48];
    int64_t launches;
    double total_ms;
    double algo_bytes;   /* summed over the launches */
} qai_kernel_stat;

qai_status qai_profile_enable(int on);
int qai_profile_read(qai_kernel_stat* out, int cap);

/* Restricts the per-kernel timing to the kernels named `name` (a copy is
 * kept; NULL or "" times every kernel again). Fewer events on the stream
 * disturb the timed work less. */
qai_status qai_profile_select(const char* name);

/* Number of kernel launches made by the library since load (all entry points). */
int64_t qai_launch_count(void);

/* Human-readable name of a status code; a static string. */
const char* qai_status_string(qai_status s);

/* Detail of the last error on the calling host thread ("" if none). */
const char* qai_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* QAI_H */
