/*
 * stencil.h -- C ABI of the GB300 stencil-matrixization library.
 *
 * The library advances structured-grid stencils (Sec. 2.2 of "Stencil
 * Matrixization", arXiv 2310.16298): a field A at time t is mapped to B at
 * time t+1 by
 *
 *     B[x] = sum over o in [0, 2r]^d of C^g[o] * A[x + o - r]          (Eq. (stencil-2d9p))
 *
 * with C^g the (2r+1)^d gather-mode coefficient tensor (Eq. (stencil-2d9p-cm)),
 * r the stencil order (radius), d = 2 or 3.  The matrixized implementation
 * evaluates the same sum in scatter mode as outer products of coefficient
 * vectors and input vectors accumulated into resident output tiles (Sec. 3,
 * Eq. (final)); the gather implementation is the plain CUDA-core form.
 *
 * Conventions for every entry point:
 *  - Arrays are C-ordered, last index contiguous (the footnote of Sec. 4.1),
 *    and hold only the interior points listed in `shape`; rows are packed
 *    unless the plan was created with a pitch (stencil_options.pitch), which
 *    then applies to every grid passed to the plan.  Points outside the interior are 0 at every step
 *    (STENCIL_BC_DIRICHLET_ZERO) or the interior taken modulo the extent
 *    (STENCIL_BC_PERIODIC).
 *  - Device pointers are CUDA device (or managed) addresses on the device
 *    that was current when the plan was created; host pointers are ordinary
 *    host memory.  The caller keeps ownership of every buffer it passes.
 *  - Every call returns a stencil_status; nothing aborts or exits.  After a
 *    non-OK status, stencil_last_error() returns a message for the calling
 *    thread.
 *  - No call needs or takes PyTorch types.
 */
#ifndef STENCIL_GB300_H
#define STENCIL_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define STENCIL_API __attribute__((visibility("default")))
#else
#define STENCIL_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stencil_plan_s *stencil_plan_t;
typedef struct CUstream_st *stencil_stream_t; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
    STENCIL_OK = 0,
    STENCIL_EINVAL = 1,       /* invalid argument (message says which)              */
    STENCIL_ENOMEM = 2,       /* device or host allocation failed, or over budget    */
    STENCIL_ECUDA = 3,        /* a CUDA call failed (message has the CUDA error)     */
    STENCIL_EBUSY = 4,        /* resource in use (e.g. no free serving slot)         */
    STENCIL_ENOTREADY = 5,    /* submitted work has not finished yet                 */
    STENCIL_ETIMEDOUT = 6,    /* a wait ran out its host-side deadline               */
    STENCIL_EUNSUPPORTED = 7  /* valid request, but no kernel for this combination   */
} stencil_status;

typedef enum { STENCIL_STAR = 0, STENCIL_BOX = 1 } stencil_kind;
typedef enum { STENCIL_F32 = 0, STENCIL_F64 = 1 } stencil_dtype;
typedef enum { STENCIL_BC_DIRICHLET_ZERO = 0, STENCIL_BC_PERIODIC = 1 } stencil_boundary;

/* Arithmetic used by the outer-product (matrixized) kernels.  NATIVE is the
 * storage type on CUDA cores (FP32 FMA or FP64 DFMA).  TF32 / BF16 run the
 * outer products on the tensor cores with FP32 accumulation; the X2/X3 forms
 * split each operand into 2 or 3 parts (hi + lo [+ lo2]) and keep the partial
 * products listed in the design notes, which restores FP32-level accuracy.
 * BF16_W2 rounds the field to one BF16 part but keeps the weights as two BF16
 * parts (two products per MMA step): plain-BF16 inputs without the amplitude
 * drift that BF16-rounded weights cause over many steps (their sum is off by
 * up to 2^-9, an error that grows linearly with the step count). */
typedef enum {
    STENCIL_PREC_NATIVE = 0,
    STENCIL_PREC_TF32 = 1,
    STENCIL_PREC_TF32X3 = 2,
    STENCIL_PREC_BF16 = 3,
    STENCIL_PREC_BF16X2 = 4,
    STENCIL_PREC_BF16X3 = 5,
    STENCIL_PREC_BF16_W2 = 6
} stencil_precision;

typedef enum {
    STENCIL_IMPL_AUTO = 0,       /* matrixized where built for the request, else gather */
    STENCIL_IMPL_GATHER = 1,     /* CUDA-core gather kernel (baseline form)             */
    STENCIL_IMPL_MATRIXIZED = 2  /* tensor-core outer-product kernel                    */
} stencil_impl;

/* Coefficient-line cover of a star stencil on the matrixized kernel (Sec. 4.1,
 * Tables cls-2d / cls-3d).  PARALLEL: every line along the contiguous axis
 * goes to the tensor cores (off-axis weights as one-diagonal bands).  HYBRID:
 * only the contiguous-axis line (and an identity band that returns the input
 * rows) goes to the tensor cores; the 2*ndim*r - 2r off-axis weights are
 * applied on the CUDA cores to those rows in FP32.  Built for 3D stars;
 * 2D stars and box stencils always use PARALLEL.  AUTO for a 3D star times
 * one sweep of each cover on the plan's own grids when the plan is created
 * and keeps the faster (the choice is cached per order, precision, boundary
 * and grid size class); stencil_plan_info reports the cover that runs. */
typedef enum {
    STENCIL_COVER_AUTO = 0,      /* library choice (3D stars: the faster, by timing)   */
    STENCIL_COVER_PARALLEL = 1,
    STENCIL_COVER_HYBRID = 2
} stencil_cover;

typedef struct {
    int32_t prec;     /* stencil_precision; default NATIVE for GATHER, TF32X3 for F32 MATRIXIZED */
    int32_t bc;       /* stencil_boundary; default DIRICHLET_ZERO                              */
    int32_t impl;     /* stencil_impl; default AUTO                                            */
    int32_t tb;       /* time steps fused per sweep (temporal blocking); 0 = library choice     */
    int32_t cover;    /* stencil_cover; default AUTO (EINVAL when out of range)                 */
    int32_t pitch;    /* row stride of the grids, in elements (0 = packed rows); >= the
                         contiguous extent and a multiple of 16 bytes, else EINVAL.  Padding
                         elements are neither read nor written.  Packed grids whose rows are
                         not 16-byte multiples run on the tensor-core kernels through two
                         padded grids the plan owns (one strided copy in, one out per apply) */
    int32_t unit_planes; /* 3D matrixized kernel: output planes per work unit, 1..1024 (0 = the
                         library's 32).  Each unit streams its planes plus 2r halo planes, so
                         the depth trades re-read halo planes against the number of units
                         (load balance); exposed for the scheduling ablation          */
    int32_t reserved[1];
} stencil_options;

/* Plan introspection (filled by stencil_plan_info). */
typedef struct {
    int32_t impl;         /* stencil_impl actually used (GATHER or MATRIXIZED)          */
    int32_t prec;         /* stencil_precision actually used                            */
    int32_t tb;           /* time steps per sweep                                       */
    int32_t n_lines;      /* coefficient lines run as outer products (0 for GATHER)     */
    int32_t n_scalar;     /* coefficients applied on CUDA cores beside the lines        */
    int32_t tile_n;       /* output columns per outer-product block (0 for GATHER)      */
    int64_t scratch_bytes;/* device scratch owned by the plan                           */
    int32_t device_error; /* error bits: nonzero once a kernel of the plan gave up a
                             bounded wait (or stencil_plan_raise_error set bits)        */
    int32_t cover;        /* stencil_cover the matrixized kernel runs (0 for GATHER)    */
    int32_t kernels_per_sweep; /* kernel launches per sweep: 2 for MATRIXIZED plans with
                             a periodic boundary (the tensor-core kernel, whose TMA
                             loads see zeros outside the grid in x and y, then a
                             kernel over the boundary strips that adds the wrapped
                             terms), else 1                                             */
} stencil_plan_info_t;

/* ---------------------------------------------------------------------------
 * Plans.
 *
 * stencil_plan_create -- validate a problem and build everything a sweep needs
 * (Sec. 3.1-3.4: C^s = J C^g J, Eq. (stencil-2d9p-gm2sm); the coefficient
 * lines; the banded operand of every line, the windows of C^o of Eq. (co);
 * the operand splits for the chosen precision).
 *   out     [out] receives the plan handle.
 *   ndim    2 or 3.
 *   shape   ndim interior extents, C order (slowest first); each >= 2r+1.
 *   radius  the order r, 1..4.
 *   kind    STAR requires every off-axis coefficient to be exactly 0.
 *   coeffs  host array of (2r+1)^ndim doubles: dense C^g in C order, gather
 *           orientation (coeffs[o] multiplies A[x + o - r]).  Copied; the
 *           caller may free it after the call.  All must be finite.
 *   dtype   storage type of the fields passed to apply.
 *   opt     NULL for defaults.
 * Errors: EINVAL (bad argument; TF32/BF16 precision with F64 storage),
 * EUNSUPPORTED (IMPL_MATRIXIZED for a shape/precision without a kernel:
 * the message says which), ENOMEM / ECUDA (device allocation of the plan's
 * scratch grid and operands).  The plan owns one scratch grid of the field's
 * size; it is freed by stencil_plan_destroy.
 */
STENCIL_API stencil_status stencil_plan_create(stencil_plan_t *out, int ndim, const int64_t *shape, int radius,
                                   stencil_kind kind, const double *coeffs, stencil_dtype dtype,
                                   const stencil_options *opt);

/* Free a plan and its device memory.  Work still queued that uses the plan
 * must have finished.  NULL is accepted. */
STENCIL_API stencil_status stencil_plan_destroy(stencil_plan_t plan);

/* Describe the plan (host only, no GPU work). */
STENCIL_API stencil_status stencil_plan_info(stencil_plan_t plan, stencil_plan_info_t *info);

/* Device errors.  Every wait inside the matrixized kernels is bounded; a
 * kernel that runs one out sets error bits in a host-mapped word of its plan,
 * drains its copies in flight, frees its tensor memory and returns, so the
 * CUDA context stays usable but the output of that sweep is not valid.  The
 * bits are sticky until the plan is destroyed, and every call that runs or
 * completes work of the plan reports them as STENCIL_ECUDA with a message:
 * stencil_apply, stencil_apply_noalloc, stencil_apply_host and
 * stencil_submit (before queueing), stencil_poll and stencil_wait (once the
 * work has finished), stencil_batch_launch (any plan of the batch),
 * stencil_batch_run (after the run), and the server's request status.
 *
 * stencil_plan_raise_error -- set error bits of a plan from the host, as a
 * kernel that gave up a wait would: host-side fault injection, used to test
 * the error paths without making a GPU fault.  bits != 0.  Errors: EINVAL. */
STENCIL_API stencil_status stencil_plan_raise_error(stencil_plan_t plan, uint32_t bits);

/* ---------------------------------------------------------------------------
 * Sweeps.
 *
 * stencil_apply -- advance d_in by `steps` time steps into d_out (Sec. 2.2:
 * two copies of the grid used alternately; the library's second copy is the
 * plan's scratch grid).  Asynchronous on `stream`; returns once the work is
 * queued.
 *   d_in    device array, dtype of the plan, read only (unless == d_out).
 *   d_out   device array of the same size; may equal d_in.
 *   steps   >= 0; 0 copies d_in to d_out.
 * Errors: EINVAL (NULL pointer, steps < 0), ECUDA (launch failure, or the
 * plan's error bits are set: see stencil_plan_raise_error).
 * Concurrent applies of one plan must be ordered by the caller: they share
 * the plan's scratch grid and, for the matrixized kernels, the plan's
 * device tile counter (tiles are handed out to the SMs at run time; the
 * counter is back at zero when a launch ends).
 */
STENCIL_API stencil_status stencil_apply(stencil_plan_t plan, const void *d_in, void *d_out, int64_t steps,
                             stencil_stream_t stream);

/* stencil_apply_noalloc -- stencil_apply for callers that cannot allocate
 * device memory while they run steps (code inside another runtime's stream
 * work, processes whose device memory is budgeted up front, real-time loops
 * that cannot take cudaMalloc's synchronisation).  The paper has no
 * counterpart.
 *
 * Same arguments, layout and result as stencil_apply, but the second grid copy
 * of the ping-pong is a file-scope device array of 16 MiB (4 Mi FP32 or 2 Mi
 * FP64 points) instead of the plan's scratch grid, and the call allocates
 * nothing (no cudaMalloc, cudaFree or allocating library routine).
 *   - Grids larger than 16 MiB return EINVAL with a message.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - Every call shares the one array per device and leaves its last contents
 *     there; a sweep writes every point of the copy before reading it, so
 *     nothing has to start at zero.  Calls whose work overlaps on the GPU (on
 *     different streams, or while an earlier call is still running) race on
 *     the array: order them.
 *   - Every GPU that loads the library holds the 16 MiB until the process
 *     exits. */
STENCIL_API stencil_status stencil_apply_noalloc(stencil_plan_t plan, const void *d_in, void *d_out, int64_t steps,
                                                 stencil_stream_t stream);

/* Host-to-host convenience: copy h_in to the device, apply, copy the result
 * to h_out (both host arrays of the plan's dtype, pinned or pageable), and
 * synchronise.  The field is advanced in place in a device staging grid that
 * the plan allocates on its first stencil_apply_host call and keeps until it
 * is destroyed (so later calls allocate nothing); the copies and sweeps run
 * on the plan's own stream.  Errors: EINVAL, ENOMEM (staging grid), ECUDA. */
STENCIL_API stencil_status stencil_apply_host(stencil_plan_t plan, const void *h_in, void *h_out, int64_t steps);

/* ---------------------------------------------------------------------------
 * Asynchronous submission.  stencil_submit queues an apply on the plan's own
 * stream and returns a ticket; stencil_poll returns OK once that work has
 * finished, ENOTREADY before; stencil_wait blocks up to timeout_ms
 * (< 0: no limit) and returns OK, or ETIMEDOUT without cancelling the work.
 * The host waits with cudaEventQuery and short sleeps; nothing spins on the
 * device.  A ticket is released by the first poll/wait that returns OK or a
 * CUDA error; using it again returns EINVAL.
 */
STENCIL_API stencil_status stencil_submit(stencil_plan_t plan, const void *d_in, void *d_out, int64_t steps,
                              uint64_t *ticket);
STENCIL_API stencil_status stencil_poll(uint64_t ticket);
STENCIL_API stencil_status stencil_wait(uint64_t ticket, int64_t timeout_ms);

/* Message describing the last non-OK status returned to this thread. */
STENCIL_API const char *stencil_last_error(void);

/* ---------------------------------------------------------------------------
 * Batches: many independent problems advanced together (problem i by steps[i]
 * time steps from d_in[i] into d_out[i], with plans[i]).  When every plan is
 * 2D with the same order, kind and dtype (order <= 3), all problems are packed
 * into shared persistent launches: launch k advances every problem that still
 * has steps left by up to `tb` steps (temporal blocking), each with its own
 * coefficients and boundary.  Otherwise each problem runs its own sweeps.  In
 * both cases the whole launch sequence is captured once in a CUDA graph and
 * replayed by stencil_batch_launch.
 *
 * stencil_batch_create_ex -- build the schedule and the graph.
 *   tb          time steps per launch (1..8); 0 = autotune.
 *   tile_shape  output tile of the packed launches: 0 = 64 x 128,
 *               1 = 32 x 64 (rows x columns); -1 = autotune.
 *   The autotuner times one launch of this batch (reading d_in, writing the
 *   plans' scratch grids) for each (tile shape, depth 1..4) pair left open
 *   that fits shared memory, and keeps the pair fastest per time step (cached
 *   per order, kind, dtype, batch size class and the fixed values).  d_in must
 *   hold the inputs when create is called if anything is autotuned.  Both
 *   values are ignored when the batch is not packed.
 *   The arrays plans/d_in/d_out/steps are copied; the buffers must stay valid
 *   while the batch exists.  d_in[i] == d_out[i] is allowed.
 * stencil_batch_create -- stencil_batch_create_ex with tile_shape = -1.
 * Errors: EINVAL (NULL or negative entries, tb or tile_shape out of range),
 * EUNSUPPORTED (tb too deep for shared memory), ENOMEM / ECUDA.
 */
typedef struct stencil_batch_s *stencil_batch_t;

typedef struct {
    int32_t packed;    /* 1: problems share persistent launches                */
    int32_t tb;        /* time steps per launch                                */
    int32_t launches;  /* packed launches per run (-1 when not packed)         */
    int32_t tile_shape;/* tile shape of the packed launches (-1: not packed)   */
    int64_t tiles;     /* output tiles processed per run (packed)              */
    int64_t updates;   /* stencil updates per run (sum of points x steps)      */
} stencil_batch_info_t;

STENCIL_API stencil_status stencil_batch_create_ex(stencil_batch_t *out, int n, const stencil_plan_t *plans,
                                                   const void *const *d_in, void *const *d_out,
                                                   const int64_t *steps, int32_t tb, int32_t tile_shape);
STENCIL_API stencil_status stencil_batch_create(stencil_batch_t *out, int n, const stencil_plan_t *plans,
                                                const void *const *d_in, void *const *d_out, const int64_t *steps,
                                                int32_t tb);
/* Queue one run of the batch (one graph launch) on `stream`; asynchronous. */
STENCIL_API stencil_status stencil_batch_launch(stencil_batch_t batch, stencil_stream_t stream);
STENCIL_API stencil_status stencil_batch_info(stencil_batch_t batch, stencil_batch_info_t *info);
/* Free the batch after its queued runs have finished.  NULL is accepted. */
STENCIL_API stencil_status stencil_batch_destroy(stencil_batch_t batch);

/* One-shot: create (autotuned), launch on `stream`, wait for it, destroy. */
STENCIL_API stencil_status stencil_batch_run(int n, const stencil_plan_t *plans, const void *const *d_in,
                                             void *const *d_out, const int64_t *steps, stencil_stream_t stream);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of stencil solves.
 *
 * A server owns a worker thread.  Submitted requests are admitted in arrival
 * order while the device-memory budget (each request is charged two grids
 * plus 1 MiB: its own grid, advanced in place, and its plan's scratch grid,
 * the second copy of the ping-pong) and the resident-slot
 * limit allow.  Every resident request advances by at most `quantum_steps`
 * time steps per issue on one of `nstreams` streams, so requests overlap on
 * the device and new ones join as soon as memory and a slot free up.  A
 * finished grid is copied to host memory and the request's device state is
 * freed.  Each request runs through the same plan and kernels as
 * stencil_apply, so its result is the same alone and in any mix.
 */
typedef struct stencil_server_s *stencil_server_t;

typedef struct {
    int32_t ndim, radius, kind, dtype, bc, impl;  /* as for stencil_plan_create / stencil_options */
    int64_t shape[3];                             /* ndim interior extents                        */
    const double *coeffs;  /* dense C^g; copied by submit                                              */
    const void *h_in;      /* host input grid (dtype, C order), read at admission; keep it valid
                              until the request finishes.  NULL: the input is the uniform[lo, hi)
                              SplitMix64 field of `seed` (element i of the seed's stream in C order),
                              generated on the device                                              */
    uint64_t seed;
    double lo, hi;
    int64_t steps;         /* time steps to advance, >= 0                                          */
} stencil_request;

typedef struct {
    double submit_s, admit_s, done_s;  /* seconds since the server was created                 */
    int32_t impl;                      /* stencil_impl that ran                                 */
    int32_t status;                    /* stencil_status of the request                         */
    int64_t updates;                   /* points x steps                                        */
} stencil_request_stats;

typedef struct {
    int64_t queued, resident, admitted, completed;
    int64_t bytes_in_use, peak_bytes, peak_resident, quanta_issued;
} stencil_server_stats_t;

/* budget_bytes > 0, max_resident >= 1, quantum_steps >= 1, 1 <= nstreams <= 64. */
STENCIL_API stencil_status stencil_server_create(stencil_server_t *out, int64_t budget_bytes, int32_t max_resident,
                                                 int32_t quantum_steps, int32_t nstreams);
/* Queue a request; *id identifies it.  EINVAL for an invalid problem, ENOMEM
 * when one request alone exceeds the budget. */
STENCIL_API stencil_status stencil_server_submit(stencil_server_t server, const stencil_request *request,
                                                 uint64_t *id);
/* OK once the request finished, ENOTREADY before, its error if it failed. */
STENCIL_API stencil_status stencil_server_poll(stencil_server_t server, uint64_t id);
/* Block up to timeout_ms (< 0: no limit); ETIMEDOUT leaves the request running. */
STENCIL_API stencil_status stencil_server_wait(stencil_server_t server, uint64_t id, int64_t timeout_ms);
/* Copy a finished result to h_out (NULL: discard), fill stats, release the id. */
STENCIL_API stencil_status stencil_server_result(stencil_server_t server, uint64_t id, void *h_out,
                                                 stencil_request_stats *stats);
STENCIL_API stencil_status stencil_server_stats(stencil_server_t server, stencil_server_stats_t *stats);
/* Finish every submitted request, then stop the worker and free the server. */
STENCIL_API stencil_status stencil_server_destroy(stencil_server_t server);

/* Fill a device array with the uniform[lo, hi) SplitMix64 field of `seed`
 * (elements offset .. offset+count-1 of the stream, rounded to dtype); the
 * same values the seeded host generator gives.  Asynchronous on stream. */
STENCIL_API stencil_status stencil_fill_uniform(void *d_out, stencil_dtype dtype, int64_t count, uint64_t seed,
                                                int64_t offset, double lo, double hi, stencil_stream_t stream);

/* ---------------------------------------------------------------------------
 * Error norms against a reference (the accuracy report attached to every
 * result).  Computes, in FP64 on the device,
 *   out[0] = sum (got - ref)^2,  out[1] = sum ref^2,
 *   out[2] = max |got - ref|,    out[3] = max |ref|
 * over `count` elements.  d_got has type got_dtype, d_ref is FP64; out is a
 * host array of 4 doubles.  Synchronises `stream` before returning.
 */
STENCIL_API stencil_status stencil_error_norms(const void *d_got, stencil_dtype got_dtype, const double *d_ref,
                                   int64_t count, double *out, stencil_stream_t stream);

/* ---------------------------------------------------------------------------
 * Host-only plan algebra (no GPU needed; used to check the plan layer).
 *
 * stencil_band_operand -- the banded (Toeplitz) operand of one coefficient
 * line.  `line` holds the 2r+1 gather-orientation weights of the line
 * (line[t] multiplies the input at offset t - r along the line's axis).
 * Writes K x n doubles, K = n + 2*pad, row-major:
 *     band[k*n + q] = line[k - q - (pad - r)]  when 0 <= k - q - (pad - r) <= 2r, else 0,
 * i.e. output q of an n-wide block receives input k of the K-wide window that
 * starts pad points before the block.  With pad = r the columns of `band`,
 * read along k, are the windows of a column of C^o (Eq. (co)) that
 * Eq. (final) multiplies with the input vectors.  pad >= r, n >= 1.
 */
STENCIL_API stencil_status stencil_band_operand(int radius, const double *line, int n, int pad, double *band);

/* stencil_line_cover -- the coefficient lines a plan would use (Sec. 3.4 and
 * Tables cls-2d / cls-3d), described for an n x n output tile (2D) or
 * 1 x n x n tile (3D).
 *   option  0 = parallel lines (every line along the contiguous axis),
 *           1 = orthogonal (star only: one line per axis, the centre weight on
 *               the contiguous-axis line), 2 = hybrid (3D star only: lines
 *               CLS(i,*,r) plus CLS(r,r,*)).
 *   n_lines         [out] lines in the cover.
 *   outer_products  [out] vector outer products per tile: a line whose
 *                   nonzeros span s consecutive positions costs n + s - 1.
 * Errors: EINVAL for an option that does not apply to the kind/ndim.
 */
STENCIL_API stencil_status stencil_line_cover(int ndim, int radius, stencil_kind kind, int option, int n,
                                  int32_t *n_lines, int64_t *outer_products);

/* stencil_min_line_cover -- a minimal set of axis-parallel coefficient lines
 * covering every weight of a 2D stencil of any pattern (Sec. 3.5: the rows
 * and columns of the weight matrix form a bipartite graph whose edges are the
 * weights, and a minimum vertex cover of it, found through a maximum matching
 * and Konig's theorem, is a minimal line cover).
 *   n        side of the weight matrix (2r+1), 1..64.
 *   mask     n x n bytes, row-major; nonzero = a weight is present.
 *   rows     [out] n entries: 1 if row line i (weights C[i][*]) is in the cover.
 *   cols     [out] n entries: 1 if column line j (weights C[*][j]) is in the cover.
 *   n_lines  [out] lines in the cover (sum of rows and cols).
 * Host only; the caller owns every array.  Errors: EINVAL (NULL, n out of
 * range).  The matrixized kernels run star and box patterns only; this is
 * the plan algebra for others.
 */
STENCIL_API stencil_status stencil_min_line_cover(int n, const uint8_t *mask, int32_t *rows, int32_t *cols,
                                                  int32_t *n_lines);

/* Library version string. */
STENCIL_API const char *stencil_version(void);

#ifdef __cplusplus
}
#endif

#endif /* STENCIL_GB300_H */
