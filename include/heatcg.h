/*
 * heatcg.h -- C ABI of the GB300 (sm_103a) heat-stencil and CG library.
 *
 * The library advances the three-dimensional heat equation of Section 4 with
 * the explicit update of Eq. 4 in its constant-coefficient form
 *
 *     u'[k,j,i] = u + r * ((u[i-1] + u[i+1]) + (u[j-1] + u[j+1]) + (u[k-1] + u[k+1]) - 6 u)
 *
 * (r = alpha*dt/h^2) on a box whose boundary values are held at zero, and
 * solves the companion system A x = b of Section 7.5 by conjugate gradients,
 * A being the 7-point Dirichlet Laplacian (CSR or matrix-free).
 *
 * Conventions shared by every entry point:
 *   - Grid sizes are INTERIOR counts nx, ny, nz (the boundary layer is not
 *     counted; h = 1/(n+1) per axis).  Fields cross the ABI as dense arrays
 *     of nx*ny*nz elements, x fastest, then y, then z (the paper's k, j, i
 *     loop order, Algorithm COMPUTE_SINGLE_GPU).
 *   - Every function returns HS_OK (0) or a negative HS_E* code.  On error,
 *     hs_last_error() returns a message for the calling thread, and nothing
 *     has been enqueued unless the code is HS_ECUDA.
 *   - "stream" arguments are cudaStream_t handles passed as void*; NULL
 *     means the legacy default stream.  Work is enqueued asynchronously on
 *     that stream unless a function says it synchronises.
 *   - Pointers marked "device" must be device (or managed) memory of the
 *     current CUDA device; the caller keeps ownership of every buffer it
 *     passes in and must keep it alive until the work that uses it is done.
 *   - The library is not thread safe per handle: one handle, one thread at a
 *     time.  Distinct handles may be used from distinct threads.
 */
#ifndef HEATCG_H
#define HEATCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define HS_OK          0
#define HS_EINVAL     (-1)  /* bad size, pointer, flag or dtype            */
#define HS_ENOMEM     (-2)  /* device or pinned-host allocation failed     */
#define HS_ECUDA      (-3)  /* a CUDA call or kernel launch failed         */
#define HS_EUNSTABLE  (-4)  /* r > 1/6 without HS_ALLOW_UNSTABLE           */
#define HS_ENOCONV    (-5)  /* CG stopped at max_iter before reaching rtol */
#define HS_ETIMEOUT   (-6)  /* a bounded device-side wait expired          */
#define HS_EBUSY      (-7)  /* the handle has work in a state that forbids the call */
#define HS_ERANGE     (-8)  /* a value lies outside the range a format can hold */

/* ---- element types ---------------------------------------------------- */
#define HS_F64 0
#define HS_F32 1

/* ---- heat handle flags ------------------------------------------------ */
/* Accept r > 1/6.  The explicit update of Eq. 4 is stable in three
 * dimensions only for r <= 1/6 (Section 4, Eq. 6 prints the one-dimensional
 * bound dt/h^2 < 0.5); larger r makes the highest grid mode grow. */
#define HS_ALLOW_UNSTABLE   0x1u
/* FP64 only: evaluate the update with one rounding per operation, in exactly
 * the order written above and without fused multiply-add (the paper compiles
 * with --fmad=false / -ffp-contract=off, Section 5, table of compiler
 * flags).  Slower (9 instead of 7 FP64 instructions per point). */
#define HS_EXACT_ROUNDING   0x2u
/* Advance each step with one kernel over the whole interior (Algorithm
 * COMPUTE_SINGLE_GPU) instead of the Interior + Boundary pair (Algorithms
 * INTERIOR and BOUNDARY).  Results are bitwise identical either way. */
#define HS_SCHED_FULL       0x4u
/* HS_F64 only: keep the FP64 interface (upload and read are doubles) but hold
 * the field as 64-bit fixed-point integers U = round(u 2^E), with E chosen at
 * each upload from max|u0| so that 12 max|U| < 2^61.  Every step is exact
 * integer arithmetic -- the neighbour sum and S - 6U exactly, r held as
 * R = round(r 2^64) (exact for r >= 2^-11) -- with one rounding per point, of
 * R (S - 6U) / 2^64 to the nearest integer.  Requires r <= 1/6 (the update is
 * then a convex combination and |U| never grows, so nothing overflows);
 * excludes HS_EXACT_ROUNDING and HS_ALLOW_UNSTABLE.  heat_read returns the
 * nearest doubles; it reports HS_ERANGE if the uploaded field held NaN or Inf.
 * Per step this costs integer instructions instead of FP64 ones, so on GPUs
 * whose FP64 pipe is narrow it runs at memory speed. */
#define HS_FIXED64          0x8u
/* The paper's variable-coefficient problem instead of the constant one
 * (Section 4, Eqs. 1-4): du/dt = div(kappa grad u) + f with
 * kappa = 0.5 + 0.45 sin(pi x) sin(pi y) sin(pi z), f = 1 + cos(pi x) cos(pi y)
 * cos(pi z), and u' = u + dt f + sum_d dt/(2 h_d^2) D_d with face-averaged
 * differences D_x = (k[i+1] + k[i])(u[i+1] - u[i]) - (k[i] + k[i-1])(u[i] - u[i-1])
 * (the paper does not print D; this is the reading consistent with its
 * beta = dt/(2h^2)).  Here r means dt / h_min^2 (the paper's choice is
 * dt = h^2/(12 kappa_max), r = 1/(12 * 0.95)); the stability bound is
 * r <= 1/(6 kappa_max).  The coefficients (on every node, boundary included)
 * and dt f live on the device beside u, as in the paper's 1-GPU Baseline:
 * kappa itself for HS_F32, for HS_F64 the three face sums k[i+1] + k[i] of
 * each node (constant in time; the same values the formula forms).  For
 * HS_F64 the operator sums are formed exactly in integers on the field's
 * fixed-point scale (its largest exponent, tracked on the device as for the
 * default FP64 arithmetic) and rounded once -- the whole sum on a cubic grid,
 * each axis's sum otherwise: error below 6 * 2 * 1.9 * 4 * 2^-57 max|u| beta
 * plus a few roundings per step; fields outside [2^-903, 2^1007] in magnitude
 * step in FP64 arithmetic.  HS_F64 or
 * HS_F32; excludes HS_FIXED64, HS_EXACT_ROUNDING, HS_SCHED_FULL and tdepth > 1;
 * cannot join a heat batch. */
#define HS_VARKAPPA         0x10u
/* HS_F64 only: do every operation of the update on the FP64 pipe (the six
 * additions and two fused multiply-adds of the written order).  Without this
 * flag a plain HS_F64 handle with tdepth <= 1 keeps its fields in FP64 but
 * forms the numerator S - 6u exactly: each value becomes a 64-bit integer
 * within two units of u 2^(1080 - e), e the largest binary exponent field in
 * the current field (tracked on the device step by step), the integer sum is
 * exact, and u' = fma(r, (S - 6U) 2^(e - 1080), u) with the numerator rounded
 * to the nearest double -- one or two FP64 instructions per point instead of
 * seven, the rest done with integer instructions.  Its error against exact
 * arithmetic on the same field is below 24 r 2^-57 max|u| + 2 ulp; values
 * more than 58 binades below the field's maximum count as 0 (or one unit) in
 * the sum, not as centre values.  Fields whose largest exponent field lies
 * outside [max(70, 1081 - exponent field of r), 2040] (all-zero or tiny
 * fields, values near overflow, NaN, Inf) are stepped on the FP64 pipe
 * instead.  Temporal blocking (tdepth >= 2) and HS_VARKAPPA always use the
 * FP64 pipe. */
#define HS_FP64_PIPE        0x20u

typedef struct hs_heat* hs_heat_t;

typedef struct {
    int32_t  nx, ny, nz;   /* interior points per axis, each >= 1              */
    double   r;            /* alpha*dt/h^2 >= 0; see HS_ALLOW_UNSTABLE         */
    uint32_t flags;        /* HS_* heat flags                                 */
    int32_t  dtype;        /* HS_F64 or HS_F32: storage and arithmetic type   */
    int32_t  tdepth;       /* time steps per pass over HBM: 0 = library choice
                              (2 for HS_F32 without HS_VARKAPPA or
                              HS_SCHED_FULL, else 1), 1 = the Interior + Boundary
                              kernels every step, or 2, 3, 4 = temporal
                              blocking (see heat_step)                     */
    void*    stream;       /* cudaStream_t for all work of this handle        */
    void*    dev_buf0;     /* optional caller-owned device buffers for the two
                              time levels (for example torch allocations):
                              both NULL (the library allocates them) or both
                              set, distinct, non-overlapping, 256-byte aligned
                              and each at least heat_buffer_bytes(desc) long */
    void*    dev_buf1;
} hs_heat_desc;

/* Create a heat handle (Algorithm "1-GPU Baseline", setup and allocation:
 * the two time levels u_old and u_new).  Uses two device buffers of (nz+2)
 * planes x (ny+2) rows x pitch elements -- the caller's dev_buf0/dev_buf1 when
 * given, else its own allocations; it zeroes both (on the handle's stream), so
 * their boundary layer holds the Dirichlet zeros, which are never written
 * again and so survive every buffer swap.  Caller-owned buffers stay the
 * caller's: the handle never frees them, and they must outlive it.
 * Errors: HS_EINVAL (desc NULL, a size < 1, r < 0 or not finite, unknown flag
 * or dtype; caller buffers not both given, equal, overlapping or misaligned),
 * HS_EUNSTABLE (r > 1/6 without HS_ALLOW_UNSTABLE), HS_ENOMEM. */
int heat_create(hs_heat_t* out, const hs_heat_desc* desc);

/* Bytes of ONE padded field buffer for desc: (nz+2) (ny+2) pitch elements of
 * the dtype, pitch = the interior row plus its boundary cells and a 32-byte
 * lead, rounded up to 128 bytes (the layout the kernels index; Section 6.1's
 * padded arrays).  The size a caller-owned dev_buf0/dev_buf1 must have. */
int heat_buffer_bytes(const hs_heat_desc* desc, size_t* bytes);

/* Device bytes heat_create would allocate for desc (for admission control):
 * the two field buffers unless the caller supplies them, and the per-step
 * state of the exact-sum and FIXED64 arithmetics (and the coefficient
 * arrays and dt f for HS_VARKAPPA: two fields' worth for HS_F32, four for
 * HS_F64). */
int heat_device_bytes(const hs_heat_desc* desc, size_t* bytes);

/* Load the interior field u (nx*ny*nz elements of the handle's dtype, x
 * fastest) as the current time level and reset the step counter.  (The paper
 * copies u_old and u_new alike, Algorithm "1-GPU Baseline"; here the spare
 * buffer needs no copy: its boundary layer is zero from creation and the next
 * step writes every interior value of it before any is read.)  u is host memory
 * if src_is_device == 0, device memory otherwise.  Device memory and pinned,
 * mapped host memory (cudaHostAlloc, cudaMallocHost, cudaHostRegister; pinned
 * torch tensors) are read by a re-layout kernel, the latter through its mapped
 * device address, so the call returns at once; pageable host memory goes
 * through one strided copy.  Enqueued on the handle's stream; a pinned source
 * must stay unchanged until the stream has passed the upload. */
int heat_upload(hs_heat_t h, const void* u, int src_is_device);

/* Advance n_steps >= 0 steps.  With tdepth 1 each step runs the Boundary
 * kernel on the first and last interior k-planes and the Interior kernel on
 * the planes between them (Algorithms BOUNDARY and INTERIOR; on one GPU the
 * planes a k-split would exchange are the outermost interior planes), then
 * swaps the buffers by pointer (Algorithm "1-GPU Baseline").  On grids of
 * 2^22 points or more the Boundary kernel runs on a side stream of the
 * handle, forked from and joined back to the handle's stream every step, so
 * it overlaps the Interior kernel (the two write disjoint planes); the
 * handle's stream still orders everything after the step.  With tdepth
 * L >= 2 each pass over HBM advances L steps (temporal blocking: tiles with
 * an L-wide halo stream up the k axis, the intermediate time levels living
 * in shared memory and registers), then swaps; a remainder of n_steps is done
 * in shallower passes.  The result equals stepping one step at a time up to
 * rounding (bit for bit for FP32, and for FP64 against an HS_FP64_PIPE handle
 * stepped one step at a time, whose per-point arithmetic is the same; FIXED64
 * may rescale at different steps).  Asynchronous: launch errors
 * are returned here, errors raised while kernels run are returned by the next
 * synchronising call (a bounded device wait that ran out: HS_ETIMEOUT). */
int heat_step(hs_heat_t h, int64_t n_steps);

/* The three parts of one step, for callers that schedule them themselves:
 * the Interior kernel, the Boundary kernel (each writes the next time level
 * into the spare buffer), and the pointer swap that makes it current.
 * heat_step(h, 1) == heat_boundary(h); heat_interior(h); heat_swap(h). */
int heat_interior(hs_heat_t h);
int heat_boundary(hs_heat_t h);
int heat_swap(hs_heat_t h);

/* Interior-kernel timing, for measuring the kernel against its roofline
 * inside a running step loop.  heat_time_interior(h, 1) makes heat_step (at
 * tdepth 1) bracket every Interior launch with a pair of timing CUDA events
 * on the handle's stream; heat_time_interior(h, 0) stops it.
 * heat_interior_time waits for the last recorded launch, writes the mean
 * duration in milliseconds of the launches recorded since the previous call
 * (0 if none) and their count, and clears the record.  Either output may be
 * NULL.  A record holds up to 8192 launches; later ones go untimed until it
 * is read.  The events belong to the handle (freed by heat_destroy). */
int heat_time_interior(hs_heat_t h, int enable);
int heat_interior_time(hs_heat_t h, double* mean_ms, int64_t* launches);

/* Copy the current interior field to dst (Algorithm "1-GPU Baseline", the
 * device-to-host copy of the result after the time loop; nx*ny*nz elements, x fastest):
 * host memory if dst_is_device == 0, device memory otherwise.  Device memory
 * and pinned, mapped host memory are written by a re-layout kernel (host
 * memory through its mapped device address); pageable host memory by one
 * strided copy.  Synchronises the handle's stream and reports any
 * asynchronous error. */
int heat_read(hs_heat_t h, void* dst, int dst_is_device);

/* Steps applied since the last heat_upload. */
int heat_steps_done(hs_heat_t h, int64_t* steps);

/* The temporal depth the handle runs with (tdepth resolved: 1 = the Interior
 * + Boundary kernels every step, L >= 2 = L steps per pass). */
int heat_get_tdepth(hs_heat_t h, int32_t* tdepth);

/* Planes each block of the one-step Interior kernel takes (the k-chunk of
 * Section 6.1's k-split, applied within one GPU): planes >= 1 sets it (capped
 * at the interior's nz - 2), 0 restores the library's choice.  It changes
 * speed only -- every point is computed the same way -- and does not apply to
 * temporally blocked passes.  heat_get_kchunk reports the value in use. */
int heat_set_kchunk(hs_heat_t h, int32_t planes);
int heat_get_kchunk(hs_heat_t h, int32_t* planes);

/* Release the handle (Algorithm "1-GPU Baseline", freeing the device arrays
 * after the time loop): synchronises its stream and frees what the library
 * allocated; caller-owned dev_buf0/dev_buf1 are left to the caller. */
int heat_destroy(hs_heat_t h);

/* ---- batched heat stepping ---------------------------------------------- */
/* Many independent grids -- their own sizes, r and step counts, FP64 or FP32
 * -- advanced together in ONE persistent kernel launch (optionally replayed
 * from a captured CUDA graph).  Each grid is a heat handle (plain HS_F64 or
 * HS_F32, not HS_FIXED64) whose field has been uploaded; a run advances
 * grid i by steps[i] steps of the update of Section 4, Eq. 4 -- the work of
 * the Interior and Boundary kernels of each step -- with the same per-point
 * arithmetic as heat_step, so the results match running each grid alone bit
 * for bit.  Work items are (step, grid, column tile -- FP64 64 x 8 or 32 x 16,
 * FP32 64 x 16 or 32 x 32 --, chunk of planes) taken from a device work counter; each item stages its planes in
 * shared memory (converted once in the exact-sum FP64 arithmetic); a grid's step starts once its previous step is complete, a wait
 * that is bounded (about a second), after which heat_batch_wait reports
 * HS_ETIMEOUT. */
typedef struct hs_batch* hs_batch_t;

/* Build the batch and its step-major work schedule.  grids[0..n) must be
 * distinct and outlive the batch; steps[i] >= 0.  The batch runs on `stream`
 * (each grid's own stream is synchronised before a run). */
int heat_batch_create(hs_batch_t* out, const hs_heat_t* grids, const int64_t* steps, int32_t n,
                      void* stream);

/* heat_batch_create with the work split chosen per grid.  kz[i] >= 1 splits
 * each step of grid i into z-chunks of kz[i] planes (each chunk of each column
 * tile is one item); 0 leaves it to the library (chunks of 32 planes).
 * tile_w[i] is the column tile width: 64 (64 x 8 columns for FP64 grids,
 * 64 x 16 for FP32), 32 (32 x 16, FP32 32 x 32) or 0 for the
 * library's choice (the one that stages fewer values per plane, so narrow
 * grids keep their warps busy).  Either array may be NULL (all 0).  The split
 * changes speed only: every point is computed the same way. */
int heat_batch_create_tiled(hs_batch_t* out, const hs_heat_t* grids, const int64_t* steps,
                            const int32_t* kz, const int32_t* tile_w, int32_t n, void* stream);

/* Enqueue one run: every grid advances by its steps (asynchronous; the
 * handles' step counters and current buffers are updated at once).  With
 * use_graph != 0 the first run captures [clear counters, persistent launch]
 * into a CUDA graph that later runs replay. */
int heat_batch_run(hs_batch_t b, int use_graph);

/* Synchronise the batch stream; HS_ETIMEOUT if a bounded wait ran out. */
int heat_batch_wait(hs_batch_t b);

/* The limit, in SM clock cycles, of the bounded step wait of batches created
 * after this call (0 restores the default of about one second at GB300
 * clocks).  A wait that runs out makes the run stop early: every block
 * finishes the item it holds and takes no other, heat_batch_wait returns
 * HS_ETIMEOUT, and the grids' fields are not valid until they are uploaded
 * again.  Nothing else is affected: the handles, the batch and the CUDA
 * context stay usable.  Meant for tests of that error path (a limit of a few
 * cycles makes a multi-step batch's waits run out).  Errors: HS_EINVAL for a
 * negative limit. */
int heat_batch_set_wait_limit(int64_t cycles);

/* Lattice-point updates per run, and blocks of the persistent launch. */
int heat_batch_info(hs_batch_t b, int64_t* lups, int32_t* blocks);

int heat_batch_destroy(hs_batch_t b);

/* ---- conjugate gradients (Section 7.5) --------------------------------- */
#define HS_OP_STENCIL7 0   /* matrix-free 7-point Dirichlet Laplacian on nx*ny*nz */
#define HS_OP_CSR      1   /* CSR matrix (rowptr, col, val), int32 indices        */

typedef struct {
    int32_t        kind;      /* HS_OP_STENCIL7 or HS_OP_CSR                     */
    int32_t        nx, ny, nz;/* STENCIL7: interior grid (n = nx*ny*nz)          */
    int64_t        n;         /* rows = unknowns (CSR; for STENCIL7 n = nx*ny*nz) */
    int64_t        nnz;       /* CSR entries                                     */
    const int32_t* rowptr;    /* CSR row starts, n+1 entries, rowptr[0] = 0      */
    const int32_t* col;       /* CSR column indices, nnz entries, each in [0, n) */
    const void*    val;       /* CSR values, nnz entries of dtype               */
    int32_t        dtype;     /* HS_F64                                          */
    int32_t        host;      /* 0: rowptr/col/val are device memory; 1: host
                                 memory that cg_create copies to the device     */
} hs_op;

typedef struct {
    int32_t iters;          /* CG iterations taken (mixed: inner iterations)  */
    int32_t status;         /* HS_OK or HS_ENOCONV                            */
    double  relres_recur;   /* sqrt(r.r)/||b|| of the recurrence at exit      */
    double  relres_true;    /* ||b - A x|| / ||b|| recomputed at exit         */
    int32_t refinements;    /* mixed precision: FP64 refinement steps; 0 for FP64 CG */
    int32_t reserved;
} hs_cg_info;

/* Options of the mixed-precision solver (zero fields take the defaults). */
typedef struct {
    double  inner_rtol;     /* each FP32 inner solve stops once its residual fell
                               by this factor; in (0, 1), default 1e-4          */
    int32_t max_inner;      /* cap on iterations of one inner solve (default 2^20) */
    int32_t reserved;
} hs_cg_mixed_opts;

typedef struct hs_cg* hs_cg_t;

/* y = A p on the device (the SpMV of a CG iteration, Algorithm "spmv" (b)
 * for CSR).  p and y are device arrays of n FP64 values; A's arrays must be
 * device memory (host == 0). */
int op_apply(const hs_op* A, const void* p, void* y, void* stream);

/* One SpMV of a CG iteration on its own: q = A p fused with the dot product
 * p.q (Section 7.5; Algorithm "spmv" (b) for CSR), through exactly one launch
 * of the kernel named by `kernel`, with the block count and work order cg_run
 * uses for A, so q and p.q are bit for bit what that kernel computes inside a
 * solve.  p's scale (its largest exponent, which the exact-sum kernels read)
 * is taken from p first, as the kernels that form p record it during a solve.
 *   HS_SPMV_AUTO    the kernel cg_run picks for A, p and q;
 *   HS_SPMV_ROWS    one row per thread in FP64 arithmetic (matrix-free: the
 *                   sum ((zm + ym) + (xm + xp)) + (yp + zp), then
 *                   fma(6, p, -sum); CSR: the row loop with FMA);
 *   HS_SPMV_STAGED  matrix-free only: planes staged in shared memory by
 *                   loads, the exact-sum arithmetic described at cg_run;
 *   HS_SPMV_TMA     matrix-free only: the same, planes staged by TMA; needs
 *                   nx even and p, q 16-byte aligned (else HS_EINVAL).
 * The staged kernels accept any grid size here (cg_run takes them only from
 * about 160^3 up).  p and q are device arrays of n FP64 values that must not
 * overlap; A's arrays must be device memory.  pq (may be NULL) receives p.q.
 * Allocates a few kilobytes of scratch on the stream, synchronises the stream.
 * Errors: HS_EINVAL, HS_ENOMEM, HS_ECUDA, HS_ETIMEOUT (a bounded wait of the
 * TMA-staged kernel ran out). */
#define HS_SPMV_AUTO   0
#define HS_SPMV_ROWS   1
#define HS_SPMV_STAGED 2
#define HS_SPMV_TMA    3
int cg_spmv(const hs_op* A, const void* p, void* q, int kernel, double* pq, void* stream);

/* Create a CG context: checks A, takes a device copy of A's arrays when
 * A->host == 1 (otherwise it keeps A's device pointers, which must outlive
 * the context), and allocates the workspace (r, p, q, reduction partials and
 * device scalars).  Errors: HS_EINVAL, HS_ENOMEM, HS_ECUDA. */
int cg_create(hs_cg_t* out, const hs_op* A, void* stream);

/* Solve A x = b by unpreconditioned FP64 CG (textbook form, Section 7.5):
 * r0 = b - A x0, p0 = r0; each iteration q = A p, alpha = rho/(p.q),
 * x += alpha p, r -= alpha q, rho' = r.r, stop when sqrt(rho')/||b|| <= rtol,
 * else p = r + (rho'/rho) p.  x holds x0 on entry (zeros allowed) and the
 * last iterate on exit.  b and x are host arrays if host_buffers != 0 (copied
 * in and out on the context's stream: by a copy kernel through the mapped
 * address when they are pinned, mapped host memory, else by cudaMemcpyAsync),
 * device arrays otherwise.  Dot products
 * accumulate in FP64 in a fixed order, so repeated runs agree bit for bit.
 * For the matrix-free operator the SpMV forms 6p - (sum of the neighbours)
 * exactly in 64-bit fixed point on p's current scale (its largest exponent,
 * tracked on the device) and rounds it once to FP64 -- error below
 * 24 2^-57 max|p| plus one rounding, where FP64 arithmetic rounds about seven
 * times; a p whose exponents fall outside the convertible range (see
 * HS_FP64_PIPE) takes FP64 arithmetic.  op_apply always computes in FP64.
 * On grids large enough for the shared-memory-staged SpMV, an even nx lets
 * the kernel stage p by TMA (same results bit for bit; a bounded wait in it
 * that runs out stops the solve with HS_ETIMEOUT).
 * Synchronises the stream.  Returns HS_OK when converged, HS_ENOCONV when
 * max_iter iterations ran without reaching rtol (x and info are still
 * filled), or an error code.  info may be NULL. */
int cg_run(hs_cg_t c, const void* b, void* x, int host_buffers, double rtol, int32_t max_iter,
           hs_cg_info* info);

/* Create a mixed-precision CG context: cg_run on it solves A x = b to rtol by
 * FP64 iterative refinement around FP32 CG -- r = b - A x in FP64, an inner CG
 * with its Krylov vectors (d, r', p, q) and operator in FP32 solves A d = r,
 * reducing its residual by inner_rtol or by just what reaching rtol needs
 * (with a factor-2 margin), whichever is less, x += d in FP64, repeat.  Dot products accumulate in FP64 (each
 * thread promotes after at most 4 FP32 products, or keeps an exact FP32
 * two-sum pair that it converts once); alpha, beta and the residual norms are
 * FP64.  The stop test and info->relres_true use the FP64 residual,
 * so the returned x meets rtol in FP64 terms; info->iters counts inner
 * iterations (max_iter bounds them) and info->refinements the inner solves.
 * A CSR operator's values are rounded to an FP32 copy the context owns.
 * Refinement converges while cond(A) times 2^-24 is well below one.  Use
 * cg_run and cg_destroy as for cg_create.  (The precision split extends the
 * paper's FP64 CG of Section 7.5.) */
int cg_create_mixed(hs_cg_t* out, const hs_op* A, const hs_cg_mixed_opts* opts, void* stream);

/* Release a CG context (synchronises its stream). */
int cg_destroy(hs_cg_t c);

/* Batched CG: n independent systems (each its own operator, device b and x)
 * solved together -- three kernel launches per iteration for the whole batch.
 * Each system uses the row partition and reduction order its own cg_run
 * would use, so its results equal solving it alone bit for bit; a system
 * stops when it reaches rtol or max_iter while the others go on.  infos (may
 * be NULL) receives one hs_cg_info per system.  Returns HS_OK when every
 * system converged, HS_ENOCONV if any did not (x and infos filled anyway).
 * Operators must be device memory and outlive the batch. */
typedef struct hs_cg_batch* hs_cg_batch_t;
int cg_batch_create(hs_cg_batch_t* out, const hs_op* ops, int32_t n, void* stream);
int cg_batch_run(hs_cg_batch_t b, const void* const* bs, void* const* xs, double rtol,
                 int32_t max_iter, hs_cg_info* infos);
int cg_batch_destroy(hs_cg_batch_t b);

/* One-shot form of the CG solve of Section 7.5 (textbook unpreconditioned
 * CG, stopping on ||r_k|| / ||b|| <= rtol): cg_create + cg_run (device b and
 * x) + cg_destroy. */
int cg_solve(const hs_op* A, const void* b, void* x, double rtol, int32_t max_iter,
             hs_cg_info* info, void* stream);

/* ---- allocation-free CG (the paper has no counterpart) ------------------- */
/* Largest system cg_solve_noalloc accepts: 2,097,152 unknowns (a 128^3 grid). */
#define HS_NOALLOC_MAX_N 2097152

/* cg_solve for callers that cannot allocate memory while they solve -- for
 * example a serving loop that reserved its device memory up front and must
 * not let cudaMalloc/cudaFree synchronise the device under its other streams,
 * or code running under another framework's memory manager or fixed budget.
 * Same arguments, same kernels and the same results as cg_solve; it calls no
 * cudaMalloc, cudaFree, cudaMallocHost or other allocating routine.  The
 * solver's scratch (r, p, q, reduction partials, device scalars) lives in one
 * fixed array of about 50 MB inside the library, which every GPU that loads
 * the library holds until the process exits.
 *   - A's arrays, b and x must be device memory (A->host == 0).
 *   - n > HS_NOALLOC_MAX_N is rejected with HS_EINVAL before any work.
 *   - The first call on a device does a one-time set-up on that device (it
 *     looks up the scratch array's device address and keeps it for the rest
 *     of the process); make that first call before any stream capture.  The
 *     kept address belongs to the device's current context: after
 *     cudaDeviceReset on that device it is stale, so do not call
 *     cg_solve_noalloc in a process that has reset the device.
 *   - Every call, on any stream, uses the same scratch array.  Calls whose
 *     work overlaps on the GPU race and corrupt each other's results:
 *     serialise them (one stream, or events between streams).  Each call
 *     clears what must start at zero, so it does not depend on what an
 *     earlier call left behind.
 *   - Synchronises the stream.  Returns HS_OK, HS_ENOCONV, or an error code. */
int cg_solve_noalloc(const hs_op* A, const void* b, void* x, double rtol, int32_t max_iter,
                     hs_cg_info* info, void* stream);

/* ---- misc ---------------------------------------------------------------- */
/* Message describing the last error on the calling thread ("" if none).  The
 * paper judges a run by comparing its result with a CPU reference (Section
 * 6.1.7) and has no error interface; this string and the HS_E* codes are the
 * library's own. */
const char* hs_last_error(void);
/* Library ABI version (major*10000 + minor*100 + patch). */
int hs_version(void);
/* Number of kernel launches this library has issued in this process. */
int64_t hs_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* HEATCG_H */
