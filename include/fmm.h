/*
 * fmm.h -- C ABI of the GB300-native unigrid fast-multipole Poisson solver.
 *
 * The solver computes the gravitational potential of a density sampled on an
 * isolated (vacuum-boundary) uniform grid by the cell-based fast multipole
 * method of Lee & Teyssier, "A Scalable Fast Multipole Method Poisson Solver
 * for the RAMSES code: I. Unigrid Algorithm":
 *
 *   P2M    multipoles of each leaf box of b^3 cells        (Sec. 2.1, eq. multipole)
 *   M2M    shift of multipoles up the FMM grid hierarchy   (Sec. 2.1, eq. M2M_general)
 *   M2L    intermediate field over the fixed 189-box list  (Sec. 2.2; Sec. 2.3, eq. M2L)
 *   L2L    far field moved from parent to child centres    (Sec. 2.3, eq. L2L)
 *   L2P    local expansion evaluated at the cell centres   (Sec. 2.3)
 *   P2P    softened cell-cell direct sum over the 27 near  (Sec. 2.3, eq. direct)
 *          leaf boxes (self cell included: g(0) = -1/dx)
 *   accel  a = -grad(phi) by the 5-point stencil            (App. C)
 *
 * so that   phi(x_i) = G dx^2 [ sum_far L2P + sum_{j near i} rho_j g(x_i - x_j) ]
 * with rho a mass density (cell mass = rho dx^3) and g(r) = -1/|r| in cell
 * units.  Expansions are Cartesian Taylor series truncated at
 * |alpha| + |beta| <= order (multipole order + local order <= order), which
 * makes the solve a symmetric linear operator.
 *
 * Conventions for every entry point:
 *  - Arrays are C-contiguous [nz][ny][nx] (x fastest); accel is [3][nz][ny][nx]
 *    (a_x block, then a_y, then a_z).
 *  - Element type: double for FMM_FP64, float for every other precision.
 *  - Device pointers are owned by the caller, must stay valid until the work
 *    enqueued on `stream` has finished, and must be 16-byte aligned.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Every call
 *    is asynchronous on that stream unless stated otherwise; none allocates
 *    device memory after fmm_plan() (fmm_solve_host and fmm_solve_host_many
 *    allocate their staging buffers on first use, see there).
 *  - Argument errors are reported synchronously by the return code; the text
 *    of the most recent error of the calling thread is fmm_last_error().
 *  - Device-side conditions (non-finite input, a spin-wait that gave up) are
 *    latched in the plan and reported by fmm_check() after the stream has
 *    been synchronised.
 */
#ifndef FMM_GB300_H
#define FMM_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fmm_plan_s* fmm_plan_t;

typedef enum {
  FMM_OK = 0,
  FMM_ERR_ARG = 1,          /* invalid argument (NULL, sizes, alignment, order) */
  FMM_ERR_UNSUPPORTED = 2,  /* valid but not supported by this build/device */
  FMM_ERR_ALLOC = 3,        /* device or host allocation failed */
  FMM_ERR_CUDA = 4,         /* a CUDA runtime call failed */
  FMM_ERR_NONFINITE = 5,    /* the density held NaN or Inf (fmm_check) */
  FMM_ERR_TIMEOUT = 6       /* a device spin-wait reached its limit (fmm_check) */
} fmm_status;

/* Arithmetic of the solve. */
typedef enum {
  FMM_FP64 = 0,        /* every step in FP64 on the CUDA cores; data are double */
  FMM_FP32 = 1,        /* every step in FP32 on the CUDA cores ("plain")        */
  FMM_M2L_TF32 = 2,    /* M2L on tcgen05 tensor cores, TF32 inputs, FP32
                          accumulation; the n_fp64_levels coarsest M2L levels on
                          the CUDA cores (FP32, or FP64 with coarse_fp32 = 0);
                          everything else FP32                                  */
  FMM_M2L_BF16X3 = 3   /* as FMM_M2L_TF32 with the M2L operands split into
                          bf16 hi + lo parts and three products
                          (hi*hi + hi*lo + lo*hi), FP32 accumulation             */
} fmm_precision;

typedef struct {
  int nx, ny, nz; /* cells per axis, each a multiple of `leaf`                    */
  double dx;      /* cell size (physical units); phi scales as G dx^2, accel G dx */
  double G;       /* gravitational constant                                      */
} fmm_grid;

typedef struct {
  int precision;      /* fmm_precision                                          */
  int n_fp64_levels;  /* mixed precisions: coarsest M2L levels kept off the
                         tensor cores (levels 2 .. 1+n_fp64_levels, never the
                         leaf level), in the precision coarse_fp32 selects;
                         default 3                                              */
  int accel;          /* 0: no accel output; 1: accel = -grad(phi) by the
                         5-point stencil (App. C); 2: analytic accel, the
                         gradient of the leaf local expansions plus the
                         near-field pair forces m (x - y)/|x - y|^3 between
                         distinct cells (no self force); with final_stage 1
                         also the gradient of the leaf interaction list's M2P
                         at the cell centres.  With 2, the near field (and
                         the M2P) computes four columns per cell           */
  int final_stage;    /* 0: M2L + L2P at the leaf level too; 1: the paper's own
                         final stage (Sec. 4): the leaf interaction list is
                         evaluated by M2P at the cell centres (more accurate,
                         ~6x the leaf-level work).
                         The truncated M2P operator is not symmetric: its
                         transpose (P2L, the leaf cells' own sources expanded
                         about the listed boxes' centres) is what
                         fmm_solve_adjoint runs at the leaf level           */
  int m2l_cartesian;  /* 0 (default): the M2L (tensor cores, and the CUDA
                         cores of FMM_FP32 / FMM_FP64; the FP64 levels of the
                         mixed precisions stay Cartesian) and the tensor-core
                         M2P contract the (p+1)^2 harmonic components
                         (multipoles folded by the Laplace identity of the
                         derivatives of 1/r, which keeps the total order; the
                         remaining locals rebuilt from the same identity before
                         L2L): the same truncated operator of Sec. 2.3, eq.
                         M2L, up to rounding, with 1.7x fewer products at
                         p = 6.  1: all nc(p) Cartesian components            */
  int mult_order;     /* -1 (default) or >= order: multipoles to `order`, the
                         symmetric truncation |alpha| + |beta| <= order.  0 ..
                         order-1: multipole components above mult_order take
                         no part in M2L / M2P (locals stay to `order`): the
                         paper keeps multipoles to 2 and locals to 3 (Sec. 2.1,
                         2.3), i.e. order 3, mult_order 2.  Not symmetric: its
                         transpose swaps the two limits, so such a plan also
                         holds M2L weights with locals to mult_order, which
                         fmm_solve_adjoint runs.  Start from fmm_default_opts
                         (a zeroed struct means monopoles only)               */
  int coarse_fp32;    /* mixed precisions: the coarse M2L levels (n_fp64_levels
                         of them) are kept off the tensor cores for accuracy
                         (they carry the bulk of phi, where the split
                         products' error counts most); 1 (default): in FP32
                         on the CUDA cores, harmonic components, which
                         already gives that accuracy (512^3 p = 6 bf16x3:
                         6.7e-7 against the oracle, 7.40 ms a step); 0: in
                         FP64, Cartesian (6.2e-7, 7.98 ms: at 1.25 TFLOP/s the
                         FP64 work runs beside the tensor-core levels and
                         slows them; at p = 8 it sets the step, 22.7 against
                         11.95 ms)                                           */
  int reserved[1];    /* must be zero */
} fmm_opts;

/* Default options: FMM_FP32, n_fp64_levels = 3, accel = 1, mult_order = -1,
 * coarse_fp32 = 1. */
void fmm_default_opts(fmm_opts* opts);

/*
 * fmm_plan -- build a solver for one grid shape.
 *   grid   : grid extents, cell size and G (read during the call only).
 *   order  : expansion order p, 0 <= p <= 8 (|alpha|+|beta| <= p).
 *   leaf   : cells per leaf-box side b (the paper's 2^dl), one of 2, 4, 8.
 *   opts   : NULL for fmm_default_opts().
 *   stream : stream used for the table uploads.
 *   out    : receives the plan; the plan owns its tables and workspace arena
 *            (device memory sized by fmm_workspace_bytes()).
 * The hierarchy follows Sec. 2: the finest FMM level has (n/b) boxes per axis,
 * each coarser level halves the box count (rounding up; boxes past the domain
 * carry no mass) until one box remains.  The M2L translation kernels are
 * precomputed once, for the unit box, from the fixed interaction geometry
 * (Sec. 2.2).  Errors: FMM_ERR_ARG, FMM_ERR_UNSUPPORTED (no sm_103 device for a
 * tensor-core precision), FMM_ERR_ALLOC, FMM_ERR_CUDA.
 */
fmm_status fmm_plan(const fmm_grid* grid, int order, int leaf, const fmm_opts* opts, void* stream,
                    fmm_plan_t* out);

/*
 * fmm_solve -- phi (and optionally accel) of the density rho.
 *   rho   : device, [nz][ny][nx] density (read only).
 *   phi   : device, [nz][ny][nx] potential (written).
 *   accel : device, [3][nz][ny][nx] or NULL; -grad(phi) by the 4th-order
 *           5-point central stencil (App. C), 2nd-order central one cell from
 *           an edge and 2nd-order one-sided at the edge.
 * Runs P2M, M2M, M2L+L2L per level, P2P+L2P and the stencil as kernels on
 * `stream`; no host synchronisation, no allocation.  Errors: FMM_ERR_ARG,
 * FMM_ERR_CUDA (launch failure).
 */
fmm_status fmm_solve(fmm_plan_t plan, const void* rho, void* phi, void* accel, void* stream);

/*
 * fmm_solve_adjoint -- gradient of a loss with respect to rho.
 *   grad_phi   : device [nz][ny][nx], dLoss/dphi (read only).
 *   grad_accel : device [3][nz][ny][nx] dLoss/daccel, or NULL.
 *   grad_rho   : device [nz][ny][nx] (written): A^T (grad_phi - FD^T grad_accel/dx) G dx^2
 *                with the stencil force (accel = 1); with the analytic force
 *                (accel = 2) the transpose of (phi, accel) applied to
 *                (grad_phi, grad_accel).
 * With |alpha|+|beta| <= order the FMM operator A is symmetric (Green's
 * function symmetry, Sec. 2.3), so A^T is the same chain of kernels applied to
 * the adjoint source; the stencil transpose FD^T is its own kernel.  The
 * analytic force's transpose enters the same chain: its L2P gradient
 * transposed is a dipole source in the P2M (and, with final_stage = 1, the
 * force columns of the P2L), its near pair forces transposed join the near
 * field's contraction (four input columns per cell, on the CUDA cores).  The
 * two truncations that break the symmetry run their transposes: final_stage =
 * 1 replaces the leaf M2P by P2L, and mult_order < order runs the M2L with the
 * multipole and local limits swapped.  Errors: FMM_ERR_ARG, FMM_ERR_CUDA.
 *
 * A plan runs one call at a time: fmm_solve, fmm_solve_adjoint,
 * fmm_solve_host, fmm_solve_host_many and fmm_plan_autotune share the plan's
 * workspace arena (and the adjoint switches the plan's M2L weights for its
 * duration), so calls on one plan are made from one host thread at a time and
 * ordered on one stream.
 * Separate plans are independent.
 */
fmm_status fmm_solve_adjoint(fmm_plan_t plan, const void* grad_phi, const void* grad_accel, void* grad_rho,
                             void* stream);

/*
 * fmm_solve_host -- fmm_solve with HOST buffers: copies rho host->device,
 * solves, copies phi (and accel) device->host, all on `stream`, then
 * synchronises `stream` before returning.  Pinned host memory gives full
 * copy bandwidth; pageable memory works but is slower.  The first call
 * allocates device staging buffers owned by the plan (freed by
 * fmm_plan_destroy).
 */
fmm_status fmm_solve_host(fmm_plan_t plan, const void* rho_host, void* phi_host, void* accel_host, void* stream);

/*
 * fmm_solve_host_many -- `count` independent densities through one plan,
 * HOST buffers: field i's rho_host[i] is solved into phi_host[i] (and
 * accel_host[i]), each with the plan's layout and element type
 * ([nz][ny][nx], accel [3][nz][ny][nx]; FP32, FP64 for FMM_FP64 plans).  The
 * results equal fmm_solve_host's field by field.  The copies overlap the
 * solves: two device staging sets (owned by the plan, allocated by the first
 * call, freed by fmm_plan_destroy), uploads on one copy stream and downloads
 * on another, so that field i + 1's upload and field i's download run beside
 * the solve of field i + 1; the solves themselves run one after another on
 * `stream`, after the work already queued there.  A pointer may repeat (the
 * same input or output buffer for several fields; output buffers that repeat
 * hold the last such field).  Pinned host memory is needed for the overlap;
 * pageable buffers work, without it.  Returns after every copy has finished,
 * also on error.  accel_host NULL: no acceleration.  count = 0 does nothing.
 * Errors: FMM_ERR_ARG (NULL plan or buffer, negative count), FMM_ERR_ALLOC,
 * FMM_ERR_CUDA, and fmm_solve's.
 */
fmm_status fmm_solve_host_many(fmm_plan_t plan, int count, const void* const* rho_host, void* const* phi_host,
                               void* const* accel_host, void* stream);

/*
 * fmm_solve_static -- the same FP32 solve as fmm_solve (CUDA-core kernels,
 * FMM_FP32 arithmetic, 5-point accel), for callers that cannot allocate
 * device memory.  The paper has no counterpart: this entry point only
 * changes where the solver's workspace lives.
 *
 * Who needs it: code that must not call cudaMalloc while it runs -- for
 * example a hot loop with a latency budget (cudaMalloc may synchronise the
 * whole device), code running inside a framework whose caching allocator
 * owns the device memory budget, or a plug-in whose host application forbids
 * device allocation after start-up.  Those callers cannot create a plan
 * (fmm_plan allocates its tables and arena), so this call takes no plan and
 * allocates nothing: no cudaMalloc, no cudaFree, no allocating library call.
 *
 * Workspace: one static device array of FMM_STATIC_WORKSPACE_BYTES (16 MiB)
 * compiled into this library.  Every device on which the library is loaded
 * holds that array until the process exits.  A solve fits when its tables
 * plus its arena fit the array: at leaf 4 that is up to 64^3 cells for
 * orders <= 6.  Orders above 6 and grid extents above 4096 return
 * FMM_ERR_ARG before any device work; a grid whose tables and arena do not
 * fit returns FMM_ERR_ARG (the byte count in fmm_last_error()) while the
 * array is being laid out, after some of its clearing and table copies may
 * already be queued on `stream` -- the array's tables are then marked stale
 * and rebuilt by the next call, but a call still running on another stream
 * would read them being overwritten (see the note on overlapping calls).
 *
 *   grid, order, leaf : as fmm_plan (order <= 6).
 *   rho, phi, accel   : device float arrays as fmm_solve (accel may be NULL),
 *                       16-byte aligned, owned by the caller.
 *   stream            : cudaStream_t for every copy and kernel of the call.
 *
 * Set-up: every call looks up the array's device address
 * (cudaGetSymbolAddress, with the device current; no allocation) and
 * rebuilds the tables when the address changed (after a device reset); make
 * the first call on a device before any stream capture.  The call keeps the array's tables from the
 * previous call when order, leaf and grid are unchanged (otherwise it
 * rebuilds them on the host and copies them in), and clears every part of
 * the array that must start at zero.  All calls share one array: calls whose
 * work overlaps on the GPU (other streams, other host threads) race and give
 * wrong results; order them on one stream.  Device-side flags (non-finite
 * input) are not reported: there is no plan to hold them.
 */
#define FMM_STATIC_WORKSPACE_BYTES (16u << 20)
fmm_status fmm_solve_static(const fmm_grid* grid, int order, int leaf, const void* rho, void* phi, void* accel,
                            void* stream);

/*
 * Autotuning of the CUDA-core contractions: the M2L levels that are not on
 * the tensor cores (Sec. 2.3, eq. M2L) and the near-field sum (Sec. 2.3, the
 * direct cell-cell part), when it is not on the tensor cores.
 *   fmm_plan_autotune   : times every applicable variant of each contraction
 *                         on the plan's own workspace (3 timed launches after
 *                         one warm-up) and keeps the fastest.  Overwrites the
 *                         workspace (no solve state survives a solve anyway);
 *                         synchronises `stream`.  Results are cached per
 *                         process by contraction geometry (grid of rows, row
 *                         length, columns, order, leaf), so further plans of
 *                         the same shape only look the choice up.
 *   fmm_plan_tuning     : reads the variant of level `level` (2..leaf level;
 *                         -1 = near field): shape 0 = 4x4x4 rows per block,
 *                         shapes 1 and 2 = z-run register tiles
 *                         (8x4x8 / 8x4x4 rows for FP32, 8x4x4 / 8x4x2 for
 *                         FP64), shape 3 = one output column per lane, 16
 *                         rows per block, no shared memory (the coarse FP64
 *                         levels of the tensor-core precisions default to
 *                         it; shapes 1 and 2 are not used there), and the
 *                         number of blocks sharing the 27 neighbours of a row
 *                         tile (shapes 0, 3: 1 or 27; shapes 1, 2: 1, 3 or 9).
 *   fmm_plan_set_tuning : sets it; FMM_ERR_ARG if the variant does not apply
 *                         (level on the tensor cores, reduction lengths not a
 *                         multiple of 8, split scratch too small).
 * All variants compute the same sums; they differ in summation order only
 * through the neighbour split (partials added in a fixed order).
 * The paper has no counterpart (its M2L runs on CPU cores).
 */
fmm_status fmm_plan_autotune(fmm_plan_t plan, void* stream);

/*
 * Tensor-core schedules.  Each tensor-core contraction -- `what` 0: the M2L
 * of the tensor-core levels (Sec. 2.3, eq. M2L), 1: the near field (Sec. 2.3,
 * the direct cell-cell part), 2: the final-stage M2P (Sec. 4) -- has up to two
 * schedules with the same arithmetic: the span schedule (k_m2l_tc.cu: column
 * groups of one order range, one MMA per group and K step) and the prefix
 * schedule (k_nbr_tc.cu: all columns of a pass in one accumulator set, one
 * wide MMA per K step over the prefix of columns it feeds).  The near field
 * of leaf-4 plans without the analytic force also has a third, dedicated
 * kernel (k_near_tc.cu: four row tiles per weight copy, one accumulation
 * segment per neighbour column).  A plan starts with the one measured
 * fastest on GB300 at 512^3 (M2L and M2P: prefix; near field: the dedicated
 * kernel where it exists, else span) and fmm_plan_autotune times them all.
 *   fmm_plan_tc_schedule     : *available = bit 0 span, bit 1 prefix, bit 2
 *                              dedicated; *prefix = 2 dedicated, 1 prefix,
 *                              0 span, -1 none (the contraction is not on the
 *                              tensor cores).  Either pointer may be NULL.
 *   fmm_plan_set_tc_schedule : selects one (`prefix` 0, 1 or 2 as above);
 *                              FMM_ERR_ARG if that schedule does not exist
 *                              for the contraction (or, for the M2L of a plan
 *                              with mult_order < order, for its transposed
 *                              form).
 * All schedules give the same sums up to the order of the FP32 additions.
 * The paper has no counterpart.
 */
fmm_status fmm_plan_tc_schedule(fmm_plan_t plan, int what, int* prefix, int* available);

/*
 * fmm_plan_debug_timeout -- test hook for the bounded device waits.  The
 * next solve's first prefix-schedule M2L launch leaves the first activation
 * stage of every CTA unloaded: no copy or MMA is issued for it, so the
 * issuers' wait on it reaches its time limit (2 s) with nothing in flight,
 * the CTAs give up (each lets its own copies land and frees its tensor
 * memory) and fmm_check then returns FMM_ERR_TIMEOUT naming the wait sites.
 * That solve's output is invalid; the plan stays usable and the next solve is
 * an ordinary one.  FMM_ERR_ARG if no M2L level runs the prefix schedule.
 */
fmm_status fmm_plan_debug_timeout(fmm_plan_t plan);
fmm_status fmm_plan_set_tc_schedule(fmm_plan_t plan, int what, int prefix);
fmm_status fmm_plan_tuning(fmm_plan_t plan, int level, int* shape, int* dsplit);
fmm_status fmm_plan_set_tuning(fmm_plan_t plan, int level, int shape, int dsplit);

/*
 * Batched solves (many independent densities, uneven grid sizes).
 *   fmm_batch_create  : groups `count` existing plans (not copied, not owned;
 *                       they must outlive the batch).
 *   fmm_batch_solve   : solves every plan's density with one graph launch.
 *                       rho[i], phi[i] (and accel[i] if `accel` is non-NULL and
 *                       accel[i] is non-NULL) are plan i's device buffers as in
 *                       fmm_solve.  Two forms, chosen per call:
 *                       - fused: when every plan runs all its contractions on
 *                         the CUDA cores (no tensor-core level, near field or
 *                         final-stage M2P), the plans share the order and
 *                         precision, every level holds the data's precision and
 *                         a force, if asked for, is the FP32 stencil on rows of
 *                         a multiple of 4 cells (all buffers 16-byte aligned,
 *                         every accel[i] non-NULL), each step kind of Sec. 2.3
 *                         is one kernel launch over every field: P2M, M2M per
 *                         depth below the leaf level, the M2L levels and near
 *                         fields of all fields together (one launch per
 *                         contraction tile shape, without neighbour split),
 *                         L2L per level, the leaf evaluation and the stencil;
 *                       - otherwise one CUDA graph of the per-plan solves, each
 *                         plan on its own branch.
 *                       The first call with a given set of buffers runs the
 *                       work once, then captures it into a CUDA graph and
 *                       launches that; later calls with the same buffers only
 *                       launch the graph (new buffers: a new capture, and for
 *                       the fused form a new upload of its item table).
 *                       Asynchronous on `stream`.
 *   fmm_batch_set_fused : enable (default) or disable the fused form
 *                       (disabled: always the graph of per-plan solves).
 *   fmm_batch_is_fused : 1 if the batch's current graph is the fused form,
 *                       0 if it is the per-plan one, -1 before the first solve
 *                       (or for a NULL batch).
 *   fmm_batch_destroy : frees the graph, the item table and the batch's
 *                       streams/events (NULL: no-op).
 * Errors: FMM_ERR_ARG (NULL batch, plan or buffer array, a NULL rho[i] /
 * phi[i], count < 1), FMM_ERR_ALLOC (host memory), FMM_ERR_CUDA (stream,
 * event, capture, instantiation or launch failure; the solve errors of
 * fmm_solve pass through from the first, uncaptured run).
 * The batch is the multi-field form of the solve; the paper solves one field
 * per call (this is the data-parallel batch of many problems).
 */
typedef struct fmm_batch_s* fmm_batch_t;
fmm_status fmm_batch_create(const fmm_plan_t* plans, int count, fmm_batch_t* out);
fmm_status fmm_batch_solve(fmm_batch_t batch, const void* const* rho, void* const* phi, void* const* accel,
                           void* stream);
fmm_status fmm_batch_destroy(fmm_batch_t batch);
fmm_status fmm_batch_set_fused(fmm_batch_t batch, int enable);
int fmm_batch_is_fused(fmm_batch_t batch);
/* Kernel launches one fmm_batch_solve graph holds: the fused form's step
 * count when the plans qualify for it (and it is enabled), else the sum over
 * the plans. */
int fmm_batch_launches(fmm_batch_t batch, int with_accel);

/* fmm_check -- synchronises the plan's last stream and reports device-side
 * flags (FMM_ERR_NONFINITE, FMM_ERR_TIMEOUT), clearing them.  FMM_ERR_ARG for
 * a NULL plan, FMM_ERR_CUDA for an error the synchronisation returns. */
fmm_status fmm_check(fmm_plan_t plan);

/* Bytes of device memory the plan holds (tables + workspace arena). */
size_t fmm_workspace_bytes(fmm_plan_t plan);

/* Number of kernel launches one fmm_solve() enqueues for this plan. */
int fmm_solve_launches(fmm_plan_t plan, int with_accel);

/*
 * Per-stage timing with CUDA events recorded on the solve's own stream around
 * every kernel launch (for benchmarks; off by default).
 *   fmm_timing_enable : 1 starts recording (and clears totals), 0 stops.
 *                       Creates its event pool here, not during solves.
 *   fmm_timing_read   : synchronises, then writes for each stage i < nstages
 *                       the summed milliseconds ms[i] and launch count
 *                       launches[i] since the last enable/read, and clears them.
 * Stages (index: name): see fmm_timing_stage_name().  Errors: FMM_ERR_ARG
 * (NULL plan or arrays), FMM_ERR_CUDA (event creation or timing failure).
 */
fmm_status fmm_timing_enable(fmm_plan_t plan, int enable);
fmm_status fmm_timing_read(fmm_plan_t plan, double* ms, int* launches, int nstages);
int fmm_timing_stage_count(void);
const char* fmm_timing_stage_name(int stage);

/* Frees every resource of the plan (synchronises the device first). */
fmm_status fmm_plan_destroy(fmm_plan_t plan);

/* Text of the most recent error on the calling thread ("" if none). */
const char* fmm_last_error(void);

/*
 * fmm_debug_level -- copy one level's expansions to host memory in the
 * canonical layout [box z][box y][box x][coef] (coefficients ordered by total
 * order, then a descending, then b descending), as double, in cell units
 * about each box centre (M_alpha = sum m (x-c)^alpha, L_beta as in eq. M2L).
 *   what: 0 = multipoles M, 1 = local expansions L.  level: 2..L.
 * Synchronises the device.  For tests that localise a mismatch.  Errors:
 * FMM_ERR_ARG (NULL plan, `what` not 0 or 1, a level that is not stored, a
 * host buffer shorter than nbox * ncoef), FMM_ERR_CUDA (copy failure).
 */
fmm_status fmm_debug_level(fmm_plan_t plan, int what, int level, double* host_out, size_t host_count);

/* Number of FMM levels minus one (index of the leaf level), or -1. */
int fmm_plan_leaf_level(fmm_plan_t plan);

/* How the M2L of one level runs: 0 none (levels 0, 1), 1 CUDA cores FP32,
 * 2 CUDA cores FP64, 3 tcgen05 tensor cores; -1 for a bad plan or level. */
int fmm_plan_level_kind(fmm_plan_t plan, int level);

/* 1 when the near field runs on the tensor cores (bf16x3), else 0. */
int fmm_plan_near_on_tensor_cores(fmm_plan_t plan);

#ifdef __cplusplus
}
#endif

#endif /* FMM_GB300_H */
