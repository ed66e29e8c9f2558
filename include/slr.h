/*
 * slr.h -- C ABI of the GB300-native Loop-of-stencil-reduce library (libslr.so).
 *
 * The pattern (Aldinucci et al., "A Parallel Pattern for Iterative Stencil +
 * Reduce", arXiv 1609.04567, Sec. 3.1, procedures loop-of-stencil-reduce-d and
 * -s): repeat { one stencil sweep over the grid; reduce the per-item change
 * (or the new items) with an associative operator; count the iteration } until
 * the convergence test on the reduced value and the iteration count passes.
 * The library runs the sweep, the reduce and the test on one GPU; the loop
 * stays on the device.
 *
 * Conventions for every call:
 *   - Pointers named u, aux, workspace are DEVICE pointers owned by the caller.
 *     The library never allocates, frees or retains device memory beyond the
 *     handle's lifetime; the handle owns only host metadata.
 *   - Grids are dense row-major arrays: item (z, y, x) is at index
 *     (z * ny + y) * nx + x, x contiguous.  u must be 16-byte aligned.
 *   - All device work is enqueued on the CUDA stream given at creation
 *     (a cudaStream_t passed as void*, NULL = legacy default stream) and is
 *     asynchronous; slr_reduce_value() is the only call that waits.
 *   - Calls return an slr_status and never abort.  After an error,
 *     slr_last_error() returns a message.
 *   - A handle is not thread-safe; distinct handles may be used concurrently
 *     from distinct threads on distinct streams.
 */
#ifndef SLR_H
#define SLR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct slr_ctx *slr_handle;

typedef enum {
    SLR_OK = 0,                /* converged (the test, not the cap, stopped the loop) */
    SLR_NOT_CONVERGED = 1,     /* the iteration cap stopped the loop; state is valid */
    SLR_ERR_INVALID_ARG = -1,  /* bad descriptor, pointer or size */
    SLR_ERR_WORKSPACE = -2,    /* workspace smaller than slr_workspace_size() */
    SLR_ERR_CUDA = -3,         /* a CUDA call failed; see slr_last_error() */
    SLR_ERR_TIMEOUT = -4,      /* a device-side wait ran out its limit */
    SLR_ERR_UNSUPPORTED = -5   /* valid but unimplemented combination */
} slr_status;

/* Elemental functions (the f of stencil(sigma_1, f), Sec. 3.1). */
typedef enum {
    /* 2D 5-point Helmholtz Jacobi (Sec. 4.1):
     *   u' = (h^2 f + ((u_N + u_S) + u_W) + u_E) / (4 + sigma h^2)
     * aux = f (same storage type as u). */
    SLR_J2D5 = 0,
    /* 3D 7-point form: u' = (h^2 f + sum of 6 neighbours) / (6 + sigma h^2),
     * neighbours summed x-, x+, y-, y+, z-, z+.  aux = f. */
    SLR_J3D7 = 1,
    /* Game of Life B3/S23 over the 8 Moore neighbours (Fig. 1).  Cells are
     * uint8 0/1 (any non-zero input reads as alive; outputs are 0/1).
     * aux = NULL. */
    SLR_LIFE = 2,
    /* Restoration update of the two-phase denoiser (Sec. 4.3), binary32 state:
     * for masked pixels u' = sum_j w_j u_j / sum_j w_j over the in-range
     * 8-neighbours, w_j = 1/sqrt(alpha + (u - u_j)^2); unmasked pixels are
     * copied.  aux = uint8 mask (non-zero = noisy). */
    SLR_RESTORE8 = 3
} slr_stencil;

/* What lies beyond the grid (the bottom items of the stencil operator). */
typedef enum {
    SLR_DIRICHLET = 0,  /* a fixed ghost value (desc.ghost; Life: dead cell) */
    SLR_WRAP = 1        /* toroidal wrap_around */
} slr_boundary;

/* The reduce operator applied to the per-item change (delta) or item. */
typedef enum {
    SLR_RED_MAX_ABS_DELTA = 0,          /* max |u' - u|, identity 0 (Jacobi) */
    SLR_RED_MEAN_ABS_DELTA_MASKED = 1,  /* sum over mask of |u'-u| (each truncated to a
                                           multiple of 2^-24, summed as uint64) / #mask */
    SLR_RED_LIVE_COUNT = 2              /* live count (+ on uint64) and any-changed (or) */
} slr_reduce_op;

typedef enum { SLR_U8 = 0, SLR_BF16 = 1, SLR_F16 = 2, SLR_F32 = 3, SLR_F64 = 4 } slr_dtype;

/* How the loop is driven. */
typedef enum {
    SLR_LOOP_AUTO = 0,        /* library choice: the autotuner's, else PERSISTENT */
    SLR_LOOP_HOST = 1,        /* plain schema of Fig. 2: one sweep launch, one reduce
                                 launch and a host-side test per iteration */
    SLR_LOOP_PERSISTENT = 2   /* one cooperative launch; sweep, reduce, test and buffer
                                 swap stay on the device, one grid barrier per pass */
} slr_loop;

/* Precision mode of the floating-point elemental functions. */
typedef enum {
    SLR_MATH_EXACT = 0,  /* IEEE ops in the oracle's order, no contraction: bit-exact */
    SLR_MATH_FAST = 1    /* fused multiply-add and hardware approximations allowed */
} slr_math;

typedef struct {
    int32_t stencil;       /* slr_stencil */
    int32_t storage;       /* slr_dtype of u and aux-f: J2D5/J3D7 F64, F32, BF16, F16
                              (BF16/F16 store the state, arithmetic is binary32);
                              LIFE U8; RESTORE8 F32 */
    int32_t reduce;        /* slr_reduce_op; must be the one of the stencil */
    int32_t boundary;      /* slr_boundary */
    int64_t nx, ny, nz;    /* extents, nz = 1 for 2D stencils; each >= 1 */
    double ghost;          /* Dirichlet ghost value (Jacobi) */
    double tol;            /* convergence: stop when reduced value < tol (delta reduces);
                              Life stops when no cell changed */
    double sigma;          /* Helmholtz sigma */
    double h;              /* mesh width; <= 0 selects 1/(nx + 1) */
    float alpha;           /* restoration constant (100) */
    int32_t loop;          /* slr_loop */
    int32_t math;          /* slr_math */
    int32_t temporal_k;    /* sweeps per HBM pass, 1 = one.  Life: 1 .. 32.  SLR_J2D5 with
                              binary32 arithmetic (storage F32, BF16 or F16), a Dirichlet
                              ghost exact in the storage type, rows of whole 16-byte
                              groups: 1 .. 8.  SLR_RESTORE8 with nx a multiple of 16:
                              1 .. 8.  (Larger values run 8; a solve that stops inside a
                              pass recomputes that pass up to the stopping sweep, so
                              results equal those of k = 1.)
                              0 = library choice: the autotuner's, else for Life the
                              largest k in [4, 32] whose tiles fit the co-resident CTAs,
                              for SLR_J2D5 and SLR_RESTORE8 8 when tiling is
                              SLR_TILING_AUTO (1 otherwise) */
    int64_t wait_limit_ns; /* device-side barrier wait limit; <= 0 selects 2 s */
    int32_t debug_flags;   /* SLR_DEBUG_* bits; 0 in normal use */
    int32_t defect_correction; /* 1: FP64 defect correction around FP32 Jacobi inner solves
                                  (SLR_J2D5, storage F64, Dirichlet ghost 0).  One iteration:
                                  inner_sweeps binary32 Jacobi sweeps of A e = r from e = 0,
                                  then u += e and r = f - A u in binary64; the reduced value
                                  is the scaled defect max |h^2 r / (4 + sigma h^2)| (the
                                  change the next FP64 Jacobi sweep would make); stop when
                                  it is < tol or at the cap */
    int32_t inner_sweeps;  /* binary32 sweeps per correction; 0 selects 50 */
    int32_t grid_ctas;     /* CTAs of the persistent launch, capped at the number that can
                              be co-resident; 0 = library choice (all co-resident CTAs).
                              Results do not depend on it. */
    int32_t tiling;        /* slr_tiling of the RESTORE8 and Jacobi persistent sweeps; Life
                              ignores it */
    int32_t reserved;      /* 0 */
} slr_desc;

/* How a persistent sweep stages its input.  Results do not depend on it.
 * RESTORE8: TMA = 32x64 tiles with halo in shared memory (nx a multiple of 16).
 * J2D5/J3D7: TMA = a CTA marches a 256-cell-wide column along y (2D, blocks of
 * rows) or z (3D, plane tiles with their y-halo), every step staged by TMA
 * in a 4-stage ring; needs a Dirichlet ghost of +0, rows of whole 16-byte
 * groups and 16-byte aligned u, f and workspace.  NONE = warps march row
 * segments with the rows in registers (any boundary).  Where TMA does not
 * apply the sweep falls back to NONE. */
typedef enum {
    SLR_TILING_AUTO = 0,   /* library choice: TMA where it applies (Jacobi: grids of at least
                              about 2 x (SMs x 768) 16-byte groups) */
    SLR_TILING_NONE = 1,
    SLR_TILING_TMA = 2
} slr_tiling;

/* Fault injection for tests of the device-side wait limit: the last CTA of a
 * persistent launch leaves before its first barrier arrival, so every other
 * CTA's wait runs out after wait_limit_ns and the run reports SLR_ERR_TIMEOUT.
 * The handle is then unusable (create a new one); the GPU context is not. */
#define SLR_DEBUG_SKIP_ARRIVAL 1

/* Fill *d with defaults for a stencil: the matching reduce operator and
 * storage, Dirichlet ghost 0, tol 1e-6 (Jacobi), 1e-3 (restoration), sigma 1,
 * h = 1/(nx+1), alpha 100, AUTO loop, EXACT math. */
void slr_desc_init(slr_desc *d, int32_t stencil, int64_t nx, int64_t ny, int64_t nz);

/* Bytes of device workspace a handle for *d needs (control block, second
 * state buffer; Life: two bit-packed buffers; defect correction: three binary32
 * buffers; SLR_RESTORE8: one 12,352-byte record per 64 x 64 tile, the tile's
 * noisy-pixel list built in a run's first pass and read by its later ones,
 * the records rounded up to 256 bytes; when nx is not a multiple of 16 also
 * a copy of the mask with rows padded to a multiple of 16 bytes, and when nx
 * is not a multiple of 4 two copies of the state with rows padded to a
 * multiple of 4 floats, each rounded up to 256 bytes: the temporal-blocked
 * loop reads rows that start on 16-byte boundaries).  Returns 0 for an
 * invalid descriptor. */
size_t slr_workspace_size(const slr_desc *d);

/* Create a handle (constructor of Sec. 3.2: elemental function, combinator
 * with identity, iteration condition and sizes).
 *   u          device state, in/out; holds the result after each run.
 *   aux        device f (Jacobi), mask (restoration) or NULL (Life); read-only.
 *   workspace  device buffer of at least slr_workspace_size(d) bytes, 256-byte
 *              aligned, owned by the caller, not touched by anyone else while
 *              the handle lives.
 *   stream     cudaStream_t for all work of this handle.
 * The iteration counter starts at 0.  Enqueues a small workspace reset. */
slr_status slr_create(const slr_desc *d, void *u, const void *aux, void *workspace,
                      size_t workspace_bytes, void *stream, slr_handle *out);

/* Enqueue the loop until the test passes or the TOTAL iteration count of the
 * handle reaches max_iters (a call with a higher cap resumes from the state
 * left in u).  Asynchronous.  A converged handle returns at once. */
slr_status slr_run_until(slr_handle h, int64_t max_iters);

/* Wait for the handle's stream and read the result of the last iteration:
 * reduced value (max or mean |delta|; live count for Life), total iterations,
 * converged flag (1 when the test stopped the loop) and the integer count
 * (live cells for Life, masked pixels for the restoration, else 0).  Any
 * output pointer may be NULL.  Returns SLR_OK when converged,
 * SLR_NOT_CONVERGED when stopped by the cap, or an error (SLR_ERR_TIMEOUT if
 * a device barrier wait ran out). */
slr_status slr_reduce_value(slr_handle h, double *value, int64_t *iters,
                            int32_t *converged, uint64_t *count);

/* Release the handle (host memory only; waits for nothing). */
slr_status slr_destroy(slr_handle h);

/* Message of the last error on h (or of the last failed create when h is
 * NULL).  Never NULL. */
const char *slr_last_error(slr_handle h);

/* ---- Noise detection (the detection phase of the Sec. 4.3 denoiser) ----------
 * The paper's two-phase restoration marks noisy pixels with a traditional
 * adaptive median filter before RESTORE8 restores them (its mask input).  For
 * every pixel z of the uint8 image img (nx x ny, row-major): square windows of
 * side 3, 5, ..., wmax centred on z and clipped to the image give zmin, zmax
 * and zmed, the lower median (element floor((n-1)/2) of the n window values in
 * ascending order); the first window with zmin < zmed < zmax decides: the
 * filter keeps z when zmin < z < zmax and outputs zmed otherwise; when no
 * window qualifies it outputs zmed of the largest window.  mask (uint8, same
 * layout) receives 1 where the output differs from z, else 0.  state, when
 * not NULL, receives the image as binary32 values (float, same layout, 4-byte
 * aligned): the restoration's initial state, written in the same pass.  img,
 * mask and state are device pointers that must not overlap; wmax odd in
 * [3, 15].  Enqueued on `stream` (nothing waits); returns SLR_OK, or
 * SLR_ERR_INVALID_ARG / SLR_ERR_CUDA with the message in slr_last_error(NULL). */
slr_status slr_detect_noise(const void *img, void *mask, void *state, int64_t nx, int64_t ny, int32_t wmax,
                            void *stream);

/* A restored binary32 state (n values, device, 4-byte aligned) written back as
 * a uint8 frame: img[i] = u[i] rounded to the nearest integer (ties to even)
 * and clamped to [0, 255] (NaN gives 0).  Enqueued on `stream`; SLR_OK or SLR_ERR_INVALID_ARG
 * / SLR_ERR_CUDA (message in slr_last_error(NULL)). */
slr_status slr_state_to_frame(const void *state, void *img, int64_t n, void *stream);

/* ---- Sobel edge detector (Sec. 4.2): one stencil sweep, no reduce ----------
 * out (uint8, nx x ny, row-major) = the edge magnitude of the uint8 image img:
 * with the 3x3 gradients Gx = (z[i-1][j+1] - z[i-1][j-1]) + 2 (z[i][j+1] -
 * z[i][j-1]) + (z[i+1][j+1] - z[i+1][j-1]) and Gy = (z[i+1][j-1] - z[i-1][j-1])
 * + 2 (z[i+1][j] - z[i-1][j]) + (z[i+1][j+1] - z[i-1][j+1]) in integers,
 * out = min(255, floor(sqrt(Gx^2 + Gy^2))) where the 3x3 neighbourhood lies in
 * the image and 0 on its border.  img and out are device pointers that must not
 * overlap.  Enqueued on `stream`; SLR_OK or SLR_ERR_INVALID_ARG / SLR_ERR_CUDA
 * (message in slr_last_error(NULL)). */
slr_status slr_sobel(const void *img, void *out, int64_t nx, int64_t ny, void *stream);

/* ---- User-defined elemental functions (Sec. 3.2, Fig. 1) --------------------
 * The paper's pattern takes the elemental stencil and reduce functions from the
 * user as source code compiled for the device at run time.  slr_user_create
 * compiles (NVRTC, sm_103a, no floating-point contraction: every operation
 * rounds as written) CUDA C++ source that defines
 *
 *   __device__ slr_t  slr_update(const slr_nbr &u, slr_t aux, long long i, long long j,
 *                                const double *p);
 *   __device__ double slr_delta(slr_t new_value, slr_t old_value);
 *
 * where slr_t is float (dtype SLR_F32) or double (SLR_F64); u(di, dj) returns
 * the state at row i + di, column j + dj under the boundary rule (the ghost
 * value outside the grid, or wrapped); aux is the item of the aux array (0
 * when aux is NULL); p[0..7] are desc.params.  One iteration sets every item
 * to slr_update(...) of the previous state (ping-pong buffers), reduces
 * slr_delta(new, old) over all items by max (identity -inf, NaN skipped) or
 * sum (identity 0; per-CTA partials then a fold, in a fixed order: the same
 * inputs give the same value on every run), and stops when the value is below
 * tol or at the cap, in one cooperative launch by default or with the host
 * reading the value after every iteration (the schema of Fig. 2; desc.loop).
 * Programs are cached per (source, dtype).  Compile errors
 * return SLR_ERR_INVALID_ARG with the compiler's log in
 * slr_user_last_error(NULL). */
typedef enum { SLR_USER_MAX = 0, SLR_USER_SUM = 1 } slr_user_reduce;

typedef struct {
    int32_t dtype;         /* SLR_F32 or SLR_F64: state and aux elements */
    int32_t boundary;      /* SLR_DIRICHLET (ghost) or SLR_WRAP */
    int64_t nx, ny;        /* extents, row-major, nx contiguous; nx * ny < 2^40 */
    double ghost;          /* value outside the grid for SLR_DIRICHLET */
    double tol;            /* stop when the reduced value < tol */
    int32_t reduce;        /* slr_user_reduce */
    int32_t loop;          /* slr_loop: AUTO or PERSISTENT = the whole loop in one cooperative
                              launch (bounded grid barrier, the test on the device); HOST =
                              a sweep and a fold launch and a host test per iteration.  Both
                              give the same values. */
    double params[8];      /* constants handed to slr_update as p */
} slr_user_desc;

typedef struct slr_user_handle_s *slr_user_handle;

/* Device workspace bytes for d (0 for an invalid descriptor). */
size_t slr_user_workspace_size(const slr_user_desc *d);
/* Compile (or reuse) the program and bind the caller's u (in/out), aux (may be
 * NULL) and workspace (256-byte aligned, slr_user_workspace_size bytes), all
 * device memory owned by the caller; work is enqueued on `stream`. */
slr_status slr_user_create(const slr_user_desc *d, const char *source, void *u, const void *aux, void *workspace,
                           size_t workspace_bytes, void *stream, slr_user_handle *out);
/* Iterate until the test passes or the handle has run max_iters iterations in
 * all (waits for the stream; u holds the state on return).  SLR_OK when
 * converged, SLR_NOT_CONVERGED at the cap. */
slr_status slr_user_run_until(slr_user_handle h, int64_t max_iters);
/* The last iteration's reduced value, the iterations run, the convergence flag. */
slr_status slr_user_reduce_value(slr_user_handle h, double *value, int64_t *iters, int32_t *converged);
slr_status slr_user_destroy(slr_user_handle h);
/* Message of the last error on h (of the last failed create when h is NULL). */
const char *slr_user_last_error(slr_user_handle h);

/* Library build string (architecture, version). */
const char *slr_version(void);

/* ---- Batches: many instances in one persistent launch -----------------------
 * A batch holds up to max_instances independent loops (SLR_J2D5, SLR_J3D7 in
 * any storage, with or without FP64 defect correction, SLR_RESTORE8 in EXACT
 * math), each with its own grid, tolerance and iteration cap.  slr_batch_run
 * enqueues the launches that run up to `sweeps` more steps of every running
 * instance: the Jacobi instances of at most 64K cells (32K with defect
 * correction) each on a thread-block cluster of 1-16 CTAs holding the grid in
 * shared memory (with defect correction: its binary32 defect and
 * corrections), one cluster
 * barrier per sweep or phase (one launch per cluster size,
 * on side streams the batch's stream then waits for), and the others in ONE
 * cooperative launch with one grid barrier per step for all of them: a step
 * is one sweep, or for a defect-correction instance one phase
 * of its loop (the initial defect, one of its inner binary32 sweeps, or the
 * correction with its new defect; its test follows each correction and its
 * iteration count is the number of corrections).  An instance stops when its
 * test passes or its cap is reached (the per-instance -d/-s tests of Sec.
 * 3.1), and its result is then in its u.  Instances may be added and removed between runs,
 * which is how a serving loop admits new work while earlier work is still
 * running (continuous batching).  Results are identical to slr_create runs of
 * the same descriptors.
 *
 * Ownership: the caller owns u, aux and a scratch buffer per instance
 * (slr_batch_scratch_size bytes: the second state buffer, plus the binary32
 * defect and corrections of a defect-correction instance), and the batch
 * workspace (slr_batch_workspace_size bytes, 256-byte aligned).  None of them
 * may be freed or reused while the instance is in the batch and a run may be
 * in flight.  The batch handle owns host metadata only. */
typedef struct slr_batch_ctx *slr_batch;
size_t slr_batch_workspace_size(int32_t max_instances);       /* 0 if out of [1, 1024] */
size_t slr_batch_scratch_size(const slr_desc *d);             /* 0 for an invalid/unsupported d */
slr_status slr_batch_create(int32_t max_instances, void *workspace, size_t workspace_bytes, void *stream,
                            slr_batch *out);
/* Add an instance with its own absolute iteration cap; returns its slot. */
slr_status slr_batch_add(slr_batch b, const slr_desc *d, void *u, const void *aux, void *scratch,
                         int64_t max_iters, int32_t *slot);
/* Enqueue up to `sweeps` steps of all running instances (asynchronous). */
slr_status slr_batch_run(slr_batch b, int64_t sweeps);
/* Wait for the batch's stream; list (up to max_finished) slots that finished
 * since the last poll, and count the instances still running. */
slr_status slr_batch_poll(slr_batch b, int32_t *finished, int32_t max_finished, int32_t *n_finished,
                          int32_t *n_running);
/* Result of a slot as of the last poll (same meaning as slr_reduce_value). */
slr_status slr_batch_result(slr_batch b, int32_t slot, double *value, int64_t *iters, int32_t *converged,
                            uint64_t *count);
slr_status slr_batch_remove(slr_batch b, int32_t slot);
slr_status slr_batch_destroy(slr_batch b);
const char *slr_batch_last_error(slr_batch b);

/* ---- One grid over n devices: the device step of a row-block split ----------
 * The 1:n deployment of Sec. 3.3 (Fig. 2) cuts one grid into row blocks (3D:
 * slabs of z-planes), one per device; before each sweep (or each pass of k
 * sweeps) the rows next to a block are copied in from the blocks that own
 * them, and the partial reduces of the devices are combined into the value
 * the convergence test reads.  slr_block_sweep is the device step: one sweep
 * of one block.  The halo exchange, the combination of the partials and the
 * test run on the host (paper_1609_04567_gb300/split.py drives them over
 * torch.distributed or, for several blocks on one device, local copies).
 *
 * d describes the whole grid (stencil, storage, boundary, nx, ny, nz, sigma,
 * h, ghost, alpha; defect correction is not accepted).  src, dst and aux are
 * device arrays of b->rows consecutive grid rows (3D: z-planes of ny x nx
 * items), row-major like the grid; aux (f or mask) has the same layout as the
 * state.  Rows [b->lo, b->hi) of dst receive the update of the same rows of
 * src, item for item the whole-grid sweep's; rows of dst outside that range
 * are not written.  The change is reduced over rows [b->own_lo, b->own_hi)
 * into *partial (a device pointer, cleared by the call): the maximum
 * |u' - u| as binary64 bits (Jacobi), the 2^-24 fixed-point sum of |u' - u|
 * and the masked count (restoration), the live count (Life) and "any item
 * changed".  Block row r is global row b->row0 + r; a row beyond the grid's
 * first or last row is the boundary (the Dirichlet ghost, a dead cell, or
 * left out of the restoration's sums) and is never updated; with SLR_WRAP the
 * caller's copied-in rows hold the wrapped rows.  Enqueued on `stream`;
 * SLR_ERR_INVALID_ARG when the ranges are inconsistent or an updated row's
 * neighbour row lies outside the block array (message in
 * slr_last_error(NULL)). */
typedef struct {
    int64_t rows;            /* rows (3D: z-planes) in the block arrays, copied-in rows included */
    int64_t row0;            /* global index of block row 0 */
    int64_t lo, hi;          /* block rows updated: [lo, hi) */
    int64_t own_lo, own_hi;  /* block rows reduced: [own_lo, own_hi), inside [lo, hi) */
} slr_block;

typedef struct {
    uint64_t maxbits;        /* max |delta| as binary64 bits (Jacobi) */
    uint64_t sum;            /* sum of |delta| truncated to multiples of 2^-24 (restoration) */
    uint64_t count;          /* live cells (Life), masked pixels (restoration) */
    uint32_t changed;        /* any item changed */
    uint32_t reserved;
} slr_partial;

slr_status slr_block_sweep(const slr_desc *d, const slr_block *b, const void *src, void *dst, const void *aux,
                           slr_partial *partial, void *stream);

/* ---- A Jacobi solve that allocates nothing ---------------------------------
 * The paper has no counterpart to this call; it serves callers that cannot
 * allocate device memory when they need a solve (a device-memory budget owned
 * by another framework's allocator, a real-time loop that forbids allocation
 * after start-up, or a host thread where cudaMalloc/cudaFree would synchronise
 * the device and stall other streams).  The second state buffer and the
 * control block live in one static device array inside the library, of
 * SLR_STATIC_STATE_BYTES + 4 KiB, which every GPU that loads the library keeps
 * until the process exits.  The call makes no cudaMalloc, cudaFree or other
 * allocating call.
 *
 * Runs d's loop (SLR_J2D5 or SLR_J3D7, any storage, persistent device loop)
 * from the state in u with right-hand side f (both device pointers owned by
 * the caller, layout as for slr_create) until the test passes or max_iters
 * iterations, on `stream`.  Every call then reads the control block back and
 * waits for the stream before it returns the reduced value, the iterations
 * run and the converged flag (NULL outputs are skipped).  Returns SLR_OK /
 * SLR_NOT_CONVERGED like slr_reduce_value, SLR_ERR_INVALID_ARG for a grid
 * whose state exceeds SLR_STATIC_STATE_BYTES (message from
 * slr_static_last_error()), SLR_ERR_UNSUPPORTED for other stencils, for
 * defect correction and for loop = SLR_LOOP_HOST.  Descriptor fields are
 * read as slr_create reads them (grid_ctas, temporal_k and tiling
 * included), except that library-choice fields take the built-in defaults,
 * never the autotuner's cache, and debug_flags is ignored.
 *
 * The first call on each device looks up the array's device address (once per
 * device, with that device current).  The address is kept for the life of the process, so the
 * call must not be used on a device after a cudaDeviceReset of it.  Every
 * call shares the one array: each call clears the control block before it
 * starts, and calls whose GPU work overlaps (several streams or host threads
 * on one device) race on it. */
#define SLR_STATIC_STATE_BYTES (4u << 20)
slr_status slr_run_static(const slr_desc *d, void *u, const void *f, int64_t max_iters, void *stream,
                          double *value, int64_t *iters, int32_t *converged);
/* Message of the last failed slr_run_static on this host thread. */
const char *slr_static_last_error(void);

/* ---- Autotuner -------------------------------------------------------------
 * The paper sizes its OpenCL work-groups with fixed heuristics (Sec. 3.3); this
 * library instead times the launch choices that do not change results on the
 * caller's own data and keeps the fastest in a process-wide cache.
 *
 * slr_tune searches the fields of *d left at their library-choice value:
 *   loop        (SLR_LOOP_AUTO: persistent device loop or the host-driven loop;
 *                defect correction keeps the persistent loop),
 *   temporal_k  (0, Life, SLR_J2D5 and SLR_RESTORE8: sweeps per HBM pass, 1 = none),
 *   tiling      (SLR_TILING_AUTO, RESTORE8 and Jacobi without defect correction:
 *                TMA tiles or none),
 *   grid_ctas   (0: CTAs of the persistent launch),
 * first loop x temporal_k x tiling with all co-resident CTAs, then grid_ctas
 * for the winner.  Fields set explicitly are held fixed.  Each candidate runs
 * trial_iters iterations (<= 0 selects 64, or 4 with defect correction) from a
 * copy of u taken into `scratch`, with the convergence test disabled (Life
 * still stops at a still state), once untimed and twice timed with CUDA events
 * on `stream`; its score is the shorter time per iteration run.  A candidate
 * replaces the best so far only when it is more than 1% faster, so the library
 * default (timed first) is kept on a tie.  u and aux are only read.
 *   scratch     device buffer of slr_tune_scratch_size(d) bytes, 256-byte
 *               aligned, owned by the caller; free to reuse after return.
 *   out         receives the choice with every searched field explicit (loop
 *               HOST or PERSISTENT, temporal_k >= 1 for Life, SLR_J2D5 and SLR_RESTORE8, tiling NONE or TMA
 *               for RESTORE8, grid_ctas >= 0 where 0 kept the default), the
 *               number of candidates timed and the two scores; may be NULL.
 * The call waits for `stream`.  It stores the choice under (device, SM count,
 * stencil, storage, boundary, math, defect correction, nx, ny, nz) and under
 * the same key with each extent replaced by its power-of-two bucket
 * (floor(log2)).  slr_create then fills the library-choice fields of a
 * descriptor from the exact entry, else from the bucket entry, else from the
 * built-in defaults; grid_ctas only when the descriptor then names the
 * choice's loop, temporal_k (Life, SLR_J2D5, SLR_RESTORE8) and tiling, the kernel that
 * grid size was timed with.  Returns SLR_OK, SLR_ERR_INVALID_ARG / UNSUPPORTED for a
 * descriptor slr_create would refuse or a NULL/misaligned pointer,
 * SLR_ERR_WORKSPACE for a short scratch, or the error of a failed trial
 * (message from slr_tune_last_error()), and leaves the cache unchanged then.  The
 * cache is guarded by a mutex; concurrent slr_tune calls on one device time
 * each other's work and should be avoided. */
typedef struct {
    int32_t loop, temporal_k, tiling, grid_ctas;  /* the choice */
    int32_t trials;                               /* candidates timed */
    int32_t reserved;
    double ms_per_iter;                           /* score of the choice */
    double default_ms_per_iter;                   /* score of the library default */
} slr_tune_result;
size_t slr_tune_scratch_size(const slr_desc *d);  /* 0 for an invalid descriptor */
slr_status slr_tune(const slr_desc *d, const void *u, const void *aux, void *scratch, size_t scratch_bytes,
                    void *stream, int64_t trial_iters, slr_tune_result *out);
/* Copy the cached choice for *d (exact key, else bucket) into *out; returns 1
 * when one exists, 0 otherwise.  Needs no GPU work. */
int32_t slr_tune_lookup(const slr_desc *d, slr_tune_result *out);
/* Empty the cache. */
void slr_tune_clear(void);
/* Message of the last failed slr_tune on this host thread. */
const char *slr_tune_last_error(void);

/* ---- Self-check of the restoration's EXACT arithmetic ----------------------
 * EXACT RESTORE8 sweeps form each weight 1 / sqrt(alpha + t*t) with the two
 * IEEE roundings of a sequential 1.0f / sqrtf(x), from the hardware estimates
 * plus one fused-multiply-add correction each (Markstein's method).  This
 * call checks that arithmetic on the device against CUDA's IEEE operations
 * __frcp_rn(__fsqrt_rn(x)) for every non-negative binary32 x (2^31 inputs):
 * mismatches[0] counts inputs whose weight bits differ, mismatches[1] and
 * mismatches[2] the square roots and reciprocals on the inputs that take the
 * estimate route; *checked receives the number of inputs (2^31).  All three
 * counts are 0 on a correct build.  Waits for `stream`; the counters live in a
 * static device array (no allocation).  Either pointer may be NULL. */
slr_status slr_check_exact_math(uint64_t *mismatches, uint64_t *checked, void *stream);

/* Self-check of the Jacobi sweeps' division by the constant d = 2n + sigma h^2:
 * EXACT sweeps form RN(a / d) from the correctly rounded reciprocal of d and
 * two fused-multiply-add corrections (Markstein's method) when |a| and |d|
 * lie in [2^-40, 2^40) (binary32) or [2^-400, 2^400) (binary64), and call the
 * IEEE division otherwise.  For the given d this compares that quotient with
 * CUDA's __fdiv_rn for every binary32 numerator (2^32) and with __ddiv_rn for
 * 2^26 binary64 numerators spread over exponents -600..600; mismatches[0]
 * and [1] count differing quotients (binary32, binary64; NaN quotients agree
 * as NaNs), checked[0] and [1] the numerators tried.  Both counts are 0 on a
 * correct build.  Returns SLR_ERR_INVALID_ARG when d (or (float)d) is outside
 * the range above.  Waits for `stream`; static device counters. */
slr_status slr_check_exact_division(double d, uint64_t *mismatches, uint64_t *checked, void *stream);

/* Self-check of the Sobel magnitude's clamped integer square root (the
 * hardware estimate of sqrt(n + 1/2), truncated): compares it with
 * min(255, floor(sqrt(n))) for every integer 0 <= n < 2^22; *mismatches
 * counts differences (0 on a correct build), *checked the values tried.
 * Waits for `stream`; static device counters. */
slr_status slr_check_exact_isqrt(uint64_t *mismatches, uint64_t *checked, void *stream);

/* Measured throughput of the integer logic pipe on the current device, the
 * denominator of the Game of Life roofline (the bit-sliced update of Fig. 1's
 * rule is three-input logic operations and funnel shifts, which issue to that
 * pipe): a kernel of independent three-input logic operations on every SM
 * (64 warps per SM), timed with CUDA events on `stream` after one warm-up
 * launch.  *ops_per_s receives the logic operations per second (thread
 * operations), *ms the timed kernel's duration; either may be NULL.  Waits
 * for `stream`.  Returns SLR_OK or SLR_ERR_CUDA. */
slr_status slr_measure_logic_rate(double *ops_per_s, double *ms, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SLR_H */
