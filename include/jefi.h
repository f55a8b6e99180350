/*
 * jefi.h -- C ABI of libjefi: Jefimenko field evaluation on one GB300 GPU.
 *
 * What the library computes (JefiGPU, Sec. 2.2, Eqs. E-1, B-1, tr-1): for
 * every observation point r_o and evaluation time t, the midpoint sum over
 * all source cells r_s of a uniform grid
 *
 *   E(r_o,t) = k_e dV sum_s [ D (rho/R^3 + drho/(c R^2)) - dJ/(c^2 R) ]
 *   B(r_o,t) = k_b dV sum_s [ (J/R^3 + dJ/(c R^2)) x D ]
 *
 * with D = r_o - r_s, R = |D| and every source quantity read at the
 * retarded slice
 *
 *   n = floor(((t - t0) - R/c) / dt)                                (Eq. tr-1)
 *
 * of a history of source snapshots pushed one slice at a time (slice n
 * holds the sources at t0 + n dt; sources are zero before slice 0).  Time
 * derivatives are the backward difference (f[n] - f[n-1])/dt of Eq. E-1
 * (f[-1] = 0) or are supplied by the caller.  Pairs inside the screening box
 * |D_a| <= delta_a on all three axes contribute nothing (coarse screening,
 * Sec. 2.1 and Sec. 3).  The paper's units are k_e = k_b = 1/(4 pi), c = 1
 * (Eqs. E and B); any positive c and any k_e, k_b are accepted.
 *
 * Exactness contract.  Cell centres are x_i = lo + (i + 0.5) d rounded as
 * written (product, then sum); the slot n is the FP64 value of the formula
 * above with R = sqrt((Dx*Dx + Dy*Dy) + Dz*Dz), every operation rounded
 * (no FMA).  Every precision selects exactly that slot for every pair;
 * screening decisions are made in FP64 the same way.
 *
 * Threading and streams.  A handle is not thread-safe; issue all calls for
 * one handle from one host thread and on one CUDA stream (or serialise the
 * streams yourself).  `stream` arguments are cudaStream_t values (NULL is the
 * legacy default stream).
 *
 * Errors.  Every call returns a jefi_status; on error nothing has been
 * enqueued unless the code is JEFI_ECUDA.  jefi_strerror() gives a message.
 */
#ifndef JEFI_H
#define JEFI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    JEFI_OK = 0,
    JEFI_EINVAL = 1,       /* bad argument (NULL, non-finite, size or mode)       */
    JEFI_ENOMEM = 2,       /* device or host allocation failed                    */
    JEFI_ENOTYET = 3,      /* t needs a slice that has not been pushed yet        */
    JEFI_EEVICTED = 4,     /* t needs a slice already overwritten in the ring     */
    JEFI_ECUDA = 5,        /* a CUDA runtime call failed                          */
    JEFI_ETIMEOUT = 6,     /* a bounded device wait expired                       */
    JEFI_EINTERNAL = 7,    /* internal consistency check failed                   */
    JEFI_EUNSUPPORTED = 8  /* valid request outside what this library supports    */
} jefi_status;

typedef struct jefi_problem* jefi_handle;

/* Cell-centred uniform grid: centre of cell i on axis a is lo[a] + (i+0.5) d[a].
 * Arrays over a grid are x fastest: index = (k*n[1] + j)*n[0] + i. */
typedef struct {
    int32_t n[3];
    double lo[3];
    double d[3];
} jefi_grid;

typedef enum {
    JEFI_FP64 = 0,       /* FP64 ring and FP64 arithmetic                          */
    JEFI_FP32 = 1,       /* FP32 ring, FP32 sums, FP64 cross-block reduction        */
    JEFI_FP32_COMP = 2   /* as JEFI_FP32 with compensated (Kahan) per-thread sums   */
} jefi_precision;

typedef enum {
    JEFI_DERIV_BACKWARD = 0, /* d/dt = (f[n] - f[n-1]) / dt, f[-1] = 0 (Eq. E-1)  */
    JEFI_DERIV_SUPPLIED = 1  /* caller passes drho/dt and dJ/dt with each slice   */
} jefi_deriv_mode;

/* Optional device allocator (e.g. a framework's caching allocator).  Both
 * NULL: the library uses cudaMalloc / cudaFree. */
typedef void* (*jefi_alloc_fn)(size_t bytes, void* ctx);
typedef void (*jefi_free_fn)(void* ptr, void* ctx);

typedef struct {
    double c;                 /* signal speed, > 0                                  */
    double k_e;               /* E prefactor (1/(4 pi eps0); paper: 1/(4 pi))       */
    double k_b;               /* B prefactor (mu0/(4 pi); paper: 1/(4 pi))          */
    double dt;                /* slice spacing, > 0                                 */
    double t0;                /* time of slice 0                                    */
    int32_t history_slots;    /* H: resident slices in the device ring, >= 1 (FP32
                                 problems on the direct-gather kernel: the ring's
                                 rows, P + mirror + 4 with P = H rounded up to a
                                 multiple of 4, at most 65536, else jefi_create
                                 returns JEFI_EUNSUPPORTED)                       */
    int32_t precision;        /* jefi_precision                                     */
    int32_t deriv;            /* jefi_deriv_mode                                    */
    int32_t flags;            /* JEFI_FLAG_* bits                                   */
    double screen[3];         /* screening half-widths; < 0 selects d_src/2         */
    jefi_alloc_fn alloc;
    jefi_free_fn free;
    void* alloc_ctx;
    /* First cell of the source grid in its lattice: cell i of axis a is
     * centred at lo[a] + (src_origin[a] + i + 0.5) d[a].  0 for a grid of
     * its own; a source sub-box of a larger grid (an S-O pair, paper Sec. 2.2,
     * Fig. 2; see jefi_so_partition) keeps the large grid's lo and d and
     * names its first cell here, so its cell centres are bit-identical to the
     * large grid's. */
    int32_t src_origin[3];
    /* Observation grids only: the shape of the 256-point tiles one CTA
     * evaluates, JEFI_TILE_8x8x4 ... JEFI_TILE_4x4x16 (boxes of the grid),
     * JEFI_TILE_PACKED (4x4x2-point blocks of the grid in Morton order,
     * eight per tile: fewer padding lanes where the grid's sides are not
     * multiples of a box), or JEFI_TILE_AUTO (0): for FP32 problems the
     * tiling with the least predicted time, tiles x the cost of the slot band
     * its widest tile needs (the band the staged kernel copies), else 8x8x4.
     * Point lists are tiled in Morton order (or by distance from the sources
     * when that narrows the bands clearly).  The tiling changes which CTA
     * sums a point, never the slots. */
    int32_t tile_shape;
} jefi_params;

#define JEFI_TILE_AUTO 0
#define JEFI_TILE_8x8x4 1
#define JEFI_TILE_16x4x4 2
#define JEFI_TILE_4x8x8 3
#define JEFI_TILE_8x4x8 4
#define JEFI_TILE_4x16x4 5
#define JEFI_TILE_16x8x2 6
#define JEFI_TILE_8x16x2 7
#define JEFI_TILE_4x4x16 8
#define JEFI_TILE_PACKED 9

#define JEFI_FLAG_STATS 1u    /* time the sum kernel with CUDA events on the call's stream */
#define JEFI_FLAG_DIRECT_GATHER 2u  /* FP32: never use the TMA-staged kernel (for comparisons) */
#define JEFI_FLAG_SHARED_RING 4u    /* FP32: size the ring's mirror for views of any staged band */
/* Second-order retarded time (opt-in; the default floor rule of Eq. tr-1 is
 * the parity contract).  With u = ((t - t0) - R/c)/dt, n = floor(u) (the same
 * exact slot as the floor rule) and w = u - n, every source channel is read as
 *   f = (1 - w) f[n] + w f[n+1],
 * derivatives included: supplied derivatives are interpolated as given;
 * with JEFI_DERIV_BACKWARD the library stores central differences
 * (f[k+1] - f[k-1]) / (2 dt) instead, one slice late (slice k's derivative is
 * written when slice k+1 is pushed).  Slices before the first are zero,
 * values and derivatives alike.  An evaluation needs slices up to n+1
 * (supplied) or n+2 (central) to be pushed: the valid window ends one or two
 * slices earlier than with the floor rule.  Every path supports it (FP64,
 * FP32 staged and direct gather, single, batched and planned evaluations; a
 * batch may mix both rules); a view inherits the setting of its base. */
#define JEFI_FLAG_INTERP 8u

/* Fills p with: c = 1, k_e = k_b = 1, dt = 1, t0 = 0, H = 64, FP32_COMP,
 * backward differences, default screening, cudaMalloc. */
void jefi_default_params(jefi_params* p);

/*
 * Create a problem: a source grid, observation points, and an empty history.
 *
 * src         source grid (n[a] >= 0; a zero extent gives zero fields)
 * obs_grid    observation grid, or NULL when obs_points is given
 * obs_points  [n_obs][3] FP64 host array of observation points (used when
 *             obs_grid is NULL); n_obs >= 0
 * p           parameters (copied)
 * stream      stream for the initial uploads (the call synchronises it)
 * out         receives the handle
 *
 * Allocates the ring (history_slots+1 slots x padded cells x 8 channels of
 * FP32 or FP64) and per-point tables on the device.  Host work is
 * O(N_obs + N_src).
 */
int jefi_create(const jefi_grid* src, const jefi_grid* obs_grid, const double* obs_points,
                int64_t n_obs, const jefi_params* p, void* stream, jefi_handle* out);

/*
 * A second set of observation points over the same resident source history:
 * the view shares `base`'s ring, parameters and pushed slices (pushes go to
 * the base; a view always sees the latest), and has its own tiles, tables
 * and scratch.  The paper keeps rho and J resident across calls (Sec. 2.2);
 * views let many observation regions use one resident history.
 * obs_grid / obs_points / n_obs as in jefi_create.  Destroy every view of a
 * base before the base (jefi_destroy of a base with live views returns
 * JEFI_EINVAL).  Pushing to a view returns JEFI_EINVAL.  A view keeps
 * scratch for 2 evaluation times per launch (a base handle for 8).  A view uses the
 * staged kernel only if its band fits the base ring's mirror (create the
 * base with JEFI_FLAG_SHARED_RING).
 */
int jefi_create_view(jefi_handle base, const jefi_grid* obs_grid, const double* obs_points,
                     int64_t n_obs, void* stream, jefi_handle* out);

/*
 * Append the next slice n_latest+1 of the source history (paper Sec. 2.2:
 * rho and J stay resident on the device between evaluations).
 *
 * rho [N_src], J [N_src][3]: FP64, x-fastest over the source grid.
 * drho_dt, dJ_dt: same layouts; required iff deriv == JEFI_DERIV_SUPPLIED,
 *   must be NULL otherwise.
 * on_device: 1 if the pointers are device memory (read asynchronously on
 *   `stream`), 0 if host memory (copied before the call returns).
 * Backward differences use the previously pushed slice.
 */
int jefi_push_sources(jefi_handle h, const double* rho, const double* J, const double* drho_dt,
                      const double* dJ_dt, int on_device, void* stream);

/*
 * E and B at time t for every observation point (input order).
 *
 * E, B: [N_obs][3] FP64.  on_device = 1: device pointers, results written
 * asynchronously on `stream`.  on_device = 0: host pointers, the call
 * returns when they are filled.
 * JEFI_ENOTYET / JEFI_EEVICTED when some pair's retarded slice is not
 * resident; nothing is written then.
 */
int jefi_eval_fields(jefi_handle h, double t, double* E, double* B, int on_device, void* stream);

/*
 * Several evaluation times in one launch: t[n_t] (host array); E, B are
 * [n_t][N_obs][3].  Same semantics as n_t calls of jefi_eval_fields.
 */
int jefi_eval_fields_multi(jefi_handle h, int32_t n_t, const double* t, double* E, double* B,
                           int on_device, void* stream);

/*
 * Several problems, each at its own time, in one persistent launch per
 * kernel variant present (problems sharing precision and staging share a
 * launch) plus one reduction launch: the many-problem form of
 * jefi_eval_fields (Eqs. E-1, B-1, tr-1 for every problem).
 *
 * hs[n], t[n]: problem i is evaluated at time t[i] (a handle may appear up
 *   to 8 times, a view up to 2 times).  E[i], B[i]: device [N_obs_i][3]
 *   FP64 outputs.
 * Asynchronous on `stream`.  Every problem's result is bit-identical to
 * jefi_eval_fields on the same handle and time: the work items run the same
 * code in the same order whatever else is in the batch.  Batches issued on
 * different streams may run concurrently (each stream has its own batch
 * metadata); a handle must not be in two batches in flight at once.
 */
int jefi_eval_batch(const jefi_handle* hs, const double* t, double* const* E, double* const* B,
                    int32_t n, void* stream);

/*
 * Interval [t_lo, t_hi] of evaluation times whose every retarded slice is
 * resident (all slots >= n_latest-H+1 or < 0, all <= n_latest).  Returns
 * JEFI_ENOTYET if no time qualifies (e.g. nothing pushed yet).
 */
int jefi_valid_window(jefi_handle h, double* t_lo, double* t_hi);

/* Problem sizes and counters. */
typedef struct {
    int64_t n_src;            /* source cells                                      */
    int64_t n_obs;            /* observation points                                */
    int64_t n_latest;         /* index of the newest pushed slice (-1 if none)      */
    int64_t pairs_per_eval;   /* n_src * n_obs                                     */
    int64_t device_bytes;     /* bytes allocated on the device                     */
    int64_t kernel_launches;  /* kernels launched by this handle so far            */
    int64_t slot_fallbacks;   /* pairs whose slot the FP32 path recomputed in FP64  */
    int64_t sum_launches;     /* timed sum-kernel launches (JEFI_FLAG_STATS)        */
    double sum_ms_total;      /* their summed device time, ms (JEFI_FLAG_STATS)     */
    int32_t n_split;          /* source splits per observation tile                */
    int32_t precision;
    int32_t device_status;    /* first error a kernel reported (0 = none), sticky  */
    int32_t staged_band;      /* FP32 sum kernel: history rows staged per cell by
                                 TMA, or 0 for the direct-gather kernel            */
    int32_t tile_shape;       /* observation grids: the JEFI_TILE_* shape of the
                                 256-point tiles; 0 for point lists               */
} jefi_info;

/* Fills *out (waits for the handle's outstanding work).  Kernel-side errors
 * (a bounded wait that expired, a failed internal check) are reported in
 * device_status; calls with host outputs also return them directly. */
int jefi_get_info(jefi_handle h, jefi_info* out);

/* Zeroes the fall-back counter and the kernel timing totals. */
int jefi_reset_stats(jefi_handle h);

/*
 * Diagnostic: the retarded slot the evaluation kernel selects for every
 * pair at time t, through the same code path as jefi_eval_fields.
 * slots: host array [N_obs][N_src] int32 (source index x fastest);
 * screened pairs are INT32_MIN.  Intended for small problems.
 */
int jefi_debug_slots(jefi_handle h, double t, int32_t* slots, void* stream);

/*
 * Diagnostic of the bounded device waits: launches a kernel that waits on a
 * barrier nothing completes, with the same bounded wait the staged sum
 * kernel uses for its TMA copies, limited to limit_s seconds (0 < limit_s
 * <= 10).  Returns JEFI_ETIMEOUT when the wait expired and was reported
 * (the expected outcome), JEFI_OK if it did not expire.
 */
int jefi_debug_wait_timeout(double limit_s, void* stream);

/*
 * Host reference of the exact slot rule above for explicit pairs (no GPU
 * needed): xo, xs [n][3]; out[n].
 */
void jefi_host_pair_slots(int64_t n, const double* xo, const double* xs, double t, double t0,
                          double c, double dt, int64_t* out);

/*
 * Host rule of the source splits (no GPU needed).  The direct sum of
 * Eqs. E-1/B-1 runs over every source cell for every observation tile; the
 * library cuts the source bricks of a tile into splits whose FP64 partial
 * sums the reduction adds in split order (the paper has no counterpart: its
 * kernel sums all cells in one thread).  For n_tiles tiles of 256 points
 * over n_bricks 4x4x4 source bricks, at most max_splits splits, launches of
 * 1, 2, 4, ... times_per_launch evaluation times and resident_ctas CTAs
 * resident at once, this returns the split count jefi_create picks for a
 * staged FP32 handle (*n_split, the one whose launches fill their waves of
 * equal work items best, the fewest among equals), its bricks per split
 * (*bricks_per_split) and the consecutive splits one work item of a
 * single-time launch merges (*merge).  jefi_create takes max_splits as
 * twice the count that gives 8 waves (4 for a view) at one time, capped at
 * one split per brick and 256 MB of partial sums (32 MB for a view), and
 * resident_ctas as 2 per SM.  Returns JEFI_EINVAL for a non-positive size
 * or a NULL output.
 */
int jefi_host_split_plan(int64_t n_tiles, int64_t n_bricks, int64_t max_splits, int32_t times_per_launch,
                         int64_t resident_ctas, int32_t* n_split, int32_t* bricks_per_split, int32_t* merge);

/*
 * Push one slice given as a region of larger arrays: rho, J (and drho, dJ
 * when supplied) cover full_n[0] x full_n[1] x full_n[2] cells, x fastest,
 * and the handle's cell (i, j, k) is their cell offset + (i, j, k).  The
 * source side of an S-O pair (paper Sec. 2.2, Fig. 2) pushes its sub-box
 * straight from the whole grid's slice this way.  offset + the handle's grid
 * extents must lie within full_n (JEFI_EINVAL otherwise).  Otherwise as
 * jefi_push_sources; host arrays (on_device = 0) are gathered on the host
 * and the call returns once they have been copied.
 */
int jefi_push_sources_region(jefi_handle h, const double* rho, const double* J, const double* drho,
                             const double* dJ, const int32_t full_n[3], const int32_t offset[3], int on_device,
                             void* stream);

/*
 * Source/observation (S-O) decomposition (paper Sec. 2.2, Fig. 2: the source
 * and observation regions are cut into rectangular sub-boxes and every pair
 * of a source box and an observation box is evaluated on its own, e.g. one
 * pair per GPU; the fields of the pairs that share an observation box add).
 *
 * jefi_so_partition cuts the source grid into parts[0] x parts[1] x parts[2]
 * boxes along whole 4-cell bricks (box k = (kz parts[1] + ky) parts[0] + kx,
 * x fastest; a box may be empty when there are fewer bricks than parts).
 * Box k is sub[k] with origin[3k .. 3k+2]: sub[k] keeps src's lo and d and
 * its first cell is src cell origin[3k + a] -- create its handle with
 * jefi_params.src_origin = that origin so its cell centres are bit-identical
 * to src's, and push its slices with jefi_push_sources_region.  sub holds
 * parts[0] parts[1] parts[2] grids and origin three times as many int32.
 * Host-only; JEFI_EINVAL for parts outside [1, 4096].
 */
int jefi_so_partition(const jefi_grid* src, const int32_t parts[3], jefi_grid* sub, int32_t* origin);

/*
 * E = E_parts[0] + E_parts[1] + ... and the same for B, summed in FP64 in
 * that order, element by element over n_obs points ([n_obs][3] device
 * arrays, caller-owned): the fields of S-O pairs that share their
 * observation points, summed in source-box order whatever the number of
 * ranks that produced them (deterministic).  1 <= n_parts <= 64; enqueued
 * on `stream`.
 */
int jefi_sum_fields(int32_t n_parts, const double* const* E_parts, const double* const* B_parts, int64_t n_obs,
                    double* E, double* B, void* stream);

/*
 * One-shot FP64 evaluation that allocates no device memory.  The paper has
 * no counterpart: it is for callers that cannot allocate device memory when
 * they need fields -- a host application whose own pool allocator owns the
 * device memory and forbids other cudaMalloc calls, or a time-critical loop
 * where cudaMalloc/cudaFree would synchronise the device.
 *
 * Computes the same sum as jefi_eval_fields with precision JEFI_FP64 and
 * backward differences, for one time t, from the caller's device buffers:
 *   src        source grid (host struct)
 *   obs        device [n_obs][3] FP64 observation points (any order)
 *   rho, J     device [n_slices][N_src] and [n_slices][N_src][3] FP64: the
 *              whole history, slice n at time p->t0 + n*p->dt, cells x fastest
 *   p          uses c, k_e, k_b, dt, t0 and screen; other fields are ignored
 *              (flags included: this entry runs the floor rule of Eq. tr-1)
 *   E, B       device [n_obs][3] FP64 outputs
 * The call is synchronous on `stream` (it returns after E and B are written).
 *
 * Working memory is one file-scope device array of JEFI_NOALLOC_SCRATCH_BYTES
 * per GPU that loads the library, held until the process exits.  The first
 * call on a device, with that device current, does the set-up: it finds the
 * array's address (cudaGetSymbolAddress, which also loads the module) and the
 * device's SM count; make that first call before any stream capture begins.
 * All calls share the array and it keeps the last call's contents (the call
 * clears its status word itself); calls that overlap on the GPU race on it,
 * so callers on several streams or threads must serialise them.  The library
 * cannot check the sizes of the caller's device buffers: they must hold the
 * element counts above.
 *
 * Limits: ceil(n_obs/256)*256 <= (JEFI_NOALLOC_SCRATCH_BYTES - 256)/48 (that
 * is n_obs <= 698880), and 4*(ceil(nx/4)+ceil(ny/4)+ceil(nz/4)) <= 6144;
 * larger requests return JEFI_EUNSUPPORTED without touching the GPU.
 * JEFI_ENOTYET if some pair needs a slice >= n_slices (E, B then incomplete).
 */
#define JEFI_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
int jefi_eval_fields_noalloc(const jefi_grid* src, const double* obs, int64_t n_obs,
                             const double* rho, const double* J, int64_t n_slices,
                             const jefi_params* p, double t, double* E, double* B, void* stream);

/*
 * Checkpoint and resume of a handle's resident history (paper Sec. 2.2: rho
 * and J stay on the device between evaluations; a serving process that
 * restarts keeps them this way instead of pushing the last H slices again).
 *
 * The image is opaque bytes owned by the caller: a header (format version,
 * the source grid, c, dt, t0, H, precision, derivative mode, interpolation
 * setting, the index of the newest slice) followed by ring slots 0..H-1 of
 * every cell (FP32 or FP64, 8 channels) and the FP64 state of the
 * difference rule (the last one or two slices).  Observation points are not
 * part of it.
 *
 * jefi_checkpoint_bytes: size of the image of h.
 * jefi_checkpoint: writes the image into host memory dst (bytes >= the
 *   size); synchronous on `stream`.
 * jefi_restore: loads an image into h, which must have been created with the
 *   same source grid, c, dt, t0, H, precision, derivative mode and
 *   interpolation setting (its observation points may differ); the handle
 *   then holds exactly the history of the checkpointed one and continues
 *   from its newest slice.  Synchronous on `stream`.  Views of h see it.
 * Errors: JEFI_EINVAL for a view (views hold no history; checkpoint the
 * base), a buffer that is too small, or an image that is corrupt or was
 * taken under other parameters (h is then unchanged).
 */
int jefi_checkpoint_bytes(jefi_handle h, size_t* bytes);
int jefi_checkpoint(jefi_handle h, void* dst, size_t bytes, void* stream);
int jefi_restore(jefi_handle h, const void* src, size_t bytes, void* stream);

/*
 * Choice of the FP32 sum kernel of a handle after creation.  At creation a
 * geometry rule picks the TMA-staged kernel whenever every (tile, brick)
 * slot band fits 48 rows, else the direct gather.  On wide bands either can
 * be the faster (Eqs. E-1, B-1, tr-1 are computed the same way by both:
 * identical slots, fields equal to FP32 rounding, not bit for bit).
 *
 * mode JEFI_KERNEL_MEASURE: time one evaluation at t with each candidate --
 *   the staged band of creation, the next wider compiled band when the
 *   ring's mirror holds it (other stages, other shared-memory layout) and
 *   the direct gather -- after one untimed evaluation each, and keep the
 *   fastest; t must be in the valid window.  The call synchronises `stream`.
 * mode JEFI_KERNEL_DIRECT: switch to the direct gather (t unused).
 * mode JEFI_KERNEL_STAGED: switch back to the staged kernel of creation (t
 *   unused).
 * staged_band (may be NULL) receives the band of the kernel in use, 0 for
 *   the direct gather (the value jefi_get_info reports as staged_band).
 * Errors: JEFI_EINVAL for a bad mode or an FP64 handle; for
 *   JEFI_KERNEL_MEASURE a t outside the window gives JEFI_ENOTYET /
 *   JEFI_EEVICTED as in jefi_eval_fields.  JEFI_EUNSUPPORTED when the kernel
 *   a switch asks for cannot run this handle (no staged band at creation;
 *   for the direct gather a ring of more than 65536 rows or tables beyond
 *   its shared memory): the choice is then unchanged.  Where there is no
 *   alternative, JEFI_KERNEL_MEASURE keeps the kernel in use and returns
 *   JEFI_OK.  Later evaluations, single or batched, use the chosen kernel.
 */
#define JEFI_KERNEL_MEASURE 0
#define JEFI_KERNEL_DIRECT 1
#define JEFI_KERNEL_STAGED 2
int jefi_select_kernel(jefi_handle h, int32_t mode, double t, int32_t* staged_band, void* stream);

/*
 * Batch plans: a fixed set of problems evaluated again and again, each call
 * at new times, as one CUDA graph (Eqs. E-1, B-1, tr-1 for every problem,
 * exactly as jefi_eval_batch computes them).
 *
 * jefi_batch_plan_create records, once, everything jefi_eval_batch issues
 * for hs[n] with outputs E[i], B[i] (device [N_obs_i][3] FP64, fixed for the
 * plan's life): one host-to-device copy of the batch's metadata and slot
 * tables, one persistent launch per kernel variant and the reduction.  It
 * captures that sequence into two CUDA graphs (the metadata of call k is
 * written on the host while call k-1 may still run on the device) and
 * allocates the plan's own device and pinned host buffers.  In the graphs
 * the launches of different kernel variants are parallel branches between
 * the copy and the reduction (their work items are independent), so one
 * variant's first items can run beside another's last ones.  A handle may
 * appear up to 8 times (a view up to 2 times), as in jefi_eval_batch; FP64,
 * FP32 and compensated FP32 handles mix freely, with and without
 * JEFI_FLAG_INTERP.
 *
 * jefi_batch_plan_launch evaluates problem i at t[i] (host array [n]):
 * checks every time against its handle's window (JEFI_ENOTYET /
 * JEFI_EEVICTED, nothing enqueued), builds the exact slot tables on the
 * host and replays the graph with one cudaGraphLaunch on `stream`.
 * Asynchronous; every result is bit-identical to jefi_eval_batch (and to
 * jefi_eval_fields) on the same handles and times.  If a handle's kernel or
 * source-split count changed since the graphs were recorded
 * (jefi_select_kernel, a tuner), the call first waits for the plan's
 * earlier launches and records the graphs again.  Launches of one plan must
 * be issued on one stream (or serialised by the caller); a handle must not
 * be in two plans or batches in flight at once (they share its scratch).
 *
 * jefi_batch_plan_tune is the autotuner of the batched launch.  It times the
 * plan, on the device, at times t[n] (which it evaluates, overwriting the
 * outputs) in each of these configurations and keeps the fastest:
 *   - the kernel variants' launches as parallel graph branches or one after
 *     another (decided first, then kept for the candidates below);
 *   - kernel choice per problem: the handles' current choice, and the one
 *     jefi_select_kernel(JEFI_KERNEL_MEASURE) makes for each FP32 handle
 *     that has alternatives (staged band of creation, the next wider
 *     compiled band, direct gather);
 *   - source splits per observation tile (the work-item shape): every
 *     handle's creation-time split count divided by 1, 2, 4 or 8 (a batch
 *     fills the GPU with many problems, so fewer and larger items can win).
 * (The observation tile shape is the third work-item dimension; it is
 * chosen when a handle is created, see jefi_params.tile_shape.)
 * The choice stays with the handles: later single, batched and planned
 * evaluations use it.  Fields then differ from the untuned ones at the
 * rounding level of the precision (the split sums change), still within
 * the accuracy contract.  `report` (may be NULL) receives what was tried
 * and kept.  The call synchronises `stream`.
 *
 * Tune cache: when the environment variable JEFI_TUNE_CACHE names a file,
 * the tuner first looks there for the plan's key (a hash of every entry's
 * geometry -- source grid and origin, observation points, history, dt, c,
 * precision, derivative rule, creation bands and splits -- and the
 * device's SM count).  On a hit it applies the stored choice (branches,
 * per-problem kernel, split divisor), times it once and returns with
 * from_cache = 1; otherwise it tunes and appends one line with the choice.
 * The file is plain text, one line per plan; an unreadable or malformed
 * file counts as a miss.
 *
 * jefi_batch_plan_destroy waits for the plan's launches and frees it.
 * Destroy every plan before the handles it holds: jefi_destroy of a handle
 * in a live plan returns JEFI_EINVAL.
 */
typedef struct jefi_batch_plan_s* jefi_batch_plan;

typedef struct {
    int32_t candidates;       /* configurations timed                                */
    int32_t split_divisor;    /* kept: creation-time split counts divided by this
                                 (1, 2, 4, 8), or 0 if the splits the handles had
                                 at the call were kept                             */
    int32_t measured_kernels; /* kept: 1 = per-problem measured kernel choice,
                                 0 = the handles' choice at the call               */
    int32_t staged_problems;  /* batch entries on the staged kernel after tuning      */
    int32_t concurrent_groups;/* kept: 1 = kernel variants as parallel graph
                                 branches, 0 = one after another                   */
    double ms_initial;        /* device time of one launch as the handles were       */
    double ms_tuned;          /* device time of one launch as kept                   */
    int32_t from_cache;       /* 1: the choice came from the JEFI_TUNE_CACHE file    */
    int32_t widened_bands;    /* batch entries kept on the wider staged band         */
} jefi_tune_report;

int jefi_batch_plan_create(const jefi_handle* hs, double* const* E, double* const* B, int32_t n,
                           jefi_batch_plan* out);
int jefi_batch_plan_launch(jefi_batch_plan plan, const double* t, void* stream);
int jefi_batch_plan_tune(jefi_batch_plan plan, const double* t, void* stream, jefi_tune_report* report);
int jefi_batch_plan_destroy(jefi_batch_plan plan);

/* Release every device and host resource of the handle.  Waits for the
 * work enqueued on the handle (on any stream) to finish, not for the whole
 * device: other handles' work keeps running.  A base with live views
 * returns JEFI_EINVAL (destroy the views first), and so does a handle that
 * a live batch plan holds. */
int jefi_destroy(jefi_handle h);

const char* jefi_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* JEFI_H */
