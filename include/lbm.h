/*
 * lbm.h -- C ABI of the GB300 D3Q27 cumulant lattice Boltzmann library.
 *
 * The library advances the channel flow of the paper's data pipeline
 * (Sec. 2 "Pipeline description": simulation, capture of mean velocity and
 * pressure, strided snapshots and obstacle forces; Sec. 3.1 "Generated
 * dataset": velocity inlet, outflow, no-slip lateral walls, Re set through
 * the lattice viscosity at constant inlet velocity; Sec. 3.2: D3Q27 stencil,
 * cumulant collision operator, bounce-back on the obstacle).
 *
 * Conventions shared by every entry point
 *   - Grid (nx, ny, nz), x streamwise.  Cell index c = x + nx*(y + ny*z).
 *   - Velocities c_i in {-1,0,1}^3 with i = (cx+1) + 3(cy+1) + 9(cz+1); the
 *     opposite of i is 26 - i.
 *   - Every call returns lbm_status and never throws.  Argument errors are
 *     reported synchronously; device-side conditions (non-finite or
 *     out-of-range density) are latched in a device word and reported by the
 *     next lbm_sync or read as LBM_ERR_UNSTABLE, after which lbm_step refuses
 *     to run (LBM_ERR_STATE) but reads still work.
 *   - Work is enqueued on the CUDA stream given at creation (borrowed, never
 *     destroyed; NULL = legacy default stream).  lbm_step is asynchronous;
 *     every read synchronises that stream.
 *   - Destination/source buffers of reads and writes may live in host memory
 *     or device memory (detected per call); the caller owns them.
 *   - Masks and parameters are copied at creation; the caller keeps them.
 */
#ifndef GB300_LBM_H
#define GB300_LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = 1,       /* invalid argument (nothing was enqueued)          */
    LBM_ERR_CUDA = 2,      /* a CUDA runtime call failed                        */
    LBM_ERR_OOM = 3,       /* device allocation failed / workspace too small    */
    LBM_ERR_UNSTABLE = 4,  /* density left (0.5, 1.5) or became non-finite     */
    LBM_ERR_TIMEOUT = 5,   /* a bounded device-side wait expired               */
    LBM_ERR_STATE = 6,     /* call not valid in the context's current state    */
    LBM_ERR_IO = 7         /* checkpoint file could not be written or read     */
} lbm_status;

/* Storage of the shifted populations f_i - w_i (arithmetic is FP32 for the
 * reduced formats, FP64 for LBM_F64).  LBM_F16S is IEEE binary16, LBM_BF16S
 * bfloat16, LBM_F16C a 16-bit float with 4 exponent bits (bias 15) and 11
 * mantissa bits (range +-2, subnormal step 2^-25, saturating): one mantissa
 * bit more than binary16 for values that never leave (-1, 1). */
typedef enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F16S = 2, LBM_BF16S = 3, LBM_F16C = 4 } lbm_storage;

/* Boundary kind of a pair of faces (x has a low and a high face).
 *
 * x high, LBM_FACE_OUTFLOW (the default; Sec. 3.1: the outflow "employs
 * extrapolation"): the convective outflow of Geier et al. 2015 (App. F), the
 * paper's cited cumulant reference.  For each link of an outlet cell x_b
 * through the face (cx = -1 and the source not beyond a lateral wall), the
 * incoming population is f_i(x_b, t+1) = c_s f_i(x_b - e_x, t) +
 * (1 - c_s) f_i(x_b, t) from pre-collision values, c_s = 1/sqrt(3): waves
 * leave the domain instead of reflecting.  A solid cell next to the outlet
 * makes the outlet cell extrapolate from itself.
 * x high, LBM_FACE_OUTLET: anti-bounce-back at the fixed density rho_out
 * (a pressure node; it reflects sound, and with lattice viscosities below
 * about 2.5e-3 the channel diverges from the outlet corners). */
typedef enum {
    LBM_FACE_WALL = 0,      /* no-slip halfway bounce-back                       */
    LBM_FACE_PERIODIC = 1,  /* wrap-around                                       */
    LBM_FACE_INLET = 2,     /* x low only: bounce-back from a wall moving at u_in */
    LBM_FACE_OUTLET = 3,    /* x high only: anti-bounce-back at rho_out           */
    LBM_FACE_OUTFLOW = 4    /* x high only: convective extrapolation outflow      */
} lbm_face;

typedef struct { int32_t nx, ny, nz; } lbm_grid;

typedef struct {
    /* Sec. 3.1: nu = u_in * l_ref / re, omega1 = 1 / (3 nu + 1/2) */
    double re, u_in, l_ref;
    double omega1;          /* > 0 overrides the Re-derived shear rate          */
    double omega_bulk;      /* bulk rate (default 1)                            */
    double omega_higher;    /* rate of every cumulant of order 3..6 (default 1) */
    double rho_in;          /* density of the moving inlet wall (default 1)     */
    double rho_out;         /* outlet density (default 1)                       */
    int32_t storage;        /* lbm_storage (default LBM_F32)                    */
    int32_t galilean_correction; /* 1 (default): corrected diagonal relaxation  */
    int32_t face_x_lo, face_x_hi, face_y, face_z; /* lbm_face; default inlet/outflow/wall/wall */
    /* time average (Sec. 2: mean velocity and pressure): steps t with
     * mean_start <= t < mean_end and (t - mean_start) % mean_every == 0 are
     * sampled from the pre-collision state of step t; mean_every = 0: off */
    int64_t mean_start, mean_end, mean_every;
    /* snapshots (Sec. 2: 20 snapshots 25 steps apart): u, v, w, p of the
     * pre-collision state at t = snap_first + k * snap_every, k < snap_count */
    int64_t snap_first, snap_every, snap_count;
    int32_t snap_halfres;   /* 1: 2x2x2 box mean (Sec. 3.1: half resolution)    */
    int32_t force_every;    /* record the obstacle force every n steps (0: off) */
    int64_t force_capacity; /* rows kept on the device between host flushes     */
    int32_t block_x;        /* threads per block along x, multiple of 32 (0: 128) */
    int32_t block_y;        /* rows per block (0: 1); block_x * block_y <= 256   */
    int32_t stats;          /* 1: also accumulate the velocity products of the
                               averaged samples (lbm_read_stats)                */
    /* Sec. 3.2: the fourth-order parametrisation with limiter (Geier,
     * Pasquali & Schoenherr 2017) in place of omega_higher: third-order
     * cumulants relax in the combinations C_210 +- C_012, C_201 +- C_021,
     * C_120 +- C_102 (sums with omega3, differences with omega4) and C_111
     * (omega5), each rate limited as w + (1 - w)|X| / (|X| + limiter); the
     * fourth-order cumulants are set to C_220 = -(2/3) A (1/w1 - 1/2)(dxu + dyv)
     * (and permutations) and C_211 = B (1 - w1/2) C_011 (and permutations),
     * with dxu, dyv, dzw the velocity-derivative estimates of the Galilean
     * correction; fifth and sixth orders to 0.  omega3..5, A and B are the
     * published functions of omega1 and omega_bulk; they are undefined at
     * omega1 = omega_bulk (LBM_ERR_ARG).  The paper switches it on for
     * Re_c >= 3000 only: at elevated viscosity (omega1 below about 1.8 with
     * omega_bulk = 1) some of these rates leave (0, 2). */
    int32_t param4;         /* 1: the parametrisation above (default 0)          */
    double limiter;         /* its limiter lambda (default 0.01)                 */
    int32_t xface_edge;     /* 1: the inlet/outlet cells go through the boundary-
                               cell records instead of the bulk kernel's face
                               warps (default 0: the face warps, whose accesses
                               are coalesced with their rows; batch members
                               follow their own setting) */
    int32_t reserved[1];
} lbm_params;

/* Fill *p with the defaults listed above (re = 1000, u_in = 0.05, l_ref = 1,
 * averaging and snapshots off, force off). */
void lbm_params_default(lbm_params *p);

/* Bytes of device memory a context with these arguments needs (pdfs,
 * cell flags, boundary-cell records, accumulators, snapshot ring, scratch).
 * mask as for lbm_create (host, device or NULL): the boundary records are
 * bounded by the face cells plus 26 per solid cell.  0 on invalid input. */
size_t lbm_workspace_bytes(const lbm_grid *grid, const uint8_t *mask, const lbm_params *p);

/* Create a context.  mask: nx*ny*nz bytes, 1 = solid obstacle cell, host or
 * device, may be NULL (no obstacle).  State starts at rest (f = w, t = 0).
 * The library allocates its own device memory. */
lbm_status lbm_create(const lbm_grid *grid, const uint8_t *mask, const lbm_params *p,
                      void *cuda_stream, lbm_ctx **out);

/* As lbm_create, but every device buffer is carved from the caller's
 * device allocation `workspace` of `workspace_bytes` (at least
 * lbm_workspace_bytes(); 256-byte aligned).  The caller keeps ownership and
 * must keep it alive until lbm_destroy. */
lbm_status lbm_create_in(const lbm_grid *grid, const uint8_t *mask, const lbm_params *p,
                         void *cuda_stream, void *workspace, size_t workspace_bytes,
                         lbm_ctx **out);

lbm_status lbm_destroy(lbm_ctx *ctx);

/* Advance n time steps (fused collide + stream in place, AA pattern; the
 * epilogues sample means, forces and snapshots as configured).  Async. */
lbm_status lbm_step(lbm_ctx *ctx, int64_t n);

/* Wait for the stream; report latched device conditions. */
lbm_status lbm_sync(lbm_ctx *ctx);

/* Number of steps taken so far. */
int64_t lbm_time(const lbm_ctx *ctx);

/* Time-averaged fields: 4 values per cell (ux, uy, uz, p), cell-major
 * [z][y][x][4], p = (rho - 1)/3; solid cells give 0.  dtype 0 = double,
 * 1 = float.  halfres = 1: 2x2x2 box means on a ceil(n/2) grid.
 * samples (may be NULL) receives the sample count. */
lbm_status lbm_read_mean(lbm_ctx *ctx, int32_t dtype, int32_t halfres, void *dst,
                         int64_t *samples);

/* Interpolated bounce-back on obstacle links (Sec. 3.2: a quadratic
 * bounce-back with wall distances).  Link k runs from fluid cell cell[k]
 * along direction dir[k] (index (cx+1) + 3(cy+1) + 9(cz+1)) into an obstacle
 * cell inside the grid; q[k] in (0, 1] is the fraction of the link on the
 * fluid side of the wall.  After every step the population returned into the
 * opposite direction becomes the quadratic interpolation of Bouzidi,
 * Firdaouss & Lallemand (2001) from the post-collision populations of the
 * cell and of the two cells behind it (x - c, x - 2c; linear when only the
 * first is a fluid cell, halfway bounce-back when neither is; periodic faces
 * are crossed, other faces end the stencil), and the obstacle force becomes
 * the momentum exchange c (f* + f_returned).  Links not listed keep halfway
 * bounce-back; n = 0 restores it everywhere; a repeated link takes its last
 * entry.  Host arrays; the list is copied to device memory the context owns
 * (kept across lbm_reset and lbm_load).  LBM_ERR_ARG for a link that is not
 * fluid -> obstacle or q outside (0, 1]; LBM_ERR_STATE on a batch member (use
 * lbm_batch_set_wall_distances).  Stepped by an extra kernel after each step
 * (for batches, in the end-of-step kernel that also runs the outflow). */
lbm_status lbm_set_wall_distances(lbm_ctx *ctx, int64_t n, const int64_t *cell, const int8_t *dir,
                                  const double *q);

/* Probes (Sec. 3.3: the Strouhal number from the velocity in the wake; a
 * monitor of chosen cells): every `every` steps, (ux, uy, uz, p) of the
 * state before the step at the n listed cells (x + nx (y + ny z)), FP32,
 * the time-average convention (p = (rho - 1)/3; solid cells give 0).  Rows
 * are kept on the device, `capacity` at a time, and moved to the host when
 * full.  A call replaces the probe set and clears the record; n = 0 turns
 * probes off.  Host cell array, copied.  Not supported on batch members
 * (LBM_ERR_STATE); not part of checkpoints. */
lbm_status lbm_set_probes(lbm_ctx *ctx, int64_t n, const int64_t *cells, int64_t every, int64_t capacity);

/* The probe record so far, rows of n x 4 floats (host or device dst, at most
 * max_rows rows); n_rows (may be NULL) receives the rows recorded. */
lbm_status lbm_read_probes(lbm_ctx *ctx, float *dst, int64_t max_rows, int64_t *n_rows);

/* Monitor plane (Sec. 2: "2D snapshots of the center x-y plane for
 * monitoring the development of the entire simulation"): before every step t
 * with t % every == 0, the (ux, uy, uz, p) of the plane z (z < 0: nz / 2) of
 * the state at t are recorded as FP32 [ny][nx][4] (solid cells 0) into a
 * device ring of `capacity` planes that is flushed to host memory when full.
 * every = 0 switches it off.  Not on batch members (LBM_ERR_STATE).  Setting
 * it discards the planes recorded so far. */
lbm_status lbm_set_plane_monitor(lbm_ctx *ctx, int32_t z, int64_t every, int64_t capacity);

/* The planes recorded so far, oldest first: dst [k][ny][nx][4] floats (host or
 * device), at most max_planes; *n_planes (may be NULL) receives the number
 * recorded and steps[k] (host, may be NULL) the step of plane k. */
lbm_status lbm_read_plane_monitor(lbm_ctx *ctx, float *dst, int64_t max_planes, int64_t *n_planes,
                                  int64_t *steps);

/* Turbulence statistics (Sec. 3.3 validates turbulent fluctuations): the
 * velocity covariances over the same samples as the time average, per cell
 * <ux ux> - <ux>^2, <uy uy> - <uy>^2, <uz uz> - <uz>^2, <ux uy> - <ux><uy>,
 * <ux uz> - <ux><uz>, <uy uz> - <uy><uz>, cell-major [z][y][x][6], from FP64
 * running sums; solid cells give 0.  Needs params.stats = 1 and a time
 * average (LBM_ERR_STATE otherwise).  dtype 0 = double, 1 = float. */
lbm_status lbm_read_stats(lbm_ctx *ctx, int32_t dtype, void *dst, int64_t *samples);

/* Snapshot k (0 <= k < snap_count) as float [z][y][x][4] (ux, uy, uz, p) at
 * full or half resolution (params.snap_halfres); LBM_ERR_STATE if not taken. */
lbm_status lbm_read_snapshot(lbm_ctx *ctx, int32_t k, float *dst);

/* Density and velocity of the current state: rho [N], u [N][3] (doubles). */
lbm_status lbm_read_macros(lbm_ctx *ctx, double *rho, double *u);

/* Obstacle force by momentum exchange (Sec. 2: forces on the object),
 * F(t) = sum over obstacle links (x, i) of c_i (f*_i(x) + f_back), where f_back
 * is the population returned into the opposite direction: f*_i itself on
 * halfway bounce-back links (2 c_i f*_i), the interpolated value on links
 * with wall distances (lbm_set_wall_distances).  Walls are not part of the
 * body.  One row (Fx, Fy, Fz) per recorded step, oldest first.  Writes at
 * most max_rows rows; *n_rows receives the number recorded. */
lbm_status lbm_read_forces(lbm_ctx *ctx, double *dst, int64_t max_rows, int64_t *n_rows);

/* Full populations f_i (stored value + w_i) of the current state in natural
 * order, direction-major [27][N] doubles. */
lbm_status lbm_get_pdfs(lbm_ctx *ctx, double *dst);

/* Start from given fields (e.g. a surrogate's prediction of the mean flow):
 * fields [z][y][x][4] floats (ux, uy, uz, p), host or device; every fluid
 * cell takes the product-form equilibrium at rho = 1 + 3 p and u (the
 * equilibrium whose cumulants above second order vanish).  Only at even t
 * (LBM_ERR_STATE otherwise). */
lbm_status lbm_init_equilibrium(lbm_ctx *ctx, const float *fields);

/* Overwrite the state with full populations [27][N] (values of solid cells
 * are ignored).  Only at even t (LBM_ERR_STATE otherwise). */
lbm_status lbm_set_pdfs(lbm_ctx *ctx, const double *src);

/* Full populations of n selected cells: dst [n][27] doubles; cells [n]
 * (host or device int64 cell indices, each in [0, N)). */
lbm_status lbm_get_cells(lbm_ctx *ctx, int64_t n, const int64_t *cells, double *dst);

/* Seeded near-rest state: stored f_i - w_i = amplitude * r, r uniform in
 * [-1, 1) from SplitMix64 started at `seed`, stream counter cell*27 + i;
 * solid cells 0.  Only at even t. */
lbm_status lbm_init_noise(lbm_ctx *ctx, uint64_t seed, double amplitude);

/* Totals over fluid cells of the current state: out[0] = sum_i (f_i - w_i)
 * (mass minus the rest mass), out[1..3] = momentum.  Two-pass deterministic
 * FP64 reduction. */
lbm_status lbm_totals(lbm_ctx *ctx, double out[4]);

/* Sizes and counters of a context. */
typedef struct {
    int64_t cells;           /* nx*ny*nz                                          */
    int64_t fluid_cells;     /* cells that are not obstacle                       */
    int64_t edge_cells;      /* fluid cells handled by the boundary-aware kernel  */
    int64_t bulk_cells;      /* fluid cells handled by the bulk kernel (incl. inlet/outlet plane cells) */
    int64_t launches;        /* kernels launched by lbm_step so far               */
    uint64_t workspace_bytes;
    int32_t storage, block_x;
    double omega1;           /* shear rate in use                                 */
    int64_t interior_cells;  /* equal to bulk_cells (kept for layout stability)     */
    int64_t wall_cells;      /* fluid cells in the rows next to no-slip lateral walls,
                                updated in extra blocks of the edge kernel's
                                launch (fluid_cells = bulk_cells + wall_cells +
                                edge_cells) */
} lbm_info;

lbm_status lbm_get_info(const lbm_ctx *ctx, lbm_info *out);

/* Kernel timing.  While enabled, lbm_step records CUDA events on the
 * context's stream around the bulk kernel and the edge kernel of every step
 * (events only; no sync). */
lbm_status lbm_timing(lbm_ctx *ctx, int32_t enable);

/* Durations accumulated since the last reset (synchronises the stream).
 * bulk_ms / bulk_n (bulk kernel) are indexed by (odd step) + 2 * (epilogue
 * active); edge_ms is summed over all steps; rowend_ms is always 0. */
typedef struct {
    int64_t steps;
    double bulk_ms[4];
    int64_t bulk_n[4];
    double rowend_ms;
    double edge_ms;
} lbm_timing_report;

lbm_status lbm_timing_read(lbm_ctx *ctx, lbm_timing_report *out, int32_t reset);

/* Checkpoint: pdfs, time step, outlet plane, accumulators, force rows. */
lbm_status lbm_save(lbm_ctx *ctx, const char *path);
lbm_status lbm_load(lbm_ctx *ctx, const char *path);

/* ------------------------------------------------------------------------
 * Batches: many independent lattices (e.g. generated geometries on uneven
 * grids at different Re, Sec. 2-3.1) stepped together.  Every step is one
 * bulk launch and one edge launch over all unfinished members (blocks are
 * numbered member after member); a chunk of steps is captured once as a CUDA
 * graph on the batch's own stream and replayed.  Step-dependent work (time
 * average sampling, force rows) is driven by a device step counter.
 *
 * Members are ordinary contexts owned by the batch: read them with the
 * lbm_read_* / lbm_get_* calls through lbm_batch_member; do not step them
 * directly.  Requirements: one storage for all members; the same
 * omega_higher == 1 choice; no snapshots; if any member averages, all share
 * one even mean_every and each mean_start is a multiple of it (the chunk
 * length is mean_every, else 2); force_capacity must hold every recorded row.
 * ------------------------------------------------------------------------ */
typedef struct lbm_batch lbm_batch;

lbm_status lbm_batch_create(int32_t n, const lbm_grid *grids, const uint8_t *const *masks,
                            const lbm_params *params, void *cuda_stream, lbm_batch **out);
lbm_status lbm_batch_destroy(lbm_batch *b);

/* Last step of every member: member g runs t_end[g] steps (rounded up to a
 * multiple of the chunk length).  An end at or before the batch's current
 * step retires the member where it is (e.g. after it became unstable). */
lbm_status lbm_batch_set_end(lbm_batch *b, const int64_t *t_end);

/* t_end[g] = ceil(n_ft * nx_g / u_in_g): n_ft flow-through times. */
lbm_status lbm_batch_set_flowthroughs(lbm_batch *b, double n_ft);

/* Advance every unfinished member by n steps (rounded up to whole chunks,
 * stopping members at their end).  Asynchronous on the caller's stream. */
lbm_status lbm_batch_run(lbm_batch *b, int64_t n);

/* Run until every member reached its end. */
lbm_status lbm_batch_run_to_end(lbm_batch *b);

/* Wait for the batch; report latched device conditions of any member.  A
 * run is refused only while an unstable member is still live. */
lbm_status lbm_batch_sync(lbm_batch *b);

/* Wall distances of member g (as lbm_set_wall_distances); the next run
 * captures the step sequence again. */
lbm_status lbm_batch_set_wall_distances(lbm_batch *b, int32_t g, int64_t n, const int64_t *cell,
                                        const int8_t *dir, const double *q);

/* Borrow member g's context (valid until lbm_batch_destroy). */
lbm_status lbm_batch_member(lbm_batch *b, int32_t g, lbm_ctx **ctx);

typedef struct {
    int64_t t;               /* steps taken by the batch                           */
    int64_t chunk;           /* steps per captured graph                          */
    int32_t members, live;   /* members, members not yet at their end             */
    int32_t block_x, block_y;
    int64_t graph_captures, graph_launches, kernel_launches;
    int64_t lattice_updates; /* fluid cell updates performed so far               */
} lbm_batch_info;

lbm_status lbm_batch_get_info(const lbm_batch *b, lbm_batch_info *out);

/* Autotuner.  Times each candidate block shape (block_x, block_y) for
 * `trials` chunks (batch) or steps (context) on the real lattices, picks the
 * fastest, and resets the lattices to rest (t = 0, accumulators cleared), so
 * call it before the run.  With the environment variable LBM_AUTOTUNE_CACHE
 * set to a file path, results are read from / written to that JSON file,
 * keyed by device, storage, collision variant and grid sizes. */
lbm_status lbm_batch_autotune(lbm_batch *b, int32_t trials, int32_t *best_block_x, int32_t *best_block_y,
                              double *best_ms);
lbm_status lbm_autotune(lbm_ctx *ctx, int32_t trials, int32_t *best_block_x, int32_t *best_block_y,
                        double *best_ms);

/* Return a context to rest: f = w, t = 0, accumulators, forces and
 * snapshots cleared, instability latch reset. */
lbm_status lbm_reset(lbm_ctx *ctx);

/* Totals of a caller-owned population array, allocating nothing.
 *
 * The paper has no counterpart: this is a service for callers that cannot
 * call cudaMalloc where they need the totals -- a monitor thread checking
 * conservation between the steps of a solver it does not own (cudaMalloc and
 * cudaFree may synchronise the whole device and stall that solver), or an
 * application whose device memory is owned entirely by a host framework's
 * pool (a side allocation could fail or fragment it).  It computes the same
 * quantities as lbm_totals: out[0] = sum of f_i - w_i over fluid cells,
 * out[1..3] = momentum, by a deterministic two-pass FP64 reduction.
 *
 *   pdf          device (or managed) array of 27 slots x slot_stride values
 *                of `storage` type (any lbm_storage, LBM_F16C included)
 *                holding f_i - w_i in natural order (the layout a context
 *                holds at even time steps), cell c of direction i at
 *                i * slot_stride + c; slot_stride >= nx*ny*nz.
 *   mask         device (or managed) array of nx*ny*nz bytes, 1 = solid
 *                (skipped), or NULL.  A host pdf or mask returns LBM_ERR_ARG
 *                before anything is launched.
 *   out          4 doubles, host or device; for a host buffer the call waits
 *                for the stream (cudaStreamSynchronize), for a device buffer
 *                it does not.  Only a device `out` can be used while the
 *                stream is being captured into a graph.
 *
 * Its only scratch is a fixed array compiled into the library (512 KiB, held
 * by every GPU that loads the library until the process exits), which limits
 * grids to 2^30 cells: larger grids return LBM_ERR_ARG with a message in
 * lbm_last_error(NULL).  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture begins.  All calls share the array and
 * it keeps the last call's contents (each call writes every slot it reads, so
 * nothing needs clearing), but calls that overlap on the GPU race: serialise
 * them, e.g. on one stream.  Errors go to lbm_last_error(NULL). */
lbm_status lbm_totals_noalloc(const void *pdf, int32_t storage, int64_t slot_stride,
                              const uint8_t *mask, int32_t nx, int32_t ny, int32_t nz,
                              void *cuda_stream, double *out);

/* Last error message of this context (never NULL). */
/* Resampling of mean fields onto another grid (App. B: the simulated fields
 * are scaled down to the surrogate's 128x64x64 grid): cell-centred trilinear
 * interpolation.  Target cell o of an axis with n source and m target cells
 * samples the source at s = (o + 1/2) n/m - 1/2 clamped to [0, n - 1],
 * linearly between floor(s) and floor(s) + 1 (a factor 2 is the 2-cell mean,
 * a factor 1 the identity); the 3D map is the product of the three axes.
 *   src    device array of `channels` fields on the nx x ny x nz grid:
 *          src_layout 0 = [z][y][x][channels] (the layout of lbm_read_mean),
 *          1 = [channels][z][y][x].
 *   dst    device array [channels][mz][my][mx] (the FNO's input layout).
 * FP32 arithmetic; asynchronous on cuda_stream.  Host pointers, empty grids
 * or an unknown layout return LBM_ERR_ARG (message in lbm_last_error(NULL)). */
lbm_status lbm_resample(const float *src, int32_t nx, int32_t ny, int32_t nz, int32_t channels, int32_t src_layout,
                        float *dst, int32_t mx, int32_t my, int32_t mz, void *cuda_stream);

const char *lbm_last_error(const lbm_ctx *ctx);
const char *lbm_status_string(lbm_status s);

#ifdef __cplusplus
}
#endif
#endif /* GB300_LBM_H */
