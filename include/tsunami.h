/*
 * tsunami.h -- C ABI of the GB300 shallow-water AMR library.
 *
 * The library advances the shallow water equations over bathymetry (Sec. 2.1,
 * Eq. swe, without the drag term) with the wave-propagation form of Godunov's
 * method, limited second-order corrections and Godunov dimensional splitting
 * (Sec. 2.2, Eqs. wave_propagation_form, wave_propagation_2nd_order, _x, _y,
 * theta), on block-structured AMR patches (Sec. 3: hierarchy, recursive time
 * integration of Sec. 3.1 steps 1-4 -- refluxing (step 5) is omitted as in the
 * paper's GPU code -- and the regridding of Sec. 3.2).  All state lives in
 * device memory; every step of the method runs in the library's CUDA kernels.
 *
 * Conventions for every entry point:
 *   - returns TSU_OK (0) or a negative TSU_ERR_* code; nothing throws across
 *     the ABI; tsu_last_error() describes the last failure of a context;
 *   - the library owns all device memory (a pooled arena, Sec. 4.2 "Memory
 *     Pool"); the caller owns every host buffer it passes and the library
 *     never keeps a caller pointer after the call returns;
 *   - host arrays are row-major, x fastest: element (i, j) at [j * nx + i];
 *   - grids passed in (topography, surface, uplift) are node grids: value k
 *     sits at x0 + i dx, y0 + j dy and is sampled bilinearly; nx, ny >= 2;
 *   - levels are 1-based (level 1 covers the whole domain), scenarios 0-based;
 *   - a context is not thread-safe; calls on one context must be serialised.
 *
 * Error codes: TSU_ERR_ARG (bad argument or call order), TSU_ERR_CUDA (a CUDA
 * runtime error; the message names it), TSU_ERR_CFL (a level step ran with
 * Courant number above cfl_max; the step is kept and the run continues),
 * TSU_ERR_NESTING (an AMR invariant failed), TSU_ERR_OOM (device memory),
 * TSU_ERR_NOT_BUILT (the CUDA library is not loaded on a GPU), TSU_ERR_NAN (the
 * state is no longer finite), TSU_ERR_TIMEOUT (a kernel's bounded wait on the
 * device gave up), TSU_ERR_NEGDEPTH (a state the caller supplied has a
 * negative depth).
 */
#ifndef TSUNAMI_H
#define TSUNAMI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TSU_MAX_LEVELS 8
#define TSU_MAX_REGIONS 8

enum {
    TSU_OK = 0,
    TSU_ERR_ARG = -1,
    TSU_ERR_CUDA = -2,
    TSU_ERR_CFL = -3,
    TSU_ERR_NESTING = -4,
    TSU_ERR_OOM = -5,
    TSU_ERR_NOT_BUILT = -6,
    TSU_ERR_NAN = -7,           /* a wave speed or a cell's depth (surface) is not a finite number: the run
                                   has blown up; the context keeps returning this code */
    TSU_ERR_TIMEOUT = -8,       /* a kernel gave up waiting on the device (a row's bulk copy into shared
                                   memory did not complete within the poll budget of tsu_set_bulk_copies):
                                   that step's state is not valid; the context keeps returning this code */
    TSU_ERR_NEGDEPTH = -9       /* a state the caller supplied (written through tsu_level1_buffers, or
                                   restored by tsu_checkpoint_restore) has an interior cell with a negative
                                   depth, which the library never stores (it clips depths at zero): the
                                   step did nothing */
};

enum { TSU_F64 = 0, TSU_F32P = 1 };              /* precision of the state */
enum { TSU_BC_WALL = 0, TSU_BC_EXTRAP = 1 };     /* physical boundary rule */
enum { TSU_H = 0, TSU_HU = 1, TSU_HV = 2, TSU_ETA = 3, TSU_ZETA = 4, TSU_B = 5 };

typedef struct tsu_ctx tsu_ctx;

/* Run configuration.  Units: metres, seconds. */
typedef struct tsu_config {
    int precision;              /* TSU_F64: state (h, hu, hv) and B in FP64.
                                   TSU_F32P: state (eta' = h + B, hu, hv) and B in
                                   FP32 -- the surface-perturbation form */
    int nx, ny;                 /* level-1 cells */
    double x0, y0, dx, dy;      /* lower-left corner and level-1 cell size */
    int num_levels;             /* 1 .. TSU_MAX_LEVELS */
    int ratios[TSU_MAX_LEVELS]; /* ratios[k] refines level k+1 into level k+2 (space and time, Sec. 3) */
    int bc[4];                  /* left, right, bottom, top */
    double g;                   /* gravity, 9.81 */
    double drytol;              /* a cell is dry if h < drytol */
    double cfl_desired;         /* nu_d used to choose dt (Sec. 2.2 CFL condition) */
    double cfl_max;             /* largest Courant number accepted (Sec. 2.2: nu <= 1); see cfl_retake */
    double dt_max;              /* cap on the level-1 time step */
    int regrid_interval;        /* b: regrid every b steps of a level; also the flag buffer (Sec. 3.2) */
    double flag_eta_tol;        /* flag wet cells with |eta| > tol; <= 0 disables */
    double flag_depth_below;    /* flag cells with still-water depth -B < value; <= 0 disables */
    int patch_max;              /* largest fine patch side in fine cells */
    int level1_tile;            /* 0: level 1 is one patch; else square tiles of this side */
    int n_regions;
    double regions[TSU_MAX_REGIONS][6]; /* x1, y1, x2, y2, min_level, max_level (1-based levels) */
    int n_scenarios;            /* independent scenarios advanced together (>= 1) */
    int transverse;             /* 0: dimensional splitting, x then y (the paper's GPU scheme);
                                   1: unsplit update with transverse corrections (the original
                                   GeoClaw scheme Sec. 5 compares against; corner transport
                                   upwind, LeVeque 1997) */
    double cluster_eff;         /* Berger-Rigoutsos box efficiency, 0.7 if <= 0 */
    int use_graphs;             /* replay coarse steps as CUDA graphs: pairs of steps within one tsu_step
                                   call, and single steps (one graph per buffer-parity pattern) when no
                                   regrid falls in the next three; recaptured after every regrid */
    int use_cnn;                /* add the flag predictor's cells to the flags (tsu_cnn_set_weights) */
    int cnn_buffer;             /* flag buffer width used together with the predictor (instead of b) */
    double manning_n;           /* Manning coefficient of the drag (Sec. 2.1; the paper's runs use 0.025),
                                   applied after every level step as hu, hv <- hu, hv / (1 + dt D),
                                   D = n^2 g sqrt(hu^2 + hv^2) / h^(7/3), on wet cells; 0: none */
    int spherical;              /* 1: latitude-longitude grid -- x0, dx longitude and y0, dy latitude in
                                   degrees, the domain inside (-90, 90) -- advanced in capacity form
                                   (cell capacity = zone area over an equatorial cell's, latitude edges
                                   weighted by cos of their latitude); split scheme only */
    double earth_radius;        /* metres, spherical grids (<= 0: 6371 km) */
    int cfl_retake;             /* 1: a level-1 step whose Courant number exceeds cfl_max is discarded
                                   before any finer level moves and taken again from the same state with
                                   dt^1 = cfl_desired / (the largest speed / dx it saw); the decision is
                                   made on the device.  A retaken step that still exceeds cfl_max, and a
                                   finer level's step (its dt is fixed by the level-1 step), are kept and
                                   counted.  0: every step is kept and counted.  tsu_step returns
                                   TSU_ERR_CFL when a kept step exceeded cfl_max during the call */
} tsu_config;

typedef struct tsu_stats {
    double dt;                  /* last level-1 time step */
    double t;                   /* simulated time */
    double mass;                /* sum of h dx dy over level 1 (finer levels are averaged into it), FP64,
                                   summed in a fixed order: the same state gives the same bits */
    double cell_updates;        /* interior cells x steps summed over levels */
    long long cfl_violations;
    int patches[TSU_MAX_LEVELS];
    long long kernel_launches;  /* kernels this context has launched */
    long long regrids;          /* level rebuilds from flags (all scenarios of one call count once) */
    double regrid_host_ms;      /* host wall time inside those rebuilds, without regrid_wait_ms */
    double cluster_ms;          /* of which clustering the flag masks */
    long long cfl_retakes;      /* level-1 steps discarded and taken again (cfl_retake) */
    double regrid_wait_ms;      /* host time the rebuilds spent waiting for the queued steps to finish
                                   before the flags could be read (device time, not regrid work) */
    long long patches_renewed;  /* patches the rebuilds created (all levels and scenarios) */
    long long patches_reused;   /* of which had the box of an old patch and kept its memory block */
} tsu_stats;

/* Create a context.  cfg is copied.  cuda_stream: a cudaStream_t (for example
 * torch.cuda.current_stream().cuda_stream) or NULL for a stream the library
 * creates.  Allocates the device arena lazily.  Errors: TSU_ERR_ARG for an
 * invalid configuration, TSU_ERR_CUDA, TSU_ERR_NOT_BUILT. */
int tsu_create(const tsu_config *cfg, void *cuda_stream, tsu_ctx **out);

/* Destroy a context and release its device memory.  NULL is accepted. */
int tsu_destroy(tsu_ctx *ctx);

/* Message of the last failure of ctx (owned by ctx; valid until the next call). */
const char *tsu_last_error(tsu_ctx *ctx);

/* Add a bathymetry/topography grid B (metres, B < 0 under sea level; Sec. 2.1).
 * Where several grids cover a point the finest wins (later grids win ties).
 * Before tsu_init only.  B: nx*ny host doubles, copied. */
int tsu_add_topo(tsu_ctx *ctx, const double *B, int nx, int ny, double x0, double y0, double dx, double dy);

/* Initial sea surface eta of one scenario (default 0); h = max(0, eta - B).
 * Before tsu_init only.  eta: nx*ny host doubles, copied. */
int tsu_set_eta(tsu_ctx *ctx, int scenario, const double *eta, int nx, int ny,
                double x0, double y0, double dx, double dy);

/* Initial depth-averaged velocities u, v of one scenario (default 0), on one
 * node grid (both nx*ny host doubles, copied; same convention as tsu_set_eta):
 * at tsu_init every wet cell gets hu = h u, hv = h v.  Before tsu_init only. */
int tsu_set_velocity(tsu_ctx *ctx, int scenario, const double *u, const double *v, int nx, int ny,
                     double x0, double y0, double dx, double dy);

/* Instantaneous seafloor deformation (Sec. 5.1.1 dtopo, applied at once):
 * B += dB on every cell of every level with h unchanged, so the surface rises
 * with the seafloor; later patches sample it too.  May be called before or
 * after tsu_init.  dB: nx*ny host doubles, copied. */
int tsu_add_uplift(tsu_ctx *ctx, int scenario, const double *dB, int nx, int ny,
                   double x0, double y0, double dx, double dy);

/* Build level 1 (tiled per cfg), sample B, set the state, and build the finer
 * levels by flagging and clustering (Sec. 3.2).  Requires one tsu_add_topo. */
int tsu_init(tsu_ctx *ctx);

/* Advance n coarse (level-1) steps with the recursive integration of Sec. 3.1,
 * regridding every regrid_interval steps of each level.  t_out (may be NULL)
 * receives n_scenarios doubles: the simulated time of each scenario.
 * Returns TSU_ERR_CFL if a kept level step exceeded cfl_max (the work is done;
 * see cfl_retake), TSU_ERR_NAN if a speed or a depth is not a finite number,
 * TSU_ERR_TIMEOUT if a kernel gave up waiting (tsu_set_bulk_copies),
 * TSU_ERR_ARG after tsu_step_level left a coarse step unfinished.  The first
 * step after tsu_level1_buffers or tsu_checkpoint_restore checks every level's
 * interior depths first and returns TSU_ERR_NEGDEPTH, doing nothing, if one is
 * negative. */
int tsu_step(tsu_ctx *ctx, int n_coarse_steps, double *t_out);

/* One step of one level (1-based), the unit of the recursion of Sec. 3.1
 * (step 1 of its algorithm: advance level l by one step of dt^l = dt^1 / R_l),
 * for debugging and tests.  Calls must follow the recursion's order:
 *   - level 1 only between coarse steps: it chooses dt^1 (Sec. 2.2 CFL
 *     condition) and takes the level-1 step (with its retake);
 *   - level l > 1 only while the step of level l - 1 has substeps of level l
 *     pending (r_{l-1} per step of level l - 1) and level l has none of its own
 *     pending; the substep's ghost cells are interpolated at time fraction
 *     k / r_{l-1}.
 * A step whose next finer level has patches leaves that level's r_l substeps
 * pending.  The last pending substep of a level completes its parent's step:
 * averaging onto the parent, the step count, the regrids every
 * regrid_interval steps, and -- when the parent is level 1 -- the end of the
 * coarse step (time advanced, gauges sampled).  Steps taken in this order
 * give tsu_step's results bit for bit.  t_out (may be NULL): n_scenarios
 * doubles, the time of each scenario at the end of the last finished coarse
 * step.  Out of order, an empty level, or a level outside 1..num_levels:
 * TSU_ERR_ARG, nothing done.  tsu_step fails with TSU_ERR_ARG while a coarse
 * step is unfinished.  Other codes as tsu_step. */
int tsu_step_level(tsu_ctx *ctx, int level, double *t_out);

/* Regenerate levels level+1 .. num_levels from flags on `level` (Sec. 3.2). */
int tsu_regrid(tsu_ctx *ctx, int scenario, int level);

/* The host step of a regrid on its own (Sec. 3.2, Berger-Rigoutsos
 * clustering as read in the library): cluster the 0/1 mask `flags` (ny rows of
 * nx bytes, row-major, host memory) into rectangles, accepting a tight box
 * when its flags fill at least `eff` of it and every cell of it is nonzero in
 * `nestable` (same layout; NULL = everywhere nestable), then split boxes into
 * near-equal pieces of at most patch_max / ratio cells per side.  Writes
 * (i0, j0, w, h) per box to `boxes` (4 ints each, caller-owned, room for
 * max_boxes) and the count to *n_boxes.  Needs no GPU and no context.
 * Errors: TSU_ERR_ARG (bad sizes, NULL flags or outputs, or more than
 * max_boxes boxes; *n_boxes then holds the count needed). */
int tsu_cluster_flags(const unsigned char *flags, const unsigned char *nestable, int nx, int ny, double eff,
                      int ratio, int patch_max, int *boxes, int max_boxes, int *n_boxes);

/* Number of patches of a level, and their boxes: 4 ints per patch (i0, j0, nx,
 * ny) in global cell indices of that level, in the library's patch order. */
int tsu_num_patches(tsu_ctx *ctx, int scenario, int level, int *n);
int tsu_get_patches(tsu_ctx *ctx, int scenario, int level, int *boxes, int max_patches, int *n);

/* Copy the interior of patch k of a level to host: h, hu, hv, B, each
 * nx*ny doubles (any may be NULL).  h is the depth in both precisions. */
int tsu_get_patch(tsu_ctx *ctx, int scenario, int level, int k, double *h, double *hu, double *hv, double *B);

/* Sample a field on the points (x0 + i dx, y0 + j dy), i < nx, j < ny:
 * piecewise constant from the finest patch (level == 0) or from level
 * `level` only; NaN where nothing covers a point.  Fields: TSU_H, TSU_HU,
 * TSU_HV, TSU_ETA (h + B), TSU_ZETA (Eq. zeta: h where B > 0, else h + B),
 * TSU_B.  dst: nx*ny host doubles, owned by the caller; the call writes
 * every element and returns after the copy has landed.  Large fields are
 * copied straight into dst where the device reaches pageable host memory
 * through the host's page tables (coherent CPU-GPU platforms), else through
 * a page-locked staging buffer. */
int tsu_read_field(tsu_ctx *ctx, int scenario, int level, int field, double *dst, int nx, int ny,
                   double x0, double y0, double dx, double dy);

/* Gauges (Sec. 5.1.2): points xy[2k], xy[2k+1]; before the first tsu_step.
 * After every coarse step the library records eta at each gauge from the
 * finest patch containing it (bilinear between cell centres). */
int tsu_add_gauges(tsu_ctx *ctx, const double *xy, int n);

/* Read the recorded samples: t[s*ns + scen], eta[(s*ns + scen)*ngauges + g]
 * for samples s < *n_written <= max_samples. */
int tsu_read_gauges(tsu_ctx *ctx, double *t, double *eta, int max_samples, int *n_written);

/* Statistics of one scenario (synchronises the stream). */
int tsu_get_stats(tsu_ctx *ctx, int scenario, tsu_stats *out);

/* Launch shape of the patch update (the autotuner's knobs): step_threads
 * threads per CTA and seg_rows rows per CTA (patches taller than that are cut
 * into row segments).  step_threads is 64, 128 or 256, or also 32 for the
 * split FP32 update.  A CTA updates a strip of 2 step_threads - 4 columns in
 * the split FP32 update (two columns per thread), step_threads - 4 otherwise.
 * The split FP32 update runs as two kernels: the knobs shape its x-sweep
 * kernel (rows counted over the patch's ghost rows too); its y-sweep kernel
 * always takes strips of 64 columns and 64 rows.  0 restores the defaults.
 * Results do not depend on either.  Returns TSU_ERR_ARG for any other value. */
int tsu_set_tuning(tsu_ctx *ctx, int step_threads, int seg_rows);

/* How the FP32 split update's x-sweep kernel brings rows into shared memory.
 * enable = 0 (the default): every thread copies its own columns with
 * cp.async.  enable = 1: one thread copies each field's row segment with a
 * bulk copy (cp.async.bulk) that completes on an mbarrier, and every thread
 * polls that barrier at most `polls` times before it gives up (2^22 is far
 * above what a copy takes).  A wait that runs out stops the work item's
 * further copies, waits for those in flight, and makes tsu_step return
 * TSU_ERR_TIMEOUT; polls = 0 gives up at the first wait (a test of that path;
 * no GPU fault is involved).  Results are the same bits either way; the bulk
 * copies measured slower on GB300.  Errors: TSU_ERR_ARG for enable not 0 or 1
 * or polls outside [0, 2^32 - 1]. */
int tsu_set_bulk_copies(tsu_ctx *ctx, int enable, long long polls);

/* Autotuner: time every launch shape of the patch update (threads per CTA
 * 64/128/256, and 32 for the split FP32 update, x rows per work item
 * 32/64/128/256, or 16/32/64/128 for the split FP32 update) on the context's current
 * levels with `reps` zero-length steps each -- the kernels do all their work
 * but the state is unchanged -- and keep the fastest.  Outputs (any may be
 * NULL): the chosen shape and its time per step of all levels in ms. */
int tsu_autotune(tsu_ctx *ctx, int reps, int *best_threads, int *best_seg_rows, double *best_ms);

/* Checkpoint and restart of a whole simulation, between tsu_step calls
 * (after tsu_init).  tsu_checkpoint_save writes every patch of every level and
 * scenario -- its box and its current state and B, ghost cells included --
 * with the time, time step, wave-speed rates, step and regrid counters and
 * the gauge records into buf (caller-owned host memory, cap bytes) and the
 * size into *written.  buf = NULL with cap = 0 only queries the size.  A
 * checkpoint is taken between coarse steps, where the state before the next
 * step is all that the next step reads, so one time level suffices.
 * tsu_checkpoint_restore replaces the hierarchy of an initialised context
 * with a checkpoint's.  The context must have the same tsu_config (compared
 * byte for byte), the same topography and uplift layers (new patches sample
 * B from them at later regrids) and the same gauges; predictor weights are
 * set again with tsu_cnn_set_weights.  The run then continues exactly as the
 * saved one would have.  Errors: TSU_ERR_ARG (buffer too small, not a
 * checkpoint, another configuration, truncated or corrupt data).  The next
 * tsu_step or tsu_step_level checks the restored depths (TSU_ERR_NEGDEPTH). */
int tsu_checkpoint_save(tsu_ctx *ctx, void *buf, size_t cap, size_t *written);
int tsu_checkpoint_restore(tsu_ctx *ctx, const void *buf, size_t n);

/* Synchronise the context's stream. */
int tsu_sync(tsu_ctx *ctx);

/* Device pointer of level-1 patch 0's current state buffers, for tests and
 * the benchmark (fields h|eta', hu, hv, B; element type by precision;
 * row pitch in elements; interior cell (i, j) at [(j + 2) * pitch + i + 2]).
 * The caller may write the state through them; the next tsu_step or
 * tsu_step_level checks its depths (TSU_ERR_NEGDEPTH). */
int tsu_level1_buffers(tsu_ctx *ctx, void **h, void **hu, void **hv, void **B, int *pitch);

/* Per-level timing of the patch update, for measurement.  enable != 0 starts
 * recording a pair of CUDA events on the library's stream around the update
 * launches of every level step (the x- and y-sweep kernels of the FP32 split
 * update, the fused FP64 kernel, and on level 1 the retake launch with its
 * bookkeeping kernel); coarse steps then run without graphs.  Either call
 * drops what was recorded so far.  Synchronises the stream. */
int tsu_profile_levels(tsu_ctx *ctx, int enable);

/* What tsu_profile_levels recorded since it was enabled or last read, per
 * level l < max_levels (0-based): ms[l] the summed device time of its update
 * launches (CUDA events), cells[l] the interior cells they updated (one count
 * per level step, all scenarios), steps[l] the level steps, kernels[l] the
 * kernels launched.  All four are host arrays of max_levels entries; the
 * record is cleared.  Synchronises the stream. */
int tsu_level_update_times(tsu_ctx *ctx, double *ms, double *cells, long long *steps, long long *kernels,
                           int max_levels);

/* Halo exchange of a level split over ranks (one process per GPU).  Before
 * each level step a rank needs, in its patches' 2-cell ghost rings (Sec. 3.1
 * step 2: ghost cells from same-level neighbours), the cells that patches on
 * other ranks own.  These two calls move such boxes between the patches'
 * current state buffers and a contiguous device buffer that the caller owns
 * and sends or receives (for example with NCCL through torch.distributed):
 *   msgs: n_msgs messages of 5 host ints (k, i0, j0, i1, j1) -- patch k of the
 *         scenario on the level (the order of tsu_get_patches) and a
 *         half-open box in level indices inside that patch and its ghost ring
 *         (pack: normally in the interior; unpack: in the ghost ring);
 *   dev_buf: device memory of buf_elems elements of the state's precision
 *         (double for TSU_F64, float for TSU_F32P, where q0 is eta'), holding
 *         per message in order the fields q0, hu, hv, each a row-major
 *         (j1 - j0) x (i1 - i0) block: 3 sum (i1 - i0)(j1 - j0) elements.
 * tsu_halo_pack copies the boxes out of the patches, tsu_halo_unpack into
 * them.  Both run on the library's stream and return after it finishes.
 * Errors: TSU_ERR_ARG (no such patch, a box outside the patch's storage, a
 * buffer too small, before tsu_init), TSU_ERR_CUDA. */
int tsu_halo_pack(tsu_ctx *ctx, int scenario, int level, const int *msgs, int n_msgs, void *dev_buf,
                  long long buf_elems);
int tsu_halo_unpack(tsu_ctx *ctx, int scenario, int level, const int *msgs, int n_msgs, const void *dev_buf,
                    long long buf_elems);

/* Time n steps of a one-level context with CUDA events on the library's stream
 * after `warmup` untimed steps, each step the kernels tsu_step launches for it
 * (start of the step, ghost fill, boundaries, the patch update, the CFL check
 * and, with cfl_retake, the retake launch and its check, end of the step);
 * kernel_ms_out gets the mean milliseconds of the patch update's launches per
 * step and step_ms_out those of the whole step.  Advances the solution.
 * Errors: TSU_ERR_ARG (more than one level, n < 1, before tsu_init). */
int tsu_time_level1_steps(tsu_ctx *ctx, int warmup, int n, double *kernel_ms_out, double *step_ms_out);

/* ---------------------------------------------------------------------------
 * Refinement-flag predictor.  The buffer of b cells around flagged cells
 * (Sec. 3.2) is there so waves do not leave the refined region before the next
 * regrid; it widens every patch by 2b cells.  A small CNN -- three 3x3
 * convolutions with 16 channels and ReLU, a 1x1 head to one logit per cell --
 * predicts, from 5 features of a level (eta / 0.1 m on wet cells,
 * clip(-B / 1000 m, -1, 5), |hu| / 10, |hv| / 10 m^2/s, the criterion flag),
 * which cells the criterion will flag at the next regrid.  With use_cnn the
 * flags become criterion(now) OR prediction, dilated by cnn_buffer instead of
 * b; the criterion stays both the fallback and the arbiter (cells it flags are
 * always refined).  Parameters: a flat FP32 vector (per layer W (C_out, C_in,
 * k, k) then b (C_out); layers 5->16 3x3, 16->16 3x3, 16->16 3x3, 16->1 1x1).
 * ------------------------------------------------------------------------- */

/* Number of parameters of the predictor: 5,393 (three 3x3 layers 5->16, 16->16,
 * 16->16 with biases: 736 + 2,320 + 2,320; the 1x1 head 16->1: 17). */
int tsu_cnn_num_params(void);

/* Logits (n, h, w) of host inputs x (n, 5, h, w); fp16 != 0: FP16 activations
 * and weights with FP32 accumulation (the inference path), else FP32. */
int tsu_cnn_forward(const float *theta, const float *x, int n, int h, int w, int fp16, float *logits);

/* Mean binary cross-entropy with logits over the cells where m = 1 and its
 * gradient with respect to theta (host buffers; targets t in {0, 1}). */
int tsu_cnn_loss_grad(const float *theta, const float *x, const float *t, const float *m, int n, int h, int w,
                      double *loss, float *grad);

/* Train theta in place on the GPU: `steps` Adam updates (lr) on mini-batches
 * of `batch` planes drawn from the host dataset (x, t, m) with a generator
 * seeded by `seed`; returns the loss of the first and last batch. */
int tsu_cnn_train(float *theta, const float *x, const float *t, const float *m, int n, int h, int w, int steps,
                  int batch, float lr, unsigned seed, double *loss_first, double *loss_last);

/* Give a context the predictor's parameters (n = tsu_cnn_num_params()). */
int tsu_cnn_set_weights(tsu_ctx *ctx, const float *theta, int n);

/* The predictor's input planes of one level (5 planes of nx_l x ny_l floats,
 * zero where no patch covers a cell) and the criterion flags before the
 * buffer (nx_l x ny_l bytes), both to host; either may be NULL. */
int tsu_cnn_features(tsu_ctx *ctx, int scenario, int level, float *features, unsigned char *flags);

/* ---------------------------------------------------------------------------
 * Stepping without allocating.  The paper has no counterpart to this entry
 * point; it exists for callers that must not call cudaMalloc: applications
 * whose device memory is owned end to end by their own allocator (a
 * framework's caching allocator, or a service that reserves all of HBM up
 * front), and latency-critical loops where a cudaMalloc could block or fail.
 *
 * One dimensionally split step (the same kernels as tsu_step) of a single
 * uniform grid of nx x ny cells held in the caller's device memory `block`:
 * 7 fields of field_stride elements each -- buffer 0 (q0, hu, hv), buffer 1
 * (q0, hu, hv), B -- with element (i, j), -2 <= i < nx + 2, -2 <= j < ny + 2,
 * at (j + 2) * pitch + (i + 2).  Elements are double (TSU_F64: q0 = h) or
 * float (TSU_F32P: q0 = eta' = h + B).  The step reads buffer `cur`, first
 * overwriting the ghost rings of buffer `cur` and of B with the boundary rules
 * bc[4] (host ints, left, right, bottom, top) -- so the caller fills interiors
 * only -- and writes the interior of buffer 1 - cur.  dt is the
 * caller's; max_speeds (2 host doubles) receives the largest |wave speed| of
 * the x and y sweeps, from which the caller picks the next dt (+infinity:
 * a cell's depth or surface came out not a finite number).  The call copies
 * the speeds to the host and synchronises `cuda_stream` (NULL: the default
 * stream) before it returns, so it must not be issued while that stream is
 * being captured into a CUDA graph.
 *
 * It allocates nothing: its scratch (about 1 MiB, mostly the work-item table)
 * is a file-scope __device__ array that every GPU loading the library holds
 * until the process exits.  The first call on a device looks up that array's
 * address (once per device, with that device current).  Every call shares the
 * array and leaves its contents behind; each call rewrites what it uses and
 * clears the speed accumulator, but calls that overlap on the GPU (other
 * streams or host threads) race on it -- serialise them.
 *
 * Limits: 1 <= nx, ny <= TSU_NOALLOC_MAX_SIDE; pitch >= nx + 4; field_stride
 * >= pitch * (ny + 4); block aligned to its element size.  Anything else,
 * including a larger grid, returns TSU_ERR_ARG without launching work.
 * TSU_ERR_CUDA reports a CUDA failure.
 * ------------------------------------------------------------------------- */
#define TSU_NOALLOC_MAX_SIDE 16384
int tsu_grid_step_noalloc(int precision, void *block, int nx, int ny, int pitch, long long field_stride, int cur,
                          double dx, double dy, double dt, double g, double drytol, const int *bc,
                          double *max_speeds, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
