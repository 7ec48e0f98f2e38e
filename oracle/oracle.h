/*
 * oracle.h -- plain FP64 CPU oracle for the shallow-water wave-propagation
 * update on block-structured AMR patches (Qin, LeVeque & Motley, "Efficient
 * Tsunami Modeling on Adaptive Grids with GPUs").
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the slow, obviously-correct
 * statement of what the GPU library computes.  Only the test suite, the
 * package smoke check and the benchmark's CPU-baseline leg may build, load
 * or call it.  It shares no source with the CUDA library and includes
 * nothing from it.
 *
 * Everything is double precision, compiled with -ffp-contract=off so the
 * arithmetic is exactly the IEEE sequence written in the source.
 *
 * Parity status per function (see the pins in tests/test_oracle_*.py):
 *   ora_riemann       pinned: equal states, lake at rest over a step,
 *                     mirror symmetry, wall reflection, conservation of
 *                     the flux jump (sum of f-waves == flux difference),
 *                     non-negative depths of every state of its fan (bed
 *                     steps, dry fronts, overtopping, supersonic flow) and
 *                     of the first-order update built on it at Courant 1/2
 *                     (Sec. 2.2); a single shock is one wave at the
 *                     Rankine-Hugoniot speed.  Agreement with George's
 *                     (2008) augmented solver in particular is not checked:
 *                     the paper cites that solver without stating it, and
 *                     the construction here is the one the design records
 *                     (reading r1).
 *   ora_mc_limiter    pinned: MC table values (textbook closed form).
 *   patch step        pinned: 1D dam break (Stoker, Ritter) closed forms,
 *                     mass conservation with walls, lake at rest,
 *                     Gaussian-hump mirror symmetry; the CFL retake: a dam
 *                     break onto a dry bed retakes its first step with the
 *                     closed-form dt of its front speed (Sec. 2.2).
 *   multi-patch level pinned: one patch == tiled level, bitwise.
 *   AMR               pinned: lake at rest through regrid/interp/average,
 *                     full-coverage level 2 == uniform fine grid.
 *   clustering        pinned: hand-drawn masks, coverage/efficiency/
 *                     disjointness invariants.
 */
#ifndef ORACLE_H
#define ORACLE_H

#define ORA_MAX_LEVELS 8
#define ORA_MAX_REGIONS 8

enum { ORA_BC_WALL = 0, ORA_BC_EXTRAP = 1 };
enum { ORA_F_H = 0, ORA_F_HU = 1, ORA_F_HV = 2, ORA_F_ETA = 3, ORA_F_ZETA = 4, ORA_F_B = 5 };

typedef struct ora_config {
    int nx, ny;                 /* level-1 cells */
    double x0, y0, dx, dy;      /* level-1 lower-left corner and cell size */
    int num_levels;
    int ratios[ORA_MAX_LEVELS]; /* ratios[l] refines level l+1 -> l+2 (1-based levels) */
    int bc[4];                  /* left, right, bottom, top */
    double g, drytol, cfl_desired, cfl_max, dt_max;
    int regrid_interval;        /* b: regrid every b steps of a level; also the flag buffer width */
    double flag_eta_tol;        /* flag wet cells with |eta| > tol (<= 0 disables) */
    double flag_depth_below;    /* flag cells with -B < value (<= 0 disables) */
    int patch_max;              /* max fine-patch side in fine cells */
    int level1_tile;            /* 0: level 1 is one patch; else tiles of this side */
    int n_regions;
    double regions[ORA_MAX_REGIONS][6]; /* x1, y1, x2, y2, min_level, max_level */
    int n_scenarios;
    int transverse;             /* 0: dimensional splitting (the paper's GPU scheme) */
    double cluster_eff;         /* Berger-Rigoutsos acceptance efficiency */
    double manning_n;           /* Manning coefficient of the drag D (Sec. 2.1); 0: no friction */
    int spherical;              /* 1: x = longitude, y = latitude in degrees (capacity form) */
    double earth_radius;        /* metres (spherical; <= 0: 6371 km) */
    int reflux;                 /* 1: refluxing of the mass (Sec. 3.1 step 5; split scheme, plane grids) */
    int cfl_retake;             /* 1: a level-1 step with nu > cfl_max is discarded and taken again */
} ora_config;

typedef struct ora_rp {
    double Z[3][3];  /* f-wave p, component (mass, normal momentum, transverse momentum) */
    double s[3];     /* speeds s1 <= s2 <= s3 */
    int wallL, wallR;
} ora_rp;

/* low-level pieces, exported for the pins */
void ora_riemann(double g, double drytol,
                 double hL, double hnL, double htL, double BL,
                 double hR, double hnR, double htR, double BR, ora_rp *out);
double ora_mc_limiter(double theta);
int ora_cluster(const unsigned char *flags, const unsigned char *nestable, int nx, int ny,
                double eff, int ratio, int patch_max, int *boxes, int max_boxes);

/* whole-method driver */
void *ora_create(const ora_config *cfg);
void ora_destroy(void *o);
int ora_add_topo(void *o, const double *B, int nx, int ny, double x0, double y0, double dx, double dy);
int ora_set_eta(void *o, int scen, const double *eta, int nx, int ny, double x0, double y0, double dx, double dy);
/* initial velocities u, v (same node-grid convention as the surface): at
 * init every wet cell gets hu = h u, hv = h v */
int ora_set_velocity(void *o, int scen, const double *u, const double *v, int nx, int ny, double x0, double y0,
                     double dx, double dy);
int ora_add_uplift(void *o, int scen, const double *dB, int nx, int ny, double x0, double y0, double dx, double dy);
int ora_init(void *o);
int ora_step(void *o, int n_coarse, double *t_out);
int ora_regrid(void *o, int scen, int level);
int ora_num_patches(void *o, int scen, int level);
int ora_get_patch(void *o, int scen, int level, int k, int *box, double *h, double *hu, double *hv, double *B);
int ora_read_field(void *o, int scen, int level, int field, double *dst, int nx, int ny,
                   double x0, double y0, double dx, double dy);
int ora_add_gauges(void *o, const double *xy, int n);
int ora_read_gauges(void *o, double *t, double *eta, int max_samples, int *n_written);
int ora_stats(void *o, int scen, double *out /* [dt, t, mass_l1, cfl_violations, cell_updates,
                                                n_patches[ORA_MAX_LEVELS], cfl_retakes, neg_clips] */);

#endif
