// amr_kernels.h -- views and launchers of the kernels around the patch update.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "tsu_device.h"

namespace tsu {

constexpr int kMaxLevels = 8;

// Where one ghost cell of a patch takes its value from, found once per patch
// table (the search over the neighbour boxes does not run at every fill):
// src >= 0 is the element offset in the arena of the same-level neighbour's
// interior cell in field 0 of buffer 0, sfs that patch's field stride; the
// negative codes below mark the other cases.
struct __align__(16) GhostSrc {
    long long src;
    long long sfs;
};
constexpr long long kGhostSkip = -1;     // outside the level's index space (physical boundary)
constexpr long long kGhostInterp = -2;   // no same-level neighbour: space-time interpolation from the coarser level
constexpr long long kGhostNone = -3;     // no neighbour on the coarsest level: a tiling error

// Device view of one level's tables (all scenarios).
struct LevelView {
    const PatchDesc *descs;
    void *arena;
    int nxl, nyl;           // level index space
    const int *nbrs;        // same-level neighbour lists
    const int *cmap;        // coarse-level patch index maps
    const int *olds;        // regrid: overlapping old patches
    const double *kap;      // latitude-longitude grids: capacity of row J at [J + 2]; null on Cartesian grids
    const double *ced;      // latitude-longitude grids: relative length of the latitude edge below row J at [J + 2]
    const GhostSrc *gmap;   // ghost-cell sources, patch after patch in ghost-ring order
    const long long *goff;  // first entry of each patch in gmap
    const int2 *ilist;      // ghost cells interpolated from the coarser level: (patch, ghost-ring index)
    const int *icount;      // entries of ilist
};

// Device control block of a context: per scenario dt, time, rates, counters.
struct CtrlView {
    double *dt1, *t;
    float *dt1f;                 // FP32 copy of dt1 for the perturbation-form kernel
    double *rate;                // [scen][max_levels]
    double *cell_updates;        // [scen]
    const double *cells;         // [scen][max_levels] interior cells per level
    long long *cfl_viol;         // [scen]
    unsigned long long *smax;    // [scen][2]
    int *retake;                 // [scen] 1: the level-1 step is being retaken (the step kernels' gate)
    long long *retakes;          // [scen] level-1 steps retaken
    int *err;                    // device error flag (TSU_DEV_ERR_*)
    int max_levels;
};


struct TopoDev {
    int nx, ny;
    double x0, y0, dx, dy;
    const double *v;
};

// Sampling grid k at the cell centres of one level is separable: whether the
// centre lies in the grid's extent, and the clamped node index and fraction
// of the bilinear interpolation, depend on the column alone in x and on the
// row alone in y.  AxisTab holds them per grid and column ([k nx + I]) and per
// grid and row ([k ny + J]), computed by the same operations as at the cell.
struct AxisTab {
    int *ci, *rj;                // node index i of column I, j of row J
    double *ct, *rt;             // interpolation fractions tx, ty
    unsigned char *cin, *rin;    // x_I within [x0, x0 + (nx - 1) dx], y_J likewise
    int nx, ny;                  // the level's columns and rows
};

// Base topography grids [0, nbase), then uplift layers and surface grids;
// scen[k] tells which scenario a layer belongs to (-1: not an uplift layer).
struct TopoSet {
    const TopoDev *grids;
    const int *scen;
    const int *eta_index;        // per scenario s: [3s] initial surface, [3s+1] u, [3s+2] v grid index or -1
    int nbase, ngrids;
    double drytol;               // initial velocities apply to wet cells only
    AxisTab tab;                 // storage for k_init_patches: ngrids (nx + ny) entries of each array
};

// Window of a level plane on which the flag predictor runs (x0, y0, w, h), and
// the target box inside it whose predictions are used (tx0, ty0, tw, th; the
// window adds the predictor's 3-cell receptive margin where the plane allows)
struct CnnWindow {
    int x0, y0, w, h;
    int tx0, ty0, tw, th;
};

struct FlagArgs {
    uint8_t *raw, *cov;
    const int *scen_slot;        // plane of each scenario or -1
    double eta_tol, depth_below, drytol;
    // FP32 state: the largest floats <= eta_tol and <= -depth_below, and drytol in FP32
    float eta_tol_f, depth_neg_f, drytol_f;
    double x0, y0, dxl, dyl;
    int n_regions, newlev;
    double regions[6 * kMaxLevels];
};

struct BcArgs {
    const int *list;             // patches with a side on the domain boundary
    int bc[4];
};

struct GaugeLoc {
    int level, patch;            // finest patch containing the gauge, or patch = -1
};

struct GaugeArgs {
    const GaugeLoc *loc;         // [scen][gauge]
    const double *xy;
    double *eta, *t;
    long long *nsamp;
    int nscen, ngauges;
    double x0, y0;
    LevelView levels[kMaxLevels];
    int curs[kMaxLevels];
    double dxl[kMaxLevels], dyl[kMaxLevels];
};

// ghost-cell sources of every patch of a level (L.gmap, L.goff), after its patch table or neighbour lists
// change; ratio 0 on the coarsest level
// (ilist, icount: the interpolated cells' list and its length, zeroed here; ilist holds one entry per ghost cell)
int k_ghost_map(const LevelView &L, GhostSrc *gmap, int2 *ilist, int *icount, int npatch, int maxring, int ratio,
                cudaStream_t st);
int k_ghost_fill(int prec, const LevelView &L, const LevelView &C, int npatch, int maxring, int cur, int cur_c,
                 int ratio, double alpha, double drytol, int *err, cudaStream_t st);
int k_bc(int prec, const LevelView &L, const BcArgs &b, int nlist, int maxring, int cur, int do_state, int do_B,
         cudaStream_t st);
int k_average(int prec, const LevelView &F, const LevelView &C, int npatch, int maxcells, int cur_f, int cur_c, int r,
              double drytol, int *err, cudaStream_t st);
// Old: the level's previous patch table at a regrid (B copied where an old patch held the cell), or a view
// with null descs
int k_init_patches(int prec, const LevelView &L, const LevelView &Old, const int *list, int nlist, int maxcells,
                   const TopoSet &ts, int cur, int set_state, double x0, double y0, double dxl, double dyl,
                   cudaStream_t st);
int k_uplift(int prec, const LevelView &L, int npatch, int maxcells, const TopoDev &U, int scen, int cur, double x0,
             double y0, double dxl, double dyl, cudaStream_t st);
int k_regrid_init(int prec, const LevelView &L, const LevelView &Old, const LevelView &C, const int *list, int nlist,
                  int maxcells, int cur, int cur_c, int ratio, double drytol, int *err, cudaStream_t st);
int k_flag(int prec, const LevelView &L, int npatch, int maxcells, int cur, const FlagArgs &fa, cudaStream_t st);
// a window (i0, j0, w, h) of a level's index plane
struct Win {
    int i0, j0, w, h;
};
// dilation along x (dir 0) or y (dir 1) over the window W of every plane
int k_dilate(const uint8_t *src, uint8_t *dst, int nx, int ny, int nplanes, int b, int dir, const Win &W,
             cudaStream_t st);
// bounding box (min i, min j, max i, max j) of the flagged cells of each plane
// (within the window W, null: the whole plane); box preset to (nx, ny, -1, -1)
int k_flag_bbox(const uint8_t *F, int nx, int ny, int nplanes, int *box, cudaStream_t st, const Win *W = nullptr);
// coarse maps of a level's npatch patches from their coarse candidate lists
int k_fill_cmap(const PatchDesc *descs, const PatchDesc *cdescs, const int *cand, int npatch, int *cmap, cudaStream_t st);
// box (i0, j0, w, h) of the nx-wide byte plane N (bit 0 flag, bit 1 nestable)
// packed 4 cells per byte, rows ps bytes apart (ps >= (w + 3) / 4)
int k_pack_flags(const uint8_t *N, int nx, int i0, int j0, int w, int h, int ps, uint8_t *out, cudaStream_t st);
// proper nesting over the window W (tmp: a plane set of scratch, the x pass of the erosion)
int k_nest(uint8_t *F, uint8_t *N, const uint8_t *cov, uint8_t *tmp, int nx, int ny, int nplanes, const FlagArgs &fa,
           const Win &W, cudaStream_t st);
// count of interior cells with a negative depth over a level's patches (into *count)
int k_depth_check(int prec, const LevelView &L, int npatch, int maxcells, int cur, int *count, cudaStream_t st);
int k_cell_speed(int prec, const LevelView &L, const int *list, int nlist, int maxcells, int cur, double g,
                 double drytol, unsigned long long *smax, cudaStream_t st);
// one box of a halo exchange: patch (index in the level), box origin and
// size in level indices, element offset of its three fields in the buffer
struct HaloMsg {
    int patch, i0, j0, w, h;
    long long off;
};
// pack (unpack = 0: patch buffers -> buf) or unpack (buf -> patch buffers) n boxes
int k_halo(int prec, const LevelView &L, const HaloMsg *msgs, int n, int cur, void *buf, int unpack, cudaStream_t st);

// end_step 1 (modes 0 and 3): the step was a one-level grid's whole coarse step (mode 3: after its
// retake launch), and the kernel also advances t by dt^1 (the work of k_end_step, saving its launch)
int k_post_level(const CtrlView &cv, int level, int nscen, double R, double dx, double dy, double cfl_max,
                 double cfl_desired, int mode,
                 cudaStream_t st, int end_step = 0);
int k_begin_step(const CtrlView &cv, int nscen, int nlev, const double *Rl, double cfl_desired, double dt_max,
                 cudaStream_t st);
int k_end_step(const CtrlView &cv, int nscen, cudaStream_t st);
int k_gauges(int prec, const GaugeArgs &ga, const CtrlView &cv, cudaStream_t st);
// maxpts: an upper bound on the output points one patch covers (sizes the grid)
int k_read_field(int prec, const LevelView &L, int npatch, int maxpts, int cur, int scen, int field, double *dst, int nx,
                 int ny, double x0, double y0, double dx, double dy, double X0, double Y0, double dxl, double dyl,
                 cudaStream_t st);
int k_fill(double *p, long long n, double v, cudaStream_t st);
int k_patch_out(int prec, const LevelView &L, int p, int ncells, int cur, double *out, cudaStream_t st);
int k_cnn_features(int prec, const LevelView &L, int npatch, int maxcells, int cur, const int *scen_slot,
                   const uint8_t *raw, float *feat, double drytol, const CnnWindow &win, cudaStream_t st);
int k_cnn_union(uint8_t *raw, const uint8_t *cov, const float *logits, int nx, int ny, int np, const CnnWindow &win,
                cudaStream_t st);
// mass per scenario over level 1 in a fixed summation order; parts: k_mass_parts(npatch, maxcells) doubles
int k_mass_parts(int npatch, int maxcells);
int k_mass(int prec, const LevelView &L, int npatch, int maxcells, int cur, double *parts, double *mass, int nscen,
           cudaStream_t st);

}  // namespace tsu
