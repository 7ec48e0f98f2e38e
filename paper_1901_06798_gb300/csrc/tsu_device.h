// tsu_device.h -- structures shared by the library's host code and kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tsu {

// One patch of a level: interior box [i0, i0+nx) x [j0, j0+ny) in global
// level indices, stored with 2 ghost cells per side.  The patch's block in the
// arena holds 7 fields of fs elements each: buffer 0 (q0, q1, q2), buffer 1
// (q0, q1, q2), B.  q0 is h (FP64 form) or eta' = h + B (FP32 perturbation
// form); q1 = hu, q2 = hv.  Element (i, j), -2 <= i < nx+2, at
// (j + 2) * pitch + (i + 2).
struct PatchDesc {
    long long off;      // element offset of the block in the arena
    long long fs;       // elements per field
    int i0, j0, nx, ny, pitch;
    int scen;
    int bcmask;         // 1 left, 2 right, 4 bottom, 8 top: ghost cells reach past that domain edge
    int nbr_off, nbr_cnt;      // same-level patches whose interior may feed this patch's ghosts
    int cmap_off, cmap_i0, cmap_j0, cmap_w, cmap_h;  // coarse-level patch index per coarse cell (levels >= 2)
    int ccand_off, ccand_cnt;  // coarse patches overlapping the coarse map's footprint (the map's painters)
    int old_off, old_cnt;      // old same-level patches overlapping (regrid initialisation)
    long long soff;            // FP32 split update: element offset of the patch's Q* (3 fields of fs) in the scratch
};

// One work item of the patch update: a strip of columns [x0, x0+w) and a row
// segment [y0, y0+h) of one patch (patch-local interior indices).
struct StepItem {
    int patch;
    int x0, y0, w, h;
};

struct StepArgs {
    const PatchDesc *descs;
    const StepItem *items;
    void *arena;
    int cur;                    // current buffer of this level (0 or 1)
    const double *dt1;          // level-1 time step per scenario
    unsigned long long *smax;   // per scenario: [2] max speed bits (x, y)
    double R;                   // refinement of this level relative to level 1
    double dx, dy, g, drytol;
    // FP32 copies for the perturbation-form kernel (no FP64 work per CTA)
    const float *dt1f;          // level-1 time step per scenario, FP32
    float rdx, rdy;             // 1 / (R dx), 1 / (R dy)
    float gf, drytolf, sqrtgf;
    int transverse;             // 1: unsplit update with transverse corrections
    double manning;             // n^2 g of the friction step (0: none)
    float manningf;
    float rR;                   // 1 / R (FP32 level time step = dt1f * rR)
    // latitude-longitude grids (capacity form): dx, dy above are the physical
    // sizes of an equatorial cell; capacity of global row J at kap[J + 2], relative
    // length of the latitude edge below row J at ced[J + 2]; null on Cartesian grids
    const double *kap, *ced;
    const float *kapf, *cedf;
    // FP32 split update (two kernels): the level's Q* scratch and the y kernel's
    // work items (strips of 64 columns x row segments); null scratch: fused kernel
    float *scratch;
    const StepItem *items_y;
    int n_items_y;
    // CFL retake of a level-1 step: when set, a work item of scenario s runs
    // only if gate[s] != 0 (null: every item runs)
    const int *gate;
    // device error flag (TSU_DEV_ERR_* bits; null: not reported); FP32 split
    // update: bulk row copies in the x-sweep kernel (0: per-thread cp.async) and
    // the polls it spends waiting for one before it gives up
    int *err;
    int bulk_rows;
    unsigned wait_polls;
};

// device error flag bits: 1, 2, 4 a ghost, coarse or parent cell without a
// covering patch (nesting); 8 a non-finite wave speed or depth; 16 a wait for a
// bulk copy ran out of polls; 32 patch storage not aligned for bulk copies
enum { TSU_DEV_ERR_NESTING = 7, TSU_DEV_ERR_NAN = 8, TSU_DEV_ERR_TIMEOUT = 16, TSU_DEV_ERR_LAYOUT = 32 };

// FP32 launch constants of a level
inline void set_f32_constants(StepArgs &a)
{
    a.rdx = (float)(1.0 / (a.R * a.dx));
    a.rdy = (float)(1.0 / (a.R * a.dy));
    a.gf = (float)a.g;
    a.drytolf = (float)a.drytol;
    a.sqrtgf = (float)__builtin_sqrt(a.g);
    a.manningf = (float)a.manning;
    a.rR = (float)(1.0 / a.R);
}

// Launch helpers implemented in the .cu files.
int launch_step_f64(const StepArgs &a, int n_items, int threads, cudaStream_t st);
int launch_step_f32p(const StepArgs &a, int n_items, int threads, cudaStream_t st);
int launch_unsplit_f64(const StepArgs &a, int n_items, int threads, cudaStream_t st);
int launch_unsplit_f32p(const StepArgs &a, int n_items, int threads, cudaStream_t st);
int step_threads_f64();
int step_threads_f32p();
// columns one work item of the patch update covers, for a launch of `threads`
// per CTA (the unsplit kernels take one column per thread in both precisions)
int step_strip_width_f64(int threads, int transverse);
int step_strip_width_f32p(int threads, int transverse);

}  // namespace tsu
