/* Private declarations of the FP64 CPU oracle (test infrastructure only). */
#ifndef ORA_INTERNAL_H
#define ORA_INTERNAL_H
#include "oracle.h"

typedef struct OPatch {
    int level, scen;            /* level is 0-based here */
    int i0, j0, nx, ny;         /* interior box in global level indices */
    int pitch;                  /* nx + 4 */
    double *h, *hu, *hv, *B;    /* (nx+4)*(ny+4) with 2 ghost cells each side */
    double *h0, *hu0, *hv0;     /* state at the start of the patch's last step */
} OPatch;

/* running count of depths that came out of a sweep negative and were clipped
 * to zero (the post-processing after each sweep); the driver reads differences */
extern long ora_neg_clips;

#define OIDX(p, i, j) ((size_t)((i) + 2) + (size_t)((j) + 2) * (size_t)(p)->pitch)

/* one dimensionally split step (x sweep then y sweep) of one patch whose
 * ghost cells are already filled; returns the max wave speeds seen on the
 * edges that update interior cells. */
void ora_step_patch(OPatch *p, double g, double drytol, double dt, double dx, double dy,
                    double *sx, double *sy);

/* the same step, also returning the edge mass fluxes of the interior rows (xf:
 * ny (nx + 1) x-edges) and columns (yf: nx (ny + 1) y-edges), two per edge: as
 * the lower/left cell's update uses it, and as the upper/right cell's does */
void ora_step_patch_flux(OPatch *p, double g, double drytol, double dt, double dx, double dy,
                         double *sx, double *sy, double *xf, double *yf);

/* split step on a latitude-longitude grid in capacity form: kap[j + 2] is the
 * capacity of patch row j (-2 <= j < ny + 2), ced[j + 2] the relative length of
 * the latitude edge below row j (-2 <= j <= ny + 2); dxp, dyp are the physical
 * cell sizes at the equator.  sx, sy: largest speeds scaled to those sizes. */
void ora_step_patch_geo(OPatch *p, double g, double drytol, double dt, double dxp, double dyp, const double *kap,
                        const double *ced, double *sx, double *sy);

/* Manning friction of the interior cells after a step (Sec. 2.1 drag D) */
void ora_friction_patch(OPatch *p, double g, double drytol, double n, double dt);

/* one unsplit step with transverse corrections (the original GeoClaw scheme) */
void ora_step_patch_unsplit(OPatch *p, double g, double drytol, double dt, double dx, double dy,
                            double *sx, double *sy);

#endif
