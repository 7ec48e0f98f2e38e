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

#define OIDX(p, i, j) ((size_t)((i) + 2) + (size_t)((j) + 2) * (size_t)(p)->pitch)

/* one dimensionally split step (x sweep then y sweep) of one patch whose
 * ghost cells are already filled; returns the max wave speeds seen on the
 * edges that update interior cells. */
void ora_step_patch(OPatch *p, double g, double drytol, double dt, double dx, double dy,
                    double *sx, double *sy);

/* Manning friction of the interior cells after a step (Sec. 2.1 drag D) */
void ora_friction_patch(OPatch *p, double g, double drytol, double n, double dt);

/* one unsplit step with transverse corrections (the original GeoClaw scheme) */
void ora_step_patch_unsplit(OPatch *p, double g, double drytol, double dt, double dx, double dy,
                            double *sx, double *sy);

#endif
