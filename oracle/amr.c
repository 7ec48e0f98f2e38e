/*
 * amr.c -- FP64 CPU oracle: block-structured AMR around the patch update.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Plain loops and linear searches;
 * nothing is precomputed, blocked or fused.
 *
 *   Sec. 3      patch hierarchy, dx^{l+1} = dx^l / r^l, dt^{l+1} = dt^l / r^l
 *   Sec. 3.1    recursive time integration: (1) advance level l, (2) fill the
 *               level-l+1 ghost cells by copy or by space-time interpolation
 *               from level l at t_n and t_n + dt^l, (3) advance level l+1 r
 *               times, (4) average level l+1 onto level l; (5) refluxing is
 *               dropped as in the paper's GPU code.
 *   Sec. 3.2    regridding every b steps, flag buffer of b cells, clustering
 *               (Berger & Rigoutsos), new cells copied from old same-level
 *               patches or interpolated from level l; surface-elevation
 *               interpolation and averaging that keep the ocean at rest.
 *   Sec. 5.1.2  zeta output field (Eq. zeta) and gauges.
 *
 * Readings where the paper is silent:
 *   - interpolation: linear in time of (h, hu, hv) as q0 + a (q1 - q0), then
 *     minmod-limited linear in space of (eta, hu, hv) using wet neighbours
 *     only; fine h = max(0, eta - B_f); momenta zeroed below drytol.  A dry
 *     coarse centre takes the lowest surface of the wet cells in its 3x3
 *     coarse neighbourhood (zero slope, zero momenta), or stays dry if there
 *     is none, so fine cells below the sea surface next to the shore are
 *     filled to it and the ocean at rest stays exactly at rest.
 *   - averaging: eta averaged over wet fine cells, momenta over all fine
 *     cells; h_c = max(0, eta - B_c).
 *   - dt: dt^1 = min(dt_max, nu_d / max_l(rate_l / R_l)) from the largest
 *     max(s_x/dx, s_y/dy) seen on each level during the previous coarse step
 *     (cell speeds |u| + sqrt(gh) at start-up and for new patches); a step
 *     with nu > cfl_max is counted as a CFL violation (not retaken).
 *   - flags: wet and |eta| > tol, or -B < depth_below, or inside a forcing
 *     region; Chebyshev dilation by b; region caps; proper nesting (every
 *     level-l cell within 2 of a flagged cell is covered by level l or lies
 *     outside the domain).
 *   - clustering: see ora_cluster below.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include "ora_internal.h"

typedef struct TopoGrid {
    int nx, ny;
    double x0, y0, dx, dy;
    double *v;
} TopoGrid;

typedef struct Level {
    OPatch **p;
    int n, cap;
} Level;

typedef struct Scen {
    Level lev[ORA_MAX_LEVELS];
    TopoGrid *up;               /* uplift layers (additive) */
    int nup;
    TopoGrid eta0;
    int has_eta0;
    TopoGrid u0, v0;            /* initial velocities (node grids) */
    int has_uv0;
    double t, dt1;
    double rate[ORA_MAX_LEVELS];
    long nsteps[ORA_MAX_LEVELS];
    int substep[ORA_MAX_LEVELS];
    long cfl_viol;
    long cfl_retakes;           /* level-1 steps discarded and taken again (CFL) */
    long neg_clips;             /* depths clipped to zero after a sweep */
    double cell_updates;
    /* refluxing registers of level l as the coarse level of l+1, over its whole
     * index space, 4 faces (W, E, S, N) per cell: dt times the mass flux the
     * cell's own update used (cflux), the time- and length-weighted sum of the
     * fine fluxes through that face (fflux), and which faces are coarse-fine
     * interfaces this step (fset) */
    double *cflux[ORA_MAX_LEVELS], *fflux[ORA_MAX_LEVELS];
    unsigned char *fset[ORA_MAX_LEVELS];
} Scen;

typedef struct Ora {
    ora_config c;
    TopoGrid *topo;
    int ntopo;
    Scen *sc;
    int R[ORA_MAX_LEVELS];      /* cumulative refinement of each level vs level 1 */
    int nxl[ORA_MAX_LEVELS], nyl[ORA_MAX_LEVELS];
    double dxl[ORA_MAX_LEVELS], dyl[ORA_MAX_LEVELS];
    int initialized;
    double *gxy;
    int ngauge;
    double *gt, *geta;
    int nsamp, capsamp;
} Ora;

/* ------------------------------------------------------------------ */
/* topography                                                          */

static int grid_contains(const TopoGrid *g, double x, double y)
{
    return x >= g->x0 && x <= g->x0 + (double)(g->nx - 1) * g->dx &&
           y >= g->y0 && y <= g->y0 + (double)(g->ny - 1) * g->dy;
}

static double grid_bilinear(const TopoGrid *g, double x, double y)
{
    double fx = (x - g->x0) / g->dx, fy = (y - g->y0) / g->dy;
    int i = (int)floor(fx), j = (int)floor(fy);
    if (i < 0) i = 0;
    if (i > g->nx - 2) i = g->nx - 2;
    if (j < 0) j = 0;
    if (j > g->ny - 2) j = g->ny - 2;
    double tx = fx - (double)i, ty = fy - (double)j;
    if (tx < 0.0) tx = 0.0;
    if (tx > 1.0) tx = 1.0;
    if (ty < 0.0) ty = 0.0;
    if (ty > 1.0) ty = 1.0;
    const double *v = g->v;
    double v00 = v[(size_t)j * g->nx + i], v10 = v[(size_t)j * g->nx + i + 1];
    double v01 = v[(size_t)(j + 1) * g->nx + i], v11 = v[(size_t)(j + 1) * g->nx + i + 1];
    double a = v00 + tx * (v10 - v00);
    double b = v01 + tx * (v11 - v01);
    return a + ty * (b - a);
}

/* base topography: the finest grid containing the point (later grids win ties) */
static double base_topo(const Ora *o, double x, double y)
{
    int best = -1;
    double barea = 0.0;
    for (int k = 0; k < o->ntopo; k++) {
        if (!grid_contains(&o->topo[k], x, y)) continue;
        double area = o->topo[k].dx * o->topo[k].dy;
        if (best < 0 || area <= barea) { best = k; barea = area; }
    }
    if (best < 0) best = 0;
    return grid_bilinear(&o->topo[best], x, y);
}

static double uplift_sum(const Scen *S, double B, double x, double y)
{
    for (int k = 0; k < S->nup; k++)
        if (grid_contains(&S->up[k], x, y)) B = B + grid_bilinear(&S->up[k], x, y);
    return B;
}

static double xc(const Ora *o, int l, int I) { return o->c.x0 + ((double)I + 0.5) * o->dxl[l]; }
static double yc(const Ora *o, int l, int J) { return o->c.y0 + ((double)J + 0.5) * o->dyl[l]; }

/* ------------------------------------------------------------------ */
/* patches                                                             */

static OPatch *patch_new(int level, int scen, int i0, int j0, int nx, int ny)
{
    OPatch *p = (OPatch *)calloc(1, sizeof *p);
    p->level = level; p->scen = scen; p->i0 = i0; p->j0 = j0; p->nx = nx; p->ny = ny;
    p->pitch = nx + 4;
    size_t n = (size_t)(nx + 4) * (size_t)(ny + 4);
    p->h = calloc(n, sizeof(double)); p->hu = calloc(n, sizeof(double)); p->hv = calloc(n, sizeof(double));
    p->B = calloc(n, sizeof(double));
    p->h0 = calloc(n, sizeof(double)); p->hu0 = calloc(n, sizeof(double)); p->hv0 = calloc(n, sizeof(double));
    return p;
}

static void patch_free(OPatch *p)
{
    if (!p) return;
    free(p->h); free(p->hu); free(p->hv); free(p->B); free(p->h0); free(p->hu0); free(p->hv0);
    free(p);
}

static void level_push(Level *L, OPatch *p)
{
    if (L->n == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 16;
        L->p = (OPatch **)realloc(L->p, (size_t)L->cap * sizeof *L->p);
    }
    L->p[L->n++] = p;
}

static void save_old(OPatch *p)
{
    size_t n = (size_t)(p->nx + 4) * (size_t)(p->ny + 4);
    memcpy(p->h0, p->h, n * sizeof(double));
    memcpy(p->hu0, p->hu, n * sizeof(double));
    memcpy(p->hv0, p->hv, n * sizeof(double));
}

static int inside_domain(const Ora *o, int l, int I, int J)
{
    return I >= 0 && I < o->nxl[l] && J >= 0 && J < o->nyl[l];
}

static OPatch *find_patch(const Ora *o, int s, int l, int I, int J, const OPatch *skip)
{
    const Level *L = &o->sc[s].lev[l];
    for (int k = 0; k < L->n; k++) {
        OPatch *q = L->p[k];
        if (q == skip) continue;
        if (I >= q->i0 && I < q->i0 + q->nx && J >= q->j0 && J < q->j0 + q->ny) return q;
    }
    return NULL;
}

/* Physical boundary conditions on the ghost cells outside the domain, in
 * global indices: a ghost cell beyond the left edge at I < 0 takes cell -1-I
 * (wall: mirror, normal momentum negated) or cell 0 (extrapolation); beyond
 * the right edge at I >= nx_l it takes 2 nx_l - 1 - I or nx_l - 1; the same in
 * y.  The source lies in the patch's own storage (interior or a ghost cell
 * already filled by copy or interpolation), also when a thin neighbour patch
 * sits between this patch and the boundary.  Left/right ghost columns on
 * every row first, then bottom/top ghost rows on every column, so corners end
 * up defined by the y rule.  normal_x/normal_y: negate under a wall (never
 * for B). */
static void apply_bc_field(const Ora *o, OPatch *p, double *f, int normal_x, int normal_y)
{
    int l = p->level, nx = p->nx, ny = p->ny, nxl = o->nxl[l], nyl = o->nyl[l];
    for (int j = -2; j < ny + 2; j++)
        for (int i = -2; i < nx + 2; i++) {
            int I = p->i0 + i, src, neg = 0;
            if (I < 0) {
                if (o->c.bc[0] == ORA_BC_WALL) { src = -1 - I; neg = normal_x; } else src = 0;
            } else if (I >= nxl) {
                if (o->c.bc[1] == ORA_BC_WALL) { src = 2 * nxl - 1 - I; neg = normal_x; } else src = nxl - 1;
            } else continue;
            double v = f[OIDX(p, src - p->i0, j)];
            f[OIDX(p, i, j)] = neg ? -v : v;
        }
    for (int i = -2; i < nx + 2; i++)
        for (int j = -2; j < ny + 2; j++) {
            int J = p->j0 + j, src, neg = 0;
            if (J < 0) {
                if (o->c.bc[2] == ORA_BC_WALL) { src = -1 - J; neg = normal_y; } else src = 0;
            } else if (J >= nyl) {
                if (o->c.bc[3] == ORA_BC_WALL) { src = 2 * nyl - 1 - J; neg = normal_y; } else src = nyl - 1;
            } else continue;
            double v = f[OIDX(p, i, src - p->j0)];
            f[OIDX(p, i, j)] = neg ? -v : v;
        }
}

/* The x rule must run on all three fields before the y rule, field order
 * does not matter because each field is handled independently. */
static void apply_bc_state(const Ora *o, OPatch *p)
{
    apply_bc_field(o, p, p->h, 0, 0);
    apply_bc_field(o, p, p->hu, 1, 0);
    apply_bc_field(o, p, p->hv, 0, 1);
}

/* B at every cell of a new patch: sampled topography (base + the scenario's
 * uplift layers) inside the domain, boundary rule outside. */
static void patch_set_B(const Ora *o, OPatch *p)
{
    const Scen *S = &o->sc[p->scen];
    for (int j = -2; j < p->ny + 2; j++)
        for (int i = -2; i < p->nx + 2; i++) {
            int I = p->i0 + i, J = p->j0 + j;
            if (!inside_domain(o, p->level, I, J)) continue;
            double x = xc(o, p->level, I), y = yc(o, p->level, J);
            p->B[OIDX(p, i, j)] = uplift_sum(S, base_topo(o, x, y), x, y);
        }
    apply_bc_field(o, p, p->B, 0, 0);
}

/* ------------------------------------------------------------------ */
/* coarse -> fine interpolation (Sec. 3.1 step 2, Sec. 3.2)            */

typedef struct CVal {
    int found, wet;
    double q[3];   /* eta, hu, hv */
} CVal;

static CVal coarse_value(const Ora *o, int s, int lc, int I, int J, double alpha)
{
    CVal v;
    memset(&v, 0, sizeof v);
    if (!inside_domain(o, lc, I, J)) return v;
    OPatch *c = find_patch(o, s, lc, I, J, NULL);
    if (!c) return v;
    size_t k = OIDX(c, I - c->i0, J - c->j0);
    double h, hu, hv;
    if (alpha == 1.0) { h = c->h[k]; hu = c->hu[k]; hv = c->hv[k]; }
    else {
        h = c->h0[k] + alpha * (c->h[k] - c->h0[k]);
        hu = c->hu0[k] + alpha * (c->hu[k] - c->hu0[k]);
        hv = c->hv0[k] + alpha * (c->hv[k] - c->hv0[k]);
    }
    v.found = 1;
    v.wet = h >= o->c.drytol;
    v.q[0] = h + c->B[k];
    v.q[1] = hu;
    v.q[2] = hv;
    return v;
}

static double minmod(double a, double b)
{
    if (a > 0.0 && b > 0.0) return fmin(a, b);
    if (a < 0.0 && b < 0.0) return fmax(a, b);
    return 0.0;
}

/* fine cell (I, J) on level lf > 0 with bed Bf, from level lf-1 at time
 * fraction alpha of the coarse step; returns 0 if the coarse centre is not
 * covered (a nesting error). */
static int interp_fine(const Ora *o, int s, int lf, int I, int J, double Bf, double alpha,
                       double *h, double *hu, double *hv)
{
    int lc = lf - 1, r = o->c.ratios[lc];
    int Ic = I / r, Jc = J / r;
    CVal c = coarse_value(o, s, lc, Ic, Jc, alpha);
    if (!c.found) return 0;
    if (!c.wet) {
        /* dry coarse centre: take the lowest surface among the wet cells of
         * the 3x3 coarse neighbourhood (zero slope, no momentum); dry if none */
        double eref = 0.0;
        int any = 0;
        for (int dj = -1; dj <= 1; dj++)
            for (int di = -1; di <= 1; di++) {
                if (di == 0 && dj == 0) continue;
                CVal nb = coarse_value(o, s, lc, Ic + di, Jc + dj, alpha);
                if (nb.found && nb.wet && (!any || nb.q[0] < eref)) { eref = nb.q[0]; any = 1; }
            }
        double hf = any ? eref - Bf : 0.0;
        if (hf < 0.0) hf = 0.0;
        *h = hf; *hu = 0.0; *hv = 0.0;
        return 1;
    }
    CVal xm = coarse_value(o, s, lc, Ic - 1, Jc, alpha), xp = coarse_value(o, s, lc, Ic + 1, Jc, alpha);
    CVal ym = coarse_value(o, s, lc, Ic, Jc - 1, alpha), yp = coarse_value(o, s, lc, Ic, Jc + 1, alpha);
    double xi = ((double)(I - Ic * r) + 0.5) / (double)r - 0.5;
    double et = ((double)(J - Jc * r) + 0.5) / (double)r - 0.5;
    double qf[3];
    for (int m = 0; m < 3; m++) {
        double dxp = (xp.found && xp.wet) ? xp.q[m] - c.q[m] : 0.0;
        double dxm = (xm.found && xm.wet) ? c.q[m] - xm.q[m] : 0.0;
        double dyp = (yp.found && yp.wet) ? yp.q[m] - c.q[m] : 0.0;
        double dym = (ym.found && ym.wet) ? c.q[m] - ym.q[m] : 0.0;
        double sx = minmod(dxp, dxm), sy = minmod(dyp, dym);
        qf[m] = (c.q[m] + xi * sx) + et * sy;
    }
    double hf = qf[0] - Bf;
    if (hf < 0.0) hf = 0.0;
    *h = hf;
    if (hf < o->c.drytol) { *hu = 0.0; *hv = 0.0; }
    else { *hu = qf[1]; *hv = qf[2]; }
    return 1;
}

/* ------------------------------------------------------------------ */
/* ghost fill (Sec. 3.1 step 2)                                        */

static int fill_ghosts(Ora *o, int s, int l, double alpha)
{
    Level *L = &o->sc[s].lev[l];
    for (int k = 0; k < L->n; k++) {
        OPatch *p = L->p[k];
        for (int j = -2; j < p->ny + 2; j++)
            for (int i = -2; i < p->nx + 2; i++) {
                if (i >= 0 && i < p->nx && j >= 0 && j < p->ny) continue;
                int I = p->i0 + i, J = p->j0 + j;
                if (!inside_domain(o, l, I, J)) continue;
                size_t kk = OIDX(p, i, j);
                OPatch *q = find_patch(o, s, l, I, J, p);
                if (q) {
                    size_t kq = OIDX(q, I - q->i0, J - q->j0);
                    p->h[kk] = q->h[kq]; p->hu[kk] = q->hu[kq]; p->hv[kk] = q->hv[kq];
                } else if (l > 0) {
                    if (!interp_fine(o, s, l, I, J, p->B[kk], alpha, &p->h[kk], &p->hu[kk], &p->hv[kk]))
                        return -1;
                } else {
                    return -1;
                }
            }
        apply_bc_state(o, p);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* updating: fine -> coarse averaging (Sec. 3.1 step 4)                */

/* ------------------------------------------------------------------ */
/* latitude-longitude geometry (spherical coordinates)                  */
/*   row J of level l spans latitudes y0 + J dy .. y0 + (J + 1) dy (deg); */
/*   its capacity is the zone area over the area of an equatorial cell,   */
/*   (sin phi_top - sin phi_bottom) / dphi; the latitude edge below row J  */
/*   has relative length cos(y0 + J dy).                                  */

#define ORA_D2R (3.14159265358979323846 / 180.0)

static double geo_kap(const Ora *o, int l, int J)
{
    const double a = (o->c.y0 + (double)J * o->dyl[l]) * ORA_D2R;
    const double b = (o->c.y0 + (double)(J + 1) * o->dyl[l]) * ORA_D2R;
    return (sin(b) - sin(a)) / (o->dyl[l] * ORA_D2R);
}

static double geo_ced(const Ora *o, int l, int J) { return cos((o->c.y0 + (double)J * o->dyl[l]) * ORA_D2R); }

static double earth_r(const Ora *o) { return o->c.earth_radius > 0.0 ? o->c.earth_radius : 6371.0e3; }

/* physical cell sizes (at the equator on the sphere) */
static double phys_dx(const Ora *o, int l) { return o->c.spherical ? earth_r(o) * (o->dxl[l] * ORA_D2R) : o->dxl[l]; }
static double phys_dy(const Ora *o, int l) { return o->c.spherical ? earth_r(o) * (o->dyl[l] * ORA_D2R) : o->dyl[l]; }

static void average_down(Ora *o, int s, int lf)
{
    int lc = lf - 1, r = o->c.ratios[lc];
    Level *L = &o->sc[s].lev[lf];
    double drytol = o->c.drytol;
    for (int k = 0; k < L->n; k++) {
        OPatch *f = L->p[k];
        for (int Jc = f->j0 / r; Jc < (f->j0 + f->ny) / r; Jc++)
            for (int Ic = f->i0 / r; Ic < (f->i0 + f->nx) / r; Ic++) {
                OPatch *c = find_patch(o, s, lc, Ic, Jc, NULL);
                if (!c) continue;
                double se = 0.0, su = 0.0, sv = 0.0;
                int nwet = 0;
                double kw = 0.0, ka = 0.0;   /* spherical: capacity of the wet fine cells and of all */
                for (int jj = 0; jj < r; jj++) {
                    const double kf_ = o->c.spherical ? geo_kap(o, lf, Jc * r + jj) : 1.0;
                    for (int ii = 0; ii < r; ii++) {
                        size_t kf = OIDX(f, Ic * r + ii - f->i0, Jc * r + jj - f->j0);
                        if (o->c.spherical) {
                            if (f->h[kf] >= drytol) { se = se + kf_ * (f->h[kf] + f->B[kf]); kw = kw + kf_; nwet++; }
                            su = su + kf_ * f->hu[kf];
                            sv = sv + kf_ * f->hv[kf];
                            ka = ka + kf_;
                        } else {
                            if (f->h[kf] >= drytol) { se = se + (f->h[kf] + f->B[kf]); nwet++; }
                            su = su + f->hu[kf];
                            sv = sv + f->hv[kf];
                        }
                    }
                }
                size_t kc = OIDX(c, Ic - c->i0, Jc - c->j0);
                double hc = 0.0;
                if (nwet > 0) {
                    hc = (o->c.spherical ? se / kw : se / (double)nwet) - c->B[kc];
                    if (hc < 0.0) hc = 0.0;
                }
                double rr = o->c.spherical ? ka : (double)(r * r);
                c->h[kc] = hc;
                if (hc < drytol) { c->hu[kc] = 0.0; c->hv[kc] = 0.0; }
                else { c->hu[kc] = su / rr; c->hv[kc] = sv / rr; }
            }
    }
}

/* ------------------------------------------------------------------ */
/* clustering (Sec. 3.2, Berger & Rigoutsos 1991)                      */
/*
 * Reading used here (deterministic, written out so that two independent
 * implementations agree box for box):
 *   - box = tight bounding box of the flags inside the search region;
 *     accept it if flags >= eff * area and every cell is nestable;
 *   - otherwise cut: (1) at an empty column/row (signature hole) closest to
 *     the box centre, in the longer dimension when both exist (x on ties);
 *     (2) else at the strongest sign change of the signature Laplacian
 *     sig[i-1] - 2 sig[i] + sig[i+1] (strength |lap[i+1] - lap[i]|; ties:
 *     closer to the centre, then the smaller index; x vs y: stronger, then
 *     longer, then x); (3) else bisect the longer side (x on ties);
 *   - recurse on the lower/left part first;
 *   - finally split every box into near-equal pieces whose fine size is at
 *     most patch_max (pieces ordered row by row).
 */

typedef struct BoxList {
    int *b;
    int n, cap, overflow;
} BoxList;

static void box_push(BoxList *L, int i0, int j0, int w, int h)
{
    if (L->n >= L->cap) { L->overflow = 1; return; }
    L->b[4 * L->n + 0] = i0; L->b[4 * L->n + 1] = j0; L->b[4 * L->n + 2] = w; L->b[4 * L->n + 3] = h;
    L->n++;
}

static void cluster_rec(const unsigned char *F, const unsigned char *N, int nx,
                        int ri0, int rj0, int ri1, int rj1, double eff, BoxList *out)
{
    /* tight bounding box in [ri0, ri1] x [rj0, rj1] (inclusive) */
    int i0 = ri1 + 1, i1 = ri0 - 1, j0 = rj1 + 1, j1 = rj0 - 1;
    long nf = 0;
    for (int j = rj0; j <= rj1; j++)
        for (int i = ri0; i <= ri1; i++)
            if (F[(size_t)j * nx + i]) {
                nf++;
                if (i < i0) i0 = i;
                if (i > i1) i1 = i;
                if (j < j0) j0 = j;
                if (j > j1) j1 = j;
            }
    if (nf == 0) return;
    int w = i1 - i0 + 1, h = j1 - j0 + 1;
    long area = (long)w * (long)h;
    int nested = 1;
    for (int j = j0; j <= j1 && nested; j++)
        for (int i = i0; i <= i1; i++)
            if (!N[(size_t)j * nx + i]) { nested = 0; break; }
    if ((double)nf >= eff * (double)area && nested) {
        box_push(out, i0, j0, w, h);
        return;
    }

    long *sx = (long *)calloc((size_t)w, sizeof(long));
    long *sy = (long *)calloc((size_t)h, sizeof(long));
    for (int j = j0; j <= j1; j++)
        for (int i = i0; i <= i1; i++)
            if (F[(size_t)j * nx + i]) { sx[i - i0]++; sy[j - j0]++; }

    int cut_dim = -1, cut_at = 0;   /* cut between cut_at and cut_at+1 (box-relative) */

    /* (1) holes */
    int hx = -1, hy = -1;
    long bdx = 0, bdy = 0;
    for (int i = 1; i < w - 1; i++)
        if (sx[i] == 0) {
            long d = labs(2L * i - (long)(w - 1));
            if (hx < 0 || d < bdx) { hx = i; bdx = d; }
        }
    for (int j = 1; j < h - 1; j++)
        if (sy[j] == 0) {
            long d = labs(2L * j - (long)(h - 1));
            if (hy < 0 || d < bdy) { hy = j; bdy = d; }
        }
    if (hx >= 0 && (hy < 0 || w >= h)) { cut_dim = 0; cut_at = hx; }
    else if (hy >= 0) { cut_dim = 1; cut_at = hy; }

    /* (2) inflection of the signature Laplacian */
    if (cut_dim < 0) {
        long bsx = -1, bsy = -1, cdx = 0, cdy = 0;
        int ix = -1, iy = -1;
        for (int i = 1; i + 2 <= w - 1; i++) {
            long la = sx[i - 1] - 2 * sx[i] + sx[i + 1];
            long lb = sx[i] - 2 * sx[i + 1] + sx[i + 2];
            if ((la < 0 && lb > 0) || (la > 0 && lb < 0)) {
                long st = labs(lb - la), d = labs(2L * i + 1 - (long)(w - 1));
                if (st > bsx || (st == bsx && d < cdx)) { bsx = st; cdx = d; ix = i; }
            }
        }
        for (int j = 1; j + 2 <= h - 1; j++) {
            long la = sy[j - 1] - 2 * sy[j] + sy[j + 1];
            long lb = sy[j] - 2 * sy[j + 1] + sy[j + 2];
            if ((la < 0 && lb > 0) || (la > 0 && lb < 0)) {
                long st = labs(lb - la), d = labs(2L * j + 1 - (long)(h - 1));
                if (st > bsy || (st == bsy && d < cdy)) { bsy = st; cdy = d; iy = j; }
            }
        }
        if (ix >= 0 && (iy < 0 || bsx > bsy || (bsx == bsy && w >= h))) { cut_dim = 0; cut_at = ix; }
        else if (iy >= 0) { cut_dim = 1; cut_at = iy; }
    }

    /* (3) bisection of the longer side */
    if (cut_dim < 0) {
        if (w >= h) { cut_dim = 0; cut_at = w / 2 - 1; }
        else { cut_dim = 1; cut_at = h / 2 - 1; }
    }
    free(sx);
    free(sy);

    if (cut_dim == 0) {
        cluster_rec(F, N, nx, i0, j0, i0 + cut_at, j1, eff, out);
        cluster_rec(F, N, nx, i0 + cut_at + 1, j0, i1, j1, eff, out);
    } else {
        cluster_rec(F, N, nx, i0, j0, i1, j0 + cut_at, eff, out);
        cluster_rec(F, N, nx, i0, j0 + cut_at + 1, i1, j1, eff, out);
    }
}

int ora_cluster(const unsigned char *flags, const unsigned char *nestable, int nx, int ny,
                double eff, int ratio, int patch_max, int *boxes, int max_boxes)
{
    BoxList raw;
    raw.cap = nx * ny + 1;
    raw.b = (int *)malloc((size_t)raw.cap * 4 * sizeof(int));
    raw.n = 0; raw.overflow = 0;
    cluster_rec(flags, nestable, nx, 0, 0, nx - 1, ny - 1, eff, &raw);
    int pm = patch_max / ratio;
    if (pm < 1) pm = 1;
    BoxList out;
    out.b = boxes; out.cap = max_boxes; out.n = 0; out.overflow = 0;
    for (int k = 0; k < raw.n; k++) {
        int i0 = raw.b[4 * k], j0 = raw.b[4 * k + 1], w = raw.b[4 * k + 2], h = raw.b[4 * k + 3];
        int npx = (w + pm - 1) / pm, npy = (h + pm - 1) / pm;
        for (int b = 0; b < npy; b++)
            for (int a = 0; a < npx; a++) {
                int xa = i0 + (int)((long)a * w / npx), xb = i0 + (int)((long)(a + 1) * w / npx);
                int ya = j0 + (int)((long)b * h / npy), yb = j0 + (int)((long)(b + 1) * h / npy);
                box_push(&out, xa, ya, xb - xa, yb - ya);
            }
    }
    free(raw.b);
    return out.overflow ? -1 : out.n;
}

/* ------------------------------------------------------------------ */
/* flagging and regridding (Sec. 3.2)                                  */

static double cell_rate(const Ora *o, const OPatch *p, double *sxo, double *syo)
{
    double g = o->c.g, sx = 0.0, sy = 0.0;
    for (int j = 0; j < p->ny; j++) {
        /* on the sphere a row's x speeds count relative to its capacity, its y
         * speeds like those of its y-edges: times ced_e / kap, the larger of
         * its two edges (the Courant numbers of the capacity-form sweeps) */
        const double kj = o->c.spherical ? geo_kap(o, p->level, p->j0 + j) : 1.0;
        const double cj = o->c.spherical ? fmax(geo_ced(o, p->level, p->j0 + j), geo_ced(o, p->level, p->j0 + j + 1)) / kj
                                         : 1.0;
        for (int i = 0; i < p->nx; i++) {
            size_t k = OIDX(p, i, j);
            double h = p->h[k];
            if (h < o->c.drytol) continue;
            double c = sqrt(g * h);
            double ax = fabs(p->hu[k] / h) + c, ay = fabs(p->hv[k] / h) + c;
            if (o->c.spherical) { ax = ax / kj; ay = ay * cj; }
            sx = fmax(sx, ax);
            sy = fmax(sy, ay);
        }
    }
    *sxo = sx; *syo = sy;
    return 0.0;
}

static void level_cell_rate(Ora *o, int s, int l)
{
    Level *L = &o->sc[s].lev[l];
    double sx = 0.0, sy = 0.0;
    for (int k = 0; k < L->n; k++) {
        double a, b;
        cell_rate(o, L->p[k], &a, &b);
        sx = fmax(sx, a);
        sy = fmax(sy, b);
    }
    double r = fmax(sx / phys_dx(o, l), sy / phys_dy(o, l));
    o->sc[s].rate[l] = fmax(o->sc[s].rate[l], r);
}

/* flags on level l (0-based) for building level l+1; returns a mask over the
 * whole level-l index space and the nestable mask. */
static void make_flags(const Ora *o, int s, int l, unsigned char *F, unsigned char *N)
{
    int nx = o->nxl[l], ny = o->nyl[l];
    size_t n = (size_t)nx * ny;
    const ora_config *c = &o->c;
    const Level *L = &o->sc[s].lev[l];
    int newlev = l + 2;  /* 1-based level being created */
    unsigned char *raw = (unsigned char *)calloc(n, 1);
    unsigned char *cov = (unsigned char *)calloc(n, 1);
    for (int k = 0; k < L->n; k++) {
        const OPatch *p = L->p[k];
        for (int j = 0; j < p->ny; j++)
            for (int i = 0; i < p->nx; i++) {
                size_t kk = OIDX(p, i, j);
                int I = p->i0 + i, J = p->j0 + j;
                cov[(size_t)J * nx + I] = 1;
                double h = p->h[kk], B = p->B[kk];
                int f = 0;
                if (c->flag_eta_tol > 0.0 && h >= c->drytol && fabs(h + B) > c->flag_eta_tol) f = 1;
                if (c->flag_depth_below > 0.0 && -B < c->flag_depth_below) f = 1;
                double x = xc(o, l, I), y = yc(o, l, J);
                for (int rg = 0; rg < c->n_regions; rg++) {
                    const double *R = c->regions[rg];
                    if (x >= R[0] && x <= R[2] && y >= R[1] && y <= R[3] && (double)newlev <= R[4]) f = 1;
                }
                raw[(size_t)J * nx + I] = (unsigned char)f;
            }
    }
    /* Chebyshev dilation by b */
    int b = c->regrid_interval > 0 ? c->regrid_interval : 0;
    memset(F, 0, n);
    for (int J = 0; J < ny; J++)
        for (int I = 0; I < nx; I++) {
            if (!raw[(size_t)J * nx + I]) continue;
            for (int dj = -b; dj <= b; dj++)
                for (int di = -b; di <= b; di++) {
                    int a = I + di, bb = J + dj;
                    if (a >= 0 && a < nx && bb >= 0 && bb < ny) F[(size_t)bb * nx + a] = 1;
                }
        }
    /* region caps, then proper nesting */
    for (int J = 0; J < ny; J++)
        for (int I = 0; I < nx; I++) {
            size_t kk = (size_t)J * nx + I;
            double x = xc(o, l, I), y = yc(o, l, J);
            for (int rg = 0; rg < c->n_regions; rg++) {
                const double *R = c->regions[rg];
                if (x >= R[0] && x <= R[2] && y >= R[1] && y <= R[3] && (double)newlev > R[5]) F[kk] = 0;
            }
            int ok = 1;
            for (int dj = -2; dj <= 2 && ok; dj++)
                for (int di = -2; di <= 2; di++) {
                    int a = I + di, bb = J + dj;
                    if (a < 0 || a >= nx || bb < 0 || bb >= ny) continue;
                    if (!cov[(size_t)bb * nx + a]) { ok = 0; break; }
                }
            N[kk] = (unsigned char)ok;
            if (!ok) F[kk] = 0;
        }
    free(raw);
    free(cov);
}

/* build level l+1 of scenario s from flags on level l: new cells copy the
 * old level-l+1 patches where they overlap, else interpolate from level l. */
static int regrid_one(Ora *o, int s, int l)
{
    int lf = l + 1, r = o->c.ratios[l];
    int nx = o->nxl[l], ny = o->nyl[l];
    unsigned char *F = (unsigned char *)malloc((size_t)nx * ny);
    unsigned char *N = (unsigned char *)malloc((size_t)nx * ny);
    make_flags(o, s, l, F, N);
    int maxb = nx * ny + 1;
    int *boxes = (int *)malloc((size_t)maxb * 4 * sizeof(int));
    int nb = ora_cluster(F, N, nx, ny, o->c.cluster_eff, r, o->c.patch_max, boxes, maxb);
    free(F);
    free(N);
    if (nb < 0) { free(boxes); return -1; }

    Scen *S = &o->sc[s];
    Level old = S->lev[lf];
    Level nw;
    memset(&nw, 0, sizeof nw);
    int rc = 0;
    for (int k = 0; k < nb; k++) {
        OPatch *p = patch_new(lf, s, boxes[4 * k] * r, boxes[4 * k + 1] * r, boxes[4 * k + 2] * r, boxes[4 * k + 3] * r);
        patch_set_B(o, p);
        for (int j = 0; j < p->ny; j++)
            for (int i = 0; i < p->nx; i++) {
                int I = p->i0 + i, J = p->j0 + j;
                size_t kk = OIDX(p, i, j);
                OPatch *q = NULL;
                for (int m = 0; m < old.n; m++) {
                    OPatch *c = old.p[m];
                    if (I >= c->i0 && I < c->i0 + c->nx && J >= c->j0 && J < c->j0 + c->ny) { q = c; break; }
                }
                if (q) {
                    size_t kq = OIDX(q, I - q->i0, J - q->j0);
                    p->h[kk] = q->h[kq]; p->hu[kk] = q->hu[kq]; p->hv[kk] = q->hv[kq];
                } else if (!interp_fine(o, s, lf, I, J, p->B[kk], 1.0, &p->h[kk], &p->hu[kk], &p->hv[kk])) {
                    rc = -1;
                }
            }
        save_old(p);
        level_push(&nw, p);
    }
    free(boxes);
    for (int m = 0; m < old.n; m++) patch_free(old.p[m]);
    free(old.p);
    S->lev[lf] = nw;
    level_cell_rate(o, s, lf);
    return rc;
}

/* regrid based on level l: rebuild levels l+1 .. L-1 in turn */
static int regrid_from(Ora *o, int s, int l)
{
    for (int k = l; k + 1 < o->c.num_levels; k++)
        if (regrid_one(o, s, k)) return -1;
    return 0;
}

/* ------------------------------------------------------------------ */
/* refluxing (Sec. 3.1 step 5), optional: the mass only                */
/*                                                                     */
/* Reading: the paper describes step 5 (replace a coarse cell's flux   */
/* through a face it shares with finer cells by the finer fluxes) and  */
/* drops it on the GPU.  In the wave-propagation form a cell's update  */
/* is a difference of edge "fluxes" seen from that cell (sweep_1d_flux:*/
/* G- for the left/lower cell, G+ for the right/upper one).  For the   */
/* mass they are the same flux up to rounding (the f-waves of the mass */
/* sum to the jump of hu: the bed source enters the momentum only).    */
/* Momentum is not refluxed: with the bed source its edge fluxes are   */
/* not one flux, and the coarse and fine flux of a lake at rest differ */
/* by the hydrostatic term of the two beds, which refluxing would turn */
/* into motion.  Per coarse step of level l: the flux each level-l     */
/* cell used through each face (dt_l G), the sum over the fine steps   */
/* and the r fine edges of a face of dt_{l+1} G / r, taken as the fine */
/* cells used it, then after averaging every uncovered level-l cell    */
/* next to a fine patch gets h += (used - fine) / dx (signs by face);  */
/* a depth driven below zero is clamped, as after a sweep.             */

static void reflux_clear(Ora *o, int s, int l)
{
    Scen *S = &o->sc[s];
    const size_t n = (size_t)o->nxl[l] * o->nyl[l] * 4;
    if (!S->cflux[l]) {
        S->cflux[l] = calloc(n, sizeof(double));
        S->fflux[l] = calloc(n, sizeof(double));
        S->fset[l] = calloc(n, 1);
    } else {
        memset(S->cflux[l], 0, n * sizeof(double));
        memset(S->fflux[l], 0, n * sizeof(double));
        memset(S->fset[l], 0, n);
    }
}

enum { FACE_W = 0, FACE_E = 1, FACE_S = 2, FACE_N = 3 };

static size_t reg_index(const Ora *o, int l, int I, int J, int face)
{
    return ((size_t)J * o->nxl[l] + I) * 4 + face;
}

/* level l as the coarse level: the flux each interior cell's update used through each face */
static void reflux_record_coarse(Ora *o, int s, int l, const OPatch *p, double dt, const double *xf,
                                 const double *yf)
{
    Scen *S = &o->sc[s];
    const int nx = p->nx, ny = p->ny;
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            const int I = p->i0 + i, J = p->j0 + j;
            double *c = S->cflux[l] + reg_index(o, l, I, J, 0);
            c[FACE_W] = dt * xf[2 * ((size_t)j * (nx + 1) + i) + 1];       /* as the right cell of x-edge i */
            c[FACE_E] = dt * xf[2 * ((size_t)j * (nx + 1) + i + 1)];       /* as the left cell of x-edge i+1 */
            c[FACE_S] = dt * yf[2 * ((size_t)i * (ny + 1) + j) + 1];       /* as the upper cell of y-edge j */
            c[FACE_N] = dt * yf[2 * ((size_t)i * (ny + 1) + j + 1)];       /* as the lower cell of y-edge j+1 */
        }
}

/* one fine boundary edge: the outside level-l cell (Io, Jo) decides whether it is
 * a coarse-fine interface (inside the domain, in no other level-l patch) */
static void reflux_add_fine(Ora *o, int s, int l, const OPatch *p, int Io, int Jo, int face, double v)
{
    if (!inside_domain(o, l, Io, Jo)) return;
    if (find_patch(o, s, l, Io, Jo, p)) return;
    const int r = o->c.ratios[l - 1];
    const int Ic = Io / r, Jc = Jo / r;
    Scen *S = &o->sc[s];
    const size_t k = reg_index(o, l - 1, Ic, Jc, face);
    S->fflux[l - 1][k] = S->fflux[l - 1][k] + v / (double)r;
    S->fset[l - 1][k] = 1;
}

/* level l as the fine level: its boundary edges' fluxes, as its own cells used them */
static void reflux_record_fine(Ora *o, int s, int l, const OPatch *p, double dt, const double *xf,
                               const double *yf)
{
    const int nx = p->nx, ny = p->ny;
    for (int j = 0; j < ny; j++) {
        /* west boundary: the coarse cell outside sees the patch on its east face */
        reflux_add_fine(o, s, l, p, p->i0 - 1, p->j0 + j, FACE_E, dt * xf[2 * ((size_t)j * (nx + 1)) + 1]);
        reflux_add_fine(o, s, l, p, p->i0 + nx, p->j0 + j, FACE_W, dt * xf[2 * ((size_t)j * (nx + 1) + nx)]);
    }
    for (int i = 0; i < nx; i++) {
        reflux_add_fine(o, s, l, p, p->i0 + i, p->j0 - 1, FACE_N, dt * yf[2 * ((size_t)i * (ny + 1)) + 1]);
        reflux_add_fine(o, s, l, p, p->i0 + i, p->j0 + ny, FACE_S, dt * yf[2 * ((size_t)i * (ny + 1) + ny)]);
    }
}

/* after the fine steps and the averaging: correct the uncovered level-l cells */
static void reflux_apply(Ora *o, int s, int l)
{
    Scen *S = &o->sc[s];
    const int r = o->c.ratios[l];
    const double dx = o->dxl[l], dy = o->dyl[l];
    Level *L = &S->lev[l];
    for (int k = 0; k < L->n; k++) {
        OPatch *p = L->p[k];
        for (int j = 0; j < p->ny; j++)
            for (int i = 0; i < p->nx; i++) {
                const int I = p->i0 + i, J = p->j0 + j;
                const size_t b = reg_index(o, l, I, J, 0);
                const unsigned char *f = S->fset[l] + b;
                if (!(f[0] | f[1] | f[2] | f[3])) continue;
                if (find_patch(o, s, l + 1, I * r, J * r, NULL)) continue;   /* covered: averaged */
                const double *c = S->cflux[l] + b, *fi = S->fflux[l] + b;
                double h = p->h[OIDX(p, i, j)];
                if (f[FACE_W]) h = h + (fi[FACE_W] - c[FACE_W]) / dx;
                if (f[FACE_E]) h = h + (c[FACE_E] - fi[FACE_E]) / dx;
                if (f[FACE_S]) h = h + (fi[FACE_S] - c[FACE_S]) / dy;
                if (f[FACE_N]) h = h + (c[FACE_N] - fi[FACE_N]) / dy;
                if (h < 0.0) h = 0.0;
                p->h[OIDX(p, i, j)] = h;
            }
    }
}

/* ------------------------------------------------------------------ */
/* recursive time stepping (Sec. 3.1)                                  */

static void restore_old(OPatch *p)
{
    size_t n = (size_t)(p->nx + 4) * (size_t)(p->ny + 4);
    memcpy(p->h, p->h0, n * sizeof(double));
    memcpy(p->hu, p->hu0, n * sizeof(double));
    memcpy(p->hv, p->hv0, n * sizeof(double));
}

/* One step of level l (all its patches) and, recursively, the r_l steps of
 * level l+1, the averaging and the regrids (Sec. 3.1).
 * CFL retake (Sec. 2.2: nu <= 1 must hold): a level-1 step whose Courant
 * number nu = dt * max(sx/dx, sy/dy) exceeds cfl_max is discarded before any
 * finer level moves; dt^1 becomes cfl_desired / max(sx/dx, sy/dy) with the
 * speeds that step saw, and the step is taken again from the same state.  A
 * retaken step that still exceeds cfl_max, and a step of a finer level (whose
 * dt^l = dt^1 / R_l is fixed by the level-1 step already taken), are kept and
 * counted as violations. */
static int advance(Ora *o, int s, int l)
{
    Scen *S = &o->sc[s];
    Level *L = &S->lev[l];
    double alpha = l > 0 ? (double)S->substep[l] / (double)o->c.ratios[l - 1] : 0.0;
    if (fill_ghosts(o, s, l, alpha)) return -1;
    const int coarse_of_next = o->c.reflux && l + 1 < o->c.num_levels && S->lev[l + 1].n > 0;
    for (int attempt = 0;; attempt++) {
        double dt = S->dt1 / (double)o->R[l];
        if (coarse_of_next) reflux_clear(o, s, l);
        double sx = 0.0, sy = 0.0;
        const long clips0 = ora_neg_clips;
        for (int k = 0; k < L->n; k++) {
            OPatch *p = L->p[k];
            save_old(p);
            double a, b;
            if (o->c.reflux && (coarse_of_next || l > 0)) {
                double *xf = malloc(2 * (size_t)p->ny * (p->nx + 1) * sizeof(double));
                double *yf = malloc(2 * (size_t)p->nx * (p->ny + 1) * sizeof(double));
                ora_step_patch_flux(p, o->c.g, o->c.drytol, dt, o->dxl[l], o->dyl[l], &a, &b, xf, yf);
                if (coarse_of_next) reflux_record_coarse(o, s, l, p, dt, xf, yf);
                if (l > 0) reflux_record_fine(o, s, l, p, dt, xf, yf);
                free(xf);
                free(yf);
            } else if (o->c.spherical) {
                double *kap = malloc((size_t)(p->ny + 4) * sizeof(double));
                double *ced = malloc((size_t)(p->ny + 5) * sizeof(double));
                for (int j = -2; j < p->ny + 2; j++) kap[j + 2] = geo_kap(o, l, p->j0 + j);
                for (int j = -2; j <= p->ny + 2; j++) ced[j + 2] = geo_ced(o, l, p->j0 + j);
                ora_step_patch_geo(p, o->c.g, o->c.drytol, dt, phys_dx(o, l), phys_dy(o, l), kap, ced, &a, &b);
                free(kap);
                free(ced);
            } else if (o->c.transverse)
                ora_step_patch_unsplit(p, o->c.g, o->c.drytol, dt, o->dxl[l], o->dyl[l], &a, &b);
            else
                ora_step_patch(p, o->c.g, o->c.drytol, dt, o->dxl[l], o->dyl[l], &a, &b);
            if (o->c.manning_n > 0.0) ora_friction_patch(p, o->c.g, o->c.drytol, o->c.manning_n, dt);
            sx = fmax(sx, a);
            sy = fmax(sy, b);
        }
        double rate = fmax(sx / phys_dx(o, l), sy / phys_dy(o, l));
        if (dt * rate > o->c.cfl_max) {
            if (l == 0 && o->c.cfl_retake && attempt == 0) {
                for (int k = 0; k < L->n; k++) restore_old(L->p[k]);
                ora_neg_clips = clips0;
                S->dt1 = o->c.cfl_desired / rate;
                S->cfl_retakes++;
                continue;
            }
            S->cfl_viol++;
        }
        S->neg_clips += ora_neg_clips - clips0;
        for (int k = 0; k < L->n; k++) S->cell_updates += (double)L->p[k]->nx * (double)L->p[k]->ny;
        S->rate[l] = fmax(S->rate[l], rate);
        break;
    }

    if (l + 1 < o->c.num_levels && S->lev[l + 1].n > 0) {
        for (int k = 0; k < o->c.ratios[l]; k++) {
            S->substep[l + 1] = k;
            if (advance(o, s, l + 1)) return -1;
        }
        average_down(o, s, l + 1);
        if (coarse_of_next) reflux_apply(o, s, l);
    }
    S->nsteps[l]++;
    if (l + 1 < o->c.num_levels && o->c.regrid_interval > 0 && S->nsteps[l] % o->c.regrid_interval == 0)
        if (regrid_from(o, s, l)) return -1;
    return 0;
}

/* ------------------------------------------------------------------ */
/* gauges and fields (Sec. 5.1.2)                                      */

static const OPatch *finest_at(const Ora *o, int s, int lmax, double x, double y, int *lout)
{
    for (int l = lmax; l >= 0; l--) {
        int I = (int)floor((x - o->c.x0) / o->dxl[l]);
        int J = (int)floor((y - o->c.y0) / o->dyl[l]);
        if (!inside_domain(o, l, I, J)) continue;
        OPatch *p = find_patch(o, s, l, I, J, NULL);
        if (p) { *lout = l; return p; }
    }
    return NULL;
}

static double gauge_eta(const Ora *o, int s, double x, double y)
{
    int l;
    const OPatch *p = finest_at(o, s, o->c.num_levels - 1, x, y, &l);
    if (!p) return NAN;
    double fx = (x - o->c.x0) / o->dxl[l] - 0.5, fy = (y - o->c.y0) / o->dyl[l] - 0.5;
    int ia = (int)floor(fx), ja = (int)floor(fy);
    double tx = fx - (double)ia, ty = fy - (double)ja;
    if (ia < p->i0) { ia = p->i0; tx = 0.0; }
    if (ia > p->i0 + p->nx - 2) { ia = p->i0 + p->nx - 2; tx = 1.0; }
    if (ja < p->j0) { ja = p->j0; ty = 0.0; }
    if (ja > p->j0 + p->ny - 2) { ja = p->j0 + p->ny - 2; ty = 1.0; }
    int i = ia - p->i0, j = ja - p->j0;
    double e00 = p->h[OIDX(p, i, j)] + p->B[OIDX(p, i, j)];
    double e10 = p->h[OIDX(p, i + 1, j)] + p->B[OIDX(p, i + 1, j)];
    double e01 = p->h[OIDX(p, i, j + 1)] + p->B[OIDX(p, i, j + 1)];
    double e11 = p->h[OIDX(p, i + 1, j + 1)] + p->B[OIDX(p, i + 1, j + 1)];
    double a = e00 + tx * (e10 - e00);
    double b = e01 + tx * (e11 - e01);
    return a + ty * (b - a);
}

static void sample_gauges(Ora *o)
{
    if (o->ngauge == 0) return;
    int ns = o->c.n_scenarios;
    if (o->nsamp == o->capsamp) {
        o->capsamp = o->capsamp ? 2 * o->capsamp : 64;
        o->gt = (double *)realloc(o->gt, (size_t)o->capsamp * ns * sizeof(double));
        o->geta = (double *)realloc(o->geta, (size_t)o->capsamp * ns * o->ngauge * sizeof(double));
    }
    for (int s = 0; s < ns; s++) {
        o->gt[(size_t)o->nsamp * ns + s] = o->sc[s].t;
        for (int g = 0; g < o->ngauge; g++)
            o->geta[((size_t)o->nsamp * ns + s) * o->ngauge + g] = gauge_eta(o, s, o->gxy[2 * g], o->gxy[2 * g + 1]);
    }
    o->nsamp++;
}

/* ------------------------------------------------------------------ */
/* public driver                                                       */

void *ora_create(const ora_config *cfg)
{
    if (cfg->num_levels < 1 || cfg->num_levels > ORA_MAX_LEVELS || cfg->nx < 2 || cfg->ny < 2 ||
        cfg->n_scenarios < 1)
        return NULL;
    Ora *o = (Ora *)calloc(1, sizeof *o);
    o->c = *cfg;
    if (o->c.cluster_eff <= 0.0) o->c.cluster_eff = 0.7;
    if (!(o->c.manning_n >= 0.0)) { free(o); return NULL; }
    if (o->c.spherical && (o->c.transverse || !(cfg->y0 > -90.0) || !(cfg->y0 + cfg->ny * cfg->dy < 90.0))) {
        free(o);
        return NULL;
    }
    if (o->c.reflux && (o->c.transverse || o->c.spherical)) {   /* refluxing: split scheme on plane grids */
        free(o);
        return NULL;
    }
    o->R[0] = 1;
    for (int l = 1; l < cfg->num_levels; l++) o->R[l] = o->R[l - 1] * cfg->ratios[l - 1];
    for (int l = 0; l < cfg->num_levels; l++) {
        o->nxl[l] = cfg->nx * o->R[l];
        o->nyl[l] = cfg->ny * o->R[l];
        o->dxl[l] = cfg->dx / (double)o->R[l];
        o->dyl[l] = cfg->dy / (double)o->R[l];
    }
    o->sc = (Scen *)calloc((size_t)cfg->n_scenarios, sizeof(Scen));
    return o;
}

static void grid_free(TopoGrid *g) { free(g->v); }

void ora_destroy(void *vo)
{
    Ora *o = (Ora *)vo;
    if (!o) return;
    for (int s = 0; s < o->c.n_scenarios; s++) {
        Scen *S = &o->sc[s];
        for (int l = 0; l < ORA_MAX_LEVELS; l++) {
            for (int k = 0; k < S->lev[l].n; k++) patch_free(S->lev[l].p[k]);
            free(S->lev[l].p);
        }
        for (int k = 0; k < S->nup; k++) grid_free(&S->up[k]);
        free(S->up);
        if (S->has_eta0) grid_free(&S->eta0);
        if (S->has_uv0) { grid_free(&S->u0); grid_free(&S->v0); }
        for (int l = 0; l < ORA_MAX_LEVELS; l++) { free(S->cflux[l]); free(S->fflux[l]); free(S->fset[l]); }
    }
    for (int k = 0; k < o->ntopo; k++) grid_free(&o->topo[k]);
    free(o->topo);
    free(o->sc);
    free(o->gxy);
    free(o->gt);
    free(o->geta);
    free(o);
}

static TopoGrid grid_copy(const double *v, int nx, int ny, double x0, double y0, double dx, double dy)
{
    TopoGrid g;
    g.nx = nx; g.ny = ny; g.x0 = x0; g.y0 = y0; g.dx = dx; g.dy = dy;
    g.v = (double *)malloc((size_t)nx * ny * sizeof(double));
    memcpy(g.v, v, (size_t)nx * ny * sizeof(double));
    return g;
}

int ora_add_topo(void *vo, const double *B, int nx, int ny, double x0, double y0, double dx, double dy)
{
    Ora *o = (Ora *)vo;
    if (o->initialized || nx < 2 || ny < 2) return -1;
    o->topo = (TopoGrid *)realloc(o->topo, (size_t)(o->ntopo + 1) * sizeof(TopoGrid));
    o->topo[o->ntopo++] = grid_copy(B, nx, ny, x0, y0, dx, dy);
    return 0;
}

int ora_set_eta(void *vo, int s, const double *eta, int nx, int ny, double x0, double y0, double dx, double dy)
{
    Ora *o = (Ora *)vo;
    if (o->initialized || s < 0 || s >= o->c.n_scenarios || nx < 2 || ny < 2) return -1;
    Scen *S = &o->sc[s];
    if (S->has_eta0) grid_free(&S->eta0);
    S->eta0 = grid_copy(eta, nx, ny, x0, y0, dx, dy);
    S->has_eta0 = 1;
    return 0;
}

/* initial depth-averaged velocities: hu = h u, hv = h v on wet cells at init */
int ora_set_velocity(void *vo, int s, const double *u, const double *v, int nx, int ny, double x0, double y0,
                     double dx, double dy)
{
    Ora *o = (Ora *)vo;
    if (o->initialized || s < 0 || s >= o->c.n_scenarios || nx < 2 || ny < 2) return -1;
    Scen *S = &o->sc[s];
    if (S->has_uv0) { grid_free(&S->u0); grid_free(&S->v0); }
    S->u0 = grid_copy(u, nx, ny, x0, y0, dx, dy);
    S->v0 = grid_copy(v, nx, ny, x0, y0, dx, dy);
    S->has_uv0 = 1;
    return 0;
}

/* seafloor uplift: B += dB with h unchanged (eta rises with the seafloor) */
int ora_add_uplift(void *vo, int s, const double *dB, int nx, int ny, double x0, double y0, double dx, double dy)
{
    Ora *o = (Ora *)vo;
    if (s < 0 || s >= o->c.n_scenarios || nx < 2 || ny < 2) return -1;
    Scen *S = &o->sc[s];
    S->up = (TopoGrid *)realloc(S->up, (size_t)(S->nup + 1) * sizeof(TopoGrid));
    S->up[S->nup] = grid_copy(dB, nx, ny, x0, y0, dx, dy);
    const TopoGrid *U = &S->up[S->nup];
    S->nup++;
    if (!o->initialized) return 0;
    for (int l = 0; l < o->c.num_levels; l++)
        for (int k = 0; k < S->lev[l].n; k++) {
            OPatch *p = S->lev[l].p[k];
            for (int j = -2; j < p->ny + 2; j++)
                for (int i = -2; i < p->nx + 2; i++) {
                    int I = p->i0 + i, J = p->j0 + j;
                    if (!inside_domain(o, l, I, J)) continue;
                    double x = xc(o, l, I), y = yc(o, l, J);
                    if (grid_contains(U, x, y)) p->B[OIDX(p, i, j)] = p->B[OIDX(p, i, j)] + grid_bilinear(U, x, y);
                }
            apply_bc_field(o, p, p->B, 0, 0);
        }
    return 0;
}

int ora_init(void *vo)
{
    Ora *o = (Ora *)vo;
    if (o->initialized || o->ntopo == 0) return -1;
    int T = o->c.level1_tile > 0 ? o->c.level1_tile : (o->c.nx > o->c.ny ? o->c.nx : o->c.ny);
    for (int s = 0; s < o->c.n_scenarios; s++) {
        Scen *S = &o->sc[s];
        for (int j0 = 0; j0 < o->c.ny; j0 += T)
            for (int i0 = 0; i0 < o->c.nx; i0 += T) {
                int w = o->c.nx - i0 < T ? o->c.nx - i0 : T;
                int h = o->c.ny - j0 < T ? o->c.ny - j0 : T;
                OPatch *p = patch_new(0, s, i0, j0, w, h);
                for (int j = -2; j < h + 2; j++)
                    for (int i = -2; i < w + 2; i++) {
                        int I = i0 + i, J = j0 + j;
                        if (!inside_domain(o, 0, I, J)) continue;
                        double x = xc(o, 0, I), y = yc(o, 0, J);
                        size_t k = OIDX(p, i, j);
                        double B0 = base_topo(o, x, y);
                        double eta = 0.0;
                        if (S->has_eta0 && grid_contains(&S->eta0, x, y)) eta = grid_bilinear(&S->eta0, x, y);
                        double hh = eta - B0;
                        if (hh < 0.0) hh = 0.0;
                        p->h[k] = hh;
                        if (S->has_uv0 && hh >= o->c.drytol && grid_contains(&S->u0, x, y)) {
                            p->hu[k] = hh * grid_bilinear(&S->u0, x, y);
                            p->hv[k] = hh * grid_bilinear(&S->v0, x, y);
                        }
                        p->B[k] = uplift_sum(S, B0, x, y);
                    }
                apply_bc_field(o, p, p->B, 0, 0);
                save_old(p);
                level_push(&S->lev[0], p);
            }
        level_cell_rate(o, s, 0);
    }
    o->initialized = 1;
    for (int s = 0; s < o->c.n_scenarios; s++)
        if (regrid_from(o, s, 0)) return -1;
    return 0;
}

int ora_step(void *vo, int n, double *t_out)
{
    Ora *o = (Ora *)vo;
    if (!o->initialized) return -1;
    for (int it = 0; it < n; it++) {
        for (int s = 0; s < o->c.n_scenarios; s++) {
            Scen *S = &o->sc[s];
            double m = 0.0;
            for (int l = 0; l < o->c.num_levels; l++) m = fmax(m, S->rate[l] / (double)o->R[l]);
            double dt = m > 0.0 ? o->c.cfl_desired / m : o->c.dt_max;
            S->dt1 = fmin(dt, o->c.dt_max);
            for (int l = 0; l < o->c.num_levels; l++) S->rate[l] = 0.0;
            if (advance(o, s, 0)) return -1;
            S->t = S->t + S->dt1;
        }
        sample_gauges(o);
    }
    if (t_out)
        for (int s = 0; s < o->c.n_scenarios; s++) t_out[s] = o->sc[s].t;
    return 0;
}

int ora_regrid(void *vo, int s, int level)
{
    Ora *o = (Ora *)vo;
    if (!o->initialized || s < 0 || s >= o->c.n_scenarios || level < 1 || level >= o->c.num_levels) return -1;
    return regrid_from(o, s, level - 1);
}

int ora_num_patches(void *vo, int s, int level)
{
    Ora *o = (Ora *)vo;
    if (s < 0 || s >= o->c.n_scenarios || level < 1 || level > o->c.num_levels) return -1;
    return o->sc[s].lev[level - 1].n;
}

int ora_get_patch(void *vo, int s, int level, int k, int *box, double *h, double *hu, double *hv, double *B)
{
    Ora *o = (Ora *)vo;
    if (s < 0 || s >= o->c.n_scenarios || level < 1 || level > o->c.num_levels) return -1;
    Level *L = &o->sc[s].lev[level - 1];
    if (k < 0 || k >= L->n) return -1;
    OPatch *p = L->p[k];
    box[0] = p->i0; box[1] = p->j0; box[2] = p->nx; box[3] = p->ny;
    for (int j = 0; j < p->ny; j++)
        for (int i = 0; i < p->nx; i++) {
            size_t kk = OIDX(p, i, j), d = (size_t)j * p->nx + i;
            if (h) h[d] = p->h[kk];
            if (hu) hu[d] = p->hu[kk];
            if (hv) hv[d] = p->hv[kk];
            if (B) B[d] = p->B[kk];
        }
    return 0;
}

int ora_read_field(void *vo, int s, int level, int field, double *dst, int nx, int ny,
                   double x0, double y0, double dx, double dy)
{
    Ora *o = (Ora *)vo;
    if (s < 0 || s >= o->c.n_scenarios || level < 0 || level > o->c.num_levels) return -1;
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            double x = x0 + (double)i * dx, y = y0 + (double)j * dy;
            double v = NAN;
            int l;
            const OPatch *p = NULL;
            if (level == 0) p = finest_at(o, s, o->c.num_levels - 1, x, y, &l);
            else {
                l = level - 1;
                int I = (int)floor((x - o->c.x0) / o->dxl[l]), J = (int)floor((y - o->c.y0) / o->dyl[l]);
                if (inside_domain(o, l, I, J)) p = find_patch(o, s, l, I, J, NULL);
            }
            if (p) {
                int I = (int)floor((x - o->c.x0) / o->dxl[l]), J = (int)floor((y - o->c.y0) / o->dyl[l]);
                size_t k = OIDX(p, I - p->i0, J - p->j0);
                double hh = p->h[k], B = p->B[k];
                switch (field) {
                case ORA_F_H: v = hh; break;
                case ORA_F_HU: v = p->hu[k]; break;
                case ORA_F_HV: v = p->hv[k]; break;
                case ORA_F_ETA: v = hh + B; break;
                case ORA_F_ZETA: v = B > 0.0 ? hh : hh + B; break;
                case ORA_F_B: v = B; break;
                default: return -1;
                }
            }
            dst[(size_t)j * nx + i] = v;
        }
    return 0;
}

int ora_add_gauges(void *vo, const double *xy, int n)
{
    Ora *o = (Ora *)vo;
    if (o->nsamp > 0 || n < 0) return -1;
    o->gxy = (double *)realloc(o->gxy, (size_t)(o->ngauge + n) * 2 * sizeof(double));
    memcpy(o->gxy + 2 * o->ngauge, xy, (size_t)n * 2 * sizeof(double));
    o->ngauge += n;
    return 0;
}

int ora_read_gauges(void *vo, double *t, double *eta, int max_samples, int *n_written)
{
    Ora *o = (Ora *)vo;
    int ns = o->c.n_scenarios;
    int n = o->nsamp < max_samples ? o->nsamp : max_samples;
    memcpy(t, o->gt, (size_t)n * ns * sizeof(double));
    memcpy(eta, o->geta, (size_t)n * ns * o->ngauge * sizeof(double));
    *n_written = n;
    return 0;
}

/* out: dt1, t, mass on level 1, cfl violations, cell updates, patches per level
 * (ORA_MAX_LEVELS entries), CFL retakes, clipped depths */
int ora_stats(void *vo, int s, double *out)
{
    Ora *o = (Ora *)vo;
    if (s < 0 || s >= o->c.n_scenarios) return -1;
    Scen *S = &o->sc[s];
    double mass = 0.0;
    Level *L = &S->lev[0];
    for (int k = 0; k < L->n; k++) {
        OPatch *p = L->p[k];
        for (int j = 0; j < p->ny; j++) {
            const double kj = o->c.spherical ? geo_kap(o, 0, p->j0 + j) : 1.0;
            for (int i = 0; i < p->nx; i++)
                mass = o->c.spherical ? mass + kj * p->h[OIDX(p, i, j)] : mass + p->h[OIDX(p, i, j)];
        }
    }
    out[0] = S->dt1;
    out[1] = S->t;
    out[2] = mass * phys_dx(o, 0) * phys_dy(o, 0);
    out[3] = (double)S->cfl_viol;
    out[4] = S->cell_updates;
    for (int l = 0; l < ORA_MAX_LEVELS; l++) out[5 + l] = l < o->c.num_levels ? (double)S->lev[l].n : 0.0;
    out[5 + ORA_MAX_LEVELS] = (double)S->cfl_retakes;
    out[6 + ORA_MAX_LEVELS] = (double)S->neg_clips;
    return 0;
}
