/*
 * swe.c -- FP64 CPU oracle: Riemann solver, MC wave limiter and the
 * dimensionally split wave-propagation update of one patch.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Plain loops, no blocking, no
 * fusion: each function follows the paper's equations in order.
 *
 *   Sec. 2.1, Eq. (swe)                      shallow water equations with bathymetry B
 *   Sec. 2.2, Eq. (wave_propagation_form)    first-order fluctuation update
 *   Sec. 2.2, Eq. (wave_propagation_2nd_order) and the correction flux
 *                                            F~ = 1/2 sum (1 - dt/dx |l|) |l| W~
 *   Sec. 2.2, Eq. (theta) and the upwind index I   wave limiter ratio
 *   Sec. 2.2, Eqs. (..._x), (..._y)          Godunov dimensional splitting, x then y
 *   Sec. 2.2, CFL condition                  nu = |s dt / dx| <= 1
 *   Sec. 2.1, drag D (Manning, n)           friction step after each level step
 *   spherical coordinates (Sec. 1, supported for transoceanic runs): capacity-form split step
 *
 * Readings of points the paper leaves open:
 *   - f-wave form: the solver decomposes the flux jump (including the
 *     bathymetry source -g hbar dB folded into the momentum flux jump as
 *     g hbar d(eta)) into f-waves Z^p = s^p W^p, so A-dQ/A+dQ are the sums of
 *     the left/right-going Z^p and the correction flux is
 *     1/2 sum sgn(s)(1 - dt/dx|s|) Z~^p, which equals the paper's form when
 *     Z = s W.  theta uses the squared norm Z_I.Z_i / Z_i.Z_i (the printed
 *     single-norm form is not dimensionless).
 *   - MC limiter phi(theta) = max(0, min((1+theta)/2, 2, 2 theta)).
 *   - Upwind edge: s >= 0 -> I = i-1, s < 0 -> I = i+1.
 *   - Riemann solver (the paper only cites George 2008): Einfeldt-type speeds
 *     from Roe averages, two acoustic f-waves from an HLLE-type decomposition
 *     of the augmented jump (d eta, d hu) and the flux jump with the bed
 *     source, a contact wave carrying the transverse momentum at the Roe
 *     speed, dry-bed speeds u - c, u + 2c (mirrored for a dry left side), and a
 *     reflecting wall when a dry cell's bed lies above the wet side's
 *     two-rarefaction middle-state surface.  The bed step is a stationary
 *     wave whose depth jump keeps the surface continuous (still water stays
 *     still), bounded so that every constant state of the fan has a
 *     non-negative depth.  A wave of speed exactly 0 is split half into each
 *     cell.
 *   - After each sweep: h < 0 -> 0, and h < drytol -> zero momenta.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "ora_internal.h"

/* depths that came out of a sweep negative and were clipped to zero; the
 * driver reports them with the run's statistics */
long ora_neg_clips = 0;

/* Augmented f-wave Riemann solver for the normal direction.
 * Inputs per side: depth h, normal momentum hn, transverse momentum ht, bed B.
 * Output: f-waves Z[p][m] (m = mass, normal, transverse), speeds s[p], and
 * wall flags (the dry side was replaced by the mirror of the wet side). */
void ora_riemann(double g, double drytol,
                 double hL, double hnL, double htL, double BL,
                 double hR, double hnR, double htR, double BR, ora_rp *r)
{
    memset(r, 0, sizeof *r);
    int wetL = hL >= drytol;
    int wetR = hR >= drytol;
    if (!wetL && !wetR)
        return;

    double uL = 0.0, vL = 0.0, uR = 0.0, vR = 0.0;
    if (wetL) { uL = hnL / hL; vL = htL / hL; }
    if (wetR) { uR = hnR / hR; vR = htR / hR; }

    /* wet/dry: can the wet water reach the dry cell?  Two-rarefaction
     * estimate of the middle depth against a wall: sqrt(g hm) = c + u/2
     * (u measured toward the dry cell). */
    if (wetL && !wetR) {
        double a = sqrt(g * hL) + 0.5 * uL;
        double hm = a > 0.0 ? a * a / g : 0.0;
        if (hm + BL <= BR) {
            r->wallR = 1;
            hR = hL; hnR = -hnL; htR = htL; BR = BL; uR = -uL; vR = vL; wetR = 1;
        }
    } else if (!wetL && wetR) {
        double a = sqrt(g * hR) - 0.5 * uR;
        double hm = a > 0.0 ? a * a / g : 0.0;
        if (hm + BR <= BL) {
            r->wallL = 1;
            hL = hR; hnL = -hnR; htL = htR; BL = BR; uL = -uR; vL = vR; wetL = 1;
        }
    }

    double s1, s2, s3;
    if (wetL && wetR) {
        double cL = sqrt(g * hL), cR = sqrt(g * hR);
        double sqL = sqrt(hL), sqR = sqrt(hR);
        double uhat = (sqL * uL + sqR * uR) / (sqL + sqR);
        double chat = sqrt(g * (0.5 * (hL + hR)));
        s1 = fmin(uL - cL, uhat - chat);
        s3 = fmax(uR + cR, uhat + chat);
        s2 = uhat;
    } else if (wetL) {              /* right side is a dry bed below the water */
        double cL = sqrt(g * hL);
        s1 = uL - cL;
        s3 = uL + 2.0 * cL;
        s2 = uL;
    } else {                        /* left side is a dry bed */
        double cR = sqrt(g * hR);
        s1 = uR - 2.0 * cR;
        s3 = uR + cR;
        s2 = uR;
    }

    /* Augmented jump: the bed step is a stationary wave at x = 0 across which
     * the depth jumps by delta; the acoustic waves carry the rest of the depth
     * jump, dh - delta.  Still water over a step is a steady state, so delta
     * is BL - BR (the surface is continuous through the stationary wave) and
     * the mass jump to decompose is d(eta).  The momentum flux jump has the
     * bathymetry source folded in: d(hu^2 + g h^2/2) + g hbar dB =
     * d(hu^2) + g hbar d(eta).
     * HLLE-type decomposition into two acoustic f-waves: W1 = Q* - Q_l with
     * the middle state of the two-speed approximation, W3 = dQ - W1,
     * Z = s W, so Z1 + Z3 equals the flux jump exactly; a third (contact)
     * wave at the Roe speed carries what remains of the transverse momentum
     * flux after each acoustic wave has advected v of its upwind side. */
    double hbar = 0.5 * (hL + hR);
    double deta = (hR + BR) - (hL + BL);
    double d2 = hnR - hnL;
    double d3 = (hnR * uR - hnL * uL) + (g * hbar) * deta;
    double d4 = hnR * vR - hnL * vL;
    double den = s3 - s1;

    /* Non-negative depth (Sec. 2.2: the solver keeps depths non-negative).
     * With M = s3 hR - s1 hL - d(hu) ((s3 - s1) times the two-speed middle
     * depth of a flat bed), the depths of the constant states of the fan are
     *   s1 < 0 < s3:  (M - s3 delta)/den left of the bed step, (M - s1 delta)/den right of it;
     *   s1 >= 0:      hL + delta between x = 0 and s1, (M - s1 delta)/den between s1 and s3;
     *   s3 <= 0:      (M - s3 delta)/den between s1 and s3, hR - delta between s3 and x = 0.
     * Where the still-water delta would make one of them negative, delta is
     * moved to the value that makes it zero. */
    double M = (s3 * hR - s1 * hL) - d2;
    double delta = BL - BR;
    int bounded = 0;
    if (s1 < 0.0 && s3 > 0.0) {
        if (M - s3 * delta < 0.0) { delta = M / s3; bounded = 1; }
        else if (M - s1 * delta < 0.0) { delta = M / s1; bounded = 1; }
    } else if (s1 >= 0.0) {
        if (hL + delta < 0.0) { delta = -hL; bounded = 1; }
        else if (s1 > 0.0 && M - s1 * delta < 0.0) { delta = M / s1; bounded = 1; }
    } else {
        if (hR - delta < 0.0) { delta = hR; bounded = 1; }
        else if (s3 < 0.0 && M - s3 * delta < 0.0) { delta = M / s3; bounded = 1; }
    }
    double d1 = bounded ? (hR - hL) - delta : deta;
    double w1m = (s3 * d1 - d2) / den;
    double w1n = (s3 * d2 - d3) / den;
    double b1 = s1 * w1m, g1 = s1 * w1n;
    double b3 = s3 * (d1 - w1m), g3 = s3 * (d2 - w1n);

    r->Z[0][0] = b1;  r->Z[0][1] = g1;  r->Z[0][2] = b1 * vL;
    r->Z[2][0] = b3;  r->Z[2][1] = g3;  r->Z[2][2] = b3 * vR;
    r->Z[1][0] = 0.0; r->Z[1][1] = 0.0; r->Z[1][2] = (d4 - b1 * vL) - b3 * vR;
    r->s[0] = s1; r->s[1] = s2; r->s[2] = s3;
}

/* MC limiter, Sec. 2.2 (limiter named in Sec. 5.1.1) */
double ora_mc_limiter(double theta)
{
    double t = 0.5 * (1.0 + theta);
    t = fmin(t, 2.0);
    t = fmin(t, 2.0 * theta);
    return fmax(0.0, t);
}

/* share of a wave of speed s going left (A-dQ) and right (A+dQ) */
static double w_left(double s) { return s < 0.0 ? 1.0 : (s == 0.0 ? 0.5 : 0.0); }
static double w_right(double s) { return s > 0.0 ? 1.0 : (s == 0.0 ? 0.5 : 0.0); }

/* One 1D sweep over n interior cells with 2 ghost cells on each side.
 * Input arrays have n+4 entries (cell c at index c+2).  The updated interior
 * is written to the output arrays (n entries).  Returns max |s| over the
 * edges 0..n (the edges that touch an interior cell).
 * gflux (NULL: not wanted; 2 (n+1) entries): the mass flux of edge e as each
 * neighbour's update uses it -- the update of cell i is
 * h_i - dtdx (G-_{i+1} - G+_i) with G-_e = hn_{e-1} + (A-dQ)_e + F~_e (seen
 * from the left cell) and G+_e = hn_e - (A+dQ)_e + F~_e (from the right):
 * gflux[2e] = G-_e, gflux[2e+1] = G+_e.  Used by the refluxing option. */
static double sweep_1d_flux(double g, double drytol, int n, double dtdx,
                            const double *h, const double *hn, const double *ht, const double *B,
                            double *ho, double *hno, double *hto, double *gflux)
{
    /* Riemann problems at edges e = -1 .. n+1 (edge e between cells e-1 and e) */
    ora_rp *rp = (ora_rp *)malloc((size_t)(n + 3) * sizeof *rp);
    for (int e = -1; e <= n + 1; e++) {
        int cl = e - 1 + 2, cr = e + 2;
        ora_riemann(g, drytol, h[cl], hn[cl], ht[cl], B[cl], h[cr], hn[cr], ht[cr], B[cr], &rp[e + 1]);
    }

    double (*amdq)[3] = malloc((size_t)(n + 1) * sizeof *amdq);
    double (*apdq)[3] = malloc((size_t)(n + 1) * sizeof *apdq);
    double (*F)[3] = malloc((size_t)(n + 1) * sizeof *F);
    double smax = 0.0;

    for (int e = 0; e <= n; e++) {
        const ora_rp *r = &rp[e + 1];
        /* fluctuations, Eq. (wave_propagation_form) in f-wave form */
        for (int m = 0; m < 3; m++) {
            amdq[e][m] = (w_left(r->s[0]) * r->Z[0][m] + w_left(r->s[1]) * r->Z[1][m]) + w_left(r->s[2]) * r->Z[2][m];
            apdq[e][m] = (w_right(r->s[0]) * r->Z[0][m] + w_right(r->s[1]) * r->Z[1][m]) + w_right(r->s[2]) * r->Z[2][m];
        }
        if (r->wallR) { apdq[e][0] = 0.0; apdq[e][1] = 0.0; apdq[e][2] = 0.0; }
        if (r->wallL) { amdq[e][0] = 0.0; amdq[e][1] = 0.0; amdq[e][2] = 0.0; }

        /* limited second-order correction flux */
        double c[3] = {0.0, 0.0, 0.0};
        if (!r->wallL && !r->wallR) {
            for (int p = 0; p < 3; p++) {
                const double *Zi = r->Z[p];
                double dii = (Zi[0] * Zi[0] + Zi[1] * Zi[1]) + Zi[2] * Zi[2];
                double phi = 0.0;
                if (dii != 0.0) {
                    int I = r->s[p] >= 0.0 ? e - 1 : e + 1;
                    const double *ZI = rp[I + 1].Z[p];
                    double dIi = (ZI[0] * Zi[0] + ZI[1] * Zi[1]) + ZI[2] * Zi[2];
                    phi = ora_mc_limiter(dIi / dii);
                }
                double s = r->s[p];
                double cp = (1.0 - dtdx * fabs(s)) * phi;
                if (s < 0.0) cp = -cp;
                else if (s == 0.0) cp = 0.0;
                c[p] = cp;
            }
        }
        for (int m = 0; m < 3; m++)
            F[e][m] = 0.5 * ((c[0] * r->Z[0][m] + c[1] * r->Z[1][m]) + c[2] * r->Z[2][m]);

        double se = fmax(-r->s[0], r->s[2]);
        smax = fmax(smax, se);
        if (gflux) {
            gflux[2 * e] = (hn[e - 1 + 2] + amdq[e][0]) + F[e][0];
            gflux[2 * e + 1] = (hn[e + 2] - apdq[e][0]) + F[e][0];
        }
    }

    /* cell update, Eq. (wave_propagation_2nd_order) */
    for (int i = 0; i < n; i++) {
        const double *q[3] = {h, hn, ht};
        double *qo[3] = {ho, hno, hto};
        for (int m = 0; m < 3; m++) {
            double upd = (apdq[i][m] + amdq[i + 1][m]) + (F[i + 1][m] - F[i][m]);
            qo[m][i] = q[m][i + 2] - dtdx * upd;
        }
        if (ho[i] < 0.0) {
#pragma omp atomic
            ora_neg_clips++;
            ho[i] = 0.0;
        }
        if (ho[i] < drytol) { hno[i] = 0.0; hto[i] = 0.0; }
    }
    free(rp); free(amdq); free(apdq); free(F);
    return smax;
}

static double sweep_1d(double g, double drytol, int n, double dtdx,
                       const double *h, const double *hn, const double *ht, const double *B,
                       double *ho, double *hno, double *hto)
{
    return sweep_1d_flux(g, drytol, n, dtdx, h, hn, ht, B, ho, hno, hto, NULL);
}

/* The y sweep on a latitude-longitude grid (capacity form).  Cell c of the
 * column has capacity kap[c + 2] (its area over the area of an equatorial
 * cell), edge e (between cells e-1 and e) the relative length ced[e]
 * (cos of its latitude).  Fluctuations and correction fluxes are weighted by
 * their edge's length and the update divided by the cell's capacity; the
 * Courant number of edge e is dt |s| ced[e] / (dyp kbar_e), kbar_e the mean
 * capacity of its two cells; the mass gets the divergence term
 * (ced[i+1] - ced[i]) hv_i of the varying edge length, so that it is
 * conserved exactly.  Returns max |s| ced / kbar over the edges 0..n. */
static double sweep_1d_geo(double g, double drytol, int n, double dt, double dyp, const double *kap,
                           const double *ced, const double *h, const double *hn, const double *ht, const double *B,
                           double *ho, double *hno, double *hto)
{
    if (n < 1) return 0.0;
    ora_rp *rp = (ora_rp *)malloc((size_t)(n + 3) * sizeof *rp);
    for (int e = -1; e <= n + 1; e++) {
        int cl = e - 1 + 2, cr = e + 2;
        ora_riemann(g, drytol, h[cl], hn[cl], ht[cl], B[cl], h[cr], hn[cr], ht[cr], B[cr], &rp[e + 1]);
    }
    double (*amdq)[3] = malloc((size_t)(n + 1) * sizeof *amdq);
    double (*apdq)[3] = malloc((size_t)(n + 1) * sizeof *apdq);
    double (*F)[3] = malloc((size_t)(n + 1) * sizeof *F);
    double smax = 0.0;
    for (int e = 0; e <= n; e++) {
        const ora_rp *r = &rp[e + 1];
        for (int m = 0; m < 3; m++) {
            amdq[e][m] = (w_left(r->s[0]) * r->Z[0][m] + w_left(r->s[1]) * r->Z[1][m]) + w_left(r->s[2]) * r->Z[2][m];
            apdq[e][m] = (w_right(r->s[0]) * r->Z[0][m] + w_right(r->s[1]) * r->Z[1][m]) + w_right(r->s[2]) * r->Z[2][m];
        }
        if (r->wallR) { apdq[e][0] = 0.0; apdq[e][1] = 0.0; apdq[e][2] = 0.0; }
        if (r->wallL) { amdq[e][0] = 0.0; amdq[e][1] = 0.0; amdq[e][2] = 0.0; }
        const double kbar = 0.5 * (kap[e - 1 + 2] + kap[e + 2]);
        const double dtdy = (dt * ced[e]) / (kbar * dyp);
        double c[3] = {0.0, 0.0, 0.0};
        if (!r->wallL && !r->wallR) {
            for (int p = 0; p < 3; p++) {
                const double *Zi = r->Z[p];
                double dii = (Zi[0] * Zi[0] + Zi[1] * Zi[1]) + Zi[2] * Zi[2];
                double phi = 0.0;
                if (dii != 0.0) {
                    int I = r->s[p] >= 0.0 ? e - 1 : e + 1;
                    const double *ZI = rp[I + 1].Z[p];
                    double dIi = (ZI[0] * Zi[0] + ZI[1] * Zi[1]) + ZI[2] * Zi[2];
                    phi = ora_mc_limiter(dIi / dii);
                }
                double s = r->s[p];
                double cp = (1.0 - dtdy * fabs(s)) * phi;
                if (s < 0.0) cp = -cp;
                else if (s == 0.0) cp = 0.0;
                c[p] = cp;
            }
        }
        for (int m = 0; m < 3; m++)
            F[e][m] = 0.5 * ((c[0] * r->Z[0][m] + c[1] * r->Z[1][m]) + c[2] * r->Z[2][m]);
        smax = fmax(smax, fmax(-r->s[0], r->s[2]) * (ced[e] / kbar));
    }
    for (int i = 0; i < n; i++) {
        const double *q[3] = {h, hn, ht};
        double *qo[3] = {ho, hno, hto};
        const double dtk = dt / (kap[i + 2] * dyp);
        for (int m = 0; m < 3; m++) {
            double upd = (ced[i] * apdq[i][m] + ced[i + 1] * amdq[i + 1][m]) +
                         (ced[i + 1] * F[i + 1][m] - ced[i] * F[i][m]);
            if (m == 0) upd = upd + (ced[i + 1] - ced[i]) * hn[i + 2];
            qo[m][i] = q[m][i + 2] - dtk * upd;
        }
        if (ho[i] < 0.0) {
#pragma omp atomic
            ora_neg_clips++;
            ho[i] = 0.0;
        }
        if (ho[i] < drytol) { hno[i] = 0.0; hto[i] = 0.0; }
    }
    free(rp); free(amdq); free(apdq); free(F);
    return smax;
}

/* The split step on a latitude-longitude grid: the x sweep of row j is the
 * plane sweep with dt / (kap_j dxp) (all longitude edges have the same
 * length), its speeds scaled by 1 / kap_j; the y sweep is sweep_1d_geo. */
void ora_step_patch_geo(OPatch *p, double g, double drytol, double dt, double dxp, double dyp, const double *kap,
                        const double *ced, double *sx_out, double *sy_out)
{
    int nx = p->nx, ny = p->ny;
    int nmax = (nx > ny ? nx : ny) + 4;
    double *a = malloc(4 * (size_t)nmax * sizeof(double));
    double *o = malloc(3 * (size_t)nmax * sizeof(double));
    double *ah = a, *an = a + nmax, *at = a + 2 * nmax, *aB = a + 3 * nmax;
    double *oh = o, *on = o + nmax, *ot = o + 2 * nmax;
    double sx = 0.0, sy = 0.0;
    for (int j = -2; j < ny + 2; j++) {
        for (int i = -2; i < nx + 2; i++) {
            size_t k = OIDX(p, i, j);
            ah[i + 2] = p->h[k]; an[i + 2] = p->hu[k]; at[i + 2] = p->hv[k]; aB[i + 2] = p->B[k];
        }
        const double kj = kap[j + 2];
        double s = sweep_1d(g, drytol, nx, dt / (kj * dxp), ah, an, at, aB, oh, on, ot);
        if (j >= 0 && j < ny) sx = fmax(sx, s / kj);
        for (int i = 0; i < nx; i++) {
            size_t k = OIDX(p, i, j);
            p->h[k] = oh[i]; p->hu[k] = on[i]; p->hv[k] = ot[i];
        }
    }
    for (int i = 0; i < nx; i++) {
        for (int j = -2; j < ny + 2; j++) {
            size_t k = OIDX(p, i, j);
            ah[j + 2] = p->h[k]; an[j + 2] = p->hv[k]; at[j + 2] = p->hu[k]; aB[j + 2] = p->B[k];
        }
        double s = sweep_1d_geo(g, drytol, ny, dt, dyp, kap, ced + 2, ah, an, at, aB, oh, on, ot);
        sy = fmax(sy, s);
        for (int j = 0; j < ny; j++) {
            size_t k = OIDX(p, i, j);
            p->h[k] = oh[j]; p->hv[k] = on[j]; p->hu[k] = ot[j];
        }
    }
    free(a); free(o);
    *sx_out = sx; *sy_out = sy;
}

/* Q* = x-sweep(Q^n) on every row including the ghost rows (so the y-sweep
 * sees Q* in its ghost cells), then Q^{n+1} = y-sweep(Q*) on the interior,
 * Eqs. (wave_propagation_2nd_order_x/_y). */
void ora_step_patch(OPatch *p, double g, double drytol, double dt, double dx, double dy,
                    double *sx_out, double *sy_out)
{
    ora_step_patch_flux(p, g, drytol, dt, dx, dy, sx_out, sy_out, NULL, NULL);
}

/* ora_step_patch, also returning the edge mass fluxes of the interior rows and
 * columns (xf, yf may be NULL): xf[2 ((j (nx + 1)) + e) + side] for x-edge e
 * (0..nx) of row j (0..ny-1), yf[2 ((i (ny + 1)) + e) + side] for y-edge e of
 * column i; side 0 as the lower/left cell uses it, 1 as the upper/right cell
 * does (sweep_1d_flux; the y sweep's fluxes are those of Q*). */
void ora_step_patch_flux(OPatch *p, double g, double drytol, double dt, double dx, double dy,
                         double *sx_out, double *sy_out, double *xf, double *yf)
{
    int nx = p->nx, ny = p->ny;
    int nmax = (nx > ny ? nx : ny) + 4;
    double sx = 0.0, sy = 0.0;
    double dtdx = dt / dx, dtdy = dt / dy;
    /* Every row's x sweep, and then every column's y sweep, is independent of
     * the others: the timing build (built with OpenMP) shares them out over
     * host threads; the maxima are order-independent.  Without OpenMP the
     * pragmas are ignored and this is the plain loop. */
#pragma omp parallel
    {
        double *a = malloc(4 * (size_t)nmax * sizeof(double));
        double *o = malloc(3 * (size_t)nmax * sizeof(double));
        double *ah = a, *an = a + nmax, *at = a + 2 * nmax, *aB = a + 3 * nmax;
        double *oh = o, *on = o + nmax, *ot = o + 2 * nmax;
        double sxl = 0.0, syl = 0.0;
#pragma omp for schedule(static)
        for (int j = -2; j < ny + 2; j++) {
            for (int i = -2; i < nx + 2; i++) {
                size_t k = OIDX(p, i, j);
                ah[i + 2] = p->h[k]; an[i + 2] = p->hu[k]; at[i + 2] = p->hv[k]; aB[i + 2] = p->B[k];
            }
            double *gx = (xf && j >= 0 && j < ny) ? xf + 2 * (size_t)j * (nx + 1) : NULL;
            double s = sweep_1d_flux(g, drytol, nx, dtdx, ah, an, at, aB, oh, on, ot, gx);
            if (j >= 0 && j < ny) sxl = fmax(sxl, s);
            for (int i = 0; i < nx; i++) {
                size_t k = OIDX(p, i, j);
                p->h[k] = oh[i]; p->hu[k] = on[i]; p->hv[k] = ot[i];
            }
        }
#pragma omp for schedule(static)
        for (int i = 0; i < nx; i++) {
            for (int j = -2; j < ny + 2; j++) {
                size_t k = OIDX(p, i, j);
                ah[j + 2] = p->h[k]; an[j + 2] = p->hv[k]; at[j + 2] = p->hu[k]; aB[j + 2] = p->B[k];
            }
            double *gy = yf ? yf + 2 * (size_t)i * (ny + 1) : NULL;
            double s = sweep_1d_flux(g, drytol, ny, dtdy, ah, an, at, aB, oh, on, ot, gy);
            syl = fmax(syl, s);
            for (int j = 0; j < ny; j++) {
                size_t k = OIDX(p, i, j);
                p->h[k] = oh[j]; p->hv[k] = on[j]; p->hu[k] = ot[j];
            }
        }
#pragma omp critical
        {
            sx = fmax(sx, sxl);
            sy = fmax(sy, syl);
        }
        free(a); free(o);
    }
    *sx_out = sx; *sy_out = sy;
}

/* ------------------------------------------------------------------------
 * Unsplit wave propagation with transverse corrections (the scheme of the
 * original GeoClaw that the paper compares against, Sec. 5; corner transport
 * upwind of LeVeque 1997).  Reading: the fluctuations A+-dQ of every x-edge are
 * split in y by a Roe decomposition of the two cells above/below the cell they
 * enter, B-+ parts update the correction fluxes G of that cell's y-edges with
 * -(dt/dx)/2; likewise y-edge fluctuations split in x update F with
 * -(dt/dy)/2 (eigenstructure and dry cells: tsplit below).  As in GeoClaw's default, the second-order corrections are
 * propagated transversely too: the split fluctuations are A-dQ + 2F~ and
 * A+dQ - 2F~ (2F~ = sum_p c_p Z_p, the limited correction of the edge).
 * Accumulation order (fixed so two implementations agree bit for bit):
 *   G(i, j-1/2) = (((Gc - h*B-A+(i-1/2, j)) - h*B-A-(i+1/2, j))
 *                 - h*B+A+(i-1/2, j-1)) - h*B+A-(i+1/2, j-1),  h = dt/dx / 2
 *   F(i-1/2, j) = (((Fc - k*A-B+(i, j-1/2)) - k*A-B-(i, j+1/2))
 *                 - k*A+B+(i-1, j-1/2)) - k*A+B-(i-1, j+1/2),  k = dt/dy / 2
 * where A+- here are the second-order fluctuations above
 *   Q = (Q - dt/dx ((A+dQ_l + A-dQ_r) + (F_r - F_l))) - dt/dy ((B+dQ_b + B-dQ_t) + (G_t - G_b))
 * ------------------------------------------------------------------------ */

/* split fluctuation d (mass, n, t) along direction n between cells a (low) and
 * b (high) into the parts going towards a (minus) and towards b (plus), with
 * the eigenvectors of the Roe average of the two cells (both wet), or of the
 * wet cell alone (one dry cell whose bed lies below the wet surface).  Both
 * dry, or a dry cell whose bed reaches the wet surface (a wall): no transverse
 * wave. */
static void tsplit(double g, double drytol, const double d[3],
                   double ha, double na, double ta, double Ba, double hb, double nb, double tb, double Bb,
                   double minus[3], double plus[3])
{
    for (int m = 0; m < 3; m++) { minus[m] = 0.0; plus[m] = 0.0; }
    int wa = ha >= drytol, wb = hb >= drytol;
    double un, ut, c;
    if (wa && wb) {
        double sa = sqrt(ha), sb = sqrt(hb);
        un = (sa * (na / ha) + sb * (nb / hb)) / (sa + sb);
        ut = (sa * (ta / ha) + sb * (tb / hb)) / (sa + sb);
        c = sqrt(g * (0.5 * (ha + hb)));
    } else if (wa) {
        if (Bb >= ha + Ba) return;
        un = na / ha; ut = ta / ha; c = sqrt(g * ha);
    } else if (wb) {
        if (Ba >= hb + Bb) return;
        un = nb / hb; ut = tb / hb; c = sqrt(g * hb);
    } else {
        return;
    }
    double l1 = un - c, l2 = un, l3 = un + c;
    double b1 = ((un + c) * d[0] - d[1]) / (2.0 * c);
    double b3 = (d[1] - (un - c) * d[0]) / (2.0 * c);
    double b2 = d[2] - ut * d[0];
    double w1[3] = {b1, b1 * l1, b1 * ut}, w3[3] = {b3, b3 * l3, b3 * ut};
    double w2[3] = {0.0, 0.0, b2};
    double m1 = fmin(l1, 0.0), m2 = fmin(l2, 0.0), m3 = fmin(l3, 0.0);
    double p1 = fmax(l1, 0.0), p2 = fmax(l2, 0.0), p3 = fmax(l3, 0.0);
    for (int m = 0; m < 3; m++) {
        minus[m] = (m1 * w1[m] + m2 * w2[m]) + m3 * w3[m];
        plus[m] = (p1 * w1[m] + p2 * w2[m]) + p3 * w3[m];
    }
}

typedef struct EdgeTerms {
    double am[3], ap[3], F[3];   /* fluctuations and limited correction, edge frame (mass, normal, transverse) */
    double am2[3], ap2[3];       /* A-dQ + 2F~, A+dQ - 2F~: what is split transversely */
    double s0, s2;
} EdgeTerms;

/* edge terms of one 1D row of n interior cells (arrays of n+4 with 2 ghosts):
 * out[e] for edges e = 0..n (fluctuations, limited correction) */
static void row_terms(double g, double drytol, int n, double dtdx,
                      const double *h, const double *hn, const double *ht, const double *B, EdgeTerms *out)
{
    ora_rp *rp = (ora_rp *)malloc((size_t)(n + 3) * sizeof *rp);
    for (int e = -1; e <= n + 1; e++) {
        int cl = e - 1 + 2, cr = e + 2;
        ora_riemann(g, drytol, h[cl], hn[cl], ht[cl], B[cl], h[cr], hn[cr], ht[cr], B[cr], &rp[e + 1]);
    }
    for (int e = 0; e <= n; e++) {
        const ora_rp *r = &rp[e + 1];
        EdgeTerms *o = &out[e];
        for (int m = 0; m < 3; m++) {
            o->am[m] = (w_left(r->s[0]) * r->Z[0][m] + w_left(r->s[1]) * r->Z[1][m]) + w_left(r->s[2]) * r->Z[2][m];
            o->ap[m] = (w_right(r->s[0]) * r->Z[0][m] + w_right(r->s[1]) * r->Z[1][m]) + w_right(r->s[2]) * r->Z[2][m];
        }
        if (r->wallR) { o->ap[0] = 0.0; o->ap[1] = 0.0; o->ap[2] = 0.0; }
        if (r->wallL) { o->am[0] = 0.0; o->am[1] = 0.0; o->am[2] = 0.0; }
        double c[3] = {0.0, 0.0, 0.0};
        if (!r->wallL && !r->wallR) {
            for (int p = 0; p < 3; p++) {
                const double *Zi = r->Z[p];
                double dii = (Zi[0] * Zi[0] + Zi[1] * Zi[1]) + Zi[2] * Zi[2];
                double phi = 0.0;
                if (dii != 0.0) {
                    int I = r->s[p] >= 0.0 ? e - 1 : e + 1;
                    const double *ZI = rp[I + 1].Z[p];
                    double dIi = (ZI[0] * Zi[0] + ZI[1] * Zi[1]) + ZI[2] * Zi[2];
                    phi = ora_mc_limiter(dIi / dii);
                }
                double s = r->s[p];
                double cp = (1.0 - dtdx * fabs(s)) * phi;
                if (s < 0.0) cp = -cp;
                else if (s == 0.0) cp = 0.0;
                c[p] = cp;
            }
        }
        for (int m = 0; m < 3; m++) {
            double cq = (c[0] * r->Z[0][m] + c[1] * r->Z[1][m]) + c[2] * r->Z[2][m];
            o->F[m] = 0.5 * cq;
            o->am2[m] = o->am[m] + cq;
            o->ap2[m] = o->ap[m] - cq;
        }
        o->s0 = r->s[0];
        o->s2 = r->s[2];
    }
    free(rp);
}

void ora_step_patch_unsplit(OPatch *p, double g, double drytol, double dt, double dx, double dy,
                            double *sx_out, double *sy_out)
{
    int nx = p->nx, ny = p->ny;
    double dtdx = dt / dx, dtdy = dt / dy;
    int nmax = (nx > ny ? nx : ny) + 4;
    double *a = malloc(4 * (size_t)nmax * sizeof(double));
    double *ah = a, *an = a + nmax, *at = a + 2 * nmax, *aB = a + 3 * nmax;
    /* x-edge terms X[j+1][e] for rows j = -1..ny, edges e = 0..nx (storage frame: mass, hu, hv) */
    EdgeTerms *X = malloc((size_t)(ny + 2) * (nx + 1) * sizeof *X);
    EdgeTerms *Y = malloc((size_t)(nx + 2) * (ny + 1) * sizeof *Y);   /* Y[i+1][e], frame (mass, hv, hu) */
    EdgeTerms *tmp = malloc((size_t)(nmax + 1) * sizeof *tmp);
    double sx = 0.0, sy = 0.0;
    for (int j = -1; j <= ny; j++) {
        for (int i = -2; i < nx + 2; i++) {
            size_t k = OIDX(p, i, j);
            ah[i + 2] = p->h[k]; an[i + 2] = p->hu[k]; at[i + 2] = p->hv[k]; aB[i + 2] = p->B[k];
        }
        row_terms(g, drytol, nx, dtdx, ah, an, at, aB, tmp);
        for (int e = 0; e <= nx; e++) {
            X[(size_t)(j + 1) * (nx + 1) + e] = tmp[e];
            if (j >= 0 && j < ny) sx = fmax(sx, fmax(-tmp[e].s0, tmp[e].s2));
        }
    }
    for (int i = -1; i <= nx; i++) {
        for (int j = -2; j < ny + 2; j++) {
            size_t k = OIDX(p, i, j);
            ah[j + 2] = p->h[k]; an[j + 2] = p->hv[k]; at[j + 2] = p->hu[k]; aB[j + 2] = p->B[k];
        }
        row_terms(g, drytol, ny, dtdy, ah, an, at, aB, tmp);
        for (int e = 0; e <= ny; e++) {
            Y[(size_t)(i + 1) * (ny + 1) + e] = tmp[e];
            if (i >= 0 && i < nx) sy = fmax(sy, fmax(-tmp[e].s0, tmp[e].s2));
        }
    }
#define XT(j, e) X[(size_t)((j) + 1) * (nx + 1) + (e)]
#define YT(i, e) Y[(size_t)((i) + 1) * (ny + 1) + (e)]
#define H(i, j) p->h[OIDX(p, i, j)]
#define HU(i, j) p->hu[OIDX(p, i, j)]
#define HV(i, j) p->hv[OIDX(p, i, j)]
#define BB(i, j) p->B[OIDX(p, i, j)]
    double hx = 0.5 * dtdx, hy = 0.5 * dtdy;
    /* x-edge fluctuation of edge (e, j) split in y for the cell column c it enters: returns B- and B+
     * parts in storage frame (mass, hu, hv); frame for tsplit: (mass, hv, hu) */
#define XSPLIT(fl, c, j, lo, hi_)                                                              \
    do {                                                                                       \
        double d_[3] = {(fl)[0], (fl)[2], (fl)[1]}, mi_[3], pl_[3];                            \
        tsplit(g, drytol, d_, H(c, (j) - 1), HV(c, (j) - 1), HU(c, (j) - 1), BB(c, (j) - 1), H(c, j), HV(c, j), HU(c, j), BB(c, j), mi_, pl_); \
        lo[0] = mi_[0]; lo[1] = mi_[2]; lo[2] = mi_[1];                                        \
        tsplit(g, drytol, d_, H(c, j), HV(c, j), HU(c, j), BB(c, j), H(c, (j) + 1), HV(c, (j) + 1), HU(c, (j) + 1), BB(c, (j) + 1), mi_, pl_); \
        hi_[0] = pl_[0]; hi_[1] = pl_[2]; hi_[2] = pl_[1];                                     \
    } while (0)
    /* G(i, e) for y-edges e = 0..ny of columns i = 0..nx-1, in storage frame (mass, hu, hv) */
    double (*G)[3] = malloc((size_t)nx * (ny + 1) * sizeof *G);
    for (int i = 0; i < nx; i++)
        for (int e = 0; e <= ny; e++) {
            const EdgeTerms *yt = &YT(i, e);
            double gv[3] = {yt->F[0], yt->F[2], yt->F[1]};   /* to storage frame */
            int j = e;   /* y-edge between rows j-1 and j */
            double lo[3], hi[3];
            /* (a) x-edge (i-1/2, j): A+ into (i, j), down part */
            XSPLIT(XT(j, i).ap2, i, j, lo, hi);
            for (int m = 0; m < 3; m++) gv[m] = gv[m] - hx * lo[m];
            /* (b) x-edge (i+1/2, j): A- into (i, j), down part */
            XSPLIT(XT(j, i + 1).am2, i, j, lo, hi);
            for (int m = 0; m < 3; m++) gv[m] = gv[m] - hx * lo[m];
            /* (c) x-edge (i-1/2, j-1): A+ into (i, j-1), up part */
            XSPLIT(XT(j - 1, i).ap2, i, j - 1, lo, hi);
            for (int m = 0; m < 3; m++) gv[m] = gv[m] - hx * hi[m];
            /* (d) x-edge (i+1/2, j-1): A- into (i, j-1), up part */
            XSPLIT(XT(j - 1, i + 1).am2, i, j - 1, lo, hi);
            for (int m = 0; m < 3; m++) gv[m] = gv[m] - hx * hi[m];
            G[(size_t)i * (ny + 1) + e][0] = gv[0];
            G[(size_t)i * (ny + 1) + e][1] = gv[1];
            G[(size_t)i * (ny + 1) + e][2] = gv[2];
        }
    /* y-edge fluctuation split in x, frame for tsplit (mass, hu, hv) */
#define YSPLIT(fl, c, r, lo, hi_)                                                              \
    do {                                                                                       \
        double d_[3] = {(fl)[0], (fl)[2], (fl)[1]}, mi_[3], pl_[3];                            \
        tsplit(g, drytol, d_, H((c) - 1, r), HU((c) - 1, r), HV((c) - 1, r), BB((c) - 1, r), H(c, r), HU(c, r), HV(c, r), BB(c, r), mi_, pl_); \
        lo[0] = mi_[0]; lo[1] = mi_[1]; lo[2] = mi_[2];                                        \
        tsplit(g, drytol, d_, H(c, r), HU(c, r), HV(c, r), BB(c, r), H((c) + 1, r), HU((c) + 1, r), HV((c) + 1, r), BB((c) + 1, r), mi_, pl_); \
        hi_[0] = pl_[0]; hi_[1] = pl_[1]; hi_[2] = pl_[2];                                     \
    } while (0)
    double (*Fx)[3] = malloc((size_t)ny * (nx + 1) * sizeof *Fx);
    for (int j = 0; j < ny; j++)
        for (int e = 0; e <= nx; e++) {
            const EdgeTerms *xt = &XT(j, e);
            double fv[3] = {xt->F[0], xt->F[1], xt->F[2]};
            int i = e;   /* x-edge between columns i-1 and i */
            double lo[3], hi[3];
            /* (a) y-edge (i, j-1/2): B+ into (i, j), left part */
            YSPLIT(YT(i, j).ap2, i, j, lo, hi);
            for (int m = 0; m < 3; m++) fv[m] = fv[m] - hy * lo[m];
            /* (b) y-edge (i, j+1/2): B- into (i, j), left part */
            YSPLIT(YT(i, j + 1).am2, i, j, lo, hi);
            for (int m = 0; m < 3; m++) fv[m] = fv[m] - hy * lo[m];
            /* (c) y-edge (i-1, j-1/2): B+ into (i-1, j), right part */
            YSPLIT(YT(i - 1, j).ap2, i - 1, j, lo, hi);
            for (int m = 0; m < 3; m++) fv[m] = fv[m] - hy * hi[m];
            /* (d) y-edge (i-1, j+1/2): B- into (i-1, j), right part */
            YSPLIT(YT(i - 1, j + 1).am2, i - 1, j, lo, hi);
            for (int m = 0; m < 3; m++) fv[m] = fv[m] - hy * hi[m];
            Fx[(size_t)j * (nx + 1) + e][0] = fv[0];
            Fx[(size_t)j * (nx + 1) + e][1] = fv[1];
            Fx[(size_t)j * (nx + 1) + e][2] = fv[2];
        }
    /* update (new values to temporary arrays, then copy) */
    double *qn = malloc(3 * (size_t)nx * ny * sizeof(double));
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            const EdgeTerms *xl = &XT(j, i), *xr = &XT(j, i + 1);
            const EdgeTerms *yb = &YT(i, j), *ytp = &YT(i, j + 1);
            const double *Fl = Fx[(size_t)j * (nx + 1) + i], *Fr = Fx[(size_t)j * (nx + 1) + i + 1];
            const double *Gb = G[(size_t)i * (ny + 1) + j], *Gt = G[(size_t)i * (ny + 1) + j + 1];
            double q[3] = {H(i, j), HU(i, j), HV(i, j)};
            for (int m = 0; m < 3; m++) {
                int my = m == 0 ? 0 : (m == 1 ? 2 : 1);   /* storage component m in the y-edge frame */
                double ux = (xl->ap[m] + xr->am[m]) + (Fr[m] - Fl[m]);
                double uy = (yb->ap[my] + ytp->am[my]) + (Gt[m] - Gb[m]);
                q[m] = (q[m] - dtdx * ux) - dtdy * uy;
            }
            if (q[0] < 0.0) { ora_neg_clips++; q[0] = 0.0; }
            if (q[0] < drytol) { q[1] = 0.0; q[2] = 0.0; }
            for (int m = 0; m < 3; m++) qn[(size_t)m * nx * ny + (size_t)j * nx + i] = q[m];
        }
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            size_t k = OIDX(p, i, j), d = (size_t)j * nx + i;
            p->h[k] = qn[d];
            p->hu[k] = qn[(size_t)nx * ny + d];
            p->hv[k] = qn[2 * (size_t)nx * ny + d];
        }
#undef XT
#undef YT
#undef H
#undef HU
#undef HV
#undef BB
#undef XSPLIT
#undef YSPLIT
    free(qn); free(G); free(Fx); free(X); free(Y); free(tmp); free(a);
    *sx_out = sx; *sy_out = sy;
}

/* Manning friction (Sec. 2.1: the momentum equations carry -D hu and -D hv).
 * Reading: the printed D = n^2 g h^(-7/3) sqrt(u^2 + v^2) is not
 * dimensionally consistent with -D hu; with the momentum magnitude,
 * D = n^2 g h^(-7/3) sqrt((hu)^2 + (hv)^2) = g n^2 |u| / h^(4/3), it is the
 * Manning law.  Applied as a pointwise step after each wave-propagation step
 * of a level, implicit in the momentum with D from the updated state:
 * hu <- hu / (1 + dt D), hv <- hv / (1 + dt D), on wet interior cells. */
void ora_friction_patch(OPatch *p, double g, double drytol, double n, double dt)
{
    const double coef = (n * n) * g;
    for (int j = 0; j < p->ny; j++)
        for (int i = 0; i < p->nx; i++) {
            size_t k = OIDX(p, i, j);
            double h = p->h[k];
            if (!(h >= drytol)) continue;
            double hu = p->hu[k], hv = p->hv[k];
            double D = (coef * pow(h, -7.0 / 3.0)) * sqrt(hu * hu + hv * hv);
            double f = 1.0 + dt * D;
            p->hu[k] = hu / f;
            p->hv[k] = hv / f;
        }
}
