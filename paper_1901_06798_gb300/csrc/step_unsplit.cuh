// step_unsplit.cuh -- one unsplit wave-propagation step with transverse
// corrections (corner transport upwind, LeVeque 1997) of every patch of a
// level in one launch: the scheme of the original GeoClaw that Sec. 5 compares
// the dimensionally split GPU scheme against.
//
// Update of cell (i, j), all terms from Q^n:
//   Q -= dt/dx ((A+dQ_{i-1/2} + A-dQ_{i+1/2}) + (F_{i+1/2} - F_{i-1/2}))
//   Q -= dt/dy ((B+dQ_{j-1/2} + B-dQ_{j+1/2}) + (G_{j+1/2} - G_{j-1/2}))
// where F and G are the limited correction fluxes of the edge (Sec. 2.2 Eq.
// wave_propagation_2nd_order) minus one half dt/dy (dt/dx) times the
// transverse splits of the neighbouring edges' fluctuations:
//   * each x-edge fluctuation A-+dQ + -2F~ (the second-order correction is
//     propagated too) entering a cell is split by the Roe eigenvectors in y of
//     that cell and its neighbour above / below into up- and down-going parts,
//     which enter G of the y-edge between the two;
//   * symmetrically for y-edge fluctuations and F.
// Every transverse contribution to the flux of an edge uses the
// eigenstructure of the two cells that share that edge, so the stencil stays
// within the 2-cell ghost ring of the split scheme.
//
// Per CTA: a strip of W = NT - 4 columns of one patch and a segment of rows;
// thread t owns ring column t (patch column x0 - 2 + t).  The CTA marches
// down the rows; at iteration k (patch row r = y0 - 2 + k) it
//   1. solves the x-edge Riemann problems of row r and limits them
//      (shared memory, as the split kernel), keeping A-+dQ, F~ and the
//      second-order fluctuations of rows r-2 .. r in a shared ring;
//   2. solves the y-edge problem of edge r of its column and limits edge r-1
//      (registers: the column's waves stay with its thread);
//   3. forms G of y-edge r-1 of its column from the x-terms of rows r-2, r-1;
//   4. forms F of x-edge t of row r-2 from the y-terms of columns t-1, t;
//   5. updates cell (t, r-2).
// Four barriers per row.  The arithmetic follows the FP64 oracle operation by
// operation (same association, same order of the four transverse terms); the
// FP64 instantiation is compiled without contraction so the two agree to the
// last bit.  The FP32 perturbation form has its own kernel with the same
// pipeline and fewer shared-memory terms (step_unsplit_f32.cuh).
#pragma once
#include "step_kernel.cuh"

namespace tsu {

// Eigenstructure of a transverse pair (a low, b high) in the split
// direction's roles: both wet -> Roe average; one wet -> the wet cell alone,
// unless the dry cell's bed reaches the wet surface (a wall: no transverse
// wave); both dry -> none.
template <typename T> struct TEig {
    T un, ut, c;
    bool on;
};

template <typename T>
__device__ __forceinline__ TEig<T> teig(T g, T ha, T ua, T va, T ca, T sqa, T Ba, bool wa,
                                        T hb, T ub, T vb, T cb, T sqb, T Bb, bool wb)
{
    TEig<T> e;
    e.un = T(0); e.ut = T(0); e.c = T(0); e.on = false;
    if (wa && wb) {
        e.un = (sqa * ua + sqb * ub) / (sqa + sqb);
        e.ut = (sqa * va + sqb * vb) / (sqa + sqb);
        e.c = dsqrt<T>(g * (T(0.5) * (ha + hb)));
        e.on = true;
    } else if (wa) {
        if (!(Bb >= ha + Ba)) { e.un = ua; e.ut = va; e.c = ca; e.on = true; }
    } else if (wb) {
        if (!(Ba >= hb + Bb)) { e.un = ub; e.ut = vb; e.c = cb; e.on = true; }
    }
    return e;
}

// Part of fluctuation d (frame: mass, normal, transverse) carried by the
// waves going to the high side (PLUS) or the low side.
template <typename T, bool PLUS>
__device__ __forceinline__ void tpart(const TEig<T> &e, const T (&d)[3], T (&out)[3])
{
    if (!e.on) { out[0] = T(0); out[1] = T(0); out[2] = T(0); return; }
    const T l1 = e.un - e.c, l2 = e.un, l3 = e.un + e.c;
    const T b1 = ((e.un + e.c) * d[0] - d[1]) / (T(2) * e.c);
    const T b3 = (d[1] - (e.un - e.c) * d[0]) / (T(2) * e.c);
    const T b2 = d[2] - e.ut * d[0];
    const T w1[3] = {b1, b1 * l1, b1 * e.ut}, w3[3] = {b3, b3 * l3, b3 * e.ut};
    const T w2[3] = {T(0), T(0), b2};
    const T k1 = PLUS ? dmax<T>(l1, T(0)) : dmin<T>(l1, T(0));
    const T k2 = PLUS ? dmax<T>(l2, T(0)) : dmin<T>(l2, T(0));
    const T k3 = PLUS ? dmax<T>(l3, T(0)) : dmin<T>(l3, T(0));
#pragma unroll
    for (int m = 0; m < 3; m++) out[m] = (k1 * w1[m] + k2 * w2[m]) + k3 * w3[m];
}

// Fluctuations, limited correction and the second-order fluctuations
// A-dQ + 2F~, A+dQ - 2F~ of one edge.
template <typename T>
__device__ __forceinline__ void limit2(const Wave<T> &r, const T (&ZI)[3][3], T dtdx, T (&am)[3], T (&ap)[3],
                                       T (&F)[3], T (&am2)[3], T (&ap2)[3])
{
    T wl0 = wleft<T>(r.s[0]), wl1 = wleft<T>(r.s[1]), wl2 = wleft<T>(r.s[2]);
    T wr0 = wright<T>(r.s[0]), wr1 = wright<T>(r.s[1]), wr2 = wright<T>(r.s[2]);
#pragma unroll
    for (int m = 0; m < 3; m++) {
        am[m] = (wl0 * r.Z[0][m] + wl1 * r.Z[1][m]) + wl2 * r.Z[2][m];
        ap[m] = (wr0 * r.Z[0][m] + wr1 * r.Z[1][m]) + wr2 * r.Z[2][m];
    }
    if (r.wall == 2) { ap[0] = T(0); ap[1] = T(0); ap[2] = T(0); }
    if (r.wall == 1) { am[0] = T(0); am[1] = T(0); am[2] = T(0); }
    T c[3] = {T(0), T(0), T(0)};
    if (r.wall == 0) {
#pragma unroll
        for (int p = 0; p < 3; p++) {
            const T *Zi = r.Z[p];
            T dii = (Zi[0] * Zi[0] + Zi[1] * Zi[1]) + Zi[2] * Zi[2];
            T phi = T(0);
            if (dii != T(0)) {
                T dIi = (ZI[p][0] * Zi[0] + ZI[p][1] * Zi[1]) + ZI[p][2] * Zi[2];
                phi = mc_limiter<T>(dIi / dii);
            }
            T s = r.s[p];
            T cp = (T(1) - dtdx * dabs<T>(s)) * phi;
            if (s < T(0)) cp = -cp;
            else if (s == T(0)) cp = T(0);
            c[p] = cp;
        }
    }
#pragma unroll
    for (int m = 0; m < 3; m++) {
        T cq = (c[0] * r.Z[0][m] + c[1] * r.Z[1][m]) + c[2] * r.Z[2][m];
        F[m] = T(0.5) * cq;
        am2[m] = am[m] + cq;
        ap2[m] = ap[m] - cq;
    }
}

// shared-memory layout of the unsplit kernel, in elements of T
template <int NT, int RING> struct UnsplitSmem {
    static constexpr int ring = 0;                    // [RING][4][NT] q0, hu, hv, B
    static constexpr int der = ring + RING * 4 * NT;  // [RING][4][NT] u, v, c, sqrt(h) (x roles)
    static constexpr int z = der + RING * 4 * NT;     // [9][NT] x-edge f-waves of the current row
    static constexpr int xt = z + 9 * NT;             // [3][15][NT] x-edge am, ap, F, am2, ap2 by row mod 3
    static constexpr int ys = xt + 3 * 15 * NT;       // [2][6][NT] y-edge am2, ap2 (y frame) by edge parity
    static constexpr int fx = ys + 2 * 6 * NT;        // [3][NT] transverse-corrected F of x-edge t
    static constexpr int red = fx + 3 * NT;           // [2][NT / 32] speed maxima
    static constexpr int total = red + 2 * (NT / 32);
};

template <typename T> __device__ __forceinline__ T dt_over(const StepArgs &a, int scen, bool ydir);
template <> __device__ __forceinline__ double dt_over<double>(const StepArgs &a, int scen, bool ydir)
{
    const double dt = a.dt1[scen] / a.R;
    return ydir ? dt / a.dy : dt / a.dx;
}
template <> __device__ __forceinline__ float dt_over<float>(const StepArgs &a, int scen, bool ydir)
{
    return a.dt1f[scen] * (ydir ? a.rdy : a.rdx);
}

template <typename T> __device__ __forceinline__ T dt_level(const StepArgs &a, int scen);
template <> __device__ __forceinline__ double dt_level<double>(const StepArgs &a, int scen) { return a.dt1[scen] / a.R; }
template <> __device__ __forceinline__ float dt_level<float>(const StepArgs &a, int scen) { return a.dt1f[scen] * a.rR; }

template <typename T, bool PERT, int NT, int RING>
__global__ void __launch_bounds__(NT) step_unsplit_kernel(StepArgs a)
{
    static_assert(RING >= 5, "rows r-2 .. r are read while rows r+1, r+2 are in flight");
    using S = UnsplitSmem<NT, RING>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    auto RG = [&](int slot, int f, int t) -> T & { return sm[S::ring + (slot * 4 + f) * NT + t]; };
    auto DV = [&](int slot, int f, int t) -> T & { return sm[S::der + (slot * 4 + f) * NT + t]; };
    auto ZS = [&](int pm, int t) -> T & { return sm[S::z + pm * NT + t]; };
    auto XT = [&](int slot, int f, int t) -> T & { return sm[S::xt + (slot * 15 + f) * NT + t]; };
    auto YS = [&](int slot, int f, int t) -> T & { return sm[S::ys + (slot * 6 + f) * NT + t]; };
    auto FX = [&](int m, int t) -> T & { return sm[S::fx + m * NT + t]; };
    T *red = sm + S::red;

    const StepItem it = a.items[blockIdx.x];
    if (it.w > NT - 4 || it.w < 1 || it.h < 1) return;   // not a work item of this launch shape
    const PatchDesc P = a.descs[it.patch];
    if (a.gate != nullptr && a.gate[P.scen] == 0) return;   // not retaken (uniform over the CTA)
    const int t = threadIdx.x;
    const int cur = a.cur;
    T *base = reinterpret_cast<T *>(a.arena) + P.off;
    const T *qin0 = base + (long long)(cur * 3 + 0) * P.fs;
    const T *qin1 = base + (long long)(cur * 3 + 1) * P.fs;
    const T *qin2 = base + (long long)(cur * 3 + 2) * P.fs;
    const T *Bg = base + 6LL * P.fs;
    T *qo0 = base + (long long)((1 - cur) * 3 + 0) * P.fs;
    T *qo1 = base + (long long)((1 - cur) * 3 + 1) * P.fs;
    T *qo2 = base + (long long)((1 - cur) * 3 + 2) * P.fs;

    const T dtdx = dt_over<T>(a, P.scen, false), dtdy = dt_over<T>(a, P.scen, true);
    const T hx = T(0.5) * dtdx, hy = T(0.5) * dtdy;
    const T g = PERT ? (T)a.gf : (T)a.g;
    const T drytol = PERT ? (T)a.drytolf : (T)a.drytol;
    const int x0 = it.x0, y0 = it.y0, w = it.w, h = it.h;
    const int pitch = P.pitch;
    const int nrows = h + 4;
    const bool loader = t < w + 4;
    const long long colofs = (long long)(x0 + t);

    auto prefetch = [&](int k) {
        if (k < nrows && loader) {
            const int slot = k % RING;
            const long long gi = (long long)(y0 + k) * pitch + colofs;
            cp_async_elem(&RG(slot, 0, t), qin0 + gi, sizeof(T));
            cp_async_elem(&RG(slot, 1, t), qin1 + gi, sizeof(T));
            cp_async_elem(&RG(slot, 2, t), qin2 + gi, sizeof(T));
            cp_async_elem(&RG(slot, 3, t), Bg + gi, sizeof(T));
        }
        cp_async_commit();
    };
    // derived values (x roles) of this thread's ring cell of row k
    auto derive_own = [&](int k) {
        if (k < nrows && loader) {
            const int slot = k % RING;
            Cell<T> z;
            z.q0 = RG(slot, 0, t); z.hn = RG(slot, 1, t); z.ht = RG(slot, 2, t); z.B = RG(slot, 3, t);
            derive<T, PERT>(z, g, drytol);
            DV(slot, 0, t) = z.u; DV(slot, 1, t) = z.v; DV(slot, 2, t) = z.c; DV(slot, 3, t) = z.sq;
        }
    };
    // ring cell c of row k in x roles (hn = hu) or y roles (hn = hv)
    auto cell = [&](int k, int c, bool yroles) {
        const int slot = k % RING;
        Cell<T> z;
        z.q0 = RG(slot, 0, c);
        z.hn = RG(slot, yroles ? 2 : 1, c);
        z.ht = RG(slot, yroles ? 1 : 2, c);
        z.B = RG(slot, 3, c);
        z.h = PERT ? z.q0 - z.B : z.q0;
        z.wet = z.h >= drytol;
        z.u = DV(slot, yroles ? 1 : 0, c);
        z.v = DV(slot, yroles ? 0 : 1, c);
        z.c = DV(slot, 2, c);
        z.sq = DV(slot, 3, c);
        return z;
    };

    prefetch(0);
    prefetch(1);
    cp_async_wait<1>();
    derive_own(0);

    const bool xsolve = t >= 1 && t < w + 4;   // x-edge between ring cells t-1 and t
    const bool xlim = t >= 2 && t < w + 3;     // x-edges x0 .. x0 + w
    const bool ycol = t >= 1 && t < w + 3;     // columns x0 - 1 .. x0 + w
    const bool out = t >= 2 && t < w + 2;      // columns x0 .. x0 + w - 1

    Wave<T> yold, ymid;
    T yap_prev[3] = {T(0), T(0), T(0)};
    T G_prev[3] = {T(0), T(0), T(0)};
    T smx = T(0), smy = T(0);

    for (int k = 0; k < nrows; k++) {
        __syncthreads();   // row k (ring + derived) visible; iteration k-1 finished everywhere
        prefetch(k + 2);
        const int r = y0 - 2 + k;
        const bool rowint = r >= y0 && r < y0 + h;

        // ---- 1a. x-edge Riemann problem of row r between ring cells t-1 and t
        Wave<T> xw;
        if (xsolve) {
            Cell<T> cl = cell(k, t - 1, false), cr = cell(k, t, false);
            riemann<T, PERT>(g, cl, cr, xw);
#pragma unroll
            for (int p = 0; p < 3; p++)
#pragma unroll
                for (int m = 0; m < 3; m++) ZS(p * 3 + m, t) = xw.Z[p][m];
        }

        // ---- 2. y-edge r of this column; limit edge r-1
        T yam[3], yap[3], yF[3], yam2[3], yap2[3];
        bool yready = false;
        if (ycol && k >= 1) {
            Cell<T> lo = cell(k - 1, t, true), hi = cell(k, t, true);
            Wave<T> ynew;
            riemann<T, PERT>(g, lo, hi, ynew);
            if (k >= 3) {
                T ZI[3][3];
#pragma unroll
                for (int p = 0; p < 3; p++)
#pragma unroll
                    for (int m = 0; m < 3; m++) ZI[p][m] = ymid.s[p] >= T(0) ? yold.Z[p][m] : ynew.Z[p][m];
                limit2<T>(ymid, ZI, dtdy, yam, yap, yF, yam2, yap2);
                yready = true;
                const int e = r - 1;
                if (out && e >= y0 && e <= y0 + h) smy = dmax<T>(smy, dmax<T>(-ymid.s[0], ymid.s[2]));
#pragma unroll
                for (int m = 0; m < 3; m++) { YS(k & 1, m, t) = yam2[m]; YS(k & 1, 3 + m, t) = yap2[m]; }
            }
            yold = ymid;
            ymid = ynew;
        }

        // ---- 3. G of y-edge r-1 of this column (x-terms of rows r-2 and r-1)
        T Gc[3] = {T(0), T(0), T(0)};
        if (out && yready) {
            const Cell<T> ca = cell(k - 2, t, true), cb = cell(k - 1, t, true);
            const TEig<T> ev = teig<T>(g, ca.h, ca.u, ca.v, ca.c, ca.sq, ca.B, ca.wet,
                                       cb.h, cb.u, cb.v, cb.c, cb.sq, cb.B, cb.wet);
            const int se = (k - 1) % 3, sb = (k - 2) % 3;   // rows r-1 (edge's upper cell) and r-2
            Gc[0] = yF[0]; Gc[1] = yF[2]; Gc[2] = yF[1];    // y frame -> storage frame
            T d[3], part[3];
            // (a) A+dQ entering (t, r-1) through its left edge: down-going part
            d[0] = XT(se, 9 + 3 + 0, t); d[1] = XT(se, 9 + 3 + 2, t); d[2] = XT(se, 9 + 3 + 1, t);
            tpart<T, false>(ev, d, part);
            Gc[0] = Gc[0] - hx * part[0]; Gc[1] = Gc[1] - hx * part[2]; Gc[2] = Gc[2] - hx * part[1];
            // (b) A-dQ entering (t, r-1) through its right edge: down-going part
            d[0] = XT(se, 9 + 0, t + 1); d[1] = XT(se, 9 + 2, t + 1); d[2] = XT(se, 9 + 1, t + 1);
            tpart<T, false>(ev, d, part);
            Gc[0] = Gc[0] - hx * part[0]; Gc[1] = Gc[1] - hx * part[2]; Gc[2] = Gc[2] - hx * part[1];
            // (c) A+dQ entering (t, r-2) through its left edge: up-going part
            d[0] = XT(sb, 9 + 3 + 0, t); d[1] = XT(sb, 9 + 3 + 2, t); d[2] = XT(sb, 9 + 3 + 1, t);
            tpart<T, true>(ev, d, part);
            Gc[0] = Gc[0] - hx * part[0]; Gc[1] = Gc[1] - hx * part[2]; Gc[2] = Gc[2] - hx * part[1];
            // (d) A-dQ entering (t, r-2) through its right edge: up-going part
            d[0] = XT(sb, 9 + 0, t + 1); d[1] = XT(sb, 9 + 2, t + 1); d[2] = XT(sb, 9 + 1, t + 1);
            tpart<T, true>(ev, d, part);
            Gc[0] = Gc[0] - hx * part[0]; Gc[1] = Gc[1] - hx * part[2]; Gc[2] = Gc[2] - hx * part[1];
        }
        __syncthreads();   // x-waves of row r and y-terms of edge r-1 published

        // ---- 1b. limit x-edges of row r
        if (xlim) {
            T ZI[3][3];
#pragma unroll
            for (int p = 0; p < 3; p++) {
                const int nb = xw.s[p] >= T(0) ? t - 1 : t + 1;
#pragma unroll
                for (int m = 0; m < 3; m++) ZI[p][m] = ZS(p * 3 + m, nb);
            }
            T am[3], ap[3], F[3], am2[3], ap2[3];
            limit2<T>(xw, ZI, dtdx, am, ap, F, am2, ap2);
            const int sx = k % 3;
#pragma unroll
            for (int m = 0; m < 3; m++) {
                XT(sx, m, t) = am[m]; XT(sx, 3 + m, t) = ap[m]; XT(sx, 6 + m, t) = F[m];
                XT(sx, 9 + m, t) = am2[m]; XT(sx, 12 + m, t) = ap2[m];
            }
            if (rowint) smx = dmax<T>(smx, dmax<T>(-xw.s[0], xw.s[2]));
        }

        // ---- 4. F of x-edge t in row r-2 (y-terms of columns t-1, t at edges r-2, r-1)
        if (xlim && k >= 4) {
            const Cell<T> ca = cell(k - 2, t - 1, false), cb = cell(k - 2, t, false);
            const TEig<T> ev = teig<T>(g, ca.h, ca.u, ca.v, ca.c, ca.sq, ca.B, ca.wet,
                                       cb.h, cb.u, cb.v, cb.c, cb.sq, cb.B, cb.wet);
            const int sj = (k - 2) % 3, yb = (k - 1) & 1, yt = k & 1;   // row r-2; edges r-2, r-1
            T Fc[3] = {XT(sj, 6 + 0, t), XT(sj, 6 + 1, t), XT(sj, 6 + 2, t)};
            T d[3], part[3];
            // (a) B+dQ entering (t, r-2) from below: left-going part
            d[0] = YS(yb, 3 + 0, t); d[1] = YS(yb, 3 + 2, t); d[2] = YS(yb, 3 + 1, t);
            tpart<T, false>(ev, d, part);
#pragma unroll
            for (int m = 0; m < 3; m++) Fc[m] = Fc[m] - hy * part[m];
            // (b) B-dQ entering (t, r-2) from above: left-going part
            d[0] = YS(yt, 0, t); d[1] = YS(yt, 2, t); d[2] = YS(yt, 1, t);
            tpart<T, false>(ev, d, part);
#pragma unroll
            for (int m = 0; m < 3; m++) Fc[m] = Fc[m] - hy * part[m];
            // (c) B+dQ entering (t-1, r-2) from below: right-going part
            d[0] = YS(yb, 3 + 0, t - 1); d[1] = YS(yb, 3 + 2, t - 1); d[2] = YS(yb, 3 + 1, t - 1);
            tpart<T, true>(ev, d, part);
#pragma unroll
            for (int m = 0; m < 3; m++) Fc[m] = Fc[m] - hy * part[m];
            // (d) B-dQ entering (t-1, r-2) from above: right-going part
            d[0] = YS(yt, 0, t - 1); d[1] = YS(yt, 2, t - 1); d[2] = YS(yt, 1, t - 1);
            tpart<T, true>(ev, d, part);
#pragma unroll
            for (int m = 0; m < 3; m++) Fc[m] = Fc[m] - hy * part[m];
#pragma unroll
            for (int m = 0; m < 3; m++) FX(m, t) = Fc[m];
        }
        __syncthreads();   // F of row r-2 published

        // ---- 5. update cell (t, r-2)
        if (out && k >= 4) {
            const int j = r - 2;
            const int sj = (k - 2) % 3;
            const int slot = (k - 2) % RING;
            T q[3] = {RG(slot, 0, t), RG(slot, 1, t), RG(slot, 2, t)};
            const T Bc = RG(slot, 3, t);
#pragma unroll
            for (int m = 0; m < 3; m++) {
                const int my = m == 0 ? 0 : (m == 1 ? 2 : 1);
                const T ux = (XT(sj, 3 + m, t) + XT(sj, m, t + 1)) + (FX(m, t + 1) - FX(m, t));
                const T uy = (yap_prev[my] + yam[my]) + (Gc[m] - G_prev[m]);
                q[m] = (q[m] - dtdx * ux) - dtdy * uy;
            }
            postprocess<T, PERT>(q[0], q[1], q[2], Bc, drytol);
            if (a.manning > 0.0)
                friction<T, PERT>(q[0], q[1], q[2], Bc, drytol, PERT ? (T)a.manningf : (T)a.manning,
                                  dt_level<T>(a, P.scen));
            if (j >= y0 && j < y0 + h) {
                // a depth that is not a finite number reaches the host as an infinite speed
                if (!(dabs<T>(q[0]) < T(1e30))) smy = T(INFINITY);
                const long long gi = (long long)(j + 2) * pitch + (x0 + t);
                qo0[gi] = q[0];
                qo1[gi] = q[1];
                qo2[gi] = q[2];
            }
        }
        if (yready) {
#pragma unroll
            for (int m = 0; m < 3; m++) { yap_prev[m] = yap[m]; G_prev[m] = Gc[m]; }
        }
        // row k+1 of this thread has landed (row k+2 may still be in flight)
        cp_async_wait<1>();
        derive_own(k + 1);
    }
    cp_async_wait<0>();

    // CTA max of the wave speeds: warp shuffles, then one atomic per CTA
    if (!(smx > T(0))) smx = T(0);
    if (!(smy > T(0))) smy = T(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        smx = dmax<T>(smx, __shfl_xor_sync(0xffffffffu, smx, o));
        smy = dmax<T>(smy, __shfl_xor_sync(0xffffffffu, smy, o));
    }
    if ((t & 31) == 0) { red[t >> 5] = smx; red[NT / 32 + (t >> 5)] = smy; }
    __syncthreads();
    if (t == 0) {
        T mx = T(0), my = T(0);
        for (int k = 0; k < NT / 32; k++) { mx = dmax<T>(mx, red[k]); my = dmax<T>(my, red[NT / 32 + k]); }
        atomic_max_speed(a.smax + 2 * P.scen + 0, (double)mx);
        atomic_max_speed(a.smax + 2 * P.scen + 1, (double)my);
    }
}

template <typename T, bool PERT, int NT>
int launch_unsplit_nt(const StepArgs &a, int n_items, cudaStream_t st)
{
    constexpr int RING = 5;
    const size_t bytes = sizeof(T) * (size_t)UnsplitSmem<NT, RING>::total;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(step_unsplit_kernel<T, PERT, NT, RING>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return (int)e;
        configured = true;
    }
    step_unsplit_kernel<T, PERT, NT, RING><<<n_items, NT, bytes, st>>>(a);
    return (int)cudaGetLastError();
}

}  // namespace tsu
