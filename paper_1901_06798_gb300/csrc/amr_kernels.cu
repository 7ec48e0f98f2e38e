// amr_kernels.cu -- the kernels around the patch update: ghost-cell fill
// (same-level copy, coarse-to-fine space-time interpolation, physical
// boundaries), fine-to-coarse averaging, flagging with buffer dilation and
// proper nesting, topography sampling, seafloor uplift, the CFL / dt
// bookkeeping that keeps dt on the device, gauges and field reads.
//
// Built with --fmad=false: the FP64 instantiations round every operation as
// the FP64 oracle does.  Each kernel batches all patches of a level (and all
// scenarios) into one launch.
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>
#include <type_traits>
#include "amr_kernels.h"

namespace tsu {

// ---------------------------------------------------------------- helpers

template <typename T> struct Acc {
    T *base;
    long long fs;
    int pitch;
    __device__ __forceinline__ long long idx(int i, int j) const { return (long long)(j + 2) * pitch + (i + 2); }
    __device__ __forceinline__ T *f(int buf, int m) const { return base + (long long)(buf * 3 + m) * fs; }
    __device__ __forceinline__ T *Bp() const { return base + 6LL * fs; }
};

template <typename T> __device__ __forceinline__ Acc<T> acc(void *arena, const PatchDesc &P)
{
    Acc<T> a;
    a.base = reinterpret_cast<T *>(arena) + P.off;
    a.fs = P.fs;
    a.pitch = P.pitch;
    return a;
}

__device__ __forceinline__ int ring_count(const PatchDesc &P) { return (P.nx + 4) * (P.ny + 4) - P.nx * P.ny; }

// ghost cell g of a patch -> (i, j): 2 bottom rows, 2 top rows, then the 2+2
// side columns of the interior rows.
__device__ __forceinline__ void ring_cell(const PatchDesc &P, int g, int &i, int &j)
{
    int W = P.nx + 4;
    if (g < 2 * W) { j = -2 + g / W; i = -2 + g % W; return; }
    g -= 2 * W;
    if (g < 2 * W) { j = P.ny + g / W; i = -2 + g % W; return; }
    g -= 2 * W;
    j = g / 4;
    int k = g % 4;
    i = k < 2 ? -2 + k : P.nx + (k - 2);
}

// Arithmetic of the coarse-to-fine interpolation: double for the FP64 state
// (the oracle's operations exactly), float for the FP32 perturbation form
// (GB300's FP64 rate is a small fraction of its FP32 rate; eta' values are O(1 m))
template <bool PERT> using InterpT = typename std::conditional<PERT, float, double>::type;

template <typename W> __device__ __forceinline__ W minmod(W a, W b)
{
    if (a > W(0) && b > W(0)) return a < b ? a : b;
    if (a < W(0) && b < W(0)) return a > b ? a : b;
    return W(0);
}

// one coarse cell's (eta, hu, hv) at time fraction alpha
template <typename W> struct CVal {
    int found, wet;
    W q[3];
};

template <typename T, bool PERT>
__device__ CVal<InterpT<PERT>> coarse_value(const LevelView &C, int cur_c, const int *cmap, const PatchDesc &F, int I,
                                            int J, InterpT<PERT> alpha, InterpT<PERT> drytol)
{
    using W = InterpT<PERT>;
    CVal<W> v;
    v.found = 0; v.wet = 0; v.q[0] = v.q[1] = v.q[2] = W(0);
    if (I < 0 || I >= C.nxl || J < 0 || J >= C.nyl) return v;
    int mi = I - F.cmap_i0, mj = J - F.cmap_j0;
    if (mi < 0 || mi >= F.cmap_w || mj < 0 || mj >= F.cmap_h) return v;
    int cp = cmap[F.cmap_off + mj * F.cmap_w + mi];
    if (cp < 0) return v;
    const PatchDesc P = C.descs[cp];
    Acc<T> a = acc<T>(C.arena, P);
    long long k = a.idx(I - P.i0, J - P.j0);
    W B = (W)a.Bp()[k];
    W q0n = (W)a.f(cur_c, 0)[k], q1n = (W)a.f(cur_c, 1)[k], q2n = (W)a.f(cur_c, 2)[k];
    W q0, q1, q2;
    if (alpha == W(1)) { q0 = q0n; q1 = q1n; q2 = q2n; }
    else {
        W q0o = (W)a.f(1 - cur_c, 0)[k], q1o = (W)a.f(1 - cur_c, 1)[k], q2o = (W)a.f(1 - cur_c, 2)[k];
        q0 = q0o + alpha * (q0n - q0o);
        q1 = q1o + alpha * (q1n - q1o);
        q2 = q2o + alpha * (q2n - q2o);
    }
    v.found = 1;
    W h = PERT ? q0 - B : q0;
    v.wet = h >= drytol;
    v.q[0] = PERT ? q0 : h + B;
    v.q[1] = q1;
    v.q[2] = q2;
    return v;
}

// Space-time interpolation of fine cell (I, J) of level F from the coarse
// level (minmod-limited linear in space of eta, hu, hv over wet neighbours;
// a dry coarse centre takes the lowest wet surface of its 3x3 neighbourhood).
// Writes q0 (h or eta'), q1, q2; returns false on a nesting error.  In the
// perturbation form the surface is written as eta' itself, not as
// (eta' - B) + B, which in FP32 would round eta' to the ulp of the depth.
template <typename T, bool PERT>
__device__ bool interp_fine(const LevelView &C, int cur_c, const int *cmap, const PatchDesc &F, int r, int I, int J,
                            double Bfd, double alphad, double drytold, T &o0, T &o1, T &o2)
{
    using W = InterpT<PERT>;
    const W Bf = (W)Bfd, alpha = (W)alphad, drytol = (W)drytold;
    int Ic = I / r, Jc = J / r;
    CVal<W> c = coarse_value<T, PERT>(C, cur_c, cmap, F, Ic, Jc, alpha, drytol);
    if (!c.found) return false;
    W hf, hu, hv, ef;   // ef: the surface eta when hf > 0
    if (!c.wet) {
        W eref = W(0);
        int any = 0;
        for (int dj = -1; dj <= 1; dj++)
            for (int di = -1; di <= 1; di++) {
                if (di == 0 && dj == 0) continue;
                CVal<W> nb = coarse_value<T, PERT>(C, cur_c, cmap, F, Ic + di, Jc + dj, alpha, drytol);
                if (nb.found && nb.wet && (!any || nb.q[0] < eref)) { eref = nb.q[0]; any = 1; }
            }
        hf = any ? eref - Bf : W(0);
        ef = eref;
        if (hf < W(0)) hf = W(0);
        hu = W(0); hv = W(0);
    } else {
        CVal<W> xm = coarse_value<T, PERT>(C, cur_c, cmap, F, Ic - 1, Jc, alpha, drytol);
        CVal<W> xp = coarse_value<T, PERT>(C, cur_c, cmap, F, Ic + 1, Jc, alpha, drytol);
        CVal<W> ym = coarse_value<T, PERT>(C, cur_c, cmap, F, Ic, Jc - 1, alpha, drytol);
        CVal<W> yp = coarse_value<T, PERT>(C, cur_c, cmap, F, Ic, Jc + 1, alpha, drytol);
        W xi = ((W)(I - Ic * r) + W(0.5)) / (W)r - W(0.5);
        W et = ((W)(J - Jc * r) + W(0.5)) / (W)r - W(0.5);
        W qf[3];
        for (int m = 0; m < 3; m++) {
            W dxp = (xp.found && xp.wet) ? xp.q[m] - c.q[m] : W(0);
            W dxm = (xm.found && xm.wet) ? c.q[m] - xm.q[m] : W(0);
            W dyp = (yp.found && yp.wet) ? yp.q[m] - c.q[m] : W(0);
            W dym = (ym.found && ym.wet) ? c.q[m] - ym.q[m] : W(0);
            W sx = minmod<W>(dxp, dxm), sy = minmod<W>(dyp, dym);
            qf[m] = (c.q[m] + xi * sx) + et * sy;
        }
        hf = qf[0] - Bf;
        ef = qf[0];
        if (hf < W(0)) hf = W(0);
        if (hf < drytol) { hu = W(0); hv = W(0); }
        else { hu = qf[1]; hv = qf[2]; }
    }
    if (PERT) o0 = (T)(hf > W(0) ? ef : Bf);
    else o0 = (T)hf;
    o1 = (T)hu;
    o2 = (T)hv;
    return true;
}

// ---------------------------------------------------------------- ghost fill

// The source of every ghost cell of a patch (blockIdx.x the patch): a
// same-level neighbour whose interior holds the cell, else the coarser level
// (space-time interpolation), else none (a tiling error on the coarsest
// level).  Same-level patches do not overlap, so the source is unique.  The
// interpolated cells also go to a compact list (in no particular order: each
// is computed on its own).  Runs once per patch table; the fills gather.
__global__ void ghost_map_kernel(LevelView L, GhostSrc *gmap, int2 *ilist, int *icount, int ratio)
{
    const PatchDesc P = L.descs[blockIdx.x];
    const int n = ring_count(P);
    GhostSrc *out = gmap + L.goff[blockIdx.x];
    // the patch's neighbour boxes, staged once per CTA (each ghost cell searches them)
    constexpr int kStaged = 32;
    __shared__ int4 nbox[kStaged];
    __shared__ int nid[kStaged];
    const int ns = P.nbr_cnt < kStaged ? P.nbr_cnt : kStaged;
    for (int m = threadIdx.x; m < ns; m += blockDim.x) {
        const int qi = L.nbrs[P.nbr_off + m];
        const PatchDesc &Q = L.descs[qi];
        nbox[m] = make_int4(Q.i0, Q.j0, Q.i0 + Q.nx, Q.j0 + Q.ny);
        nid[m] = qi;
    }
    __syncthreads();
    for (int g = blockIdx.y * blockDim.x + threadIdx.x; g < n; g += gridDim.y * blockDim.x) {
        int i, j;
        ring_cell(P, g, i, j);
        const int I = P.i0 + i, J = P.j0 + j;
        GhostSrc e;
        e.src = kGhostSkip;
        e.sfs = 0;
        if (I >= 0 && I < L.nxl && J >= 0 && J < L.nyl) {
            int src = -1;
            for (int m = 0; m < ns; m++) {
                const int4 b = nbox[m];
                if (I >= b.x && I < b.z && J >= b.y && J < b.w) { src = nid[m]; break; }
            }
            for (int m = ns; src < 0 && m < P.nbr_cnt; m++) {   // more neighbours than staged
                const int qi = L.nbrs[P.nbr_off + m];
                const PatchDesc &Q = L.descs[qi];
                if (I >= Q.i0 && I < Q.i0 + Q.nx && J >= Q.j0 && J < Q.j0 + Q.ny) { src = qi; break; }
            }
            if (src >= 0) {
                const PatchDesc &Q = L.descs[src];
                e.src = Q.off + (long long)(J - Q.j0 + 2) * Q.pitch + (I - Q.i0 + 2);
                e.sfs = Q.fs;
            } else if (ratio > 0) {
                e.src = kGhostInterp;
                ilist[atomicAdd(icount, 1)] = make_int2((int)blockIdx.x, g);
            } else {
                e.src = kGhostNone;
            }
        }
        out[g] = e;
    }
}

// Ghost cells of the current state copied from the same-level interior cells
// the map names.  The interpolated cells are left to the kernel below, so
// that no CTA here waits on their long chains of dependent loads.
template <typename T>
__global__ void ghost_copy_kernel(LevelView L, int cur, int *err)
{
    const PatchDesc P = L.descs[blockIdx.x];
    const int n = ring_count(P);
    Acc<T> a = acc<T>(L.arena, P);
    T *q0 = a.f(cur, 0), *q1 = a.f(cur, 1), *q2 = a.f(cur, 2);
    const T *ar = reinterpret_cast<const T *>(L.arena);
    const GhostSrc *gm = L.gmap + L.goff[blockIdx.x];
    for (int g = blockIdx.y * blockDim.x + threadIdx.x; g < n; g += gridDim.y * blockDim.x) {
        const GhostSrc s = gm[g];
        if (s.src == kGhostSkip || s.src == kGhostInterp) continue;
        if (s.src < 0) { atomicOr(err, 1); continue; }
        int i, j;
        ring_cell(P, g, i, j);
        const long long k = a.idx(i, j);
        const T *q = ar + s.src + (long long)(cur * 3) * s.sfs;
        const T v0 = q[0], v1 = q[s.sfs], v2 = q[2 * s.sfs];
        q0[k] = v0; q1[k] = v1; q2[k] = v2;
    }
}

// The ghost cells with no same-level source, one thread each: space-time
// interpolation from the coarser level at time fraction alpha.
template <typename T, bool PERT>
__global__ void ghost_interp_kernel(LevelView L, LevelView C, int cur, int cur_c, int ratio, double alpha,
                                    double drytol, int *err)
{
    const int ni = *L.icount;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ni; e += gridDim.x * blockDim.x) {
        const int2 pg = L.ilist[e];
        const PatchDesc P = L.descs[pg.x];
        Acc<T> a = acc<T>(L.arena, P);
        int i, j;
        ring_cell(P, pg.y, i, j);
        const long long k = a.idx(i, j);
        T o0, o1, o2;
        if (interp_fine<T, PERT>(C, cur_c, L.cmap, P, ratio, P.i0 + i, P.j0 + j, (double)a.Bp()[k], alpha, drytol, o0,
                                 o1, o2)) {
            a.f(cur, 0)[k] = o0; a.f(cur, 1)[k] = o1; a.f(cur, 2)[k] = o2;
        } else {
            atomicOr(err, 1);
        }
    }
}

// Physical boundaries: every ghost cell outside the domain takes the value of
// its source cell in global indices -- wall: the mirror image across the
// domain edge with the normal momentum negated; extrapolation: the edge cell
// -- applied in x and then in y (the composition gives the corners).  The
// source always lies in the patch's own storage: an interior cell or a ghost
// cell inside the domain that the fill kernel wrote before.
__device__ __forceinline__ bool bc_source(const PatchDesc &P, int nxl, int nyl, const int *bc, int i, int j, int &si,
                                          int &sj, bool &negx, bool &negy)
{
    int I = P.i0 + i, J = P.j0 + j;
    bool out = false;
    si = i; sj = j; negx = false; negy = false;
    if (I < 0) {
        out = true;
        if (bc[0] == 0) { si = (-1 - I) - P.i0; negx = true; } else si = -P.i0;
    } else if (I >= nxl) {
        out = true;
        if (bc[1] == 0) { si = (2 * nxl - 1 - I) - P.i0; negx = true; } else si = nxl - 1 - P.i0;
    }
    if (J < 0) {
        out = true;
        if (bc[2] == 0) { sj = (-1 - J) - P.j0; negy = true; } else sj = -P.j0;
    } else if (J >= nyl) {
        out = true;
        if (bc[3] == 0) { sj = (2 * nyl - 1 - J) - P.j0; negy = true; } else sj = nyl - 1 - P.j0;
    }
    return out;
}

template <typename T>
__global__ void bc_kernel(LevelView L, int cur, BcArgs bcs, int do_state, int do_B)
{
    const PatchDesc P = L.descs[bcs.list[blockIdx.x]];
    const int n = ring_count(P);
    Acc<T> a = acc<T>(L.arena, P);
    for (int g = blockIdx.y * blockDim.x + threadIdx.x; g < n; g += gridDim.y * blockDim.x) {
        int i, j, si, sj;
        bool nx_, ny_;
        ring_cell(P, g, i, j);
        if (!bc_source(P, L.nxl, L.nyl, bcs.bc, i, j, si, sj, nx_, ny_)) continue;
        long long k = a.idx(i, j), ks = a.idx(si, sj);
        if (do_state) {
            T *q0 = a.f(cur, 0), *q1 = a.f(cur, 1), *q2 = a.f(cur, 2);
            T v1 = q1[ks], v2 = q2[ks];
            q0[k] = q0[ks];
            q1[k] = nx_ ? -v1 : v1;
            q2[k] = ny_ ? -v2 : v2;
        }
        if (do_B) a.Bp()[k] = a.Bp()[ks];
    }
}

// ---------------------------------------------------------------- averaging

// Averaging of each fine patch onto the coarse cells it covers: surface over
// the wet fine cells, momenta over all (capacity-weighted on latitude-longitude
// grids).  Arithmetic in the state's precision (InterpT); in the perturbation
// form the coarse surface is written as the mean eta' itself, not as
// (mean - B) + B.
template <typename T, bool PERT>
__global__ void average_kernel(LevelView Fv, LevelView C, int cur_f, int cur_c, int r, double drytold, int *err)
{
    using W = InterpT<PERT>;
    const W drytol = (W)drytold;
    const PatchDesc F = Fv.descs[blockIdx.x];
    const int cw = F.nx / r, ch = F.ny / r;
    const int n = cw * ch;
    Acc<T> fa = acc<T>(Fv.arena, F);
    const T *f0 = fa.f(cur_f, 0), *f1 = fa.f(cur_f, 1), *f2 = fa.f(cur_f, 2), *fB = fa.Bp();
    for (int c = blockIdx.y * blockDim.x + threadIdx.x; c < n; c += gridDim.y * blockDim.x) {
        int Ic = F.i0 / r + c % cw, Jc = F.j0 / r + c / cw;
        int mi = Ic - F.cmap_i0, mj = Jc - F.cmap_j0;
        int cp = Fv.cmap[F.cmap_off + mj * F.cmap_w + mi];
        if (cp < 0) { atomicOr(err, 2); continue; }
        W se = W(0), su = W(0), sv = W(0);
        int nwet = 0;
        W kw = W(0), ka = W(0);   // latitude-longitude grids: capacities of the wet and of all fine cells
        for (int jj = 0; jj < r; jj++) {
            const W kf_ = Fv.kap ? (W)Fv.kap[Jc * r + jj + 2] : W(1);
            for (int ii = 0; ii < r; ii++) {
                long long kf = fa.idx(Ic * r + ii - F.i0, Jc * r + jj - F.j0);
                W B = (W)fB[kf];
                W q0 = (W)f0[kf];
                W h = PERT ? q0 - B : q0;
                if (Fv.kap) {
                    if (h >= drytol) { se = se + kf_ * (PERT ? q0 : h + B); kw = kw + kf_; nwet++; }
                    su = su + kf_ * (W)f1[kf];
                    sv = sv + kf_ * (W)f2[kf];
                    ka = ka + kf_;
                } else {
                    if (h >= drytol) { se = se + (PERT ? q0 : h + B); nwet++; }
                    su = su + (W)f1[kf];
                    sv = sv + (W)f2[kf];
                }
            }
        }
        const PatchDesc P = C.descs[cp];
        Acc<T> ca = acc<T>(C.arena, P);
        long long kc = ca.idx(Ic - P.i0, Jc - P.j0);
        W Bc = (W)ca.Bp()[kc];
        W hc = W(0), ec = Bc;   // ec: the coarse surface
        if (nwet > 0) {
            ec = Fv.kap ? se / kw : se / (W)nwet;
            hc = ec - Bc;
            if (hc < W(0)) hc = W(0);
        }
        W rr = Fv.kap ? ka : (W)(r * r);
        if (PERT) ca.f(cur_c, 0)[kc] = (T)(hc > W(0) ? ec : Bc);
        else ca.f(cur_c, 0)[kc] = (T)hc;
        if (hc < drytol) { ca.f(cur_c, 1)[kc] = T(0); ca.f(cur_c, 2)[kc] = T(0); }
        else { ca.f(cur_c, 1)[kc] = (T)(su / rr); ca.f(cur_c, 2)[kc] = (T)(sv / rr); }
    }
}

// ---------------------------------------------------------------- topography

__device__ __forceinline__ bool grid_contains(const TopoDev &g, double x, double y)
{
    return x >= g.x0 && x <= g.x0 + (double)(g.nx - 1) * g.dx && y >= g.y0 && y <= g.y0 + (double)(g.ny - 1) * g.dy;
}

__device__ double grid_bilinear(const TopoDev &g, double x, double y)
{
    double fx = (x - g.x0) / g.dx, fy = (y - g.y0) / g.dy;
    int i = (int)floor(fx), j = (int)floor(fy);
    if (i < 0) i = 0;
    if (i > g.nx - 2) i = g.nx - 2;
    if (j < 0) j = 0;
    if (j > g.ny - 2) j = g.ny - 2;
    double tx = fx - (double)i, ty = fy - (double)j;
    if (tx < 0.0) tx = 0.0;
    if (tx > 1.0) tx = 1.0;
    if (ty < 0.0) ty = 0.0;
    if (ty > 1.0) ty = 1.0;
    const double *v = g.v;
    double v00 = v[(long long)j * g.nx + i], v10 = v[(long long)j * g.nx + i + 1];
    double v01 = v[(long long)(j + 1) * g.nx + i], v11 = v[(long long)(j + 1) * g.nx + i + 1];
    double a = v00 + tx * (v10 - v00);
    double b = v01 + tx * (v11 - v01);
    return a + ty * (b - a);
}

// The per-column and per-row parts of sampling every grid at a level's cell
// centres (x_I = x0 + (I + 1/2) dx, y_J likewise): the operations of
// grid_contains and grid_bilinear on one coordinate, so the values are the ones
// computed at each cell.
__global__ void axis_tab_kernel(TopoSet ts, double x0, double y0, double dxl, double dyl)
{
    const AxisTab &T = ts.tab;
    const long long ncol = (long long)ts.ngrids * T.nx, nall = ncol + (long long)ts.ngrids * T.ny;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nall; q += (long long)gridDim.x * blockDim.x) {
        const bool col = q < ncol;
        const long long r = col ? q : q - ncol;
        const int n = col ? T.nx : T.ny;
        const int k = (int)(r / n), I = (int)(r - (long long)k * n);
        const TopoDev &g = ts.grids[k];
        const double o = col ? g.x0 : g.y0, d = col ? g.dx : g.dy;
        const int gn = col ? g.nx : g.ny;
        const double x = col ? x0 + ((double)I + 0.5) * dxl : y0 + ((double)I + 0.5) * dyl;
        const unsigned char in = x >= o && x <= o + (double)(gn - 1) * d;
        const double f = (x - o) / d;
        int i = (int)floor(f);
        if (i < 0) i = 0;
        if (i > gn - 2) i = gn - 2;
        double t = f - (double)i;
        if (t < 0.0) t = 0.0;
        if (t > 1.0) t = 1.0;
        if (col) { T.ci[r] = i; T.ct[r] = t; T.cin[r] = in; }
        else { T.rj[r] = i; T.rt[r] = t; T.rin[r] = in; }
    }
}

__device__ __forceinline__ bool tab_contains(const TopoSet &ts, int k, int I, int J)
{
    return ts.tab.cin[(long long)k * ts.tab.nx + I] && ts.tab.rin[(long long)k * ts.tab.ny + J];
}

// grid_bilinear of grid k at the centre of cell (I, J), from the axis table
__device__ double tab_bilinear(const TopoSet &ts, int k, int I, int J)
{
    const TopoDev &g = ts.grids[k];
    const long long c = (long long)k * ts.tab.nx + I, r = (long long)k * ts.tab.ny + J;
    const int i = ts.tab.ci[c], j = ts.tab.rj[r];
    const double tx = ts.tab.ct[c], ty = ts.tab.rt[r];
    const double *v = g.v;
    double v00 = v[(long long)j * g.nx + i], v10 = v[(long long)j * g.nx + i + 1];
    double v01 = v[(long long)(j + 1) * g.nx + i], v11 = v[(long long)(j + 1) * g.nx + i + 1];
    double a = v00 + tx * (v10 - v00);
    double b = v01 + tx * (v11 - v01);
    return a + ty * (b - a);
}

// base_topo and uplift_sum at the centre of cell (I, J), from the axis table
__device__ double base_topo_tab(const TopoSet &ts, int I, int J)
{
    int best = -1;
    double barea = 0.0;
    for (int k = 0; k < ts.nbase; k++) {
        if (!tab_contains(ts, k, I, J)) continue;
        double area = ts.grids[k].dx * ts.grids[k].dy;
        if (best < 0 || area <= barea) { best = k; barea = area; }
    }
    if (best < 0) best = 0;
    return tab_bilinear(ts, best, I, J);
}

__device__ double uplift_sum_tab(const TopoSet &ts, int scen, double B, int I, int J)
{
    for (int k = ts.nbase; k < ts.ngrids; k++) {
        if (ts.scen[k] != scen) continue;
        if (tab_contains(ts, k, I, J)) B = B + tab_bilinear(ts, k, I, J);
    }
    return B;
}

// B (and, for level-1 initialisation, the state: h from the initial surface,
// hu = h u, hv = h v from the initial velocities on wet cells) of the patches in `list`
// at every cell inside the domain; cells outside are filled by bc_kernel.  At a
// regrid (Old.descs set) a cell that an old patch of the level held in its
// interior takes that patch's B -- the same value, without sampling the
// topography again -- and only the other cells are sampled.  Sampling picks the
// finest base grid holding the cell centre (the last of equal ones), adds the
// scenario's uplift layers holding it, and reads the per-column and per-row
// parts of each grid's bilinear interpolation from the axis table.
template <typename T, bool PERT>
__global__ void init_patch_kernel(LevelView L, LevelView Old, const int *list, TopoSet ts, int cur, int set_state,
                                  double x0, double y0, double dxl, double dyl)
{
    const PatchDesc P = L.descs[list[blockIdx.x]];
    const int n = (P.nx + 4) * (P.ny + 4);
    Acc<T> a = acc<T>(L.arena, P);
    for (int c = blockIdx.y * blockDim.x + threadIdx.x; c < n; c += gridDim.y * blockDim.x) {
        int i = c % (P.nx + 4) - 2, j = c / (P.nx + 4) - 2;
        int I = P.i0 + i, J = P.j0 + j;
        if (I < 0 || I >= L.nxl || J < 0 || J >= L.nyl) continue;
        long long k = a.idx(i, j);
        if (!set_state && Old.descs) {
            bool held = false;
            for (int m = 0; m < P.old_cnt && !held; m++) {
                const PatchDesc Q = Old.descs[L.olds[P.old_off + m]];
                if (I >= Q.i0 && I < Q.i0 + Q.nx && J >= Q.j0 && J < Q.j0 + Q.ny) {
                    Acc<T> b = acc<T>(L.arena, Q);
                    a.Bp()[k] = b.Bp()[b.idx(I - Q.i0, J - Q.j0)];
                    held = true;
                }
            }
            if (held) continue;
        }
        double B0 = base_topo_tab(ts, I, J);
        double B = uplift_sum_tab(ts, P.scen, B0, I, J);
        a.Bp()[k] = (T)B;
        if (set_state) {
            double eta = 0.0;
            int eg = ts.eta_index[3 * P.scen];
            if (eg >= 0 && tab_contains(ts, eg, I, J)) eta = tab_bilinear(ts, eg, I, J);
            double hh = eta - B0;
            if (hh < 0.0) hh = 0.0;
            double hu = 0.0, hv = 0.0;
            const int ug = ts.eta_index[3 * P.scen + 1], vg = ts.eta_index[3 * P.scen + 2];
            if (ug >= 0 && hh >= ts.drytol && tab_contains(ts, ug, I, J)) {
                hu = hh * tab_bilinear(ts, ug, I, J);
                hv = hh * tab_bilinear(ts, vg, I, J);
            }
            a.f(cur, 0)[k] = PERT ? (T)(hh + B) : (T)hh;
            a.f(cur, 1)[k] = (T)hu;
            a.f(cur, 2)[k] = (T)hv;
        }
    }
}

// seafloor uplift of one layer on the patches of a level: B += dB, h unchanged
template <typename T, bool PERT>
__global__ void uplift_kernel(LevelView L, TopoDev U, int scen, int cur, double x0, double y0, double dxl, double dyl)
{
    const PatchDesc P = L.descs[blockIdx.x];
    if (P.scen != scen) return;
    const int n = (P.nx + 4) * (P.ny + 4);
    Acc<T> a = acc<T>(L.arena, P);
    for (int c = blockIdx.y * blockDim.x + threadIdx.x; c < n; c += gridDim.y * blockDim.x) {
        int i = c % (P.nx + 4) - 2, j = c / (P.nx + 4) - 2;
        int I = P.i0 + i, J = P.j0 + j;
        if (I < 0 || I >= L.nxl || J < 0 || J >= L.nyl) continue;
        double x = x0 + ((double)I + 0.5) * dxl, y = y0 + ((double)J + 0.5) * dyl;
        if (!grid_contains(U, x, y)) continue;
        double d = grid_bilinear(U, x, y);
        long long k = a.idx(i, j);
        double Bo = (double)a.Bp()[k];
        a.Bp()[k] = (T)(Bo + d);
        if (PERT) {
            // eta' = h + B moves with the bed: shift both buffers by the deformation
            a.f(0, 0)[k] = (T)((double)a.f(0, 0)[k] + d);
            a.f(1, 0)[k] = (T)((double)a.f(1, 0)[k] + d);
        }
    }
}

// New patches of a regridded level: copy from old same-level patches where
// they overlap, else interpolate from the coarse level at its current time.
template <typename T, bool PERT>
__global__ void regrid_init_kernel(LevelView L, LevelView Old, LevelView C, const int *list, int cur, int cur_c,
                                   int ratio, double drytol, int *err)
{
    const PatchDesc P = L.descs[list[blockIdx.x]];
    const int n = P.nx * P.ny;
    Acc<T> a = acc<T>(L.arena, P);
    for (int c = blockIdx.y * blockDim.x + threadIdx.x; c < n; c += gridDim.y * blockDim.x) {
        int i = c % P.nx, j = c / P.nx;
        int I = P.i0 + i, J = P.j0 + j;
        long long k = a.idx(i, j);
        int src = -1;
        for (int m = 0; m < P.old_cnt; m++) {
            int qi = L.olds[P.old_off + m];
            const PatchDesc &Q = Old.descs[qi];
            if (I >= Q.i0 && I < Q.i0 + Q.nx && J >= Q.j0 && J < Q.j0 + Q.ny) { src = qi; break; }
        }
        if (src >= 0) {
            const PatchDesc Q = Old.descs[src];
            Acc<T> b = acc<T>(Old.arena, Q);
            long long kq = b.idx(I - Q.i0, J - Q.j0);
            a.f(cur, 0)[k] = b.f(cur, 0)[kq];
            a.f(cur, 1)[k] = b.f(cur, 1)[kq];
            a.f(cur, 2)[k] = b.f(cur, 2)[kq];
        } else {
            T o0, o1, o2;
            if (interp_fine<T, PERT>(C, cur_c, L.cmap, P, ratio, I, J, (double)a.Bp()[k], 1.0, drytol, o0, o1, o2)) {
                a.f(cur, 0)[k] = o0; a.f(cur, 1)[k] = o1; a.f(cur, 2)[k] = o2;
            } else {
                atomicOr(err, 4);
            }
        }
    }
}

// ---------------------------------------------------------------- flagging

template <typename T, bool PERT>
__global__ void flag_kernel(LevelView L, int cur, FlagArgs fa)
{
    const PatchDesc P = L.descs[blockIdx.x];
    const int n = P.nx * P.ny;
    Acc<T> a = acc<T>(L.arena, P);
    const long long plane = (long long)L.nxl * L.nyl;
    uint8_t *raw = fa.raw + plane * fa.scen_slot[P.scen];
    uint8_t *cov = fa.cov + plane * fa.scen_slot[P.scen];
    if (fa.scen_slot[P.scen] < 0) return;
    for (int c = blockIdx.y * blockDim.x + threadIdx.x; c < n; c += gridDim.y * blockDim.x) {
        int i = c % P.nx, j = c / P.nx;
        int I = P.i0 + i, J = P.j0 + j;
        long long k = a.idx(i, j);
        int f = 0;
        if (PERT) {
            // the FP64 tests below decided in FP32: a float exceeds a double t
            // exactly when it exceeds the largest float <= t; the depth eta' - B,
            // rounded in FP32, decides unless it lies within rounding of drytol,
            // where the exact FP64 difference does
            const float qf = (float)a.f(cur, 0)[k], Bf = (float)a.Bp()[k];
            if (fa.eta_tol > 0.0 && fabsf(qf) > fa.eta_tol_f) {
                const float hf = qf - Bf;
                bool wet;
                if (fa.drytol_f > 0.0f && hf > fa.drytol_f * 1.000001f) wet = true;
                else if (fa.drytol_f > 0.0f && hf < fa.drytol_f * 0.999999f) wet = false;
                else wet = (double)qf - (double)Bf >= fa.drytol;
                if (wet) f = 1;
            }
            if (fa.depth_below > 0.0 && Bf > fa.depth_neg_f) f = 1;
        } else {
            double B = (double)a.Bp()[k];
            double h = (double)a.f(cur, 0)[k];
            double eta = h + B;
            if (fa.eta_tol > 0.0 && h >= fa.drytol && fabs(eta) > fa.eta_tol) f = 1;
            if (fa.depth_below > 0.0 && -B < fa.depth_below) f = 1;
        }
        if (fa.n_regions > 0) {
            double x = fa.x0 + ((double)I + 0.5) * fa.dxl, y = fa.y0 + ((double)J + 0.5) * fa.dyl;
            for (int rg = 0; rg < fa.n_regions; rg++) {
                const double *R = fa.regions + 6 * rg;
                if (x >= R[0] && x <= R[2] && y >= R[1] && y <= R[3] && (double)fa.newlev <= R[4]) f = 1;
            }
        }
        long long gk = (long long)J * L.nxl + I;
        raw[gk] = (uint8_t)f;
        cov[gk] = 1;
    }
}

// Chebyshev dilation, separable, over the window W = (wi0, wj0, ww, wh) of each
// plane (plane blockIdx.y).
//   dir 0 (along x): a warp holds 32 consecutive cells of a row; its lanes'
//     flags, and those of the b cells on either side, form one 64-bit mask
//     (warp ballots), and a cell is set when any of the 2b + 1 bits around it
//     is (b <= 16; larger b reads the cells one by one).
//   dir 1 (along y): a thread walks down a column segment keeping the count of
//     set cells among rows J - b .. J + b: two reads per cell.
__global__ void dilate_x_kernel(const uint8_t *src, uint8_t *dst, int nx, int ny, int b, Win W)
{
    const int ncb = (W.w + blockDim.x - 1) / blockDim.x;
    const size_t pl = (size_t)blockIdx.y * nx * ny;
    const uint8_t *s = src + pl;
    uint8_t *d = dst + pl;
    const int lane = threadIdx.x & 31;
    for (int rb = blockIdx.x; rb < W.h * ncb; rb += gridDim.x) {   // uniform over the block
        const int jr = rb / ncb, ir = (rb - jr * ncb) * blockDim.x + threadIdx.x;
        const int J = W.j0 + jr, I = W.i0 + ir;
        const uint8_t *r = s + (size_t)J * nx;
        uint8_t v = 0;
        if (b <= 16) {
            const int I0 = I - lane;   // the warp's first cell
            const bool own = I < nx && r[I] != 0;
            const int il = I0 - b + lane, irr = I0 + 32 + (lane - (32 - b));
            const bool left = lane < b && il >= 0 && r[il] != 0;
            const bool right = lane >= 32 - b && irr < nx && r[irr] != 0;
            const unsigned mo = __ballot_sync(0xffffffffu, own);
            const unsigned ml = __ballot_sync(0xffffffffu, left) & ((1u << b) - 1u);
            const unsigned mr = b > 0 ? (__ballot_sync(0xffffffffu, right) >> (32 - b)) : 0u;
            const unsigned long long m = (unsigned long long)ml | ((unsigned long long)mo << b) |
                                         ((unsigned long long)mr << (32 + b));
            const unsigned long long win = (2ull << (2 * b)) - 1ull;   // 2b + 1 bits
            v = ((m >> lane) & win) != 0ull;
        } else if (ir < W.w) {
            for (int a = max(I - b, 0); a <= min(I + b, nx - 1) && !v; a++) v = r[a];
        }
        if (ir < W.w) d[(size_t)J * nx + I] = v ? 1 : 0;
    }
}

__global__ void dilate_y_kernel(const uint8_t *src, uint8_t *dst, int nx, int ny, int b, Win W, int seg)
{
    const size_t pl = (size_t)blockIdx.y * nx * ny;
    const uint8_t *s = src + pl;
    uint8_t *d = dst + pl;
    const int ncb = (W.w + blockDim.x - 1) / blockDim.x, nseg = (W.h + seg - 1) / seg;
    for (int q = blockIdx.x; q < ncb * nseg; q += gridDim.x) {
        const int sg = q / ncb, ir = (q - sg * ncb) * blockDim.x + threadIdx.x;
        if (ir >= W.w) continue;
        const int I = W.i0 + ir, ja = W.j0 + sg * seg, jb = min(W.j0 + W.h, ja + seg);
        int cnt = 0;   // set cells among rows J - b .. J + b (inside the plane)
        for (int a = max(ja - b, 0); a <= min(ja + b, ny - 1); a++) cnt += s[(size_t)a * nx + I] ? 1 : 0;
        for (int J = ja; J < jb; J++) {
            d[(size_t)J * nx + I] = cnt > 0 ? 1 : 0;
            if (J - b >= 0) cnt -= s[(size_t)(J - b) * nx + I] ? 1 : 0;
            if (J + b + 1 < ny) cnt += s[(size_t)(J + b + 1) * nx + I] ? 1 : 0;
        }
    }
}

// Proper nesting, separable: E(I, J) = every in-domain cell within 2 of I in row J
// is covered (the x pass, over the rows within 2 of the window W) ...
__global__ void erode_x_kernel(const uint8_t *cov, uint8_t *E, int nx, int ny, Win W)
{
    const int ncb = (W.w + blockDim.x - 1) / blockDim.x;
    const size_t pl = (size_t)blockIdx.y * nx * ny;
    for (int rb = blockIdx.x; rb < W.h * ncb; rb += gridDim.x) {
        const int jr = rb / ncb, ir = (rb - jr * ncb) * blockDim.x + threadIdx.x;
        if (ir >= W.w) continue;
        const int J = W.j0 + jr, I = W.i0 + ir;
        const uint8_t *r = cov + pl + (size_t)J * nx;
        uint8_t ok = 1;
        for (int a2 = max(I - 2, 0); a2 <= min(I + 2, nx - 1) && ok; a2++) ok = r[a2] ? 1 : 0;
        E[pl + (size_t)J * nx + I] = ok;
    }
}

// ... then over W: N = every in-domain cell within 2 is covered (E of the rows
// within 2), region caps and F &= N
__global__ void nest_kernel(uint8_t *F, uint8_t *N, const uint8_t *E, int nx, int ny, FlagArgs fa, Win W)
{
    const int ncb = (W.w + blockDim.x - 1) / blockDim.x;
    const size_t pl = (size_t)blockIdx.y * nx * ny;
    const uint8_t *ep = E + pl;
    for (int rb = blockIdx.x; rb < W.h * ncb; rb += gridDim.x) {
        const int jr = rb / ncb, ir = (rb - jr * ncb) * blockDim.x + threadIdx.x;
        if (ir >= W.w) continue;
        const int J = W.j0 + jr, I = W.i0 + ir;
        const size_t c = pl + (size_t)J * nx + I;
        uint8_t f = F[c];
        if (fa.n_regions > 0) {
            const double x = fa.x0 + ((double)I + 0.5) * fa.dxl, y = fa.y0 + ((double)J + 0.5) * fa.dyl;
            for (int rg = 0; rg < fa.n_regions; rg++) {
                const double *R = fa.regions + 6 * rg;
                if (x >= R[0] && x <= R[2] && y >= R[1] && y <= R[3] && (double)fa.newlev > R[5]) f = 0;
            }
        }
        int ok = 1;
        for (int b2 = max(J - 2, 0); b2 <= min(J + 2, ny - 1) && ok; b2++) ok = ep[(size_t)b2 * nx + I] ? 1 : 0;
        // N: bit 0 the final flag, bit 1 nestable -- the one plane the host clusters
        const uint8_t ff = ok ? f : 0;
        N[c] = (uint8_t)((ok << 1) | (ff ? 1 : 0));
        F[c] = ff;
    }
}

// Input planes of the refinement-flag predictor for the scenarios being
// regridded (one plane set per slot): eta/0.1 on wet cells, clip(-B/1000, -1, 5),
// |hu|/10, |hv|/10 and the criterion flag, zero where no patch covers a cell.
template <typename T, bool PERT>
__global__ void cnn_features_kernel(LevelView L, int cur, const int *scen_slot, const uint8_t *raw, float *feat,
                                    double drytol, CnnWindow win)
{
    const PatchDesc P = L.descs[blockIdx.x];
    const int slot = scen_slot[P.scen];
    if (slot < 0) return;
    if (P.i0 >= win.x0 + win.w || P.i0 + P.nx <= win.x0 || P.j0 >= win.y0 + win.h || P.j0 + P.ny <= win.y0) return;
    const int n = P.nx * P.ny;
    Acc<T> a = acc<T>(L.arena, P);
    const long long lplane = (long long)L.nxl * L.nyl;
    const long long plane = (long long)win.w * win.h;   // features of the window only
    float *f = feat + (long long)slot * 5 * plane;
    const uint8_t *rw = raw + (long long)slot * lplane;
    for (int c = blockIdx.y * blockDim.x + threadIdx.x; c < n; c += gridDim.y * blockDim.x) {
        int i = c % P.nx, j = c / P.nx;
        const int I = P.i0 + i - win.x0, J = P.j0 + j - win.y0;
        if (I < 0 || J < 0 || I >= win.w || J >= win.h) continue;
        long long k = a.idx(i, j);
        double B = (double)a.Bp()[k], q0 = (double)a.f(cur, 0)[k];
        double h = PERT ? q0 - B : q0;
        double eta = PERT ? q0 : h + B;
        long long gk = (long long)J * win.w + I;                         // in the window
        long long lk = (long long)(P.j0 + j) * L.nxl + (P.i0 + i);      // in the level plane
        double dep = -B / 1000.0;
        dep = dep < -1.0 ? -1.0 : (dep > 5.0 ? 5.0 : dep);
        f[gk] = h >= drytol ? (float)(eta / 0.1) : 0.0f;
        f[plane + gk] = (float)dep;
        f[2 * plane + gk] = (float)(fabs((double)a.f(cur, 1)[k]) / 10.0);
        f[3 * plane + gk] = (float)(fabs((double)a.f(cur, 2)[k]) / 10.0);
        f[4 * plane + gk] = rw[lk] ? 1.0f : 0.0f;
    }
}

// raw flags |= (logit > 0) on covered cells of the target box (logits of the
// window, one plane per flag plane)
__global__ void cnn_union_kernel(uint8_t *raw, const uint8_t *cov, const float *logits, int nx, int ny, int np,
                                 CnnWindow win)
{
    const long long tn = (long long)win.tw * win.th, n = tn * np;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const long long pl = q / tn, r = q % tn;
        const int I = win.tx0 + (int)(r % win.tw), J = win.ty0 + (int)(r / win.tw);
        const long long g = pl * (long long)nx * ny + (long long)J * nx + I;
        const long long w = pl * (long long)win.w * win.h + (long long)(J - win.y0) * win.w + (I - win.x0);
        if (cov[g] && logits[w] > 0.0f) raw[g] = 1;
    }
}

// ---------------------------------------------------------------- rates, dt

// Largest cell wave speeds (x, y) of the patches in `list`, for the first dt
// of a level or of new patches.  Blocks walk patches (blockIdx.y) and, within
// a patch, interleaved groups of 8 rows (blockIdx.x; 32 x 8 threads over
// columns and rows, no index division), then reduce in shared memory: one
// atomic pair per block and patch, not per warp (thousands of patches from a
// regrid would otherwise queue on the same two words).  Many small patches
// take one block each; one large patch spreads over many.
// Interior cells of the level's patches whose depth is negative (h < 0; in the
// perturbation form eta' - B < 0 in FP32, the operation the sweeps derive h
// with), counted into *count.  No state the library stores has one: the
// sweeps, the averaging and the interpolation clip depths at zero.
template <typename T, bool PERT>
__global__ void __launch_bounds__(256) depth_check_kernel(LevelView L, int npatch, int cur, int *count)
{
    const int tx = threadIdx.x, ty = threadIdx.y;
    int n = 0;
    for (int pi = blockIdx.y; pi < npatch; pi += gridDim.y) {
        const PatchDesc P = L.descs[pi];
        Acc<T> a = acc<T>(L.arena, P);
        for (int j = blockIdx.x * 8 + ty; j < P.ny; j += gridDim.x * 8) {
            const T *r0 = a.f(cur, 0) + a.idx(0, j), *rB = a.Bp() + a.idx(0, j);
            for (int i = tx; i < P.nx; i += 32) {
                const T h = PERT ? r0[i] - rB[i] : r0[i];
                n += h < T(0) ? 1 : 0;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if (tx == 0 && n) atomicAdd(count, n);
}

// Max wave speeds of a list of patches (new patches after a regrid, or all of
// them at initialisation).  One CTA row per patch; the CTAs of a row split its
// interior cells, flat in row-major order, and each thread loads the fields
// of kU cells before it uses any, so that many loads are in flight.  The
// maxima are order-free (a speed that is not a number never wins a compare).
template <typename T, bool PERT>
__global__ void __launch_bounds__(256) cell_speed_kernel(LevelView L, const int *list, int nlist, int cur, double g,
                                                         double drytol, unsigned long long *smax)
{
    constexpr int kU = 4;
    __shared__ double red[2][8];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int pi = blockIdx.y; pi < nlist; pi += gridDim.y) {
        const PatchDesc P = L.descs[list ? list[pi] : pi];
        Acc<T> a = acc<T>(L.arena, P);
        const T *r0 = a.f(cur, 0), *r1 = a.f(cur, 1), *r2 = a.f(cur, 2), *rB = a.Bp();
        const int ncell = P.nx * P.ny;
        const int stride = gridDim.x * blockDim.x;
        T sxT = T(0), syT = T(0);   // running maxima in the state's precision (no FP64 work per cell in FP32)
        for (int e0 = blockIdx.x * blockDim.x + t; e0 < ncell; e0 += kU * stride) {
            T q0[kU], qB[kU], qu[kU], qv[kU];
            int jr[kU];
#pragma unroll
            for (int u = 0; u < kU; u++) {
                const int e = e0 + u * stride;
                const int j = e < ncell ? e / P.nx : 0, i = e < ncell ? e - j * P.nx : 0;
                const long long k = a.idx(i, j);
                jr[u] = e < ncell ? j : -1;
                q0[u] = r0[k]; qB[u] = rB[k]; qu[u] = r1[k]; qv[u] = r2[k];
            }
#pragma unroll
            for (int u = 0; u < kU; u++) {
                if (jr[u] < 0) continue;
                const T h = PERT ? q0[u] - qB[u] : q0[u];
                if (h < (T)drytol) continue;
                const T cc = PERT ? (T)sqrtf((float)((T)g * h)) : (T)sqrt((double)((T)g * h));
                const T ux = qu[u] / h, uy = qv[u] / h;
                T ax = (ux < T(0) ? -ux : ux) + cc, ay = (uy < T(0) ? -uy : uy) + cc;
                if (L.kap) {   // latitude-longitude grids: x speeds over the row's capacity, y speeds
                               // times the larger edge length over it (the sweeps' Courant numbers)
                    const int jj = P.j0 + jr[u] + 2;
                    const double kd = L.kap[jj];
                    const T kj = (T)kd;
                    const T cj = (T)(fmax(L.ced[jj], L.ced[jj + 1]) / kd);
                    ax = ax / kj;
                    ay = ay * cj;
                }
                sxT = ax > sxT ? ax : sxT;
                syT = ay > syT ? ay : syT;
            }
        }
        double sx = (double)sxT, sy = (double)syT;
        for (int o = 16; o > 0; o >>= 1) {
            sx = fmax(sx, __shfl_xor_sync(0xffffffffu, sx, o));
            sy = fmax(sy, __shfl_xor_sync(0xffffffffu, sy, o));
        }
        if (lane == 0) { red[0][warp] = sx; red[1][warp] = sy; }
        __syncthreads();
        if (t == 0) {
            double mx = 0.0, my = 0.0;
            for (int k = 0; k < (int)(blockDim.x >> 5); k++) { mx = fmax(mx, red[0][k]); my = fmax(my, red[1][k]); }
            if (mx > 0.0) atomicMax(smax + 2 * P.scen, (unsigned long long)__double_as_longlong(mx));
            if (my > 0.0) atomicMax(smax + 2 * P.scen + 1, (unsigned long long)__double_as_longlong(my));
        }
        __syncthreads();   // red is reused by the next patch
    }
}

// After a level step (mode 0) or a cell-speed scan (mode 1): fold the level's
// max speeds into its rate max(sx/dx, sy/dy), check the CFL number of the step
// just taken and count cell updates (mode 0).
// After a level's step: the level's rate max(sx/dx, sy/dy) from the speeds
// the step kernels reduced (smax is cleared for the next step).
//   mode 0: a kept step -- count its cells, a violation if dt rate > cfl_max,
//           and fold the rate into the level's maximum;
//   mode 1: cell speeds of new patches -- the rate only;
//   mode 2: a level-1 step that may be retaken (Sec. 2.2 CFL condition): if
//           dt rate > cfl_max, mark the scenario for a retake and set
//           dt^1 = cfl_desired / rate (the state is still in the untouched
//           buffer); otherwise keep it as in mode 0;
//   mode 3: after the retake launch -- keep the retaken steps as in mode 0.
// A rate that is not a finite number (a NaN or infinite speed) sets the error
// flag to TSU_DEV_ERR_NAN.  end_step (modes 0 and 3, every scenario): then
// t += dt^1, as end_step_kernel.
__global__ void post_level_kernel(CtrlView cv, int level, int nscen, double R, double dx, double dy, double cfl_max,
                                  double cfl_desired, int mode, int end_step)
{
    for (int s = threadIdx.x; s < nscen; s += blockDim.x) {
        do {
            unsigned long long *sm = cv.smax + 2 * s;
            double sx = __longlong_as_double((long long)sm[0]);
            double sy = __longlong_as_double((long long)sm[1]);
            sm[0] = 0ull;
            sm[1] = 0ull;
            if (mode == 3 && cv.retake[s] == 0) break;
            double rate = fmax(sx / dx, sy / dy);
            if (!(sx <= 1.0e300 && sy <= 1.0e300)) atomicOr(cv.err, TSU_DEV_ERR_NAN);
            double *ra = cv.rate + (long long)s * cv.max_levels + level;
            if (mode != 1) {
                double dt = cv.dt1[s] / R;
                if (dt * rate > cfl_max) {
                    if (mode == 2) {
                        cv.retake[s] = 1;
                        cv.retakes[s] += 1;
                        cv.dt1[s] = cfl_desired / rate;
                        cv.dt1f[s] = (float)cv.dt1[s];
                        break;
                    }
                    cv.cfl_viol[s] += 1;
                }
                if (mode == 2 || mode == 3) cv.retake[s] = 0;
                cv.cell_updates[s] += cv.cells[(long long)s * cv.max_levels + level];
            }
            *ra = fmax(*ra, rate);
        } while (false);
        if (end_step) cv.t[s] = cv.t[s] + cv.dt1[s];
    }
}

// Start of a coarse step: dt^1 = min(dt_max, nu_d / max_l(rate_l / R_l)).
__global__ void begin_step_kernel(CtrlView cv, int nscen, int nlev, const double *Rl, double cfl_desired,
                                  double dt_max)
{
    for (int s = threadIdx.x; s < nscen; s += blockDim.x) {
        double m = 0.0;
        for (int l = 0; l < nlev; l++) m = fmax(m, cv.rate[(long long)s * cv.max_levels + l] / Rl[l]);
        double dt = m > 0.0 ? cfl_desired / m : dt_max;
        cv.dt1[s] = fmin(dt, dt_max);
        cv.dt1f[s] = (float)cv.dt1[s];
        for (int l = 0; l < cv.max_levels; l++) cv.rate[(long long)s * cv.max_levels + l] = 0.0;
    }
}

__global__ void end_step_kernel(CtrlView cv, int nscen)
{
    for (int s = threadIdx.x; s < nscen; s += blockDim.x) cv.t[s] = cv.t[s] + cv.dt1[s];
}

// ---------------------------------------------------------------- gauges, fields

template <typename T, bool PERT>
__global__ void gauge_kernel(GaugeArgs ga, CtrlView cv)
{
    const int total = ga.nscen * ga.ngauges;
    const long long sidx = *ga.nsamp;
    for (int c = threadIdx.x; c < total; c += blockDim.x) {
        int s = c / ga.ngauges;
        const GaugeLoc gl = ga.loc[c];
        double eta = __longlong_as_double(0x7ff8000000000000LL);
        if (gl.patch >= 0) {
            const LevelView &L = ga.levels[gl.level];
            const PatchDesc P = L.descs[gl.patch];
            Acc<T> a = acc<T>(L.arena, P);
            int cur = ga.curs[gl.level];
            double dxl = ga.dxl[gl.level], dyl = ga.dyl[gl.level];
            double x = ga.xy[2 * (c % ga.ngauges)], y = ga.xy[2 * (c % ga.ngauges) + 1];
            double fx = (x - ga.x0) / dxl - 0.5, fy = (y - ga.y0) / dyl - 0.5;
            int ia = (int)floor(fx), ja = (int)floor(fy);
            double tx = fx - (double)ia, ty = fy - (double)ja;
            if (ia < P.i0) { ia = P.i0; tx = 0.0; }
            if (ia > P.i0 + P.nx - 2) { ia = P.i0 + P.nx - 2; tx = 1.0; }
            if (ja < P.j0) { ja = P.j0; ty = 0.0; }
            if (ja > P.j0 + P.ny - 2) { ja = P.j0 + P.ny - 2; ty = 1.0; }
            int i = ia - P.i0, j = ja - P.j0;
            const T *q0 = a.f(cur, 0), *B = a.Bp();
            double e[4];
            int di[4] = {0, 1, 0, 1}, dj[4] = {0, 0, 1, 1};
            for (int m = 0; m < 4; m++) {
                long long k = a.idx(i + di[m], j + dj[m]);
                e[m] = PERT ? (double)q0[k] : (double)q0[k] + (double)B[k];
            }
            double aa = e[0] + tx * (e[1] - e[0]);
            double bb = e[2] + tx * (e[3] - e[2]);
            eta = aa + ty * (bb - aa);
        }
        ga.eta[(sidx * ga.nscen + s) * ga.ngauges + (c % ga.ngauges)] = eta;
        if (c % ga.ngauges == 0) ga.t[sidx * ga.nscen + s] = cv.t[s];
    }
    __syncthreads();
    if (threadIdx.x == 0) *ga.nsamp = sidx + 1;
}

template <typename T, bool PERT>
__global__ void read_field_kernel(LevelView L, int cur, int scen, int field, double *dst, int nx, int ny, double x0,
                                  double y0, double dx, double dy, double X0, double Y0, double dxl, double dyl)
{
    const PatchDesc P = L.descs[blockIdx.x];
    if (P.scen != scen) return;
    // output index range whose points fall inside the patch interior
    double xl = X0 + (double)P.i0 * dxl, xh = X0 + (double)(P.i0 + P.nx) * dxl;
    double yl = Y0 + (double)P.j0 * dyl, yh = Y0 + (double)(P.j0 + P.ny) * dyl;
    int ia = (int)floor((xl - x0) / dx) - 1, ib = (int)ceil((xh - x0) / dx) + 1;
    int ja = (int)floor((yl - y0) / dy) - 1, jb = (int)ceil((yh - y0) / dy) + 1;
    if (ia < 0) ia = 0;
    if (ja < 0) ja = 0;
    if (ib > nx) ib = nx;
    if (jb > ny) jb = ny;
    if (ia >= ib || ja >= jb) return;
    Acc<T> a = acc<T>(L.arena, P);
    const int w = ib - ia, n = w * (jb - ja);
    for (int c = blockIdx.y * blockDim.x + threadIdx.x; c < n; c += gridDim.y * blockDim.x) {
        int i = ia + c % w, j = ja + c / w;
        double x = x0 + (double)i * dx, y = y0 + (double)j * dy;
        int I = (int)floor((x - X0) / dxl), J = (int)floor((y - Y0) / dyl);
        if (I < P.i0 || I >= P.i0 + P.nx || J < P.j0 || J >= P.j0 + P.ny) continue;
        long long k = a.idx(I - P.i0, J - P.j0);
        double B = (double)a.Bp()[k], q0 = (double)a.f(cur, 0)[k];
        double h = PERT ? q0 - B : q0;
        double v;
        switch (field) {
        case 0: v = h; break;
        case 1: v = (double)a.f(cur, 1)[k]; break;
        case 2: v = (double)a.f(cur, 2)[k]; break;
        case 3: v = PERT ? q0 : h + B; break;
        case 4: v = B > 0.0 ? h : (PERT ? q0 : h + B); break;
        default: v = B; break;
        }
        dst[(long long)j * nx + i] = v;
    }
}

// interior of one patch to FP64 staging (h, hu, hv, B), for reads to host
template <typename T, bool PERT>
__global__ void patch_out_kernel(LevelView L, int p, int cur, double *out)
{
    const PatchDesc P = L.descs[p];
    const int n = P.nx * P.ny;
    Acc<T> a = acc<T>(L.arena, P);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        int i = c % P.nx, j = c / P.nx;
        long long k = a.idx(i, j);
        double B = (double)a.Bp()[k], q0 = (double)a.f(cur, 0)[k];
        out[c] = PERT ? q0 - B : q0;
        out[n + c] = (double)a.f(cur, 1)[k];
        out[2 * n + c] = (double)a.f(cur, 2)[k];
        out[3 * n + c] = B;
    }
}

// Mass of each scenario over level 1 (the composite mass once finer levels
// are averaged down), in FP64 and in a fixed order, so it is reproducible to
// the last bit: block b of patch p sums its cells (capacity-weighted on
// latitude-longitude grids), reduces by a fixed tree and writes parts[p B + b]
// (p = blockIdx.x, b = blockIdx.y, B CTAs per patch);
// mass_sum_kernel adds the parts of each scenario in (p, b) order.
template <typename T, bool PERT>
__global__ void __launch_bounds__(256) mass_kernel(LevelView L, int cur, double *parts)
{
    __shared__ double red[256];
    const PatchDesc P = L.descs[blockIdx.x];
    const int n = P.nx * P.ny;
    Acc<T> a = acc<T>(L.arena, P);
    double s = 0.0;
    for (int c = blockIdx.y * blockDim.x + threadIdx.x; c < n; c += gridDim.y * blockDim.x) {
        long long k = a.idx(c % P.nx, c / P.nx);
        double q0 = (double)a.f(cur, 0)[k];
        double h = PERT ? q0 - (double)a.Bp()[k] : q0;
        s += L.kap ? L.kap[P.j0 + c / P.nx + 2] * h : h;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] = red[threadIdx.x] + red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) parts[(size_t)blockIdx.x * gridDim.y + blockIdx.y] = red[0];
}

__global__ void mass_sum_kernel(const PatchDesc *descs, int npatch, int nb, const double *parts, double *mass,
                                int nscen)
{
    for (int sc = blockIdx.x * blockDim.x + threadIdx.x; sc < nscen; sc += gridDim.x * blockDim.x) {
        double m = 0.0;
        for (int p = 0; p < npatch; p++)
            if (descs[p].scen == sc)
                for (int b = 0; b < nb; b++) m = m + parts[(size_t)p * nb + b];
        mass[sc] = m;
    }
}

// ---------------------------------------------------------------- launchers

// Grid of a patch-batched launch: blockIdx.x is the patch (or list entry), so
// a level may hold more patches than a grid's y extent allows, and blockIdx.y
// the CTA within it: enough CTAs to cover its work, at most 64 when there are
// many patches, and up to 16 per SM over the whole grid when there are few (a
// single large patch must still fill the GPU)
static dim3 grid_for(int per_patch, int npatch, int threads)
{
    int by = (per_patch + threads - 1) / threads;
    const int cap = npatch >= 38 ? 64 : (152 * 16) / (npatch > 0 ? npatch : 1);
    if (by < 1) by = 1;
    if (by > cap) by = cap;
    return dim3(npatch, by);
}

// ---------------------------------------------------------------- halo exchange
// A level split over ranks (one process per GPU) exchanges, before each level
// step, the parts of its patches' 2-cell ghost rings that patches on other
// ranks own.  These kernels move those boxes between the patches' current
// buffers and one contiguous device buffer in message order: per message, the
// fields q0, hu, hv, each a row-major h x w block.  One CTA per message.
template <typename T, bool PERT>
__global__ void halo_pack_kernel(LevelView L, const HaloMsg *msgs, int cur, T *buf)
{
    const HaloMsg m = msgs[blockIdx.x];
    const PatchDesc P = L.descs[m.patch];
    Acc<T> a = acc<T>(L.arena, P);
    const int n = m.w * m.h;
    for (int c = threadIdx.x; c < 3 * n; c += blockDim.x) {
        const int f = c / n, e = c - f * n;
        const int j = m.j0 - P.j0 + e / m.w, i = m.i0 - P.i0 + e % m.w;
        buf[m.off + c] = a.f(cur, f)[a.idx(i, j)];
    }
}

template <typename T, bool PERT>
__global__ void halo_unpack_kernel(LevelView L, const HaloMsg *msgs, int cur, const T *buf)
{
    const HaloMsg m = msgs[blockIdx.x];
    const PatchDesc P = L.descs[m.patch];
    Acc<T> a = acc<T>(L.arena, P);
    const int n = m.w * m.h;
    for (int c = threadIdx.x; c < 3 * n; c += blockDim.x) {
        const int f = c / n, e = c - f * n;
        const int j = m.j0 - P.j0 + e / m.w, i = m.i0 - P.i0 + e % m.w;
        a.f(cur, f)[a.idx(i, j)] = buf[m.off + c];
    }
}

#define TSU_DISPATCH(PREC, KERNEL, ...)                                  \
    do {                                                                 \
        if (PREC == 0) KERNEL<double, false>__VA_ARGS__;                 \
        else KERNEL<float, true>__VA_ARGS__;                             \
    } while (0)

int k_ghost_map(const LevelView &L, GhostSrc *gmap, int2 *ilist, int *icount, int npatch, int maxring, int ratio,
                cudaStream_t st)
{
    int e = (int)cudaMemsetAsync(icount, 0, sizeof(int), st);
    if (e != 0 || npatch <= 0) return e;
    // many patches: one CTA per patch (its neighbour boxes are staged once);
    // few: their ghost rings spread over more CTAs
    dim3 g = npatch >= 152 * 8 ? dim3(npatch, 1) : grid_for(maxring, npatch, 128);
    ghost_map_kernel<<<g, 128, 0, st>>>(L, gmap, ilist, icount, ratio);
    return (int)cudaGetLastError();
}

int k_ghost_fill(int prec, const LevelView &L, const LevelView &C, int npatch, int maxring, int cur, int cur_c,
                 int ratio, double alpha, double drytol, int *err, cudaStream_t st)
{
    if (npatch <= 0) return 0;
    dim3 g = npatch >= 152 * 8 ? dim3(npatch, 1) : grid_for(maxring, npatch, 128);
    if (prec == 0) ghost_copy_kernel<double><<<g, 128, 0, st>>>(L, cur, err);
    else ghost_copy_kernel<float><<<g, 128, 0, st>>>(L, cur, err);
    int e = (int)cudaGetLastError();
    if (e != 0 || ratio <= 0) return e;
    // the list's length is known on the device only: a fixed grid strides over it
    TSU_DISPATCH(prec, ghost_interp_kernel, <<<152 * 8, 128, 0, st>>>(L, C, cur, cur_c, ratio, alpha, drytol, err));
    return (int)cudaGetLastError();
}

int k_bc(int prec, const LevelView &L, const BcArgs &b, int nlist, int maxring, int cur, int do_state, int do_B,
         cudaStream_t st)
{
    if (nlist <= 0) return 0;
    dim3 g = grid_for(maxring, nlist, 128);
    if (prec == 0) bc_kernel<double><<<g, 128, 0, st>>>(L, cur, b, do_state, do_B);
    else bc_kernel<float><<<g, 128, 0, st>>>(L, cur, b, do_state, do_B);
    return (int)cudaGetLastError();
}

int k_average(int prec, const LevelView &F, const LevelView &C, int npatch, int maxcells, int cur_f, int cur_c, int r,
              double drytol, int *err, cudaStream_t st)
{
    if (npatch <= 0) return 0;
    // one thread per coarse cell: a patch has about maxcells / r^2 of them
    dim3 g = grid_for((maxcells + r * r - 1) / (r * r), npatch, 128);
    TSU_DISPATCH(prec, average_kernel, <<<g, 128, 0, st>>>(F, C, cur_f, cur_c, r, drytol, err));
    return (int)cudaGetLastError();
}

int k_init_patches(int prec, const LevelView &L, const LevelView &Old, const int *list, int nlist, int maxcells,
                   const TopoSet &ts, int cur,
                   int set_state, double x0, double y0, double dxl, double dyl, cudaStream_t st)
{
    if (nlist <= 0) return 0;
    // the sampling's per-column and per-row parts at this level's cell centres
    TopoSet t = ts;
    t.tab.nx = L.nxl;
    t.tab.ny = L.nyl;
    const long long nt = (long long)ts.ngrids * (L.nxl + L.nyl);
    axis_tab_kernel<<<(int)std::min<long long>((nt + 255) / 256, 152 * 8), 256, 0, st>>>(t, x0, y0, dxl, dyl);
    int e = (int)cudaGetLastError();
    if (e != 0) return e;
    dim3 g = grid_for(maxcells, nlist, 128);
    TSU_DISPATCH(prec, init_patch_kernel, <<<g, 128, 0, st>>>(L, Old, list, t, cur, set_state, x0, y0, dxl, dyl));
    return (int)cudaGetLastError();
}

int k_uplift(int prec, const LevelView &L, int npatch, int maxcells, const TopoDev &U, int scen, int cur, double x0,
             double y0, double dxl, double dyl, cudaStream_t st)
{
    if (npatch <= 0) return 0;
    dim3 g = grid_for(maxcells, npatch, 128);
    TSU_DISPATCH(prec, uplift_kernel, <<<g, 128, 0, st>>>(L, U, scen, cur, x0, y0, dxl, dyl));
    return (int)cudaGetLastError();
}

int k_regrid_init(int prec, const LevelView &L, const LevelView &Old, const LevelView &C, const int *list, int nlist,
                  int maxcells, int cur, int cur_c, int ratio, double drytol, int *err, cudaStream_t st)
{
    if (nlist <= 0) return 0;
    dim3 g = grid_for(maxcells, nlist, 128);
    TSU_DISPATCH(prec, regrid_init_kernel, <<<g, 128, 0, st>>>(L, Old, C, list, cur, cur_c, ratio, drytol, err));
    return (int)cudaGetLastError();
}

int k_flag(int prec, const LevelView &L, int npatch, int maxcells, int cur, const FlagArgs &fa, cudaStream_t st)
{
    if (npatch <= 0) return 0;
    dim3 g = grid_for(maxcells, npatch, 128);
    TSU_DISPATCH(prec, flag_kernel, <<<g, 128, 0, st>>>(L, cur, fa));
    return (int)cudaGetLastError();
}

int k_dilate(const uint8_t *src, uint8_t *dst, int nx, int ny, int nplanes, int b, int dir, const Win &W,
             cudaStream_t st)
{
    if (nplanes <= 0 || W.w <= 0 || W.h <= 0) return 0;
    if (dir == 0) {
        const long long rows = (long long)W.h * ((W.w + 255) / 256);
        const int blocks = (int)std::min<long long>(rows, 152LL * 16);
        dilate_x_kernel<<<dim3(blocks, nplanes), 256, 0, st>>>(src, dst, nx, ny, b, W);
    } else {
        constexpr int kSeg = 64;   // rows per column segment
        const long long items = (long long)((W.h + kSeg - 1) / kSeg) * ((W.w + 255) / 256);
        const int blocks = (int)std::min<long long>(items, 152LL * 16);
        dilate_y_kernel<<<dim3(blocks, nplanes), 256, 0, st>>>(src, dst, nx, ny, b, W, kSeg);
    }
    return (int)cudaGetLastError();
}

int k_nest(uint8_t *F, uint8_t *N, const uint8_t *cov, uint8_t *tmp, int nx, int ny, int nplanes, const FlagArgs &fa,
           const Win &W, cudaStream_t st)
{
    if (nplanes <= 0 || W.w <= 0 || W.h <= 0) return 0;
    const int ja = std::max(0, W.j0 - 2), jb = std::min(ny, W.j0 + W.h + 2);
    const Win Wx{W.i0, ja, W.w, jb - ja};
    long long rows = (long long)Wx.h * ((W.w + 255) / 256);
    int blocks = (int)std::min<long long>(rows, 152LL * 16);
    erode_x_kernel<<<dim3(blocks, nplanes), 256, 0, st>>>(cov, tmp, nx, ny, Wx);
    rows = (long long)W.h * ((W.w + 255) / 256);
    blocks = (int)std::min<long long>(rows, 152LL * 16);
    nest_kernel<<<dim3(blocks, nplanes), 256, 0, st>>>(F, N, tmp, nx, ny, fa, W);
    return (int)cudaGetLastError();
}

// Bounding box of the flagged cells of each plane: box[4p .. 4p+3] = min i,
// min j, max i, max j (left at nx, ny, -1, -1 when nothing is flagged).  One
// block per (row group, plane); warp minima/maxima, then one atomic per warp.
__global__ void flag_bbox_kernel(const uint8_t *F, int nx, int ny, int rows_per_block, int *box, Win W)
{
    const int p = blockIdx.y;
    const uint8_t *Fp = F + (size_t)p * nx * ny;
    int i0 = nx, j0 = ny, i1 = -1, j1 = -1;
    const int ja = W.j0 + blockIdx.x * rows_per_block, jb = min(W.j0 + W.h, ja + rows_per_block);
    for (int j = ja; j < jb; j++)
        for (int i = W.i0 + threadIdx.x; i < W.i0 + W.w; i += blockDim.x)
            if (Fp[(size_t)j * nx + i]) {
                i0 = min(i0, i); i1 = max(i1, i);
                j0 = min(j0, j); j1 = max(j1, j);
            }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        i0 = min(i0, __shfl_xor_sync(0xffffffffu, i0, o));
        j0 = min(j0, __shfl_xor_sync(0xffffffffu, j0, o));
        i1 = max(i1, __shfl_xor_sync(0xffffffffu, i1, o));
        j1 = max(j1, __shfl_xor_sync(0xffffffffu, j1, o));
    }
    if ((threadIdx.x & 31) == 0 && i1 >= 0) {
        atomicMin(box + 4 * p + 0, i0);
        atomicMin(box + 4 * p + 1, j0);
        atomicMax(box + 4 * p + 2, i1);
        atomicMax(box + 4 * p + 3, j1);
    }
}

// The box (i0, j0, w, h) of one nx-wide byte plane N (bit 0 the flag, bit 1
// nestable), packed 4 cells per byte: cell i of box row j at byte
// j * ps + i / 4, bits 2 (i % 4) (flag) and 2 (i % 4) + 1 (nestable); the
// bytes past the row's last cell are zero.  One thread per packed byte.
__global__ void pack_flags_kernel(const uint8_t *N, int nx, int i0, int j0, int w, int h, int ps, uint8_t *out)
{
    const long long n = (long long)ps * h;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(k / ps), b = (int)(k % ps);
        const uint8_t *r = N + (size_t)(j0 + j) * nx + i0;
        unsigned v = 0;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int i = 4 * b + q;
            if (i < w) v |= (unsigned)(r[i] & 3) << (2 * q);
        }
        out[k] = (uint8_t)v;
    }
}

int k_pack_flags(const uint8_t *N, int nx, int i0, int j0, int w, int h, int ps, uint8_t *out, cudaStream_t st)
{
    const long long n = (long long)ps * h;
    if (n <= 0) return 0;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 152LL * 16);
    pack_flags_kernel<<<blocks, 256, 0, st>>>(N, nx, i0, j0, w, h, ps, out);
    return (int)cudaGetLastError();
}

// Coarse maps of a level (levels >= 2): cell (mi, mj) of patch p's map holds
// the coarse patch covering coarse cell (cmap_i0 + mi, cmap_j0 + mj), or -1.
// The few coarse patches overlapping the footprint come as the patch's
// candidate list; coarse patches of a scenario do not overlap, so the first
// candidate containing the cell is the only one.  One block per patch.
__global__ void fill_cmap_kernel(const PatchDesc *descs, const PatchDesc *cdescs, const int *cand, int npatch,
                                 int *cmap)
{
    __shared__ int4 cb[32];
    __shared__ int cid[32];
    for (int p = blockIdx.x; p < npatch; p += gridDim.x) {
        const PatchDesc P = descs[p];
        const int nc = P.ccand_cnt < 32 ? P.ccand_cnt : 32;
        __syncthreads();
        for (int m = threadIdx.x; m < nc; m += blockDim.x) {
            const int q = cand[P.ccand_off + m];
            const PatchDesc &Q = cdescs[q];
            cb[m] = make_int4(Q.i0, Q.j0, Q.i0 + Q.nx, Q.j0 + Q.ny);
            cid[m] = q;
        }
        __syncthreads();
        const int n = P.cmap_w * P.cmap_h;
        for (int c = threadIdx.x; c < n; c += blockDim.x) {
            const int mj = c / P.cmap_w, mi = c - mj * P.cmap_w;
            const int I = P.cmap_i0 + mi, J = P.cmap_j0 + mj;
            int v = -1;
            for (int m = 0; m < nc && v < 0; m++) {
                const int4 b = cb[m];
                if (I >= b.x && I < b.z && J >= b.y && J < b.w) v = cid[m];
            }
            for (int m = nc; m < P.ccand_cnt && v < 0; m++) {   // more candidates than staged
                const int q = cand[P.ccand_off + m];
                const PatchDesc &Q = cdescs[q];
                if (I >= Q.i0 && I < Q.i0 + Q.nx && J >= Q.j0 && J < Q.j0 + Q.ny) v = q;
            }
            cmap[(size_t)P.cmap_off + c] = v;
        }
    }
}

int k_fill_cmap(const PatchDesc *descs, const PatchDesc *cdescs, const int *cand, int npatch, int *cmap, cudaStream_t st)
{
    if (npatch <= 0) return 0;
    const int blocks = npatch < 152 * 16 ? npatch : 152 * 16;
    fill_cmap_kernel<<<blocks, 128, 0, st>>>(descs, cdescs, cand, npatch, cmap);
    return (int)cudaGetLastError();
}

int k_flag_bbox(const uint8_t *F, int nx, int ny, int nplanes, int *box, cudaStream_t st, const Win *W)
{
    const Win w = W ? *W : Win{0, 0, nx, ny};
    if (nplanes <= 0 || w.w <= 0 || w.h <= 0) return 0;
    const int rpb = 8;
    dim3 grid((w.h + rpb - 1) / rpb, nplanes);
    flag_bbox_kernel<<<grid, 256, 0, st>>>(F, nx, ny, rpb, box, w);
    return (int)cudaGetLastError();
}

int k_depth_check(int prec, const LevelView &L, int npatch, int maxcells, int cur, int *count, cudaStream_t st)
{
    if (npatch <= 0) return 0;
    constexpr int kBlocks = 152 * 8;
    const int by = npatch < kBlocks ? npatch : kBlocks;
    int bx = (maxcells + 256 * 32 - 1) / (256 * 32);
    if (bx > kBlocks / by) bx = kBlocks / by;
    if (bx < 1) bx = 1;
    TSU_DISPATCH(prec, depth_check_kernel, <<<dim3(bx, by), dim3(32, 8), 0, st>>>(L, npatch, cur, count));
    return (int)cudaGetLastError();
}

int k_cell_speed(int prec, const LevelView &L, const int *list, int nlist, int maxcells, int cur, double g,
                 double drytol, unsigned long long *smax, cudaStream_t st)
{
    if (nlist <= 0) return 0;
    // one CTA row per patch (up to the grid's limit); a large patch spreads over
    // more CTAs, about 16 cells per thread, while the launch stays near 32 CTAs
    // of 256 threads per SM
    const int by = nlist < 65535 ? nlist : 65535;
    int bx = (maxcells + 256 * 16 - 1) / (256 * 16);
    const int cap = (152 * 32) / by;
    if (bx > cap) bx = cap;
    if (bx < 1) bx = 1;
    TSU_DISPATCH(prec, cell_speed_kernel, <<<dim3(bx, by), 256, 0, st>>>(L, list, nlist, cur, g, drytol, smax));
    return (int)cudaGetLastError();
}

int k_post_level(const CtrlView &cv, int level, int nscen, double R, double dx, double dy, double cfl_max,
                 double cfl_desired, int mode,
                 cudaStream_t st, int end_step)
{
    post_level_kernel<<<1, 128, 0, st>>>(cv, level, nscen, R, dx, dy, cfl_max, cfl_desired, mode,
                                         (mode == 0 || mode == 3) ? end_step : 0);
    return (int)cudaGetLastError();
}

int k_begin_step(const CtrlView &cv, int nscen, int nlev, const double *Rl, double cfl_desired, double dt_max,
                 cudaStream_t st)
{
    begin_step_kernel<<<1, 128, 0, st>>>(cv, nscen, nlev, Rl, cfl_desired, dt_max);
    return (int)cudaGetLastError();
}

int k_end_step(const CtrlView &cv, int nscen, cudaStream_t st)
{
    end_step_kernel<<<1, 128, 0, st>>>(cv, nscen);
    return (int)cudaGetLastError();
}

int k_gauges(int prec, const GaugeArgs &ga, const CtrlView &cv, cudaStream_t st)
{
    TSU_DISPATCH(prec, gauge_kernel, <<<1, 256, 0, st>>>(ga, cv));
    return (int)cudaGetLastError();
}

int k_read_field(int prec, const LevelView &L, int npatch, int maxpts, int cur, int scen, int field, double *dst, int nx,
                 int ny, double x0, double y0, double dx, double dy, double X0, double Y0, double dxl, double dyl,
                 cudaStream_t st)
{
    if (npatch <= 0) return 0;
    dim3 g = grid_for(maxpts, npatch, 128);
    TSU_DISPATCH(prec, read_field_kernel,
                 <<<g, 128, 0, st>>>(L, cur, scen, field, dst, nx, ny, x0, y0, dx, dy, X0, Y0, dxl, dyl));
    return (int)cudaGetLastError();
}

__global__ void fill_kernel(double *p, long long n, double v)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        p[k] = v;
}

int k_fill(double *p, long long n, double v, cudaStream_t st)
{
    if (n <= 0) return 0;
    long long b = (n + 255) / 256;
    fill_kernel<<<(int)(b < 152 * 8 ? b : 152 * 8), 256, 0, st>>>(p, n, v);
    return (int)cudaGetLastError();
}

int k_patch_out(int prec, const LevelView &L, int p, int ncells, int cur, double *out, cudaStream_t st)
{
    int blocks = (ncells + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    if (blocks < 1) blocks = 1;
    TSU_DISPATCH(prec, patch_out_kernel, <<<blocks, 256, 0, st>>>(L, p, cur, out));
    return (int)cudaGetLastError();
}

int k_cnn_features(int prec, const LevelView &L, int npatch, int maxcells, int cur, const int *scen_slot,
                   const uint8_t *raw, float *feat, double drytol, const CnnWindow &win, cudaStream_t st)
{
    if (npatch <= 0) return 0;
    dim3 g = grid_for(maxcells, npatch, 128);
    TSU_DISPATCH(prec, cnn_features_kernel, <<<g, 128, 0, st>>>(L, cur, scen_slot, raw, feat, drytol, win));
    return (int)cudaGetLastError();
}

int k_cnn_union(uint8_t *raw, const uint8_t *cov, const float *logits, int nx, int ny, int np, const CnnWindow &win,
                cudaStream_t st)
{
    long long n = (long long)win.tw * win.th * np;
    if (n <= 0) return 0;
    long long b = (n + 255) / 256;
    if (b > 152 * 32) b = 152 * 32;
    cnn_union_kernel<<<(int)(b < 1 ? 1 : b), 256, 0, st>>>(raw, cov, logits, nx, ny, np, win);
    return (int)cudaGetLastError();
}

int k_mass_parts(int npatch, int maxcells) { return npatch * (int)grid_for(maxcells, npatch, 256).y; }

int k_mass(int prec, const LevelView &L, int npatch, int maxcells, int cur, double *parts, double *mass, int nscen,
           cudaStream_t st)
{
    if (npatch <= 0) return 0;
    dim3 g = grid_for(maxcells, npatch, 256);
    TSU_DISPATCH(prec, mass_kernel, <<<g, 256, 0, st>>>(L, cur, parts));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return (int)e;
    mass_sum_kernel<<<(nscen + 127) / 128, 128, 0, st>>>(L.descs, npatch, (int)g.y, parts, mass, nscen);
    return (int)cudaGetLastError();
}

int k_halo(int prec, const LevelView &L, const HaloMsg *msgs, int n, int cur, void *buf, int unpack, cudaStream_t st)
{
    if (n <= 0) return 0;
    if (unpack) {
        if (prec == 0) halo_unpack_kernel<double, false><<<n, 128, 0, st>>>(L, msgs, cur, (const double *)buf);
        else halo_unpack_kernel<float, true><<<n, 128, 0, st>>>(L, msgs, cur, (const float *)buf);
    } else {
        if (prec == 0) halo_pack_kernel<double, false><<<n, 128, 0, st>>>(L, msgs, cur, (double *)buf);
        else halo_pack_kernel<float, true><<<n, 128, 0, st>>>(L, msgs, cur, (float *)buf);
    }
    return (int)cudaGetLastError();
}

}  // namespace tsu
