// step_kernel.cuh -- one dimensionally split wave-propagation step of every
// patch of a level in one launch (Sec. 2.2 Eqs. wave_propagation_2nd_order_x
// then _y), with the per-patch CFL wave-speed reduction fused in.
//
// Per CTA: a strip of W = NT - 4 columns of one patch and a segment of rows.
// The CTA streams down the rows:
//   * row r (W + 4 cells of q0, q1, q2, B) is prefetched into a ring of
//     shared-memory slots with cp.async, RING - 1 rows ahead, so every
//     state value is read from HBM once (plus the 4-row / 4-column halo);
//   * x sweep of row r: thread t solves the Riemann problem of x-edge t
//     (between ring cells t and t+1) and publishes its f-waves; after a
//     barrier it limits them with the upwind neighbour's waves (Eq. theta,
//     MC limiter), publishes A+dQ and the correction flux, and after a second
//     barrier updates cell t from its own A-dQ / correction (registers) and
//     its left neighbour's A+dQ / correction (shared memory) -- the
//     edge-then-cell thread mapping of Sec. 4.3.3, no redundant solves;
//   * the same thread owns column t for the y sweep: Q* of rows r-2 .. r and
//     the y-edge waves of rows r-2 .. r stay in its registers, so the y sweep
//     needs neither shared memory nor barriers and Q* never goes to HBM --
//     the x and y sweeps are fused in one kernel;
//   * the max |s| of the edges touching interior cells is reduced with warp
//     shuffles, then one atomicMax per CTA (Sec. 4.3 reduction).
// GEO: latitude-longitude grid in capacity form (Sec. 2.1 spherical
// coordinates; LeVeque's capacity-form wave propagation): row j has capacity
// kap_j, the latitude edge below it the relative length ced_j.  The x sweep of
// row j runs with dt / (kap_j dx) and reports speeds / kap_j; each y-edge's
// fluctuations and correction flux are weighted by ced_e, its Courant number
// uses dt ced_e / (kbar_e dy) (kbar_e the mean capacity of its two cells), the
// cell update divides by kap_j, and the mass gets the term
// (ced_{j+1} - ced_j) hv_j of the varying edge length.
// The arithmetic of riemann()/limit() follows the FP64 oracle operation by
// operation; the FP64 instantiation is compiled without contraction so the
// two agree to the last bit.
#pragma once
#include <cuda_runtime.h>
#include "tsu_device.h"

namespace tsu {

template <typename T> struct Wave {
    T Z[3][3];   // f-wave p, component (mass, normal, transverse)
    T s[3];
    int wall;    // 1: left side replaced by the wall mirror, 2: right side
};

template <typename T> __device__ __forceinline__ T dsqrt(T x);
template <> __device__ __forceinline__ double dsqrt<double>(double x) { return sqrt(x); }
template <> __device__ __forceinline__ float dsqrt<float>(float x) { return sqrtf(x); }
template <typename T> __device__ __forceinline__ T dmin(T a, T b);
template <> __device__ __forceinline__ double dmin<double>(double a, double b) { return fmin(a, b); }
template <> __device__ __forceinline__ float dmin<float>(float a, float b) { return fminf(a, b); }
template <typename T> __device__ __forceinline__ T dmax(T a, T b);
template <> __device__ __forceinline__ double dmax<double>(double a, double b) { return fmax(a, b); }
template <> __device__ __forceinline__ float dmax<float>(float a, float b) { return fmaxf(a, b); }
template <typename T> __device__ __forceinline__ T dabs(T a);
template <> __device__ __forceinline__ double dabs<double>(double a) { return fabs(a); }
template <> __device__ __forceinline__ float dabs<float>(float a) { return fabsf(a); }

// One cell as seen by a normal-direction Riemann problem: stored state (q0 is
// h, or eta' in the perturbation form), bed, and the quantities derived from
// it once per sweep -- depth, velocities, sqrt(g h), sqrt(h).
template <typename T> struct Cell {
    T q0, hn, ht, B;
    T h, u, v, c, sq;
    bool wet;
};

template <typename T, bool PERT>
__device__ __forceinline__ void derive(Cell<T> &z, T g, T drytol)
{
    z.h = PERT ? z.q0 - z.B : z.q0;
    z.wet = z.h >= drytol;
    z.u = T(0); z.v = T(0); z.c = T(0); z.sq = T(0);
    if (z.wet) {
        z.u = z.hn / z.h;
        z.v = z.ht / z.h;
        z.c = dsqrt<T>(g * z.h);
        z.sq = dsqrt<T>(z.h);
    }
}

// Normal-direction Riemann solver.  Augmented HLLE-type f-wave decomposition
// with the bathymetry source folded into the momentum flux jump,
// Einfeldt-type speeds from Roe averages, dry-bed speeds, a reflecting wall
// where a dry bed lies above the wet side's middle-state surface, a bed-step
// depth jump bounded so every state of the fan keeps h >= 0 (Sec. 2.2), and a
// contact wave at the Roe speed for the transverse momentum.
template <typename T, bool PERT>
__device__ __forceinline__ void riemann(const T g, const Cell<T> &cl, const Cell<T> &cr, Wave<T> &r)
{
    const T zero = T(0);
    r.wall = 0;
    if (!cl.wet && !cr.wet) {
#pragma unroll
        for (int p = 0; p < 3; p++) {
            r.s[p] = zero;
#pragma unroll
            for (int m = 0; m < 3; m++) r.Z[p][m] = zero;
        }
        return;
    }
    T qL = cl.q0, hnL = cl.hn, BL = cl.B, hL = cl.h, uL = cl.u, vL = cl.v, cL = cl.c, sqL = cl.sq;
    T qR = cr.q0, hnR = cr.hn, BR = cr.B, hR = cr.h, uR = cr.u, vR = cr.v, cR = cr.c, sqR = cr.sq;
    bool wetL = cl.wet, wetR = cr.wet;
    if (wetL && !wetR) {
        T a = cL + T(0.5) * uL;
        T hm = a > zero ? a * a / g : zero;
        if (hm + BL <= BR) {
            r.wall = 2;
            hR = hL; hnR = -hnL; BR = BL; uR = -uL; vR = vL; wetR = true; qR = qL; cR = cL; sqR = sqL;
        }
    } else if (!wetL && wetR) {
        T a = cR - T(0.5) * uR;
        T hm = a > zero ? a * a / g : zero;
        if (hm + BR <= BL) {
            r.wall = 1;
            hL = hR; hnL = -hnR; BL = BR; uL = -uR; vL = vR; wetL = true; qL = qR; cL = cR; sqL = sqR;
        }
    }

    T s1, s2, s3;
    if (wetL && wetR) {
        T uhat = (sqL * uL + sqR * uR) / (sqL + sqR);
        T chat = dsqrt<T>(g * (T(0.5) * (hL + hR)));
        s1 = dmin<T>(uL - cL, uhat - chat);
        s3 = dmax<T>(uR + cR, uhat + chat);
        s2 = uhat;
    } else if (wetL) {
        s1 = uL - cL;
        s3 = uL + T(2) * cL;
        s2 = uL;
    } else {
        s1 = uR - T(2) * cR;
        s3 = uR + cR;
        s2 = uR;
    }

    T hbar = T(0.5) * (hL + hR);
    T deta = PERT ? qR - qL : (hR + BR) - (hL + BL);
    T d2 = hnR - hnL;
    T d3 = (hnR * uR - hnL * uL) + (g * hbar) * deta;
    T d4 = hnR * vR - hnL * vL;
    T den = s3 - s1;
    // Non-negative depth: the bed step is a stationary wave across which the
    // depth jumps by delta (BL - BR keeps still water still).  With
    // M = s3 hR - s1 hL - d(hu), the fan's constant states have depths
    //   s1 < 0 < s3: (M - s3 delta)/den and (M - s1 delta)/den either side of x = 0;
    //   s1 >= 0:     hL + delta, then (M - s1 delta)/den;
    //   s3 <= 0:     (M - s3 delta)/den, then hR - delta.
    // A delta that would make one negative is moved to make it zero, and the
    // acoustic waves carry dh - delta instead of d(eta).
    T M = (s3 * hR - s1 * hL) - d2;
    T delta = BL - BR;
    bool bounded = false;
    if (s1 < zero && s3 > zero) {
        if (M - s3 * delta < zero) { delta = M / s3; bounded = true; }
        else if (M - s1 * delta < zero) { delta = M / s1; bounded = true; }
    } else if (s1 >= zero) {
        if (hL + delta < zero) { delta = -hL; bounded = true; }
        else if (s1 > zero && M - s1 * delta < zero) { delta = M / s1; bounded = true; }
    } else {
        if (hR - delta < zero) { delta = hR; bounded = true; }
        else if (s3 < zero && M - s3 * delta < zero) { delta = M / s3; bounded = true; }
    }
    T d1 = bounded ? (hR - hL) - delta : deta;
    T w1m = (s3 * d1 - d2) / den;
    T w1n = (s3 * d2 - d3) / den;
    T b1 = s1 * w1m, g1 = s1 * w1n;
    T b3 = s3 * (d1 - w1m), g3 = s3 * (d2 - w1n);

    r.Z[0][0] = b1; r.Z[0][1] = g1; r.Z[0][2] = b1 * vL;
    r.Z[2][0] = b3; r.Z[2][1] = g3; r.Z[2][2] = b3 * vR;
    r.Z[1][0] = zero; r.Z[1][1] = zero; r.Z[1][2] = (d4 - b1 * vL) - b3 * vR;
    r.s[0] = s1; r.s[1] = s2; r.s[2] = s3;
}

template <typename T> __device__ __forceinline__ T wleft(T s) { return s < T(0) ? T(1) : (s == T(0) ? T(0.5) : T(0)); }
template <typename T> __device__ __forceinline__ T wright(T s) { return s > T(0) ? T(1) : (s == T(0) ? T(0.5) : T(0)); }

template <typename T> __device__ __forceinline__ T mc_limiter(T theta)
{
    T t = T(0.5) * (T(1) + theta);
    t = dmin<T>(t, T(2));
    t = dmin<T>(t, T(2) * theta);
    return dmax<T>(T(0), t);
}

// Fluctuations and limited correction flux of one edge.  ZI[p][m]: the f-waves
// of the upwind neighbour chosen per wave (I = i-1 if s >= 0, else i+1).
template <typename T>
__device__ __forceinline__ void limit(const Wave<T> &r, const T (&ZI)[3][3], T dtdx,
                                      T (&amdq)[3], T (&apdq)[3], T (&F)[3])
{
    T wl0 = wleft<T>(r.s[0]), wl1 = wleft<T>(r.s[1]), wl2 = wleft<T>(r.s[2]);
    T wr0 = wright<T>(r.s[0]), wr1 = wright<T>(r.s[1]), wr2 = wright<T>(r.s[2]);
#pragma unroll
    for (int m = 0; m < 3; m++) {
        amdq[m] = (wl0 * r.Z[0][m] + wl1 * r.Z[1][m]) + wl2 * r.Z[2][m];
        apdq[m] = (wr0 * r.Z[0][m] + wr1 * r.Z[1][m]) + wr2 * r.Z[2][m];
    }
    if (r.wall == 2) { apdq[0] = T(0); apdq[1] = T(0); apdq[2] = T(0); }
    if (r.wall == 1) { amdq[0] = T(0); amdq[1] = T(0); amdq[2] = T(0); }
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
    for (int m = 0; m < 3; m++)
        F[m] = T(0.5) * ((c[0] * r.Z[0][m] + c[1] * r.Z[1][m]) + c[2] * r.Z[2][m]);
}

template <typename T, bool PERT>
__device__ __forceinline__ void postprocess(T &q0, T &qn, T &qt, T B, T drytol)
{
    if (PERT) {
        T h = q0 - B;
        if (h < T(0)) { q0 = B; h = T(0); }
        if (h < drytol) { qn = T(0); qt = T(0); }
    } else {
        if (q0 < T(0)) q0 = T(0);
        if (q0 < drytol) { qn = T(0); qt = T(0); }
    }
}

// Manning friction of one updated cell (Sec. 2.1 drag, read with the momentum
// magnitude: D = n^2 g sqrt(hu^2 + hv^2) / h^(7/3)), implicit in the
// momentum: hu, hv <- hu, hv / (1 + dt D) on a wet cell.  coef = n^2 g.
template <typename T> __device__ __forceinline__ T dpow(T x, T y);
template <> __device__ __forceinline__ double dpow<double>(double x, double y) { return pow(x, y); }
template <> __device__ __forceinline__ float dpow<float>(float x, float y) { return powf(x, y); }
template <typename T, bool PERT>
__device__ __forceinline__ void friction(T q0, T &hu, T &hv, T B, T drytol, T coef, T dt)
{
    const T h = PERT ? q0 - B : q0;
    if (!(h >= drytol)) return;
    const T D = (coef * dpow<T>(h, T(-7.0 / 3.0))) * dsqrt<T>(hu * hu + hv * hv);
    const T f = T(1) + dt * D;
    hu = hu / f;
    hv = hv / f;
}

__device__ __forceinline__ void cp_async_elem(void *smem, const void *gmem, int bytes)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    if (bytes == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Bulk copies into shared memory completing on an mbarrier (one thread arms
// the barrier with the bytes to expect and issues the copies; every consumer
// polls the phase).  Waits are bounded: mbar_wait gives up after `polls` tests.
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long *b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
// makes initialised barriers visible to the bulk copies (the async proxy)
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *b, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
// bytes (a multiple of 16) from 16-byte aligned global src to 16-byte aligned shared dst
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *b)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(b))
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long *b, unsigned parity)
{
    unsigned r;
    asm volatile("{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(r)
                 : "r"(smem_u32(b)), "r"(parity)
                 : "memory");
    return r != 0;
}
// true once the phase of the given parity has completed; false if it has not
// after `polls` tests
__device__ __forceinline__ bool mbar_wait(unsigned long long *b, unsigned parity, unsigned polls)
{
    for (unsigned i = 0; i < polls; i++)
        if (mbar_test(b, parity)) return true;
    return false;
}
// polls of the final wait for copies still in flight after a wait gave up
constexpr unsigned kDrainPolls = 1u << 26;

__device__ __forceinline__ void atomic_max_speed(unsigned long long *dst, double v)
{
    atomicMax(dst, (unsigned long long)__double_as_longlong(v));
}

template <typename T> __device__ __forceinline__ const T *geo_table(const double *d, const float *f);
template <> __device__ __forceinline__ const double *geo_table<double>(const double *d, const float *) { return d; }
template <> __device__ __forceinline__ const float *geo_table<float>(const double *, const float *f) { return f; }

template <typename T, bool PERT, int NT, int RING, bool GEO = false>
__global__ void __launch_bounds__(NT) step_kernel(StepArgs a)
{
    static_assert(RING >= 3, "the derived values of row k+1 need its copy complete at iteration k");
    __shared__ T ring[RING][4][NT];
    __shared__ T sZ[9][NT];
    __shared__ T sAp[3][NT];
    __shared__ T sF[3][NT];
    __shared__ T sD[2][4][NT];     // derived u, v, c, sqrt(h) of the ring cells, by row parity
    __shared__ T red[2][NT / 32];

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

    const double dt = a.dt1[P.scen] / a.R;
    const T dtdx = (T)(dt / a.dx), dtdy = (T)(dt / a.dy);
    const T g = (T)a.g, drytol = (T)a.drytol;
    const int x0 = it.x0, y0 = it.y0, w = it.w, h = it.h;
    const int pitch = P.pitch;
    const int nrows = h + 4;
    // capacity of patch row j at kapP[j], relative length of the y-edge below it at cedP[j]
    const T *kapP = GEO ? geo_table<T>(a.kap, a.kapf) + (P.j0 + 2) : nullptr;
    const T *cedP = GEO ? geo_table<T>(a.ced, a.cedf) + (P.j0 + 2) : nullptr;
    // ring cell t <-> patch column x0 - 2 + t (storage column x0 + t)
    const bool loader = t < w + 4;
    const long long colofs = (long long)(x0 + t);

    auto prefetch = [&](int k) {
        if (k < nrows && loader) {
            int slot = k % RING;
            long long gi = (long long)(y0 + k) * pitch + colofs;  // storage row (y0 - 2 + k) + 2
            cp_async_elem(&ring[slot][0][t], qin0 + gi, sizeof(T));
            cp_async_elem(&ring[slot][1][t], qin1 + gi, sizeof(T));
            cp_async_elem(&ring[slot][2][t], qin2 + gi, sizeof(T));
            cp_async_elem(&ring[slot][3][t], Bg + gi, sizeof(T));
        }
        cp_async_commit();
    };
    // own ring cell of row k (x-sweep roles: normal hu, transverse hv), derived
    // and published for the left neighbour's edge
    auto own_cell = [&](int k, Cell<T> &z) {
        const int slot = k % RING;
        z.q0 = ring[slot][0][t]; z.hn = ring[slot][1][t]; z.ht = ring[slot][2][t]; z.B = ring[slot][3][t];
        derive<T, PERT>(z, g, drytol);
        sD[k & 1][0][t] = z.u; sD[k & 1][1][t] = z.v; sD[k & 1][2][t] = z.c; sD[k & 1][3][t] = z.sq;
    };

#pragma unroll
    for (int k = 0; k < RING - 1; k++) prefetch(k);
    Cell<T> xc;   // this thread's ring cell of the current row
    cp_async_wait<RING - 2>();
    if (loader) own_cell(0, xc);

    // y-sweep state of column t (valid for update threads 2 <= t < w + 2)
    Cell<T> ym1;                 // Q* of row r-1 with derived values (y roles)
    T qm2[3], Bm2 = T(0);
    Wave<T> yold, ymid;
    T yap[3] = {T(0), T(0), T(0)}, yF[3] = {T(0), T(0), T(0)};
    T smx = T(0), smy = T(0);
    const bool upd = t >= 2 && t < w + 2;
    const bool rsolve = t < w + 3;
    const bool lim = t >= 1 && t < w + 2;

    for (int k = 0; k < nrows; k++) {
        prefetch(k + RING - 1);
        cp_async_wait<RING - 2>();   // rows <= k+1 of this thread have landed
        __syncthreads();
        const int slot = k % RING;
        const int r = y0 - 2 + k;            // patch-local row of this iteration
        const bool rowint = r >= y0 && r < y0 + h;
        const T kr = GEO ? kapP[r] : T(1);
        const T dtdxr = GEO ? (T)(dt / (kr * a.dx)) : dtdx;

        // ---- x sweep: Riemann problem at edge t (ring cells t, t+1)
        Wave<T> xw;
        if (rsolve) {
            Cell<T> xr;
            xr.q0 = ring[slot][0][t + 1]; xr.hn = ring[slot][1][t + 1]; xr.ht = ring[slot][2][t + 1];
            xr.B = ring[slot][3][t + 1];
            xr.h = PERT ? xr.q0 - xr.B : xr.q0;
            xr.wet = xr.h >= drytol;
            xr.u = sD[k & 1][0][t + 1]; xr.v = sD[k & 1][1][t + 1]; xr.c = sD[k & 1][2][t + 1];
            xr.sq = sD[k & 1][3][t + 1];
            riemann<T, PERT>(g, xc, xr, xw);
#pragma unroll
            for (int p = 0; p < 3; p++)
#pragma unroll
                for (int m = 0; m < 3; m++) sZ[p * 3 + m][t] = xw.Z[p][m];
        }
        __syncthreads();

        T xam[3], xap[3], xF[3];
        if (lim) {
            T ZI[3][3];
#pragma unroll
            for (int p = 0; p < 3; p++) {
                int nb = xw.s[p] >= T(0) ? t - 1 : t + 1;
#pragma unroll
                for (int m = 0; m < 3; m++) ZI[p][m] = sZ[p * 3 + m][nb];
            }
            limit<T>(xw, ZI, dtdxr, xam, xap, xF);
#pragma unroll
            for (int m = 0; m < 3; m++) { sAp[m][t] = xap[m]; sF[m][t] = xF[m]; }
            if (rowint) {
                const T se = dmax<T>(-xw.s[0], xw.s[2]);
                smx = dmax<T>(smx, GEO ? se / kr : se);
            }
        }
        __syncthreads();

        if (upd) {
            // cell t: left edge t-1 (shared memory), right edge t (registers)
            T qs[3] = {xc.q0, xc.hn, xc.ht};
#pragma unroll
            for (int m = 0; m < 3; m++) {
                T u = (sAp[m][t - 1] + xam[m]) + (xF[m] - sF[m][t - 1]);
                qs[m] = qs[m] - dtdxr * u;
            }
            postprocess<T, PERT>(qs[0], qs[1], qs[2], xc.B, drytol);

            // ---- y sweep of column t: y-edge between rows r-1 and r
            Cell<T> yc;
            yc.q0 = qs[0]; yc.hn = qs[2]; yc.ht = qs[1]; yc.B = xc.B;
            derive<T, PERT>(yc, g, drytol);
            if (k >= 1) {
                Wave<T> ynew;
                riemann<T, PERT>(g, ym1, yc, ynew);
                if (k >= 3) {
                    // limit y-edge r-1 (ymid) with neighbours r-2 (yold) and r (ynew)
                    const int e = r - 1;
                    if (e >= y0 && e <= y0 + h) {
                        T ZI[3][3];
#pragma unroll
                        for (int p = 0; p < 3; p++)
#pragma unroll
                            for (int m = 0; m < 3; m++) ZI[p][m] = ymid.s[p] >= T(0) ? yold.Z[p][m] : ynew.Z[p][m];
                        T yam[3], yapn[3], yFn[3];
                        T dtdye = dtdy, cratio = T(1);
                        if (GEO) {
                            const T kbar = T(0.5) * (kapP[e - 1] + kapP[e]);
                            dtdye = ((T)dt * cedP[e]) / (kbar * (T)a.dy);
                            cratio = cedP[e] / kbar;
                        }
                        limit<T>(ymid, ZI, dtdye, yam, yapn, yFn);
                        const T se = dmax<T>(-ymid.s[0], ymid.s[2]);
                        smy = dmax<T>(smy, GEO ? se * cratio : se);
                        const int rc = r - 2;   // cell between y-edges r-2 and r-1
                        if (rc >= y0 && rc < y0 + h) {
                            T qn[3] = {qm2[0], qm2[2], qm2[1]};   // (mass, normal = hv, transverse = hu)
                            if (GEO) {
                                const T clo = cedP[rc], chi = cedP[e];
                                const T dtk = (T)dt / (kapP[rc] * (T)a.dy);
                                const T hv = qm2[2];
#pragma unroll
                                for (int m = 0; m < 3; m++) {
                                    T u = (clo * yap[m] + chi * yam[m]) + (chi * yFn[m] - clo * yF[m]);
                                    if (m == 0) u = u + (chi - clo) * hv;
                                    qn[m] = qn[m] - dtk * u;
                                }
                            } else {
#pragma unroll
                                for (int m = 0; m < 3; m++) {
                                    T u = (yap[m] + yam[m]) + (yFn[m] - yF[m]);
                                    qn[m] = qn[m] - dtdy * u;
                                }
                            }
                            postprocess<T, PERT>(qn[0], qn[1], qn[2], Bm2, drytol);
                            if (a.manning > 0.0)   // y frame: qn[2] = hu, qn[1] = hv
                                friction<T, PERT>(qn[0], qn[2], qn[1], Bm2, drytol, (T)a.manning, (T)dt);
                            // a depth that is not a finite number reaches the host as an infinite speed
                            if (!(dabs<T>(qn[0]) < T(1e30))) smy = T(INFINITY);
                            long long gi = (long long)(rc + 2) * pitch + (x0 + t);
                            qo0[gi] = qn[0];
                            qo2[gi] = qn[1];
                            qo1[gi] = qn[2];
                        }
#pragma unroll
                        for (int m = 0; m < 3; m++) { yap[m] = yapn[m]; yF[m] = yFn[m]; }
                    }
                }
                yold = ymid;
                ymid = ynew;
            }
            qm2[0] = ym1.q0; qm2[1] = ym1.ht; qm2[2] = ym1.hn;
            Bm2 = ym1.B;
            ym1 = yc;
        }
        // derived values of this thread's cell in the next row (its own copy has landed)
        if (loader && k + 1 < nrows) own_cell(k + 1, xc);
    }

    // CTA max of the wave speeds: warp shuffles, then one atomic per CTA
    if (!(smx > T(0))) smx = T(0);
    if (!(smy > T(0))) smy = T(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        smx = dmax<T>(smx, __shfl_xor_sync(0xffffffffu, smx, o));
        smy = dmax<T>(smy, __shfl_xor_sync(0xffffffffu, smy, o));
    }
    if ((t & 31) == 0) { red[0][t >> 5] = smx; red[1][t >> 5] = smy; }
    __syncthreads();
    if (t == 0) {
        T mx = T(0), my = T(0);
        for (int k = 0; k < NT / 32; k++) { mx = dmax<T>(mx, red[0][k]); my = dmax<T>(my, red[1][k]); }
        atomic_max_speed(a.smax + 2 * P.scen + 0, (double)mx);
        atomic_max_speed(a.smax + 2 * P.scen + 1, (double)my);
    }
}

}  // namespace tsu
