// step_f32x2.cuh -- the FP32 surface-perturbation patch update with two
// columns per thread and Blackwell's paired FP32 arithmetic.
//
// The method is the dimensionally split update of Sec. 2.2 (x then y),
// fused: rows stream through a cp.async shared-memory ring, x-edge waves are
// exchanged through shared memory, and the y sweep of each column stays in
// registers, with the wave-speed reduction fused in.  The arithmetic is
// reorganised where FP32 rounding is held to the 1e-4 m surface bar rather
// than to the FP64 oracle's operation order:
//   * the wet-wet Riemann problem (the ocean) takes a short branch; dry beds,
//     walls and dry pairs take the general solver;
//   * fluctuations from the wave signs: A-dQ = (sum Z - sum sgn(s) Z) / 2,
//     A+dQ = (sum Z + sum sgn(s) Z) / 2 (a speed of 0 splits the wave in
//     half, as in the oracle);
//   * the contact wave has only a transverse component, so an edge publishes
//     7 wave components, and its limiter ratio is a quotient of scalars;
//   * no zero-norm test before theta = Z_I.Z / Z.Z: a zero wave contributes
//     0 to the correction whatever phi becomes (phi stays finite);
//   * phi / 2 = sat(min((1 + theta) / 4, theta)) is the MC limiter halved,
//     with the clamps to [0, 1] as one saturation.
// The work each thread carries:
//   * thread t owns the adjacent ring columns 2t and 2t+1 (lanes .x, .y of a
//     float2).  Both cells' fields come in with one 8-byte cp.async each, and
//     the thread solves the two x-edges to their left: 2t (cells 2t-1 | 2t)
//     and 2t+1 (cells 2t | 2t+1);
//   * every per-cell and per-edge formula runs on float2 with the paired
//     FP32 instructions (__ffma2_rn, __fadd2_rn, __fmul2_rn): one issue slot
//     for two edges or two cells.  Per-lane operations (reciprocal, square
//     root, min/max, compares, selects) stay scalar;
//   * exchange through shared memory shrinks: cell 2t's both edges are the
//     thread's own, so only the neighbours' outer edges cross threads (the
//     left cell of edge 2t, the upwind waves of edges 2t-1 and 2t+2, and
//     A-dQ + F~ of edge 2t+2);
//   * the y sweeps of the two columns run side by side in registers, paired
//     the same way.
// GEO: latitude-longitude grid in capacity form (Sec. 2.1 spherical
// coordinates): the x sweep of row j runs with dt / (kap_j dx) and reports
// speeds / kap_j; each y-edge's A-dQ, A+dQ and F~ are weighted by its relative
// length ced_e once, right after the limiter (its Courant number uses
// dt ced_e / (kbar_e dy), kbar_e the mean capacity of its two cells); the cell
// update divides by kap_j and adds (ced_{j+1} - ced_j) hv_j to the mass.
// Strip width W = 2 NT - 4 columns.  Registers are capped so that 12 warps fit
// on an SM (at the uncapped ~220 registers only 8 do and the kernel waits on
// latency; more than 12 spills).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include "step_kernel.cuh"

namespace tsu {
namespace x2 {

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b as one paired FMA
__device__ __forceinline__ float2 sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
// c - a b
__device__ __forceinline__ float2 fnma(float2 a, float2 b, float2 c)
{
    return __ffma2_rn(make_float2(-a.x, -a.y), b, c);
}
__device__ __forceinline__ float2 fmin2(float2 a, float2 b) { return make_float2(fminf(a.x, b.x), fminf(a.y, b.y)); }
__device__ __forceinline__ float2 fmax2(float2 a, float2 b) { return make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y)); }
__device__ __forceinline__ float2 rcp(float2 a) { return make_float2(__fdividef(1.0f, a.x), __fdividef(1.0f, a.y)); }
__device__ __forceinline__ float2 sqrt2(float2 a) { return make_float2(sqrtf(a.x), sqrtf(a.y)); }

// two cells in the roles of one sweep: q0 = eta', hn normal, ht transverse
// momentum, B; derived h, velocities, sqrt(g h), sqrt(h)
struct C2 {
    float2 q0, hn, ht, B;
    float2 h, u, v, c, sq;
    bool wx, wy;
};

// two edges' waves (layout of LWave, paired)
struct W2 {
    float2 z0m, z0n, z0t, z1t, z2m, z2n, z2t;
    float2 s0, s1, s2;
    int wallx, wally;
};

__device__ __forceinline__ void derive(C2 &z, float sqrtg, float drytol)
{
    z.h = sub(z.q0, z.B);
    z.wx = z.h.x >= drytol;
    z.wy = z.h.y >= drytol;
    float2 rh = make_float2(z.wx ? __fdividef(1.0f, z.h.x) : 0.0f, z.wy ? __fdividef(1.0f, z.h.y) : 0.0f);
    z.u = mul(z.hn, rh);
    z.v = mul(z.ht, rh);
    z.sq = make_float2(sqrtf(z.wx ? z.h.x : 0.0f), sqrtf(z.wy ? z.h.y : 0.0f));
    z.c = mul(f2(sqrtg), z.sq);
}

__device__ __forceinline__ void lane_in(const C2 &z, int l, Cell<float> &o)
{
    o.q0 = l ? z.q0.y : z.q0.x; o.hn = l ? z.hn.y : z.hn.x; o.ht = l ? z.ht.y : z.ht.x; o.B = l ? z.B.y : z.B.x;
    o.h = l ? z.h.y : z.h.x; o.u = l ? z.u.y : z.u.x; o.v = l ? z.v.y : z.v.x; o.c = l ? z.c.y : z.c.x;
    o.sq = l ? z.sq.y : z.sq.x; o.wet = l ? z.wy : z.wx;
}

// the general solver on lane l (0: x, 1: y) of two edges, into that lane of r
__device__ __forceinline__ void riemann2_lane(float g, const C2 &L, const C2 &R, int l, W2 &r)
{
    Cell<float> a, b;
    lane_in(L, l, a);
    lane_in(R, l, b);
    Wave<float> w;
    riemann<float, true>(g, a, b, w);
    if (l == 0) {
        r.z0m.x = w.Z[0][0]; r.z0n.x = w.Z[0][1]; r.z0t.x = w.Z[0][2]; r.z1t.x = w.Z[1][2];
        r.z2m.x = w.Z[2][0]; r.z2n.x = w.Z[2][1]; r.z2t.x = w.Z[2][2];
        r.s0.x = w.s[0]; r.s1.x = w.s[1]; r.s2.x = w.s[2];
        r.wallx = w.wall;
    } else {
        r.z0m.y = w.Z[0][0]; r.z0n.y = w.Z[0][1]; r.z0t.y = w.Z[0][2]; r.z1t.y = w.Z[1][2];
        r.z2m.y = w.Z[2][0]; r.z2n.y = w.Z[2][1]; r.z2t.y = w.Z[2][2];
        r.s0.y = w.s[0]; r.s1.y = w.s[1]; r.s2.y = w.s[2];
        r.wally = w.wall;
    }
}

// Riemann problems of two edges (L[i] | R[i]) for lanes i = x, y.  The
// wet-wet short branch runs paired on both lanes; a lane keeps its result
// when both its cells are wet, it is subsonic (s1 < 0 < s3) and the middle
// depths either side of the bed step with the still-water jump, hL + W1 and
// hR - W3, are positive (the depth bound is not needed).  Any other lane is
// solved again by the general solver.  The choice is made per edge, so an
// edge's waves do not depend on which edge shares its pair.
__device__ __forceinline__ void riemann2(float g, const C2 &L, const C2 &R, W2 &r)
{
    const float2 num = fma(L.sq, L.u, mul(R.sq, R.u));
    const float2 uhat = mul(num, rcp(add(L.sq, R.sq)));
    const float2 hbar = mul(f2(0.5f), add(L.h, R.h));
    const float2 ghb = mul(f2(g), hbar);
    const float2 chat = sqrt2(ghb);
    const float2 s1 = fmin2(sub(L.u, L.c), sub(uhat, chat));
    const float2 s3 = fmax2(add(R.u, R.c), add(uhat, chat));
    const float2 d1 = sub(R.q0, L.q0);
    const float2 d2 = sub(R.hn, L.hn);
    const float2 d3 = fma(ghb, d1, sub(mul(R.hn, R.u), mul(L.hn, L.u)));
    const float2 d4 = sub(mul(R.hn, R.v), mul(L.hn, L.v));
    const float2 rden = rcp(sub(s3, s1));
    const float2 w1m = mul(sub(mul(s3, d1), d2), rden);
    const float2 w1n = mul(sub(mul(s3, d2), d3), rden);
    const float2 w3m = sub(d1, w1m);
    const float2 hl = add(L.h, w1m), hr = sub(R.h, w3m);
    const bool okx = L.wx && R.wx && fminf(fminf(hl.x, hr.x), fminf(-s1.x, s3.x)) > 0.0f;
    const bool oky = L.wy && R.wy && fminf(fminf(hl.y, hr.y), fminf(-s1.y, s3.y)) > 0.0f;
    r.z0m = mul(s1, w1m); r.z0n = mul(s1, w1n); r.z0t = mul(r.z0m, L.v);
    r.z2m = mul(s3, w3m); r.z2n = mul(s3, sub(d2, w1n)); r.z2t = mul(r.z2m, R.v);
    r.z1t = sub(sub(d4, r.z0t), r.z2t);
    r.s0 = s1; r.s1 = uhat; r.s2 = s3;
    r.wallx = 0; r.wally = 0;
    if (!okx) riemann2_lane(g, L, R, 0, r);
    if (!oky) riemann2_lane(g, L, R, 1, r);
}

__device__ __forceinline__ float sgnf(float s) { return s > 0.0f ? 1.0f : (s < 0.0f ? -1.0f : 0.0f); }
// half the MC limiter: phi / 2 = max(0, min((1 + th) / 4, 1, th)) = sat(min((1 + th) / 4, th))
__device__ __forceinline__ float2 mc_half(float2 th)
{
    const float2 a = fma(f2(0.25f), th, f2(0.25f));
    return make_float2(__saturatef(fminf(a.x, th.x)), __saturatef(fminf(a.y, th.y)));
}

// upwind neighbour waves per lane and family
struct I2 {
    float2 m0, n0, t0, t1, m2, n2, t2;
};

// fluctuations and limited correction flux of two edges (as llimit)
__device__ __forceinline__ void limit2(const W2 &r, const I2 &I, float2 dtdx, float2 (&am)[3], float2 (&ap)[3],
                                       float2 (&F)[3])
{
    const float2 g0 = make_float2(copysignf(1.0f, r.s0.x), copysignf(1.0f, r.s0.y));
    const float2 g1 = make_float2(sgnf(r.s1.x), sgnf(r.s1.y));
    const float2 g2 = make_float2(copysignf(1.0f, r.s2.x), copysignf(1.0f, r.s2.y));
    const float2 sm = add(r.z0m, r.z2m), sn = add(r.z0n, r.z2n), st = add(add(r.z0t, r.z1t), r.z2t);
    const float2 gm = fma(g0, r.z0m, mul(g2, r.z2m));
    const float2 gn = fma(g0, r.z0n, mul(g2, r.z2n));
    const float2 gt = fma(g0, r.z0t, fma(g1, r.z1t, mul(g2, r.z2t)));
    const float2 h = f2(0.5f);
    am[0] = mul(h, sub(sm, gm)); ap[0] = mul(h, add(sm, gm));
    am[1] = mul(h, sub(sn, gn)); ap[1] = mul(h, add(sn, gn));
    am[2] = mul(h, sub(st, gt)); ap[2] = mul(h, add(st, gt));
    const float2 n0 = fma(r.z0m, r.z0m, fma(r.z0n, r.z0n, mul(r.z0t, r.z0t)));
    const float2 n2 = fma(r.z2m, r.z2m, fma(r.z2n, r.z2n, mul(r.z2t, r.z2t)));
    const float2 d0 = fma(I.m0, r.z0m, fma(I.n0, r.z0n, mul(I.t0, r.z0t)));
    const float2 d2 = fma(I.m2, r.z2m, fma(I.n2, r.z2n, mul(I.t2, r.z2t)));
    const float2 ph0 = mc_half(mul(d0, rcp(n0)));
    const float2 ph1 = mc_half(mul(I.t1, rcp(r.z1t)));
    const float2 ph2 = mc_half(mul(d2, rcp(n2)));
    // c_p = 1/2 sgn(s)(1 - dt/dx |s|) phi = sgn(s)(1 - dt/dx |s|)(phi / 2), |s| = sgn(s) s
    const float2 mdt = make_float2(-dtdx.x, -dtdx.y);
    const float2 c0 = mul(g0, mul(fma(mdt, mul(g0, r.s0), f2(1.0f)), ph0));
    const float2 c1 = mul(g1, mul(fma(mdt, mul(g1, r.s1), f2(1.0f)), ph1));
    const float2 c2 = mul(g2, mul(fma(mdt, mul(g2, r.s2), f2(1.0f)), ph2));
    F[0] = fma(c0, r.z0m, mul(c2, r.z2m));
    F[1] = fma(c0, r.z0n, mul(c2, r.z2n));
    F[2] = fma(c0, r.z0t, fma(c1, r.z1t, mul(c2, r.z2t)));
    if (r.wallx | r.wally) {
        // a wall edge: no fluctuation into the dry side, no correction
#pragma unroll
        for (int m = 0; m < 3; m++) {
            if (r.wallx == 2) ap[m].x = 0.0f;
            if (r.wallx == 1) am[m].x = 0.0f;
            if (r.wallx) F[m].x = 0.0f;
            if (r.wally == 2) ap[m].y = 0.0f;
            if (r.wally == 1) am[m].y = 0.0f;
            if (r.wally) F[m].y = 0.0f;
        }
    }
}

// Manning friction of two updated cells (as friction() in step_kernel.cuh)
__device__ __forceinline__ void friction2(float2 q0, float2 &hu, float2 &hv, float2 B, float drytol, float coef,
                                          float dt)
{
    const float2 h = sub(q0, B);
    const float2 m2 = fma(hu, hu, mul(hv, hv));
    float fx = 1.0f, fy = 1.0f;
    if (h.x >= drytol) fx = fmaf(dt, coef * __powf(h.x, -7.0f / 3.0f) * sqrtf(m2.x), 1.0f);
    if (h.y >= drytol) fy = fmaf(dt, coef * __powf(h.y, -7.0f / 3.0f) * sqrtf(m2.y), 1.0f);
    const float2 r = make_float2(__fdividef(1.0f, fx), __fdividef(1.0f, fy));
    hu = mul(hu, r);
    hv = mul(hv, r);
}

// wet/dry post-processing of two updated cells (perturbation form)
__device__ __forceinline__ void post2(float2 &q0, float2 &qn, float2 &qt, float2 B, float drytol)
{
    const float2 h = sub(q0, B);
    if (h.x < 0.0f) q0.x = B.x;
    if (h.y < 0.0f) q0.y = B.y;
    if (!(h.x >= drytol)) { qn.x = 0.0f; qt.x = 0.0f; }
    if (!(h.y >= drytol)) { qn.y = 0.0f; qt.y = 0.0f; }
}

__device__ __forceinline__ float2 ld2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
__device__ __forceinline__ void st2(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }

}  // namespace x2

template <int NT, int RING, bool GEO = false>
__global__ void __launch_bounds__(NT, (12 * 32) / NT) step_kernel_f32x2(StepArgs a)
{
    using namespace x2;
    static_assert(RING >= 3, "the derived values of row k+1 need its copy complete at iteration k");
    constexpr int NC = 2 * NT;   // ring columns
    __shared__ __align__(16) float ring[RING][4][NC];
    __shared__ float sDb[2][4][NT];   // derived u, v, c, sqrt(h) of cell 2t+1, by row parity
    __shared__ float sZx[7][NT];      // waves of edge 2t
    __shared__ float sZy[7][NT];      // waves of edge 2t+1
    __shared__ float sP[3][NT];       // A-dQ + F~ of edge 2t
    __shared__ float red[2][NT / 32];

    const StepItem it = a.items[blockIdx.x];
    if (it.w > 2 * NT - 4 || it.w < 1 || it.h < 1) return;   // not a work item of this launch shape
    const PatchDesc P = a.descs[it.patch];
    if (a.gate != nullptr && a.gate[P.scen] == 0) return;   // not retaken (uniform over the CTA)
    const int t = threadIdx.x;
    const int cur = a.cur;
    float *base = reinterpret_cast<float *>(a.arena) + P.off;
    const float *qin0 = base + (long long)(cur * 3 + 0) * P.fs;
    float *qo0 = base + (long long)((1 - cur) * 3 + 0) * P.fs;
    const long long fs = P.fs;

    const float dt1 = a.dt1f[P.scen];
    const float dtdx = dt1 * a.rdx, dtdy = dt1 * a.rdy;
    const float2 dtdx2 = f2(dtdx), dtdy2 = f2(dtdy);
    // capacity of patch row j at kapP[j], relative length of the y-edge below it at cedP[j]
    const float *kapP = GEO ? a.kapf + (P.j0 + 2) : nullptr;
    const float *cedP = GEO ? a.cedf + (P.j0 + 2) : nullptr;
    const float g = a.gf, drytol = a.drytolf, sqrtg = a.sqrtgf;
    const int x0 = it.x0, y0 = it.y0, w = it.w, h = it.h;
    const int pitch = P.pitch;
    const int nrows = h + 4;
    const int ncols = w + 4;                     // ring columns loaded
    const int c0 = 2 * t;                        // this thread's first ring column
    // 8-byte transfers need every field row to start on an even element
    const bool v8 = ((reinterpret_cast<uintptr_t>(qin0) & 7) == 0) && ((pitch & 1) == 0) && ((fs & 1) == 0) &&
                    ((x0 & 1) == 0);
    const float *src = qin0 + (long long)y0 * pitch + (x0 + c0);
    const long long fo[4] = {0, fs, 2 * fs, (6 - cur * 3) * fs};   // q0, q1, q2, B relative to q0 of buffer cur

    auto prefetch = [&](int k) {
        if (k < nrows) {
            const int slot = k % RING;
            const float *s = src + (long long)k * pitch;
            if (c0 + 1 < ncols && v8) {
#pragma unroll
                for (int f = 0; f < 4; f++) cp_async_elem(&ring[slot][f][c0], s + fo[f], 8);
            } else if (c0 < ncols) {
                // past an odd last column the second slot repeats the first: a
                // stale slot could send the valid lane down the other Riemann path
                // (general instead of paired), which rounds differently
                const int c1 = c0 + 1 < ncols ? 1 : 0;
#pragma unroll
                for (int f = 0; f < 4; f++) {
                    cp_async_elem(&ring[slot][f][c0], s + fo[f], 4);
                    cp_async_elem(&ring[slot][f][c0 + 1], s + fo[f] + c1, 4);
                }
            }
        }
        cp_async_commit();
    };
    // this thread's two cells of row k in x roles; publishes cell 2t+1's derived values
    auto own_cells = [&](int k, C2 &z) {
        const int slot = k % RING;
        z.q0 = ld2(&ring[slot][0][c0]); z.hn = ld2(&ring[slot][1][c0]);
        z.ht = ld2(&ring[slot][2][c0]); z.B = ld2(&ring[slot][3][c0]);
        derive(z, sqrtg, drytol);
        sDb[k & 1][0][t] = z.u.y; sDb[k & 1][1][t] = z.v.y; sDb[k & 1][2][t] = z.c.y; sDb[k & 1][3][t] = z.sq.y;
    };

#pragma unroll
    for (int k = 0; k < RING - 1; k++) prefetch(k);
    C2 xc;
    cp_async_wait<RING - 2>();
    own_cells(0, xc);

    // lane validity
    const int tl = t > 0 ? t - 1 : 0, tr = t + 1 < NT ? t + 1 : NT - 1;
    const bool limx = c0 >= 2 && c0 <= w + 2, limy = c0 + 1 >= 2 && c0 + 1 <= w + 2;   // edges x0 .. x0+w
    const bool outx = c0 >= 2 && c0 < w + 2, outy = c0 + 1 >= 2 && c0 + 1 < w + 2;     // columns x0 .. x0+w-1
    const bool upd = outx || outy;
    const bool w8 = v8 && outx && outy;
    float *dst = qo0 + (long long)(y0 + 2) * pitch + (x0 + c0);
    const long long go[3] = {0, fs, 2 * fs};

    // y sweep state of the two columns (y roles: hn = hv, ht = hu): Q* cells of
    // rows r-2, r-1, the waves of y-edges r-2, r-1 and A+dQ - F~ of y-edge r-2
    C2 yq2, yq1, yq0;
    W2 ywo, ywm, ywn;
    float2 yDo[3], yDm[3];
#pragma unroll
    for (int m = 0; m < 3; m++) { yDo[m] = f2(0.0f); yDm[m] = f2(0.0f); }
    float smx = 0.0f, smy = 0.0f;

    // ring row k: ycm2, ycm1, ycur = Q* cells of rows r-2, r-1, r; wo, wm, wn =
    // waves of y-edges r-2, r-1, r; Do = A+dQ - F~ of y-edge r-2; Dm receives
    // that of y-edge r-1
    auto row = [&](const int k, const C2 &ycm2, const C2 &ycm1, C2 &ycur, const W2 &wo, const W2 &wm, W2 &wn,
                   const float2 (&Do)[3], float2 (&Dm)[3]) {
        prefetch(k + RING - 1);
        cp_async_wait<RING - 2>();
        __syncthreads();
        const int slot = k % RING;
        const int r = y0 - 2 + k;
        const bool rowint = r >= y0 && r < y0 + h;
        float rk = 1.0f;
        float2 dtdxr = dtdx2;
        if (GEO) {
            rk = 1.0f / kapP[r];
            dtdxr = f2(dtdx * rk);
        }

        // ---- x edges 2t (cells 2t-1 | 2t) and 2t+1 (cells 2t | 2t+1)
        C2 L;
        L.q0 = make_float2(ring[slot][0][c0 > 0 ? c0 - 1 : 0], xc.q0.x);
        L.hn = make_float2(ring[slot][1][c0 > 0 ? c0 - 1 : 0], xc.hn.x);
        L.ht = make_float2(ring[slot][2][c0 > 0 ? c0 - 1 : 0], xc.ht.x);
        L.B = make_float2(ring[slot][3][c0 > 0 ? c0 - 1 : 0], xc.B.x);
        L.h = sub(L.q0, L.B);
        L.wx = L.h.x >= drytol; L.wy = xc.wx;
        L.u = make_float2(sDb[k & 1][0][tl], xc.u.x); L.v = make_float2(sDb[k & 1][1][tl], xc.v.x);
        L.c = make_float2(sDb[k & 1][2][tl], xc.c.x); L.sq = make_float2(sDb[k & 1][3][tl], xc.sq.x);
        W2 xw;
        riemann2(g, L, xc, xw);
        sZx[0][t] = xw.z0m.x; sZx[1][t] = xw.z0n.x; sZx[2][t] = xw.z0t.x; sZx[3][t] = xw.z1t.x;
        sZx[4][t] = xw.z2m.x; sZx[5][t] = xw.z2n.x; sZx[6][t] = xw.z2t.x;
        sZy[0][t] = xw.z0m.y; sZy[1][t] = xw.z0n.y; sZy[2][t] = xw.z0t.y; sZy[3][t] = xw.z1t.y;
        sZy[4][t] = xw.z2m.y; sZy[5][t] = xw.z2n.y; sZy[6][t] = xw.z2t.y;
        __syncthreads();

        // ---- limit both edges.  Upwind of edge 2t: 2t-1 (thread t-1, lane y) or
        // 2t+1 (own lane y), both in sZy; upwind of edge 2t+1: 2t (own lane x)
        // or 2t+2 (thread t+1, lane x), both in sZx
        float2 xam[3], xap[3], xF[3];
        {
            I2 I;
            const int a0 = xw.s0.x >= 0.0f ? tl : t, a1 = xw.s1.x >= 0.0f ? tl : t, a2 = xw.s2.x >= 0.0f ? tl : t;
            const int b0 = xw.s0.y >= 0.0f ? t : tr, b1 = xw.s1.y >= 0.0f ? t : tr, b2 = xw.s2.y >= 0.0f ? t : tr;
            I.m0 = make_float2(sZy[0][a0], sZx[0][b0]);
            I.n0 = make_float2(sZy[1][a0], sZx[1][b0]);
            I.t0 = make_float2(sZy[2][a0], sZx[2][b0]);
            I.t1 = make_float2(sZy[3][a1], sZx[3][b1]);
            I.m2 = make_float2(sZy[4][a2], sZx[4][b2]);
            I.n2 = make_float2(sZy[5][a2], sZx[5][b2]);
            I.t2 = make_float2(sZy[6][a2], sZx[6][b2]);
            limit2(xw, I, dtdxr, xam, xap, xF);
            sP[0][t] = xam[0].x + xF[0].x; sP[1][t] = xam[1].x + xF[1].x; sP[2][t] = xam[2].x + xF[2].x;
            if (rowint) {
                if (limx) smx = fmaxf(smx, fmaxf(-xw.s0.x, xw.s2.x) * rk);
                if (limy) smx = fmaxf(smx, fmaxf(-xw.s0.y, xw.s2.y) * rk);
            }
        }
        __syncthreads();

        if (upd) {
            // cell 2t: edges 2t (lane x) and 2t+1 (lane y); cell 2t+1: edges 2t+1
            // (lane y) and 2t+2 (thread t+1, lane x)
            float2 q0 = xc.q0, q1 = xc.hn, q2 = xc.ht;
            {
                const float2 r0 = make_float2(xam[0].y + xF[0].y, sP[0][tr]);
                const float2 r1 = make_float2(xam[1].y + xF[1].y, sP[1][tr]);
                const float2 r2 = make_float2(xam[2].y + xF[2].y, sP[2][tr]);
                q0 = fnma(dtdxr, add(sub(xap[0], xF[0]), r0), q0);
                q1 = fnma(dtdxr, add(sub(xap[1], xF[1]), r1), q1);
                q2 = fnma(dtdxr, add(sub(xap[2], xF[2]), r2), q2);
            }
            post2(q0, q1, q2, xc.B, drytol);

            // ---- y sweep of the two columns: y-edge r between rows r-1 and r
            ycur.q0 = q0; ycur.hn = q2; ycur.ht = q1; ycur.B = xc.B;
            derive(ycur, sqrtg, drytol);
            if (k >= 1) {
                riemann2(g, ycm1, ycur, wn);
                if (k >= 3) {
                    const int e = r - 1;
                    if (e >= y0 && e <= y0 + h) {
                        I2 I;
                        const bool a0 = wm.s0.x >= 0.0f, a1 = wm.s1.x >= 0.0f, a2 = wm.s2.x >= 0.0f;
                        const bool b0 = wm.s0.y >= 0.0f, b1 = wm.s1.y >= 0.0f, b2 = wm.s2.y >= 0.0f;
                        I.m0 = make_float2(a0 ? wo.z0m.x : wn.z0m.x, b0 ? wo.z0m.y : wn.z0m.y);
                        I.n0 = make_float2(a0 ? wo.z0n.x : wn.z0n.x, b0 ? wo.z0n.y : wn.z0n.y);
                        I.t0 = make_float2(a0 ? wo.z0t.x : wn.z0t.x, b0 ? wo.z0t.y : wn.z0t.y);
                        I.t1 = make_float2(a1 ? wo.z1t.x : wn.z1t.x, b1 ? wo.z1t.y : wn.z1t.y);
                        I.m2 = make_float2(a2 ? wo.z2m.x : wn.z2m.x, b2 ? wo.z2m.y : wn.z2m.y);
                        I.n2 = make_float2(a2 ? wo.z2n.x : wn.z2n.x, b2 ? wo.z2n.y : wn.z2n.y);
                        I.t2 = make_float2(a2 ? wo.z2t.x : wn.z2t.x, b2 ? wo.z2t.y : wn.z2t.y);
                        float2 yam[3], yap[3], yF[3], S[3];
                        float2 dtdye = dtdy2;
                        float cr = 1.0f, ce = 1.0f;
                        if (GEO) {
                            ce = cedP[e];
                            cr = ce / (0.5f * (kapP[e - 1] + kapP[e]));
                            dtdye = f2(dtdy * cr);
                        }
                        limit2(wm, I, dtdye, yam, yap, yF);
                        if (outx) smy = fmaxf(smy, fmaxf(-wm.s0.x, wm.s2.x) * cr);
                        if (outy) smy = fmaxf(smy, fmaxf(-wm.s0.y, wm.s2.y) * cr);
                        if (GEO) {
                            const float2 ce2 = f2(ce);
#pragma unroll
                            for (int m = 0; m < 3; m++) { yam[m] = mul(ce2, yam[m]); yap[m] = mul(ce2, yap[m]); yF[m] = mul(ce2, yF[m]); }
                        }
#pragma unroll
                        for (int m = 0; m < 3; m++) { S[m] = add(yam[m], yF[m]); Dm[m] = sub(yap[m], yF[m]); }
                        const int rc = r - 2;
                        if (rc >= y0 && rc < y0 + h) {
                            // cell row r-2: (A+dQ - F~) of y-edge r-2 plus (A-dQ + F~) of y-edge r-1
                            float2 dtk = dtdy2, m0 = add(Do[0], S[0]);
                            if (GEO) {
                                dtk = f2(dtdy / kapP[rc]);
                                m0 = fma(f2(ce - cedP[rc]), ycm2.hn, m0);   // divergence of the edge length
                            }
                            float2 n0 = fnma(dtk, m0, ycm2.q0);
                            float2 n1 = fnma(dtk, add(Do[1], S[1]), ycm2.hn);
                            float2 n2 = fnma(dtk, add(Do[2], S[2]), ycm2.ht);
                            post2(n0, n1, n2, ycm2.B, drytol);
                            if (a.manningf > 0.0f)   // y frame: n2 = hu, n1 = hv
                                friction2(n0, n2, n1, ycm2.B, drytol, a.manningf, dt1 * a.rR);
                            // a surface that is not a finite number reaches the host as an infinite speed
                            if ((outx && !(fabsf(n0.x) < 1e30f)) || (outy && !(fabsf(n0.y) < 1e30f))) smy = INFINITY;
                            float *d = dst + (long long)(rc - y0) * pitch;
                            if (w8) {
                                st2(d + go[0], n0);
                                st2(d + go[2], n1);
                                st2(d + go[1], n2);
                            } else {
                                if (outx) { d[go[0]] = n0.x; d[go[2]] = n1.x; d[go[1]] = n2.x; }
                                if (outy) { d[go[0] + 1] = n0.y; d[go[2] + 1] = n1.y; d[go[1] + 1] = n2.y; }
                            }
                        }
                    }
                }
            }
        }
        if (k + 1 < nrows) own_cells(k + 1, xc);
    };

    for (int k = 0; k < nrows; k++) {
        row(k, yq2, yq1, yq0, ywo, ywm, ywn, yDo, yDm);
        yq2 = yq1; yq1 = yq0;
        ywo = ywm; ywm = ywn;
#pragma unroll
        for (int m = 0; m < 3; m++) yDo[m] = yDm[m];
    }
    cp_async_wait<0>();

    if (!(smx > 0.0f)) smx = 0.0f;
    if (!(smy > 0.0f)) smy = 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        smx = fmaxf(smx, __shfl_xor_sync(0xffffffffu, smx, o));
        smy = fmaxf(smy, __shfl_xor_sync(0xffffffffu, smy, o));
    }
    if ((t & 31) == 0) { red[0][t >> 5] = smx; red[1][t >> 5] = smy; }
    __syncthreads();
    if (t == 0) {
        float mx = 0.0f, my = 0.0f;
        for (int k = 0; k < NT / 32; k++) { mx = fmaxf(mx, red[0][k]); my = fmaxf(my, red[1][k]); }
        atomic_max_speed(a.smax + 2 * P.scen + 0, (double)mx);
        atomic_max_speed(a.smax + 2 * P.scen + 1, (double)my);
    }
}

}  // namespace tsu
