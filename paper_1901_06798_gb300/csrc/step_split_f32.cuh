// step_split_f32.cuh -- the FP32 surface-perturbation split step (Sec. 2.2,
// x sweep then y sweep) as two kernels, with Q* through a scratch copy in HBM.
//
// step_x_f32x2: one CTA per strip of 2 NT - 4 columns and a segment of rows,
//   ghost rows included (Q* is needed there by the y sweep).  Rows stream
//   through a cp.async ring as in the fused kernel, two columns per thread on
//   the paired FP32 instructions, x-edge waves exchanged in shared memory.  A
//   row needs no other row, so segments carry no halo rows.  It writes Q* of
//   its interior columns and reduces the max x wave speed of interior rows.
// step_y_f32x2: one CTA of 32 threads per strip of 64 columns (two per
//   thread) and a segment of interior rows; reads Q* and B of the segment plus
//   two rows above and below, runs the y sweep of its columns in registers
//   (no halo columns, no barriers) and writes Q^{n+1}.  Each thread streams
//   its own two columns through a cp.async ring in shared memory, YRING - 1
//   rows ahead, so the loads' latency hides behind the rows in flight.
//
// Against the fused kernel (step_f32x2.cuh) the split pays 24 B per cell more
// HBM traffic (Q* out and back in), which the 4096^2 update has room for: the
// fused kernel is bound by instruction issue and latency.  What the split
// saves is the recomputed halo work (4 rows per row segment, 4 columns per
// y strip) and the register pressure of carrying both sweeps: the x kernel
// runs at about 84 registers (24 warps per SM) instead of 168 (12).  The
// arithmetic per cell is the fused kernel's, operation for operation, so the
// two give the same bits.  GEO: latitude-longitude grid in capacity form, as
// in the fused kernel.
#pragma once
#include "step_f32x2.cuh"

namespace tsu {

template <int NT, int RING, bool GEO>
__global__ void __launch_bounds__(NT) step_x_f32x2(StepArgs a)
{
    using namespace x2;
    static_assert(RING >= 3, "the derived values of row k+1 need its copy complete at iteration k");
    constexpr int NC = 2 * NT;
    __shared__ __align__(16) float ring[RING][4][NC];
    __shared__ float sDb[2][4][NT];   // derived u, v, c, sqrt(h) of cell 2t+1, by row parity
    __shared__ float sZx[7][NT];      // waves of edge 2t
    __shared__ float sZy[7][NT];      // waves of edge 2t+1
    __shared__ float sP[3][NT];       // A-dQ + F~ of edge 2t
    __shared__ float red[NT / 32];

    const StepItem it = a.items[blockIdx.x];
    if (it.w > 2 * NT - 4 || it.w < 1 || it.h < 1) return;   // not a work item of this launch shape
    const PatchDesc P = a.descs[it.patch];
    if (a.gate != nullptr && a.gate[P.scen] == 0) return;   // not retaken (uniform over the CTA)
    const int t = threadIdx.x;
    const int cur = a.cur;
    float *base = reinterpret_cast<float *>(a.arena) + P.off;
    const float *qin0 = base + (long long)(cur * 3) * P.fs;
    float *qs0 = a.scratch + P.soff;   // Q*: eta', hu, hv at 0, fs, 2 fs
    const long long fs = P.fs;
    const float dt1 = a.dt1f[P.scen];
    const float dtdx = dt1 * a.rdx;
    const float *kapP = GEO ? a.kapf + (P.j0 + 2) : nullptr;
    const float g = a.gf, drytol = a.drytolf, sqrtg = a.sqrtgf;
    const int x0 = it.x0, y0 = it.y0, w = it.w;   // y0 may be -2: ghost rows are swept too
    const int pitch = P.pitch;
    const int nrows = it.h;
    const int ncols = w + 4;
    const int c0 = 2 * t;
    const bool v8 = ((reinterpret_cast<uintptr_t>(qin0) & 7) == 0) && ((pitch & 1) == 0) && ((fs & 1) == 0) &&
                    ((x0 & 1) == 0);
    // ring column c <-> patch column x0 - 2 + c (storage column x0 + c); patch row j at storage row j + 2
    const long long row0 = (long long)(y0 + 2) * pitch + (x0 + c0);
    const float *src = qin0 + row0;
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

    const int tl = t > 0 ? t - 1 : 0, tr = t + 1 < NT ? t + 1 : NT - 1;
    const bool limx = c0 >= 2 && c0 <= w + 2, limy = c0 + 1 >= 2 && c0 + 1 <= w + 2;   // edges x0 .. x0+w
    const bool outx = c0 >= 2 && c0 < w + 2, outy = c0 + 1 >= 2 && c0 + 1 < w + 2;     // columns x0 .. x0+w-1
    const bool upd = outx || outy;
    const bool w8 = v8 && outx && outy;
    float smx = 0.0f;

    for (int k = 0; k < nrows; k++) {
        prefetch(k + RING - 1);
        cp_async_wait<RING - 2>();
        __syncthreads();
        const int slot = k % RING;
        const int j = y0 + k;
        const bool rowint = j >= 0 && j < P.ny;
        float rk = 1.0f;
        float2 dtdxr = f2(dtdx);
        if (GEO) {
            rk = 1.0f / kapP[j];
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

        // ---- limit both edges (upwind neighbours as in the fused kernel)
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
            float2 q0 = xc.q0, q1 = xc.hn, q2 = xc.ht;
            const float2 r0 = make_float2(xam[0].y + xF[0].y, sP[0][tr]);
            const float2 r1 = make_float2(xam[1].y + xF[1].y, sP[1][tr]);
            const float2 r2 = make_float2(xam[2].y + xF[2].y, sP[2][tr]);
            q0 = fnma(dtdxr, add(sub(xap[0], xF[0]), r0), q0);
            q1 = fnma(dtdxr, add(sub(xap[1], xF[1]), r1), q1);
            q2 = fnma(dtdxr, add(sub(xap[2], xF[2]), r2), q2);
            post2(q0, q1, q2, xc.B, drytol);
            float *d = qs0 + row0 + (long long)k * pitch;
            if (w8) {
                st2(d, q0); st2(d + fs, q1); st2(d + 2 * fs, q2);
            } else {
                if (outx) { d[0] = q0.x; d[fs] = q1.x; d[2 * fs] = q2.x; }
                if (outy) { d[1] = q0.y; d[fs + 1] = q1.y; d[2 * fs + 1] = q2.y; }
            }
        }
        if (k + 1 < nrows) own_cells(k + 1, xc);
    }
    cp_async_wait<0>();

    if (!(smx > 0.0f)) smx = 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) smx = fmaxf(smx, __shfl_xor_sync(0xffffffffu, smx, o));
    if ((t & 31) == 0) red[t >> 5] = smx;
    __syncthreads();
    if (t == 0) {
        float mx = 0.0f;
        for (int q = 0; q < NT / 32; q++) mx = fmaxf(mx, red[q]);
        atomic_max_speed(a.smax + 2 * P.scen + 0, (double)mx);
    }
}

// threads per CTA of the y kernel: one warp, two columns per thread
constexpr int kSplitYThreads = 32;
constexpr int kSplitYRing = 4;   // rows in flight per thread

template <bool GEO>
__global__ void __launch_bounds__(kSplitYThreads) step_y_f32x2(StepArgs a)
{
    using namespace x2;
    constexpr int NT = kSplitYThreads, YRING = kSplitYRing;
    // ring[slot][field][2 t .. 2 t + 1]: fields Q* eta', hu, hv and B; thread t
    // only ever reads its own two columns, so its cp.async waits suffice
    __shared__ __align__(16) float ring[YRING][4][2 * NT];
    const StepItem it = a.items_y[blockIdx.x];
    if (it.w > 2 * NT || it.w < 1 || it.h < 1) return;   // uniform over the CTA
    const PatchDesc P = a.descs[it.patch];
    if (a.gate != nullptr && a.gate[P.scen] == 0) return;   // not retaken (uniform over the CTA)
    const int t = threadIdx.x;
    const int cur = a.cur;
    float *base = reinterpret_cast<float *>(a.arena) + P.off;
    const long long fs = P.fs;
    const float *qs0 = a.scratch + P.soff;
    const float *Bg = base + 6 * fs;
    float *qo0 = base + (long long)((1 - cur) * 3) * fs;
    const float dt1 = a.dt1f[P.scen];
    const float dtdy = dt1 * a.rdy;
    const float2 dtdy2 = f2(dtdy);
    const float *kapP = GEO ? a.kapf + (P.j0 + 2) : nullptr;
    const float *cedP = GEO ? a.cedf + (P.j0 + 2) : nullptr;
    const float g = a.gf, drytol = a.drytolf, sqrtg = a.sqrtgf;
    const int y0 = it.y0, h = it.h;
    const int pitch = P.pitch;
    const bool vx = 2 * t < it.w, vy = 2 * t + 1 < it.w;
    const int col = it.x0 + 2 * t;
    // patch row y0 - 2 + k of column col at storage [(y0 + k) * pitch + col + 2]
    const long long cbase = (long long)y0 * pitch + (col + 2);
    const bool w8 = vx && vy && ((reinterpret_cast<uintptr_t>(qs0 + cbase) & 7) == 0) &&
                    ((reinterpret_cast<uintptr_t>(qo0 + cbase) & 7) == 0) && ((pitch & 1) == 0) && ((fs & 1) == 0);
    const int nrows = h + 4;
    const float *fsrc[4] = {qs0, qs0 + fs, qs0 + 2 * fs, Bg};
    const int c0 = 2 * t;
    auto prefetch = [&](int k) {
        if (k < nrows) {
            const int slot = k % YRING;
            const long long o = cbase + (long long)k * pitch;
            if (w8) {
#pragma unroll
                for (int f = 0; f < 4; f++) cp_async_elem(&ring[slot][f][c0], fsrc[f] + o, 8);
            } else {
                if (vx) {
#pragma unroll
                    for (int f = 0; f < 4; f++) cp_async_elem(&ring[slot][f][c0], fsrc[f] + o, 4);
                }
                if (vy) {
#pragma unroll
                    for (int f = 0; f < 4; f++) cp_async_elem(&ring[slot][f][c0 + 1], fsrc[f] + o + 1, 4);
                }
            }
        }
        cp_async_commit();
    };
#pragma unroll
    for (int k = 0; k < YRING - 1; k++) prefetch(k);

    C2 yq2, yq1, yq0;
    W2 ywo, ywm, ywn;
    float2 yao[3], yfo[3], yam1[3], yfm1[3];
#pragma unroll
    for (int m = 0; m < 3; m++) { yao[m] = f2(0.0f); yfo[m] = f2(0.0f); yam1[m] = f2(0.0f); yfm1[m] = f2(0.0f); }
    float smy = 0.0f;

    // row k: ycm2, ycm1, ycur = Q* cells of rows r-2, r-1, r; wo, wm, wn = waves of
    // y-edges r-2, r-1, r; apo, Fo = A+dQ, F~ of y-edge r-2; apm, Fm receive those of r-1
    auto row = [&](const int k, const C2 &ycm2, const C2 &ycm1, C2 &ycur, const W2 &wo, const W2 &wm, W2 &wn,
                   const float2 (&apo)[3], const float2 (&Fo)[3], float2 (&apm)[3], float2 (&Fm)[3]) {
        const int r = y0 - 2 + k;
        prefetch(k + YRING - 1);
        cp_async_wait<YRING - 1>();   // row k of this thread has landed
        {
            const int slot = k % YRING;
            // lanes outside the strip read zeros: a dry cell whose results are not stored
            ycur.q0 = vx ? ld2(&ring[slot][0][c0]) : f2(0.0f);
            ycur.ht = vx ? ld2(&ring[slot][1][c0]) : f2(0.0f);
            ycur.hn = vx ? ld2(&ring[slot][2][c0]) : f2(0.0f);
            ycur.B = vx ? ld2(&ring[slot][3][c0]) : f2(0.0f);
            if (!vy) { ycur.q0.y = 0.0f; ycur.ht.y = 0.0f; ycur.hn.y = 0.0f; ycur.B.y = 0.0f; }
        }
        derive(ycur, sqrtg, drytol);
        if (k >= 1) {
            riemann2(g, ycm1, ycur, wn);
            if (k >= 3) {
                const int e = r - 1;   // y0 <= e <= y0 + h
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
                float2 yam[3];
                float2 dtdye = dtdy2;
                float cr = 1.0f, ce = 1.0f;
                if (GEO) {
                    ce = cedP[e];
                    cr = ce / (0.5f * (kapP[e - 1] + kapP[e]));
                    dtdye = f2(dtdy * cr);
                }
                limit2(wm, I, dtdye, yam, apm, Fm);
                if (vx) smy = fmaxf(smy, fmaxf(-wm.s0.x, wm.s2.x) * cr);
                if (vy) smy = fmaxf(smy, fmaxf(-wm.s0.y, wm.s2.y) * cr);
                if (GEO) {
                    const float2 ce2 = f2(ce);
#pragma unroll
                    for (int m = 0; m < 3; m++) { yam[m] = mul(ce2, yam[m]); apm[m] = mul(ce2, apm[m]); Fm[m] = mul(ce2, Fm[m]); }
                }
                const int rc = r - 2;
                if (rc >= y0) {   // rc < y0 + h always
                    // cell row r-2: y-edges r-2 (A+dQ, F~ from the last row) and r-1
                    float2 dtk = dtdy2, m0 = add(add(apo[0], yam[0]), sub(Fm[0], Fo[0]));
                    if (GEO) {
                        dtk = f2(dtdy / kapP[rc]);
                        m0 = fma(f2(ce - cedP[rc]), ycm2.hn, m0);   // divergence of the edge length
                    }
                    float2 n0 = fnma(dtk, m0, ycm2.q0);
                    float2 n1 = fnma(dtk, add(add(apo[1], yam[1]), sub(Fm[1], Fo[1])), ycm2.hn);
                    float2 n2 = fnma(dtk, add(add(apo[2], yam[2]), sub(Fm[2], Fo[2])), ycm2.ht);
                    post2(n0, n1, n2, ycm2.B, drytol);
                    if (a.manningf > 0.0f)   // y frame: n2 = hu, n1 = hv
                        friction2(n0, n2, n1, ycm2.B, drytol, a.manningf, dt1 * a.rR);
                    // a surface that is not a finite number reaches the host as an infinite speed
                    if ((vx && !(fabsf(n0.x) < 1e30f)) || (vy && !(fabsf(n0.y) < 1e30f))) smy = INFINITY;
                    float *d = qo0 + cbase + (long long)(k - 2) * pitch;
                    if (w8) {
                        st2(d, n0); st2(d + 2 * fs, n1); st2(d + fs, n2);
                    } else {
                        if (vx) { d[0] = n0.x; d[2 * fs] = n1.x; d[fs] = n2.x; }
                        if (vy) { d[1] = n0.y; d[2 * fs + 1] = n1.y; d[fs + 1] = n2.y; }
                    }
                }
            }
        }
    };

    for (int k = 0; k < nrows; k++) {
        row(k, yq2, yq1, yq0, ywo, ywm, ywn, yao, yfo, yam1, yfm1);
        yq2 = yq1; yq1 = yq0;
        ywo = ywm; ywm = ywn;
#pragma unroll
        for (int m = 0; m < 3; m++) { yao[m] = yam1[m]; yfo[m] = yfm1[m]; }
    }
    cp_async_wait<0>();

    if (!(smy > 0.0f)) smy = 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) smy = fmaxf(smy, __shfl_xor_sync(0xffffffffu, smy, o));
    if (t == 0) atomic_max_speed(a.smax + 2 * P.scen + 1, (double)smy);
}

}  // namespace tsu
