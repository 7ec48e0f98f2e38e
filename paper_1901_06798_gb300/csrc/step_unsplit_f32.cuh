// step_unsplit_f32.cuh -- the unsplit update with transverse corrections
// (corner transport upwind) in the FP32 surface-perturbation form.
//
// Same work items, thread roles, row pipeline and barriers as the generic
// kernel of step_unsplit.cuh (thread t owns ring column t, the CTA marches
// down the rows, cell (t, r-2) is updated at iteration k, patch row r); what
// changes is what goes through shared memory.
//
// The transverse split is linear in the fluctuation, and the two fluctuations
// that enter a cell through opposite edges meet the same eigenstructure, so
// their sum is split once: 4 splits per cell instead of 8.  Those sums are per
// cell, so a thread keeps its own x-edge's and its own column's terms in
// registers and publishes only what a neighbour needs:
//   * per x-edge t: A-dQ and A-dQ + 2F~ (thread t-1 adds them to its cell);
//   * per column t: the second-order y-fluctuations entering cell (t, r-2)
//     (threads t and t+1 split them for the x-edges on either side).
// Shared memory per thread falls from 109 to 61 floats, and the transverse
// terms are read from registers instead of a three-row shared ring.
#pragma once
#include "step_unsplit.cuh"

namespace tsu {

// tpart for FP32: the same three waves with 1/(2c) taken once per pair and the
// second wave's zero mass and normal components left out.
template <bool PLUS>
__device__ __forceinline__ void tpart_f32(const TEig<float> &e, float i2c, const float (&d)[3], float (&out)[3])
{
    if (!e.on) { out[0] = 0.f; out[1] = 0.f; out[2] = 0.f; return; }
    const float l1 = e.un - e.c, l3 = e.un + e.c;
    const float b1 = (l3 * d[0] - d[1]) * i2c;
    const float b3 = (d[1] - l1 * d[0]) * i2c;
    const float b2 = d[2] - e.ut * d[0];
    const float k1 = PLUS ? fmaxf(l1, 0.f) : fminf(l1, 0.f);
    const float k2 = PLUS ? fmaxf(e.un, 0.f) : fminf(e.un, 0.f);
    const float k3 = PLUS ? fmaxf(l3, 0.f) : fminf(l3, 0.f);
    const float kb1 = k1 * b1, kb3 = k3 * b3;
    out[0] = kb1 + kb3;
    out[1] = kb1 * l1 + kb3 * l3;
    out[2] = out[0] * e.ut + k2 * b2;
}

// shared-memory layout, in floats
template <int NT, int RING> struct UnsplitF32Smem {
    static constexpr int ring = 0;                    // [RING][4][NT] eta', hu, hv, B
    static constexpr int der = ring + RING * 4 * NT;  // [RING][4][NT] u, v, c, sqrt(h) (x roles)
    static constexpr int z = der + RING * 4 * NT;     // [9][NT] x-edge f-waves of the current row
    static constexpr int xa = z + 9 * NT;             // [6][NT] A-dQ, A-dQ + 2F~ of x-edge t, last limited row
    static constexpr int by = xa + 6 * NT;            // [3][NT] y-fluctuations entering (t, r-2), x frame
    static constexpr int fx = by + 3 * NT;            // [3][NT] transverse-corrected F of x-edge t
    static constexpr int red = fx + 3 * NT;           // [2][NT / 32] speed maxima
    static constexpr int total = red + 2 * (NT / 32);
};

template <int NT, int RING>
__global__ void __launch_bounds__(NT) step_unsplit_f32_kernel(StepArgs a)
{
    static_assert(RING >= 5, "rows r-2 .. r are read while rows r+1, r+2 are in flight");
    using T = float;
    constexpr bool PERT = true;
    using S = UnsplitF32Smem<NT, RING>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *sm = reinterpret_cast<float *>(smem_raw);
    auto RG = [&](int slot, int f, int t) -> float & { return sm[S::ring + (slot * 4 + f) * NT + t]; };
    auto DV = [&](int slot, int f, int t) -> float & { return sm[S::der + (slot * 4 + f) * NT + t]; };
    auto ZS = [&](int pm, int t) -> float & { return sm[S::z + pm * NT + t]; };
    auto XA = [&](int f, int t) -> float & { return sm[S::xa + f * NT + t]; };
    auto BY = [&](int m, int t) -> float & { return sm[S::by + m * NT + t]; };
    auto FX = [&](int m, int t) -> float & { return sm[S::fx + m * NT + t]; };
    float *red = sm + S::red;

    const StepItem it = a.items[blockIdx.x];
    if (it.w > NT - 4 || it.w < 1 || it.h < 1) return;   // not a work item of this launch shape
    const PatchDesc P = a.descs[it.patch];
    if (a.gate != nullptr && a.gate[P.scen] == 0) return;   // not retaken (uniform over the CTA)
    const int t = threadIdx.x;
    const int cur = a.cur;
    float *base = reinterpret_cast<float *>(a.arena) + P.off;
    const float *qin0 = base + (long long)(cur * 3 + 0) * P.fs;
    const float *qin1 = base + (long long)(cur * 3 + 1) * P.fs;
    const float *qin2 = base + (long long)(cur * 3 + 2) * P.fs;
    const float *Bg = base + 6LL * P.fs;
    float *qo0 = base + (long long)((1 - cur) * 3 + 0) * P.fs;
    float *qo1 = base + (long long)((1 - cur) * 3 + 1) * P.fs;
    float *qo2 = base + (long long)((1 - cur) * 3 + 2) * P.fs;

    const float dtdx = dt_over<float>(a, P.scen, false), dtdy = dt_over<float>(a, P.scen, true);
    const float hx = 0.5f * dtdx, hy = 0.5f * dtdy;
    const float g = a.gf;
    const float drytol = a.drytolf;
    const int x0 = it.x0, y0 = it.y0, w = it.w, h = it.h;
    const int pitch = P.pitch;
    const int nrows = h + 4;
    const bool loader = t < w + 4;
    const long long colofs = (long long)(x0 + t);

    auto prefetch = [&](int k) {
        if (k < nrows && loader) {
            const int slot = k % RING;
            const long long gi = (long long)(y0 + k) * pitch + colofs;
            cp_async_elem(&RG(slot, 0, t), qin0 + gi, sizeof(float));
            cp_async_elem(&RG(slot, 1, t), qin1 + gi, sizeof(float));
            cp_async_elem(&RG(slot, 2, t), qin2 + gi, sizeof(float));
            cp_async_elem(&RG(slot, 3, t), Bg + gi, sizeof(float));
        }
        cp_async_commit();
    };
    auto derive_own = [&](int k) {
        if (k < nrows && loader) {
            const int slot = k % RING;
            Cell<float> z;
            z.q0 = RG(slot, 0, t); z.hn = RG(slot, 1, t); z.ht = RG(slot, 2, t); z.B = RG(slot, 3, t);
            derive<float, PERT>(z, g, drytol);
            DV(slot, 0, t) = z.u; DV(slot, 1, t) = z.v; DV(slot, 2, t) = z.c; DV(slot, 3, t) = z.sq;
        }
    };
    auto cell = [&](int k, int c, bool yroles) {
        const int slot = k % RING;
        Cell<float> z;
        z.q0 = RG(slot, 0, c);
        z.hn = RG(slot, yroles ? 2 : 1, c);
        z.ht = RG(slot, yroles ? 1 : 2, c);
        z.B = RG(slot, 3, c);
        z.h = z.q0 - z.B;
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

    Wave<float> yold, ymid;
    float yap_prev[3] = {0.f, 0.f, 0.f};   // B+dQ of y-edge r-2 (y frame)
    float yap2_prev[3] = {0.f, 0.f, 0.f};  // its second-order form B+dQ - 2G~
    float G_prev[3] = {0.f, 0.f, 0.f};     // corrected G of y-edge r-2 (storage frame)
    float ap_own[3] = {0.f, 0.f, 0.f};     // A+dQ of x-edge t, last limited row
    float ap2_own[3] = {0.f, 0.f, 0.f};    // A+dQ - 2F~ of x-edge t, last limited row
    float Fq1[3] = {0.f, 0.f, 0.f};        // F~ of x-edge t in row r-1
    float Fq2[3] = {0.f, 0.f, 0.f};        // F~ of x-edge t in row r-2
    float Sx_old[3] = {0.f, 0.f, 0.f};     // A+dQ + A-dQ entering cell (t, r-2)
    float ax_old[3] = {0.f, 0.f, 0.f};     // second-order x-fluctuations entering cell (t, r-2)
    float smx = 0.f, smy = 0.f;

    for (int k = 0; k < nrows; k++) {
        __syncthreads();   // row k (ring + derived) visible; iteration k-1 finished everywhere
        prefetch(k + 2);
        const int r = y0 - 2 + k;
        const bool rowint = r >= y0 && r < y0 + h;

        // ---- 1a. x-edge Riemann problem of row r between ring cells t-1 and t
        Wave<float> xw;
        if (xsolve) {
            Cell<float> cl = cell(k, t - 1, false), cr = cell(k, t, false);
            riemann<float, PERT>(g, cl, cr, xw);
#pragma unroll
            for (int p = 0; p < 3; p++)
#pragma unroll
                for (int m = 0; m < 3; m++) ZS(p * 3 + m, t) = xw.Z[p][m];
        }

        // ---- 2. y-edge r of this column; limit edge r-1; publish the
        //         y-fluctuations entering cell (t, r-2)
        float yam[3], yap[3], yF[3], yam2[3], yap2[3];
        bool yready = false;
        if (ycol && k >= 1) {
            Cell<float> lo = cell(k - 1, t, true), hi = cell(k, t, true);
            Wave<float> ynew;
            riemann<float, PERT>(g, lo, hi, ynew);
            if (k >= 3) {
                float ZI[3][3];
#pragma unroll
                for (int p = 0; p < 3; p++)
#pragma unroll
                    for (int m = 0; m < 3; m++) ZI[p][m] = ymid.s[p] >= 0.f ? yold.Z[p][m] : ynew.Z[p][m];
                limit2<float>(ymid, ZI, dtdy, yam, yap, yF, yam2, yap2);
                yready = true;
                const int e = r - 1;
                if (out && e >= y0 && e <= y0 + h) smy = fmaxf(smy, fmaxf(-ymid.s[0], ymid.s[2]));
                // from below through edge r-2, from above through edge r-1; y frame -> x frame
                BY(0, t) = yap2_prev[0] + yam2[0];
                BY(1, t) = yap2_prev[2] + yam2[2];
                BY(2, t) = yap2_prev[1] + yam2[1];
            }
            yold = ymid;
            ymid = ynew;
        }

        // ---- 3. x-terms of cell (t, r-1); G of y-edge r-1 of this column
        float Sx_new[3] = {0.f, 0.f, 0.f}, ax_new[3] = {0.f, 0.f, 0.f};
        if (out && k >= 1) {
            // x-edge t of row r-1 is this thread's own; x-edge t+1 is thread t+1's
#pragma unroll
            for (int m = 0; m < 3; m++) {
                Sx_new[m] = ap_own[m] + XA(m, t + 1);
                ax_new[m] = ap2_own[m] + XA(3 + m, t + 1);
            }
        }
        float Gc[3] = {0.f, 0.f, 0.f};
        if (out && yready) {
            const Cell<float> ca = cell(k - 2, t, true), cb = cell(k - 1, t, true);
            const TEig<float> ev = teig<float>(g, ca.h, ca.u, ca.v, ca.c, ca.sq, ca.B, ca.wet,
                                               cb.h, cb.u, cb.v, cb.c, cb.sq, cb.B, cb.wet);
            const float i2c = ev.on ? 0.5f / ev.c : 0.f;
            Gc[0] = yF[0]; Gc[1] = yF[2]; Gc[2] = yF[1];    // y frame -> storage frame
            float part[3];
            // entering (t, r-1), the edge's upper cell: down-going part
            const float du[3] = {ax_new[0], ax_new[2], ax_new[1]};
            tpart_f32<false>(ev, i2c, du, part);
            Gc[0] = Gc[0] - hx * part[0]; Gc[1] = Gc[1] - hx * part[2]; Gc[2] = Gc[2] - hx * part[1];
            // entering (t, r-2), the edge's lower cell: up-going part
            const float dl[3] = {ax_old[0], ax_old[2], ax_old[1]};
            tpart_f32<true>(ev, i2c, dl, part);
            Gc[0] = Gc[0] - hx * part[0]; Gc[1] = Gc[1] - hx * part[2]; Gc[2] = Gc[2] - hx * part[1];
        }
        __syncthreads();   // x-waves of row r and y-fluctuations of row r-2 published; XA read

        // ---- 1b. limit x-edge t of row r; publish what thread t-1 needs
        float Fnew[3] = {0.f, 0.f, 0.f};
        if (xlim) {
            float ZI[3][3];
#pragma unroll
            for (int p = 0; p < 3; p++) {
                const int nb = xw.s[p] >= 0.f ? t - 1 : t + 1;
#pragma unroll
                for (int m = 0; m < 3; m++) ZI[p][m] = ZS(p * 3 + m, nb);
            }
            float am[3], ap[3], am2[3], ap2[3];
            limit2<float>(xw, ZI, dtdx, am, ap, Fnew, am2, ap2);
#pragma unroll
            for (int m = 0; m < 3; m++) {
                XA(m, t) = am[m];
                XA(3 + m, t) = am2[m];
                ap_own[m] = ap[m];
                ap2_own[m] = ap2[m];
            }
            if (rowint) smx = fmaxf(smx, fmaxf(-xw.s[0], xw.s[2]));
        }

        // ---- 4. F of x-edge t in row r-2 (y-fluctuations of columns t-1, t)
        if (xlim && k >= 4) {
            const Cell<float> ca = cell(k - 2, t - 1, false), cb = cell(k - 2, t, false);
            const TEig<float> ev = teig<float>(g, ca.h, ca.u, ca.v, ca.c, ca.sq, ca.B, ca.wet,
                                               cb.h, cb.u, cb.v, cb.c, cb.sq, cb.B, cb.wet);
            const float i2c = ev.on ? 0.5f / ev.c : 0.f;
            float Fc[3] = {Fq2[0], Fq2[1], Fq2[2]};
            float part[3];
            // entering (t, r-2), the edge's right cell: left-going part
            const float dr[3] = {BY(0, t), BY(1, t), BY(2, t)};
            tpart_f32<false>(ev, i2c, dr, part);
#pragma unroll
            for (int m = 0; m < 3; m++) Fc[m] = Fc[m] - hy * part[m];
            // entering (t-1, r-2), the edge's left cell: right-going part
            const float dl[3] = {BY(0, t - 1), BY(1, t - 1), BY(2, t - 1)};
            tpart_f32<true>(ev, i2c, dl, part);
#pragma unroll
            for (int m = 0; m < 3; m++) Fc[m] = Fc[m] - hy * part[m];
#pragma unroll
            for (int m = 0; m < 3; m++) FX(m, t) = Fc[m];
        }
        __syncthreads();   // F of row r-2 published

        // ---- 5. update cell (t, r-2)
        if (out && k >= 4) {
            const int j = r - 2;
            const int slot = (k - 2) % RING;
            float q[3] = {RG(slot, 0, t), RG(slot, 1, t), RG(slot, 2, t)};
            const float Bc = RG(slot, 3, t);
#pragma unroll
            for (int m = 0; m < 3; m++) {
                const int my = m == 0 ? 0 : (m == 1 ? 2 : 1);
                const float ux = Sx_old[m] + (FX(m, t + 1) - FX(m, t));
                const float uy = (yap_prev[my] + yam[my]) + (Gc[m] - G_prev[m]);
                q[m] = (q[m] - dtdx * ux) - dtdy * uy;
            }
            postprocess<float, PERT>(q[0], q[1], q[2], Bc, drytol);
            if (a.manning > 0.0)
                friction<float, PERT>(q[0], q[1], q[2], Bc, drytol, (float)a.manningf, dt_level<float>(a, P.scen));
            if (j >= y0 && j < y0 + h) {
                // a surface that is not a finite number reaches the host as an infinite speed
                if (!(fabsf(q[0]) < 1e30f)) smy = INFINITY;
                const long long gi = (long long)(j + 2) * pitch + (x0 + t);
                qo0[gi] = q[0];
                qo1[gi] = q[1];
                qo2[gi] = q[2];
            }
        }

        // ---- carry this iteration's terms one row down
        if (yready) {
#pragma unroll
            for (int m = 0; m < 3; m++) { yap_prev[m] = yap[m]; yap2_prev[m] = yap2[m]; G_prev[m] = Gc[m]; }
        }
#pragma unroll
        for (int m = 0; m < 3; m++) {
            Sx_old[m] = Sx_new[m];
            ax_old[m] = ax_new[m];
            Fq2[m] = Fq1[m];
            Fq1[m] = Fnew[m];
        }
        // row k+1 of this thread has landed (row k+2 may still be in flight)
        cp_async_wait<1>();
        derive_own(k + 1);
    }
    cp_async_wait<0>();

    // CTA max of the wave speeds: warp shuffles, then one atomic per CTA
    if (!(smx > 0.f)) smx = 0.f;
    if (!(smy > 0.f)) smy = 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        smx = fmaxf(smx, __shfl_xor_sync(0xffffffffu, smx, o));
        smy = fmaxf(smy, __shfl_xor_sync(0xffffffffu, smy, o));
    }
    if ((t & 31) == 0) { red[t >> 5] = smx; red[NT / 32 + (t >> 5)] = smy; }
    __syncthreads();
    if (t == 0) {
        float mx = 0.f, my = 0.f;
        for (int k = 0; k < NT / 32; k++) { mx = fmaxf(mx, red[k]); my = fmaxf(my, red[NT / 32 + k]); }
        atomic_max_speed(a.smax + 2 * P.scen + 0, (double)mx);
        atomic_max_speed(a.smax + 2 * P.scen + 1, (double)my);
    }
}

template <int NT>
int launch_unsplit_f32_nt(const StepArgs &a, int n_items, cudaStream_t st)
{
    constexpr int RING = 5;
    const size_t bytes = sizeof(float) * (size_t)UnsplitF32Smem<NT, RING>::total;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(step_unsplit_f32_kernel<NT, RING>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return (int)e;
        configured = true;
    }
    step_unsplit_f32_kernel<NT, RING><<<n_items, NT, bytes, st>>>(a);
    return (int)cudaGetLastError();
}

}  // namespace tsu
