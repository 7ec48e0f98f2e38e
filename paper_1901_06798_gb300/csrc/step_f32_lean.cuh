// step_f32_lean.cuh -- the FP32 surface-perturbation patch update, written
// for instruction count.
//
// Same method and the same streaming structure as step_kernel.cuh (rows
// through a cp.async ring, x-edge waves exchanged in shared memory, the y
// sweep of each column in registers, fused wave-speed reduction); the
// arithmetic is reorganised where FP32 rounding is held to the 1e-4 m
// surface bar rather than to the FP64 oracle's operation order:
//   * the wet-wet Riemann problem (the ocean) takes a short branch; dry beds,
//     walls and dry pairs take the general solver;
//   * fluctuations from the wave signs: A-dQ = (sum Z - sum sgn(s) Z) / 2,
//     A+dQ = (sum Z + sum sgn(s) Z) / 2 (a speed of 0 splits the wave in
//     half, as in the oracle);
//   * the contact wave has only a transverse component, so an edge publishes
//     7 wave components, and its limiter ratio is a quotient of scalars;
//   * no zero-norm test before theta = Z_I.Z / Z.Z: a zero wave contributes
//     0 to the correction whatever phi becomes.
#pragma once
#include <cuda_runtime.h>
#include "step_kernel.cuh"

namespace tsu {

struct LWave {
    float z0m, z0n, z0t;   // acoustic wave 1 (mass, normal, transverse)
    float z1t;             // contact wave (transverse only)
    float z2m, z2n, z2t;   // acoustic wave 3
    float s0, s1, s2;
    int wall;              // 1: left side mirrored, 2: right side mirrored
};

struct LCell {
    float q0, hn, ht, B;   // eta', normal and transverse momentum, bed
    float h, u, v, c, sq;
    bool wet;
};

__device__ __forceinline__ void lderive(LCell &z, float sqrtg, float drytol)
{
    z.h = z.q0 - z.B;
    z.wet = z.h >= drytol;
    float hp = z.wet ? z.h : 0.0f;
    float rh = z.wet ? __fdividef(1.0f, z.h) : 0.0f;
    z.u = z.hn * rh;
    z.v = z.ht * rh;
    z.sq = sqrtf(hp);
    z.c = sqrtg * z.sq;
}

__device__ __forceinline__ void lriemann(float g, const LCell &L, const LCell &R, LWave &r)
{
    if (L.wet && R.wet) {
        float uhat = __fdividef(L.sq * L.u + R.sq * R.u, L.sq + R.sq);
        float hbar = 0.5f * (L.h + R.h);
        float chat = sqrtf(g * hbar);
        float s1 = fminf(L.u - L.c, uhat - chat);
        float s3 = fmaxf(R.u + R.c, uhat + chat);
        float d1 = R.q0 - L.q0;
        float d2 = R.hn - L.hn;
        float d3 = (R.hn * R.u - L.hn * L.u) + (g * hbar) * d1;
        float d4 = R.hn * R.v - L.hn * L.v;
        float rden = __fdividef(1.0f, s3 - s1);
        float w1m = (s3 * d1 - d2) * rden;
        float w1n = (s3 * d2 - d3) * rden;
        r.z0m = s1 * w1m; r.z0n = s1 * w1n; r.z0t = r.z0m * L.v;
        r.z2m = s3 * (d1 - w1m); r.z2n = s3 * (d2 - w1n); r.z2t = r.z2m * R.v;
        r.z1t = (d4 - r.z0t) - r.z2t;
        r.s0 = s1; r.s1 = uhat; r.s2 = s3;
        r.wall = 0;
        return;
    }
    // dry bed, wall or dry pair: the general solver
    Cell<float> a, b;
    a.q0 = L.q0; a.hn = L.hn; a.ht = L.ht; a.B = L.B; a.h = L.h; a.u = L.u; a.v = L.v; a.c = L.c; a.sq = L.sq; a.wet = L.wet;
    b.q0 = R.q0; b.hn = R.hn; b.ht = R.ht; b.B = R.B; b.h = R.h; b.u = R.u; b.v = R.v; b.c = R.c; b.sq = R.sq; b.wet = R.wet;
    Wave<float> w;
    riemann<float, true>(g, a, b, w);
    r.z0m = w.Z[0][0]; r.z0n = w.Z[0][1]; r.z0t = w.Z[0][2];
    r.z1t = w.Z[1][2];
    r.z2m = w.Z[2][0]; r.z2n = w.Z[2][1]; r.z2t = w.Z[2][2];
    r.s0 = w.s[0]; r.s1 = w.s[1]; r.s2 = w.s[2];
    r.wall = w.wall;
}

__device__ __forceinline__ float sgnf(float s) { return s > 0.0f ? 1.0f : (s < 0.0f ? -1.0f : 0.0f); }
// sign of an acoustic wave's speed: at s = 0 its f-wave Z = s W is zero, so
// where it goes does not matter and copysign suffices
__device__ __forceinline__ float sgna(float s) { return copysignf(1.0f, s); }

__device__ __forceinline__ float mcf(float th)
{
    return fmaxf(0.0f, fminf(fminf(fmaf(0.5f, th, 0.5f), 2.0f), 2.0f * th));
}

// fluctuations and limited correction flux of one edge; I0/I1/I2: the
// upwind neighbours' waves for wave 1, contact, wave 3
__device__ __forceinline__ void llimit(const LWave &r, float i0m, float i0n, float i0t, float i1t, float i2m,
                                       float i2n, float i2t, float dtdx, float (&amdq)[3], float (&apdq)[3],
                                       float (&F)[3])
{
    float g0 = sgna(r.s0), g1 = sgnf(r.s1), g2 = sgna(r.s2);
    float sm = r.z0m + r.z2m, sn = r.z0n + r.z2n, st = (r.z0t + r.z1t) + r.z2t;
    float gm = g0 * r.z0m + g2 * r.z2m;
    float gn = g0 * r.z0n + g2 * r.z2n;
    float gt = fmaf(g0, r.z0t, fmaf(g1, r.z1t, g2 * r.z2t));
    amdq[0] = 0.5f * (sm - gm); apdq[0] = 0.5f * (sm + gm);
    amdq[1] = 0.5f * (sn - gn); apdq[1] = 0.5f * (sn + gn);
    amdq[2] = 0.5f * (st - gt); apdq[2] = 0.5f * (st + gt);
    if (r.wall) {
        if (r.wall == 2) { apdq[0] = 0.0f; apdq[1] = 0.0f; apdq[2] = 0.0f; }
        else { amdq[0] = 0.0f; amdq[1] = 0.0f; amdq[2] = 0.0f; }
        F[0] = 0.0f; F[1] = 0.0f; F[2] = 0.0f;
        return;
    }
    float n0 = fmaf(r.z0m, r.z0m, fmaf(r.z0n, r.z0n, r.z0t * r.z0t));
    float n2 = fmaf(r.z2m, r.z2m, fmaf(r.z2n, r.z2n, r.z2t * r.z2t));
    float d0 = fmaf(i0m, r.z0m, fmaf(i0n, r.z0n, i0t * r.z0t));
    float d2 = fmaf(i2m, r.z2m, fmaf(i2n, r.z2n, i2t * r.z2t));
    float ph0 = mcf(__fdividef(d0, n0));
    float ph1 = mcf(__fdividef(i1t, r.z1t));
    float ph2 = mcf(__fdividef(d2, n2));
    float c0 = 0.5f * g0 * (1.0f - dtdx * fabsf(r.s0)) * ph0;
    float c1 = 0.5f * g1 * (1.0f - dtdx * fabsf(r.s1)) * ph1;
    float c2 = 0.5f * g2 * (1.0f - dtdx * fabsf(r.s2)) * ph2;
    F[0] = fmaf(c0, r.z0m, c2 * r.z2m);
    F[1] = fmaf(c0, r.z0n, c2 * r.z2n);
    F[2] = fmaf(c0, r.z0t, fmaf(c1, r.z1t, c2 * r.z2t));
}

__device__ __forceinline__ void lpost(float &q0, float &qn, float &qt, float B, float drytol)
{
    float h = q0 - B;
    if (h < 0.0f) { q0 = B; h = 0.0f; }
    if (h < drytol) { qn = 0.0f; qt = 0.0f; }
}

template <int NT, int RING>
__global__ void __launch_bounds__(NT) step_kernel_f32(StepArgs a)
{
    static_assert(RING >= 3, "the derived values of row k+1 need its copy complete at iteration k");
    __shared__ float ring[RING][4][NT];
    __shared__ float sZ[7][NT];
    __shared__ float sAp[3][NT];
    __shared__ float sF[3][NT];
    __shared__ float sD[2][4][NT];
    __shared__ float red[2][NT / 32];

    const StepItem it = a.items[blockIdx.x];
    const PatchDesc P = a.descs[it.patch];
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

    // dt / dx of this level in FP32: the level-1 step (an FP32 copy kept by the
    // step-start kernel) times 1 / (R dx) prepared on the host
    const float dt1 = a.dt1f[P.scen];
    const float dtdx = dt1 * a.rdx, dtdy = dt1 * a.rdy;
    const float g = a.gf, drytol = a.drytolf, sqrtg = a.sqrtgf;
    const int x0 = it.x0, y0 = it.y0, w = it.w, h = it.h;
    const int pitch = P.pitch;
    const int nrows = h + 4;
    const bool loader = t < w + 4;
    const float *src0 = qin0 + (long long)y0 * pitch + (x0 + t);
    const long long fo1 = qin1 - qin0, fo2 = qin2 - qin0, foB = Bg - qin0;

    auto prefetch = [&](int k) {
        if (k < nrows && loader) {
            int slot = k % RING;
            const float *s = src0 + (long long)k * pitch;
            cp_async_elem(&ring[slot][0][t], s, 4);
            cp_async_elem(&ring[slot][1][t], s + fo1, 4);
            cp_async_elem(&ring[slot][2][t], s + fo2, 4);
            cp_async_elem(&ring[slot][3][t], s + foB, 4);
        }
        cp_async_commit();
    };
    auto own_cell = [&](int k, LCell &z) {
        const int slot = k % RING;
        z.q0 = ring[slot][0][t]; z.hn = ring[slot][1][t]; z.ht = ring[slot][2][t]; z.B = ring[slot][3][t];
        lderive(z, sqrtg, drytol);
        sD[k & 1][0][t] = z.u; sD[k & 1][1][t] = z.v; sD[k & 1][2][t] = z.c; sD[k & 1][3][t] = z.sq;
    };

#pragma unroll
    for (int k = 0; k < RING - 1; k++) prefetch(k);
    LCell xc;
    cp_async_wait<RING - 2>();
    if (loader) own_cell(0, xc);

    LCell ym1;
    float m2q0 = 0.0f, m2hu = 0.0f, m2hv = 0.0f, Bm2 = 0.0f;
    LWave yold, ymid;
    float yap[3] = {0.0f, 0.0f, 0.0f}, yF[3] = {0.0f, 0.0f, 0.0f};
    float smx = 0.0f, smy = 0.0f;
    const bool upd = t >= 2 && t < w + 2;
    const bool rsolve = t < w + 3;
    const bool lim = t >= 1 && t < w + 2;
    float *dst0 = qo0 + (long long)(y0 + 2) * pitch + (x0 + t);
    const long long go1 = qo1 - qo0, go2 = qo2 - qo0;

    for (int k = 0; k < nrows; k++) {
        prefetch(k + RING - 1);
        cp_async_wait<RING - 2>();
        __syncthreads();
        const int slot = k % RING;
        const int r = y0 - 2 + k;
        const bool rowint = r >= y0 && r < y0 + h;

        LWave xw;
        if (rsolve) {
            LCell xr;
            xr.q0 = ring[slot][0][t + 1]; xr.hn = ring[slot][1][t + 1]; xr.ht = ring[slot][2][t + 1];
            xr.B = ring[slot][3][t + 1];
            xr.h = xr.q0 - xr.B;
            xr.wet = xr.h >= drytol;
            xr.u = sD[k & 1][0][t + 1]; xr.v = sD[k & 1][1][t + 1]; xr.c = sD[k & 1][2][t + 1];
            xr.sq = sD[k & 1][3][t + 1];
            lriemann(g, xc, xr, xw);
            sZ[0][t] = xw.z0m; sZ[1][t] = xw.z0n; sZ[2][t] = xw.z0t; sZ[3][t] = xw.z1t;
            sZ[4][t] = xw.z2m; sZ[5][t] = xw.z2n; sZ[6][t] = xw.z2t;
        }
        __syncthreads();

        float xam[3], xap[3], xF[3];
        if (lim) {
            const int n0 = xw.s0 >= 0.0f ? t - 1 : t + 1;
            const int n1 = xw.s1 >= 0.0f ? t - 1 : t + 1;
            const int n2 = xw.s2 >= 0.0f ? t - 1 : t + 1;
            llimit(xw, sZ[0][n0], sZ[1][n0], sZ[2][n0], sZ[3][n1], sZ[4][n2], sZ[5][n2], sZ[6][n2], dtdx, xam, xap, xF);
            sAp[0][t] = xap[0]; sAp[1][t] = xap[1]; sAp[2][t] = xap[2];
            sF[0][t] = xF[0]; sF[1][t] = xF[1]; sF[2][t] = xF[2];
            if (rowint) smx = fmaxf(smx, fmaxf(-xw.s0, xw.s2));
        }
        __syncthreads();

        if (upd) {
            float qs0 = xc.q0 - dtdx * ((sAp[0][t - 1] + xam[0]) + (xF[0] - sF[0][t - 1]));
            float qs1 = xc.hn - dtdx * ((sAp[1][t - 1] + xam[1]) + (xF[1] - sF[1][t - 1]));
            float qs2 = xc.ht - dtdx * ((sAp[2][t - 1] + xam[2]) + (xF[2] - sF[2][t - 1]));
            lpost(qs0, qs1, qs2, xc.B, drytol);

            LCell yc;
            yc.q0 = qs0; yc.hn = qs2; yc.ht = qs1; yc.B = xc.B;
            lderive(yc, sqrtg, drytol);
            if (k >= 1) {
                LWave ynew;
                lriemann(g, ym1, yc, ynew);
                if (k >= 3) {
                    const int e = r - 1;
                    if (e >= y0 && e <= y0 + h) {
                        const LWave &u0 = ymid.s0 >= 0.0f ? yold : ynew;
                        const LWave &u1 = ymid.s1 >= 0.0f ? yold : ynew;
                        const LWave &u2 = ymid.s2 >= 0.0f ? yold : ynew;
                        float yam[3], yapn[3], yFn[3];
                        llimit(ymid, u0.z0m, u0.z0n, u0.z0t, u1.z1t, u2.z2m, u2.z2n, u2.z2t, dtdy, yam, yapn, yFn);
                        smy = fmaxf(smy, fmaxf(-ymid.s0, ymid.s2));
                        const int rc = r - 2;
                        if (rc >= y0 && rc < y0 + h) {
                            float n0 = m2q0 - dtdy * ((yap[0] + yam[0]) + (yFn[0] - yF[0]));
                            float n1 = m2hv - dtdy * ((yap[1] + yam[1]) + (yFn[1] - yF[1]));
                            float n2 = m2hu - dtdy * ((yap[2] + yam[2]) + (yFn[2] - yF[2]));
                            lpost(n0, n1, n2, Bm2, drytol);
                            float *d = dst0 + (long long)(rc - y0) * pitch;
                            d[0] = n0;
                            d[go2] = n1;
                            d[go1] = n2;
                        }
                        yap[0] = yapn[0]; yap[1] = yapn[1]; yap[2] = yapn[2];
                        yF[0] = yFn[0]; yF[1] = yFn[1]; yF[2] = yFn[2];
                    }
                }
                yold = ymid;
                ymid = ynew;
            }
            m2q0 = ym1.q0; m2hu = ym1.ht; m2hv = ym1.hn; Bm2 = ym1.B;
            ym1 = yc;
        }
        if (loader && k + 1 < nrows) own_cell(k + 1, xc);
    }

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
