// step_split_f32.cuh -- the FP32 surface-perturbation split step (Sec. 2.2,
// x sweep then y sweep) as two kernels, with Q* through a scratch copy in HBM.
//
// step_x_f32x2: one CTA per strip of 2 NT - 4 columns and a segment of rows,
//   ghost rows included (Q* is needed there by the y sweep).  Rows stream
//   through a cp.async ring as in the fused kernel, two columns per thread on
//   the paired FP32 instructions.  With one warp per CTA (NT = 32, the default)
//   the neighbours' x-edge values move by warp shuffles and the row loop has
//   no block barrier; wider CTAs exchange them in shared memory.  A row needs
//   no other row, so segments carry no halo rows.  It writes Q* of its
//   interior columns and reduces the max x wave speed of interior rows.
//   BULK: one thread copies each field's row segment into the ring with a bulk
//   copy (cp.async.bulk) that completes on the slot's mbarrier, which every
//   thread polls with a bounded budget (patch rows start 16-byte aligned, the
//   pitch is a multiple of 4 floats and strips start at multiples of 4
//   columns).  Measured slower than the per-thread copies; kept as an option.
// step_y_f32x2: one CTA of 64 threads per strip of 64 columns (one per
//   thread) and a segment of interior rows; reads Q* and B of the segment plus
//   two rows above and below, runs the y sweep of its column in registers, two
//   rows per iteration on the paired instructions (no halo columns, no
//   barriers), and writes Q^{n+1}.  Each thread streams its own column through
//   a cp.async ring in shared memory, two row pairs ahead, so the loads'
//   latency hides behind the rows in flight.
//
// Against the fused kernel (step_f32x2.cuh) the split pays 24 B per cell more
// HBM traffic (Q* out and back in), which the 4096^2 update has room for: the
// fused kernel is bound by instruction issue and latency.  What the split
// saves is the recomputed halo work (4 rows per row segment, 4 columns per
// y strip) and the register pressure of carrying both sweeps: the x kernel
// runs at about 82 registers and the y kernel at 124 instead of 168.  The
// arithmetic per cell is the fused kernel's, operation for operation, so the
// two give the same bits.  GEO: latitude-longitude grid in capacity form, as
// in the fused kernel.
#pragma once
#include "step_f32x2.cuh"

namespace tsu {

template <int NT, int RING, bool GEO, bool BULK = false>
__global__ void __launch_bounds__(NT) step_x_f32x2(StepArgs a)
{
    using namespace x2;
    // one warp per CTA: neighbours' values move by warp shuffles, and each thread
    // reads only its own ring columns, so the row loop needs no block barrier
    constexpr bool WARP = NT == 32 && !BULK;
    static_assert(RING >= 3, "the derived values of row k+1 need its copy complete at iteration k");
    constexpr int NC = 2 * NT;
    __shared__ __align__(16) float ring[RING][4][NC];
    __shared__ __align__(8) unsigned long long rbar[BULK ? RING : 1];   // BULK: one barrier per ring slot
    __shared__ int gave_up;           // BULK: a wait ran out of polls (no further copies)
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

    // BULK: a row copy is the strip's ncols floats rounded up to 16 bytes,
    // which stays inside the row (x0 and the pitch are multiples of 4 floats)
    const float *col0 = qin0 + (long long)(y0 + 2) * pitch + x0;
    const unsigned nb = (unsigned)((ncols * 4 + 15) & ~15);
    int issued = 0;   // BULK: rows issued (thread 0)
    if (BULK) {
        if (((reinterpret_cast<uintptr_t>(col0) & 15) != 0) || ((pitch & 3) != 0) || ((fs & 3) != 0)) {
            if (t == 0 && a.err) atomicOr(a.err, TSU_DEV_ERR_LAYOUT);   // uniform over the CTA
            return;
        }
        if (t == 0) {
#pragma unroll
            for (int q = 0; q < RING; q++) mbar_init(&rbar[q], 1);
            gave_up = 0;
            mbar_init_fence();
        }
        __syncthreads();
    }
    auto prefetch = [&](int k) {
        if (BULK) {
            if (t == 0 && k < nrows && !*(volatile int *)&gave_up) {
                const int slot = k % RING;
                const float *s = col0 + (long long)k * pitch;
                mbar_expect_tx(&rbar[slot], 4 * nb);
#pragma unroll
                for (int f = 0; f < 4; f++) bulk_g2s(&ring[slot][f][0], s + fo[f], nb, &rbar[slot]);
                issued = k + 1;
            }
            return;
        }
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
    // row k has landed (cp.async: this thread's copies of rows up to k); BULK:
    // after one wait gives up, no thread waits again
    auto await_row = [&](int k) {
        if (BULK) {
            if (k < nrows && !*(volatile int *)&gave_up &&
                !mbar_wait(&rbar[k % RING], (unsigned)(k / RING) & 1u, a.wait_polls))
                *(volatile int *)&gave_up = 1;
        } else {
            cp_async_wait<RING - 2>();
        }
    };
    auto own_cells = [&](int k, C2 &z) {
        const int slot = k % RING;
        z.q0 = ld2(&ring[slot][0][c0]); z.hn = ld2(&ring[slot][1][c0]);
        z.ht = ld2(&ring[slot][2][c0]); z.B = ld2(&ring[slot][3][c0]);
        derive(z, sqrtg, drytol);
        if (!WARP) {
            sDb[k & 1][0][t] = z.u.y; sDb[k & 1][1][t] = z.v.y; sDb[k & 1][2][t] = z.c.y; sDb[k & 1][3][t] = z.sq.y;
        }
    };
    // from the thread on the left (lane 0: its own value), on the right (lane 31: its own)
    auto from_left = [](float v) { return __shfl_up_sync(0xffffffffu, v, 1); };
    auto from_right = [](float v) { return __shfl_down_sync(0xffffffffu, v, 1); };

#pragma unroll
    for (int k = 0; k < RING - 1; k++) prefetch(k);
    C2 xc;
    await_row(0);
    own_cells(0, xc);

    const int tl = t > 0 ? t - 1 : 0, tr = t + 1 < NT ? t + 1 : NT - 1;
    const bool limx = c0 >= 2 && c0 <= w + 2, limy = c0 + 1 >= 2 && c0 + 1 <= w + 2;   // edges x0 .. x0+w
    const bool outx = c0 >= 2 && c0 < w + 2, outy = c0 + 1 >= 2 && c0 + 1 < w + 2;     // columns x0 .. x0+w-1
    const bool upd = outx || outy;
    const bool w8 = v8 && outx && outy;
    float smx = 0.0f;

    for (int k = 0; k < nrows; k++) {
        prefetch(k + RING - 1);
        await_row(k + 1);
        if (!WARP) __syncthreads();
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
        if (WARP) {   // the left cell is the left thread's lane y
            L.q0 = make_float2(from_left(xc.q0.y), xc.q0.x);
            L.hn = make_float2(from_left(xc.hn.y), xc.hn.x);
            L.ht = make_float2(from_left(xc.ht.y), xc.ht.x);
            L.B = make_float2(from_left(xc.B.y), xc.B.x);
            L.u = make_float2(from_left(xc.u.y), xc.u.x); L.v = make_float2(from_left(xc.v.y), xc.v.x);
            L.c = make_float2(from_left(xc.c.y), xc.c.x); L.sq = make_float2(from_left(xc.sq.y), xc.sq.x);
        } else {
            L.q0 = make_float2(ring[slot][0][c0 > 0 ? c0 - 1 : 0], xc.q0.x);
            L.hn = make_float2(ring[slot][1][c0 > 0 ? c0 - 1 : 0], xc.hn.x);
            L.ht = make_float2(ring[slot][2][c0 > 0 ? c0 - 1 : 0], xc.ht.x);
            L.B = make_float2(ring[slot][3][c0 > 0 ? c0 - 1 : 0], xc.B.x);
            L.u = make_float2(sDb[k & 1][0][tl], xc.u.x); L.v = make_float2(sDb[k & 1][1][tl], xc.v.x);
            L.c = make_float2(sDb[k & 1][2][tl], xc.c.x); L.sq = make_float2(sDb[k & 1][3][tl], xc.sq.x);
        }
        L.h = sub(L.q0, L.B);
        L.wx = L.h.x >= drytol; L.wy = xc.wx;
        W2 xw;
        riemann2(g, L, xc, xw);
        if (!WARP) {
            sZx[0][t] = xw.z0m.x; sZx[1][t] = xw.z0n.x; sZx[2][t] = xw.z0t.x; sZx[3][t] = xw.z1t.x;
            sZx[4][t] = xw.z2m.x; sZx[5][t] = xw.z2n.x; sZx[6][t] = xw.z2t.x;
            sZy[0][t] = xw.z0m.y; sZy[1][t] = xw.z0n.y; sZy[2][t] = xw.z0t.y; sZy[3][t] = xw.z1t.y;
            sZy[4][t] = xw.z2m.y; sZy[5][t] = xw.z2n.y; sZy[6][t] = xw.z2t.y;
            __syncthreads();
        }

        // ---- limit both edges (upwind neighbours as in the fused kernel)
        float2 xam[3], xap[3], xF[3];
        float sPr[3];   // WARP: A-dQ + F~ of the right thread's edge 2t + 2
        {
            I2 I;
            if (WARP) {
                // upwind of edge 2t: 2t-1 (left thread's lane y) or 2t+1 (own lane y);
                // of edge 2t+1: 2t (own lane x) or 2t+2 (right thread's lane x)
                const bool a0 = xw.s0.x >= 0.0f, a1 = xw.s1.x >= 0.0f, a2 = xw.s2.x >= 0.0f;
                const bool b0 = xw.s0.y >= 0.0f, b1 = xw.s1.y >= 0.0f, b2 = xw.s2.y >= 0.0f;
                const float l0 = from_left(xw.z0m.y), l1 = from_left(xw.z0n.y), l2 = from_left(xw.z0t.y);
                const float l3 = from_left(xw.z1t.y), l4 = from_left(xw.z2m.y), l5 = from_left(xw.z2n.y);
                const float l6 = from_left(xw.z2t.y);
                const float r0_ = from_right(xw.z0m.x), r1_ = from_right(xw.z0n.x), r2_ = from_right(xw.z0t.x);
                const float r3_ = from_right(xw.z1t.x), r4_ = from_right(xw.z2m.x), r5_ = from_right(xw.z2n.x);
                const float r6_ = from_right(xw.z2t.x);
                I.m0 = make_float2(a0 ? l0 : xw.z0m.y, b0 ? xw.z0m.x : r0_);
                I.n0 = make_float2(a0 ? l1 : xw.z0n.y, b0 ? xw.z0n.x : r1_);
                I.t0 = make_float2(a0 ? l2 : xw.z0t.y, b0 ? xw.z0t.x : r2_);
                I.t1 = make_float2(a1 ? l3 : xw.z1t.y, b1 ? xw.z1t.x : r3_);
                I.m2 = make_float2(a2 ? l4 : xw.z2m.y, b2 ? xw.z2m.x : r4_);
                I.n2 = make_float2(a2 ? l5 : xw.z2n.y, b2 ? xw.z2n.x : r5_);
                I.t2 = make_float2(a2 ? l6 : xw.z2t.y, b2 ? xw.z2t.x : r6_);
            } else {
                const int a0 = xw.s0.x >= 0.0f ? tl : t, a1 = xw.s1.x >= 0.0f ? tl : t, a2 = xw.s2.x >= 0.0f ? tl : t;
                const int b0 = xw.s0.y >= 0.0f ? t : tr, b1 = xw.s1.y >= 0.0f ? t : tr, b2 = xw.s2.y >= 0.0f ? t : tr;
                I.m0 = make_float2(sZy[0][a0], sZx[0][b0]);
                I.n0 = make_float2(sZy[1][a0], sZx[1][b0]);
                I.t0 = make_float2(sZy[2][a0], sZx[2][b0]);
                I.t1 = make_float2(sZy[3][a1], sZx[3][b1]);
                I.m2 = make_float2(sZy[4][a2], sZx[4][b2]);
                I.n2 = make_float2(sZy[5][a2], sZx[5][b2]);
                I.t2 = make_float2(sZy[6][a2], sZx[6][b2]);
            }
            limit2(xw, I, dtdxr, xam, xap, xF);
            if (WARP) {
#pragma unroll
                for (int m = 0; m < 3; m++) sPr[m] = from_right(xam[m].x + xF[m].x);
            } else {
                sP[0][t] = xam[0].x + xF[0].x; sP[1][t] = xam[1].x + xF[1].x; sP[2][t] = xam[2].x + xF[2].x;
            }
            if (rowint) {
                if (limx) smx = fmaxf(smx, fmaxf(-xw.s0.x, xw.s2.x) * rk);
                if (limy) smx = fmaxf(smx, fmaxf(-xw.s0.y, xw.s2.y) * rk);
            }
        }
        if (!WARP) {
            __syncthreads();
#pragma unroll
            for (int m = 0; m < 3; m++) sPr[m] = sP[m][tr];
        }

        if (upd) {
            float2 q0 = xc.q0, q1 = xc.hn, q2 = xc.ht;
            const float2 r0 = make_float2(xam[0].y + xF[0].y, sPr[0]);
            const float2 r1 = make_float2(xam[1].y + xF[1].y, sPr[1]);
            const float2 r2 = make_float2(xam[2].y + xF[2].y, sPr[2]);
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
    if (BULK) {
        // after a wait gave up, the copies still in flight land before the CTA
        // exits: each slot's last issued row (a slot is armed again only after
        // its previous phase completed); then the launch reports the timeout
        __syncthreads();
        if (t == 0 && gave_up) {
            for (int r = issued - 1; r >= 0 && r >= issued - RING; r--)
                mbar_wait(&rbar[r % RING], (unsigned)(r / RING) & 1u, kDrainPolls);
            if (a.err) atomicOr(a.err, TSU_DEV_ERR_TIMEOUT);
        }
    } else {
        cp_async_wait<0>();
    }

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

// threads per CTA of the y kernel: two warps, one column per thread
constexpr int kSplitYThreads = 64;
constexpr int kSplitYAhead = 2;              // row pairs in flight per thread
constexpr int kSplitYRing = kSplitYAhead + 3;   // ring slots: pairs j - 2 .. j + 2

// The y sweep pairs along the sweep: thread t owns column t of the strip and
// takes two rows per iteration, so lane x of every float2 is an even ring row
// (or the y-edge below it) and lane y the odd row above.  Ring row k = 0 ..
// h + 3 is patch row y0 - 2 + k; y-edge k lies between ring rows k - 1 and k.
// Iteration j (row pair j = ring rows 2j, 2j + 1):
//   * solves the y-edge pair (2j, 2j + 1): left states (row 2j - 1, row 2j),
//     right states the pair itself;
//   * limits the edge pair (2j - 2, 2j - 1): the upwind neighbour of edge
//     2j - 2 is edge 2j - 3 (the previous pair's lane y) or 2j - 1, that of
//     edge 2j - 1 is edge 2j - 2 or 2j (this iteration's lane x);
//   * updates the row pair (2j - 4, 2j - 3) from A+dQ - F~ of its lower edges
//     (the edge pair 2j - 4, 2j - 3) and A-dQ + F~ of its upper edges (2j - 3,
//     2j - 2).
// The state carried from one iteration to the next is one cell (row 2j - 1),
// one edge pair's waves plus one edge's, and the limited terms of one edge
// pair; the row pair being updated is read back from the ring, which keeps
// the two pairs before the current one.
template <bool GEO>
__global__ void __launch_bounds__(kSplitYThreads) step_y_f32x2(StepArgs a)
{
    using namespace x2;
    constexpr int NT = kSplitYThreads, YRING = kSplitYRing, AHEAD = kSplitYAhead;
    // ring[slot][field][t] = rows 2i, 2i + 1 of column t: Q* eta', hu, hv and B.
    // Thread t only ever reads its own column, so its cp.async waits suffice.
    __shared__ __align__(16) float2 ring[YRING][4][NT];
    const StepItem it = a.items_y[blockIdx.x];
    if (it.w > NT || it.w < 1 || it.h < 1) return;   // uniform over the CTA
    const PatchDesc P = a.descs[it.patch];
    if (a.gate != nullptr && a.gate[P.scen] == 0) return;   // not retaken (uniform over the CTA)
    const int t = threadIdx.x;
    const bool valid = t < it.w;
    const int tc = valid ? t : it.w - 1;   // threads past the strip repeat its last column and store nothing
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
    // ring row k of this column at storage [(y0 + k) * pitch + x0 + tc + 2]
    const long long cbase = (long long)y0 * pitch + (it.x0 + tc + 2);
    const int klast = h + 3;
    // interior rows are ring rows 2 .. h + 1; the last row pair holding one is
    // updated at iteration (h + 1) / 2 + 2
    const int niter = (h + 1) / 2 + 3;
    const float *fsrc[4] = {qs0 + cbase, qs0 + fs + cbase, qs0 + 2 * fs + cbase, Bg + cbase};
    auto prefetch = [&](int i) {
        if (i < niter) {
            const int slot = i % YRING;
            // rows past the segment's last ring row repeat it (no waves between them)
            const long long o0 = (long long)min(2 * i, klast) * pitch;
            const long long o1 = (long long)min(2 * i + 1, klast) * pitch;
#pragma unroll
            for (int f = 0; f < 4; f++) {
                cp_async_elem(&ring[slot][f][t].x, fsrc[f] + o0, 4);
                cp_async_elem(&ring[slot][f][t].y, fsrc[f] + o1, 4);
            }
        }
        cp_async_commit();
    };
#pragma unroll
    for (int i = 0; i < AHEAD; i++) prefetch(i);

    Cell<float> pv;            // ring row 2j - 1: the lower cell of y-edge 2j
    W2 wm;                     // waves of the edge pair (2j - 2, 2j - 1)
    float wo[7];               // waves of edge 2j - 3 (lane y of the pair before)
    float2 Dp[3];              // A+dQ - F~ of the edge pair (2j - 4, 2j - 3)
    float Spy[3];              // A-dQ + F~ of edge 2j - 3
    float smy = 0.0f;
#pragma unroll
    for (int m = 0; m < 7; m++) wo[m] = 0.0f;
#pragma unroll
    for (int m = 0; m < 3; m++) { Dp[m] = f2(0.0f); Spy[m] = 0.0f; }

    for (int j = 0; j < niter; j++) {
        prefetch(j + AHEAD);   // into the slot of row pair j - 3
        cp_async_wait<AHEAD>();   // row pair j of this thread has landed
        const int slot = j % YRING;
        C2 cj;   // y roles: hn = hv, ht = hu
        cj.q0 = ring[slot][0][t];
        cj.ht = ring[slot][1][t];
        cj.hn = ring[slot][2][t];
        cj.B = ring[slot][3][t];
        derive(cj, sqrtg, drytol);
        if (j == 0) lane_in(cj, 0, pv);   // no row below ring row 0: repeat it (edge 0 is never used)

        // ---- y-edges 2j (rows 2j - 1 | 2j) and 2j + 1 (rows 2j | 2j + 1)
        C2 L;
        L.q0 = make_float2(pv.q0, cj.q0.x); L.hn = make_float2(pv.hn, cj.hn.x);
        L.ht = make_float2(pv.ht, cj.ht.x); L.B = make_float2(pv.B, cj.B.x);
        L.h = make_float2(pv.h, cj.h.x); L.u = make_float2(pv.u, cj.u.x);
        L.v = make_float2(pv.v, cj.v.x); L.c = make_float2(pv.c, cj.c.x);
        L.sq = make_float2(pv.sq, cj.sq.x);
        L.wx = pv.wet; L.wy = cj.wx;
        W2 wn;
        riemann2(g, L, cj, wn);

        if (j >= 2) {
            // ---- limit the edge pair (2j - 2, 2j - 1)
            const int e0 = 2 * j - 2;   // ring index of lane x's edge
            I2 I;
            const bool a0 = wm.s0.x >= 0.0f, a1 = wm.s1.x >= 0.0f, a2 = wm.s2.x >= 0.0f;
            const bool b0 = wm.s0.y >= 0.0f, b1 = wm.s1.y >= 0.0f, b2 = wm.s2.y >= 0.0f;
            I.m0 = make_float2(a0 ? wo[0] : wm.z0m.y, b0 ? wm.z0m.x : wn.z0m.x);
            I.n0 = make_float2(a0 ? wo[1] : wm.z0n.y, b0 ? wm.z0n.x : wn.z0n.x);
            I.t0 = make_float2(a0 ? wo[2] : wm.z0t.y, b0 ? wm.z0t.x : wn.z0t.x);
            I.t1 = make_float2(a1 ? wo[3] : wm.z1t.y, b1 ? wm.z1t.x : wn.z1t.x);
            I.m2 = make_float2(a2 ? wo[4] : wm.z2m.y, b2 ? wm.z2m.x : wn.z2m.x);
            I.n2 = make_float2(a2 ? wo[5] : wm.z2n.y, b2 ? wm.z2n.x : wn.z2n.x);
            I.t2 = make_float2(a2 ? wo[6] : wm.z2t.y, b2 ? wm.z2t.x : wn.z2t.x);
            float2 am[3], ap[3], F[3], S[3], D[3];
            float2 dtdye = dtdy2, cr = f2(1.0f), ce = f2(1.0f);
            if (GEO) {
                // patch rows above the two edges; an edge past the last one an
                // interior row needs (ring edge h + 2) is not used: clamp it there
                const int ea = min(y0 - 2 + e0, y0 + h), eb = min(y0 - 1 + e0, y0 + h);
                ce = make_float2(cedP[ea], cedP[eb]);
                cr = make_float2(ce.x / (0.5f * (kapP[ea - 1] + kapP[ea])), ce.y / (0.5f * (kapP[eb - 1] + kapP[eb])));
                dtdye = make_float2(dtdy * cr.x, dtdy * cr.y);
            }
            limit2(wm, I, dtdye, am, ap, F);
            // speeds of the edges of interior rows: ring edges 2 .. h + 2
            if (valid && e0 <= h + 2) smy = fmaxf(smy, fmaxf(-wm.s0.x, wm.s2.x) * cr.x);
            if (valid && e0 + 1 <= h + 2) smy = fmaxf(smy, fmaxf(-wm.s0.y, wm.s2.y) * cr.y);
            if (GEO) {
#pragma unroll
                for (int m = 0; m < 3; m++) { am[m] = mul(ce, am[m]); ap[m] = mul(ce, ap[m]); F[m] = mul(ce, F[m]); }
            }
#pragma unroll
            for (int m = 0; m < 3; m++) { S[m] = add(am[m], F[m]); D[m] = sub(ap[m], F[m]); }

            if (j >= 3) {
                // ---- rows 2j - 4 (lane x) and 2j - 3 (lane y)
                const int kx = 2 * j - 4;
                const int s2 = (j - 2) % YRING;
                const float2 q0 = ring[s2][0][t], qt = ring[s2][1][t], qn = ring[s2][2][t], qB = ring[s2][3][t];
                float2 dtk = dtdy2;
                float2 m0 = add(Dp[0], make_float2(Spy[0], S[0].x));
                if (GEO) {
                    const int rc = y0 - 2 + kx;
                    dtk = make_float2(dtdy / kapP[rc], dtdy / kapP[rc + 1]);
                    // divergence of the edge length
                    m0 = fma(make_float2(cedP[rc + 1] - cedP[rc], cedP[rc + 2] - cedP[rc + 1]), qn, m0);
                }
                float2 n0 = fnma(dtk, m0, q0);
                float2 n1 = fnma(dtk, add(Dp[1], make_float2(Spy[1], S[1].x)), qn);
                float2 n2 = fnma(dtk, add(Dp[2], make_float2(Spy[2], S[2].x)), qt);
                post2(n0, n1, n2, qB, drytol);
                if (a.manningf > 0.0f)   // y frame: n2 = hu, n1 = hv
                    friction2(n0, n2, n1, qB, drytol, a.manningf, dt1 * a.rR);
                const bool sy = kx + 1 <= h + 1;   // lane y's row is interior
                // a surface that is not a finite number reaches the host as an infinite speed
                if (valid && (!(fabsf(n0.x) < 1e30f) || (sy && !(fabsf(n0.y) < 1e30f)))) smy = INFINITY;
                if (valid) {
                    float *d = qo0 + cbase + (long long)kx * pitch;
                    d[0] = n0.x; d[2 * fs] = n1.x; d[fs] = n2.x;
                    if (sy) { d[pitch] = n0.y; d[2 * fs + pitch] = n1.y; d[fs + pitch] = n2.y; }
                }
            }
#pragma unroll
            for (int m = 0; m < 3; m++) { Dp[m] = D[m]; Spy[m] = S[m].y; }
        }
        // carry: waves and the upper cell
        wo[0] = wm.z0m.y; wo[1] = wm.z0n.y; wo[2] = wm.z0t.y; wo[3] = wm.z1t.y;
        wo[4] = wm.z2m.y; wo[5] = wm.z2n.y; wo[6] = wm.z2t.y;
        wm = wn;
        lane_in(cj, 1, pv);
    }
    cp_async_wait<0>();

    if (!(smy > 0.0f)) smy = 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) smy = fmaxf(smy, __shfl_xor_sync(0xffffffffu, smy, o));
    __shared__ float red[NT / 32];
    if ((t & 31) == 0) red[t >> 5] = smy;
    __syncthreads();
    if (t == 0) {
        float my = 0.0f;
#pragma unroll
        for (int q = 0; q < NT / 32; q++) my = fmaxf(my, red[q]);
        atomic_max_speed(a.smax + 2 * P.scen + 1, (double)my);
    }
}

}  // namespace tsu
