// cluster.cpp -- Berger-Rigoutsos clustering of a level's flag mask into
// rectangular boxes (Sec. 3.2), host side of the regrid.
//
// Reading of the algorithm (the paper only cites it):
//   accept the tight bounding box of the flags in a region when
//   flags >= eff * area and every cell is nestable; otherwise cut it --
//   (1) at an empty signature column/row closest to the box centre (in the
//   longer dimension when both exist, x on ties), (2) else at the strongest
//   sign change of the signature Laplacian (strength |lap[i+1] - lap[i]|,
//   ties: closer to the centre, then lower index; x vs y: stronger, then
//   longer, then x), (3) else in the middle of the longer side (x on ties) --
//   and recurse, lower/left part first.  Boxes are finally split into
//   near-equal pieces whose fine size is at most patch_max.
//
// The flags and the nestable mask come packed, 4 cells per byte (cell i of row
// j at byte j * ps + i / 4, bit 2 (i % 4) the flag and bit 2 (i % 4) + 1
// nestable): the plane the regrid packs on the device and copies out.
// 2D prefix sums of the flags and of the nestable mask make every count and
// signature O(w + h) per box, so the cost is dominated by one pass over the
// mask.  They are built only over the flags' bounding box (the recursion's
// first step takes that box anyway), as 32-bit counts, with rows and column
// blocks split across host threads.
#include <algorithm>
#include <array>
#include <cstdint>
#include <cstdlib>
#include <thread>
#include <vector>

#include "host_pool.h"

namespace tsu {

namespace {

struct Sums {
    int nx, ny;
    // 2D prefix sums ((ny+1) x (nx+1)) of the flags (.f) and of the nestable
    // mask (.n), interleaved: P[j][i] counts cells in rows < j, columns < i
    struct Pair {
        int32_t f, n;
    };
    Pair *P;

    const Pair &at(int j, int i) const { return P[(size_t)j * (nx + 1) + i]; }
    int colsum(int i, int ja, int jb) const
    {
        return at(jb + 1, i + 1).f - at(jb + 1, i).f - at(ja, i + 1).f + at(ja, i).f;
    }
    int rowsum(int j, int ia, int ib) const
    {
        return at(j + 1, ib + 1).f - at(j + 1, ia).f - at(j, ib + 1).f + at(j, ia).f;
    }
    int64_t nestsum(int ia, int ja, int ib, int jb) const
    {
        return (int64_t)at(jb + 1, ib + 1).n - at(ja, ib + 1).n - at(jb + 1, ia).n + at(ja, ia).n;
    }
};

struct Region {
    int i0, j0, i1, j1;   // inclusive
};

// run f(lo, hi) over [0, n) split into `threads` contiguous parts on the host pool
template <typename Fn> void parallel_for(int n, int threads, Fn f)
{
    if (threads <= 1 || n < 2 * threads) { f(0, n); return; }
    tsu::HostPool::get().run(threads, [&](int k) {
        f((int)((long long)n * k / threads), (int)((long long)n * (k + 1) / threads));
    });
}

}  // namespace

void cluster_boxes(const uint8_t *Fg, int nxg, int nyg, int ps, double eff, int ratio, int patch_max,
                   std::vector<std::array<int, 4>> &out, int max_threads, std::vector<int32_t> *workspace)
{
    auto cell = [&](const uint8_t *row, int i) { return (row[i >> 2] >> (2 * (i & 3))) & 3; };
    out.clear();
    // threads only pay off on large masks (handing a loop to the pool costs
    // about as much as scanning some tens of thousands of cells)
    const int hw = std::max(1, std::min(16, (int)std::thread::hardware_concurrency()));
    const int threads = std::max(1, std::min({max_threads, hw, (int)((size_t)nxg * nyg / (1u << 18)) + 1}));
    // bounding box of the flags: the recursion's first step takes the tight box
    // of the whole mask, so the prefix sums are only needed inside it
    std::vector<int> rmin(nyg, nxg), rmax(nyg, -1);
    parallel_for(nyg, threads, [&](int ja, int jb) {
        for (int j = ja; j < jb; j++) {
            const uint8_t *r = Fg + (size_t)j * ps;
            const int nb = (nxg + 3) >> 2;
            int lo = -1, hi = -1;
            for (int b = 0; b < nb && lo < 0; b++)
                if (r[b] & 0x55)
                    for (int q = 0; q < 4; q++)
                        if ((r[b] >> (2 * q)) & 1) { lo = 4 * b + q; break; }
            if (lo < 0) continue;
            for (int b = nb - 1; b >= 0 && hi < 0; b--)
                if (r[b] & 0x55)
                    for (int q = 3; q >= 0; q--)
                        if ((r[b] >> (2 * q)) & 1) { hi = 4 * b + q; break; }
            rmin[j] = lo;
            rmax[j] = hi;
        }
    });
    int bi0 = nxg, bi1 = -1, bj0 = -1, bj1 = -1;
    for (int j = 0; j < nyg; j++)
        if (rmax[j] >= 0) {
            if (bj0 < 0) bj0 = j;
            bj1 = j;
            bi0 = std::min(bi0, rmin[j]);
            bi1 = std::max(bi1, rmax[j]);
        }
    if (bj0 < 0) return;
    const int nx = bi1 - bi0 + 1, ny = bj1 - bj0 + 1;

    // workspace kept between calls by the caller, or per thread (regrids
    // repeat with similar sizes): no fresh pages once grown; every entry is
    // written below
    static thread_local std::vector<int32_t> own;
    std::vector<int32_t> &work = workspace ? *workspace : own;
    const size_t W = (size_t)nx + 1, npair = (size_t)(ny + 1) * W;
    if (work.size() < 2 * npair) work.resize(2 * npair);
    Sums S;
    S.nx = nx;
    S.ny = ny;
    S.P = reinterpret_cast<Sums::Pair *>(work.data());
    // row prefixes into rows 1..ny, then accumulated down the columns
    parallel_for(ny, threads, [&](int ja, int jb) {
        for (int j = ja; j < jb; j++) {
            Sums::Pair *r = S.P + (size_t)(j + 1) * W;
            const uint8_t *fr = Fg + (size_t)(j + bj0) * ps;
            int32_t fa = 0, na = 0;
            r[0] = {0, 0};
            for (int i = 0; i < nx; i++) {
                const int v = cell(fr, bi0 + i);
                fa += v & 1;
                na += v >> 1;
                r[i + 1] = {fa, na};
            }
        }
    });
    parallel_for((int)W, threads, [&](int ia, int ib) {
        for (int i = ia; i < ib; i++) S.P[i] = {0, 0};
        for (int j = 1; j <= ny; j++) {
            Sums::Pair *r = S.P + (size_t)j * W;
            const Sums::Pair *u = r - W;
            for (int i = ia; i < ib; i++) { r[i].f += u[i].f; r[i].n += u[i].n; }
        }
    });

    std::vector<std::array<int, 4>> raw;
    std::vector<Region> stack;
    stack.push_back({0, 0, nx - 1, ny - 1});
    std::vector<int> sx, sy;
    while (!stack.empty()) {
        Region R = stack.back();
        stack.pop_back();
        // tight bounding box from the region's signatures
        int i0 = -1, i1 = -1, j0 = -1, j1 = -1;
        for (int i = R.i0; i <= R.i1; i++)
            if (S.colsum(i, R.j0, R.j1)) { if (i0 < 0) i0 = i; i1 = i; }
        if (i0 < 0) continue;
        for (int j = R.j0; j <= R.j1; j++)
            if (S.rowsum(j, R.i0, R.i1)) { if (j0 < 0) j0 = j; j1 = j; }
        const int w = i1 - i0 + 1, h = j1 - j0 + 1;
        sx.assign(w, 0);
        sy.assign(h, 0);
        long long nf = 0;
        for (int i = 0; i < w; i++) { sx[i] = S.colsum(i0 + i, j0, j1); nf += sx[i]; }
        for (int j = 0; j < h; j++) sy[j] = S.rowsum(j0 + j, i0, i1);
        const long long area = (long long)w * h;
        const bool nested = S.nestsum(i0, j0, i1, j1) == area;
        if ((double)nf >= eff * (double)area && nested) {
            raw.push_back({i0, j0, w, h});
            continue;
        }
        int dim = -1, at = 0;
        // (1) signature holes
        int hx = -1, hy = -1;
        long bx = 0, by = 0;
        for (int i = 1; i <= w - 2; i++)
            if (sx[i] == 0) {
                long d = std::labs(2L * i - (w - 1));
                if (hx < 0 || d < bx) { hx = i; bx = d; }
            }
        for (int j = 1; j <= h - 2; j++)
            if (sy[j] == 0) {
                long d = std::labs(2L * j - (h - 1));
                if (hy < 0 || d < by) { hy = j; by = d; }
            }
        if (hx >= 0 && (hy < 0 || w >= h)) { dim = 0; at = hx; }
        else if (hy >= 0) { dim = 1; at = hy; }
        // (2) Laplacian inflections
        if (dim < 0) {
            auto best = [](const std::vector<int> &s, int n, long &strength, int &pos) {
                strength = -1;
                pos = -1;
                long dist = 0;
                for (int i = 1; i + 2 <= n - 1; i++) {
                    long la = (long)s[i - 1] - 2L * s[i] + s[i + 1];
                    long lb = (long)s[i] - 2L * s[i + 1] + s[i + 2];
                    if ((la < 0 && lb > 0) || (la > 0 && lb < 0)) {
                        long st = std::labs(lb - la), d = std::labs(2L * i + 1 - (n - 1));
                        if (st > strength || (st == strength && d < dist)) { strength = st; dist = d; pos = i; }
                    }
                }
            };
            long stx, sty;
            int ix, iy;
            best(sx, w, stx, ix);
            best(sy, h, sty, iy);
            if (ix >= 0 && (iy < 0 || stx > sty || (stx == sty && w >= h))) { dim = 0; at = ix; }
            else if (iy >= 0) { dim = 1; at = iy; }
        }
        // (3) bisection
        if (dim < 0) {
            if (w >= h) { dim = 0; at = w / 2 - 1; }
            else { dim = 1; at = h / 2 - 1; }
        }
        // depth first, lower/left part first: push the second part first
        if (dim == 0) {
            stack.push_back({i0 + at + 1, j0, i1, j1});
            stack.push_back({i0, j0, i0 + at, j1});
        } else {
            stack.push_back({i0, j0 + at + 1, i1, j1});
            stack.push_back({i0, j0, i1, j0 + at});
        }
    }

    const int pm = patch_max / ratio > 0 ? patch_max / ratio : 1;
    for (const auto &b : raw) {
        const int i0 = b[0] + bi0, j0 = b[1] + bj0, w = b[2], h = b[3];   // back to level indices
        const int npx = (w + pm - 1) / pm, npy = (h + pm - 1) / pm;
        for (int q = 0; q < npy; q++)
            for (int p = 0; p < npx; p++) {
                int xa = i0 + (int)((long long)p * w / npx), xb = i0 + (int)((long long)(p + 1) * w / npx);
                int ya = j0 + (int)((long long)q * h / npy), yb = j0 + (int)((long long)(q + 1) * h / npy);
                out.push_back({xa, ya, xb - xa, yb - ya});
            }
    }
}

}  // namespace tsu
