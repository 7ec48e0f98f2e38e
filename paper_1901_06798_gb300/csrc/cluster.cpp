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
// Column/row prefix sums make every count and signature O(w + h) per box, so
// the cost is dominated by one pass over the mask.
#include <array>
#include <cstdint>
#include <cstdlib>
#include <vector>

namespace tsu {

namespace {

struct Sums {
    int nx, ny;
    std::vector<int32_t> col;   // col[j * nx + i]: flags in column i, rows < j   ((ny+1) x nx)
    std::vector<int32_t> row;   // row[j * (nx+1) + i]: flags in row j, columns < i (ny x (nx+1))
    std::vector<int64_t> nest;  // 2D prefix of the nestable mask ((ny+1) x (nx+1))

    int colsum(int i, int ja, int jb) const { return col[(size_t)(jb + 1) * nx + i] - col[(size_t)ja * nx + i]; }
    int rowsum(int j, int ia, int ib) const
    {
        return row[(size_t)j * (nx + 1) + ib + 1] - row[(size_t)j * (nx + 1) + ia];
    }
    int64_t nestsum(int ia, int ja, int ib, int jb) const
    {
        size_t W = (size_t)nx + 1;
        return nest[(size_t)(jb + 1) * W + ib + 1] - nest[(size_t)ja * W + ib + 1] - nest[(size_t)(jb + 1) * W + ia] +
               nest[(size_t)ja * W + ia];
    }
};

struct Region {
    int i0, j0, i1, j1;   // inclusive
};

}  // namespace

void cluster_boxes(const uint8_t *F, const uint8_t *N, int nx, int ny, double eff, int ratio, int patch_max,
                   std::vector<std::array<int, 4>> &out)
{
    Sums S;
    S.nx = nx;
    S.ny = ny;
    S.col.assign((size_t)(ny + 1) * nx, 0);
    S.row.assign((size_t)ny * (nx + 1), 0);
    S.nest.assign((size_t)(ny + 1) * (nx + 1), 0);
    for (int j = 0; j < ny; j++) {
        int32_t acc = 0;
        int64_t nacc = 0;
        for (int i = 0; i < nx; i++) {
            uint8_t f = F[(size_t)j * nx + i] ? 1 : 0;
            S.col[(size_t)(j + 1) * nx + i] = S.col[(size_t)j * nx + i] + f;
            acc += f;
            S.row[(size_t)j * (nx + 1) + i + 1] = acc;
            nacc += N[(size_t)j * nx + i] ? 1 : 0;
            S.nest[(size_t)(j + 1) * (nx + 1) + i + 1] = S.nest[(size_t)j * (nx + 1) + i + 1] + nacc;
        }
    }

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
    out.clear();
    for (const auto &b : raw) {
        const int i0 = b[0], j0 = b[1], w = b[2], h = b[3];
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
