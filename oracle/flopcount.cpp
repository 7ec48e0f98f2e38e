// flopcount.cpp -- the oracle's patch update (swe.c) compiled with a counting
// scalar type, to state how many floating-point operations of each kind one
// interior cell update of the split scheme takes (the algorithmic flop count of
// the measurement).  Test infrastructure like the rest of oracle/: swe.c is
// included unchanged; only the meaning of `double` and `malloc` changes in this
// translation unit.  Operations are counted as the oracle performs them, without
// contraction: a*b + c is one multiply and one add.
#include <cmath>
#include <cstddef>
#include <cstdlib>
#include <cstring>
#include <math.h>
#include <stdlib.h>
#include <string.h>

namespace fc {

struct Counts {
    long long add, mul, div, sqrt, cmp, minmax, abs, neg;
};
static Counts N;

struct cd {
    double v;
    cd() = default;
    cd(double x) : v(x) {}
    cd(int x) : v(x) {}
    explicit operator double() const { return v; }
    cd &operator+=(cd o) { N.add++; v += o.v; return *this; }
    cd &operator-=(cd o) { N.add++; v -= o.v; return *this; }
    cd &operator*=(cd o) { N.mul++; v *= o.v; return *this; }
    cd &operator/=(cd o) { N.div++; v /= o.v; return *this; }
};
inline cd operator+(cd a, cd b) { N.add++; return cd(a.v + b.v); }
inline cd operator-(cd a, cd b) { N.add++; return cd(a.v - b.v); }
inline cd operator*(cd a, cd b) { N.mul++; return cd(a.v * b.v); }
inline cd operator/(cd a, cd b) { N.div++; return cd(a.v / b.v); }
inline cd operator-(cd a) { N.neg++; return cd(-a.v); }
inline bool operator<(cd a, cd b) { N.cmp++; return a.v < b.v; }
inline bool operator>(cd a, cd b) { N.cmp++; return a.v > b.v; }
inline bool operator<=(cd a, cd b) { N.cmp++; return a.v <= b.v; }
inline bool operator>=(cd a, cd b) { N.cmp++; return a.v >= b.v; }
inline bool operator==(cd a, cd b) { N.cmp++; return a.v == b.v; }
inline bool operator!=(cd a, cd b) { N.cmp++; return a.v != b.v; }
inline cd sqrt(cd a) { N.sqrt++; return cd(std::sqrt(a.v)); }
inline cd fabs(cd a) { N.abs++; return cd(std::fabs(a.v)); }
inline cd fmin(cd a, cd b) { N.minmax++; return cd(std::fmin(a.v, b.v)); }
inline cd fmax(cd a, cd b) { N.minmax++; return cd(std::fmax(a.v, b.v)); }
inline cd pow(cd a, cd b) { N.div++; N.mul++; return cd(std::pow(a.v, b.v)); }

// malloc's result converts to any object pointer, as in C
struct vp {
    void *p;
    template <class T> operator T *() const { return static_cast<T *>(p); }
};

}  // namespace fc

namespace ora {
using fc::cd;
using fc::sqrt;
using fc::fabs;
using fc::fmin;
using fc::fmax;
using fc::pow;
#define double cd
#define malloc(n) (fc::vp{std::malloc(n)})
#include "swe.c"
#undef malloc
#undef double
}  // namespace ora

// One split step of an nx x ny patch (arrays of (nx + 4) x (ny + 4) doubles,
// ghost cells filled, row pitch nx + 4).  out[8] receives the operation counts
// (add/sub, mul, div, sqrt, compare, min/max, abs, negate); the updated state
// is written back to h, hu, hv.
extern "C" int flop_count_step(int nx, int ny, double *h, double *hu, double *hv, const double *B, double g,
                               double drytol, double dt, double dx, double dy, long long *out)
{
    if (nx < 1 || ny < 1 || !h || !hu || !hv || !B || !out) return 1;
    const size_t n = (size_t)(nx + 4) * (ny + 4);
    fc::cd *a = static_cast<fc::cd *>(std::malloc(4 * n * sizeof(fc::cd)));
    if (!a) return 2;
    for (size_t k = 0; k < n; k++) {
        a[k] = fc::cd(h[k]);
        a[n + k] = fc::cd(hu[k]);
        a[2 * n + k] = fc::cd(hv[k]);
        a[3 * n + k] = fc::cd(B[k]);
    }
    ora::OPatch p;
    std::memset(static_cast<void *>(&p), 0, sizeof p);
    p.nx = nx; p.ny = ny; p.pitch = nx + 4;
    p.h = a; p.hu = a + n; p.hv = a + 2 * n; p.B = a + 3 * n;
    fc::cd sx(0.0), sy(0.0);
    fc::N = fc::Counts{};
    ora::ora_step_patch(&p, fc::cd(g), fc::cd(drytol), fc::cd(dt), fc::cd(dx), fc::cd(dy), &sx, &sy);
    const fc::Counts c = fc::N;
    out[0] = c.add; out[1] = c.mul; out[2] = c.div; out[3] = c.sqrt;
    out[4] = c.cmp; out[5] = c.minmax; out[6] = c.abs; out[7] = c.neg;
    for (size_t k = 0; k < n; k++) {
        h[k] = a[k].v;
        hu[k] = a[n + k].v;
        hv[k] = a[2 * n + k].v;
    }
    std::free(a);
    return 0;
}
