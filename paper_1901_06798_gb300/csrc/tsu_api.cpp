// tsu_api.cpp -- host runtime of the library behind the C ABI of tsunami.h.
//
// It owns the device memory pool (Sec. 4.2), the per-level patch tables, the
// recursive level integration of Sec. 3.1 (steps 1-4; refluxing omitted as
// in the paper's GPU code), the regridding of Sec. 3.2 (flags, buffer and
// nesting on the device, clustering on the host, new patches initialised on
// the device) and CUDA-graph replay of repeated coarse steps.  dt, t, wave
// speeds and CFL checks stay on the device; the host only reads them back at
// the end of a call.  Every numerical step runs in the library's kernels.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <map>
#include <set>
#include <stdexcept>
#include <string>
#include <vector>
#include <unordered_map>
#include <chrono>
#include <thread>

#include <cuda_runtime.h>

#include "../../include/tsunami.h"
#include "amr_kernels.h"
#include "cnn.h"
#include "host_pool.h"
#include "tsu_device.h"

namespace tsu {
// FN: 4 cells per byte, rows ps bytes apart; cell i: bit 2 (i % 4) the flag, bit 2 (i % 4) + 1 nestable
void cluster_boxes(const uint8_t *FN, int nx, int ny, int ps, double eff, int ratio, int patch_max,
                   std::vector<std::array<int, 4>> &out, int max_threads, std::vector<int32_t> *workspace);
}

using namespace tsu;

namespace {

struct Err : std::runtime_error {
    int code;
    Err(int c, const std::string &m) : std::runtime_error(m), code(c) {}
};

#define CK(x)                                                                                           \
    do {                                                                                                \
        cudaError_t e_ = (x);                                                                           \
        if (e_ != cudaSuccess) throw Err(TSU_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    } while (0)

int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// the largest float <= t: a float x exceeds t exactly when x exceeds it
float float_at_most(double t)
{
    float f = (float)t;
    if ((double)f > t) f = std::nextafter(f, -std::numeric_limits<float>::infinity());
    return f;
}

// f(q, begin, end) over contiguous ranges of [0, n), ranges in order q = 0, 1, ..;
// on the host pool (up to 16 threads) when n is large enough to pay for it
template <typename F> void parallel_ranges(int n, F &&f)
{
    const int T = n < 512 ? 1 : tsu::HostPool::get().size();
    if (T == 1) {
        f(0, 0, n);
        return;
    }
    tsu::HostPool::get().run(T, [&](int q) { f(q, (int)((long long)n * q / T), (int)((long long)n * (q + 1) / T)); });
}

// Host-to-device uploads of the tables a regrid rebuilds go through a
// page-locked ring.  A copy from pageable memory first waits for all the work
// queued on the stream; one from page-locked memory does not, so the host goes
// on building the next tables while the device runs the regrid's kernels.  A
// part of the ring is written again only once the copies out of it have
// landed: the ring is filled front to back, and before it starts over (or
// grows) the host waits for the last copy queued.
struct UploadRing {
    uint8_t *p = nullptr;
    size_t cap = 0, head = 0;
    cudaEvent_t ev = nullptr;
    bool pending = false;
    void copy(void *dst, const void *src, size_t bytes, cudaStream_t st)
    {
        if (bytes == 0) return;
        const size_t need = (bytes + 255) & ~(size_t)255;
        if (head + need > cap) {
            if (pending) {
                CK(cudaEventSynchronize(ev));
                pending = false;
            }
            head = 0;
            if (need > cap) {
                const size_t nc = std::max(need, std::max((size_t)16 << 20, cap * 2));
                if (p) cudaFreeHost(p);
                p = nullptr;
                cap = 0;
                CK(cudaMallocHost((void **)&p, nc));
                cap = nc;
            }
        }
        std::memcpy(p + head, src, bytes);
        CK(cudaMemcpyAsync(dst, p + head, bytes, cudaMemcpyHostToDevice, st));
        if (!ev) CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        CK(cudaEventRecord(ev, st));
        pending = true;
        head += need;
    }
    ~UploadRing()
    {
        if (ev) {
            cudaEventSynchronize(ev);
            cudaEventDestroy(ev);
        }
        if (p) cudaFreeHost(p);
    }
};

template <typename T> struct DevBuf {
    T *p = nullptr;
    size_t cap = 0;
    cudaStream_t st = nullptr;
    void ensure(size_t n, cudaStream_t s)
    {
        st = s;
        if (n <= cap && p) return;
        size_t nc = std::max<size_t>(n, 16);
        if (p) CK(cudaFreeAsync(p, s));
        p = nullptr;
        CK(cudaMallocAsync((void **)&p, nc * sizeof(T), s));
        cap = nc;
    }
    void upload(const std::vector<T> &v, cudaStream_t s)
    {
        ensure(v.size(), s);
        if (!v.empty()) CK(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    }
    // through the page-locked ring: no wait for the stream's queued work
    void upload(const std::vector<T> &v, cudaStream_t s, UploadRing &r)
    {
        ensure(v.size(), s);
        r.copy(p, v.data(), v.size() * sizeof(T), s);
    }
    void release()
    {
        if (p) cudaFreeAsync(p, st);
        p = nullptr;
        cap = 0;
    }
};

// Device memory pool (Sec. 4.2): one chunk sub-allocated first-fit; when it is
// full it is replaced by a chunk twice as large and the contents are copied,
// so patch offsets stay valid and regrids never call the CUDA allocator for
// individual patches.
struct Arena {
    char *base = nullptr;
    size_t cap = 0;
    // free blocks by offset (for coalescing) and by size (best fit); the two
    // always hold the same blocks
    std::map<size_t, size_t> freel;             // offset -> bytes
    std::set<std::pair<size_t, size_t>> bysize;  // (bytes, offset)
    static size_t rnd(size_t b) { return (b + 255) & ~(size_t)255; }
    void add_free(size_t off, size_t bytes)
    {
        freel[off] = bytes;
        bysize.emplace(bytes, off);
    }
    void drop_free(std::map<size_t, size_t>::iterator it)
    {
        bysize.erase({it->second, it->first});
        freel.erase(it);
    }
    // insert a free block and merge it with its neighbours
    void insert_free(size_t off, size_t bytes)
    {
        auto nx = freel.lower_bound(off);
        if (nx != freel.end() && off + bytes == nx->first) {
            bytes += nx->second;
            drop_free(nx);
        }
        auto it = freel.lower_bound(off);
        if (it != freel.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == off) {
                off = pv->first;
                bytes += pv->second;
                drop_free(pv);
            }
        }
        add_free(off, bytes);
    }
    void reserve(size_t bytes, cudaStream_t st)
    {
        if (bytes <= cap) return;
        size_t nc = std::max(bytes, cap * 2);
        char *nb = nullptr;
        CK(cudaMallocAsync((void **)&nb, nc, st));
        if (base) {
            CK(cudaMemcpyAsync(nb, base, cap, cudaMemcpyDeviceToDevice, st));
            CK(cudaFreeAsync(base, st));
        }
        // the new tail is free
        const size_t tail = cap;
        base = nb;
        cap = nc;
        insert_free(tail, nc - tail);
    }
    // the smallest free block that fits (patches of a level come in a few sizes,
    // so a released block of the same size is usually reused exactly)
    size_t alloc(size_t bytes, cudaStream_t st)
    {
        bytes = rnd(bytes);
        for (int pass = 0; pass < 2; pass++) {
            auto it = bysize.lower_bound({bytes, 0});
            if (it != bysize.end()) {
                const size_t sz = it->first, off = it->second;
                bysize.erase(it);
                freel.erase(off);
                if (sz > bytes) add_free(off + bytes, sz - bytes);
                return off;
            }
            reserve(cap + bytes, st);
        }
        throw Err(TSU_ERR_OOM, "arena allocation failed");
    }
    void release(size_t off, size_t bytes) { insert_free(off, rnd(bytes)); }
};

struct Grid {
    int nx, ny;
    double x0, y0, dx, dy;
    std::vector<double> v;
    int scen;   // -1 base topography, >= 0 uplift layer of that scenario, -2 surface grid
    double *dev = nullptr;
};

// page-locked host buffer, grown on demand (device-to-host copies at full link speed)
struct PinnedHost {
    uint8_t *p = nullptr;
    size_t cap = 0;
    // grows by half again at least: page-locked allocation is slow and freeing
    // synchronises the device, and the staged sizes creep up from regrid to regrid
    void ensure(size_t n)
    {
        if (n <= cap) return;
        const size_t nc = std::max(n, cap + cap / 2);
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        CK(cudaMallocHost((void **)&p, nc));
        cap = nc;
    }
    ~PinnedHost()
    {
        if (p) cudaFreeHost(p);
    }
};

// Spatial buckets of one scenario's patches on one level, for neighbour and
// covering-patch lookups while tables are rebuilt.
struct BoxIndex {
    // patches bucketed by bs x bs cell tiles, in compressed rows: bucket k
    // holds ids[start[k] .. start[k+1])
    int bs = 64, nbx = 0, nby = 0;
    std::vector<int> start, ids, fillv;   // kept between builds (no fresh pages per regrid)
    const std::vector<PatchDesc> *P = nullptr;
    void build(const std::vector<PatchDesc> &Pv, const std::vector<int> &which, int nxl, int nyl)
    {
        P = &Pv;
        // tiles of 64 cells, doubled until there are at most 2^14 of them: a
        // build is linear in the tiles, a query in the patches per tile
        bs = 64;
        while ((size_t)((nxl + bs - 1) / bs) * (size_t)((nyl + bs - 1) / bs) > (1u << 14)) bs *= 2;
        nbx = (nxl + bs - 1) / bs;
        nby = (nyl + bs - 1) / bs;
        start.assign((size_t)nbx * nby + 1, 0);
        auto each = [&](auto f) {
            for (int id : which) {
                const PatchDesc &q = Pv[id];
                for (int by = q.j0 / bs; by <= (q.j0 + q.ny - 1) / bs; by++)
                    for (int bx = q.i0 / bs; bx <= (q.i0 + q.nx - 1) / bs; bx++) f((size_t)by * nbx + bx, id);
            }
        };
        each([&](size_t k, int) { start[k + 1]++; });
        for (size_t k = 0; k + 1 < start.size(); k++) start[k + 1] += start[k];
        ids.resize(start.back());
        fillv.assign(start.begin(), start.end() - 1);
        each([&](size_t k, int id) { ids[fillv[k]++] = id; });
    }
    int find(int I, int J) const
    {
        if (I < 0 || J < 0 || I >= nbx * bs || J >= nby * bs) return -1;
        const size_t k = (size_t)(J / bs) * nbx + I / bs;
        for (int e = start[k]; e < start[k + 1]; e++) {
            const PatchDesc &q = (*P)[ids[e]];
            if (I >= q.i0 && I < q.i0 + q.nx && J >= q.j0 && J < q.j0 + q.ny) return ids[e];
        }
        return -1;
    }
    void overlapping(int ia, int ja, int ib, int jb, std::vector<int> &out) const   // half-open box
    {
        out.clear();
        if (nbx == 0 || nby == 0) return;
        int bxa = std::max(0, floordiv(ia, bs)), bxb = std::min(nbx - 1, floordiv(ib - 1, bs));
        int bya = std::max(0, floordiv(ja, bs)), byb = std::min(nby - 1, floordiv(jb - 1, bs));
        for (int by = bya; by <= byb; by++)
            for (int bx = bxa; bx <= bxb; bx++) {
                const size_t k = (size_t)by * nbx + bx;
                for (int e = start[k]; e < start[k + 1]; e++) {
                    const PatchDesc &q = (*P)[ids[e]];
                    if (q.i0 < ib && q.i0 + q.nx > ia && q.j0 < jb && q.j0 + q.ny > ja) out.push_back(ids[e]);
                }
            }
        std::sort(out.begin(), out.end());
        out.erase(std::unique(out.begin(), out.end()), out.end());
    }
};

constexpr int kRetakeThreads = 256, kRetakeRows = 64;   // x-sweep shape of the level-1 retake launch

struct Lvl {
    std::vector<PatchDesc> P;
    std::vector<size_t> blk, blkbytes;
    std::vector<StepItem> items, items_y;   // patch update work items (items_y: FP32 split y kernel)
    std::vector<StepItem> items_rt;         // level 1, FP32 split update: x-sweep items of the retake launch
    std::vector<int> nbrs, bclist, olds;
    std::vector<BoxIndex> idx;   // per scenario spatial index of P, rebuilt by every finish_level of the level
    std::vector<int> ccand;   // coarse patches overlapping each patch's coarse-map footprint
    DevBuf<PatchDesc> dP;
    DevBuf<StepItem> dItems, dItemsY, dItemsRt;
    DevBuf<float> dScratch;                 // FP32 split update: Q* of every patch (3 fields each)
    DevBuf<int> dNbrs, dCmap, dCcand, dBc, dOlds, dList;
    DevBuf<GhostSrc> dGmap;      // ghost-cell sources of every patch, in ghost-ring order
    DevBuf<long long> dGoff;     // first dGmap entry of each patch
    DevBuf<int2> dGinterp;       // ghost cells interpolated from the coarser level (patch, ring index)
    DevBuf<int> dGcount;         // entries of dGinterp
    std::vector<long long> goff;
    int cur = 0, maxring = 0, maxcells = 0;
    int nxl = 0, nyl = 0;
    double dx = 0, dy = 0, R = 1;
    // latitude-longitude grids: physical equatorial cell sizes and the row tables
    double dxp = 0, dyp = 0;
    DevBuf<double> dKap, dCed;
    DevBuf<float> dKapF, dCedF;
};


}  // namespace

struct tsu_ctx {
    tsu_config c{};
    int prec = 0;
    size_t esz = 8;
    int nlev = 1, nscen = 1;
    int ratio[kMaxLevels] = {0};
    cudaStream_t st = nullptr;
    bool own_stream = false;
    std::string err;
    Arena arena;
    UploadRing uring;   // regrid table uploads (declared before the levels: destroyed after them)
    Lvl lv[kMaxLevels];
    std::vector<Grid> grids;   // base topography first, then layers and surfaces in call order
    int nbase = 0;
    std::vector<int> eta_index;   // per scenario: initial surface, u and v grid indices (-1: none)
    DevBuf<TopoDev> dGrids;
    DevBuf<int> dGridScen, dEtaIdx;
    bool topo_dirty = true;
    // control block
    DevBuf<double> dt1, t, rate, cellupd, cells, Rl, mass;
    DevBuf<float> dt1f;
    DevBuf<long long> viol, retakes;
    DevBuf<unsigned long long> smax;
    DevBuf<int> derr, retake;
    std::vector<double> cells_h;
    std::vector<std::array<long long, kMaxLevels>> nsteps;
    bool initialized = false;
    // gauges
    std::vector<double> gxy;
    DevBuf<double> dgxy, dgeta, dgt;
    DevBuf<long long> dnsamp;
    DevBuf<GaugeLoc> dgloc;
    long long samp_cap = 0, nsamp = 0;
    // flags
    DevBuf<uint8_t> fraw, fcov, ftmp, fF, fN, fpack;
    DevBuf<int> fslot, fbox;
    // statistics and graphs
    long long launches = 0;
    long long viol_seen = 0;
    PinnedHost hflags;           // page-locked staging of the flag masks for clustering
    std::vector<unsigned long long> same_keys;       // regrid: old boxes by key (open addressing)
    std::vector<int> same_ids;
    std::vector<std::vector<int32_t>> cws = std::vector<std::vector<int32_t>>(16);   // clustering workspaces
    long long n_regrids = 0;     // host-side regrid accounting (tsu_stats)
    double regrid_ms = 0.0, cluster_ms = 0.0, regrid_wait_ms = 0.0;
    long long n_patches_renewed = 0, n_patches_reused = 0;   // new patches at regrids, of which kept their block
    bool ext_state = false;           // a state came from the caller (tsu_level1_buffers, restore): check its depths
    DevBuf<int> dneg;                 // count of the depth check
    int bulk_rows = 0;                // FP32 split update: x-sweep rows by bulk copies (tsu_set_bulk_copies)
    unsigned wait_polls = 1u << 22;   // polls a kernel spends on one bulk copy before giving up
    int seg_rows = 0;  // rows per work item of the patch update (0: library default)
    int step_nt = 0;   // threads per CTA of the patch update (0: library default)
    DevBuf<double> zero_dt;
    DevBuf<float> zero_dtf;
    // refinement-flag predictor
    DevBuf<float> cnn_theta, cnn_feat, cnn_logits;
    DevBuf<char> cnn_half;
    bool cnn_ready = false;
    long long hier_version = 0;
    // graphs of one or two coarse steps, keyed by the number of steps and the
    // levels' buffer parities at their start: a captured step reads and writes
    // the buffers that were current when it was captured
    struct StepGraph {
        int m;                              // coarse steps in the graph
        unsigned key;                       // parity pattern at its start
        cudaGraphExec_t ex;
        std::array<int, kMaxLevels> post;   // the parities it leaves
        long long kernels;
    };
    std::vector<StepGraph> graphs;
    long long graphs_version = -1;
    // tsu_step_level: pend[l] = steps of level l + 2 (1-based) still to take
    // within the current step of level l + 1; all zero when the hierarchy is
    // synchronised (between coarse steps)
    std::array<int, kMaxLevels> pend{};
    // per-level timing of the patch update (tsu_profile_levels): CUDA events
    // around each level step's update launches, and the interior cells and
    // launches they covered
    bool prof = false;
    struct ProfStep {
        int level;
        cudaEvent_t e0, e1;
        double cells;
        int kernels;
    };
    std::vector<ProfStep> prof_steps;
    std::vector<cudaEvent_t> prof_pool;
    cudaEvent_t prof_event()
    {
        if (!prof_pool.empty()) {
            cudaEvent_t e = prof_pool.back();
            prof_pool.pop_back();
            return e;
        }
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        return e;
    }
    bool synchronised() const
    {
        for (int l = 0; l < nlev; l++)
            if (pend[l]) return false;
        return true;
    }
    DevBuf<double> dstage;
    DevBuf<double> massParts;                  // per-block partial masses of tsu_get_stats
    PinnedHost hsmall;                         // page-locked readback of error flag, CFL counts, times
    cudaEvent_t stage_ev[8] = {};
    int device = 0;                            // the CUDA device current at tsu_create

    // ------------------------------------------------------------ helpers
    // FP32 split scheme: the patch update runs as the x and y kernels with a Q* scratch
    bool split_f32() const { return prec != TSU_F64 && c.transverse == 0; }
    int nt() const
    {
        if (step_nt > 0) return step_nt;
        return prec == TSU_F64 ? step_threads_f64() : (split_f32() ? 32 : step_threads_f32p());
    }
    // physical cell sizes of level l (of an equatorial cell on latitude-longitude grids)
    double pdx(int l) const { return c.spherical ? lv[l].dxp : lv[l].dx; }
    double pdy(int l) const { return c.spherical ? lv[l].dyp : lv[l].dy; }
    // per-level launch data of the patch update: cell sizes, latitude-longitude
    // tables, and the FP32 split kernels' scratch and y work items
    void level_args(StepArgs &a, int l) const
    {
        a.dx = pdx(l);
        a.dy = pdy(l);
        if (c.spherical) {
            a.kap = lv[l].dKap.p; a.ced = lv[l].dCed.p; a.kapf = lv[l].dKapF.p; a.cedf = lv[l].dCedF.p;
        }
        if (split_f32()) {
            a.scratch = lv[l].dScratch.p;
            a.items_y = lv[l].dItemsY.p;
            a.n_items_y = (int)lv[l].items_y.size();
        }
        a.err = derr.p;
        a.bulk_rows = bulk_rows;
        a.wait_polls = wait_polls;
    }
    const int *retake_gate() const { return retake.p; }
    // kernels one patch-update launch of level l runs
    int step_kernels() const { return split_f32() ? 2 : 1; }
    int seg() const { return seg_rows > 0 ? seg_rows : (prec == TSU_F64 ? 128 : (split_f32() ? 16 : 64)); }
    // the level-1 retake launch (a.gate set): the FP32 split update sweeps x with
    // its own wide items, the rest as the step itself
    int retake_launch(StepArgs a, const Lvl &L)
    {
        if (prec != TSU_F64 && !L.items_rt.empty() && a.scratch != nullptr && !a.transverse) {
            a.items = L.dItemsRt.p;
            return launch_step_f32p(a, (int)L.items_rt.size(), kRetakeThreads, st);
        }
        return prec == TSU_F64 ? launch_step_f64(a, (int)L.items.size(), nt(), st)
                               : launch_step_f32p(a, (int)L.items.size(), nt(), st);
    }
    void kl(int e, const char *what)
    {
        launches++;
        if (e != 0) throw Err(TSU_ERR_CUDA, std::string("kernel launch (") + what + "): " + cudaGetErrorString((cudaError_t)e));
    }
    CtrlView ctrl()
    {
        CtrlView v;
        v.dt1 = dt1.p; v.dt1f = dt1f.p; v.t = t.p; v.rate = rate.p; v.cell_updates = cellupd.p; v.cells = cells.p;
        v.cfl_viol = viol.p; v.smax = smax.p; v.max_levels = kMaxLevels;
        v.retake = retake.p; v.retakes = retakes.p; v.err = derr.p;
        return v;
    }
    LevelView view(int l, const PatchDesc *descs = nullptr)
    {
        LevelView v;
        v.descs = descs ? descs : lv[l].dP.p;
        v.arena = arena.base;
        v.nxl = lv[l].nxl; v.nyl = lv[l].nyl;
        v.nbrs = lv[l].dNbrs.p; v.cmap = lv[l].dCmap.p; v.olds = lv[l].dOlds.p;
        v.kap = c.spherical ? lv[l].dKap.p : nullptr;
        v.ced = c.spherical ? lv[l].dCed.p : nullptr;
        v.gmap = lv[l].dGmap.p; v.goff = lv[l].dGoff.p;
        v.ilist = lv[l].dGinterp.p; v.icount = lv[l].dGcount.p;
        return v;
    }
    // the topography set with axis-table storage for a level of nx x ny cells
    DevBuf<int> tabI;
    DevBuf<double> tabT;
    DevBuf<unsigned char> tabIn;
    TopoSet topo(int l)
    {
        TopoSet ts = topo();
        const size_t n = (size_t)grids.size() * (size_t)(lv[l].nxl + lv[l].nyl);
        tabI.ensure(n, st);
        tabT.ensure(n, st);
        tabIn.ensure(n, st);
        const size_t nc = (size_t)grids.size() * lv[l].nxl;
        ts.tab.ci = tabI.p; ts.tab.rj = tabI.p + nc;
        ts.tab.ct = tabT.p; ts.tab.rt = tabT.p + nc;
        ts.tab.cin = tabIn.p; ts.tab.rin = tabIn.p + nc;
        ts.tab.nx = lv[l].nxl; ts.tab.ny = lv[l].nyl;
        return ts;
    }
    TopoSet topo()
    {
        TopoSet ts{};
        ts.grids = dGrids.p; ts.scen = dGridScen.p; ts.eta_index = dEtaIdx.p;
        ts.nbase = nbase; ts.ngrids = (int)grids.size();
        ts.drytol = c.drytol;
        return ts;
    }
    void sync() { CK(cudaStreamSynchronize(st)); }
    bool has_patches(int s, int l) const
    {
        for (const auto &p : lv[l].P) if (p.scen == s) return true;
        return false;
    }

    void upload_topo()
    {
        std::vector<TopoDev> td(grids.size());
        std::vector<int> sc(grids.size());
        for (size_t k = 0; k < grids.size(); k++) {
            Grid &g = grids[k];
            if (!g.dev) {
                CK(cudaMallocAsync((void **)&g.dev, g.v.size() * sizeof(double), st));
                CK(cudaMemcpyAsync(g.dev, g.v.data(), g.v.size() * sizeof(double), cudaMemcpyHostToDevice, st));
            }
            td[k] = TopoDev{g.nx, g.ny, g.x0, g.y0, g.dx, g.dy, g.dev};
            sc[k] = g.scen >= 0 ? g.scen : -1;
        }
        dGrids.upload(td, st);
        dGridScen.upload(sc, st);
        dEtaIdx.upload(eta_index, st);
        topo_dirty = false;
    }

    // ------------------------------------------------------------ level tables
    PatchDesc make_desc(int l, int s, int i0, int j0, int nx, int ny)
    {
        PatchDesc d{};
        d.i0 = i0; d.j0 = j0; d.nx = nx; d.ny = ny; d.scen = s;
        d.pitch = (nx + 4 + 3) & ~3;
        long long fs = (long long)d.pitch * (ny + 4);
        fs = (fs + 63) & ~63LL;
        d.fs = fs;
        // ghost cells reach outside the domain (the patch lies within 2 cells of an edge)
        d.bcmask = (i0 < 2 ? 1 : 0) | (i0 + nx > lv[l].nxl - 2 ? 2 : 0) | (j0 < 2 ? 4 : 0) |
                   (j0 + ny > lv[l].nyl - 2 ? 8 : 0);
        return d;
    }

    // Rebuild everything derived from the patch list of level l: step items,
    // same-level neighbour lists, coarse maps, boundary lists, cell counts.
    void finish_level(int l)
    {
        Lvl &L = lv[l];
        const int n = (int)L.P.size();
        L.items.clear();
        L.nbrs.clear();
        L.bclist.clear();
        L.maxring = 0;
        L.maxcells = 0;
        L.items_y.clear();
        const int W = prec == TSU_F64 ? step_strip_width_f64(nt(), c.transverse) : step_strip_width_f32p(nt(), c.transverse);
        const bool split = split_f32();
        size_t soff = 0;
        for (int k = 0; k < n; k++) {
            PatchDesc &p = L.P[k];
            p.soff = split ? (long long)soff : 0;
            if (split) soff += 3 * (size_t)p.fs;
            L.maxring = std::max(L.maxring, (p.nx + 4) * (p.ny + 4) - p.nx * p.ny);
            L.maxcells = std::max(L.maxcells, (p.nx + 4) * (p.ny + 4));
            if (p.bcmask) L.bclist.push_back(k);
        }
        // work items of the patch update in patch order, built in patch ranges on
        // host threads and joined in range order
        {
            const int sg = seg();
            std::vector<std::vector<StepItem>> xi(16), yi(16);
            std::array<std::array<int, 2>, 16> rr{};
            parallel_ranges(n, [&](int q, int b, int e) {
                rr[q] = {b, e};
                std::vector<StepItem> &ox = xi[q], &oy = yi[q];
                for (int k = b; k < e; k++) {
                    const PatchDesc &p = L.P[k];
                    if (split) {
                        // x kernel: every row including the ghost rows, no halo rows; y kernel:
                        // strips of 64 columns and segments of 64 interior rows
                        for (int x0 = 0; x0 < p.nx; x0 += W)
                            for (int y0 = -2; y0 < p.ny + 2; y0 += sg)
                                ox.push_back(StepItem{k, x0, y0, std::min(W, p.nx - x0), std::min(sg, p.ny + 2 - y0)});
                        constexpr int WY = 64, SY = 64;
                        for (int x0 = 0; x0 < p.nx; x0 += WY)
                            for (int y0 = 0; y0 < p.ny; y0 += SY)
                                oy.push_back(StepItem{k, x0, y0, std::min(WY, p.nx - x0), std::min(SY, p.ny - y0)});
                    } else {
                        for (int x0 = 0; x0 < p.nx; x0 += W)
                            for (int y0 = 0; y0 < p.ny; y0 += sg)
                                ox.push_back(StepItem{k, x0, y0, std::min(W, p.nx - x0), std::min(sg, p.ny - y0)});
                    }
                }
            });
            size_t nxi = 0, nyi = 0;
            for (int q = 0; q < 16; q++) { nxi += xi[q].size(); nyi += yi[q].size(); }
            L.items.reserve(nxi);
            L.items_y.reserve(nyi);
            for (int q = 0; q < 16; q++) {
                L.items.insert(L.items.end(), xi[q].begin(), xi[q].end());
                L.items_y.insert(L.items_y.end(), yi[q].begin(), yi[q].end());
            }
        }
        // the level-1 retake launch of the FP32 split update: its CTAs exit unless
        // their scenario is retaken, so its x sweep runs the widest CTAs (every
        // launch shape gives the same bits), about 30 times fewer than the default
        L.items_rt.clear();
        if (split && l == 0 && c.cfl_retake) {
            const int Wr = step_strip_width_f32p(kRetakeThreads, 0);
            for (int k = 0; k < n; k++) {
                const PatchDesc &p = L.P[k];
                for (int x0 = 0; x0 < p.nx; x0 += Wr)
                    for (int y0 = -2; y0 < p.ny + 2; y0 += kRetakeRows)
                        L.items_rt.push_back(StepItem{k, x0, y0, std::min(Wr, p.nx - x0), std::min(kRetakeRows, p.ny + 2 - y0)});
            }
        }
        // per scenario spatial indices of this level and the coarser one
        std::vector<std::vector<int>> ids(nscen);
        for (int k = 0; k < n; k++) ids[L.P[k].scen].push_back(k);
        // the coarser level's index was built by its own last finish_level (a
        // coarser table never changes without one, before this level's)
        L.idx.resize(nscen);
        std::vector<BoxIndex> &bis = L.idx;
        std::vector<BoxIndex> &cis = l > 0 ? lv[l - 1].idx : L.idx;
        for (int s = 0; s < nscen; s++) {
            if (ids[s].empty()) continue;
            bis[s].build(L.P, ids[s], L.nxl, L.nyl);
        }
        // patch k's tables in patch order: scenario by scenario, as the ids lists run
        std::vector<int> order;
        order.reserve(n);
        for (int s = 0; s < nscen; s++) order.insert(order.end(), ids[s].begin(), ids[s].end());
        // coarse-map footprints and their offsets first (they depend on the box only)
        size_t cmap_n = 0;
        if (l > 0) {
            const int r = ratio[l - 1];
            size_t tot = 0;
            for (int k : order) {
                PatchDesc &p = L.P[k];
                const int ci0 = floordiv(p.i0 - 2, r) - 1, cj0 = floordiv(p.j0 - 2, r) - 1;
                const int ci1 = floordiv(p.i0 + p.nx + 1, r) + 1, cj1 = floordiv(p.j0 + p.ny + 1, r) + 1;
                p.cmap_i0 = ci0; p.cmap_j0 = cj0; p.cmap_w = ci1 - ci0 + 1; p.cmap_h = cj1 - cj0 + 1;
                p.cmap_off = (int)tot;
                tot += (size_t)p.cmap_w * p.cmap_h;
            }
            cmap_n = tot;
        }
        // neighbour lists and the coarse patches overlapping each coarse-map
        // footprint, patch ranges on host threads; each range's ids go to its
        // own buffers, joined in order afterwards (the device paints the maps)
        std::vector<std::vector<int>> nb(16), cb(16);
        std::array<std::array<int, 2>, 16> rng{};
        parallel_ranges(n, [&](int q, int b, int e) {
            rng[q] = {b, e};
            std::vector<int> tmp;
            std::vector<int> &out = nb[q], &cout_ = cb[q];
            for (int o = b; o < e; o++) {
                const int k = order[o];
                PatchDesc &p = L.P[k];
                bis[p.scen].overlapping(p.i0 - 2, p.j0 - 2, p.i0 + p.nx + 2, p.j0 + p.ny + 2, tmp);
                p.nbr_off = (int)out.size();   // relative to the range's buffer for now
                p.nbr_cnt = 0;
                for (int x : tmp)
                    if (x != k) { out.push_back(x); p.nbr_cnt++; }
                p.ccand_off = (int)cout_.size();
                p.ccand_cnt = 0;
                if (l > 0) {
                    cis[p.scen].overlapping(p.cmap_i0, p.cmap_j0, p.cmap_i0 + p.cmap_w, p.cmap_j0 + p.cmap_h, tmp);
                    for (int x : tmp) { cout_.push_back(x); p.ccand_cnt++; }
                }
            }
        });
        {
            std::vector<int> shift(17, 0), cshift(17, 0);
            for (int q = 0; q < 16; q++) {
                shift[q + 1] = shift[q] + (int)nb[q].size();
                cshift[q + 1] = cshift[q] + (int)cb[q].size();
            }
            L.nbrs.reserve(shift[16]);
            L.ccand.clear();
            L.ccand.reserve(cshift[16]);
            for (int q = 0; q < 16; q++) {
                L.nbrs.insert(L.nbrs.end(), nb[q].begin(), nb[q].end());
                L.ccand.insert(L.ccand.end(), cb[q].begin(), cb[q].end());
            }
            for (int q = 0; q < 16; q++)
                for (int o = rng[q][0]; o < rng[q][1]; o++) {
                    L.P[order[o]].nbr_off += shift[q];
                    L.P[order[o]].ccand_off += cshift[q];
                }
        }
        if (split) L.dScratch.ensure(std::max<size_t>(soff, 64), st);
        L.dP.upload(L.P, st, uring);
        L.dItems.upload(L.items, st, uring);
        L.dItemsY.upload(L.items_y, st, uring);
        if (!L.items_rt.empty()) L.dItemsRt.upload(L.items_rt, st, uring);
        L.dNbrs.upload(L.nbrs, st, uring);
        if (l > 0) {
            // the coarse table's device copy is current: its finish_level ran first
            L.dCmap.ensure(std::max<size_t>(cmap_n, 1), st);
            L.dCcand.upload(L.ccand, st, uring);
            kl(k_fill_cmap(L.dP.p, lv[l - 1].dP.p, L.dCcand.p, n, L.dCmap.p, st), "coarse maps");
        }
        L.dBc.upload(L.bclist, st, uring);
        // ghost-cell sources of the new table: the fills of every step until the
        // next change gather from them
        {
            L.goff.resize(n);
            long long gtot = 0;
            for (int k = 0; k < n; k++) {
                const PatchDesc &p = L.P[k];
                L.goff[k] = gtot;
                gtot += (long long)(p.nx + 4) * (p.ny + 4) - (long long)p.nx * p.ny;
            }
            L.dGoff.upload(L.goff, st, uring);
            L.dGmap.ensure((size_t)std::max<long long>(gtot, 1), st);
            L.dGinterp.ensure((size_t)std::max<long long>(gtot, 1), st);
            L.dGcount.ensure(1, st);
            kl(k_ghost_map(view(l), L.dGmap.p, L.dGinterp.p, L.dGcount.p, n, L.maxring, l > 0 ? ratio[l - 1] : 0, st),
               "ghost map");
        }
        for (int s = 0; s < nscen; s++) cells_h[(size_t)s * kMaxLevels + l] = 0.0;
        for (const auto &p : L.P) cells_h[(size_t)p.scen * kMaxLevels + l] += (double)p.nx * p.ny;
        cells.upload(cells_h, st, uring);
        hier_version++;
    }

    // ------------------------------------------------------------ gauges
    void update_gauges()
    {
        int ng = (int)gxy.size() / 2;
        if (!ng) return;
        std::vector<GaugeLoc> loc((size_t)nscen * ng);
        for (int s = 0; s < nscen; s++)
            for (int g = 0; g < ng; g++) {
                GaugeLoc gl{0, -1};
                for (int l = nlev - 1; l >= 0 && gl.patch < 0; l--) {
                    int I = (int)std::floor((gxy[2 * g] - c.x0) / lv[l].dx);
                    int J = (int)std::floor((gxy[2 * g + 1] - c.y0) / lv[l].dy);
                    if (I < 0 || J < 0 || I >= lv[l].nxl || J >= lv[l].nyl) continue;
                    for (int k = 0; k < (int)lv[l].P.size(); k++) {
                        const PatchDesc &p = lv[l].P[k];
                        if (p.scen == s && I >= p.i0 && I < p.i0 + p.nx && J >= p.j0 && J < p.j0 + p.ny) {
                            gl = GaugeLoc{l, k};
                            break;
                        }
                    }
                }
                loc[(size_t)s * ng + g] = gl;
            }
        dgloc.upload(loc, st, uring);
    }

    void ensure_samples(long long n)
    {
        int ng = (int)gxy.size() / 2;
        if (!ng || n <= samp_cap) return;
        long long nc = std::max(n, samp_cap * 2 + 64);
        double *ne = nullptr, *nt = nullptr;
        CK(cudaMallocAsync((void **)&ne, (size_t)nc * nscen * ng * sizeof(double), st));
        CK(cudaMallocAsync((void **)&nt, (size_t)nc * nscen * sizeof(double), st));
        if (dgeta.p && samp_cap) {
            CK(cudaMemcpyAsync(ne, dgeta.p, (size_t)samp_cap * nscen * ng * sizeof(double), cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(nt, dgt.p, (size_t)samp_cap * nscen * sizeof(double), cudaMemcpyDeviceToDevice, st));
        }
        dgeta.release();
        dgt.release();
        dgeta.p = ne; dgeta.cap = (size_t)nc * nscen * ng; dgeta.st = st;
        dgt.p = nt; dgt.cap = (size_t)nc * nscen; dgt.st = st;
        samp_cap = nc;
        hier_version++;   // the gauge kernel's pointers changed
    }

    void sample_gauges()
    {
        int ng = (int)gxy.size() / 2;
        if (!ng) return;
        // room for this sample (a no-op inside a captured step: tsu_step made
        // room for all of its steps before capturing)
        ensure_samples(nsamp + 1);
        GaugeArgs ga{};
        ga.loc = dgloc.p; ga.xy = dgxy.p; ga.eta = dgeta.p; ga.t = dgt.p; ga.nsamp = dnsamp.p;
        ga.nscen = nscen; ga.ngauges = ng; ga.x0 = c.x0; ga.y0 = c.y0;
        for (int l = 0; l < nlev; l++) {
            ga.levels[l] = view(l);
            ga.curs[l] = lv[l].cur;
            ga.dxl[l] = lv[l].dx;
            ga.dyl[l] = lv[l].dy;
        }
        kl(k_gauges(prec, ga, ctrl(), st), "gauges");
        nsamp++;
    }

    // ------------------------------------------------------------ regrid
    // Predictor logits for the np planes of level l whose raw criterion flags
    // and scenario slots (fslot) are set.
    // Bounding box, on level l, of the cells where the region caps allow level
    // newlev (a superset: a coarse raster marks a cell capped only when one
    // capping region holds its whole footprint).  Returns false when none is.
    bool allowed_box(int l, int newlev, int &i0, int &j0, int &i1, int &j1) const
    {
        const Lvl &C = lv[l];
        const int G = 256, gx = std::min(G, C.nxl), gy = std::min(G, C.nyl);
        i0 = C.nxl; j0 = C.nyl; i1 = -1; j1 = -1;
        for (int b = 0; b < gy; b++)
            for (int a = 0; a < gx; a++) {
                const int ia = (int)((long long)a * C.nxl / gx), ib = (int)((long long)(a + 1) * C.nxl / gx) - 1;
                const int ja = (int)((long long)b * C.nyl / gy), jb = (int)((long long)(b + 1) * C.nyl / gy) - 1;
                const double xa = c.x0 + (ia + 0.5) * C.dx, xb = c.x0 + (ib + 0.5) * C.dx;
                const double ya = c.y0 + (ja + 0.5) * C.dy, yb = c.y0 + (jb + 0.5) * C.dy;
                bool capped = false;
                for (int k = 0; k < c.n_regions && !capped; k++) {
                    const double *R = c.regions[k];
                    capped = xa >= R[0] && xb <= R[2] && ya >= R[1] && yb <= R[3] && (double)newlev > R[5];
                }
                if (capped) continue;
                i0 = std::min(i0, ia); j0 = std::min(j0, ja); i1 = std::max(i1, ib); j1 = std::max(j1, jb);
            }
        return i1 >= 0;
    }

    // Predicted flags of the np planes of level l whose raw criterion flags
    // and scenario slots (fslot) are set, ORed into the raw flags.  The
    // predictor runs on a window only: the criterion flags' bounding box grown
    // by the regrid interval (a wave crosses at most one cell per step, so no
    // flag farther away can appear by the next regrid) and clipped to where the
    // region caps allow the new level, plus the predictor's 3-cell receptive
    // margin.
    void cnn_predict(int l, int np)
    {
        Lvl &C = lv[l];
        const int nx = C.nxl, ny = C.nyl;
        std::vector<int> bb(4 * (size_t)np);
        for (int q = 0; q < np; q++) { bb[4 * q] = nx; bb[4 * q + 1] = ny; bb[4 * q + 2] = -1; bb[4 * q + 3] = -1; }
        fbox.upload(bb, st);
        kl(k_flag_bbox(fraw.p, nx, ny, np, fbox.p, st), "criterion bbox");
        CK(cudaMemcpyAsync(bb.data(), fbox.p, bb.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
        sync();
        int ti0 = nx, tj0 = ny, ti1 = -1, tj1 = -1;
        for (int q = 0; q < np; q++)
            if (bb[4 * q + 2] >= 0) {
                ti0 = std::min(ti0, bb[4 * q]); tj0 = std::min(tj0, bb[4 * q + 1]);
                ti1 = std::max(ti1, bb[4 * q + 2]); tj1 = std::max(tj1, bb[4 * q + 3]);
            }
        if (ti1 < 0) return;
        const int b = c.regrid_interval > 0 ? c.regrid_interval : 0;
        ti0 = std::max(0, ti0 - b); tj0 = std::max(0, tj0 - b);
        ti1 = std::min(nx - 1, ti1 + b); tj1 = std::min(ny - 1, tj1 + b);
        int ai0, aj0, ai1, aj1;
        if (!allowed_box(l, l + 2, ai0, aj0, ai1, aj1)) return;
        ti0 = std::max(ti0, ai0); tj0 = std::max(tj0, aj0); ti1 = std::min(ti1, ai1); tj1 = std::min(tj1, aj1);
        if (ti0 > ti1 || tj0 > tj1) return;
        CnnWindow w;
        w.tx0 = ti0; w.ty0 = tj0; w.tw = ti1 - ti0 + 1; w.th = tj1 - tj0 + 1;
        w.x0 = std::max(0, ti0 - 3); w.y0 = std::max(0, tj0 - 3);
        w.w = std::min(nx - 1, ti1 + 3) - w.x0 + 1; w.h = std::min(ny - 1, tj1 + 3) - w.y0 + 1;
        const size_t wp = (size_t)w.w * w.h;
        cnn_feat.ensure(wp * 5 * np, st);
        cnn_logits.ensure(wp * np, st);
        cnn_half.ensure(cnn_half_workspace_bytes(np, w.h, w.w), st);
        CK(cudaMemsetAsync(cnn_feat.p, 0, wp * 5 * np * sizeof(float), st));
        kl(k_cnn_features(prec, view(l), (int)C.P.size(), C.maxcells, C.cur, fslot.p, fraw.p, cnn_feat.p, c.drytol, w,
                          st), "cnn features");
        kl(cnn_forward(cnn_theta.p, cnn_feat.p, np, w.h, w.w, true, nullptr, cnn_logits.p, cnn_half.p, st),
           "cnn forward");
        kl(k_cnn_union(fraw.p, fcov.p, cnn_logits.p, nx, ny, np, w, st), "cnn union");
    }

    // Build level l+1 of the scenarios in `which` from flags on level l.
    void regrid_one(int l, const std::vector<int> &which)
    {
        // the flags need the queued steps done: that wait is the device's time,
        // not the regrid's (the uploads below would otherwise hide it)
        {
            const auto t_w0 = std::chrono::steady_clock::now();
            sync();
            regrid_wait_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_w0).count();
        }
        const auto t_begin = std::chrono::steady_clock::now();
        const int lf = l + 1, r = ratio[l];
        Lvl &C = lv[l];
        const int nx = C.nxl, ny = C.nyl;
        std::vector<int> slot(nscen, -1);
        int np = 0;
        for (int s : which) slot[s] = np++;
        const size_t plane = (size_t)nx * ny;
        std::vector<std::vector<std::array<int, 4>>> boxes(nscen);
        if (np > 0) {
            fraw.ensure(plane * np, st); fcov.ensure(plane * np, st); ftmp.ensure(plane * np, st);
            fF.ensure(plane * np, st); fN.ensure(plane * np, st);
            fslot.upload(slot, st);
            CK(cudaMemsetAsync(fraw.p, 0, plane * np, st));
            CK(cudaMemsetAsync(fcov.p, 0, plane * np, st));
            FlagArgs fa{};
            fa.raw = fraw.p; fa.cov = fcov.p; fa.scen_slot = fslot.p;
            fa.eta_tol = c.flag_eta_tol; fa.depth_below = c.flag_depth_below; fa.drytol = c.drytol;
            fa.eta_tol_f = float_at_most(c.flag_eta_tol);
            fa.depth_neg_f = float_at_most(-c.flag_depth_below);
            fa.drytol_f = (float)c.drytol;
            fa.x0 = c.x0; fa.y0 = c.y0; fa.dxl = C.dx; fa.dyl = C.dy;
            fa.n_regions = c.n_regions; fa.newlev = l + 2;
            for (int k = 0; k < c.n_regions; k++)
                for (int m = 0; m < 6; m++) fa.regions[6 * k + m] = c.regions[k][m];
            kl(k_flag(prec, view(l), (int)C.P.size(), C.maxcells, C.cur, fa, st), "flag");
            int b = c.regrid_interval > 0 ? c.regrid_interval : 0;
            if (c.use_cnn && cnn_ready) {
                // criterion(now) OR predicted flags, then the narrower buffer
                cnn_predict(l, np);
                b = c.cnn_buffer > 0 ? c.cnn_buffer : 0;
            }
            // Flags and nestable cells can only lie where the level's patches do
            // (the nesting test clears every uncovered cell), so dilation, nesting
            // and the bounding box run over the patches' bounding box W: the y pass
            // reads the x pass's rows within b of W, which reads the fresh raw plane.
            int wi0 = nx, wj0 = ny, wi1 = 0, wj1 = 0;
            for (const auto &p : C.P)
                if (slot[p.scen] >= 0) {
                    wi0 = std::min(wi0, p.i0); wj0 = std::min(wj0, p.j0);
                    wi1 = std::max(wi1, p.i0 + p.nx); wj1 = std::max(wj1, p.j0 + p.ny);
                }
            const Win W{wi0, wj0, std::max(0, wi1 - wi0), std::max(0, wj1 - wj0)};
            const int xj0 = std::max(0, wj0 - b), xj1 = std::min(ny, wj1 + b);
            const Win Wx{wi0, xj0, W.w, std::max(0, xj1 - xj0)};
            kl(k_dilate(fraw.p, ftmp.p, nx, ny, np, b, 0, Wx, st), "dilate x");
            kl(k_dilate(ftmp.p, fF.p, nx, ny, np, b, 1, W, st), "dilate y");
            kl(k_nest(fF.p, fN.p, fcov.p, ftmp.p, nx, ny, np, fa, W, st), "nest");   // ftmp is free again
            launches++;   // k_nest runs two kernels
            // only the flags' bounding box of each plane comes to the host (the
            // clustering starts from that box, so the boxes are the same)
            std::vector<int> bb(4 * (size_t)np);
            for (int q = 0; q < np; q++) { bb[4 * q] = nx; bb[4 * q + 1] = ny; bb[4 * q + 2] = -1; bb[4 * q + 3] = -1; }
            fbox.upload(bb, st);
            kl(k_flag_bbox(fF.p, nx, ny, np, fbox.p, st, &W), "flag bbox");
            CK(cudaMemcpyAsync(bb.data(), fbox.p, bb.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
            sync();
            // each plane's box packed 4 cells per byte on the device, then one copy out
            std::vector<size_t> hoff(np + 1, 0);
            std::vector<int> pstride(np, 0);
            for (int q = 0; q < np; q++) {
                const size_t w = bb[4 * q + 2] >= 0 ? (size_t)(bb[4 * q + 2] - bb[4 * q] + 1) : 0;
                const size_t h = bb[4 * q + 2] >= 0 ? (size_t)(bb[4 * q + 3] - bb[4 * q + 1] + 1) : 0;
                pstride[q] = (int)((w + 3) / 4);
                hoff[q + 1] = hoff[q] + (size_t)pstride[q] * h;
            }
            const size_t nbytes = std::max<size_t>(hoff[np], 1);
            fpack.ensure(nbytes, st);
            hflags.ensure(nbytes);
            uint8_t *hFN = hflags.p;
            for (int q = 0; q < np; q++) {
                if (bb[4 * q + 2] < 0) continue;
                const int w = bb[4 * q + 2] - bb[4 * q] + 1, h = bb[4 * q + 3] - bb[4 * q + 1] + 1;
                kl(k_pack_flags(fN.p + plane * q, nx, bb[4 * q], bb[4 * q + 1], w, h, pstride[q], fpack.p + hoff[q], st),
                   "pack flags");
            }
            CK(cudaMemcpyAsync(hFN, fpack.p, hoff[np], cudaMemcpyDeviceToHost, st));
            sync();
            const auto t_c0 = std::chrono::steady_clock::now();
            auto cluster_one = [&](int s, int threads, std::vector<int32_t> *ws) {
                const int q = slot[s];
                if (bb[4 * q + 2] < 0) return;
                const int w = bb[4 * q + 2] - bb[4 * q] + 1, h = bb[4 * q + 3] - bb[4 * q + 1] + 1;
                cluster_boxes(hFN + hoff[q], w, h, pstride[q], c.cluster_eff, r, c.patch_max, boxes[s], threads, ws);
                for (auto &b : boxes[s]) { b[0] += bb[4 * q]; b[1] += bb[4 * q + 1]; }
            };
            if (which.size() == 1) {
                cluster_one(which[0], 16, &cws[0]);
            } else {
                // independent scenarios: one pool task per group of them (each
                // clusters on its own thread: no nested pool loops)
                const int nt = std::max(1, std::min({16, (int)which.size(), tsu::HostPool::get().size()}));
                tsu::HostPool::get().run(nt, [&](int q) {
                    for (size_t k = q; k < which.size(); k += nt) cluster_one(which[k], 1, &cws[q]);
                });
            }
            cluster_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_c0).count();
        }
        rebuild_level(lf, slot, boxes);
        n_regrids++;
        regrid_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_begin).count();
    }

    void rebuild_level(int lf, const std::vector<int> &slot, std::vector<std::vector<std::array<int, 4>>> &boxes)
    {
        Lvl &L = lv[lf];
        const int r = ratio[lf - 1];
        // the old table stays readable on the device until the initialisation kernels ran
        std::vector<PatchDesc> oldP = L.P;
        std::vector<size_t> oldblk = L.blk, oldbytes = L.blkbytes;
        DevBuf<PatchDesc> oldD = L.dP;
        L.dP.p = nullptr; L.dP.cap = 0;
        std::vector<PatchDesc> P;
        std::vector<size_t> blk, bytes;
        std::vector<int> fresh, renewed;   // patches to initialise; all new patches of regridded scenarios
        {
            size_t nb = oldP.size();
            for (const auto &bx : boxes) nb += bx.size();
            P.reserve(nb); blk.reserve(nb); bytes.reserve(nb); fresh.reserve(nb); renewed.reserve(nb);
        }
        // A new box identical to an old one keeps the old block: a fresh patch
        // would copy its state from that very patch and take the same B (B is a
        // function of the cell on a level), so nothing needs copying.  Its
        // ghost cells are refilled before every step, and its other buffer is
        // written by the level's next step before anything reads it.
        auto key = [](int s, int i0, int j0, int nx, int ny) {
            return ((unsigned long long)(unsigned)s << 60) ^ ((unsigned long long)(unsigned)i0 << 45) ^
                   ((unsigned long long)(unsigned)j0 << 30) ^ ((unsigned long long)(unsigned)nx << 15) ^
                   (unsigned long long)(unsigned)ny;
        };
        // old boxes by key in an open-addressing table (linear probing, the
        // first old patch of a key kept): no allocation per entry
        size_t cap = 16;
        int lg = 4;
        while (cap < 2 * oldP.size()) { cap <<= 1; lg++; }
        same_keys.assign(cap, 0);
        same_ids.assign(cap, -1);
        // Fibonacci hashing: the product's top bits depend on every bit of the key
        auto slot_of = [&](unsigned long long kk) {
            size_t h = (size_t)((kk * 0x9E3779B97F4A7C15ull) >> (64 - lg));
            while (same_ids[h] >= 0 && same_keys[h] != kk) h = (h + 1) & (cap - 1);
            return h;
        };
        for (size_t k = 0; k < oldP.size(); k++)
            if (slot[oldP[k].scen] >= 0) {
                const unsigned long long kk = key(oldP[k].scen, oldP[k].i0, oldP[k].j0, oldP[k].nx, oldP[k].ny);
                const size_t h = slot_of(kk);
                if (same_ids[h] < 0) { same_keys[h] = kk; same_ids[h] = (int)k; }
            }
        std::vector<char> kept(oldP.size(), 0);
        for (int s = 0; s < nscen; s++) {
            if (slot[s] < 0) {
                for (size_t k = 0; k < oldP.size(); k++)
                    if (oldP[k].scen == s) { P.push_back(oldP[k]); blk.push_back(oldblk[k]); bytes.push_back(oldbytes[k]); }
            } else {
                for (const auto &b : boxes[s]) {
                    PatchDesc d = make_desc(lf, s, b[0] * r, b[1] * r, b[2] * r, b[3] * r);
                    renewed.push_back((int)P.size());
                    const int fo = same_ids[slot_of(key(s, d.i0, d.j0, d.nx, d.ny))];
                    if (fo >= 0 && !kept[fo]) {
                        const PatchDesc &o = oldP[fo];
                        if (o.i0 == d.i0 && o.j0 == d.j0 && o.nx == d.nx && o.ny == d.ny && o.scen == s) {
                            kept[fo] = 1;
                            d.off = o.off;
                            P.push_back(d); blk.push_back(oldblk[fo]); bytes.push_back(oldbytes[fo]);
                            continue;
                        }
                    }
                    size_t by = (size_t)d.fs * 7 * esz;
                    size_t off = arena.alloc(by, st);
                    d.off = (long long)(off / esz);
                    fresh.push_back((int)P.size());
                    P.push_back(d); blk.push_back(off); bytes.push_back(by);
                }
            }
        }
        n_patches_reused += (long long)(renewed.size() - fresh.size());
        n_patches_renewed += (long long)renewed.size();
        L.P = P; L.blk = blk; L.blkbytes = bytes;
        // old patches overlapping each new one (indices into the old table)
        L.olds.clear();
        {
            std::vector<std::vector<int>> ids(nscen);
            for (int k = 0; k < (int)oldP.size(); k++) ids[oldP[k].scen].push_back(k);
            // the old table's index, built by the level's last finish_level, now
            // over the copy oldP of that table
            std::vector<BoxIndex> &oi = L.idx;
            oi.resize(nscen);
            for (int s = 0; s < nscen; s++)
                if (slot[s] >= 0 && !ids[s].empty()) oi[s].P = &oldP;
            // fresh patches in contiguous ranges on the host pool, each range's ids
            // joined in patch order afterwards
            std::vector<std::vector<int>> ob(16);
            std::array<std::array<int, 2>, 16> rng{};
            parallel_ranges((int)fresh.size(), [&](int q, int b, int e) {
                rng[q] = {b, e};
                std::vector<int> tmp;
                for (int o = b; o < e; o++) {
                    PatchDesc &p = L.P[fresh[o]];
                    p.old_off = (int)ob[q].size();
                    p.old_cnt = 0;
                    if (ids[p.scen].empty()) continue;
                    oi[p.scen].overlapping(p.i0, p.j0, p.i0 + p.nx, p.j0 + p.ny, tmp);
                    for (int x : tmp) { ob[q].push_back(x); p.old_cnt++; }
                }
            });
            for (int q = 0; q < 16; q++) {
                const int shift = (int)L.olds.size();
                for (int o = rng[q][0]; o < rng[q][1]; o++) L.P[fresh[o]].old_off += shift;
                L.olds.insert(L.olds.end(), ob[q].begin(), ob[q].end());
            }
        }
        for (auto &x : L.idx)   // no index may keep pointing at the old table's copy
            if (x.P == &oldP) { x.P = nullptr; x.nbx = 0; x.nby = 0; }
        L.dOlds.upload(L.olds, st, uring);
        finish_level(lf);
        if (!fresh.empty()) {
            L.dList.upload(fresh, st, uring);
            // B: copied where an old patch of the level held the cell, else sampled
            kl(k_init_patches(prec, view(lf), view(lf, oldD.p), L.dList.p, (int)fresh.size(), L.maxcells, topo(lf), L.cur,
                              0, c.x0, c.y0, L.dx, L.dy, st),
               "init B");
            // B outside the domain for new boundary patches
            std::vector<int> bl;
            for (int k : fresh) if (L.P[k].bcmask) bl.push_back(k);
            if (!bl.empty()) {
                DevBuf<int> dbl;
                dbl.upload(bl, st, uring);
                BcArgs ba{dbl.p, {c.bc[0], c.bc[1], c.bc[2], c.bc[3]}};
                kl(k_bc(prec, view(lf), ba, (int)bl.size(), L.maxring, L.cur, 0, 1, st), "bc B");
                dbl.release();
            }
            kl(k_regrid_init(prec, view(lf), view(lf, oldD.p), view(lf - 1), L.dList.p, (int)fresh.size(), L.maxcells,
                             L.cur, lv[lf - 1].cur, r, c.drytol, derr.p, st), "regrid init");
        }
        if (!renewed.empty()) {
            // wave-speed rate of every new patch (kept blocks included) for the next dt
            L.dList.upload(renewed, st, uring);
            kl(k_cell_speed(prec, view(lf), L.dList.p, (int)renewed.size(), L.maxcells, L.cur, c.g, c.drytol, smax.p, st),
               "cell speed");
            kl(k_post_level(ctrl(), lf, nscen, L.R, pdx(lf), pdy(lf), c.cfl_max, c.cfl_desired, 1, st), "post rate");
        }
        // release the replaced patches of the regridded scenarios
        for (size_t k = 0; k < oldP.size(); k++)
            if (slot[oldP[k].scen] >= 0 && !kept[k]) arena.release(oldblk[k], oldbytes[k]);
        oldD.release();
        // the next finer level's coarse maps point into this table
        if (lf + 1 < nlev && !lv[lf + 1].P.empty()) finish_level(lf + 1);
        update_gauges();
    }

    void regrid_from(int l, const std::vector<int> &which)
    {
        for (int k = l; k + 1 < nlev; k++) regrid_one(k, which);
    }

    // ------------------------------------------------------------ stepping
    // One step of level l alone (Sec. 3.1 step 1): ghost fill (time fraction
    // k / r_{l-1} of the coarser level's step), physical boundaries, the patch
    // update with the CFL check (and, on level 1, the retake), bookkeeping.
    void level_step(int l, int k)
    {
        Lvl &L = lv[l];
        const int n = (int)L.P.size();
        if (n > 0) {
            if (l > 0 || n > 1) {
                double alpha = l > 0 ? (double)k / (double)ratio[l - 1] : 0.0;
                LevelView Cv = l > 0 ? view(l - 1) : view(l);
                kl(k_ghost_fill(prec, view(l), Cv, n, L.maxring, L.cur, l > 0 ? lv[l - 1].cur : 0,
                                l > 0 ? ratio[l - 1] : 0, alpha, c.drytol, derr.p, st), "ghost fill");
                if (l > 0) launches++;   // the interpolated cells' kernel
            }
            if (!L.bclist.empty()) {
                BcArgs ba{L.dBc.p, {c.bc[0], c.bc[1], c.bc[2], c.bc[3]}};
                kl(k_bc(prec, view(l), ba, (int)L.bclist.size(), L.maxring, L.cur, 1, 0, st), "bc");
            }
            StepArgs a{};
            a.descs = L.dP.p; a.items = L.dItems.p; a.arena = arena.base; a.cur = L.cur; a.dt1 = dt1.p;
            a.smax = smax.p; a.R = L.R; a.g = c.g; a.drytol = c.drytol;
            a.dt1f = dt1f.p;
            a.transverse = c.transverse;
            a.manning = (c.manning_n * c.manning_n) * c.g;
            level_args(a, l);
            set_f32_constants(a);
            ProfStep ps{};
            if (prof) {
                ps.level = l;
                ps.e0 = prof_event();
                ps.e1 = prof_event();
                for (int sc = 0; sc < nscen; sc++) ps.cells += cells_h[(size_t)sc * kMaxLevels + l];
                ps.kernels = step_kernels();
                CK(cudaEventRecord(ps.e0, st));
            }
            int e = prec == TSU_F64 ? launch_step_f64(a, (int)L.items.size(), nt(), st)
                                    : launch_step_f32p(a, (int)L.items.size(), nt(), st);
            kl(e, "patch step");
            launches += step_kernels() - 1;
            // Sec. 2.2 CFL condition: a level-1 step with nu > cfl_max is taken
            // again with dt^1 = cfl_desired / rate before any finer level moves.
            // The decision stays on the device: the step's input buffer is
            // untouched, and the retake launch runs only the work items of the
            // scenarios whose post-level kernel set their gate.
            const bool retake = l == 0 && c.cfl_retake;
            // on a one-level grid the last post-level kernel also ends the coarse step
            const bool ends = l == 0 && end_in_post_;
            kl(k_post_level(ctrl(), l, nscen, L.R, pdx(l), pdy(l), c.cfl_max, c.cfl_desired, retake ? 2 : 0, st,
                            ends && !retake ? 1 : 0),
               "post step");
            if (retake) {
                a.gate = retake_gate();
                e = retake_launch(a, L);
                kl(e, "patch step (retake)");
                launches += step_kernels() - 1;
                kl(k_post_level(ctrl(), l, nscen, L.R, pdx(l), pdy(l), c.cfl_max, c.cfl_desired, 3, st, ends ? 1 : 0),
                   "post step (retake)");
                ps.kernels += step_kernels() + 1;
            }
            if (ends) end_done_ = true;
            if (prof) {
                CK(cudaEventRecord(ps.e1, st));
                prof_steps.push_back(ps);
            }
            L.cur ^= 1;
        }
    }

    // What follows the r_l substeps of level l + 1 (or level l's own step when
    // level l + 1 is empty): averaging onto level l, the step count, and a
    // regrid of the finer levels every regrid_interval steps (Sec. 3.1).
    void level_finish(int l)
    {
        Lvl &L = lv[l];
        std::vector<char> stepped(nscen, 0);
        for (const auto &p : L.P) stepped[p.scen] = 1;
        if (l == 0) std::fill(stepped.begin(), stepped.end(), 1);
        if (l + 1 < nlev && !lv[l + 1].P.empty())
            kl(k_average(prec, view(l + 1), view(l), (int)lv[l + 1].P.size(), lv[l + 1].maxcells, lv[l + 1].cur,
                         L.cur, ratio[l], c.drytol, derr.p, st), "average");
        std::vector<int> which;
        for (int s = 0; s < nscen; s++)
            if (stepped[s]) {
                nsteps[s][l]++;
                if (l + 1 < nlev && c.regrid_interval > 0 && nsteps[s][l] % c.regrid_interval == 0) which.push_back(s);
            }
        if (!which.empty()) regrid_from(l, which);
    }

    // The recursion of Sec. 3.1: a step of level l, then r_l steps of level
    // l + 1 (each with its own recursion), then the finish of level l.
    void advance(int l, int k)
    {
        level_step(l, k);
        if (l + 1 < nlev && !lv[l + 1].P.empty())
            for (int kk = 0; kk < ratio[l]; kk++) advance(l + 1, kk);
        level_finish(l);
    }

    // would a regrid fire during the next `n` coarse steps?  (host counters only)
    bool regrid_ahead(int n)
    {
        if (nlev == 1 || c.regrid_interval <= 0) return false;
        // steps of level l per coarse step
        long long per = 1;
        for (int l = 0; l + 1 < nlev; l++) {
            for (int s = 0; s < nscen; s++) {
                bool active = l == 0 || has_patches(s, l);
                if (!active) continue;
                for (long long k = 1; k <= per * n; k++)
                    if ((nsteps[s][l] + k) % c.regrid_interval == 0) return true;
            }
            per *= ratio[l];
        }
        return false;
    }

    // On a one-level grid the level-1 step's post-level kernel also ends the
    // coarse step (t += dt), which saves a launch per step.
    bool end_in_post_ = false, end_done_ = false;
    void coarse_step()
    {
        kl(k_begin_step(ctrl(), nscen, nlev, Rl.p, c.cfl_desired, c.dt_max, st), "begin step");
        end_in_post_ = nlev == 1;
        end_done_ = false;
        advance(0, 0);
        end_in_post_ = false;
        if (!end_done_) kl(k_end_step(ctrl(), nscen, st), "end step");
        sample_gauges();
    }

    void step(int n)
    {
        if (!initialized) throw Err(TSU_ERR_ARG, "tsu_init has not been called");
        if (!synchronised()) throw Err(TSU_ERR_ARG, "tsu_step_level left a coarse step unfinished");
        ensure_samples(nsamp + n + 2);
        int done = 0;
        while (done < n) {
            if (c.use_graphs && !prof && n - done >= 2 && !regrid_ahead(2)) {
                graph_steps(2);
                done += 2;
            } else if (c.use_graphs && !prof && !regrid_ahead(3)) {
                // single steps (a caller reading back every step): captured only
                // when it will be launched again before a regrid
                graph_steps(1);
                done++;
            } else {
                coarse_step();
                done++;
            }
        }
    }

    unsigned parity_key() const
    {
        unsigned k = 0;
        for (int l = 0; l < nlev; l++) k |= (unsigned)(lv[l].cur & 1) << l;
        return k;
    }

    // m (1 or 2) coarse steps as one graph launch.  A coarse step flips the
    // buffer parity of level 1 (and of any level with an odd number of substeps),
    // and a graph replays the buffers it was captured with, so one graph is kept
    // per (m, parity pattern) and reused while the hierarchy is unchanged.
    void graph_steps(int m)
    {
        if (graphs_version != hier_version) {
            for (auto &g : graphs) cudaGraphExecDestroy(g.ex);
            graphs.clear();
            graphs_version = hier_version;
        }
        const unsigned key = parity_key();
        int gi = -1;
        for (size_t k = 0; k < graphs.size(); k++)
            if (graphs[k].m == m && graphs[k].key == key) gi = (int)k;
        if (gi < 0) {
            const long long l0 = launches, ns0 = nsamp;
            const std::vector<std::array<long long, kMaxLevels>> ns = nsteps;
            std::array<int, kMaxLevels> pre{};
            for (int l = 0; l < nlev; l++) pre[l] = lv[l].cur;
            cudaGraph_t g = nullptr;
            CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            try {
                for (int k = 0; k < m; k++) coarse_step();
            } catch (...) {
                cudaStreamEndCapture(st, &g);
                if (g) cudaGraphDestroy(g);
                for (int l = 0; l < nlev; l++) lv[l].cur = pre[l];
                throw;
            }
            CK(cudaStreamEndCapture(st, &g));
            StepGraph sg{};
            sg.m = m;
            sg.key = key;
            const cudaError_t e = cudaGraphInstantiate(&sg.ex, g, 0);
            cudaGraphDestroy(g);
            // the capture only recorded the steps: put the host state back
            for (int l = 0; l < nlev; l++) sg.post[l] = lv[l].cur;
            sg.kernels = launches - l0;
            launches = l0;
            nsteps = ns;
            nsamp = ns0;
            for (int l = 0; l < nlev; l++) lv[l].cur = pre[l];
            CK(e);
            graphs.push_back(sg);
            gi = (int)graphs.size() - 1;
        }
        CK(cudaGraphLaunch(graphs[gi].ex, st));
        launches += graphs[gi].kernels;
        for (int l = 0; l < nlev; l++) lv[l].cur = graphs[gi].post[l];
        long long per = 1;
        for (int l = 0; l < nlev; l++) {
            for (int s = 0; s < nscen; s++)
                if (l == 0 || has_patches(s, l)) nsteps[s][l] += per * m;
            if (l + 1 < nlev) per *= ratio[l];
        }
        nsamp += gxy.empty() ? 0 : m;
    }

    // One step of level l (0-based) in the order of the recursion of Sec. 3.1:
    // level 1 starts a coarse step; level l + 1 takes the next of the r_l
    // substeps within the current step of level l.  A step whose level has a
    // non-empty finer level leaves that level's substeps pending; the last
    // substep of a level finishes its parent's step (averaging, regrids), and
    // finishing level 1 ends the coarse step (time, gauges).
    void step_level(int l)
    {
        if (!initialized) throw Err(TSU_ERR_ARG, "tsu_init has not been called");
        if (l < 0 || l >= nlev) throw Err(TSU_ERR_ARG, "level out of range");
        if (l == 0) {
            if (!synchronised()) throw Err(TSU_ERR_ARG, "level 1 steps only between coarse steps");
            ensure_samples(nsamp + 2);
            kl(k_begin_step(ctrl(), nscen, nlev, Rl.p, c.cfl_desired, c.dt_max, st), "begin step");
        } else {
            if (pend[l - 1] == 0) throw Err(TSU_ERR_ARG, "the coarser level has no substep of this level pending");
            if (pend[l] != 0) throw Err(TSU_ERR_ARG, "the finer level's substeps are still pending");
            if (lv[l].P.empty()) throw Err(TSU_ERR_ARG, "the level has no patches");
        }
        level_step(l, l == 0 ? 0 : ratio[l - 1] - pend[l - 1]);
        if (l + 1 < nlev && !lv[l + 1].P.empty()) {
            pend[l] = ratio[l];
            return;
        }
        for (;;) {   // finish this level, and every coarser one whose last substep this was
            level_finish(l);
            if (l == 0) {
                kl(k_end_step(ctrl(), nscen, st), "end step");
                sample_gauges();
                return;
            }
            if (--pend[l - 1] > 0) return;
            l--;
        }
    }

    // Error flag and CFL-violation counts (and, with t_out, every scenario's
    // time) in one synchronisation, through page-locked memory.
    // Before the first step after the caller could have written the state
    // (tsu_level1_buffers, tsu_checkpoint_restore): no interior cell of any
    // level may have a negative depth, which the library never stores.
    void check_external_state()
    {
        if (!ext_state) return;
        dneg.ensure(1, st);
        CK(cudaMemsetAsync(dneg.p, 0, sizeof(int), st));
        for (int l = 0; l < nlev; l++)
            if (!lv[l].P.empty())
                kl(k_depth_check(prec, view(l), (int)lv[l].P.size(), lv[l].maxcells, lv[l].cur, dneg.p, st), "depth check");
        int n = 0;
        CK(cudaMemcpyAsync(&n, dneg.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        sync();
        if (n > 0)
            throw Err(TSU_ERR_NEGDEPTH, std::to_string(n) + " interior cells of the supplied state have a negative depth");
        ext_state = false;
    }

    void check_device_errors(bool &cfl, double *t_out = nullptr)
    {
        const size_t ns = (size_t)nscen;
        hsmall.ensure(64 + ns * (sizeof(long long) + sizeof(double)));
        int *e = reinterpret_cast<int *>(hsmall.p);
        long long *v = reinterpret_cast<long long *>(hsmall.p + 64);
        double *tt = reinterpret_cast<double *>(hsmall.p + 64 + ns * sizeof(long long));
        CK(cudaMemcpyAsync(e, derr.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(v, viol.p, ns * sizeof(long long), cudaMemcpyDeviceToHost, st));
        if (t_out) CK(cudaMemcpyAsync(tt, t.p, ns * sizeof(double), cudaMemcpyDeviceToHost, st));
        sync();
        if (*e & TSU_DEV_ERR_TIMEOUT)
            throw Err(TSU_ERR_TIMEOUT, "a patch update gave up waiting for a bulk copy (tsu_set_bulk_copies)");
        if (*e & TSU_DEV_ERR_LAYOUT) throw Err(TSU_ERR_CUDA, "patch storage not aligned for bulk copies");
        if (*e & TSU_DEV_ERR_NAN) throw Err(TSU_ERR_NAN, "a wave speed or depth is not a finite number");
        if (*e) throw Err(TSU_ERR_NESTING, "a ghost cell or coarse cell had no covering patch (nesting)");
        if (t_out) std::memcpy(t_out, tt, ns * sizeof(double));
        long long tot = 0;
        for (size_t s = 0; s < ns; s++) tot += v[s];
        cfl = tot > viol_seen;
        viol_seen = tot;
    }

    // Device-to-host copy of n doubles through page-locked staging.  Chunks go
    // round-robin to up to kWorkers host threads, each with its own staging
    // slot and event: the link copies one chunk while the other threads move
    // theirs into dst (and take dst's first-touch page faults) in parallel.
    // 1 when the device reaches pageable host memory through the host's page
    // tables (coherent platforms): a copy into resident pageable pages then runs
    // at the pinned rate without a staging buffer
    int pageable_ = -1;
    bool pageable_access()
    {
        if (pageable_ < 0) {
            int a = 0, b = 0;
            if (cudaDeviceGetAttribute(&a, cudaDevAttrPageableMemoryAccess, device) != cudaSuccess) a = 0;
            if (cudaDeviceGetAttribute(&b, cudaDevAttrPageableMemoryAccessUsesHostPageTables, device) != cudaSuccess) b = 0;
            pageable_ = (a && b) ? 1 : 0;
        }
        return pageable_ == 1;
    }

    void d2h_staged(double *dst, const double *src, size_t n)
    {
        constexpr size_t kChunk = (size_t)1 << 19;   // doubles per chunk (4 MiB)
        constexpr int kWorkers = 8;
        if (n <= 4096) {
            hsmall.ensure(4096 * sizeof(double));
            CK(cudaMemcpyAsync(hsmall.p, src, n * sizeof(double), cudaMemcpyDeviceToHost, st));
            sync();
            std::memcpy(dst, hsmall.p, n * sizeof(double));
            return;
        }
        const size_t nch = (n + kChunk - 1) / kChunk;
        const int T = (int)std::min<size_t>(kWorkers, nch);
        // one page-locked staging buffer for the process, kept between contexts
        // (allocating it costs milliseconds); contexts on other threads take turns
        static std::mutex stage_mu;
        static PinnedHost *stage = new PinnedHost();   // never freed: outlives every context
        std::lock_guard<std::mutex> lk(stage_mu);
        PinnedHost &hstage = *stage;
        hstage.ensure((size_t)T * kChunk * sizeof(double));
        for (int w = 0; w < T; w++)
            if (!stage_ev[w]) CK(cudaEventCreateWithFlags(&stage_ev[w], cudaEventDisableTiming));
        double *buf = reinterpret_cast<double *>(hstage.p);
        std::vector<int> err(T, 0);
        auto work = [&](int w) {
            if (w > 0 && cudaSetDevice(device) != cudaSuccess) {
                err[w] = (int)cudaErrorInvalidDevice;
                return;
            }
            double *slot = buf + (size_t)w * kChunk;
            for (size_t k = (size_t)w; k < nch && !err[w]; k += (size_t)T) {
                const size_t off = k * kChunk, m = std::min(kChunk, n - off);
                cudaError_t e = cudaMemcpyAsync(slot, src + off, m * sizeof(double), cudaMemcpyDeviceToHost, st);
                if (e == cudaSuccess) e = cudaEventRecord(stage_ev[w], st);
                if (e == cudaSuccess) e = cudaEventSynchronize(stage_ev[w]);
                if (e != cudaSuccess) {
                    err[w] = (int)e;
                    break;
                }
                std::memcpy(dst + off, slot, m * sizeof(double));
            }
        };
        std::vector<std::thread> th;
        for (int w = 1; w < T; w++) th.emplace_back(work, w);
        work(0);
        for (auto &x : th) x.join();
        for (int w = 0; w < T; w++)
            if (err[w]) CK((cudaError_t)err[w]);
        sync();
    }

    // ------------------------------------------------------------ init
    void init()
    {
        if (initialized) throw Err(TSU_ERR_ARG, "tsu_init called twice");
        if (nbase == 0) throw Err(TSU_ERR_ARG, "no topography: call tsu_add_topo first");
        upload_topo();
        Lvl &L = lv[0];
        int T = c.level1_tile > 0 ? c.level1_tile : std::max(c.nx, c.ny);
        size_t need = 0;
        for (int s = 0; s < nscen; s++)
            for (int j0 = 0; j0 < c.ny; j0 += T)
                for (int i0 = 0; i0 < c.nx; i0 += T) {
                    PatchDesc d = make_desc(0, s, i0, j0, std::min(T, c.nx - i0), std::min(T, c.ny - j0));
                    need += Arena::rnd((size_t)d.fs * 7 * esz);
                }
        arena.reserve(need + need / 2 + (64u << 20), st);
        std::vector<int> all;
        for (int s = 0; s < nscen; s++)
            for (int j0 = 0; j0 < c.ny; j0 += T)
                for (int i0 = 0; i0 < c.nx; i0 += T) {
                    PatchDesc d = make_desc(0, s, i0, j0, std::min(T, c.nx - i0), std::min(T, c.ny - j0));
                    size_t by = (size_t)d.fs * 7 * esz;
                    size_t off = arena.alloc(by, st);
                    d.off = (long long)(off / esz);
                    all.push_back((int)L.P.size());
                    L.P.push_back(d); L.blk.push_back(off); L.blkbytes.push_back(by);
                }
        finish_level(0);
        L.dList.upload(all, st);
        LevelView none{};
        kl(k_init_patches(prec, view(0), none, L.dList.p, (int)all.size(), L.maxcells, topo(0), L.cur, 1, c.x0, c.y0,
                          L.dx, L.dy, st),
           "init level 1");
        if (!L.bclist.empty()) {
            BcArgs ba{L.dBc.p, {c.bc[0], c.bc[1], c.bc[2], c.bc[3]}};
            kl(k_bc(prec, view(0), ba, (int)L.bclist.size(), L.maxring, L.cur, 0, 1, st), "bc B");
        }
        kl(k_cell_speed(prec, view(0), L.dList.p, (int)all.size(), L.maxcells, L.cur, c.g, c.drytol, smax.p, st),
           "cell speed");
        kl(k_post_level(ctrl(), 0, nscen, L.R, pdx(0), pdy(0), c.cfl_max, c.cfl_desired, 1, st), "post rate");
        initialized = true;
        std::vector<int> everyone(nscen);
        for (int s = 0; s < nscen; s++) everyone[s] = s;
        if (nlev > 1) regrid_from(0, everyone);
        update_gauges();
        bool cfl;
        check_device_errors(cfl);
    }

    // ------------------------------------------------------------ checkpoints
    // Layout (host byte order): header, config, control block, per level the
    // patch boxes with their current state (q0, q1, q2) and B including ghost
    // cells, then the gauge records.  Taken between coarse steps, where the
    // next step's old state is the saved one, so one time level suffices.
    static constexpr uint64_t kCkptMagic = 0x3154504b43555354ull;   // "TSUCKPT1"
    struct Writer {
        std::vector<uint8_t> *out;
        template <typename T> void put(const T *p, size_t n)
        {
            const uint8_t *b = reinterpret_cast<const uint8_t *>(p);
            out->insert(out->end(), b, b + n * sizeof(T));
        }
        template <typename T> void one(T v) { put(&v, 1); }
    };
    struct Reader {
        const uint8_t *p, *end;
        template <typename T> void get(T *dst, size_t n)
        {
            size_t by = n * sizeof(T);
            if ((size_t)(end - p) < by) throw Err(TSU_ERR_ARG, "checkpoint is truncated");
            std::memcpy(dst, p, by);
            p += by;
        }
        template <typename T> T one()
        {
            T v;
            get(&v, 1);
            return v;
        }
    };
    template <typename T> std::vector<T> d2h(const T *d, size_t n)
    {
        std::vector<T> v(n);
        if (n) CK(cudaMemcpyAsync(v.data(), d, n * sizeof(T), cudaMemcpyDeviceToHost, st));
        return v;
    }
    std::vector<uint8_t> checkpoint()
    {
        if (!initialized) throw Err(TSU_ERR_ARG, "tsu_init has not been called");
        sync();
        std::vector<uint8_t> out;
        Writer w{&out};
        w.one(kCkptMagic);
        w.one<int32_t>(prec); w.one<int32_t>(nscen); w.one<int32_t>(nlev); w.one<int32_t>((int32_t)sizeof(tsu_config));
        w.put(&c, 1);
        auto dt = d2h(dt1.p, nscen); auto dtf = d2h(dt1f.p, nscen); auto tt = d2h(t.p, nscen);
        auto rt = d2h(rate.p, (size_t)nscen * kMaxLevels); auto cu = d2h(cellupd.p, nscen);
        auto vi = d2h(viol.p, nscen); auto sm = d2h(smax.p, 2 * (size_t)nscen);
        const int ng = (int)gxy.size() / 2;
        auto gt = d2h(dgt.p, (size_t)(ng ? nsamp : 0) * nscen);
        auto ge = d2h(dgeta.p, (size_t)(ng ? nsamp : 0) * nscen * ng);
        std::vector<std::vector<uint8_t>> data(nlev);
        for (int l = 0; l < nlev; l++) {
            const Lvl &L = lv[l];
            size_t tot = 0;
            for (const auto &p : L.P) tot += (size_t)p.fs * 4 * esz;
            data[l].resize(tot);
            size_t o = 0;
            for (const auto &p : L.P) {
                const uint8_t *blk = reinterpret_cast<const uint8_t *>(arena.base) + (size_t)p.off * esz;
                const size_t fb = (size_t)p.fs * esz;
                const int fld[4] = {L.cur * 3 + 0, L.cur * 3 + 1, L.cur * 3 + 2, 6};
                for (int f = 0; f < 4; f++) {
                    CK(cudaMemcpyAsync(data[l].data() + o, blk + fld[f] * fb, fb, cudaMemcpyDeviceToHost, st));
                    o += fb;
                }
            }
        }
        sync();
        w.put(dt.data(), dt.size()); w.put(dtf.data(), dtf.size()); w.put(tt.data(), tt.size());
        w.put(rt.data(), rt.size()); w.put(cu.data(), cu.size()); w.put(vi.data(), vi.size());
        w.put(sm.data(), sm.size());
        for (int s = 0; s < nscen; s++) w.put(nsteps[s].data(), kMaxLevels);
        w.one<int64_t>(viol_seen);
        for (int l = 0; l < nlev; l++) {
            const Lvl &L = lv[l];
            w.one<int64_t>((int64_t)L.P.size());
            for (const auto &p : L.P) {
                const int32_t box[5] = {p.scen, p.i0, p.j0, p.nx, p.ny};
                w.put(box, 5);
            }
            w.put(data[l].data(), data[l].size());
        }
        w.one<int32_t>(ng);
        w.one<int64_t>(ng ? nsamp : 0);
        w.put(gt.data(), gt.size());
        w.put(ge.data(), ge.size());
        return out;
    }
    void restore(const uint8_t *buf, size_t n)
    {
        if (!initialized) throw Err(TSU_ERR_ARG, "restore needs an initialised context (tsu_init)");
        Reader r{buf, buf + n};
        if (r.one<uint64_t>() != kCkptMagic) throw Err(TSU_ERR_ARG, "not a checkpoint");
        const int p_ = r.one<int32_t>(), ns = r.one<int32_t>(), nl = r.one<int32_t>(), cs = r.one<int32_t>();
        if (p_ != prec || ns != nscen || nl != nlev || cs != (int32_t)sizeof(tsu_config))
            throw Err(TSU_ERR_ARG, "checkpoint of another precision, scenario count or level count");
        tsu_config cc;
        r.get(&cc, 1);
        if (std::memcmp(&cc, &c, sizeof c) != 0) throw Err(TSU_ERR_ARG, "checkpoint of another configuration");
        std::vector<double> dt(nscen), tt(nscen), rt((size_t)nscen * kMaxLevels), cu(nscen);
        std::vector<float> dtf(nscen);
        std::vector<long long> vi(nscen);
        std::vector<unsigned long long> sm(2 * (size_t)nscen);
        r.get(dt.data(), dt.size()); r.get(dtf.data(), dtf.size()); r.get(tt.data(), tt.size());
        r.get(rt.data(), rt.size()); r.get(cu.data(), cu.size()); r.get(vi.data(), vi.size());
        r.get(sm.data(), sm.size());
        std::vector<std::array<long long, kMaxLevels>> nst(nscen);
        for (int s = 0; s < nscen; s++) r.get(nst[s].data(), kMaxLevels);
        const long long vseen = r.one<int64_t>();
        // replace the hierarchy level by level (coarse maps point into the coarser table)
        sync();
        for (int l = 0; l < nlev; l++) {
            Lvl &L = lv[l];
            for (size_t k = 0; k < L.P.size(); k++) arena.release(L.blk[k], L.blkbytes[k]);
            L.P.clear(); L.blk.clear(); L.blkbytes.clear();
        }
        for (int l = 0; l < nlev; l++) {
            Lvl &L = lv[l];
            const long long np = r.one<int64_t>();
            if (np < 0 || np > (1ll << 26)) throw Err(TSU_ERR_ARG, "checkpoint is corrupt");
            std::vector<int32_t> boxes((size_t)np * 5);
            r.get(boxes.data(), boxes.size());
            for (long long k = 0; k < np; k++) {
                const int32_t *b = &boxes[(size_t)k * 5];
                if (b[0] < 0 || b[0] >= nscen || b[3] < 1 || b[4] < 1 || b[1] < 0 || b[2] < 0 || b[1] + b[3] > L.nxl ||
                    b[2] + b[4] > L.nyl)
                    throw Err(TSU_ERR_ARG, "checkpoint is corrupt");
                PatchDesc d = make_desc(l, b[0], b[1], b[2], b[3], b[4]);
                size_t by = (size_t)d.fs * 7 * esz;
                size_t off = arena.alloc(by, st);
                d.off = (long long)(off / esz);
                L.P.push_back(d); L.blk.push_back(off); L.blkbytes.push_back(by);
            }
            L.cur = 0;
            L.olds.clear();
            L.dOlds.upload(L.olds, st);
            finish_level(l);
            for (const auto &p : L.P) {
                uint8_t *blk = reinterpret_cast<uint8_t *>(arena.base) + (size_t)p.off * esz;
                const size_t fb = (size_t)p.fs * esz;
                const int fld[4] = {0, 1, 2, 6};
                for (int f = 0; f < 4; f++) {
                    std::vector<uint8_t> tmp(fb);
                    r.get(tmp.data(), fb);
                    CK(cudaMemcpyAsync(blk + fld[f] * fb, tmp.data(), fb, cudaMemcpyHostToDevice, st));
                    sync();
                }
            }
        }
        const int ng = r.one<int32_t>();
        const long long ns_ = r.one<int64_t>();
        if (ng != (int)gxy.size() / 2 || ns_ < 0) throw Err(TSU_ERR_ARG, "checkpoint has other gauges");
        std::vector<double> gt((size_t)ns_ * nscen), ge((size_t)ns_ * nscen * ng);
        r.get(gt.data(), gt.size());
        r.get(ge.data(), ge.size());
        if (ng) {
            ensure_samples(ns_);
            if (ns_) {
                CK(cudaMemcpyAsync(dgt.p, gt.data(), gt.size() * sizeof(double), cudaMemcpyHostToDevice, st));
                CK(cudaMemcpyAsync(dgeta.p, ge.data(), ge.size() * sizeof(double), cudaMemcpyHostToDevice, st));
            }
            nsamp = ns_;
            CK(cudaMemcpyAsync(dnsamp.p, &nsamp, sizeof(long long), cudaMemcpyHostToDevice, st));
        }
        CK(cudaMemcpyAsync(dt1.p, dt.data(), nscen * sizeof(double), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(dt1f.p, dtf.data(), nscen * sizeof(float), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(t.p, tt.data(), nscen * sizeof(double), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(rate.p, rt.data(), rt.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(cellupd.p, cu.data(), nscen * sizeof(double), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(viol.p, vi.data(), nscen * sizeof(long long), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(smax.p, sm.data(), sm.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice, st));
        nsteps = nst;
        viol_seen = vseen;
        update_gauges();
        hier_version++;
        sync();
    }

    void add_uplift_now(int s, const Grid &g)
    {
        TopoDev U{g.nx, g.ny, g.x0, g.y0, g.dx, g.dy, g.dev};
        for (int l = 0; l < nlev; l++) {
            Lvl &L = lv[l];
            if (L.P.empty()) continue;
            kl(k_uplift(prec, view(l), (int)L.P.size(), L.maxcells, U, s, L.cur, c.x0, c.y0, L.dx, L.dy, st), "uplift");
            if (!L.bclist.empty()) {
                BcArgs ba{L.dBc.p, {c.bc[0], c.bc[1], c.bc[2], c.bc[3]}};
                kl(k_bc(prec, view(l), ba, (int)L.bclist.size(), L.maxring, L.cur, 0, 1, st), "bc B");
            }
        }
    }

    ~tsu_ctx()
    {
        if (st) cudaStreamSynchronize(st);
        for (auto &g : graphs) cudaGraphExecDestroy(g.ex);
        for (auto &p : prof_steps) { cudaEventDestroy(p.e0); cudaEventDestroy(p.e1); }
        for (auto &e : prof_pool) cudaEventDestroy(e);
        for (auto &e : stage_ev)
            if (e) cudaEventDestroy(e);
        for (auto &L : lv) {
            L.dP.release(); L.dItems.release(); L.dNbrs.release(); L.dCmap.release(); L.dCcand.release(); L.dBc.release();
            L.dOlds.release(); L.dList.release();
            L.dKap.release(); L.dCed.release(); L.dKapF.release(); L.dCedF.release();
            L.dItemsY.release(); L.dScratch.release();
            L.dGmap.release(); L.dGoff.release(); L.dGinterp.release(); L.dGcount.release(); L.dItemsRt.release();
        }
        for (auto &g : grids) if (g.dev) cudaFreeAsync(g.dev, st);
        dGrids.release(); dGridScen.release(); dEtaIdx.release();
        dt1.release(); dt1f.release(); t.release(); rate.release(); cellupd.release(); cells.release(); Rl.release(); mass.release();
        viol.release(); smax.release(); derr.release(); retake.release(); retakes.release(); dneg.release();
        tabI.release(); tabT.release(); tabIn.release();
        dgxy.release(); dgeta.release(); dgt.release(); dnsamp.release(); dgloc.release();
        fraw.release(); fcov.release(); ftmp.release(); fF.release(); fN.release(); fpack.release(); fslot.release(); fbox.release();
        dstage.release(); zero_dt.release(); zero_dtf.release(); massParts.release();
        cnn_theta.release(); cnn_feat.release(); cnn_logits.release(); cnn_half.release();
        if (arena.base) cudaFreeAsync(arena.base, st);
        if (st) cudaStreamSynchronize(st);
        if (own_stream && st) cudaStreamDestroy(st);
    }
};

// ------------------------------------------------------------------ C ABI

namespace {

template <typename F> int guard(tsu_ctx *ctx, F &&f)
{
    if (!ctx) return TSU_ERR_ARG;
    try {
        f();
        return TSU_OK;
    } catch (const Err &e) {
        ctx->err = e.what();
        return e.code;
    } catch (const std::exception &e) {
        ctx->err = e.what();
        return TSU_ERR_ARG;
    } catch (...) {
        ctx->err = "unknown error";
        return TSU_ERR_ARG;
    }
}

void check_grid(const double *v, int nx, int ny, double dx, double dy)
{
    if (!v || nx < 2 || ny < 2 || !(dx > 0) || !(dy > 0)) throw Err(TSU_ERR_ARG, "grid needs nx, ny >= 2 and dx, dy > 0");
}

}  // namespace

extern "C" {

int tsu_create(const tsu_config *cfg, void *cuda_stream, tsu_ctx **out)
{
    if (!cfg || !out) return TSU_ERR_ARG;
    *out = nullptr;
    const tsu_config &c = *cfg;
    if (c.precision != TSU_F64 && c.precision != TSU_F32P) return TSU_ERR_ARG;
    if (c.nx < 2 || c.ny < 2 || !(c.dx > 0) || !(c.dy > 0)) return TSU_ERR_ARG;
    if (c.num_levels < 1 || c.num_levels > TSU_MAX_LEVELS || c.n_scenarios < 1 || (c.transverse != 0 && c.transverse != 1) ||
        !(c.manning_n >= 0.0)) return TSU_ERR_ARG;
    if (c.spherical != 0 && (c.spherical != 1 || c.transverse || !(c.y0 > -90.0) || !(c.y0 + c.ny * c.dy < 90.0)))
        return TSU_ERR_ARG;
    for (int l = 0; l + 1 < c.num_levels; l++)
        if (c.ratios[l] < 2) return TSU_ERR_ARG;
    if (c.n_regions < 0 || c.n_regions > TSU_MAX_REGIONS || c.patch_max < 1) return TSU_ERR_ARG;
    if (!(c.cfl_desired > 0) || !(c.cfl_max > 0) || !(c.dt_max > 0) || !(c.g > 0) || !(c.drytol > 0)) return TSU_ERR_ARG;
    for (int k = 0; k < 4; k++)
        if (c.bc[k] != TSU_BC_WALL && c.bc[k] != TSU_BC_EXTRAP) return TSU_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return TSU_ERR_NOT_BUILT;
    tsu_ctx *x = new tsu_ctx();
    int rc = guard(x, [&] {
        x->c = c;
        if (x->c.cluster_eff <= 0) x->c.cluster_eff = 0.7;
        x->prec = c.precision;
        x->esz = c.precision == TSU_F64 ? 8 : 4;
        x->nlev = c.num_levels;
        x->nscen = c.n_scenarios;
        for (int l = 0; l + 1 < x->nlev; l++) x->ratio[l] = c.ratios[l];
        CK(cudaGetDevice(&x->device));
        if (cuda_stream) x->st = (cudaStream_t)cuda_stream;
        else {
            CK(cudaStreamCreateWithFlags(&x->st, cudaStreamNonBlocking));
            x->own_stream = true;
        }
        int R = 1;
        std::vector<double> rl(kMaxLevels, 1.0);
        for (int l = 0; l < x->nlev; l++) {
            if (l > 0) R *= x->ratio[l - 1];
            x->lv[l].R = (double)R;
            x->lv[l].nxl = c.nx * R;
            x->lv[l].nyl = c.ny * R;
            x->lv[l].dx = c.dx / (double)R;
            x->lv[l].dy = c.dy / (double)R;
            rl[l] = (double)R;
        }
        if (c.spherical) {
            // latitude-longitude geometry: rows J of level l span y0 + J dy .. y0 + (J + 1) dy degrees;
            // capacity (sin top - sin bottom) / dphi, latitude edge below row J weighted by its cos
            const double d2r = 3.14159265358979323846 / 180.0;
            const double Re = c.earth_radius > 0.0 ? c.earth_radius : 6371.0e3;
            for (int l = 0; l < x->nlev; l++) {
                Lvl &L = x->lv[l];
                L.dxp = Re * (L.dx * d2r);
                L.dyp = Re * (L.dy * d2r);
                std::vector<double> kap(L.nyl + 4), ced(L.nyl + 5);
                std::vector<float> kapf(L.nyl + 4), cedf(L.nyl + 5);
                for (int J = -2; J < L.nyl + 2; J++) {
                    const double a = (c.y0 + (double)J * L.dy) * d2r, b = (c.y0 + (double)(J + 1) * L.dy) * d2r;
                    kap[J + 2] = (std::sin(b) - std::sin(a)) / (L.dy * d2r);
                    kapf[J + 2] = (float)kap[J + 2];
                }
                for (int J = -2; J <= L.nyl + 2; J++) {
                    ced[J + 2] = std::cos((c.y0 + (double)J * L.dy) * d2r);
                    cedf[J + 2] = (float)ced[J + 2];
                }
                L.dKap.upload(kap, x->st); L.dCed.upload(ced, x->st); L.dKapF.upload(kapf, x->st); L.dCedF.upload(cedf, x->st);
            }
        }
        const int S = x->nscen;
        cudaStream_t st = x->st;
        x->dt1.ensure(S, st); x->dt1f.ensure(S, st); x->t.ensure(S, st); x->rate.ensure((size_t)S * kMaxLevels, st);
        x->cellupd.ensure(S, st); x->viol.ensure(S, st); x->smax.ensure(2 * (size_t)S, st);
        x->derr.ensure(1, st); x->mass.ensure(S, st); x->dnsamp.ensure(1, st);
        x->retake.ensure(S, st); x->retakes.ensure(S, st);
        CK(cudaMemsetAsync(x->retake.p, 0, S * sizeof(int), st));
        CK(cudaMemsetAsync(x->retakes.p, 0, S * sizeof(long long), st));
        CK(cudaMemsetAsync(x->dt1.p, 0, S * sizeof(double), st));
        CK(cudaMemsetAsync(x->dt1f.p, 0, S * sizeof(float), st));
        CK(cudaMemsetAsync(x->t.p, 0, S * sizeof(double), st));
        CK(cudaMemsetAsync(x->rate.p, 0, (size_t)S * kMaxLevels * sizeof(double), st));
        CK(cudaMemsetAsync(x->cellupd.p, 0, S * sizeof(double), st));
        CK(cudaMemsetAsync(x->viol.p, 0, S * sizeof(long long), st));
        CK(cudaMemsetAsync(x->smax.p, 0, 2 * S * sizeof(unsigned long long), st));
        CK(cudaMemsetAsync(x->derr.p, 0, sizeof(int), st));
        CK(cudaMemsetAsync(x->dnsamp.p, 0, sizeof(long long), st));
        x->Rl.upload(rl, st);
        x->cells_h.assign((size_t)S * kMaxLevels, 0.0);
        x->cells.upload(x->cells_h, st);
        x->nsteps.assign(S, {});
        x->eta_index.assign(3 * S, -1);
        x->sync();
    });
    if (rc != TSU_OK) {
        delete x;
        return rc;
    }
    *out = x;
    return TSU_OK;
}

int tsu_destroy(tsu_ctx *ctx)
{
    delete ctx;
    return TSU_OK;
}

const char *tsu_last_error(tsu_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int tsu_add_topo(tsu_ctx *ctx, const double *B, int nx, int ny, double x0, double y0, double dx, double dy)
{
    return guard(ctx, [&] {
        if (ctx->initialized) throw Err(TSU_ERR_ARG, "topography must be added before tsu_init");
        check_grid(B, nx, ny, dx, dy);
        Grid g{nx, ny, x0, y0, dx, dy, std::vector<double>(B, B + (size_t)nx * ny), -1, nullptr};
        // base grids first: insert after the existing base grids and shift layer indices
        ctx->grids.insert(ctx->grids.begin() + ctx->nbase, g);
        ctx->nbase++;
        for (auto &e : ctx->eta_index) if (e >= 0) e++;
    });
}

int tsu_set_eta(tsu_ctx *ctx, int scen, const double *eta, int nx, int ny, double x0, double y0, double dx, double dy)
{
    return guard(ctx, [&] {
        if (ctx->initialized) throw Err(TSU_ERR_ARG, "the initial surface must be set before tsu_init");
        if (scen < 0 || scen >= ctx->nscen) throw Err(TSU_ERR_ARG, "bad scenario");
        check_grid(eta, nx, ny, dx, dy);
        ctx->grids.push_back(Grid{nx, ny, x0, y0, dx, dy, std::vector<double>(eta, eta + (size_t)nx * ny), -2, nullptr});
        ctx->eta_index[3 * scen] = (int)ctx->grids.size() - 1;
    });
}

int tsu_set_velocity(tsu_ctx *ctx, int scen, const double *u, const double *v, int nx, int ny, double x0, double y0,
                     double dx, double dy)
{
    return guard(ctx, [&] {
        if (ctx->initialized) throw Err(TSU_ERR_ARG, "the initial velocities must be set before tsu_init");
        if (scen < 0 || scen >= ctx->nscen) throw Err(TSU_ERR_ARG, "bad scenario");
        check_grid(u, nx, ny, dx, dy);
        check_grid(v, nx, ny, dx, dy);
        const size_t n = (size_t)nx * ny;
        ctx->grids.push_back(Grid{nx, ny, x0, y0, dx, dy, std::vector<double>(u, u + n), -2, nullptr});
        ctx->eta_index[3 * scen + 1] = (int)ctx->grids.size() - 1;
        ctx->grids.push_back(Grid{nx, ny, x0, y0, dx, dy, std::vector<double>(v, v + n), -2, nullptr});
        ctx->eta_index[3 * scen + 2] = (int)ctx->grids.size() - 1;
    });
}

int tsu_add_uplift(tsu_ctx *ctx, int scen, const double *dB, int nx, int ny, double x0, double y0, double dx, double dy)
{
    return guard(ctx, [&] {
        if (scen < 0 || scen >= ctx->nscen) throw Err(TSU_ERR_ARG, "bad scenario");
        check_grid(dB, nx, ny, dx, dy);
        ctx->grids.push_back(Grid{nx, ny, x0, y0, dx, dy, std::vector<double>(dB, dB + (size_t)nx * ny), scen, nullptr});
        if (ctx->initialized) {
            ctx->upload_topo();
            ctx->add_uplift_now(scen, ctx->grids.back());
            ctx->sync();
        }
    });
}

int tsu_init(tsu_ctx *ctx)
{
    return guard(ctx, [&] { ctx->init(); });
}

int tsu_step(tsu_ctx *ctx, int n, double *t_out)
{
    bool cfl = false;
    int rc = guard(ctx, [&] {
        if (n < 0) throw Err(TSU_ERR_ARG, "negative step count");
        ctx->check_external_state();
        ctx->step(n);
        ctx->check_device_errors(cfl, t_out);
    });
    if (rc == TSU_OK && cfl) {
        ctx->err = "a level step ran with a Courant number above cfl_max";
        return TSU_ERR_CFL;
    }
    return rc;
}

int tsu_step_level(tsu_ctx *ctx, int level, double *t_out)
{
    bool cfl = false;
    int rc = guard(ctx, [&] {
        ctx->check_external_state();
        ctx->step_level(level - 1);
        ctx->check_device_errors(cfl, t_out);
    });
    if (rc == TSU_OK && cfl) {
        ctx->err = "a level step ran with a Courant number above cfl_max";
        return TSU_ERR_CFL;
    }
    return rc;
}

// Boxes of a halo exchange (tsu_halo_pack / tsu_halo_unpack): checked against
// the scenario's patches of the level, uploaded as HaloMsg with their offsets.
static long long halo_msgs(tsu_ctx *ctx, int scen, int level, const int *msgs, int n, DevBuf<HaloMsg> &d)
{
    if (!ctx->initialized || scen < 0 || scen >= ctx->nscen || level < 1 || level > ctx->nlev || n < 0 ||
        (n > 0 && !msgs))
        throw Err(TSU_ERR_ARG, "bad argument");
    Lvl &L = ctx->lv[level - 1];
    std::vector<int> ids;
    for (int q = 0; q < (int)L.P.size(); q++)
        if (L.P[q].scen == scen) ids.push_back(q);
    std::vector<HaloMsg> hm((size_t)n);
    long long off = 0;
    for (int k = 0; k < n; k++) {
        const int *m = msgs + 5 * (size_t)k;
        if (m[0] < 0 || m[0] >= (int)ids.size()) throw Err(TSU_ERR_ARG, "halo message: no such patch");
        const PatchDesc &P = L.P[ids[m[0]]];
        const int i0 = m[1], j0 = m[2], i1 = m[3], j1 = m[4];
        if (!(i0 < i1 && j0 < j1 && i0 >= P.i0 - 2 && j0 >= P.j0 - 2 && i1 <= P.i0 + P.nx + 2 && j1 <= P.j0 + P.ny + 2))
            throw Err(TSU_ERR_ARG, "halo message: box outside the patch and its ghost ring");
        hm[k] = HaloMsg{ids[m[0]], i0, j0, i1 - i0, j1 - j0, off};
        off += 3LL * (i1 - i0) * (j1 - j0);
    }
    d.upload(hm, ctx->st);
    return off;
}

int tsu_halo_pack(tsu_ctx *ctx, int scen, int level, const int *msgs, int n_msgs, void *dev_buf, long long buf_elems)
{
    return guard(ctx, [&] {
        DevBuf<HaloMsg> d;
        const long long need = halo_msgs(ctx, scen, level, msgs, n_msgs, d);
        if (need > buf_elems || (need > 0 && !dev_buf)) throw Err(TSU_ERR_ARG, "halo buffer too small");
        Lvl &L = ctx->lv[level - 1];
        ctx->kl(k_halo(ctx->prec, ctx->view(level - 1), d.p, n_msgs, L.cur, dev_buf, 0, ctx->st), "halo pack");
        d.release();
        ctx->sync();
    });
}

int tsu_halo_unpack(tsu_ctx *ctx, int scen, int level, const int *msgs, int n_msgs, const void *dev_buf,
                    long long buf_elems)
{
    return guard(ctx, [&] {
        DevBuf<HaloMsg> d;
        const long long need = halo_msgs(ctx, scen, level, msgs, n_msgs, d);
        if (need > buf_elems || (need > 0 && !dev_buf)) throw Err(TSU_ERR_ARG, "halo buffer too small");
        Lvl &L = ctx->lv[level - 1];
        ctx->kl(k_halo(ctx->prec, ctx->view(level - 1), d.p, n_msgs, L.cur, const_cast<void *>(dev_buf), 1, ctx->st),
                "halo unpack");
        d.release();
        ctx->sync();
    });
}

int tsu_regrid(tsu_ctx *ctx, int scen, int level)
{
    return guard(ctx, [&] {
        if (!ctx->initialized) throw Err(TSU_ERR_ARG, "tsu_init has not been called");
        if (scen < 0 || scen >= ctx->nscen || level < 1 || level >= ctx->nlev) throw Err(TSU_ERR_ARG, "bad scenario/level");
        ctx->regrid_from(level - 1, std::vector<int>{scen});
        bool cfl;
        ctx->check_device_errors(cfl);
    });
}

int tsu_num_patches(tsu_ctx *ctx, int scen, int level, int *n)
{
    return guard(ctx, [&] {
        if (scen < 0 || scen >= ctx->nscen || level < 1 || level > ctx->nlev || !n) throw Err(TSU_ERR_ARG, "bad argument");
        int k = 0;
        for (const auto &p : ctx->lv[level - 1].P) k += p.scen == scen;
        *n = k;
    });
}

int tsu_get_patches(tsu_ctx *ctx, int scen, int level, int *boxes, int max_patches, int *n)
{
    return guard(ctx, [&] {
        if (scen < 0 || scen >= ctx->nscen || level < 1 || level > ctx->nlev || !n) throw Err(TSU_ERR_ARG, "bad argument");
        int k = 0;
        for (const auto &p : ctx->lv[level - 1].P) {
            if (p.scen != scen) continue;
            if (k < max_patches && boxes) {
                boxes[4 * k] = p.i0; boxes[4 * k + 1] = p.j0; boxes[4 * k + 2] = p.nx; boxes[4 * k + 3] = p.ny;
            }
            k++;
        }
        *n = k;
    });
}

int tsu_get_patch(tsu_ctx *ctx, int scen, int level, int k, double *h, double *hu, double *hv, double *B)
{
    return guard(ctx, [&] {
        if (scen < 0 || scen >= ctx->nscen || level < 1 || level > ctx->nlev) throw Err(TSU_ERR_ARG, "bad argument");
        Lvl &L = ctx->lv[level - 1];
        int idx = -1, m = 0;
        for (int q = 0; q < (int)L.P.size(); q++)
            if (L.P[q].scen == scen) { if (m == k) { idx = q; break; } m++; }
        if (idx < 0) throw Err(TSU_ERR_ARG, "no such patch");
        const PatchDesc &p = L.P[idx];
        int nc = p.nx * p.ny;
        ctx->dstage.ensure((size_t)4 * nc, ctx->st);
        ctx->kl(k_patch_out(ctx->prec, ctx->view(level - 1), idx, nc, L.cur, ctx->dstage.p, ctx->st), "patch out");
        std::vector<double> hb((size_t)4 * nc);
        CK(cudaMemcpyAsync(hb.data(), ctx->dstage.p, hb.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
        ctx->sync();
        double *dst[4] = {h, hu, hv, B};
        for (int f = 0; f < 4; f++)
            if (dst[f]) std::memcpy(dst[f], hb.data() + (size_t)f * nc, nc * sizeof(double));
    });
}

int tsu_read_field(tsu_ctx *ctx, int scen, int level, int field, double *dst, int nx, int ny, double x0, double y0,
                   double dx, double dy)
{
    return guard(ctx, [&] {
        if (scen < 0 || scen >= ctx->nscen || level < 0 || level > ctx->nlev || field < 0 || field > 5 || !dst ||
            nx < 1 || ny < 1)
            throw Err(TSU_ERR_ARG, "bad argument");
        size_t n = (size_t)nx * ny;
        ctx->dstage.ensure(n, ctx->st);
        ctx->kl(k_fill(ctx->dstage.p, (long long)n, std::numeric_limits<double>::quiet_NaN(), ctx->st), "fill");
        int la = level == 0 ? 0 : level - 1, lb = level == 0 ? ctx->nlev - 1 : level - 1;
        for (int l = la; l <= lb; l++) {
            Lvl &L = ctx->lv[l];
            if (L.P.empty()) continue;
            // output points a patch can cover: its extent in output spacings, plus the edges
            const double sx = L.dx / dx, sy = L.dy / dy;
            long long maxpts = 1;
            for (const auto &P : L.P) {
                long long w = std::min<long long>(nx, (long long)std::ceil(P.nx * sx) + 3);
                long long h = std::min<long long>(ny, (long long)std::ceil(P.ny * sy) + 3);
                maxpts = std::max(maxpts, w * h);
            }
            ctx->kl(k_read_field(ctx->prec, ctx->view(l), (int)L.P.size(), (int)std::min<long long>(maxpts, 1LL << 30),
                                 L.cur, scen, field, ctx->dstage.p, nx, ny, x0, y0, dx, dy, ctx->c.x0, ctx->c.y0, L.dx,
                                 L.dy, ctx->st),
                    "read field");
        }
        // while the kernels run, host threads write the caller's pages once, so
        // the copies below do not stop at first-touch page faults
        const bool touched = n * sizeof(double) >= ((size_t)8 << 20);
        if (touched) {
            const int T = tsu::HostPool::get().size();
            tsu::HostPool::get().run(T, [&](int k) {
                const size_t a = n * (size_t)k / T, b = n * (size_t)(k + 1) / T;
                for (size_t i = a; i < b; i += 512) dst[i] = 0.0;   // one write per 4 KiB
            });
        }
        if (touched && ctx->pageable_access()) {
            // the copy engine reaches the caller's (now resident) pages itself; one
            // copy (copies into pageable memory issued from several threads at
            // once were measured far slower)
            CK(cudaMemcpyAsync(dst, ctx->dstage.p, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
            ctx->sync();
        } else {
            ctx->d2h_staged(dst, ctx->dstage.p, n);
        }
    });
}

int tsu_add_gauges(tsu_ctx *ctx, const double *xy, int n)
{
    return guard(ctx, [&] {
        if (n < 0 || (n > 0 && !xy)) throw Err(TSU_ERR_ARG, "bad gauges");
        if (ctx->nsamp > 0) throw Err(TSU_ERR_ARG, "gauges must be added before the first step");
        ctx->gxy.insert(ctx->gxy.end(), xy, xy + 2 * (size_t)n);
        ctx->dgxy.upload(ctx->gxy, ctx->st);
        if (ctx->initialized) ctx->update_gauges();
        ctx->hier_version++;
        ctx->sync();
    });
}

int tsu_read_gauges(tsu_ctx *ctx, double *t, double *eta, int max_samples, int *n_written)
{
    return guard(ctx, [&] {
        if (!n_written || max_samples < 0) throw Err(TSU_ERR_ARG, "bad argument");
        int ng = (int)ctx->gxy.size() / 2;
        long long n = std::min<long long>(ctx->nsamp, max_samples);
        if (ng && n > 0) {
            CK(cudaMemcpyAsync(t, ctx->dgt.p, (size_t)n * ctx->nscen * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
            CK(cudaMemcpyAsync(eta, ctx->dgeta.p, (size_t)n * ctx->nscen * ng * sizeof(double), cudaMemcpyDeviceToHost,
                               ctx->st));
        }
        ctx->sync();
        *n_written = ng ? (int)n : 0;
    });
}

int tsu_get_stats(tsu_ctx *ctx, int scen, tsu_stats *out)
{
    return guard(ctx, [&] {
        if (scen < 0 || scen >= ctx->nscen || !out) throw Err(TSU_ERR_ARG, "bad argument");
        std::memset(out, 0, sizeof *out);
        CK(cudaMemsetAsync(ctx->mass.p, 0, ctx->nscen * sizeof(double), ctx->st));
        Lvl &L = ctx->lv[0];
        if (!L.P.empty()) {
            ctx->massParts.ensure((size_t)k_mass_parts((int)L.P.size(), L.maxcells), ctx->st);
            ctx->kl(k_mass(ctx->prec, ctx->view(0), (int)L.P.size(), L.maxcells, L.cur, ctx->massParts.p, ctx->mass.p,
                           ctx->nscen, ctx->st),
                    "mass");
            ctx->launches++;   // k_mass runs two kernels
        }
        double v[4];
        long long vi, vr;
        CK(cudaMemcpyAsync(&v[0], ctx->dt1.p + scen, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaMemcpyAsync(&v[1], ctx->t.p + scen, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaMemcpyAsync(&v[2], ctx->mass.p + scen, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaMemcpyAsync(&v[3], ctx->cellupd.p + scen, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaMemcpyAsync(&vi, ctx->viol.p + scen, sizeof(long long), cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaMemcpyAsync(&vr, ctx->retakes.p + scen, sizeof(long long), cudaMemcpyDeviceToHost, ctx->st));
        ctx->sync();
        out->dt = v[0];
        out->t = v[1];
        out->mass = v[2] * ctx->pdx(0) * ctx->pdy(0);
        out->cell_updates = v[3];
        out->cfl_violations = vi;
        out->cfl_retakes = vr;
        for (int l = 0; l < ctx->nlev; l++)
            for (const auto &p : ctx->lv[l].P) out->patches[l] += p.scen == scen;
        out->kernel_launches = ctx->launches;
        out->regrids = ctx->n_regrids;
        out->regrid_host_ms = ctx->regrid_ms;
        out->regrid_wait_ms = ctx->regrid_wait_ms;
        out->patches_renewed = ctx->n_patches_renewed;
        out->patches_reused = ctx->n_patches_reused;
        out->cluster_ms = ctx->cluster_ms;
    });
}

int tsu_set_bulk_copies(tsu_ctx *ctx, int enable, long long polls)
{
    return guard(ctx, [&] {
        if ((enable != 0 && enable != 1) || polls < 0 || polls > 0xffffffffLL)
            throw Err(TSU_ERR_ARG, "enable must be 0 or 1 and polls lie in [0, 2^32 - 1]");
        ctx->bulk_rows = enable;
        ctx->wait_polls = (unsigned)polls;
        ctx->hier_version++;   // captured graphs carry the old launch arguments
    });
}

int tsu_set_tuning(tsu_ctx *ctx, int step_threads, int seg_rows)
{
    return guard(ctx, [&] {
        const bool narrow = ctx->prec != TSU_F64 && ctx->c.transverse == 0;   // the paired FP32 kernel has 32
        if (!(step_threads == 0 || step_threads == 64 || step_threads == 128 || step_threads == 256 ||
              (narrow && step_threads == 32)) || seg_rows < 0)
            throw Err(TSU_ERR_ARG, "step_threads must be 0, 64, 128 or 256 (32 for the split FP32 update) and "
                                   "seg_rows >= 0");
        ctx->step_nt = step_threads;
        ctx->seg_rows = seg_rows;
        for (int l = 0; l < ctx->nlev; l++)
            if (!ctx->lv[l].P.empty()) ctx->finish_level(l);
        ctx->sync();
    });
}

int tsu_autotune(tsu_ctx *ctx, int reps, int *best_threads, int *best_seg_rows, double *best_ms)
{
    return guard(ctx, [&] {
        if (!ctx->initialized) throw Err(TSU_ERR_ARG, "tsu_init has not been called");
        if (reps < 1) reps = 3;
        // zero time step: the kernels do all their work but leave the state as it is
        ctx->zero_dt.ensure(ctx->nscen, ctx->st);
        ctx->zero_dtf.ensure(ctx->nscen, ctx->st);
        CK(cudaMemsetAsync(ctx->zero_dt.p, 0, ctx->nscen * sizeof(double), ctx->st));
        CK(cudaMemsetAsync(ctx->zero_dtf.p, 0, ctx->nscen * sizeof(float), ctx->st));
        // threads x rows per work item; the FP32 split update's x kernel also takes
        // 32 threads and needs no halo rows, so it gets shorter segments
        const bool split = ctx->split_f32();
        const int nts[4] = {64, 128, 256, 32};
        const int segs[4] = {split ? 16 : 32, split ? 32 : 64, split ? 64 : 128, split ? 128 : 256};
        const int n_nt = split ? 4 : 3;
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        double best = 1e30;
        int bt = 0, bs = 0;
        for (int a = 0; a < n_nt; a++)
            for (int b = 0; b < 4; b++) {
                ctx->step_nt = nts[a];
                ctx->seg_rows = segs[b];
                for (int l = 0; l < ctx->nlev; l++)
                    if (!ctx->lv[l].P.empty()) ctx->finish_level(l);
                auto run = [&] {
                    for (int l = 0; l < ctx->nlev; l++) {
                        Lvl &L = ctx->lv[l];
                        if (L.P.empty()) continue;
                        StepArgs sa{};
                        sa.descs = L.dP.p; sa.items = L.dItems.p; sa.arena = ctx->arena.base; sa.cur = L.cur;
                        sa.dt1 = ctx->zero_dt.p; sa.dt1f = ctx->zero_dtf.p; sa.smax = ctx->smax.p; sa.R = L.R;
                        sa.g = ctx->c.g; sa.drytol = ctx->c.drytol;
                        sa.transverse = ctx->c.transverse;
                        sa.manning = (ctx->c.manning_n * ctx->c.manning_n) * ctx->c.g;
                        ctx->level_args(sa, l);
                        set_f32_constants(sa);
                        int e = ctx->prec == TSU_F64 ? launch_step_f64(sa, (int)L.items.size(), ctx->nt(), ctx->st)
                                                     : launch_step_f32p(sa, (int)L.items.size(), ctx->nt(), ctx->st);
                        ctx->kl(e, "autotune step");
                        ctx->launches += ctx->step_kernels() - 1;
                    }
                };
                run();
                CK(cudaEventRecord(e0, ctx->st));
                for (int k = 0; k < reps; k++) run();
                CK(cudaEventRecord(e1, ctx->st));
                CK(cudaEventSynchronize(e1));
                float ms = 0;
                CK(cudaEventElapsedTime(&ms, e0, e1));
                if (ms / reps < best) { best = ms / reps; bt = nts[a]; bs = segs[b]; }
            }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        CK(cudaMemsetAsync(ctx->smax.p, 0, 2 * ctx->nscen * sizeof(unsigned long long), ctx->st));
        ctx->step_nt = bt;
        ctx->seg_rows = bs;
        for (int l = 0; l < ctx->nlev; l++)
            if (!ctx->lv[l].P.empty()) ctx->finish_level(l);
        ctx->sync();
        if (best_threads) *best_threads = bt;
        if (best_seg_rows) *best_seg_rows = bs;
        if (best_ms) *best_ms = best;
    });
}

int tsu_cnn_set_weights(tsu_ctx *ctx, const float *theta, int n)
{
    return guard(ctx, [&] {
        if (!theta || n != cnn_n_params()) throw Err(TSU_ERR_ARG, "expected tsu_cnn_num_params() weights");
        std::vector<float> v(theta, theta + n);
        ctx->cnn_theta.upload(v, ctx->st);
        ctx->cnn_ready = true;
        ctx->sync();
    });
}

int tsu_cnn_features(tsu_ctx *ctx, int scen, int level, float *features, unsigned char *flags)
{
    return guard(ctx, [&] {
        if (!ctx->initialized) throw Err(TSU_ERR_ARG, "tsu_init has not been called");
        if (scen < 0 || scen >= ctx->nscen || level < 1 || level > ctx->nlev) throw Err(TSU_ERR_ARG, "bad scenario/level");
        const int l = level - 1;
        Lvl &C = ctx->lv[l];
        const size_t plane = (size_t)C.nxl * C.nyl;
        std::vector<int> slot(ctx->nscen, -1);
        slot[scen] = 0;
        ctx->fslot.upload(slot, ctx->st);
        ctx->fraw.ensure(plane, ctx->st);
        ctx->fcov.ensure(plane, ctx->st);
        CK(cudaMemsetAsync(ctx->fraw.p, 0, plane, ctx->st));
        CK(cudaMemsetAsync(ctx->fcov.p, 0, plane, ctx->st));
        FlagArgs fa{};
        fa.raw = ctx->fraw.p; fa.cov = ctx->fcov.p; fa.scen_slot = ctx->fslot.p;
        fa.eta_tol = ctx->c.flag_eta_tol; fa.depth_below = ctx->c.flag_depth_below; fa.drytol = ctx->c.drytol;
        fa.eta_tol_f = float_at_most(ctx->c.flag_eta_tol);
        fa.depth_neg_f = float_at_most(-ctx->c.flag_depth_below);
        fa.drytol_f = (float)ctx->c.drytol;
        fa.x0 = ctx->c.x0; fa.y0 = ctx->c.y0; fa.dxl = C.dx; fa.dyl = C.dy;
        fa.n_regions = ctx->c.n_regions; fa.newlev = level + 1;
        for (int k = 0; k < ctx->c.n_regions; k++)
            for (int m = 0; m < 6; m++) fa.regions[6 * k + m] = ctx->c.regions[k][m];
        ctx->kl(k_flag(ctx->prec, ctx->view(l), (int)C.P.size(), C.maxcells, C.cur, fa, ctx->st), "flag");
        ctx->cnn_feat.ensure(plane * 5, ctx->st);
        CK(cudaMemsetAsync(ctx->cnn_feat.p, 0, plane * 5 * sizeof(float), ctx->st));
        const CnnWindow whole{0, 0, C.nxl, C.nyl, 0, 0, C.nxl, C.nyl};
        ctx->kl(k_cnn_features(ctx->prec, ctx->view(l), (int)C.P.size(), C.maxcells, C.cur, ctx->fslot.p, ctx->fraw.p,
                               ctx->cnn_feat.p, ctx->c.drytol, whole, ctx->st), "cnn features");
        if (features)
            CK(cudaMemcpyAsync(features, ctx->cnn_feat.p, plane * 5 * sizeof(float), cudaMemcpyDeviceToHost, ctx->st));
        if (flags) CK(cudaMemcpyAsync(flags, ctx->fraw.p, plane, cudaMemcpyDeviceToHost, ctx->st));
        ctx->sync();
    });
}

int tsu_sync(tsu_ctx *ctx)
{
    return guard(ctx, [&] { ctx->sync(); });
}

int tsu_level1_buffers(tsu_ctx *ctx, void **h, void **hu, void **hv, void **B, int *pitch)
{
    return guard(ctx, [&] {
        if (ctx->lv[0].P.empty()) throw Err(TSU_ERR_ARG, "not initialised");
        const PatchDesc &p = ctx->lv[0].P[0];
        char *base = ctx->arena.base + (size_t)p.off * ctx->esz;
        int cur = ctx->lv[0].cur;
        size_t fsb = (size_t)p.fs * ctx->esz;
        if (h) *h = base + (cur * 3 + 0) * fsb;
        if (hu) *hu = base + (cur * 3 + 1) * fsb;
        if (hv) *hv = base + (cur * 3 + 2) * fsb;
        if (B) *B = base + 6 * fsb;
        if (pitch) *pitch = p.pitch;
        ctx->ext_state = true;   // the caller may write through these
    });
}

int tsu_profile_levels(tsu_ctx *ctx, int enable)
{
    return guard(ctx, [&] {
        ctx->prof = enable != 0;
        ctx->sync();
        for (auto &p : ctx->prof_steps) {
            ctx->prof_pool.push_back(p.e0);
            ctx->prof_pool.push_back(p.e1);
        }
        ctx->prof_steps.clear();
    });
}

int tsu_level_update_times(tsu_ctx *ctx, double *ms, double *cells, long long *steps, long long *kernels,
                           int max_levels)
{
    return guard(ctx, [&] {
        if (!ms || !cells || !steps || !kernels || max_levels < 1) throw Err(TSU_ERR_ARG, "bad argument");
        for (int l = 0; l < max_levels; l++) { ms[l] = 0.0; cells[l] = 0.0; steps[l] = 0; kernels[l] = 0; }
        ctx->sync();
        for (auto &p : ctx->prof_steps) {
            if (p.level < max_levels) {
                float t = 0.0f;
                CK(cudaEventElapsedTime(&t, p.e0, p.e1));
                ms[p.level] += (double)t;
                cells[p.level] += p.cells;
                steps[p.level] += 1;
                kernels[p.level] += p.kernels;
            }
            ctx->prof_pool.push_back(p.e0);
            ctx->prof_pool.push_back(p.e1);
        }
        ctx->prof_steps.clear();
    });
}

int tsu_time_level1_steps(tsu_ctx *ctx, int warmup, int n, double *kernel_ms_out, double *step_ms_out)
{
    return guard(ctx, [&] {
        if (!ctx->initialized || ctx->nlev != 1 || n < 1 || warmup < 0)
            throw Err(TSU_ERR_ARG, "single-level context after tsu_init required");
        ctx->ensure_samples(ctx->nsamp + warmup + n + 2);
        for (int k = 0; k < warmup; k++) ctx->coarse_step();
        std::vector<cudaEvent_t> ev(2 * n + 2);
        for (auto &e : ev) CK(cudaEventCreate(&e));
        Lvl &L = ctx->lv[0];
        CK(cudaEventRecord(ev[2 * n], ctx->st));
        for (int k = 0; k < n; k++) {
            ctx->kl(k_begin_step(ctx->ctrl(), ctx->nscen, ctx->nlev, ctx->Rl.p, ctx->c.cfl_desired, ctx->c.dt_max, ctx->st),
                    "begin step");
            if (L.P.size() > 1) {
                ctx->kl(k_ghost_fill(ctx->prec, ctx->view(0), ctx->view(0), (int)L.P.size(), L.maxring, L.cur, 0, 0, 0.0,
                                     ctx->c.drytol, ctx->derr.p, ctx->st), "ghost fill");
            }
            if (!L.bclist.empty()) {
                BcArgs ba{L.dBc.p, {ctx->c.bc[0], ctx->c.bc[1], ctx->c.bc[2], ctx->c.bc[3]}};
                ctx->kl(k_bc(ctx->prec, ctx->view(0), ba, (int)L.bclist.size(), L.maxring, L.cur, 1, 0, ctx->st), "bc");
            }
            StepArgs a{};
            a.descs = L.dP.p; a.items = L.dItems.p; a.arena = ctx->arena.base; a.cur = L.cur; a.dt1 = ctx->dt1.p;
            a.smax = ctx->smax.p; a.R = L.R; a.g = ctx->c.g; a.drytol = ctx->c.drytol;
            a.dt1f = ctx->dt1f.p;
            a.transverse = ctx->c.transverse;
            a.manning = (ctx->c.manning_n * ctx->c.manning_n) * ctx->c.g;
            ctx->level_args(a, 0);
            set_f32_constants(a);
            CK(cudaEventRecord(ev[2 * k], ctx->st));
            int e = ctx->prec == TSU_F64 ? launch_step_f64(a, (int)L.items.size(), ctx->nt(), ctx->st)
                                         : launch_step_f32p(a, (int)L.items.size(), ctx->nt(), ctx->st);
            ctx->kl(e, "patch step");
            ctx->launches += ctx->step_kernels() - 1;
            CK(cudaEventRecord(ev[2 * k + 1], ctx->st));
            // the rest of the step exactly as level_step and coarse_step run it: with
            // the CFL retake on, the post-level check, the retake launch (its CTAs
            // exit unless their scenario is retaken) and the check after it, then
            // the end of the coarse step; without it, the post-level kernel also ends
            // the coarse step
            const bool retake = ctx->c.cfl_retake != 0;
            ctx->kl(k_post_level(ctx->ctrl(), 0, ctx->nscen, L.R, ctx->pdx(0), ctx->pdy(0), ctx->c.cfl_max,
                                 ctx->c.cfl_desired, retake ? 2 : 0, ctx->st, retake ? 0 : 1),
                    "post step");
            if (retake) {
                a.gate = ctx->retake_gate();
                e = ctx->retake_launch(a, L);
                ctx->kl(e, "patch step (retake)");
                ctx->launches += ctx->step_kernels() - 1;
                ctx->kl(k_post_level(ctx->ctrl(), 0, ctx->nscen, L.R, ctx->pdx(0), ctx->pdy(0), ctx->c.cfl_max,
                                     ctx->c.cfl_desired, 3, ctx->st, 1),
                        "post step (retake)");
            }
            L.cur ^= 1;
            for (int s = 0; s < ctx->nscen; s++) ctx->nsteps[s][0]++;
            ctx->sample_gauges();
        }
        CK(cudaEventRecord(ev[2 * n + 1], ctx->st));
        ctx->sync();
        double ks = 0;
        for (int k = 0; k < n; k++) {
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, ev[2 * k], ev[2 * k + 1]));
            ks += ms;
        }
        float tot = 0;
        CK(cudaEventElapsedTime(&tot, ev[2 * n], ev[2 * n + 1]));
        for (auto &e : ev) cudaEventDestroy(e);
        if (kernel_ms_out) *kernel_ms_out = ks / n;
        if (step_ms_out) *step_ms_out = tot / n;
        ctx->hier_version++;
    });
}

}  // extern "C"

int tsu_cluster_flags(const unsigned char *flags, const unsigned char *nestable, int nx, int ny, double eff,
                      int ratio, int patch_max, int *boxes, int max_boxes, int *n_boxes)
{
    try {
        if (!flags || !boxes || !n_boxes || nx < 1 || ny < 1 || ratio < 1 || patch_max < 1 || max_boxes < 0)
            return TSU_ERR_ARG;
        // the packed plane the regrid clusters: 4 cells per byte, flag and nestable bits
        const int ps = (nx + 3) / 4;
        std::vector<uint8_t> fn((size_t)ps * ny, 0);
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                const size_t k = (size_t)j * nx + i;
                const int v = (flags[k] ? 1 : 0) | ((!nestable || nestable[k]) ? 2 : 0);
                fn[(size_t)j * ps + i / 4] |= (uint8_t)(v << (2 * (i % 4)));
            }
        std::vector<std::array<int, 4>> out;
        tsu::cluster_boxes(fn.data(), nx, ny, ps, eff, ratio, patch_max, out, 16, nullptr);
        *n_boxes = (int)out.size();
        if ((int)out.size() > max_boxes) return TSU_ERR_ARG;
        for (size_t k = 0; k < out.size(); k++)
            for (int m = 0; m < 4; m++) boxes[4 * k + m] = out[k][m];
        return TSU_OK;
    } catch (...) {
        return TSU_ERR_ARG;
    }
}

int tsu_checkpoint_save(tsu_ctx *ctx, void *buf, size_t cap, size_t *written)
{
    return guard(ctx, [&] {
        if (!written) throw Err(TSU_ERR_ARG, "bad argument");
        std::vector<uint8_t> v = ctx->checkpoint();
        *written = v.size();
        if (buf == nullptr && cap == 0) return;    // size query
        if (!buf || cap < v.size()) throw Err(TSU_ERR_ARG, "checkpoint buffer too small");
        std::memcpy(buf, v.data(), v.size());
    });
}

int tsu_checkpoint_restore(tsu_ctx *ctx, const void *buf, size_t n)
{
    return guard(ctx, [&] {
        if (!buf) throw Err(TSU_ERR_ARG, "bad argument");
        ctx->restore(reinterpret_cast<const uint8_t *>(buf), n);
        ctx->ext_state = true;
    });
}
