// noalloc.cu -- tsu_grid_step_noalloc: one dimensionally split step of a
// uniform grid that lives in the caller's device memory, without allocating
// anything.
//
// Who needs this: applications whose device memory is owned end to end by
// their own allocator (a framework's caching allocator, or a service that
// reserves all of HBM up front and hands out slices) must not call cudaMalloc
// behind its back, and latency-critical loops cannot afford a cudaMalloc that
// may block or fail.  The context-based entry points allocate (the patch
// arena, tables, flags); this one keeps its few bytes of scratch -- patch
// descriptor, work items, boundary list, dt and the wave-speed accumulator --
// in one file-scope __device__ array instead.
//
// The scratch array is shared by every call in the process on a given GPU
// and keeps the contents of the last call; each call rewrites all of it (and
// clears the speed accumulator) before use.  Calls whose work overlaps on the
// GPU (different streams, or different host threads) race on it.
#include <cstdint>
#include <cstring>
#include <mutex>
#include <cuda_runtime.h>

#include "../../include/tsunami.h"
#include "amr_kernels.h"
#include "tsu_device.h"

namespace tsu {

namespace {

constexpr size_t kScratchBytes = 1u << 20;          // 1 MiB per GPU
constexpr size_t kDescOff = 0;                      // PatchDesc
constexpr size_t kListOff = 256;                    // int bclist[1]
constexpr size_t kDtOff = 272;                      // double dt
constexpr size_t kDtfOff = 280;                     // float dt
constexpr size_t kSmaxOff = 288;                    // unsigned long long smax[2]
constexpr size_t kItemsOff = 512;                   // StepItem items[]
constexpr int kMaxItems = (int)((kScratchBytes - kItemsOff) / sizeof(StepItem));
constexpr int kSegRows = 128;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

// Address of the scratch array on the current device, looked up once per
// device (the host-side name of a __device__ array is not a device address).
cudaError_t scratch_for_current_device(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

__global__ void noalloc_prepare_kernel(unsigned char *scratch, long long fstride, int nx, int ny, int pitch,
                                       double dt, int W, int nsx, int nsy)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        PatchDesc d;
        memset(&d, 0, sizeof d);
        d.off = 0;
        d.fs = fstride;
        d.i0 = 0; d.j0 = 0; d.nx = nx; d.ny = ny; d.pitch = pitch;
        d.scen = 0;
        d.bcmask = 15;
        *reinterpret_cast<PatchDesc *>(scratch + kDescOff) = d;
        *reinterpret_cast<int *>(scratch + kListOff) = 0;
        *reinterpret_cast<double *>(scratch + kDtOff) = dt;
        *reinterpret_cast<float *>(scratch + kDtfOff) = (float)dt;
        unsigned long long *sm = reinterpret_cast<unsigned long long *>(scratch + kSmaxOff);
        sm[0] = 0ull;
        sm[1] = 0ull;
    }
    StepItem *items = reinterpret_cast<StepItem *>(scratch + kItemsOff);
    const int n = nsx * nsy;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        int sx = k % nsx, sy = k / nsx;
        int x0 = sx * W, y0 = sy * kSegRows;
        items[k] = StepItem{0, x0, y0, min(W, nx - x0), min(kSegRows, ny - y0)};
    }
}

}  // namespace
}  // namespace tsu

using namespace tsu;

extern "C" int tsu_grid_step_noalloc(int precision, void *block, int nx, int ny, int pitch, long long field_stride,
                                     int cur, double dx, double dy, double dt, double g, double drytol, const int *bc,
                                     double *max_speeds, void *cuda_stream)
{
    if (precision != TSU_F64 && precision != TSU_F32P) return TSU_ERR_ARG;
    if (!block || !bc || !max_speeds) return TSU_ERR_ARG;
    if (nx < 1 || ny < 1 || nx > TSU_NOALLOC_MAX_SIDE || ny > TSU_NOALLOC_MAX_SIDE) return TSU_ERR_ARG;
    if (pitch < nx + 4 || field_stride < (long long)pitch * (ny + 4) || (cur != 0 && cur != 1)) return TSU_ERR_ARG;
    if (!(dx > 0) || !(dy > 0) || !(dt >= 0) || !(g > 0) || !(drytol > 0)) return TSU_ERR_ARG;
    for (int k = 0; k < 4; k++)
        if (bc[k] != TSU_BC_WALL && bc[k] != TSU_BC_EXTRAP) return TSU_ERR_ARG;
    const size_t esz = precision == TSU_F64 ? 8 : 4;
    if (((uintptr_t)block) % esz) return TSU_ERR_ARG;
    const int nt = precision == TSU_F64 ? step_threads_f64() : step_threads_f32p();
    const int W = precision == TSU_F64 ? step_strip_width_f64(nt, 0) : step_strip_width_f32p(nt, 0);
    const int nsx = (nx + W - 1) / W, nsy = (ny + kSegRows - 1) / kSegRows;
    if ((long long)nsx * nsy > kMaxItems) return TSU_ERR_ARG;

    cudaStream_t st = (cudaStream_t)cuda_stream;
    void *sp = nullptr;
    if (scratch_for_current_device(&sp) != cudaSuccess) return TSU_ERR_CUDA;
    unsigned char *scratch = reinterpret_cast<unsigned char *>(sp);

    int blocks = (nsx * nsy + 255) / 256;
    noalloc_prepare_kernel<<<blocks, 256, 0, st>>>(scratch, field_stride, nx, ny, pitch, dt, W, nsx, nsy);
    if (cudaGetLastError() != cudaSuccess) return TSU_ERR_CUDA;

    const PatchDesc *desc = reinterpret_cast<const PatchDesc *>(scratch + kDescOff);
    LevelView L{};
    L.descs = desc;
    L.arena = block;
    L.nxl = nx;
    L.nyl = ny;
    BcArgs ba{reinterpret_cast<const int *>(scratch + kListOff), {bc[0], bc[1], bc[2], bc[3]}};
    const int ring = (nx + 4) * (ny + 4) - nx * ny;
    if (k_bc(precision, L, ba, 1, ring, cur, 1, 1, st) != 0) return TSU_ERR_CUDA;

    StepArgs a{};
    a.descs = desc;
    a.items = reinterpret_cast<const StepItem *>(scratch + kItemsOff);
    a.arena = block;
    a.cur = cur;
    a.dt1 = reinterpret_cast<const double *>(scratch + kDtOff);
    a.smax = reinterpret_cast<unsigned long long *>(scratch + kSmaxOff);
    a.R = 1.0;
    a.dx = dx;
    a.dy = dy;
    a.g = g;
    a.drytol = drytol;
    a.dt1f = reinterpret_cast<const float *>(scratch + kDtfOff);
    set_f32_constants(a);
    int e = precision == TSU_F64 ? launch_step_f64(a, nsx * nsy, nt, st) : launch_step_f32p(a, nsx * nsy, nt, st);
    if (e != 0) return TSU_ERR_CUDA;

    unsigned long long bits[2] = {0ull, 0ull};
    if (cudaMemcpyAsync(bits, scratch + kSmaxOff, sizeof bits, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return TSU_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return TSU_ERR_CUDA;
    for (int k = 0; k < 2; k++) {
        double v;
        std::memcpy(&v, &bits[k], sizeof v);
        max_speeds[k] = v;
    }
    return TSU_OK;
}
