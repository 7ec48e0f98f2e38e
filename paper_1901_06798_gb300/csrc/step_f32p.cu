// step_f32p.cu -- FP32 surface-perturbation form of the patch update: state
// (eta' = h + B, hu, hv) and B in FP32.  The surface jump that drives the waves
// is formed from eta' directly, so still water is exactly still and the
// ocean-depth cancellation of h + B never enters the flux.  Levels with a Q*
// scratch run the split step as two kernels (step_split_f32.cuh); without one
// (the allocation-free entry point) the fused kernel (step_f32x2.cuh).
#include "step_split_f32.cuh"

namespace tsu {

static constexpr int kThreadsF32 = 128;

int step_threads_f32p() { return kThreadsF32; }
int step_strip_width_f32p(int threads, int transverse) { return transverse ? threads - 4 : 2 * threads - 4; }

// threads per CTA: 32, 64, 128 or 256 (two columns per thread: strip width 2 threads - 4)
int launch_step_f32p(const StepArgs &a, int n_items, int threads, cudaStream_t st)
{
    if (n_items <= 0) return 0;
    if (a.transverse) return launch_unsplit_f32p(a, n_items, threads, st);
    if (a.scratch != nullptr) {
        // x sweep over a.items (strips of 2 threads - 4 columns), then y sweep over a.items_y
        const bool geo = a.kap != nullptr;
        if (a.bulk_rows) {   // rows by bulk copies on mbarriers (Cartesian and latitude-longitude)
            switch (threads) {
            case 32: geo ? step_x_f32x2<32, 4, true, true><<<n_items, 32, 0, st>>>(a) : step_x_f32x2<32, 4, false, true><<<n_items, 32, 0, st>>>(a); break;
            case 64: geo ? step_x_f32x2<64, 4, true, true><<<n_items, 64, 0, st>>>(a) : step_x_f32x2<64, 4, false, true><<<n_items, 64, 0, st>>>(a); break;
            case 128: geo ? step_x_f32x2<128, 4, true, true><<<n_items, 128, 0, st>>>(a) : step_x_f32x2<128, 4, false, true><<<n_items, 128, 0, st>>>(a); break;
            case 256: geo ? step_x_f32x2<256, 4, true, true><<<n_items, 256, 0, st>>>(a) : step_x_f32x2<256, 4, false, true><<<n_items, 256, 0, st>>>(a); break;
            default: return (int)cudaErrorInvalidValue;
            }
        } else {
            switch (threads) {
            case 32: geo ? step_x_f32x2<32, 4, true><<<n_items, 32, 0, st>>>(a) : step_x_f32x2<32, 4, false><<<n_items, 32, 0, st>>>(a); break;
            case 64: geo ? step_x_f32x2<64, 4, true><<<n_items, 64, 0, st>>>(a) : step_x_f32x2<64, 4, false><<<n_items, 64, 0, st>>>(a); break;
            case 128: geo ? step_x_f32x2<128, 4, true><<<n_items, 128, 0, st>>>(a) : step_x_f32x2<128, 4, false><<<n_items, 128, 0, st>>>(a); break;
            case 256: geo ? step_x_f32x2<256, 4, true><<<n_items, 256, 0, st>>>(a) : step_x_f32x2<256, 4, false><<<n_items, 256, 0, st>>>(a); break;
            default: return (int)cudaErrorInvalidValue;
            }
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess || a.n_items_y <= 0) return (int)e;
        if (geo) step_y_f32x2<true><<<a.n_items_y, kSplitYThreads, 0, st>>>(a);
        else step_y_f32x2<false><<<a.n_items_y, kSplitYThreads, 0, st>>>(a);
        return (int)cudaGetLastError();
    }
    if (a.kap != nullptr) {   // latitude-longitude grid (capacity form)
        switch (threads) {
        case 32: step_kernel_f32x2<32, 4, true><<<n_items, 32, 0, st>>>(a); break;
        case 64: step_kernel_f32x2<64, 4, true><<<n_items, 64, 0, st>>>(a); break;
        case 128: step_kernel_f32x2<128, 4, true><<<n_items, 128, 0, st>>>(a); break;
        case 256: step_kernel_f32x2<256, 4, true><<<n_items, 256, 0, st>>>(a); break;
        default: return (int)cudaErrorInvalidValue;
        }
        return (int)cudaGetLastError();
    }
    switch (threads) {
    case 32: step_kernel_f32x2<32, 4><<<n_items, 32, 0, st>>>(a); break;
    case 64: step_kernel_f32x2<64, 4><<<n_items, 64, 0, st>>>(a); break;
    case 128: step_kernel_f32x2<128, 4><<<n_items, 128, 0, st>>>(a); break;
    case 256: step_kernel_f32x2<256, 4><<<n_items, 256, 0, st>>>(a); break;
    default: return (int)cudaErrorInvalidValue;
    }
    return (int)cudaGetLastError();
}

}  // namespace tsu
