// step_f64.cu -- FP64 instantiation of the fused patch update.  Built with
// --fmad=false so every multiply and add rounds exactly as the FP64 oracle's.
#include "step_kernel.cuh"

namespace tsu {

static constexpr int kThreadsF64 = 64;

int step_threads_f64() { return kThreadsF64; }
int step_strip_width_f64(int threads, int) { return threads - 4; }

// threads per CTA: 64, 128 or 256 (strip width threads - 4 columns)
int launch_step_f64(const StepArgs &a, int n_items, int threads, cudaStream_t st)
{
    if (n_items <= 0) return 0;
    if (a.transverse) return launch_unsplit_f64(a, n_items, threads, st);
    const bool geo = a.kap != nullptr;   // latitude-longitude grid (capacity form)
    switch (threads) {
    case 64:
        if (geo) step_kernel<double, false, 64, 4, true><<<n_items, 64, 0, st>>>(a);
        else step_kernel<double, false, 64, 4><<<n_items, 64, 0, st>>>(a);
        break;
    case 128:
        if (geo) step_kernel<double, false, 128, 4, true><<<n_items, 128, 0, st>>>(a);
        else step_kernel<double, false, 128, 4><<<n_items, 128, 0, st>>>(a);
        break;
    case 256:
        if (geo) step_kernel<double, false, 256, 4, true><<<n_items, 256, 0, st>>>(a);
        else step_kernel<double, false, 256, 4><<<n_items, 256, 0, st>>>(a);
        break;
    default: return (int)cudaErrorInvalidValue;
    }
    return (int)cudaGetLastError();
}

}  // namespace tsu
