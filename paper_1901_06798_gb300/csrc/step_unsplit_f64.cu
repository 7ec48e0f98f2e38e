// step_unsplit_f64.cu -- FP64 instantiation of the unsplit update with
// transverse corrections.  Built with --fmad=false so every multiply and add
// rounds exactly as the FP64 oracle's.
#include "step_unsplit.cuh"

namespace tsu {

int launch_unsplit_f64(const StepArgs &a, int n_items, int threads, cudaStream_t st)
{
    if (n_items <= 0) return 0;
    switch (threads) {
    case 64: return launch_unsplit_nt<double, false, 64>(a, n_items, st);
    case 128: return launch_unsplit_nt<double, false, 128>(a, n_items, st);
    case 256: return launch_unsplit_nt<double, false, 256>(a, n_items, st);
    default: return (int)cudaErrorInvalidValue;
    }
}

}  // namespace tsu
