// step_unsplit_f32p.cu -- FP32 surface-perturbation instantiation of the
// unsplit update with transverse corrections (state eta' = h + B, hu, hv and
// B in FP32).
#include "step_unsplit_f32.cuh"

namespace tsu {

int launch_unsplit_f32p(const StepArgs &a, int n_items, int threads, cudaStream_t st)
{
    if (n_items <= 0) return 0;
    switch (threads) {
    case 64: return launch_unsplit_f32_nt<64>(a, n_items, st);
    case 128: return launch_unsplit_f32_nt<128>(a, n_items, st);
    case 256: return launch_unsplit_f32_nt<256>(a, n_items, st);
    default: return (int)cudaErrorInvalidValue;
    }
}

}  // namespace tsu
