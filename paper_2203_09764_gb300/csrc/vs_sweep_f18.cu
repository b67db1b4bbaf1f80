// FP32 arithmetic, 18-real link storage.
#include "vs_sweep_inst.cuh"
namespace vs {
cudaError_t launch_subsweep_f18(bool rect, int mu, const SubsweepParams &p, cudaStream_t st) {
    return launch_subsweep_tpl<float, 18>(rect, mu, p, st);
}
cudaError_t launch_aus_f18(bool rect, int mu, const AusParams &p, cudaStream_t st) {
    return launch_aus_tpl<float, 18>(rect, mu, p, st);
}
}  // namespace vs
