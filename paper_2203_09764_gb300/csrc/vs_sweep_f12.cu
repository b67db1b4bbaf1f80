// FP32 arithmetic, 12-real link storage (row 3 rebuilt on load).
#include "vs_sweep_inst.cuh"
namespace vs {
cudaError_t launch_subsweep_f12(bool rect, int mu, const SubsweepParams &p, cudaStream_t st) {
    return launch_subsweep_tpl<float, 12>(rect, mu, p, st);
}
cudaError_t launch_aus_f12(bool rect, int mu, const AusParams &p, cudaStream_t st) {
    return launch_aus_tpl<float, 12>(rect, mu, p, st);
}
}  // namespace vs
