// FP64 arithmetic, 18-real link storage (the plain FP64 path).
#include "vs_sweep_inst.cuh"
namespace vs {
cudaError_t launch_subsweep_d18(bool rect, int mu, const SubsweepParams &p, cudaStream_t st) {
    return launch_subsweep_tpl<double, 18>(rect, mu, p, st);
}
cudaError_t launch_aus_d18(bool rect, int mu, const AusParams &p, cudaStream_t st) {
    return launch_aus_tpl<double, 18>(rect, mu, p, st);
}
}  // namespace vs
