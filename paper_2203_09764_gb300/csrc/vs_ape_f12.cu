// APE / AUS with unit circle projection and Runge-Kutta flow stages:
// FP32 arithmetic, 12-real link storage.
#include "vs_ape.cuh"
namespace vs {
cudaError_t launch_ape_f12(bool rect, int mu, const ApeParams &p, cudaStream_t st) {
    return launch_ape_tpl<float, 12>(rect, mu, p, st);
}
cudaError_t launch_flow_f12(bool rect, int mu, const FlowParams &p, cudaStream_t st) {
    return launch_flow_tpl<float, 12>(rect, mu, p, st);
}
}  // namespace vs
