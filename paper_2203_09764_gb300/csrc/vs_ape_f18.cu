// APE / AUS with unit circle projection and Runge-Kutta flow stages:
// FP32 arithmetic, 18-real link storage.
#include "vs_ape.cuh"
namespace vs {
cudaError_t launch_ape_f18(bool rect, int mu, const ApeParams &p, cudaStream_t st) {
    return launch_ape_tpl<float, 18>(rect, mu, p, st);
}
cudaError_t launch_flow_f18(bool rect, int mu, const FlowParams &p, cudaStream_t st) {
    return launch_flow_tpl<float, 18>(rect, mu, p, st);
}
}  // namespace vs
