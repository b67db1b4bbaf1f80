// APE / AUS with unit circle projection and Runge-Kutta flow stages:
// FP64 arithmetic, 18-real link storage.
#include "vs_ape.cuh"
namespace vs {
cudaError_t launch_ape_d18(bool rect, int mu, const ApeParams &p, cudaStream_t st) {
    return launch_ape_tpl<double, 18>(rect, mu, p, st);
}
cudaError_t launch_flow_d18(bool rect, int mu, const FlowParams &p, cudaStream_t st) {
    return launch_flow_tpl<double, 18>(rect, mu, p, st);
}
}  // namespace vs
