// k_generic_d3.cu -- instantiations of the generic step kernel for D = 3.
#include "k_generic_step.cuh"

namespace lbmh {
cudaError_t step_generic_d3(const StepArgs &a, int blocks, int threads, cudaStream_t s) {
    switch (a.lat.P) {
    case lbmd::P_F64: return lbmd::launch_generic_dp<3, lbmd::P_F64>(a, blocks, threads, s);
    case lbmd::P_F32: return lbmd::launch_generic_dp<3, lbmd::P_F32>(a, blocks, threads, s);
    case lbmd::P_F16S: return lbmd::launch_generic_dp<3, lbmd::P_F16S>(a, blocks, threads, s);
    default: return cudaErrorInvalidValue;
    }
}
}  // namespace lbmh
