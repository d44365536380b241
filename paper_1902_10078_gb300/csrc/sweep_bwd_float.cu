// bwd sweeps, float.
#include "sweep_launch.cuh"
#include "products.cuh"

namespace bnd {
template <>
cudaError_t launch_bwd<float>(const bnd_plan *p, int fl, int K, const SweepArgs<float> &A, cudaStream_t s) {
    return dispatch_bwd<float>(p, fl, K, A, s);
}
}  // namespace bnd
