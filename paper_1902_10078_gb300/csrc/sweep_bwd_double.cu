// bwd sweeps, double.
#include "sweep_launch.cuh"
#include "products.cuh"

namespace bnd {
template <>
cudaError_t launch_bwd<double>(const bnd_plan *p, int fl, int K, const SweepArgs<double> &A, cudaStream_t s) {
    return dispatch_bwd<double>(p, fl, K, A, s);
}
}  // namespace bnd
