// Staged sweep kernels of bandwidth 8 (both dtypes, both directions).
#include "sweep_staged.cuh"

BND_STAGED_INSTANCES(8)
