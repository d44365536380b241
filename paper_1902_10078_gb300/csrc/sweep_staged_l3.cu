// Staged sweep kernels of bandwidth 3 (both dtypes, both directions).
#include "sweep_staged.cuh"

BND_STAGED_INSTANCES(3)
