// Staged sweep kernels of bandwidth 4 (both dtypes, both directions).
#include "sweep_staged.cuh"

BND_STAGED_INSTANCES(4)
