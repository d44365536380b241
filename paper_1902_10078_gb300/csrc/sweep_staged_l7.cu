// Staged sweep kernels of bandwidth 7 (both dtypes, both directions).
#include "sweep_staged.cuh"

BND_STAGED_INSTANCES(7)
