// Batched persistent kernels for dimension class 12.
#include "batched_kernel.cuh"
#include "internal.h"

PG_DEFINE_BATCHED_LAUNCH(12)
