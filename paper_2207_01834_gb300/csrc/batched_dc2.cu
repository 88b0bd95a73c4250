// Batched persistent kernels for dimension class 2.
#include "batched_kernel.cuh"
#include "internal.h"

PG_DEFINE_BATCHED_LAUNCH(2)
