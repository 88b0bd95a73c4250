// Batched persistent kernels for dimension class 5.
#include "batched_kernel.cuh"
#include "internal.h"

PG_DEFINE_BATCHED_LAUNCH(5)
