// Batched persistent kernels for dimension class 7.
#include "batched_kernel.cuh"
#include "internal.h"

PG_DEFINE_BATCHED_LAUNCH(7)
