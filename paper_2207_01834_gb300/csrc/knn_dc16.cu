// k-NN traversal kernels for dimension class 16.
#include "internal.h"
#include "knn_kernel.cuh"

PG_DEFINE_KNN_LAUNCH(16)
