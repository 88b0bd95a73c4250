// k-NN traversal kernels for dimension class 7.
#include "internal.h"
#include "knn_kernel.cuh"

PG_DEFINE_KNN_LAUNCH(7)
