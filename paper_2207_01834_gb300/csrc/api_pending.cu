// Entry points whose kernels are not built yet: they report PG_EUNSUPPORTED.
#include "internal.h"

using namespace pg;

extern "C" {

pg_status pg_knn_backward(const float *, int64_t, const float *, int64_t, int dim, int k, const int32_t *,
                          const float *, float *, float *, void *) {
    if (k < 1 || k > PG_MAX_K || dim < 1 || dim > PG_MAX_DIM) return fail(PG_EINVAL, "pg_knn_backward: invalid argument");
    return fail(PG_EUNSUPPORTED, "not built");
}
pg_status pg_batched_chamfer(const float *, const int64_t *, const float *, const int64_t *, int, int, int, int,
                             float *, int32_t *, int32_t *, float *, float *, void *) { return fail(PG_EUNSUPPORTED, "not built"); }
pg_status pg_batched_chamfer_backward(const float *, const int64_t *, const float *, const int64_t *, int, int, int,
                                      const int32_t *, const int32_t *, const float *, float *, float *, void *) {
    return fail(PG_EUNSUPPORTED, "not built");
}

}
