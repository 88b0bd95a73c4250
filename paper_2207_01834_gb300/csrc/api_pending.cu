// Entry points whose kernels are not built yet: they report PG_EUNSUPPORTED.
#include "internal.h"

using namespace pg;

extern "C" {

pg_status pg_bdl_create(int dim, int64_t X, int leaf, void *, pg_bdl **out) {
    if (out) *out = nullptr;
    if (dim < 1 || dim > PG_MAX_DIM || X < 1 || leaf < 1 || leaf > PG_MAX_LEAF || !out)
        return fail(PG_EINVAL, "pg_bdl_create: invalid argument");
    return fail(PG_EUNSUPPORTED, "pg_bdl_create: not built");
}
pg_status pg_bdl_insert(pg_bdl *, const float *, int64_t, int32_t *) { return fail(PG_EUNSUPPORTED, "not built"); }
pg_status pg_bdl_erase(pg_bdl *, const float *, int64_t) { return fail(PG_EUNSUPPORTED, "not built"); }
pg_status pg_bdl_knn(const pg_bdl *, const float *, int64_t, int, int32_t *, float *) { return fail(PG_EUNSUPPORTED, "not built"); }
pg_status pg_bdl_size(const pg_bdl *, int64_t *) { return fail(PG_EUNSUPPORTED, "not built"); }
pg_status pg_bdl_structure(const pg_bdl *, uint64_t *, int64_t *, int64_t *, int64_t *) { return fail(PG_EUNSUPPORTED, "not built"); }
pg_status pg_bdl_slot_of(const pg_bdl *, int8_t *) { return fail(PG_EUNSUPPORTED, "not built"); }
pg_status pg_bdl_free(pg_bdl *) { return PG_OK; }
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
