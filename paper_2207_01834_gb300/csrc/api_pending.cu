// Entry points whose kernels are not built yet: they report PG_EUNSUPPORTED.
#include "internal.h"

using namespace pg;

extern "C" {

pg_status pg_batched_chamfer(const float *, const int64_t *, const float *, const int64_t *, int, int, int, int,
                             float *, int32_t *, int32_t *, float *, float *, void *) { return fail(PG_EUNSUPPORTED, "not built"); }
pg_status pg_batched_chamfer_backward(const float *, const int64_t *, const float *, const int64_t *, int, int, int,
                                      const int32_t *, const int32_t *, const float *, float *, float *, void *) {
    return fail(PG_EUNSUPPORTED, "not built");
}

}
