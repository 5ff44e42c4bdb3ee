// Entry points whose kernels are not written yet: they refuse every call.
#include "host.hpp"

extern "C" boba_status_t boba_reorder_batched(const int32_t *, const int32_t *, const int64_t *,
                                              const int64_t *, int64_t, int64_t, int64_t, int64_t,
                                              int64_t, int32_t *, int32_t *, int32_t *, void *,
                                              size_t, void *)
{
    return BOBA_ERR_INVALID_ARG;
}
extern "C" size_t boba_reorder_batched_workspace_bytes(int64_t, int64_t, int64_t) { return 0; }
