// thin_serve.cu -- serving entry points (continuous batching).  Filled in below.
#include "thin_internal.h"

extern "C" {
int thin_serve_create(size_t, int, int, thin_server **out)
{
    if (out) *out = nullptr;
    return THIN_ERR_UNSUPPORTED;
}
int thin_serve_submit(thin_server *, const void *, int, int, size_t, thin_dtype, uint32_t, uint64_t *)
{
    return THIN_ERR_UNSUPPORTED;
}
int thin_serve_poll(thin_server *, uint64_t, void *, size_t, int *, thin_stats *) { return THIN_ERR_UNSUPPORTED; }
int thin_serve_destroy(thin_server *) { return THIN_ERR_UNSUPPORTED; }
}
