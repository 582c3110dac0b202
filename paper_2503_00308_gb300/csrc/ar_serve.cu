// ar_serve.cu -- serving entry points (continuous batching of requests).
#include "ar.h"
#include "ar_host.h"

int ar_serve_create(int64_t, int32_t, ar_server **out)
{
    if (out) *out = nullptr;
    return AR_EINVAL;
}
int ar_serve_destroy(ar_server *) { return AR_EINVAL; }
int ar_serve_submit(ar_server *, ar_scene *, const ar_intrinsics *, const ar_nominal_pose *, const ar_pose_box *,
                    int32_t, float *, float *, uint64_t *)
{
    return AR_EINVAL;
}
int ar_serve_poll(ar_server *, uint64_t, int *, double *) { return AR_EINVAL; }
