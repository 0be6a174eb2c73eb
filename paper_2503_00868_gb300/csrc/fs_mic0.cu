// fs_mic0.cu -- MIC(0) preconditioner (placeholder until the wavefront solve lands).
#include "fs_internal.cuh"

namespace fs {

int mic0_factor(fs_ctx *c)
{
    (void)c;
    return set_error(FS_EINVAL, "MIC(0) preconditioner is not available in this build");
}

int mic0_apply(fs_ctx *c, const float *r, float *z)
{
    (void)c; (void)r; (void)z;
    return set_error(FS_EINVAL, "MIC(0) preconditioner is not available in this build");
}

}  // namespace fs
