// Tensor-core (tcgen05) path: placeholder until the DFT-GEMM kernels land.
#include "dgfs_internal.h"

namespace dgfs {
dgfs_status tc_prepare(dgfs_plan_s *) { return DGFS_OK; }
void tc_release(dgfs_plan_s *) {}
size_t tc_workspace_bytes(const dgfs_plan_s *) { return 256; }
dgfs_status tc_collide(dgfs_plan_s *, int, const void *, void *, cudaStream_t)
{
    set_error("tensor-core path not built");
    return DGFS_EUNSUPPORTED;
}
}  // namespace dgfs
