// Mixed-precision path (tcgen05 tensor-core contraction): placeholder until
// the kernel lands; init rejects CUDISC_MIXED_TF32 with ENOTSUP meanwhile.
#include "coag_internal.h"

namespace cdc {
size_t mixed_workspace_bytes(int, int) { return 256; }
cudaError_t launch_rhs_mixed(const cudisc_coag_ctx *, const double *, double *)
{
    return cudaErrorNotSupported;
}
cudaError_t launch_step_mixed(const cudisc_coag_ctx *, double *, double, double *,
                              const double *, const long long *, long long)
{
    return cudaErrorNotSupported;
}
} // namespace cdc
