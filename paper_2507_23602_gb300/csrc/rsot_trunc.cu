// Truncated evaluation (placeholder until the cell-list kernels land).
#include "rsot_internal.cuh"

namespace rsot {
cudaError_t trunc_eval(rsot_problem *, const double *, double, double, int, double *) {
    return cudaErrorNotSupported;
}
void trunc_free(rsot_problem *) {}
cudaError_t trunc_point_L(rsot_problem *, double *) { return cudaErrorNotSupported; }
}  // namespace rsot
