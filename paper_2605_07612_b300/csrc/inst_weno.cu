// Explicit instantiations of kernel launchers (parallel build unit).
#include "launch_kernels.cuh"

namespace amrb {
template amr_status launch_weno<float, 2, 0>(amr_forest *, const StageArgs<float> &, float *, cudaStream_t);
template amr_status launch_weno<float, 3, 0>(amr_forest *, const StageArgs<float> &, float *, cudaStream_t);
template amr_status launch_weno<double, 2, 0>(amr_forest *, const StageArgs<double> &, double *, cudaStream_t);
template amr_status launch_weno<double, 3, 0>(amr_forest *, const StageArgs<double> &, double *, cudaStream_t);
template amr_status launch_weno<float, 2, 1>(amr_forest *, const StageArgs<float> &, float *, cudaStream_t);
template amr_status launch_weno<float, 3, 1>(amr_forest *, const StageArgs<float> &, float *, cudaStream_t);
template amr_status launch_weno<double, 2, 1>(amr_forest *, const StageArgs<double> &, double *, cudaStream_t);
template amr_status launch_weno<double, 3, 1>(amr_forest *, const StageArgs<double> &, double *, cudaStream_t);
}  // namespace amrb
