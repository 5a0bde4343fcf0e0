// Explicit instantiations of kernel launchers (parallel build unit).
#include "launch_kernels.cuh"

namespace amrb {
template amr_status launch_stage_pair<2, 8, 1>(amr_forest *, const StageArgs<float> &, cudaStream_t);
template amr_status launch_stage_pair<2, 16, 1>(amr_forest *, const StageArgs<float> &, cudaStream_t);
template amr_status launch_stage_pair<2, 32, 1>(amr_forest *, const StageArgs<float> &, cudaStream_t);
}  // namespace amrb
