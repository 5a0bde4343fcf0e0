// Explicit instantiations of kernel launchers (parallel build unit).
#include "launch_kernels.cuh"

namespace amrb {
template amr_status launch_stage_pair<2, 8, 0>(amr_forest *, const StageArgs<float> &, cudaStream_t);
template amr_status launch_stage_pair<2, 16, 0>(amr_forest *, const StageArgs<float> &, cudaStream_t);
template amr_status launch_stage_pair<2, 32, 0>(amr_forest *, const StageArgs<float> &, cudaStream_t);
}  // namespace amrb
