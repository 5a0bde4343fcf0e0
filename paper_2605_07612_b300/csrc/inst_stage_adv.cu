// Explicit instantiations of kernel launchers (parallel build unit): the
// per-cell stage kernel for scalar advection (runtime limiter and flux) and
// the FP32 block kernel for the MUSCL limiters.
#include "launch_kernels.cuh"

namespace amrb {
AMR_INST_STAGE_PH(float, 2, true, 1)
AMR_INST_STAGE_PH(float, 3, true, 1)
AMR_INST_STAGE_PH(double, 2, true, 1)
AMR_INST_STAGE_PH(double, 3, true, 1)
template amr_status launch_adv_pair<2, 8>(amr_forest *, const StageArgs<float> &, cudaStream_t);
template amr_status launch_adv_pair<2, 16>(amr_forest *, const StageArgs<float> &, cudaStream_t);
template amr_status launch_adv_pair<2, 32>(amr_forest *, const StageArgs<float> &, cudaStream_t);
template amr_status launch_adv_pair<3, 8>(amr_forest *, const StageArgs<float> &, cudaStream_t);
template amr_status launch_adv_pair<3, 16>(amr_forest *, const StageArgs<float> &, cudaStream_t);
}  // namespace amrb
