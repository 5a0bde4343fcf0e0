// Explicit instantiations of kernel launchers (parallel build unit): the
// per-cell stage kernel for scalar advection (runtime limiter and flux).
#include "launch_kernels.cuh"

namespace amrb {
AMR_INST_STAGE_PH(float, 2, true, 1)
AMR_INST_STAGE_PH(float, 3, true, 1)
AMR_INST_STAGE_PH(double, 2, true, 1)
AMR_INST_STAGE_PH(double, 3, true, 1)
}  // namespace amrb
