// Explicit instantiations of kernel launchers (parallel build unit).
#include "launch_kernels.cuh"

namespace amrb {
AMR_INST_STAGE(float, 2, true)
}  // namespace amrb
