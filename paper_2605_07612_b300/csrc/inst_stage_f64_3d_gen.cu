// Explicit instantiations of kernel launchers (parallel build unit).
#include "launch_kernels.cuh"

namespace amrb {
AMR_INST_STAGE(double, 3, true)
}  // namespace amrb
