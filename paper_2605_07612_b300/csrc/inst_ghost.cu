// Explicit instantiations of kernel launchers (parallel build unit).
#include "launch_kernels.cuh"

namespace amrb {
template amr_status launch_ghosts<float, 2>(amr_forest *, int, cudaStream_t, bool);
template amr_status launch_ghosts<float, 3>(amr_forest *, int, cudaStream_t, bool);
template amr_status launch_ghosts<double, 2>(amr_forest *, int, cudaStream_t, bool);
template amr_status launch_ghosts<double, 3>(amr_forest *, int, cudaStream_t, bool);
}  // namespace amrb
