// Allocation-free variant of the conserved-integral reduction.
//
// Some callers cannot call cudaMalloc at the point where they need the
// conserved sums: their device memory is fully reserved up front by another
// allocator (a framework's caching pool or a fixed arena), or they must not
// trigger the device-wide synchronisation that cudaMalloc/cudaFree may cause.
// amr_conserved_static() serves them: the caller passes the block data and
// the output, and the per-block partial sums go to a fixed-size scratch array
// that lives in this library's device image (every GPU that loads the library
// holds it until the process exits).  No memory is allocated by the call.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/amr.h"

namespace {

constexpr int64_t kStaticMaxBlocks = AMR_STATIC_MAX_BLOCKS;
constexpr int kStaticMaxVars = 5;
// Per-block, per-variable partial sums.  Each call overwrites the entries it
// uses before reading them, so nothing has to be cleared between calls.
static __device__ __align__(256) double g_partials[kStaticMaxBlocks * kStaticMaxVars];

template <class real, int D>
__global__ void __launch_bounds__(256) k_static_block(const real *u, int N, int ng, const double *vol, double *partial) {
    __shared__ double red[256];
    const int b = blockIdx.x;
    const int V = D + 2, S = N + 2 * ng;
    const int64_t ncellg = (D == 3) ? int64_t(S) * S * S : int64_t(S) * S;
    const int ncell = (D == 3) ? N * N * N : N * N;
    for (int v = 0; v < V; ++v) {
        const real *ub = u + (int64_t(b) * V + v) * ncellg;
        double s = 0.0;
        for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
            const int i = c % N, j = (c / N) % N, k = (D == 3) ? c / (N * N) : 0;
            const int64_t kk = (D == 3) ? int64_t(k + ng) * S : 0;
            s += double(ub[(kk + (j + ng)) * S + (i + ng)]);
        }
        red[threadIdx.x] = s;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[int64_t(b) * V + v] = red[0] * vol[b];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(1024) k_static_final(const double *partial, int64_t nb, int V, double *out) {
    __shared__ double red[1024];
    for (int v = 0; v < V; ++v) {
        double s = 0.0;
        for (int64_t b = threadIdx.x; b < nb; b += blockDim.x) s += partial[b * V + v];
        red[threadIdx.x] = s;
        __syncthreads();
        for (int w = 512; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[v] = red[0];
        __syncthreads();
    }
}

// Device address of the scratch array on the current device.  Looked up on
// every call (a host-side lookup once the library's device code is loaded):
// a cached address would go stale after cudaDeviceReset or when the device
// gets a new primary context in the same process.  The first lookup on a
// device loads the library's device code there.
amr_status scratch_address(double **out) {
    double *p = nullptr;
    if (cudaGetSymbolAddress((void **)&p, g_partials) != cudaSuccess || !p) {
        cudaGetLastError();
        return AMR_ECUDA;
    }
    *out = p;
    return AMR_OK;
}

template <class real, int D>
amr_status run(const void *state, int N, int ng, int64_t nb, const double *vol, double *sums, cudaStream_t st) {
    double *scratch = nullptr;
    amr_status s = scratch_address(&scratch);
    if (s != AMR_OK) return s;
    if (nb > 0) k_static_block<real, D><<<unsigned(nb), 256, 0, st>>>(static_cast<const real *>(state), N, ng, vol, scratch);
    k_static_final<<<1, 1024, 0, st>>>(scratch, nb, D + 2, sums);
    if (cudaGetLastError() != cudaSuccess) return AMR_ECUDA;
    return AMR_OK;
}

}  // namespace

extern "C" amr_status amr_conserved_static(const void *state, int precision, int ndim, int block_n, int n_ghost,
                                           int64_t n_blocks, const double *cell_volume, double *sums, amr_stream stream) {
    if (!state || !cell_volume || !sums || n_blocks < 0) return AMR_EINVAL;
    if (precision != 32 && precision != 64) return AMR_EINVAL;
    if ((ndim != 2 && ndim != 3) || block_n < 2 || (block_n & 1) || n_ghost < 1 || block_n < 2 * n_ghost) return AMR_EINVAL;
    if (n_blocks > kStaticMaxBlocks) return AMR_ECAPACITY;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (precision == 64)
        return ndim == 3 ? run<double, 3>(state, block_n, n_ghost, n_blocks, cell_volume, sums, st)
                         : run<double, 2>(state, block_n, n_ghost, n_blocks, cell_volume, sums, st);
    return ndim == 3 ? run<float, 3>(state, block_n, n_ghost, n_blocks, cell_volume, sums, st)
                     : run<float, 2>(state, block_n, n_ghost, n_blocks, cell_volume, sums, st);
}
