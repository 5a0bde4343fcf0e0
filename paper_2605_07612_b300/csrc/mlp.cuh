// Learned refinement-flag predictor: a 3-layer MLP (F -> 64 -> 64 -> 3,
// GELU, softmax over derefine / keep / refine) whose forward pass uses BF16
// weights with FP32 accumulation.  Training kernels compute the mean
// cross-entropy gradient deterministically (per-CTA partial sums reduced in a
// fixed order) and apply AdamW to FP32 master weights.  The predictor stands
// in for the refinement criterion of Sec. 3.3 (Eq. 12), which stays as the
// fallback for low-confidence blocks and as the judge of its flags.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>
#include <string>

#include "common.cuh"
#include "pattern.hpp"

namespace amrb {

constexpr int kMlpH = 64, kMlpO = 3, kMlpMaxF = 256, kMlpTile = 64;

struct MlpLayout {
    int F;
    int64_t w1, b1, w2, b2, w3, b3, n;
    __host__ __device__ explicit MlpLayout(int F_) : F(F_) {
        w1 = 0;
        b1 = w1 + int64_t(F) * kMlpH;
        w2 = b1 + kMlpH;
        b2 = w2 + kMlpH * kMlpH;
        w3 = b2 + kMlpH;
        b3 = w3 + kMlpH * kMlpO;
        n = b3 + kMlpO;
    }
};

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_prime_f(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// BF16 parameters -> FP32 in shared memory
__device__ __forceinline__ void load_params(const __nv_bfloat16 *wb, int64_t n, float *sw) {
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) sw[i] = __bfloat162float(wb[i]);
}

// forward pass of one sample (feature-major input x[k * stride + s]):
// z1, z2 pre-activations, returns softmax probabilities
__device__ __forceinline__ void mlp_sample(const float *sw, const MlpLayout &L, const float *x, int64_t stride, int64_t s,
                                           float *z1, float *z2, float *prob) {
#pragma unroll
    for (int j = 0; j < kMlpH; ++j) z1[j] = sw[L.b1 + j];
    for (int k = 0; k < L.F; ++k) {
        const float xk = x[k * stride + s];
        const float *w = sw + L.w1 + int64_t(k) * kMlpH;
#pragma unroll
        for (int j = 0; j < kMlpH; ++j) z1[j] = fmaf(xk, w[j], z1[j]);
    }
#pragma unroll
    for (int j = 0; j < kMlpH; ++j) z2[j] = sw[L.b2 + j];
#pragma unroll
    for (int i = 0; i < kMlpH; ++i) {
        const float hi = gelu_f(z1[i]);
        const float *w = sw + L.w2 + i * kMlpH;
#pragma unroll
        for (int j = 0; j < kMlpH; ++j) z2[j] = fmaf(hi, w[j], z2[j]);
    }
    float z3[kMlpO];
#pragma unroll
    for (int o = 0; o < kMlpO; ++o) z3[o] = sw[L.b3 + o];
#pragma unroll
    for (int i = 0; i < kMlpH; ++i) {
        const float hi = gelu_f(z2[i]);
#pragma unroll
        for (int o = 0; o < kMlpO; ++o) z3[o] = fmaf(hi, sw[L.w3 + i * kMlpO + o], z3[o]);
    }
    const float m = fmaxf(z3[0], fmaxf(z3[1], z3[2]));
    float e[kMlpO], sum = 0.f;
#pragma unroll
    for (int o = 0; o < kMlpO; ++o) {
        e[o] = expf(z3[o] - m);
        sum += e[o];
    }
#pragma unroll
    for (int o = 0; o < kMlpO; ++o) prob[o] = e[o] / sum;
}

// probabilities of n samples: x [F][n] -> prob [n][3]
static __global__ void __launch_bounds__(128) k_mlp_forward(const __nv_bfloat16 *wb, int F, const float *x, int64_t n, float *prob) {
    extern __shared__ float sw[];
    const MlpLayout L(F);
    load_params(wb, L.n, sw);
    __syncthreads();
    for (int64_t s = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; s < n; s += int64_t(gridDim.x) * blockDim.x) {
        float z1[kMlpH], z2[kMlpH], p[kMlpO];
        mlp_sample(sw, L, x, n, s, z1, z2, p);
#pragma unroll
        for (int o = 0; o < kMlpO; ++o) prob[s * kMlpO + o] = p[o];
    }
}

// Gradient of the mean cross-entropy over a batch (sample indices idx[0..nb)
// into x [F][n_total] and labels y, classes 0..2).  The CTA takes tiles of
// 64 samples: one thread per sample runs the forward and backward passes
// into shared memory, then all threads add the tile's outer products to
// this CTA's row of `partial` ([gridDim][P + 1], last entry = loss).
static __global__ void __launch_bounds__(128) k_mlp_grad(const __nv_bfloat16 *wb, int F, const float *x, int64_t n_total,
                                                  const int32_t *idx, const int8_t *y, int64_t nb, float *partial) {
    extern __shared__ float sm[];
    const MlpLayout L(F);
    float *sw = sm;                                   // params [P]
    float *xs = sw + ((L.n + 3) & ~int64_t(3));       // [F][64]
    float *h1 = xs + int64_t(F) * kMlpTile;           // [64][64] activations, sample-major
    float *h2 = h1 + kMlpTile * kMlpH;
    float *d1 = h2 + kMlpTile * kMlpH;                // [64][64] deltas
    float *d2 = d1 + kMlpTile * kMlpH;
    float *d3 = d2 + kMlpTile * kMlpH;                // [64][3]
    load_params(wb, L.n, sw);
    float *row = partial + int64_t(blockIdx.x) * (L.n + 1);
    const float inv_nb = 1.0f / float(nb);
    float my_loss = 0.f;
    __syncthreads();
    const int64_t ntiles = (nb + kMlpTile - 1) / kMlpTile;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t s0 = t * kMlpTile;
        for (int i = threadIdx.x; i < F * kMlpTile; i += blockDim.x) {
            const int k = i / kMlpTile, s = i % kMlpTile;
            xs[i] = (s0 + s < nb) ? x[int64_t(k) * n_total + idx[s0 + s]] : 0.f;
        }
        __syncthreads();
        if (threadIdx.x < kMlpTile) {
            const int s = threadIdx.x;
            float z1[kMlpH], z2[kMlpH], p[kMlpO];
            mlp_sample(sw, L, xs, kMlpTile, s, z1, z2, p);
            const bool valid = s0 + s < nb;
            float e3[kMlpO];
            const int lab = valid ? min(max(int(y[idx[s0 + s]]), 0), kMlpO - 1) : 0;   // classes 0..2
#pragma unroll
            for (int o = 0; o < kMlpO; ++o) e3[o] = valid ? (p[o] - (o == lab ? 1.f : 0.f)) * inv_nb : 0.f;
            if (valid) my_loss -= logf(p[lab]) * inv_nb;
#pragma unroll
            for (int o = 0; o < kMlpO; ++o) d3[s * kMlpO + o] = e3[o];
            // layer 3 -> 2
#pragma unroll
            for (int j = 0; j < kMlpH; ++j) {
                float g = 0.f;
#pragma unroll
                for (int o = 0; o < kMlpO; ++o) g = fmaf(sw[L.w3 + j * kMlpO + o], e3[o], g);
                d2[s * kMlpH + j] = g * gelu_prime_f(z2[j]);
                h2[s * kMlpH + j] = gelu_f(z2[j]);
            }
            // layer 2 -> 1
#pragma unroll
            for (int i = 0; i < kMlpH; ++i) {
                float g = 0.f;
                const float *w = sw + L.w2 + i * kMlpH;
                for (int j = 0; j < kMlpH; ++j) g = fmaf(w[j], d2[s * kMlpH + j], g);
                d1[s * kMlpH + i] = g * gelu_prime_f(z1[i]);
                h1[s * kMlpH + i] = gelu_f(z1[i]);
            }
        }
        __syncthreads();
        // tile contributions: outer products summed over the tile's samples
        for (int64_t q = threadIdx.x; q < L.n; q += blockDim.x) {
            float acc = 0.f;
            if (q < L.b1) {
                const int k = int(q / kMlpH), j = int(q % kMlpH);
                for (int s = 0; s < kMlpTile; ++s) acc = fmaf(xs[k * kMlpTile + s], d1[s * kMlpH + j], acc);
            } else if (q < L.w2) {
                const int j = int(q - L.b1);
                for (int s = 0; s < kMlpTile; ++s) acc += d1[s * kMlpH + j];
            } else if (q < L.b2) {
                const int i = int((q - L.w2) / kMlpH), j = int((q - L.w2) % kMlpH);
                for (int s = 0; s < kMlpTile; ++s) acc = fmaf(h1[s * kMlpH + i], d2[s * kMlpH + j], acc);
            } else if (q < L.w3) {
                const int j = int(q - L.b2);
                for (int s = 0; s < kMlpTile; ++s) acc += d2[s * kMlpH + j];
            } else if (q < L.b3) {
                const int i = int((q - L.w3) / kMlpO), o = int((q - L.w3) % kMlpO);
                for (int s = 0; s < kMlpTile; ++s) acc = fmaf(h2[s * kMlpH + i], d3[s * kMlpO + o], acc);
            } else {
                const int o = int(q - L.b3);
                for (int s = 0; s < kMlpTile; ++s) acc += d3[s * kMlpO + o];
            }
            row[q] += acc;
        }
        __syncthreads();
    }
    // loss of this CTA's samples (threads < 64 hold them), fixed-order tree
    __shared__ float red[128];
    red[threadIdx.x] = my_loss;
    __syncthreads();
    for (int w = 64; w > 0; w >>= 1) {
        if (int(threadIdx.x) < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) row[L.n] += red[0];
}

// grad[q] = sum over CTA rows of partial[c][q] in row order (q <= P: loss)
static __global__ void k_mlp_reduce(const float *partial, int rows, int64_t n1, float *grad) {
    for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < n1; q += int64_t(gridDim.x) * blockDim.x) {
        float s = 0.f;
        for (int c = 0; c < rows; ++c) s += partial[int64_t(c) * n1 + q];
        grad[q] = s;
    }
}

// AdamW on FP32 master weights, then their BF16 copy
static __global__ void k_adamw(float *w, float *m, float *v, __nv_bfloat16 *wb, const float *g, int64_t n, float lr, float b1, float b2,
                        float eps, float wd, float c1, float c2) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float mh = mi / c1, vh = vi / c2;
        const float wi = w[i] - lr * (mh / (sqrtf(vh) + eps) + wd * w[i]);
        w[i] = wi;
        wb[i] = __float2bfloat16_rn(wi);
    }
}

static __global__ void k_to_bf16(const float *w, __nv_bfloat16 *wb, int64_t n) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        wb[i] = __float2bfloat16_rn(w[i]);
}

// per block: class with the largest probability and whether it is confident
static __global__ void k_mlp_decide(const float *prob, int64_t n, float tau, int8_t *flags) {
    for (int64_t b = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; b < n; b += int64_t(gridDim.x) * blockDim.x) {
        const float *p = prob + b * kMlpO;
        int c = 0;
        if (p[1] > p[c]) c = 1;
        if (p[2] > p[c]) c = 2;
        flags[b] = p[c] >= tau ? int8_t(c - 1) : int8_t(2);   // 2: not confident
    }
}

// Block features: 4^d average pools of density, pressure and speed (density
// and pressure over the block mean, minus one; speed over the sound speed of
// the block-mean state) and level / max_level, written feature-major
// x[f * nb + b].  Pool t = px + 4 (py + 4 pz).
//
// One CTA of 256 threads per block (N is 8, 16 or 32).  Cells are visited
// x fastest so that a warp reads whole rows; density, pressure and speed of a
// cell are formed in the state's precision, summed over the q = N/4 cells of
// a pool row by a butterfly within q lanes (every lane of the group ends with
// the same sum), and the row sums go to shared memory.  One thread per (pool,
// quantity) then adds its q^(d-1) rows in a fixed order in double, and the
// block means are the fixed-order sums of the pools: the features do not
// depend on scheduling.
template <class real, int D>
__host__ __device__ constexpr size_t features_smem(int N) {
    return size_t(3) * size_t(D == 3 ? N * N : N) * 4 * sizeof(real);
}

template <class real, int D>
__global__ void __launch_bounds__(256) k_features(const real *u, const BlockInfo *info, Geom g, double gam, float inv_levels,
                                                  float *x, int64_t nb) {
    extern __shared__ double feat_sm[];
    __shared__ double pools[3][64];
    real *rowp = reinterpret_cast<real *>(feat_sm);  // [3][rows][4]
    const int b = blockIdx.x, t = threadIdx.x;
    const int N = g.N, q = N / 4;
    const int rows = D == 3 ? N * N : N, ncell = rows * N;
    const int npool = D == 3 ? 64 : 16;
    const real *ub = u + int64_t(b) * g.bstride;
    const real gm1 = real(gam - 1.0);
    for (int c = t; c < ncell; c += blockDim.x) {  // ncell is a multiple of 32: whole warps iterate
        const int i = c % N, row = c / N;
        const int64_t ci = cell_index<real>(g, i, row % N, D == 3 ? row / N : 0);
        const real rho = ub[ci];
        const real inv = real(1) / rho;
        real ke = real(0);
        for (int d = 0; d < D; ++d) {
            const real w = ub[int64_t(1 + d) * g.ncell + ci] * inv;
            ke += w * w;
        }
        real r = rho;
        real pr = gm1 * (ub[int64_t(D + 1) * g.ncell + ci] - real(0.5) * rho * ke);
        real sp = sqrt(ke);
        for (int o = 1; o < q; o <<= 1) {
            r += __shfl_xor_sync(0xffffffffu, r, o);
            pr += __shfl_xor_sync(0xffffffffu, pr, o);
            sp += __shfl_xor_sync(0xffffffffu, sp, o);
        }
        if (i % q == 0) {
            rowp[(0 * rows + row) * 4 + i / q] = r;
            rowp[(1 * rows + row) * 4 + i / q] = pr;
            rowp[(2 * rows + row) * 4 + i / q] = sp;
        }
    }
    __syncthreads();
    if (t < 3 * npool) {
        const int v = t / npool, pl = t % npool;
        const int px = pl % 4, py = (pl / 4) % 4, pz = D == 3 ? pl / 16 : 0;
        double acc = 0.0;
        for (int kk = 0; kk < (D == 3 ? q : 1); ++kk)
            for (int jj = 0; jj < q; ++jj) {
                const int row = D == 3 ? (pz * q + kk) * N + py * q + jj : py * q + jj;
                acc += double(rowp[(v * rows + row) * 4 + px]);
            }
        pools[v][pl] = acc;
    }
    __syncthreads();
    if (t < npool) {
        double sr = 0.0, sp = 0.0;
        for (int l = 0; l < npool; ++l) {
            sr += pools[0][l];
            sp += pools[1][l];
        }
        const double cells = double(D == 3 ? q * q * q : q * q);
        const double rm = sr / double(ncell), pm = sp / double(ncell);
        const double cm = sqrt(gam * pm / rm);
        x[int64_t(t) * nb + b] = float((pools[0][t] / cells) / rm - 1.0);
        x[int64_t(npool + t) * nb + b] = float((pools[1][t] / cells) / pm - 1.0);
        x[int64_t(2 * npool + t) * nb + b] = float((pools[2][t] / cells) / cm);
    }
    if (t == 0) x[int64_t(3 * npool) * nb + b] = float(info[b].level) * inv_levels;
}

}  // namespace amrb

// the model object of the C ABI
struct amr_mlp {
    int F = 0;
    int64_t P = 0;
    float *w = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr, *partial = nullptr;
    __nv_bfloat16 *wb = nullptr;
    int32_t *idx = nullptr;
    int64_t idx_cap = 0;
    int partial_rows = 0;
    int64_t step = 0;
    int precision = 16;   // 16: BF16 tensor-core kernels, 32: FP32 CUDA-core kernels
    std::string err;
};
