// Tensor-core forms of the learned refinement-flag predictor (the network of
// mlp.cuh): the products x W1, h1 W2, h2 W3 and, in training, the
// back-propagated deltas and the weight gradients run as BF16 x BF16 -> FP32
// warp-level matrix multiply-accumulates (mma.sync m16n8k16).  Operands are
// rounded to BF16 (round to nearest even) where they enter a product:
// features, activations h1 and h2, and the deltas d1, d2 of the hidden
// layers; accumulation, biases, GELU, softmax and the output-layer delta stay
// in FP32.
//
// Fragment layouts of m16n8k16 (g = lane / 4, t = lane % 4):
//   A (16 x 16, row): a0 = A[g][2t..2t+1], a1 = A[g+8][2t..], a2 = A[g][2t+8..],
//                     a3 = A[g+8][2t+8..]      (two BF16 per 32-bit register)
//   B (16 x 8, col):  b0 = B[2t..2t+1][g],     b1 = B[2t+8..2t+9][g]
//   C (16 x 8, FP32): c0, c1 = C[g][2t..2t+1], c2, c3 = C[g+8][2t..2t+1]
// so the C fragments of two adjacent 8-column tiles are the A fragment of a
// 16-wide K step of the next product.  Shared-memory operands are laid out
// with their K index contiguous and rows padded by 8 elements (16 bytes):
// the 8 rows an ldmatrix reads then fall into distinct 16-byte bank groups.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

#include "mlp.cuh"

namespace amrb {

constexpr int kTcTile = 64;          // samples per CTA tile (4 warps x 16)
constexpr int kTcPadS = kTcTile + 8; // row pitch of sample-contiguous operands
constexpr int kTcPadH = kMlpH + 8;   // row pitch of hidden-contiguous operands

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// four 8x8 BF16 matrices; lane L gives the address of row L % 8 of matrix L / 8
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void *row_addr) {
    const unsigned s = unsigned(__cvta_generic_to_shared(row_addr));
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(s));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void *row_addr) {
    const unsigned s = unsigned(__cvta_generic_to_shared(row_addr));
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(s));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// A fragment (16 rows x 16 K) from a K-major array Kt[k][m] (row pitch p
// elements): rows m0.., K k0..  Matrix i of the x4.trans load covers K rows
// k0 + 8 (i >> 1) .. and M columns m0 + 8 (i & 1) ..
__device__ __forceinline__ void a_frag_kmajor(uint32_t (&a)[4], const __nv_bfloat16 *Kt, int p, int k0, int m0, int lane) {
    const int i = lane >> 3, r = lane & 7;
    ldsm_x4_t(a, Kt + (k0 + r + 8 * (i >> 1)) * p + m0 + 8 * (i & 1));
}
// A fragment from an M-major array Am[m][k] (row pitch p): matrix i covers
// rows m0 + 8 (i & 1) .. and K columns k0 + 8 (i >> 1) ..
__device__ __forceinline__ void a_frag_mmajor(uint32_t (&a)[4], const __nv_bfloat16 *Am, int p, int m0, int k0, int lane) {
    const int i = lane >> 3, r = lane & 7;
    ldsm_x4(a, Am + (m0 + r + 8 * (i & 1)) * p + k0 + 8 * (i >> 1));
}
// B fragments of two 8-column tiles (n0 .. n0+15) for one K step from an
// N-major array Bn[n][k] (row pitch p): b[0], b[1] tile n0, b[2], b[3] tile n0+8
__device__ __forceinline__ void b_frag2(uint32_t (&b)[4], const __nv_bfloat16 *Bn, int p, int n0, int k0, int lane) {
    const int i = lane >> 3, r = lane & 7;
    ldsm_x4(b, Bn + (n0 + r + 8 * (i >> 1)) * p + k0 + 8 * (i & 1));
}

// Shared-memory layout of the tensor-core kernels (BF16 elements unless noted)
struct TcSmem {
    int F, KP;
    size_t w1t, w2t, w2n, w3t, xt, b1, b2, b3, end;   // byte offsets
    __host__ __device__ explicit TcSmem(int F_) : F(F_), KP((F_ + 15) & ~15) {
        size_t o = 0;
        w1t = o; o += size_t(kMlpH) * (KP + 8) * 2;        // W1 transposed [j][f]
        w2t = o; o += size_t(kMlpH) * kTcPadH * 2;         // W2 transposed [j][i]
        w2n = o; o += size_t(kMlpH) * kTcPadH * 2;         // W2 as stored [i][j]
        w3t = o; o += size_t(8) * kTcPadH * 2;             // W3 transposed [o][j], rows 3..7 zero
        xt = o; o += size_t(KP) * kTcPadS * 2;             // features [f][s] of the tile
        b1 = o; o += sizeof(float) * kMlpH;
        b2 = o; o += sizeof(float) * kMlpH;
        b3 = o; o += sizeof(float) * 8;
        end = (o + 15) & ~size_t(15);
    }
};

// weights (BF16, packed as in MlpLayout) into the tensor-core layouts
__device__ __forceinline__ void tc_load_weights(const __nv_bfloat16 *wb, const MlpLayout &L, unsigned char *sm, const TcSmem &T) {
    __nv_bfloat16 *w1t = reinterpret_cast<__nv_bfloat16 *>(sm + T.w1t);
    __nv_bfloat16 *w2t = reinterpret_cast<__nv_bfloat16 *>(sm + T.w2t);
    __nv_bfloat16 *w2n = reinterpret_cast<__nv_bfloat16 *>(sm + T.w2n);
    __nv_bfloat16 *w3t = reinterpret_cast<__nv_bfloat16 *>(sm + T.w3t);
    float *b1 = reinterpret_cast<float *>(sm + T.b1), *b2 = reinterpret_cast<float *>(sm + T.b2), *b3 = reinterpret_cast<float *>(sm + T.b3);
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
    for (int e = threadIdx.x; e < kMlpH * T.KP; e += blockDim.x) {
        const int j = e / T.KP, f = e - j * T.KP;
        w1t[j * (T.KP + 8) + f] = f < L.F ? wb[L.w1 + int64_t(f) * kMlpH + j] : zero;
    }
    for (int e = threadIdx.x; e < kMlpH * kMlpH; e += blockDim.x) {
        const int i = e / kMlpH, j = e - i * kMlpH;
        w2n[i * kTcPadH + j] = wb[L.w2 + e];
        w2t[j * kTcPadH + i] = wb[L.w2 + e];
    }
    for (int e = threadIdx.x; e < 8 * kMlpH; e += blockDim.x) {
        const int o = e / kMlpH, j = e - o * kMlpH;
        w3t[o * kTcPadH + j] = o < kMlpO ? wb[L.w3 + j * kMlpO + o] : zero;
    }
    for (int e = threadIdx.x; e < kMlpH; e += blockDim.x) {
        b1[e] = __bfloat162float(wb[L.b1 + e]);
        b2[e] = __bfloat162float(wb[L.b2 + e]);
    }
    if (threadIdx.x < 8) b3[threadIdx.x] = threadIdx.x < kMlpO ? __bfloat162float(wb[L.b3 + threadIdx.x]) : 0.f;
}

// features of samples idx(s0 + s), s < kTcTile, as BF16 into xt [f][s]
// (zero beyond the sample count; rows F .. KP-1 zero)
template <class Idx>
__device__ __forceinline__ void tc_load_tile(const float *x, int64_t n_total, int64_t s0, int64_t ns, Idx idx, unsigned char *sm,
                                             const TcSmem &T) {
    __nv_bfloat16 *xt = reinterpret_cast<__nv_bfloat16 *>(sm + T.xt);
    for (int e = threadIdx.x; e < T.KP * kTcTile; e += blockDim.x) {
        const int f = e / kTcTile, s = e - f * kTcTile;
        float v = 0.f;
        if (f < T.F && s0 + s < ns) v = x[int64_t(f) * n_total + idx(s0 + s)];
        xt[f * kTcPadS + s] = __float2bfloat16_rn(v);
    }
}

// Forward pass of the warp's 16 samples (tile rows 16 w ..): z1, z2 (FP32
// pre-activations of the hidden layers, C fragments of eight 8-column tiles)
// and the output logits z3 (one C fragment, columns 0..2 valid).
__device__ __forceinline__ void tc_forward_warp(const unsigned char *sm, const TcSmem &T, int lane, int m0, float (&z1)[8][4],
                                                float (&z2)[8][4], float (&z3)[4]) {
    const __nv_bfloat16 *w1t = reinterpret_cast<const __nv_bfloat16 *>(sm + T.w1t);
    const __nv_bfloat16 *w2t = reinterpret_cast<const __nv_bfloat16 *>(sm + T.w2t);
    const __nv_bfloat16 *w3t = reinterpret_cast<const __nv_bfloat16 *>(sm + T.w3t);
    const __nv_bfloat16 *xt = reinterpret_cast<const __nv_bfloat16 *>(sm + T.xt);
    const float *b1 = reinterpret_cast<const float *>(sm + T.b1), *b2 = reinterpret_cast<const float *>(sm + T.b2);
    const float *b3 = reinterpret_cast<const float *>(sm + T.b3);
    const int t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        z1[nt][0] = z1[nt][2] = b1[8 * nt + 2 * t];
        z1[nt][1] = z1[nt][3] = b1[8 * nt + 2 * t + 1];
        z2[nt][0] = z2[nt][2] = b2[8 * nt + 2 * t];
        z2[nt][1] = z2[nt][3] = b2[8 * nt + 2 * t + 1];
    }
    z3[0] = z3[2] = b3[2 * t];
    z3[1] = z3[3] = b3[2 * t + 1];
    // layer 1: [16 x KP] x [KP x 64]
    for (int k0 = 0; k0 < T.KP; k0 += 16) {
        uint32_t a[4];
        a_frag_kmajor(a, xt, kTcPadS, k0, m0, lane);
#pragma unroll
        for (int np = 0; np < 4; ++np) {
            uint32_t b[4];
            b_frag2(b, w1t, T.KP + 8, 16 * np, k0, lane);
            mma_bf16(z1[2 * np], a, b[0], b[1]);
            mma_bf16(z1[2 * np + 1], a, b[2], b[3]);
        }
    }
    // layer 2: GELU(z1) as the A operand, [16 x 64] x [64 x 64]
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
        uint32_t a[4];
        a[0] = pack_bf16(gelu_f(z1[2 * ks][0]), gelu_f(z1[2 * ks][1]));
        a[1] = pack_bf16(gelu_f(z1[2 * ks][2]), gelu_f(z1[2 * ks][3]));
        a[2] = pack_bf16(gelu_f(z1[2 * ks + 1][0]), gelu_f(z1[2 * ks + 1][1]));
        a[3] = pack_bf16(gelu_f(z1[2 * ks + 1][2]), gelu_f(z1[2 * ks + 1][3]));
#pragma unroll
        for (int np = 0; np < 4; ++np) {
            uint32_t b[4];
            b_frag2(b, w2t, kTcPadH, 16 * np, 16 * ks, lane);
            mma_bf16(z2[2 * np], a, b[0], b[1]);
            mma_bf16(z2[2 * np + 1], a, b[2], b[3]);
        }
    }
    // layer 3: GELU(z2) x W3 (8 output columns, 3 used)
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
        uint32_t a[4];
        a[0] = pack_bf16(gelu_f(z2[2 * ks][0]), gelu_f(z2[2 * ks][1]));
        a[1] = pack_bf16(gelu_f(z2[2 * ks][2]), gelu_f(z2[2 * ks][3]));
        a[2] = pack_bf16(gelu_f(z2[2 * ks + 1][0]), gelu_f(z2[2 * ks + 1][1]));
        a[3] = pack_bf16(gelu_f(z2[2 * ks + 1][2]), gelu_f(z2[2 * ks + 1][3]));
        // B of 8 columns: matrices 0, 1 of a x4 load over rows 0..7 (K 0-7, 8-15)
        const int i = lane >> 3, r = lane & 7;
        uint32_t b[4];
        ldsm_x4(b, w3t + r * kTcPadH + 16 * ks + 8 * (i & 1));
        mma_bf16(z3, a, b[0], b[1]);
    }
}

// softmax of the three logits of rows g and g + 8 of the warp's fragment;
// every lane of a quad ends with both rows' probabilities
__device__ __forceinline__ void tc_softmax(const float (&z3)[4], int lane, float (&p0)[3], float (&p8)[3]) {
    const int q = lane & ~3;
    float l0[3], l8[3];
    l0[0] = __shfl_sync(0xffffffffu, z3[0], q);
    l0[1] = __shfl_sync(0xffffffffu, z3[1], q);
    l0[2] = __shfl_sync(0xffffffffu, z3[0], q + 1);
    l8[0] = __shfl_sync(0xffffffffu, z3[2], q);
    l8[1] = __shfl_sync(0xffffffffu, z3[3], q);
    l8[2] = __shfl_sync(0xffffffffu, z3[2], q + 1);
    auto sm3 = [](const float (&l)[3], float (&p)[3]) {
        const float m = fmaxf(l[0], fmaxf(l[1], l[2]));
        float e[3], s = 0.f;
#pragma unroll
        for (int o = 0; o < 3; ++o) {
            e[o] = expf(l[o] - m);
            s += e[o];
        }
#pragma unroll
        for (int o = 0; o < 3; ++o) p[o] = e[o] / s;
    };
    sm3(l0, p0);
    sm3(l8, p8);
}

// probabilities of n samples x [F][n] -> prob [n][3] on tensor cores
static __global__ void __launch_bounds__(128) k_mlp_forward_tc(const __nv_bfloat16 *wb, int F, const float *x, int64_t n, float *prob) {
    extern __shared__ __align__(16) unsigned char tc_smem[];
    unsigned char *sm = tc_smem;
    const MlpLayout L(F);
    const TcSmem T(F);
    tc_load_weights(wb, L, sm, T);
    const int lane = threadIdx.x & 31, m0 = 16 * (threadIdx.x >> 5), g = lane >> 2;
    const int64_t ntiles = (n + kTcTile - 1) / kTcTile;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t s0 = tile * kTcTile;
        __syncthreads();   // the previous tile's features are consumed (and the weights are in place)
        tc_load_tile(x, n, s0, n, [](int64_t s) { return s; }, sm, T);
        __syncthreads();
        float z1[8][4], z2[8][4], z3[4], p0[3], p8[3];
        tc_forward_warp(sm, T, lane, m0, z1, z2, z3);
        tc_softmax(z3, lane, p0, p8);
        if ((lane & 3) == 0) {
            const int64_t sa = s0 + m0 + g, sb = sa + 8;
#pragma unroll
            for (int o = 0; o < 3; ++o) {
                if (sa < n) prob[sa * kMlpO + o] = p0[o];
                if (sb < n) prob[sb * kMlpO + o] = p8[o];
            }
        }
    }
}

}  // namespace amrb

namespace amrb {

// Shared memory of the tensor-core gradient kernel: the forward layout, the
// tile's activations and deltas with the sample index contiguous (the K
// operand of the weight-gradient products), and the CTA's FP32 gradient
// accumulators.
struct TcGradSmem {
    TcSmem f;
    size_t h1t, h2t, d1t, d2t, d3t, cs, gw1, gw2, gw3, gb, loss, end;
    __host__ __device__ explicit TcGradSmem(int F) : f(F) {
        size_t o = f.end;
        h1t = o; o += size_t(kMlpH) * kTcPadS * 2;    // GELU(z1) [i][s]
        h2t = o; o += size_t(kMlpH) * kTcPadS * 2;    // GELU(z2) [j][s]
        d1t = o; o += size_t(kMlpH) * kTcPadS * 2;    // delta of layer 1 [i][s]
        d2t = o; o += size_t(kMlpH) * kTcPadS * 2;    // delta of layer 2 [j][s]
        d3t = o; o += size_t(8) * kTcPadS * 2;        // delta of the output [o][s], rows 3..7 zero
        cs = o; o += sizeof(float) * 4 * (2 * kMlpH + 8);   // per-warp column sums of d1, d2, d3
        gw1 = o; o += sizeof(float) * size_t(f.KP) * kMlpH;
        gw2 = o; o += sizeof(float) * kMlpH * kMlpH;
        gw3 = o; o += sizeof(float) * kMlpH * 8;
        gb = o; o += sizeof(float) * (2 * kMlpH + 8);
        loss = o; o += sizeof(float) * 4;
        end = (o + 15) & ~size_t(15);
    }
};

// sum of a C-fragment column pair over the warp's 16 rows (both rows of each
// lane, then across the 8 row groups): lanes g = 0 hold the sums of columns
// 2t, 2t+1
__device__ __forceinline__ float2 tc_colsum(const float (&c)[4]) {
    float a = c[0] + c[2], b = c[1] + c[3];
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    return make_float2(a, b);
}

// C fragment -> BF16 K-major store dst[col][row] (pitch kTcPadS) of the
// warp's rows m0 .. m0+15, columns 8 nt ..
__device__ __forceinline__ void tc_store_kmajor(__nv_bfloat16 *dst, const float (&c)[4], int nt, int m0, int lane) {
    const int g = lane >> 2, t = lane & 3, col = 8 * nt + 2 * t;
    dst[col * kTcPadS + m0 + g] = __float2bfloat16_rn(c[0]);
    dst[(col + 1) * kTcPadS + m0 + g] = __float2bfloat16_rn(c[1]);
    dst[col * kTcPadS + m0 + g + 8] = __float2bfloat16_rn(c[2]);
    dst[(col + 1) * kTcPadS + m0 + g + 8] = __float2bfloat16_rn(c[3]);
}

// C fragment of a weight-gradient tile (rows r0 .., columns c0 ..) added to an
// FP32 accumulator acc[r][c] (pitch p); each element has one owner thread
__device__ __forceinline__ void tc_acc_add(float *acc, int p, int r0, int c0, const float (&c)[4], int lane) {
    const int g = lane >> 2, t = lane & 3;
    acc[(r0 + g) * p + c0 + 2 * t] += c[0];
    acc[(r0 + g) * p + c0 + 2 * t + 1] += c[1];
    acc[(r0 + g + 8) * p + c0 + 2 * t] += c[2];
    acc[(r0 + g + 8) * p + c0 + 2 * t + 1] += c[3];
}

// Gradient of the mean cross-entropy over samples idx[0..nb) (features x
// [F][n_total], labels y), tiles of 64 samples per CTA in a grid stride.  Per
// tile each warp runs the forward pass of its 16 samples, the output delta
// d3 = (p - onehot) / nb in FP32, d2 = (d3 W3^T) GELU'(z2) in FP32, and
// d1 = (d2 W2^T) GELU'(z1) on tensor cores; then the CTA forms the tile's
// weight gradients X^T d1, h1^T d2, h2^T d3 on tensor cores and adds them to
// its FP32 accumulators.  Bias gradients are column sums of the FP32 deltas
// (warp shuffles, then the four warps in order).  The CTA's sums go to its
// row of `partial` ([gridDim][P + 1], last entry = loss), reduced in a fixed
// order by k_mlp_reduce: the gradient does not depend on scheduling.
static __global__ void __launch_bounds__(128) k_mlp_grad_tc(const __nv_bfloat16 *wb, int F, const float *x, int64_t n_total,
                                                       const int32_t *idx, const int8_t *y, int64_t nb, float *partial) {
    extern __shared__ __align__(16) unsigned char tc_smem[];
    unsigned char *sm = tc_smem;
    const MlpLayout L(F);
    const TcGradSmem G(F);
    const TcSmem &T = G.f;
    tc_load_weights(wb, L, sm, T);
    __nv_bfloat16 *h1t = reinterpret_cast<__nv_bfloat16 *>(sm + G.h1t), *h2t = reinterpret_cast<__nv_bfloat16 *>(sm + G.h2t);
    __nv_bfloat16 *d1t = reinterpret_cast<__nv_bfloat16 *>(sm + G.d1t), *d2t = reinterpret_cast<__nv_bfloat16 *>(sm + G.d2t);
    __nv_bfloat16 *d3t = reinterpret_cast<__nv_bfloat16 *>(sm + G.d3t);
    const __nv_bfloat16 *xt = reinterpret_cast<const __nv_bfloat16 *>(sm + T.xt);
    const __nv_bfloat16 *w2n = reinterpret_cast<const __nv_bfloat16 *>(sm + T.w2n);
    const __nv_bfloat16 *w3t = reinterpret_cast<const __nv_bfloat16 *>(sm + T.w3t);
    float *cs = reinterpret_cast<float *>(sm + G.cs);          // [warp][64 d1 | 64 d2 | 8 d3]
    float *gw1 = reinterpret_cast<float *>(sm + G.gw1);        // [f][i]
    float *gw2 = reinterpret_cast<float *>(sm + G.gw2);        // [i][j]
    float *gw3 = reinterpret_cast<float *>(sm + G.gw3);        // [j][o] (8 columns, 3 used)
    float *gb = reinterpret_cast<float *>(sm + G.gb);          // b1 | b2 | b3
    float *lsum = reinterpret_cast<float *>(sm + G.loss);      // per warp
    constexpr int CSW = 2 * kMlpH + 8;
    for (size_t e = threadIdx.x; e < size_t(T.KP) * kMlpH; e += blockDim.x) gw1[e] = 0.f;
    for (int e = threadIdx.x; e < kMlpH * kMlpH; e += blockDim.x) gw2[e] = 0.f;
    for (int e = threadIdx.x; e < kMlpH * 8; e += blockDim.x) gw3[e] = 0.f;
    for (int e = threadIdx.x; e < CSW; e += blockDim.x) gb[e] = 0.f;
    for (int e = threadIdx.x; e < 8 * kTcPadS; e += blockDim.x) d3t[e] = __float2bfloat16_rn(0.f);
    if (threadIdx.x < 4) lsum[threadIdx.x] = 0.f;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int m0 = 16 * warp;
    const float inv_nb = 1.0f / float(nb);
    const int64_t ntiles = (nb + kTcTile - 1) / kTcTile;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t s0 = tile * kTcTile;
        __syncthreads();
        tc_load_tile(x, n_total, s0, nb, [&](int64_t s) { return int64_t(idx[s]); }, sm, T);
        __syncthreads();
        float z1[8][4], z2[8][4], z3[4], p0[3], p8[3];
        tc_forward_warp(sm, T, lane, m0, z1, z2, z3);
        tc_softmax(z3, lane, p0, p8);
        // output delta and loss of rows g, g + 8 (every lane of the quad)
        const int64_t sa = s0 + m0 + g, sb = sa + 8;
        const bool va = sa < nb, vb = sb < nb;
        // classes 0..2 (a label outside them is clamped rather than read past the row)
        const int la = va ? min(max(int(y[idx[sa]]), 0), kMlpO - 1) : 0;
        const int lb = vb ? min(max(int(y[idx[sb]]), 0), kMlpO - 1) : 0;
        float d3a[3], d3b[3];
#pragma unroll
        for (int o = 0; o < 3; ++o) {
            d3a[o] = va ? (p0[o] - (o == la ? 1.f : 0.f)) * inv_nb : 0.f;
            d3b[o] = vb ? (p8[o] - (o == lb ? 1.f : 0.f)) * inv_nb : 0.f;
        }
        if (t == 0) {
            float l = (va ? -logf(p0[la]) : 0.f) + (vb ? -logf(p8[lb]) : 0.f);
            for (int o = 4; o < 32; o <<= 1) l += __shfl_xor_sync(0x11111111u, l, o);
            if (lane == 0) lsum[warp] += l * inv_nb;
            // the output delta as the K-major operand of h2^T d3
#pragma unroll
            for (int o = 0; o < 3; ++o) {
                d3t[o * kTcPadS + m0 + g] = __float2bfloat16_rn(d3a[o]);
                d3t[o * kTcPadS + m0 + g + 8] = __float2bfloat16_rn(d3b[o]);
            }
        }
        // d2 = (d3 W3^T) GELU'(z2) in FP32; h2 = GELU(z2) and d2 stored K-major
        float d2[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float h[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = 8 * nt + 2 * t + (e & 1);
                const float *d3r = (e < 2) ? d3a : d3b;
                float s = 0.f;
#pragma unroll
                for (int o = 0; o < 3; ++o) s = fmaf(__bfloat162float(w3t[o * kTcPadH + j]), d3r[o], s);
                d2[nt][e] = s * gelu_prime_f(z2[nt][e]);
                h[e] = gelu_f(z2[nt][e]);
            }
            tc_store_kmajor(h2t, h, nt, m0, lane);
            tc_store_kmajor(d2t, d2[nt], nt, m0, lane);
        }
        // d1 = (d2 W2^T) GELU'(z1) on tensor cores: A = d2 (BF16, from the C
        // fragments), B[k = j][n = i] = W2[i][j]
        float d1[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) d1[nt][0] = d1[nt][1] = d1[nt][2] = d1[nt][3] = 0.f;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
            uint32_t a[4];
            a[0] = pack_bf16(d2[2 * ks][0], d2[2 * ks][1]);
            a[1] = pack_bf16(d2[2 * ks][2], d2[2 * ks][3]);
            a[2] = pack_bf16(d2[2 * ks + 1][0], d2[2 * ks + 1][1]);
            a[3] = pack_bf16(d2[2 * ks + 1][2], d2[2 * ks + 1][3]);
#pragma unroll
            for (int np = 0; np < 4; ++np) {
                uint32_t b[4];
                b_frag2(b, w2n, kTcPadH, 16 * np, 16 * ks, lane);
                mma_bf16(d1[2 * np], a, b[0], b[1]);
                mma_bf16(d1[2 * np + 1], a, b[2], b[3]);
            }
        }
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float h[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                d1[nt][e] *= gelu_prime_f(z1[nt][e]);
                h[e] = gelu_f(z1[nt][e]);
            }
            tc_store_kmajor(h1t, h, nt, m0, lane);
            tc_store_kmajor(d1t, d1[nt], nt, m0, lane);
        }
        // bias gradients: column sums of the FP32 deltas over the warp's rows
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const float2 s1 = tc_colsum(d1[nt]), s2 = tc_colsum(d2[nt]);
            if (g == 0) {
                cs[warp * CSW + 8 * nt + 2 * t] = s1.x;
                cs[warp * CSW + 8 * nt + 2 * t + 1] = s1.y;
                cs[warp * CSW + kMlpH + 8 * nt + 2 * t] = s2.x;
                cs[warp * CSW + kMlpH + 8 * nt + 2 * t + 1] = s2.y;
            }
        }
        {
            float s3[3];
#pragma unroll
            for (int o = 0; o < 3; ++o) {
                float v = d3a[o] + d3b[o];      // rows g and g + 8 (identical in the quad)
                for (int off = 4; off < 32; off <<= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                s3[o] = v;
            }
            if (lane == 0) {
                cs[warp * CSW + 2 * kMlpH] = s3[0];
                cs[warp * CSW + 2 * kMlpH + 1] = s3[1];
                cs[warp * CSW + 2 * kMlpH + 2] = s3[2];
            }
        }
        __syncthreads();
        // weight gradients of the tile (K = the 64 samples)
        // gW1 [f][i] += X^T d1: A[m = f][k = s] = xt, B[k = s][n = i] = d1t^T
        const int nm1 = T.KP / 16;
        for (int w = warp; w < nm1 * 4; w += 4) {
            const int mt = w >> 2, np = w & 3;
            float c0[4] = {0.f, 0.f, 0.f, 0.f}, c1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                uint32_t a[4], b[4];
                a_frag_mmajor(a, xt, kTcPadS, 16 * mt, 16 * ks, lane);
                b_frag2(b, d1t, kTcPadS, 16 * np, 16 * ks, lane);
                mma_bf16(c0, a, b[0], b[1]);
                mma_bf16(c1, a, b[2], b[3]);
            }
            tc_acc_add(gw1, kMlpH, 16 * mt, 16 * np, c0, lane);
            tc_acc_add(gw1, kMlpH, 16 * mt, 16 * np + 8, c1, lane);
        }
        // gW2 [i][j] += h1^T d2
        for (int w = warp; w < 16; w += 4) {
            const int mt = w >> 2, np = w & 3;
            float c0[4] = {0.f, 0.f, 0.f, 0.f}, c1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                uint32_t a[4], b[4];
                a_frag_mmajor(a, h1t, kTcPadS, 16 * mt, 16 * ks, lane);
                b_frag2(b, d2t, kTcPadS, 16 * np, 16 * ks, lane);
                mma_bf16(c0, a, b[0], b[1]);
                mma_bf16(c1, a, b[2], b[3]);
            }
            tc_acc_add(gw2, kMlpH, 16 * mt, 16 * np, c0, lane);
            tc_acc_add(gw2, kMlpH, 16 * mt, 16 * np + 8, c1, lane);
        }
        // gW3 [j][o] += h2^T d3 (8 columns; warp w takes rows 16 w ..)
        {
            float c0[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                uint32_t a[4], b[4];
                a_frag_mmajor(a, h2t, kTcPadS, 16 * warp, 16 * ks, lane);
                const int i = lane >> 3, r = lane & 7;
                ldsm_x4(b, d3t + r * kTcPadS + 16 * ks + 8 * (i & 1));
                mma_bf16(c0, a, b[0], b[1]);
            }
            tc_acc_add(gw3, 8, 16 * warp, 0, c0, lane);
        }
        // bias sums, warps in order
        for (int e = threadIdx.x; e < CSW; e += blockDim.x) {
            if (e >= 2 * kMlpH + kMlpO) continue;
            gb[e] += ((cs[e] + cs[CSW + e]) + cs[2 * CSW + e]) + cs[3 * CSW + e];
        }
    }
    __syncthreads();
    // the CTA's row: [W1 (F x H), b1, W2, b2, W3 (H x 3), b3, loss]
    float *row = partial + int64_t(blockIdx.x) * (L.n + 1);
    for (int64_t q = threadIdx.x; q < L.n; q += blockDim.x) {
        float v;
        if (q < L.b1) v = gw1[q];                                   // [f][i] with f < F
        else if (q < L.w2) v = gb[q - L.b1];
        else if (q < L.b2) v = gw2[q - L.w2];
        else if (q < L.w3) v = gb[kMlpH + (q - L.b2)];
        else if (q < L.b3) {
            const int64_t e = q - L.w3;
            v = gw3[(e / kMlpO) * 8 + e % kMlpO];
        } else v = gb[2 * kMlpH + (q - L.b3)];
        row[q] = v;
    }
    if (threadIdx.x == 0) row[L.n] = ((lsum[0] + lsum[1]) + lsum[2]) + lsum[3];
}

}  // namespace amrb
