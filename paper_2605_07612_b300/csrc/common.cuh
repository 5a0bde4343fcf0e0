// Shared device definitions of the B300 block-AMR kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pattern.hpp"

namespace amrb {


// Rounded operations that the compiler may not contract into an FMA; used
// where a result must match a plain IEEE evaluation order bit for bit.
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }

// 2-element vector type of a precision (aligned 8 / 16-byte accesses)
template <class real>
struct Vec2;
template <>
struct Vec2<float> { using type = float2; };
template <>
struct Vec2<double> { using type = double2; };

// minmod of Eq. 1 with theta = 1: zero unless both slopes have the same
// strict sign, else the one of smaller magnitude.
template <class T>
__device__ __forceinline__ T minmod(T a, T b) {
    T lo = a < b ? a : b, hi = a < b ? b : a;
    return (a > T(0) && b > T(0)) ? lo : ((a < T(0) && b < T(0)) ? hi : T(0));
}

// MUSCL slope of a cell from its one-sided differences a (left), b (right):
// lim 0 minmod; 1 monotonized central = Eq. 1 with theta = 2, i.e. for equal
// signs sign(a) min(2|a|, 2|b|, |a + b| / 2); 2 van Leer 2ab / (a + b) when
// ab > 0.  Zero when a and b differ in sign.
template <class T>
__device__ __forceinline__ T limited_slope(int lim, T a, T b) {
    if (lim == 0) return minmod(a, b);
    if (!((a > T(0) && b > T(0)) || (a < T(0) && b < T(0)))) return T(0);
    if (lim == 2) return T(2) * a * b / (a + b);
    T m = fabs(T(2) * a);
    m = fmin(m, fabs(T(2) * b));
    m = fmin(m, fabs(a + b) * T(0.5));
    return a > T(0) ? m : -m;
}

// Geometry of one forest as seen by the kernels.  A forest holds one or
// more independent mesh instances; cell sizes are looked up by geometry
// class gc = instance * kMaxLevels + level in device tables [gc][3].
struct Geom {
    int N, ng, S, D, V;
    int64_t ncell;          // S^D
    int64_t bstride;        // V * ncell
    const double *dx;       // [n_instances * kMaxLevels][3]
    const double *inv_dx;
    int phys;               // amr_physics: 0 Euler, 1 scalar advection
    double vel[3];          // advection velocity
};

// Approximate reciprocal and reciprocal square root of an FP32 value with
// denormal inputs and results flushed to zero: one special-function
// instruction each.  For normal inputs and results they equal the non-flushing
// forms (rsqrtf, __fdividef(1, x)), which add a denormal check and rescale
// around the same instruction.
__device__ __forceinline__ float rsqrt_ftz(float a) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ float rcp_ftz(float a) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}

// Device-resident scalars of a forest.
struct DevScalars {
    double dt;
    unsigned long long maxspeed_bits;   // max of a non-negative double, as bits
    int status;                         // first device-side error (amr_status)
    int pad;
};

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *p, double v) {
    atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ void raise_status(int *p, int code) { atomicCAS(p, 0, code); }

// Offset of cell (i, j, k) inside one variable of a block (ghosts included,
// i fastest); k is ignored in 2D.
template <class real>
__device__ __forceinline__ int64_t cell_index(const Geom &g, int i, int j, int k) {
    const int64_t kk = (g.D == 3) ? int64_t(k + g.ng) * g.S : int64_t(0);
    return (kk + (j + g.ng)) * g.S + (i + g.ng);
}

}  // namespace amrb
