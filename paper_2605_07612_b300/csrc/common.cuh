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

// Koren's limiter (Koren 1993) on the upwind difference a with the downwind
// difference b: a phi(b / a), phi(r) = max(0, min(2r, (1 + 2r) / 3, 2)), i.e.
// sign(a) min(2|b|, (|a| + 2|b|) / 3, 2|a|) when ab > 0, else 0.
template <class T>
__device__ __forceinline__ T koren_slope(T a, T b) {
    if (!(a * b > T(0))) return T(0);
    T m = fabs(T(2) * b);
    m = fmin(m, (fabs(a) + T(2) * fabs(b)) / T(3));
    m = fmin(m, fabs(T(2) * a));
    return a > T(0) ? m : -m;
}

// WENO3 value at the face right of cell b from cells a, b, c: candidates
// -a/2 + 3b/2 and (b + c)/2, smoothness (b - a)^2 and (c - b)^2, linear
// weights 1/3 and 2/3 over (1e-6 + beta)^2 (Jiang & Shu).
template <class T>
__device__ __forceinline__ T weno3_face(T a, T b, T c) {
    const T q0 = T(-0.5) * a + T(1.5) * b;
    const T q1 = T(0.5) * b + T(0.5) * c;
    const T b0 = (b - a) * (b - a), b1 = (c - b) * (c - b);
    const T e0 = T(1e-6) + b0, e1 = T(1e-6) + b1;
    const T a0 = T(1.0 / 3.0) / (e0 * e0), a1 = T(2.0 / 3.0) / (e1 * e1);
    return (a0 * q0 + a1 * q1) / (a0 + a1);
}

// Values of cell w0 at its left (lo) and right (hi) faces along one
// dimension from its neighbours wm, wp (two ghost layers): MUSCL w0 -/+
// slope / 2 with the limited slope (0 minmod, 1 MC, 2 van Leer), Koren's
// limiter (4), WENO3 (5) or first-order upwind (6, the cell value).
template <class T>
__device__ __forceinline__ void cell_faces(int lim, T wm, T w0, T wp, T &lo, T &hi) {
    const T a = w0 - wm, b = wp - w0;
    if (lim == 6) {
        lo = w0;
        hi = w0;
    } else if (lim == 4) {
        hi = w0 + T(0.5) * koren_slope<T>(a, b);
        lo = w0 - T(0.5) * koren_slope<T>(b, a);
    } else if (lim == 5) {
        hi = weno3_face<T>(wm, w0, wp);
        lo = weno3_face<T>(wp, w0, wm);
    } else {
        const T hs = T(0.5) * limited_slope<T>(lim, a, b);
        lo = w0 - hs;
        hi = w0 + hs;
    }
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
