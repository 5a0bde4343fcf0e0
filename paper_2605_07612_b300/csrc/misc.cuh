// Kernels around the stage: flux fixing (Sec. 2.7), the CFL time step
// (Sec. 3.2), conserved integrals (Eq. 18), the refinement criterion of
// Eq. 12 (Sec. 3.3) and the data transfer after a mesh change (Sec. 2.2).
#pragma once

#include "common.cuh"
#include "ghost.cuh"

namespace amrb {

// ---------------------------------------------------------------- flux fix
// One CTA per coarse block with refinement faces; its faces are processed in
// face order (-x, +x, -y, +y, -z, +z) with a barrier in between, so a cell on
// two such faces receives both corrections in a fixed order.  The correction
// of coarse cell c next to face f is
//   u_c += sign(f) * (w_dt dt / dx_n) * (F_coarse - mean of the fine fluxes)
// with sign +1 on high faces and -1 on low faces; the fine mean sums pairs
// along the lower tangential dimension first.
template <class real>
struct FixArgs {
    real *u;
    const BlockInfo *info;
    const FixFace *fix;
    const int32_t *fix_start;
    const real *bflux;
    double w_dt;
    DevScalars *sc;
    int update_dt;
    real gamma;
};

// sum_d |v_d| / dx_d: the CFL speed of scalar advection on geometry class gc
template <class real, int D>
__device__ __forceinline__ real advection_speed(const Geom &g, int gc) {
    real s = real(0);
    for (int d = 0; d < D; ++d) s += fabs(real(g.vel[d])) * real(g.inv_dx[3 * gc + d]);
    return s;
}

template <class real, int D>
__global__ void k_fluxfix(FixArgs<real> a, Geom g) {
    const int N = g.N, V = g.V;
    const int nface = (D == 3) ? N * N : N;
    const int first = a.fix_start[blockIdx.x], last = a.fix_start[blockIdx.x + 1];
    const int b = a.fix[first].block;
    const int gc = a.info[b].gclass, inst = a.info[b].inst;
    const real dt_eff = real(a.w_dt * a.sc[inst].dt);
    real *ub = a.u + int64_t(b) * g.bstride;
    real vmax = real(0);
    for (int q = first; q < last; ++q) {
        const FixFace ff = a.fix[q];
        const int n = ff.face >> 1, side = ff.face & 1;
        int td[2] = {-1, -1};
        for (int d = 0, c = 0; d < D; ++d)
            if (d != n) td[c++] = d;
        const real coef = dt_eff * real(g.inv_dx[3 * gc + n]);
        for (int t = threadIdx.x; t < nface; t += blockDim.x) {
            const int t0 = t % N, t1 = (D == 3) ? t / N : 0;
            const int o0 = t0 >= N / 2, o1 = (D == 3) ? (t1 >= N / 2) : 0;
            const int slot = ff.fslot[o0 | (o1 << 1)];
            const int f0 = 2 * (t0 - o0 * (N / 2)), f1 = 2 * (t1 - o1 * (N / 2));
            int x[3] = {0, 0, 0};
            x[n] = side ? N - 1 : 0;
            x[td[0]] = t0;
            if (D == 3) x[td[1]] = t1;
            const int64_t cell = cell_index<real>(g, x[0], x[1], x[2]);
            real U[5];
            for (int v = 0; v < V; ++v) {
                const real *fb = a.bflux + (int64_t(slot) * V + v) * nface;
                real mean;
                if (D == 3) {
                    mean = ((fb[f0 + N * f1] + fb[f0 + 1 + N * f1]) + (fb[f0 + N * (f1 + 1)] + fb[f0 + 1 + N * (f1 + 1)])) *
                           real(0.25);
                } else {
                    mean = (fb[f0] + fb[f0 + 1]) * real(0.5);
                }
                const real Fc = a.bflux[(int64_t(ff.cslot) * V + v) * nface + t];
                const real corr = coef * (Fc - mean);
                real &u = ub[int64_t(v) * g.ncell + cell];
                u = side ? u + corr : u - corr;
                U[v] = u;
            }
            (void)U;
        }
        __syncthreads();
    }
    if (!a.update_dt) return;
    // CFL limit of every corrected cell (cells on two faces count twice)
    for (int q = first; q < last; ++q) {
        const FixFace ff = a.fix[q];
        const int n = ff.face >> 1, side = ff.face & 1;
        int td[2] = {-1, -1};
        for (int d = 0, c = 0; d < D; ++d)
            if (d != n) td[c++] = d;
        for (int t = threadIdx.x; t < nface; t += blockDim.x) {
            int x[3] = {0, 0, 0};
            x[n] = side ? N - 1 : 0;
            x[td[0]] = t % N;
            if (D == 3) x[td[1]] = t / N;
            const int64_t cell = cell_index<real>(g, x[0], x[1], x[2]);
            real s = real(0);
            if (g.phys == 1) {
                s = advection_speed<real, D>(g, gc);
            } else {
                real U[5];
                for (int v = 0; v < V; ++v) U[v] = ub[int64_t(v) * g.ncell + cell];
                const real rho = U[0], ir = real(1) / rho;
                real ke = real(0);
                for (int d = 0; d < D; ++d) ke += U[1 + d] * U[1 + d] * ir;
                const real p = (a.gamma - real(1)) * (U[D + 1] - real(0.5) * ke);
                const real c = sqrt(a.gamma * p / rho);
                for (int d = 0; d < D; ++d) s += (fabs(U[1 + d] * ir) + c) * real(g.inv_dx[3 * gc + d]);
            }
            vmax = s > vmax ? s : vmax;
        }
    }
    double m = double(vmax);
    for (int s = 16; s > 0; s >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, s));
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(&a.sc[inst].maxspeed_bits, m);
}

// ------------------------------------------------------------------- CFL dt
// max over interior cells of sum_d (|v_d| + c) / dx_d (Sec. 3.2 step 2c);
// for scalar advection sum_d |v_d| / dx_d with the uniform velocity
template <class real, int D>
__global__ void k_maxspeed(const real *u, const BlockInfo *info, DevScalars *sc, Geom g, real gam) {
    const int b = blockIdx.x;
    const int N = g.N;
    const int ncell = (D == 3) ? N * N * N : N * N;
    const int gc = info[b].gclass, inst = info[b].inst;
    const real *ub = u + int64_t(b) * g.bstride;
    real vmax = real(0);
    for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
        const int i = c % N, j = (c / N) % N, k = (D == 3) ? c / (N * N) : 0;
        if (g.phys == 1) {
            const real s = advection_speed<real, D>(g, gc);
            vmax = s > vmax ? s : vmax;
            continue;
        }
        const int64_t cell = cell_index<real>(g, i, j, k);
        real U[5];
        for (int v = 0; v < g.V; ++v) U[v] = ub[int64_t(v) * g.ncell + cell];
        const real rho = U[0], ir = real(1) / rho;
        real ke = real(0);
        for (int d = 0; d < D; ++d) ke += U[1 + d] * U[1 + d] * ir;
        const real p = (gam - real(1)) * (U[D + 1] - real(0.5) * ke);
        const real cs = sqrt(gam * p / rho);
        real s = real(0);
        for (int d = 0; d < D; ++d) s += (fabs(U[1 + d] * ir) + cs) * real(g.inv_dx[3 * gc + d]);
        vmax = s > vmax ? s : vmax;
    }
    double m = double(vmax);
    for (int s = 16; s > 0; s >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, s));
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(&sc[inst].maxspeed_bits, m);
}

// dt = cfl / max speed per instance; resets the accumulators
__global__ void k_dt_commit(DevScalars *sc, const double *cfl, int n_inst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_inst) {
        const double m = __longlong_as_double((long long)sc[i].maxspeed_bits);
        sc[i].dt = (m > 0.0) ? cfl[i] / m : 0.0;
        sc[i].maxspeed_bits = 0ull;
    }
}

// --------------------------------------------------------- conserved sums
// Per block and variable: sum of u over interior cells in a fixed order
// (a fixed cell -> thread map, then a fixed shared-memory tree), times the
// cell volume.  Then k_conserved_final sums blocks in a fixed tree order.
template <class real, int D>
__global__ void __launch_bounds__(256) k_conserved_block(const real *u, const BlockInfo *info, double *partial, Geom g) {
    __shared__ double red[256];
    const int b = blockIdx.x;
    const int N = g.N;
    const int ncell = (D == 3) ? N * N * N : N * N;
    const int gc = info[b].gclass;
    double vol = 1.0;
    for (int d = 0; d < D; ++d) vol *= g.dx[3 * gc + d];
    for (int v = 0; v < g.V; ++v) {
        const real *ub = u + int64_t(b) * g.bstride + int64_t(v) * g.ncell;
        double s = 0.0;
        for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
            const int i = c % N, j = (c / N) % N, k = (D == 3) ? c / (N * N) : 0;
            s += double(ub[cell_index<real>(g, i, j, k)]);
        }
        red[threadIdx.x] = s;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[int64_t(b) * g.V + v] = red[0] * vol;
        __syncthreads();
    }
}

// one CTA per instance: blocks [range[i], range[i+1]) in a fixed tree order
__global__ void __launch_bounds__(1024) k_conserved_final(const double *partial, const int64_t *range, int V, double *out) {
    __shared__ double red[1024];
    const int64_t b0 = range[blockIdx.x], b1 = range[blockIdx.x + 1];
    out += int64_t(blockIdx.x) * V;
    for (int v = 0; v < V; ++v) {
        double s = 0.0;
        for (int64_t b = b0 + threadIdx.x; b < b1; b += blockDim.x) s += partial[b * V + v];
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

// ------------------------------------------------------------------- flags
// Simplified Lohner estimator (Eq. 12) on density and pressure, evaluated in
// double with every operation rounded as written (no contraction), so that
// the flag decision is the same as a plain double evaluation of the formula
// on the same stored values.  Per block: +1 if some cell exceeds c_ref, -1 if
// every cell is below c_deref, else 0.
template <class real, int D>
__device__ __forceinline__ void dprim_rn(const real *ub, const Geom &g, int64_t cell, double gam, double &rho, double &p) {
    double U[5];
    for (int v = 0; v < g.V; ++v) U[v] = double(ub[int64_t(v) * g.ncell + cell]);
    rho = U[0];
    if (g.phys == 1) {      // scalar advection: the scalar stands in for both
        p = rho;
        return;
    }
    double ke = 0.0;
    for (int d = 0; d < D; ++d) {
        const double w = __ddiv_rn(U[1 + d], rho);
        ke = __dadd_rn(ke, __dmul_rn(w, w));
    }
    ke = __dmul_rn(__dmul_rn(0.5, rho), ke);
    p = __dmul_rn(gam - 1.0, __dsub_rn(U[D + 1], ke));
}

__device__ __forceinline__ double lohner_1d(double um, double u0, double up, double eps, double eps_abs) {
    const double num = fabs(__dadd_rn(__dsub_rn(um, __dmul_rn(2.0, u0)), up));
    const double ustar = __dadd_rn(__dadd_rn(fabs(um), __dmul_rn(2.0, fabs(u0))), fabs(up));
    double den = __dadd_rn(eps_abs, fabs(__dsub_rn(u0, um)));
    den = __dadd_rn(den, fabs(__dsub_rn(up, u0)));
    den = __dadd_rn(den, __dmul_rn(eps, ustar));
    return __ddiv_rn(num, den);
}

// One CTA per block.  Density and pressure are converted to primitives once
// per cell into a ring of four z planes in shared memory; each plane holds its
// interior and the x/y face ghosts (corners are never read), the planes at
// z = -1 and z = N only their interior.  A cell's score is the larger of the
// two sums of squared 1D indicators (a NaN sum ignored, as the per-cell
// maximum of the criterion ignores it); the block keeps the largest score.
// Round-to-nearest sqrt is monotone, so one square root of the block maximum
// equals the largest per-cell sqrt and decides both thresholds exactly as a
// square root per cell would.
__host__ __device__ constexpr int flags_threads(int N) { return N * N + 4 * N < 384 ? N * N + 4 * N : 384; }
__host__ __device__ constexpr size_t flags_smem(int N, int D) {
    return size_t(D == 3 ? 4 : 1) * 2 * size_t(N + 2) * size_t(N + 2) * sizeof(double);
}

template <class real, int D>
__global__ void __launch_bounds__(384) k_flags(const real *u, Geom g, double gam, double c_ref, double c_deref, double eps,
                                               double eps_abs, int8_t *flags, const int32_t *list,
                                               const int32_t *count = nullptr) {
    extern __shared__ double fsm[];
    __shared__ double red[32];
    // with a device-side count, CTAs beyond it have no block
    if (count && int(blockIdx.x) >= *count) return;
    const int b = list ? list[blockIdx.x] : int(blockIdx.x);
    const int N = g.N, P = N + 2, plane = P * P;
    const int nslot = D == 3 ? 4 : 1;
    double *R = fsm, *Q = fsm + nslot * plane;
    const real *ub = u + int64_t(b) * g.bstride;
    // position t of a plane: t < N^2 interior (i fastest), then the four face
    // ghost rows i = -1, i = N, j = -1, j = N
    auto load = [&](int k, int slot) {
        const int n = (D == 3 && (k < 0 || k >= N)) ? N * N : N * N + 4 * N;
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            int i, j;
            if (t < N * N) {
                i = t % N;
                j = t / N;
            } else {
                const int side = (t - N * N) / N, q = (t - N * N) % N;
                i = side == 0 ? -1 : (side == 1 ? N : q);
                j = side == 2 ? -1 : (side == 3 ? N : q);
            }
            double r, p;
            dprim_rn<real, D>(ub, g, cell_index<real>(g, i, j, k), gam, r, p);
            const int c = slot * plane + (j + 1) * P + i + 1;
            R[c] = r;
            Q[c] = p;
        }
    };
    double m2 = 0.0;
    auto eval = [&](int sm, int s0, int sp) {
        for (int t = threadIdx.x; t < N * N; t += blockDim.x) {
            const int c = (t / N + 1) * P + t % N + 1;
            double best = 0.0;
            for (int which = 0; which < 2; ++which) {
                const double *A = which ? Q : R;
                const double *A0 = A + s0 * plane;
                const double a0 = A0[c];
                double e = lohner_1d(A0[c - 1], a0, A0[c + 1], eps, eps_abs);
                double e2 = __dadd_rn(0.0, __dmul_rn(e, e));
                e = lohner_1d(A0[c - P], a0, A0[c + P], eps, eps_abs);
                e2 = __dadd_rn(e2, __dmul_rn(e, e));
                if (D == 3) {
                    e = lohner_1d(A[sm * plane + c], a0, A[sp * plane + c], eps, eps_abs);
                    e2 = __dadd_rn(e2, __dmul_rn(e, e));
                }
                best = fmax(best, e2);
            }
            m2 = fmax(m2, best);
        }
    };
    if (D == 2) {
        load(0, 0);
        __syncthreads();
        eval(0, 0, 0);
    } else {
        // plane z lives in slot (z + 1) & 3; plane k - 1 is scored once plane
        // k is loaded.  The slot written at step k was last read at step k - 2,
        // and the barrier of step k - 1 lies between.
        for (int k = -1; k <= N; ++k) {
            load(k, (k + 1) & 3);
            __syncthreads();
            if (k >= 1) eval((k - 1) & 3, k & 3, (k + 1) & 3);
        }
    }
    for (int o = 16; o > 0; o >>= 1) m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double M = red[0];
        for (int w = 1; w < int(blockDim.x >> 5); ++w) M = fmax(M, red[w]);
        const double E = __dsqrt_rn(M);
        flags[b] = E > c_ref ? 1 : (E < c_deref ? -1 : 0);
    }
}

// ------------------------------------------------- criterion, FP32 screen
// Exact flags at a fraction of the FP64 work: one CTA per block evaluates
// every cell's criterion in FP32 as an interval that holds the value from
// the state's own numbers (and the FP64 value k_flags computes) for sure, and
// decides the block's flag when the interval of the block's largest value
// lies clear of both thresholds; otherwise the block goes to a list that
// k_flags then evaluates in FP64.  Bounds, with u = 2^-24:
//   rho: exact for an FP32 state, within 2^-23 |rho| for an FP64 state
//   rounded to FP32; p: |p - p~| <= 2^-18 ((g-1) ke + |p|) + 1e-30, twice
//   that for an FP64 state (rcp.approx.f32 errs by at most 2 u, each
//   rounding and each input's conversion by u; the floor covers values
//   flushed to zero in the range the screen admits);
//   indicator of (a-, a0, a+) with input bounds (b-, b0, b+), B = b- + 2 b0 + b+:
//   |num - num~| <= B + 2^-21 u*,  |den - den~| <= (1 + eps) B + 2^-20 den~,
//   so e lies in [(num~ - Bn) / (den~ + Bd), (num~ + Bn) / (den~ - Bd)],
//   widened by (1 -/+ 2^-19) for the rounding of the bounds themselves.
// A block is left to the FP64 pass when any input is not finite or outside
// 1e-6 <= rho <= 1e6, |U| <= 1e12, or some den~ <= 2 Bd.  thr: the squares
// of c_ref and c_deref (-1 for a negative threshold), each with the margin
// 2^-40 that keeps the FP64 square root's rounding on the decided side.
struct ScreenThresholds {
    double ref2_lo, ref2_hi, deref2_lo, deref2_hi;
};

template <class real, int D>
__global__ void __launch_bounds__(384) k_flags_screen(const real *u, Geom g, float gm1, float eps, float eps_abs,
                                                      ScreenThresholds thr, int8_t *flags, int32_t *list, int32_t *count) {
    constexpr bool WIDE = sizeof(real) == 8;                 // an FP64 state, rounded to FP32 here
    constexpr float KR = WIDE ? 0x1p-23f : 0.f;              // density bound per |rho|
    constexpr float KP = WIDE ? 0x1p-17f : 0x1p-18f;         // pressure bound factor
    extern __shared__ float fss[];
    __shared__ float rlo[32], rhi[32];
    __shared__ int rbad;
    const int b = int(blockIdx.x);
    const int N = g.N, P = N + 2, plane = P * P;
    const int nslot = D == 3 ? 4 : 1;
    float *R = fss, *Q = fss + nslot * plane, *Bq = fss + 2 * nslot * plane;
    const real *ub = u + int64_t(b) * g.bstride;
    if (threadIdx.x == 0) rbad = 0;
    bool bad = false;
    auto load = [&](int k, int slot) {
        const int n = (D == 3 && (k < 0 || k >= N)) ? N * N : N * N + 4 * N;
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            int i, j;
            if (t < N * N) {
                i = t % N;
                j = t / N;
            } else {
                const int side = (t - N * N) / N, q = (t - N * N) % N;
                i = side == 0 ? -1 : (side == 1 ? N : q);
                j = side == 2 ? -1 : (side == 3 ? N : q);
            }
            const int64_t cell = cell_index<real>(g, i, j, k);
            float U[5];
            bool ok = true;
            for (int v = 0; v < g.V; ++v) {
                const real x = ub[int64_t(v) * g.ncell + cell];
                // (false for NaN too; an FP32 state is range-checked in FP32,
                // since FP64 instructions run at a small fraction of the FP32
                // rate on B300)
                if constexpr (WIDE) ok = ok && fabs(x) <= 1e12;
                else ok = ok && fabsf(x) <= 1e12f;
                U[v] = ok ? float(x) : 0.f;
            }
            const float rho = U[0];
            float p = rho, bp = KR * rho;
            ok = ok && rho >= 1e-6f && rho <= 1e6f;
            if (g.phys != 1) {
                const float r = rcp_ftz(rho);
                float ke = 0.f;
                for (int d = 0; d < D; ++d) {
                    ok = ok && fabsf(U[1 + d]) <= 1e12f;
                    const float w = U[1 + d] * r;
                    ke = fmaf(w, w, ke);
                }
                ok = ok && fabsf(U[D + 1]) <= 1e12f;
                ke = 0.5f * rho * ke;
                p = gm1 * (U[D + 1] - ke);
                bp = KP * fmaf(gm1, ke, fabsf(p)) + 1e-30f;
                ok = ok && isfinite(p) && isfinite(ke);
            }
            bad = bad || !ok;
            const int c = slot * plane + (j + 1) * P + i + 1;
            R[c] = rho;
            Q[c] = p;
            Bq[c] = bp;
        }
    };
    // interval of the 1D indicator of (am, a0, ap) with bounds (bm, b0, bq)
    auto interval = [&](float am, float a0, float ap, float bm, float b0, float bq, float &lo, float &hi) {
        const float num = fabsf(am - 2.f * a0 + ap);
        const float ustar = fabsf(am) + 2.f * fabsf(a0) + fabsf(ap);
        const float den = eps_abs + fabsf(a0 - am) + fabsf(ap - a0) + eps * ustar;
        const float B = bm + 2.f * b0 + bq;
        const float Bn = B + 0x1p-21f * ustar;
        const float Bd = (1.f + eps) * B + 0x1p-20f * den;
        bad = bad || !(den > 2.f * Bd);
        hi = (num + Bn) * rcp_ftz(den - Bd) * (1.f + 0x1p-19f);
        lo = fmaxf(num - Bn, 0.f) * rcp_ftz(den + Bd) * (1.f - 0x1p-19f);
    };
    float mlo = 0.f, mhi = 0.f;
    auto eval = [&](int sm, int s0, int sp) {
        for (int t = threadIdx.x; t < N * N; t += blockDim.x) {
            const int c = (t / N + 1) * P + t % N + 1;
            for (int which = 0; which < 2; ++which) {
                const float *A = which ? Q : R;
                const float *A0 = A + s0 * plane;
                const float *BB = Bq + s0 * plane;
                float lo, hi, e2lo = 0.f, e2hi = 0.f;
                interval(A0[c - 1], A0[c], A0[c + 1], which ? BB[c - 1] : KR * A0[c - 1], which ? BB[c] : KR * A0[c],
                         which ? BB[c + 1] : KR * A0[c + 1], lo, hi);
                e2lo = fmaf(lo, lo, e2lo);
                e2hi = fmaf(hi, hi, e2hi);
                interval(A0[c - P], A0[c], A0[c + P], which ? BB[c - P] : KR * A0[c - P], which ? BB[c] : KR * A0[c],
                         which ? BB[c + P] : KR * A0[c + P], lo, hi);
                e2lo = fmaf(lo, lo, e2lo);
                e2hi = fmaf(hi, hi, e2hi);
                if (D == 3) {
                    interval(A[sm * plane + c], A0[c], A[sp * plane + c], which ? Bq[sm * plane + c] : KR * A[sm * plane + c],
                             which ? BB[c] : KR * A0[c], which ? Bq[sp * plane + c] : KR * A[sp * plane + c], lo, hi);
                    e2lo = fmaf(lo, lo, e2lo);
                    e2hi = fmaf(hi, hi, e2hi);
                }
                mlo = fmaxf(mlo, e2lo * (1.f - 0x1p-19f));
                mhi = fmaxf(mhi, e2hi * (1.f + 0x1p-19f));
                bad = bad || !isfinite(e2hi);
            }
        }
    };
    __syncthreads();
    if (D == 2) {
        load(0, 0);
        __syncthreads();
        eval(0, 0, 0);
    } else {
        for (int k = -1; k <= N; ++k) {
            load(k, (k + 1) & 3);
            __syncthreads();
            if (k >= 1) eval((k - 1) & 3, k & 3, (k + 1) & 3);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        mlo = fmaxf(mlo, __shfl_xor_sync(0xffffffffu, mlo, o));
        mhi = fmaxf(mhi, __shfl_xor_sync(0xffffffffu, mhi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        rlo[threadIdx.x >> 5] = mlo;
        rhi[threadIdx.x >> 5] = mhi;
    }
    if (bad) atomicOr(&rbad, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        float L = rlo[0], H = rhi[0];
        for (int w = 1; w < int(blockDim.x >> 5); ++w) {
            L = fmaxf(L, rlo[w]);
            H = fmaxf(H, rhi[w]);
        }
        // the block's largest squared value M (FP64, as k_flags computes it) lies in [L, H]
        const double lo = double(L), hi = double(H);
        int flag = 2;   // undecided
        if (!rbad) {
            const bool is_ref = lo > thr.ref2_hi, not_ref = hi < thr.ref2_lo;          // sqrt(M) > c_ref, <= c_ref
            const bool is_deref = hi < thr.deref2_lo, not_deref = lo > thr.deref2_hi;  // sqrt(M) < c_deref, >= c_deref
            if (is_ref) flag = 1;
            else if (not_ref && is_deref) flag = -1;
            else if (not_ref && not_deref) flag = 0;
        }
        if (flag != 2) flags[b] = int8_t(flag);
        else list[atomicAdd(count, 1)] = b;
    }
}

// ---------------------------------------------------------- regrid transfer
// For each new block: kind 0 copy old block src[0]; kind 1 prolong from old
// parent src[0] (child position `pos`, bit d = upper half along d), reading
// the parent's ghost cells at its edge; kind 2 restrict from old children
// src[0..2^D) (child c has bit d = upper half along d).  Interior cells only.
struct TransferOp {
    int32_t kind, pos;
    int32_t src[8];
};

template <class real, int D>
__global__ void __launch_bounds__(256) k_transfer(const real *uold, real *unew, const TransferOp *ops, Geom g) {
    const int b = blockIdx.x;
    const TransferOp op = ops[b];
    const int N = g.N;
    const int ncell = (D == 3) ? N * N * N : N * N;
    for (int idx = threadIdx.x; idx < ncell * g.V; idx += blockDim.x) {
        const int v = idx / ncell, c = idx - v * ncell;
        const int x[3] = {c % N, (c / N) % N, (D == 3) ? c / (N * N) : 0};
        real val;
        if (op.kind == 0) {
            val = uold[int64_t(op.src[0]) * g.bstride + int64_t(v) * g.ncell + cell_index<real>(g, x[0], x[1], x[2])];
        } else if (op.kind == 1) {
            int y[3] = {0, 0, 0}, s[3] = {0, 0, 0};
            for (int d = 0; d < D; ++d) {
                const int fine = ((op.pos >> d) & 1) * N + x[d];
                y[d] = fine >> 1;
                s[d] = fine & 1;
            }
            val = prolong_at<real, D>(uold + int64_t(op.src[0]) * g.bstride + int64_t(v) * g.ncell, g, y[0], y[1], y[2], s[0],
                                      s[1], s[2]);
        } else {
            int ch = 0, y[3] = {0, 0, 0};
            for (int d = 0; d < D; ++d) {
                const int hi = x[d] >= N / 2;
                ch |= hi << d;
                y[d] = 2 * (x[d] - hi * (N / 2));
            }
            val = restrict_at<real, D>(uold + int64_t(op.src[ch]) * g.bstride + int64_t(v) * g.ncell, g, y[0], y[1], y[2]);
        }
        unew[int64_t(b) * g.bstride + int64_t(v) * g.ncell + cell_index<real>(g, x[0], x[1], x[2])] = val;
    }
}

}  // namespace amrb
