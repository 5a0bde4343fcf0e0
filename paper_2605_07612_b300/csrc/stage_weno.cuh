// Finite-volume stage with WENO5 face reconstruction (Sec. 3.2 lists WENO5
// among the limiters; it needs three ghost layers), for Euler and for scalar
// advection.  The same sub-step of
// Eq. 5 as stage.cuh, split into three passes over global memory because the
// five-cell stencils do not fit the two-cell halo of the plane-ring kernels:
//   k_weno_prim    primitives of every cell of every block (incl. ghosts)
//   k_weno_flux    one thread per face: WENO5 states from the six cells
//                  around the face, Rusanov or HLL flux; block-boundary faces
//                  also go to the refinement-face flux slots
//   k_weno_update  one thread per cell: flux divergence, gravity source,
//                  combination with the previous states, CFL speed.
// WENO5 (Jiang & Shu 1996): candidates q_k of third order, smoothness beta_k,
// weights (1/10, 6/10, 3/10) / (1e-6 + beta_k)^2 normalised.
#pragma once

#include <type_traits>

#include "stage.cuh"

namespace amrb {

template <class real>
__device__ __forceinline__ real weno5_face(real a, real b, real c, real d, real e) {
    const real q0 = (real(2) * a - real(7) * b + real(11) * c) * real(1.0 / 6.0);
    const real q1 = (-b + real(5) * c + real(2) * d) * real(1.0 / 6.0);
    const real q2 = (real(2) * c + real(5) * d - e) * real(1.0 / 6.0);
    const real t0 = a - real(2) * b + c, u0 = a - real(4) * b + real(3) * c;
    const real t1 = b - real(2) * c + d, u1 = b - d;
    const real t2 = c - real(2) * d + e, u2 = real(3) * c - real(4) * d + e;
    const real k = real(13.0 / 12.0);
    const real b0 = k * t0 * t0 + real(0.25) * u0 * u0;
    const real b1 = k * t1 * t1 + real(0.25) * u1 * u1;
    const real b2 = k * t2 * t2 + real(0.25) * u2 * u2;
    const real eps = real(1e-6);
    if constexpr (std::is_same<real, double>::value) {
        // one division instead of four: numerator and denominator times
        // s0 s1 s2, s_k = (eps + beta_k)^2 (FP64 divisions are slow here; the
        // products stay far inside the FP64 range for any finite state)
        const real s0 = (eps + b0) * (eps + b0), s1 = (eps + b1) * (eps + b1), s2 = (eps + b2) * (eps + b2);
        const real a0 = real(0.1) * (s1 * s2), a1 = real(0.6) * (s0 * s2), a2 = real(0.3) * (s0 * s1);
        return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
    } else {
        // FP32: approximate reciprocals (the weights are normalised, so their
        // few-ulp error stays a few ulp of the face value)
        const real a0 = real(0.1) * rcp_ftz((eps + b0) * (eps + b0));
        const real a1 = real(0.6) * rcp_ftz((eps + b1) * (eps + b1));
        const real a2 = real(0.3) * rcp_ftz((eps + b2) * (eps + b2));
        return (a0 * q0 + a1 * q1 + a2 * q2) * rcp_ftz(a0 + a1 + a2);
    }
}

// primitives of all S^D cells of every block: prim[b][v][cell] (Euler only:
// for scalar advection they are the state itself)
template <class real, int D>
__global__ void __launch_bounds__(256) k_weno_prim(const real *__restrict__ u, real *__restrict__ prim, Geom g, real gam) {
    using E = Euler<real, D>;
    const int b = blockIdx.x;
    const real *ub = u + int64_t(b) * g.bstride;
    real *pb = prim + int64_t(b) * g.bstride;
    for (int64_t c = threadIdx.x; c < g.ncell; c += blockDim.x) {
        real U[D + 2], w[D + 2];
#pragma unroll
        for (int v = 0; v < D + 2; ++v) U[v] = ub[int64_t(v) * g.ncell + c];
        E::prim(U, w, gam);
#pragma unroll
        for (int v = 0; v < D + 2; ++v) pb[int64_t(v) * g.ncell + c] = w[v];
    }
}

// Faces of a block: q < D (N+1) N^(D-1); direction n = q / nf, and within
// a direction the faces are numbered with x fastest whatever the normal, so
// that a warp's loads and stores run along rows: r = fp + (N+1)(y + N z)
// for x-faces, x + N (fp + (N+1) z) for y-faces, x + N (y + N fp) for
// z-faces (fp: face position along the normal, between cells fp-1 and fp).
// flux[b][n][v][r].  blockIdx.x = block, blockIdx.y = chunk of 256 faces.
template <int D>
__device__ __forceinline__ int weno_face_index(int n, int fp, const int *x, int N) {
    if (n == 0) return fp + (N + 1) * (x[1] + N * x[2]);
    if (n == 1) return x[0] + N * (fp + (N + 1) * x[2]);
    return x[0] + N * (x[1] + N * fp);
}

template <class real, int D, int PH>
__global__ void __launch_bounds__(256) k_weno_flux(const real *__restrict__ prim, real *__restrict__ flux,
                                                   const BlockInfo *__restrict__ info, real *bflux, Geom g,
                                                   PhysCtx<real> pc, int flux_kind, DevScalars *sc) {
    using E = Phys<real, D, PH>;
    constexpr int V = E::V;
    const int N = g.N, NG = g.ng, S = g.S;
    const int nface = D == 3 ? N * N : N;            // tangential faces per position
    const int nf = (N + 1) * nface;                  // faces per direction
    const int b = blockIdx.x;
    const int q = blockIdx.y * blockDim.x + threadIdx.x;
    if (q >= D * nf) return;
    const int n = q / nf, r = q - n * nf;
    int x[3] = {0, 0, 0}, fp;
    if (n == 0) {
        fp = r % (N + 1);
        const int t = r / (N + 1);
        x[1] = t % N;
        x[2] = t / N;
    } else if (n == 1) {
        x[0] = r % N;
        const int t = r / N;
        fp = t % (N + 1);
        x[2] = t / (N + 1);
    } else {
        x[0] = r % N;
        x[1] = (r / N) % N;
        fp = r / (N * N);
    }
    // tangential index of the face (lower tangential dimension first)
    const int t = n == 0 ? x[1] + N * x[2] : (n == 1 ? x[0] + N * x[2] : x[0] + N * x[1]);
    const real *pb = prim + int64_t(b) * g.bstride;
    auto cell = [&](int along) -> int64_t {
        const int i = n == 0 ? along : x[0], j = n == 1 ? along : x[1], k = n == 2 ? along : x[2];
        return (int64_t(D == 3 ? k + NG : 0) * S + (j + NG)) * S + (i + NG);
    };
    real wL[V], wR[V], F[V];
    bool bad = false;
    const int64_t c0 = cell(fp - 3), c1 = cell(fp - 2), c2 = cell(fp - 1), c3 = cell(fp), c4 = cell(fp + 1), c5 = cell(fp + 2);
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const real *pv = pb + int64_t(v) * g.ncell;
        const real w0 = pv[c0], w1 = pv[c1], w2 = pv[c2], w3 = pv[c3], w4 = pv[c4], w5 = pv[c5];
        wL[v] = weno5_face<real>(w0, w1, w2, w3, w4);
        wR[v] = weno5_face<real>(w5, w4, w3, w2, w1);
    }
    bad = E::nonphys(wL) || E::nonphys(wR);
    if (n == 0) E::template face_flux<0>(flux_kind, wL, wR, 0, pc, F);
    else if (n == 1) E::template face_flux<1>(flux_kind, wL, wR, 1, pc, F);
    else E::template face_flux<2>(flux_kind, wL, wR, 2, pc, F);
    real *fb = flux + (int64_t(b) * D + n) * V * nf;
#pragma unroll
    for (int v = 0; v < V; ++v) fb[int64_t(v) * nf + r] = F[v];
    if (fp == 0 || fp == N) {
        const int sl = info[b].bslot[2 * n + (fp == N)];
        if (sl >= 0) {
            real *dst = bflux + int64_t(sl) * V * nface + t;
#pragma unroll
            for (int v = 0; v < V; ++v) dst[int64_t(v) * nface] = F[v];
        }
    }
    if (bad) raise_status(&sc[0].status, 7);
}

// one thread per interior cell; blockIdx.x = block, blockIdx.y = chunk of 256 cells
template <class real, int D, int PH>
__global__ void __launch_bounds__(256) k_weno_update(StageArgs<real> a, const real *__restrict__ flux, Geom g) {
    using E = Phys<real, D, PH>;
    constexpr int V = E::V;
    __shared__ double red[8];
    const int N = g.N, NG = g.ng, S = g.S;
    const int nface = D == 3 ? N * N : N;
    const int nf = (N + 1) * nface;
    const int ncint = D == 3 ? N * N * N : N * N;
    const int b = blockIdx.x;
    const int c = blockIdx.y * blockDim.x + threadIdx.x;
    const BlockInfo info = a.info[b];
    double vmax = 0.0;
    if (c < ncint) {
        const int x[3] = {c % N, (c / N) % N, D == 3 ? c / (N * N) : 0};
        const int64_t o = (int64_t(D == 3 ? x[2] + NG : 0) * S + (x[1] + NG)) * S + (x[0] + NG);
        const int64_t ob = int64_t(b) * g.bstride + o;
        const int gc = info.gclass;
        const real dt_eff = real(a.w_dt * a.sc_in[info.inst].dt);
        const real *fb = flux + int64_t(b) * D * V * nf;
        real U[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            real r = real(0);
#pragma unroll
            for (int n = 0; n < D; ++n) {
                const int lo = weno_face_index<D>(n, x[n], x, N), hi = weno_face_index<D>(n, x[n] + 1, x, N);
                const real *fv = fb + (int64_t(n) * V + v) * nf;
                r += (fv[lo] - fv[hi]) * real(g.inv_dx[3 * gc + n]);
            }
            if constexpr (E::EULER) {
                if (a.gravity_on && v > 0) {
                    if (v <= D) {
                        r += a.deriv[ob] * a.grav[v - 1];
                    } else {
                        real sg = real(0);
#pragma unroll
                        for (int d = 0; d < D; ++d) sg += a.deriv[ob + int64_t(1 + d) * g.ncell] * a.grav[d];
                        r += sg;
                    }
                }
            }
            real acc = real(0);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q < a.nprev) acc += a.wprev[q] * a.prev[q][ob + int64_t(v) * g.ncell];
            U[v] = dt_eff * r + acc;
            a.out[ob + int64_t(v) * g.ncell] = U[v];
        }
        if (a.update_dt) {
            // cells next to a coarse-side refinement face are reduced after flux fixing
            const int m = info.fixmask;
            bool fixed = ((m & 1) && x[0] == 0) || ((m & 2) && x[0] == N - 1) || ((m & 4) && x[1] == 0) ||
                         ((m & 8) && x[1] == N - 1);
            if (D == 3) fixed = fixed || ((m & 16) && x[2] == 0) || ((m & 32) && x[2] == N - 1);
            if (!fixed) {
                if constexpr (E::EULER) {
                    real w[V];
                    E::prim(U, w, a.gamma);
                    const real cs = sqrt(a.gamma * w[D + 1] / w[0]);
                    real s = real(0);
#pragma unroll
                    for (int d = 0; d < D; ++d) s += (fabs(w[1 + d]) + cs) * real(g.inv_dx[3 * gc + d]);
                    vmax = double(s);
                } else {
                    real s = real(0);
#pragma unroll
                    for (int d = 0; d < D; ++d) s += fabs(a.vel[d]) * real(g.inv_dx[3 * gc + d]);
                    vmax = double(s);
                }
            }
        }
    }
    if (a.update_dt) {
        for (int o = 16; o > 0; o >>= 1) vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = vmax;
        __syncthreads();
        if (threadIdx.x == 0) {
            double m = red[0];
            for (int w = 1; w < int(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
            atomic_max_nonneg(&a.sc[info.inst].maxspeed_bits, m);
        }
    }
}

}  // namespace amrb
