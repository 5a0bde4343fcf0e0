// Finite-volume stage with WENO5 face reconstruction (Sec. 3.2 lists WENO5
// among the limiters; it needs three ghost layers), for Euler and for scalar
// advection.  The same sub-step of
// Eq. 5 as stage.cuh, split into two passes over global memory because the
// five-cell stencils do not fit the two-cell halo of the plane-ring kernels:
//   k_weno_flux    one thread per pencil of faces along a direction:
//                  primitives of each cell as it is loaded, WENO5 states of
//                  each cell's two faces, Rusanov or HLL flux; block-boundary
//                  faces also go to the refinement-face flux slots
//   k_weno_update  one thread per cell: flux divergence, gravity source,
//                  combination with the previous states, CFL speed.
// WENO5 (Jiang & Shu 1996): candidates q_k of third order, smoothness beta_k,
// weights (1/10, 6/10, 3/10) / (1e-6 + beta_k)^2 normalised.
#pragma once

#include <type_traits>

#include "stage.cuh"
#include "stage_pair.cuh"

namespace amrb {

// WENO5 values at both faces of the centre cell c of the stencil
// (a, b, c, d, e) = cells i-2 .. i+2: `right` at face i+1/2 from the
// candidates of the left-biased stencils, `left` at face i-1/2 from their
// mirror images.  The smoothness indicators beta_k of the three 3-cell
// sub-stencils serve both values (the mirror image swaps beta_0 and
// beta_2), so a cell's stencil is evaluated once for its two faces.
template <class real>
__device__ __forceinline__ void weno5_cell(real a, real b, real c, real d, real e, real &left, real &right) {
    const real r6 = real(1.0 / 6.0);
    const real q0 = (real(2) * a - real(7) * b + real(11) * c) * r6;
    const real q1 = (-b + real(5) * c + real(2) * d) * r6;
    const real q2 = (real(2) * c + real(5) * d - e) * r6;
    const real p0 = (real(2) * e - real(7) * d + real(11) * c) * r6;   // mirror images
    const real p1 = (-d + real(5) * c + real(2) * b) * r6;
    const real p2 = (real(2) * c + real(5) * b - a) * r6;
    const real t0 = a - real(2) * b + c, u0 = a - real(4) * b + real(3) * c;
    const real t1 = b - real(2) * c + d, u1 = b - d;
    const real t2 = c - real(2) * d + e, u2 = real(3) * c - real(4) * d + e;
    const real k = real(13.0 / 12.0);
    const real b0 = k * t0 * t0 + real(0.25) * u0 * u0;
    const real b1 = k * t1 * t1 + real(0.25) * u1 * u1;
    const real b2 = k * t2 * t2 + real(0.25) * u2 * u2;
    const real eps = real(1e-6);
    if constexpr (std::is_same<real, double>::value) {
        // one division per value instead of four: weights times
        // s0 s1 s2, s_k = (eps + beta_k)^2 (FP64 divisions are slow here; the
        // products stay far inside the FP64 range for any finite state)
        const real s0 = (eps + b0) * (eps + b0), s1 = (eps + b1) * (eps + b1), s2 = (eps + b2) * (eps + b2);
        const real s12 = s1 * s2, s02 = s0 * s2, s01 = s0 * s1;
        const real a0 = real(0.1) * s12, a1 = real(0.6) * s02, a2 = real(0.3) * s01;
        right = (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
        const real m0 = real(0.1) * s01, m1 = real(0.6) * s02, m2 = real(0.3) * s12;
        left = (m0 * p0 + m1 * p1 + m2 * p2) / (m0 + m1 + m2);
    } else {
        // FP32: approximate reciprocals (the weights are normalised, so their
        // few-ulp error stays a few ulp of the face value)
        const real s0 = rcp_ftz((eps + b0) * (eps + b0));
        const real s1 = rcp_ftz((eps + b1) * (eps + b1));
        const real s2 = rcp_ftz((eps + b2) * (eps + b2));
        const real a0 = real(0.1) * s0, a1 = real(0.6) * s1, a2 = real(0.3) * s2;
        right = (a0 * q0 + a1 * q1 + a2 * q2) * rcp_ftz(a0 + a1 + a2);
        const real m0 = real(0.1) * s2, m1 = real(0.6) * s1, m2 = real(0.3) * s0;
        left = (m0 * p0 + m1 * p1 + m2 * p2) * rcp_ftz(m0 + m1 + m2);
    }
}

// weno5_cell for two FP32 stencils at once (two variables of one cell) in
// packed two-wide arithmetic: the same formulas, each product and sum an
// explicit rounded operation
__device__ __forceinline__ void weno5_cell2(float2 a, float2 b, float2 c, float2 d, float2 e, float2 &left, float2 &right) {
    const float2 r6 = PF::sp(1.f / 6.f);
    const float2 two = PF::sp(2.f), five = PF::sp(5.f);
    const float2 q0 = PF::mul(PF::fma(two, a, PF::fma(PF::sp(-7.f), b, PF::mul(PF::sp(11.f), c))), r6);
    const float2 q1 = PF::mul(PF::fma(five, c, PF::fma(two, d, PF::mul(PF::sp(-1.f), b))), r6);
    const float2 q2 = PF::mul(PF::fma(two, c, PF::fma(five, d, PF::mul(PF::sp(-1.f), e))), r6);
    const float2 p0 = PF::mul(PF::fma(two, e, PF::fma(PF::sp(-7.f), d, PF::mul(PF::sp(11.f), c))), r6);   // mirror images
    const float2 p1 = PF::mul(PF::fma(five, c, PF::fma(two, b, PF::mul(PF::sp(-1.f), d))), r6);
    const float2 p2 = PF::mul(PF::fma(two, c, PF::fma(five, b, PF::mul(PF::sp(-1.f), a))), r6);
    const float2 t0 = PF::add(PF::fma(PF::sp(-2.f), b, a), c), u0 = PF::fma(PF::sp(3.f), c, PF::fma(PF::sp(-4.f), b, a));
    const float2 t1 = PF::add(PF::fma(PF::sp(-2.f), c, b), d), u1 = PF::sub(b, d);
    const float2 t2 = PF::add(PF::fma(PF::sp(-2.f), d, c), e), u2 = PF::add(PF::fma(PF::sp(-4.f), d, PF::mul(PF::sp(3.f), c)), e);
    const float2 k = PF::sp(13.f / 12.f), q4 = PF::sp(0.25f), eps = PF::sp(1e-6f);
    const float2 e0 = PF::add(eps, PF::fma(k, PF::mul(t0, t0), PF::mul(q4, PF::mul(u0, u0))));
    const float2 e1 = PF::add(eps, PF::fma(k, PF::mul(t1, t1), PF::mul(q4, PF::mul(u1, u1))));
    const float2 e2 = PF::add(eps, PF::fma(k, PF::mul(t2, t2), PF::mul(q4, PF::mul(u2, u2))));
    // 1 / (eps + beta_k)^2 by approximate reciprocals, as in weno5_cell
    const float2 s0 = PF::rcp(PF::mul(e0, e0)), s1 = PF::rcp(PF::mul(e1, e1)), s2 = PF::rcp(PF::mul(e2, e2));
    const float2 a0 = PF::mul(PF::sp(0.1f), s0), a1 = PF::mul(PF::sp(0.6f), s1), a2 = PF::mul(PF::sp(0.3f), s2);
    right = PF::mul(PF::fma(a2, q2, PF::fma(a1, q1, PF::mul(a0, q0))), PF::rcp(PF::add(PF::add(a0, a1), a2)));
    const float2 m0 = PF::mul(PF::sp(0.1f), s2), m2 = PF::mul(PF::sp(0.3f), s0);
    left = PF::mul(PF::fma(m2, p2, PF::fma(a1, p1, PF::mul(m0, p0))), PF::rcp(PF::add(PF::add(m0, a1), m2)));
}

// Faces of a block: D (N+1) N^(D-1), N+1 positions fp per direction n
// (fp between cells fp-1 and fp) and N^(D-1) tangential positions.  Within
// a direction the faces are numbered with x fastest whatever the normal:
// r = fp + (N+1)(y + N z) for x-faces, x + N (fp + (N+1) z) for y-faces,
// x + N (y + N fp) for z-faces; flux[b][n][v][r].
template <int D>
__device__ __forceinline__ int weno_face_index(int n, int fp, const int *x, int N) {
    if (n == 0) return fp + (N + 1) * (x[1] + N * x[2]);
    if (n == 1) return x[0] + N * (fp + (N + 1) * x[2]);
    return x[0] + N * (x[1] + N * fp);
}

// One thread per pencil: the N+1 faces of one direction n at one tangential
// position t, marched along n with the five-cell stencil of the current
// cell in registers (one load per variable and cell, each cell's WENO5
// stencil evaluated once for its two faces).  Consecutive threads take
// consecutive tangential positions, so the y and z pencils load and store
// along rows.  The CTAs of one block are adjacent (blockIdx.x = block x
// chunks + chunk), so a block's cells come from DRAM once.  Each loaded cell
// is converted to primitives (once per direction).
// Block-boundary faces also go to the refinement-face flux slots.
template <class real, int D, int PH>
__global__ void __launch_bounds__(256) k_weno_flux(const real *__restrict__ u, real *__restrict__ flux,
                                                   const BlockInfo *__restrict__ info, real *bflux, Geom g,
                                                   PhysCtx<real> pc, int flux_kind, DevScalars *sc) {
    using E = Phys<real, D, PH>;
    constexpr int V = E::V;
    const int N = g.N, NG = g.ng, S = g.S;
    const int nface = D == 3 ? N * N : N;            // tangential positions per direction
    const int nf = (N + 1) * nface;                  // faces per direction
    const int npen = D * nface;
    const int chunks = (npen + int(blockDim.x) - 1) / int(blockDim.x);
    const int b = int(blockIdx.x) / chunks;
    const int p = (int(blockIdx.x) - b * chunks) * int(blockDim.x) + int(threadIdx.x);
    if (p >= npen) return;
    const int n = p / nface, t = p - n * nface;      // t: lower tangential dimension fastest
    const int ta = t % N, tb = t / N;
    int x[3] = {0, 0, 0};
    if (n == 0) {
        x[1] = ta;
        x[2] = tb;
    } else if (n == 1) {
        x[0] = ta;
        x[2] = tb;
    } else {
        x[0] = ta;
        x[1] = tb;
    }
    // cell `along` of the pencil: o0 + along * step; face fp: fb0 + fp * fstep
    const int64_t step = n == 0 ? 1 : (n == 1 ? int64_t(S) : int64_t(S) * S);
    const int64_t o0 = (int64_t(D == 3 ? x[2] + NG : 0) * S + (x[1] + NG)) * S + (x[0] + NG);
    const real *ub = u + int64_t(b) * g.bstride + o0;
    // primitives of cell `along` of the pencil
    auto load = [&](int along, real *w) {
        real U[V];
#pragma unroll
        for (int v = 0; v < V; ++v) U[v] = ub[int64_t(v) * g.ncell + along * step];
        E::prim(U, w, pc.gam);
    };
    const int fb0 = weno_face_index<D>(n, 0, x, N);
    const int fstep = n == 0 ? 1 : (n == 1 ? N : N * N);
    real *fb = flux + (int64_t(b) * D + n) * V * nf + fb0;
    const int slo = (info[b].bslot[2 * n]), shi = (info[b].bslot[2 * n + 1]);
    // stencil of the current centre cell (along c-2 .. c+2), per variable
    real st[V][5], w[V];
#pragma unroll
    for (int m = 0; m < 4; ++m) {   // cells -3 .. 0
        load(m - 3, w);
#pragma unroll
        for (int v = 0; v < V; ++v) st[v][m + 1] = w[v];
    }
    real wL[V], wR[V], wnext[V], F[V];
    bool bad = false;
    for (int fp = -1; fp <= N; ++fp) {
        // centre cell fp: load cell fp + 2, evaluate its stencil
        load(fp + 2, w);
#pragma unroll
        for (int v = 0; v < V; ++v) {
#pragma unroll
            for (int m = 0; m < 4; ++m) st[v][m] = st[v][m + 1];
            st[v][4] = w[v];
            weno5_cell<real>(st[v][0], st[v][1], st[v][2], st[v][3], st[v][4], wR[v], wnext[v]);
        }
        if (fp >= 0) {
            // face fp: left state from cell fp-1, right state from cell fp
            bad = bad || E::nonphys(wL) || E::nonphys(wR);
            if (n == 0) E::template face_flux<0>(flux_kind, wL, wR, 0, pc, F);
            else if (n == 1) E::template face_flux<1>(flux_kind, wL, wR, 1, pc, F);
            else E::template face_flux<2>(flux_kind, wL, wR, 2, pc, F);
#pragma unroll
            for (int v = 0; v < V; ++v) fb[int64_t(v) * nf + int64_t(fp) * fstep] = F[v];
            const int sl = fp == 0 ? slo : (fp == N ? shi : -1);
            if (sl >= 0) {
                real *dst = bflux + int64_t(sl) * V * nface + t;
#pragma unroll
                for (int v = 0; v < V; ++v) dst[int64_t(v) * nface] = F[v];
            }
        }
#pragma unroll
        for (int v = 0; v < V; ++v) wL[v] = wnext[v];
    }
    if (bad) raise_status(&sc[0].status, 7);
}

// one thread per interior cell; blockIdx.x = block x chunks + chunk of 256
// cells (a block's chunks adjacent, for L2 reuse of its face fluxes)
template <class real, int D, int PH>
__global__ void __launch_bounds__(256) k_weno_update(StageArgs<real> a, const real *__restrict__ flux, Geom g) {
    using E = Phys<real, D, PH>;
    constexpr int V = E::V;
    __shared__ double red[8];
    const int N = g.N, NG = g.ng, S = g.S;
    const int nface = D == 3 ? N * N : N;
    const int nf = (N + 1) * nface;
    const int ncint = D == 3 ? N * N * N : N * N;
    const int chunks = (ncint + int(blockDim.x) - 1) / int(blockDim.x);
    const int b = int(blockIdx.x) / chunks;
    const int c = (int(blockIdx.x) - b * chunks) * int(blockDim.x) + int(threadIdx.x);
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


// Single-pass WENO5 stage for 3D blocks of N^3 cells (N = 8 or 16): one CTA
// of N^2 threads per block.  The CTA sweeps the block three times with one
// thread per pencil, along x, then y, then z, with the pencil march of
// k_weno_flux (each cell's five-cell stencil evaluated once for its two
// faces); instead of going to global memory the face fluxes are differenced
// at once into the divergence of the pencil's cells, accumulated in shared
// memory across the three sweeps (barrier between sweeps).  The z sweep
// finishes each cell: gravity source, combination with the previous states
// (Eq. 5), output, CFL speed.  The stencil of a pencil end reaches three
// cells into the neighbour: in gather mode they are read from a same-level
// neighbour's interior, otherwise (and across refinement faces and domain
// boundaries) from the block's filled ghost cells.  Block-boundary face
// fluxes go to the refinement-face slots as in k_weno_flux.
template <int N, int PH>
struct WenoFused {
    static constexpr int NT = N * N;
    static constexpr int V = Phys<float, 3, PH>::V;
    // divergence of cell (x, y, z) at x + P (y + N z): rows padded to P = N + 1
    // words, so that the x sweep (consecutive threads on consecutive rows)
    // hits distinct banks; the y and z sweeps run along rows
    static constexpr int P = N + 1, NCP = P * N * N;
    static constexpr size_t smem_bytes() { return sizeof(float) * size_t(V) * NCP; }
};

template <int N, int PH>
__global__ void __launch_bounds__(N * N) k_weno_fused(StageArgs<float> a, Geom g, PhysCtx<float> pc) {
    using E = Phys<float, 3, PH>;
    constexpr int V = E::V, NC3 = WenoFused<N, PH>::NCP, PW = WenoFused<N, PH>::P;
    extern __shared__ __align__(16) float wdu[];     // [V][N^2 rows of P] divergence of the block's cells
    __shared__ double red[N * N / 32];
    const int tid = threadIdx.x, ta = tid % N, tb = tid / N;
    const int S = g.S, NG = g.ng;
    const int64_t ncell = g.ncell;
    bool bad = false;
    for (int b = blockIdx.x; b < a.n_items; b += gridDim.x) {
        const int gc = a.info[b].gclass, inst = a.info[b].inst, fixmask = a.info[b].fixmask;
        const float dte = float(a.w_dt * a.sc_in[inst].dt);
        const float *ub = a.deriv + int64_t(b) * g.bstride;
        double vmax = 0.0;
#pragma unroll 1
        for (int n = 0; n < 3; ++n) {
            // pencil along n at tangential (ta, tb) (the lower tangential dimension fastest)
            const int x0 = n == 0 ? 0 : ta, x1 = n == 0 ? ta : (n == 1 ? 0 : tb), x2 = n == 2 ? 0 : tb;
            const int64_t step = n == 0 ? 1 : (n == 1 ? int64_t(S) : int64_t(S) * S);
            const int64_t o0 = (int64_t(x2 + NG) * S + (x1 + NG)) * S + (x0 + NG);
            const int cstep = n == 0 ? 1 : (n == 1 ? PW : PW * N);
            const int c0 = x0 + PW * (x1 + N * x2);
            const float idx = float(g.inv_dx[3 * gc + n]);
            const BlockInfo *ib = a.info + b;   // fields indexed by the direction: read from memory
            const int nlo = a.gather ? ib->nbr[2 * n] : -1, nhi = a.gather ? ib->nbr[2 * n + 1] : -1;
            const float *lob = nlo >= 0 ? a.deriv + int64_t(nlo) * g.bstride + o0 + int64_t(N) * step : ub + o0;
            const float *hib = nhi >= 0 ? a.deriv + int64_t(nhi) * g.bstride + o0 - int64_t(N) * step : ub + o0;
            // conservative state of cell `along` of the pencil (-3 .. N + 2)
            auto fetch = [&](int along, float *U) {
                const float *src = along < 0 ? lob : (along >= N ? hib : ub + o0);
#pragma unroll
                for (int v = 0; v < V; ++v) U[v] = src[int64_t(v) * ncell + along * step];
            };
            auto load = [&](int along, float *w) {
                float U[V];
                fetch(along, U);
                E::prim(U, w, pc.gam);
            };
            const int slo = ib->bslot[2 * n], shi = ib->bslot[2 * n + 1];
            const int tface = ta + N * tb;
            float st[V][5], w[V], wL[V], wR[V], wnext[V], F[V], Fp[V], Un[V];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                load(m - 3, w);
#pragma unroll
                for (int v = 0; v < V; ++v) st[v][m + 1] = w[v];
            }
            fetch(1, Un);
#pragma unroll 1
            for (int fp = -1; fp <= N; ++fp) {
                // the cell entering the stencil was fetched one position
                // ahead; fetch the next one (its loads stay in flight
                // through this position's arithmetic)
                E::prim(Un, w, pc.gam);
                if (fp + 3 <= N + 2) fetch(fp + 3, Un);
#pragma unroll
                for (int v = 0; v < V; ++v) {
#pragma unroll
                    for (int m = 0; m < 4; ++m) st[v][m] = st[v][m + 1];
                    st[v][4] = w[v];
                }
                if constexpr (V == 5) {
                    // variables (0, 1) and (2, 3) as packed pairs, 4 alone
#pragma unroll
                    for (int v = 0; v < 4; v += 2) {
                        float2 l2, r2;
                        weno5_cell2(make_float2(st[v][0], st[v + 1][0]), make_float2(st[v][1], st[v + 1][1]),
                                    make_float2(st[v][2], st[v + 1][2]), make_float2(st[v][3], st[v + 1][3]),
                                    make_float2(st[v][4], st[v + 1][4]), l2, r2);
                        wR[v] = l2.x;
                        wR[v + 1] = l2.y;
                        wnext[v] = r2.x;
                        wnext[v + 1] = r2.y;
                    }
                    weno5_cell<float>(st[4][0], st[4][1], st[4][2], st[4][3], st[4][4], wR[4], wnext[4]);
                } else {
#pragma unroll
                    for (int v = 0; v < V; ++v) weno5_cell<float>(st[v][0], st[v][1], st[v][2], st[v][3], st[v][4], wR[v], wnext[v]);
                }
                if (fp >= 0) {
                    bad = bad || E::nonphys(wL) || E::nonphys(wR);
                    if (n == 0) E::template face_flux<0>(a.flux, wL, wR, 0, pc, F);
                    else if (n == 1) E::template face_flux<1>(a.flux, wL, wR, 1, pc, F);
                    else E::template face_flux<2>(a.flux, wL, wR, 2, pc, F);
                    const int sl = fp == 0 ? slo : (fp == N ? shi : -1);
                    if (sl >= 0) {
                        float *dst = a.bflux + int64_t(sl) * V * (N * N) + tface;
#pragma unroll
                        for (int v = 0; v < V; ++v) dst[int64_t(v) * (N * N)] = F[v];
                    }
                    if (fp >= 1) {
                        // cell fp - 1: its lower face flux Fp, upper face F
                        const int c = c0 + (fp - 1) * cstep;
                        float du[V];
#pragma unroll
                        for (int v = 0; v < V; ++v) {
                            du[v] = (Fp[v] - F[v]) * idx;
                            if (n > 0) du[v] += wdu[v * NC3 + c];
                        }
                        if (n < 2) {
#pragma unroll
                            for (int v = 0; v < V; ++v) wdu[v * NC3 + c] = du[v];
                        } else {
                            // the cell is complete: source, Eq. 5, output, CFL speed
                            if constexpr (E::EULER) {
                                if (a.gravity_on) {
                                    // S = (0, rho g, (rho v) . g) of the cell's conservative state
                                    const int64_t oc = int64_t(b) * g.bstride + o0 + int64_t(fp - 1) * step;
                                    float sgv = 0.f;
#pragma unroll
                                    for (int d = 0; d < 3; ++d) {
                                        du[1 + d] += a.deriv[oc] * a.grav[d];
                                        sgv += a.deriv[oc + int64_t(1 + d) * ncell] * a.grav[d];
                                    }
                                    du[4] += sgv;
                                }
                            }
                            const int64_t ob = int64_t(b) * g.bstride + o0 + int64_t(fp - 1) * step;
                            float U[V];
#pragma unroll
                            for (int v = 0; v < V; ++v) {
                                float acc = 0.f;
#pragma unroll
                                for (int q = 0; q < 4; ++q)
                                    if (q < a.nprev) acc += a.wprev[q] * a.prev[q][ob + int64_t(v) * ncell];
                                U[v] = dte * du[v] + acc;
                                a.out[ob + int64_t(v) * ncell] = U[v];
                            }
                            if (a.update_dt) {
                                const int m = fixmask, k = fp - 1;
                                const bool fixed = ((m & 1) && x0 == 0) || ((m & 2) && x0 == N - 1) || ((m & 4) && x1 == 0) ||
                                                   ((m & 8) && x1 == N - 1) || ((m & 16) && k == 0) || ((m & 32) && k == N - 1);
                                if (!fixed) {
                                    if constexpr (E::EULER) {
                                        float wv[V];
                                        E::prim(U, wv, a.gamma);
                                        const float cs = sqrtf(a.gamma * wv[4] / wv[0]);
                                        float sp = 0.f;
#pragma unroll
                                        for (int d = 0; d < 3; ++d) sp += (fabsf(wv[1 + d]) + cs) * float(g.inv_dx[3 * gc + d]);
                                        vmax = fmax(vmax, double(sp));
                                    } else {
                                        float sp = 0.f;
#pragma unroll
                                        for (int d = 0; d < 3; ++d) sp += fabsf(a.vel[d]) * float(g.inv_dx[3 * gc + d]);
                                        vmax = fmax(vmax, double(sp));
                                    }
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int v = 0; v < V; ++v) Fp[v] = F[v];
                }
#pragma unroll
                for (int v = 0; v < V; ++v) wL[v] = wnext[v];
            }
            __syncthreads();   // the sweep's divergence is complete (and the next block may overwrite it after z)
        }
        if (a.update_dt) {
            for (int o = 16; o > 0; o >>= 1) vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
            if ((tid & 31) == 0) red[tid >> 5] = vmax;
            __syncthreads();
            if (tid == 0) {
                double m = red[0];
                for (int w2 = 1; w2 < N * N / 32; ++w2) m = fmax(m, red[w2]);
                atomic_max_nonneg(&a.sc[inst].maxspeed_bits, m);
            }
            __syncthreads();
        }
    }
    if (__syncthreads_or(bad) && tid == 0) raise_status(&a.sc[0].status, 7);
}

}  // namespace amrb
