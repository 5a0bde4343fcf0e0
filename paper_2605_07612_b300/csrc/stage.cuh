// Finite-volume Runge-Kutta stage of the Euler equations (Sec. 3.1-3.5):
//   u_out = w_dt dt F(u_deriv) + sum_i w_i u_prev_i            (Eq. 4)
// F: primitive variables (Eq. 9), MUSCL face values with the minmod limiter,
// Rusanov flux with Einfeldt's wave-speed estimate, flux divergence.
//
// Work decomposition (ours, not the paper's gang/collapse loops): one CTA per
// (block, T x T column tile).  The CTA marches k through the block keeping a
// ring of 5 planes of primitives (tile plus a 2-cell x/y halo, corners
// excluded) in shared memory, so each cell is converted to primitives once
// and each face flux is evaluated once.  The next plane is prefetched into
// registers while the current plane's fluxes are computed.  The kernel also
// stores the fluxes of refinement faces for flux fixing (Sec. 2.6) and, on
// the last stage of a step, reduces the CFL limit of its output (Sec. 3.2).
// 2D blocks are the single-plane case.
#pragma once

#include "common.cuh"

namespace amrb {

template <class real>
struct StageArgs {
    real *out;
    const real *deriv;
    const real *prev[4];
    real wprev[4];
    int nprev;
    double w_dt;
    const DevScalars *sc_in;     // dt
    DevScalars *sc;              // max speed accumulation, status
    const BlockInfo *info;
    real *bflux;                 // [slot][V][N^(D-1)]
    int update_dt;
    real gamma;
};

template <class real, int D>
struct Euler {
    static constexpr int V = D + 2;

    // primitive (rho, v, p) from conservative (rho, rho v, E)
    __device__ static __forceinline__ void prim(const real *U, real *w, real gam) {
        const real rho = U[0];
        const real ir = real(1) / rho;
        real ke = real(0);
#pragma unroll
        for (int d = 0; d < D; ++d) {
            w[1 + d] = U[1 + d] * ir;
            ke += w[1 + d] * U[1 + d];
        }
        w[0] = rho;
        w[D + 1] = (gam - real(1)) * (U[D + 1] - real(0.5) * ke);
    }

    // Rusanov flux along normal n (runtime) with the Einfeldt speed
    // a = |u_roe| + d_roe (Einfeldt 1988, as cited in Sec. 3.5).
    __device__ static __forceinline__ void flux(const real *wL, const real *wR, int n, real gam, real *F) {
        real vnL = wL[1], vnR = wR[1];
        if (D >= 2 && n == 1) { vnL = wL[2]; vnR = wR[2]; }
        if (D == 3 && n == 2) { vnL = wL[3]; vnR = wR[3]; }
        const real rL = wL[0], rR = wR[0], pL = wL[D + 1], pR = wR[D + 1];
        real v2L = real(0), v2R = real(0);
#pragma unroll
        for (int d = 0; d < D; ++d) {
            v2L += wL[1 + d] * wL[1 + d];
            v2R += wR[1 + d] * wR[1 + d];
        }
        const real gm1i = real(1) / (gam - real(1));
        const real EL = pL * gm1i + real(0.5) * rL * v2L;
        const real ER = pR * gm1i + real(0.5) * rR * v2R;
        const real sL = sqrt(rL), sR = sqrt(rR);
        const real inv = real(1) / (sL + sR);
        const real uroe = (sL * vnL + sR * vnR) * inv;
        const real du = vnR - vnL;
        const real d2 = (sL * (gam * pL / rL) + sR * (gam * pR / rR)) * inv + real(0.5) * sL * sR * inv * inv * du * du;
        const real a = fabs(uroe) + sqrt(d2);
        const real mL = rL * vnL, mR = rR * vnR;
        F[0] = real(0.5) * (mL + mR) - real(0.5) * a * (rR - rL);
#pragma unroll
        for (int d = 0; d < D; ++d) {
            real fl = mL * wL[1 + d], fr = mR * wR[1 + d];
            if (d == n) { fl += pL; fr += pR; }
            F[1 + d] = real(0.5) * (fl + fr) - real(0.5) * a * (rR * wR[1 + d] - rL * wL[1 + d]);
        }
        F[D + 1] = real(0.5) * ((EL + pL) * vnL + (ER + pR) * vnR) - real(0.5) * a * (ER - EL);
    }
};

template <class real, int D, int N, int NG, int T>
struct StageShape {
    static constexpr int V = D + 2;
    static constexpr int P = T + 4;                  // plane pitch (tile + 2-cell halo each side)
    static constexpr int R = (D == 3) ? 5 : 1;       // ring depth
    static constexpr int S = N + 2 * NG;
    static constexpr int NT = T * T;                 // threads
    static constexpr int TILES = (N / T) * (N / T);  // column tiles per block
    static constexpr int HALO_CELLS = T * P + 4 * T; // cells of a halo plane (corners excluded)
    static constexpr int LOADS = (HALO_CELLS + NT - 1) / NT;
    static constexpr int NFACE = T * (T + 1);
    static constexpr size_t smem_bytes() {
        return sizeof(real) * (size_t(R) * V * P * P + 2 * size_t(V) * NFACE);
    }
};

template <class real, int D, int N, int NG, int T>
__global__ void __launch_bounds__(T * T) k_stage(StageArgs<real> a, Geom g) {
    using Sh = StageShape<real, D, N, NG, T>;
    using E = Euler<real, D>;
    constexpr int V = Sh::V, P = Sh::P, S = Sh::S, NT = Sh::NT;
    constexpr int64_t NC = (D == 3) ? int64_t(S) * S * S : int64_t(S) * S;
    constexpr int NFACE = Sh::NFACE;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real *ring = reinterpret_cast<real *>(smem_raw);              // [R][V][P*P]
    real *Fx = ring + Sh::R * V * P * P;                           // [V][T][T+1]
    real *Fy = Fx + V * NFACE;                                     // [V][T+1][T]

    const int tid = threadIdx.x;
    const int b = blockIdx.x / Sh::TILES;
    const int tile = blockIdx.x - b * Sh::TILES;
    const int tx0 = (tile % (N / T)) * T, ty0 = (tile / (N / T)) * T;
    const int ti = tid % T, tj = tid / T;
    const BlockInfo info = a.info[b];
    const int lev = info.level;
    const real idx0 = real(g.inv_dx[lev][0]), idx1 = real(g.inv_dx[lev][1]);
    const real idx2 = (D == 3) ? real(g.inv_dx[lev][2]) : real(0);
    const real gam = a.gamma;
    const real dt_eff = real(a.w_dt * a.sc_in->dt);
    const real *ub = a.deriv + int64_t(b) * V * NC;

    bool nonphys = false;
    real vmax = real(0);

    // cell c of a plane -> tile-relative (ii, jj); halo planes skip corners
    auto plane_cell = [&](int c, bool halo, int &ii, int &jj) {
        if (!halo) { ii = c % T; jj = c / T; return; }
        if (c < T * P) { jj = c / P; ii = c % P - 2; return; }
        c -= T * P;
        const int r = c / T;
        ii = c % T;
        jj = (r < 2) ? r - 2 : T + r - 2;
    };
    auto gaddr = [&](int ii, int jj, int k) -> int64_t {
        return (int64_t(D == 3 ? k + NG : 0) * S + (ty0 + jj + NG)) * S + (tx0 + ii + NG);
    };
    // plane k has an x/y halo iff it is an interior plane (z-ghost planes only
    // feed the z stencil of the tile itself)
    auto is_halo_plane = [&](int k) { return D == 2 || (k >= 0 && k < N); };

    real pre[Sh::LOADS][V];
    auto prefetch = [&](int k) {
        const bool halo = is_halo_plane(k);
        const int ncells = halo ? Sh::HALO_CELLS : T * T;
#pragma unroll
        for (int l = 0; l < Sh::LOADS; ++l) {
            const int c = tid + l * NT;
            if (c < ncells) {
                int ii, jj;
                plane_cell(c, halo, ii, jj);
                const int64_t o = gaddr(ii, jj, k);
#pragma unroll
                for (int v = 0; v < V; ++v) pre[l][v] = ub[v * NC + o];
            }
        }
    };
    auto commit = [&](int k) {
        real *pl = ring + ((k + 2) % Sh::R) * V * P * P;
        const bool halo = is_halo_plane(k);
        const int ncells = halo ? Sh::HALO_CELLS : T * T;
#pragma unroll
        for (int l = 0; l < Sh::LOADS; ++l) {
            const int c = tid + l * NT;
            if (c < ncells) {
                int ii, jj;
                plane_cell(c, halo, ii, jj);
                real w[V];
                E::prim(pre[l], w, gam);
                nonphys |= !(w[0] > real(0)) || !(w[D + 1] > real(0));
                const int o = (jj + 2) * P + (ii + 2);
#pragma unroll
                for (int v = 0; v < V; ++v) pl[v * P * P + o] = w[v];
            }
        }
    };
    // flux through the face between cells c-1 and c along n, reading the
    // primitive stencil (c-2, c-1, c, c+1) at stride st from plane pointers
    auto face = [&](const real *p0, const real *p1, const real *p2, const real *p3, int st, int n, real *F) {
        real wL[V], wR[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int o = v * P * P;
            const real a0 = p0[o], a1 = p1[o + st], a2 = p2[o + 2 * st], a3 = p3[o + 3 * st];
            wL[v] = a1 + real(0.5) * minmod<real>(a1 - a0, a2 - a1);
            wR[v] = a2 - real(0.5) * minmod<real>(a2 - a1, a3 - a2);
        }
        nonphys |= !(wL[0] > real(0)) || !(wL[D + 1] > real(0)) || !(wR[0] > real(0)) || !(wR[D + 1] > real(0));
        E::flux(wL, wR, n, gam, F);
    };
    // x- or y-face q of the current plane into Fx / Fy
    auto xy_face = [&](const real *pl, int q, int n) {
        real F[V];
        if (n == 0) {
            const int jj = q / (T + 1), fi = q - jj * (T + 1);
            const real *p = pl + (jj + 2) * P + fi;          // cell fi-2
            face(p, p, p, p, 1, 0, F);
#pragma unroll
            for (int v = 0; v < V; ++v) Fx[v * NFACE + jj * (T + 1) + fi] = F[v];
        } else {
            const int fj = q / T, ii = q - fj * T;
            const real *p = pl + fj * P + ii + 2;            // cell (ii, fj-2)
            face(p, p, p, p, P, 1, F);
#pragma unroll
            for (int v = 0; v < V; ++v) Fy[v * NFACE + fj * T + ii] = F[v];
        }
    };
    const int nface_b = (D == 3) ? N * N : N;
    auto store_bflux = [&](int f, int t, const real *F) {
        const int slot = info.bslot[f];
        if (slot < 0) return;
        real *dst = a.bflux + int64_t(slot) * V * nface_b + t;
#pragma unroll
        for (int v = 0; v < V; ++v) dst[v * nface_b] = F[v];
    };

    // ---- prologue: planes -2 .. 2 (3D) or the single plane (2D)
    real Fz_lo[V];
    if (D == 3) {
        for (int k = -2; k <= 2; ++k) { prefetch(k); commit(k); }
    } else {
        prefetch(0);
        commit(0);
    }
    __syncthreads();
    if (D == 3) {
        const real *c0 = ring + ((-2 + 2) % 5) * V * P * P + (tj + 2) * P + ti + 2;
        const real *c1 = ring + ((-1 + 2) % 5) * V * P * P + (tj + 2) * P + ti + 2;
        const real *c2 = ring + ((0 + 2) % 5) * V * P * P + (tj + 2) * P + ti + 2;
        const real *c3 = ring + ((1 + 2) % 5) * V * P * P + (tj + 2) * P + ti + 2;
        face(c0, c1 - 1, c2 - 2, c3 - 3, 1, 2, Fz_lo);
        store_bflux(4, tx0 + ti + N * (ty0 + tj), Fz_lo);
    }

    const int nk = (D == 3) ? N : 1;
    for (int k = 0; k < nk; ++k) {
        if (D == 3 && k + 3 <= N + 1) prefetch(k + 3);
        const real *pl = ring + ((k + 2) % Sh::R) * V * P * P;
        xy_face(pl, tid, 0);
        xy_face(pl, tid, 1);
        if (tid < 2 * T) xy_face(pl, NT + (tid % T), tid < T ? 0 : 1);
        real Fz_hi[V];
        if (D == 3) {
            const int base = (tj + 2) * P + ti + 2;
            const real *c0 = ring + ((k - 1 + 2) % 5) * V * P * P + base;
            const real *c1 = ring + ((k + 0 + 2) % 5) * V * P * P + base;
            const real *c2 = ring + ((k + 1 + 2) % 5) * V * P * P + base;
            const real *c3 = ring + ((k + 2 + 2) % 5) * V * P * P + base;
            face(c0, c1 - 1, c2 - 2, c3 - 3, 1, 2, Fz_hi);
            if (k == N - 1) store_bflux(5, tx0 + ti + N * (ty0 + tj), Fz_hi);
        }
        if (D == 3 && k + 3 <= N + 1) commit(k + 3);
        __syncthreads();

        // ---- divergence and Runge-Kutta combination for cell (ti, tj, k)
        const int64_t o = gaddr(ti, tj, k);
        const int64_t ob = int64_t(b) * V * NC + o;
        real U[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            real du = (Fx[v * NFACE + tj * (T + 1) + ti] - Fx[v * NFACE + tj * (T + 1) + ti + 1]) * idx0 +
                      (Fy[v * NFACE + tj * T + ti] - Fy[v * NFACE + (tj + 1) * T + ti]) * idx1;
            if (D == 3) du += (Fz_lo[v] - Fz_hi[v]) * idx2;
            real acc = real(0);
            for (int q = 0; q < a.nprev; ++q) acc += a.wprev[q] * a.prev[q][ob + v * NC];
            U[v] = dt_eff * du + acc;
            a.out[ob + v * NC] = U[v];
        }
        // refinement-face fluxes of the tile's x/y block edges
        {
            const int gj = ty0 + tj, gi = tx0 + ti;
            real F[V];
            if (tx0 + ti == 0) {
                for (int v = 0; v < V; ++v) F[v] = Fx[v * NFACE + tj * (T + 1)];
                store_bflux(0, gj + N * k, F);
            }
            if (tx0 + ti == N - 1) {
                for (int v = 0; v < V; ++v) F[v] = Fx[v * NFACE + tj * (T + 1) + T];
                store_bflux(1, gj + N * k, F);
            }
            if (ty0 + tj == 0) {
                for (int v = 0; v < V; ++v) F[v] = Fy[v * NFACE + ti];
                store_bflux(2, gi + N * k, F);
            }
            if (ty0 + tj == N - 1) {
                for (int v = 0; v < V; ++v) F[v] = Fy[v * NFACE + T * T + ti];
                store_bflux(3, gi + N * k, F);
            }
        }
        if (a.update_dt) {
            // CFL limit of the new state; cells next to a coarse-side
            // refinement face are reduced after flux fixing instead
            const int gi = tx0 + ti, gj = ty0 + tj;
            const int m = info.fixmask;
            bool fixed = ((m & 1) && gi == 0) || ((m & 2) && gi == N - 1) || ((m & 4) && gj == 0) ||
                         ((m & 8) && gj == N - 1);
            if (D == 3) fixed = fixed || ((m & 16) && k == 0) || ((m & 32) && k == N - 1);
            if (!fixed) {
                real w[V];
                E::prim(U, w, gam);
                const real c = sqrt(gam * w[D + 1] / w[0]);
                real s = (fabs(w[1]) + c) * idx0 + (fabs(w[2]) + c) * idx1;
                if (D == 3) s += (fabs(w[3]) + c) * idx2;
                vmax = s > vmax ? s : vmax;
            }
        }
        if (D == 3) {
#pragma unroll
            for (int v = 0; v < V; ++v) Fz_lo[v] = Fz_hi[v];
        }
        __syncthreads();
    }

    // ---- CTA reductions: max speed and non-physical flag
    if (a.update_dt) {
        double m = double(vmax);
        for (int s = 16; s > 0; s >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, s));
        if ((tid & 31) == 0) atomic_max_nonneg(&a.sc->maxspeed_bits, m);
    }
    if (__syncthreads_or(nonphys) && tid == 0) raise_status(&a.sc->status, 7);
}

}  // namespace amrb
