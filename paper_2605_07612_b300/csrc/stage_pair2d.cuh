// FP32 2D stage kernel for two ghost layers: the sub-step of Eq. 5 (Sec.
// 3.1-3.5) on 2D blocks, with every thread owning two cells that are
// neighbours along x and all arithmetic on a pair in packed two-wide FP32
// instructions, as the 3D kernel of stage_pair.cuh does.
//
// One CTA per (block, T x T tile), T = min(N, 16) or 8 (autotuned), T*T/2
// threads.  A 2D tile is a single plane, so there is no ring: the CTA copies
// the tile and its x/y halo (corners excluded) as conservative pairs into
// shared memory with cp.async -- together with its cells' previous states --
// converts them to primitives in place, and then
//   [x and y fluxes of the tile] barrier [update] barrier.
// The thread mapping, halo numbering, conflict-free pitches and the tile's
// edge faces in one warp are those of the 3D kernel.
#pragma once

#include "stage_pair.cuh"

namespace amrb {

// the pair flux of the configured scheme (FLX 0 Rusanov, 1 HLL) for faces
// with normal NRM (0 x, 1 y; or NRM < 0 and the runtime normal n) from
// primitive states (rho, u, v, p): the grouped form of stage_pair.cuh
template <int FLX, int NRM>
__device__ __forceinline__ void pair_face_flux2d(const float2 *wL, const float2 *wR, int n, float gam, float gm1i, float2 *F) {
    pair_flux_grouped<2, FLX, NRM>(wL, wR, n, gam, gm1i, F);
}

// conservative (rho, rho u, rho v, E) -> primitive (rho, u, v, p) for a pair
__device__ __forceinline__ void pair_prim2d(const float2 *U, float2 *w, float gam) {
    const float2 ir = PF::rcp(U[0]);
    w[0] = U[0];
    w[1] = PF::mul(U[1], ir);
    w[2] = PF::mul(U[2], ir);
    float2 ke = PF::mul(w[1], U[1]);
    ke = PF::fma(w[2], U[2], ke);
    w[3] = PF::mul(PF::sp(gam - 1.f), PF::fma(ke, PF::sp(-0.5f), U[3]));
}

template <int N, int T_ = (N < 16 ? N : 16)>
struct PairShape2D {
    static constexpr int T = T_, NG = 2, S = N + 2 * NG, P = T + 4, PL = P * P, V = 4;
    static constexpr int NT = T * T / 2;
    static constexpr int TILES = (N / T) * (N / T);
    static constexpr int FXP = T == 16 ? 20 : T + 2;
    static constexpr int NFX = T * FXP;
    static constexpr int NFY = (T + 1) * T;
    static constexpr int FBUF = V * (NFX + NFY);
    __device__ static __forceinline__ int fy(int row, int c) {
        if constexpr (T == 16) return 32 * (row >> 1) + 16 * ((row ^ (row >> 2)) & 1) + c;
        else return row * T + c;
    }
    // two tile buffers (the next item's copies land in one while the CTA
    // works on the other), one flux buffer, two previous-state buffers
    static constexpr int PLB = V * PL;
    static constexpr size_t smem_bytes(int nprev) {
        return sizeof(float) * (2 * size_t(PLB) + size_t(FBUF)) + 2 * sizeof(float2) * size_t(nprev > 0 ? nprev : 0) * V * NT;
    }
};

// halo pair p of a tile (0 <= p < NPAIR): the pairs numbered row by row, the
// tile's rows with their x halo, the two y-halo rows below and above without
// the corners
template <int T>
__device__ __forceinline__ void pair2d_rc(int p, int &ii, int &jj) {
    constexpr int HP = T / 2, WP = (T + 4) / 2;
    if (p < 2 * HP) {
        jj = p / HP - 2;
        ii = 2 * (p % HP);
    } else if (p < 2 * HP + T * WP) {
        const int q = p - 2 * HP;
        jj = q / WP;
        ii = 2 * (q % WP) - 2;
    } else {
        const int q = p - 2 * HP - T * WP;
        jj = T + q / HP;
        ii = 2 * (q % HP);
    }
}

// thread -> the pair of cells it updates (row tj, first column ci)
template <int T>
__device__ __forceinline__ void pair2d_owner(int tid, int &ci, int &tj) {
    if constexpr (T == 16) {
        const int lane = tid & 31, q = (tid >> 5) * 2 + (lane >> 4);
        ci = 2 * (lane & 7);
        tj = (q & 3) + (q >> 2) * 8 + ((lane >> 3) & 1) * 4;
    } else {
        ci = 2 * (tid % (T / 2));
        tj = tid / (T / 2);
    }
}

__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Asynchronous copies of one item into tile buffer `buf`: the tile with its
// halo (in gather mode from the same-level neighbours) and the previous
// states of the thread's pair; one commit group.
template <int N, int TT, int NPREV>
__device__ __forceinline__ void pair2d_issue(const StageArgs<float> &a, int item, int buf) {
    using Sh = PairShape2D<N, TT>;
    constexpr int T = Sh::T, NG = Sh::NG, S = Sh::S, P = Sh::P, PL = Sh::PL, V = Sh::V, NT = Sh::NT;
    constexpr int64_t NC = int64_t(S) * S;
    constexpr int HP = T / 2, WP = (T + 4) / 2;
    constexpr int NPAIR = 2 * HP + T * WP + 2 * HP, REST = NPAIR - NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *pl = reinterpret_cast<float *>(smem_raw) + buf * Sh::PLB;
    float2 *stg = reinterpret_cast<float2 *>(reinterpret_cast<float *>(smem_raw) + 2 * Sh::PLB + Sh::FBUF) +
                  buf * (NPREV > 0 ? NPREV : 0) * V * NT;
    const int tid = threadIdx.x;
    const int b = item / Sh::TILES;
    const int tile = item - b * Sh::TILES;
    const int tx0 = (tile % (N / T)) * T, ty0 = (tile / (N / T)) * T;
    const BlockInfo &info = a.info[b];
    const int nb0 = a.gather ? info.nbr[0] : -1, nb1 = a.gather ? info.nbr[1] : -1;
    const int nb2 = a.gather ? info.nbr[2] : -1, nb3 = a.gather ? info.nbr[3] : -1;
    const float *ub = a.deriv + int64_t(b) * V * NC;
    auto gofs = [&](int i, int j) -> int64_t { return int64_t(j + NG) * S + (i + NG); };
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        const int p = l == 0 ? tid : (tid >= NT - REST ? NT + tid - (NT - REST) : -1);
        if (p < 0) continue;
        int ii, jj;
        pair2d_rc<T>(p, ii, jj);
        int gi = tx0 + ii, gj = ty0 + jj, nb = -1;
        if (gi < 0) { nb = nb0; gi += N; }
        else if (gi >= N) { nb = nb1; gi -= N; }
        else if (gj < 0) { nb = nb2; gj += N; }
        else if (gj >= N) { nb = nb3; gj -= N; }
        const float *src = nb >= 0 ? a.deriv + int64_t(nb) * V * NC + gofs(gi, gj) : ub + gofs(tx0 + ii, ty0 + jj);
        const int hoff = (jj + 2) * P + ii + 2;
#pragma unroll
        for (int v = 0; v < V; ++v) cp_async8(pl + hoff + v * PL, src + v * NC);
    }
    if constexpr (NPREV > 0) {
        int ci, tj;
        pair2d_owner<T>(tid, ci, tj);
        const int64_t ob = int64_t(b) * V * NC + gofs(tx0 + ci, ty0 + tj);
#pragma unroll
        for (int q = 0; q < NPREV; ++q)
#pragma unroll
            for (int v = 0; v < V; ++v) cp_async8(stg + (q * V + v) * NT + tid, a.prev[q] + ob + v * NC);
    }
    cp_async_commit();
}

// One item whose copies (pair2d_issue into buffer `buf`) have arrived:
// conversion to primitives, fluxes, update.
template <int N, int TT, int NPREV, int LIM, int FLX>
__device__ __forceinline__ void stage_pair2d_item(const StageArgs<float> &a, const Geom &g, int item, int buf) {
    using Sh = PairShape2D<N, TT>;
    constexpr int T = Sh::T, NG = Sh::NG, S = Sh::S, P = Sh::P, PL = Sh::PL, V = Sh::V, NT = Sh::NT;
    constexpr int FXP = Sh::FXP, NFX = Sh::NFX;
    constexpr int64_t NC = int64_t(S) * S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *pl = reinterpret_cast<float *>(smem_raw) + buf * Sh::PLB;        // [V][P*P] the tile and its halo
    float *Fx = reinterpret_cast<float *>(smem_raw) + 2 * Sh::PLB;          // [V][T][FXP]
    float *Fy = Fx + V * NFX;                                               // [V][T+1][T] (rows swizzled)
    const float2 *stg = reinterpret_cast<const float2 *>(Fx + Sh::FBUF) +
                        buf * (NPREV > 0 ? NPREV : 0) * V * NT;             // [NPREV][V][NT] previous states

    const int tid = threadIdx.x;
    const int b = item / Sh::TILES;
    const int tile = item - b * Sh::TILES;
    const int tx0 = (tile % (N / T)) * T, ty0 = (tile / (N / T)) * T;
    int ci, tj;
    pair2d_owner<T>(tid, ci, tj);
    const BlockInfo info = a.info[b];
    const int gc = info.gclass;
    const float idx0 = float(g.inv_dx[3 * gc]), idx1 = float(g.inv_dx[3 * gc + 1]);
    const float gam = a.gamma;
    const float gm1i = 1.f / (gam - 1.f);
    const float dt_eff = float(a.w_dt * a.sc_in[info.inst].dt);
    bool nonphys = false;
    float vmax = 0.f;

    auto gofs = [&](int i, int j) -> int64_t { return int64_t(j + NG) * S + (i + NG); };
    auto ld2 = [&](int v, int jj, int ii) -> float2 {
        return *reinterpret_cast<const float2 *>(pl + v * PL + (jj + 2) * P + (ii + 2));
    };

    // ---- conversion of the thread's copied pairs to primitives, in place
    constexpr int HP = T / 2, WP = (T + 4) / 2;
    constexpr int NPAIR = 2 * HP + T * WP + 2 * HP, REST = NPAIR - NT;
    static_assert(REST > 0 && REST <= NT, "two load rounds");
    int hoff[2];
    bool hval[2];
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        const int p = l == 0 ? tid : (tid >= NT - REST ? NT + tid - (NT - REST) : -1);
        hval[l] = p >= 0;
        hoff[l] = 0;
        if (p < 0) continue;
        int ii, jj;
        pair2d_rc<T>(p, ii, jj);
        hoff[l] = (jj + 2) * P + ii + 2;
    }
    const int64_t ob = int64_t(b) * V * NC + gofs(tx0 + ci, ty0 + tj);
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        if (!hval[l]) continue;
        float *at = pl + hoff[l];
        float2 U[V], w[V];
#pragma unroll
        for (int v = 0; v < V; ++v) U[v] = *reinterpret_cast<const float2 *>(at + v * PL);
        pair_prim2d(U, w, gam);
        nonphys |= !PF::positive(w[0]) || !PF::positive(w[3]);
#pragma unroll
        for (int v = 0; v < V; ++v) *reinterpret_cast<float2 *>(at + v * PL) = w[v];
    }
    __syncthreads();

    // ---- fluxes
    const int nface_b = N;
    auto store_bflux1 = [&](int f, int t, const float2 *F, bool hi) {
        const int sl = info.bslot[f];
        if (sl < 0) return;
        float *dst = a.bflux + int64_t(sl) * V * nface_b + t;
#pragma unroll
        for (int v = 0; v < V; ++v) dst[v * nface_b] = hi ? F[v].y : F[v].x;
    };
    auto store_bflux2 = [&](int f, int t, const float2 *F) {
        const int sl = info.bslot[f];
        if (sl < 0) return;
        float *dst = a.bflux + int64_t(sl) * V * nface_b + t;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            dst[v * nface_b] = F[v].x;
            dst[v * nface_b + 1] = F[v].y;
        }
    };
    {
        float2 wL[V], wR[V], F[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const float2 A = ld2(v, tj, ci - 2), B = ld2(v, tj, ci), C2 = ld2(v, tj, ci + 2);
            pair_states<LIM>(A, make_float2(A.y, B.x), B, make_float2(B.y, C2.x), wL[v], wR[v]);
        }
        pair_face_flux2d<FLX, 0>(wL, wR, 0, gam, gm1i, F);
#pragma unroll
        for (int v = 0; v < V; ++v) *reinterpret_cast<float2 *>(Fx + v * NFX + tj * FXP + ci) = F[v];
        if (ci == 0 && tx0 == 0) store_bflux1(0, ty0 + tj, F, false);
#pragma unroll
        for (int v = 0; v < V; ++v)
            pair_states<LIM>(ld2(v, tj - 2, ci), ld2(v, tj - 1, ci), ld2(v, tj, ci), ld2(v, tj + 1, ci), wL[v], wR[v]);
        pair_face_flux2d<FLX, 1>(wL, wR, 1, gam, gm1i, F);
#pragma unroll
        for (int v = 0; v < V; ++v) *reinterpret_cast<float2 *>(Fy + v * (T + 1) * T + Sh::fy(tj, ci)) = F[v];
        if (tj == 0 && ty0 == 0) store_bflux2(2, tx0 + ci, F);
        // the tile's upper edge faces, both in the first warp: lanes r < T/2
        // take x-face T of rows (2r, 2r+1), lanes T/2 + r y-face T of
        // columns (2r, 2r+1); one flux evaluation with a runtime normal
        if (tid < T) {
            const bool isx = tid < T / 2;
            const int r = isx ? tid : tid - T / 2;
            const int base = isx ? (2 * r + 2) * P + T : T * P + 2 + 2 * r;
            const int st = isx ? 1 : P, po = isx ? P : 1;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const float *b0 = pl + v * PL + base;
                pair_states<LIM>(make_float2(b0[0], b0[po]), make_float2(b0[st], b0[st + po]),
                                 make_float2(b0[2 * st], b0[2 * st + po]), make_float2(b0[3 * st], b0[3 * st + po]), wL[v], wR[v]);
            }
            pair_face_flux2d<FLX, -1>(wL, wR, isx ? 0 : 1, gam, gm1i, F);
            if (isx) {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    Fx[v * NFX + (2 * r) * FXP + T] = F[v].x;
                    Fx[v * NFX + (2 * r + 1) * FXP + T] = F[v].y;
                }
                if (tx0 + T == N) {
                    store_bflux1(1, ty0 + 2 * r, F, false);
                    store_bflux1(1, ty0 + 2 * r + 1, F, true);
                }
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) *reinterpret_cast<float2 *>(Fy + v * (T + 1) * T + Sh::fy(T, 2 * r)) = F[v];
                if (ty0 + T == N) store_bflux2(3, tx0 + 2 * r, F);
            }
        }
    }
    __syncthreads();

    // ---- update of the thread's pair
    {
        const float2 i0 = PF::sp(idx0), i1 = PF::sp(idx1), dte = PF::sp(dt_eff);
        float2 U[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const float2 x0 = *reinterpret_cast<const float2 *>(Fx + v * NFX + tj * FXP + ci);
            const float2 x1 = *reinterpret_cast<const float2 *>(Fx + v * NFX + tj * FXP + ci + 2);
            const float2 y0 = *reinterpret_cast<const float2 *>(Fy + v * (T + 1) * T + Sh::fy(tj, ci));
            const float2 y1 = *reinterpret_cast<const float2 *>(Fy + v * (T + 1) * T + Sh::fy(tj + 1, ci));
            float2 du = PF::mul(PF::sub(x0, make_float2(x0.y, x1.x)), i0);
            du = PF::fma(PF::sub(y0, y1), i1, du);
            if (v > 0 && a.gravity_on) {
                // S = (0, rho g, rho g.u) from the primitives of the pair
                const float2 rho = ld2(0, tj, ci);
                if (v < 3) {
                    du = PF::fma(rho, PF::sp(a.grav[v - 1]), du);
                } else {
                    const float2 vg = PF::fma(ld2(2, tj, ci), PF::sp(a.grav[1]), PF::mul(ld2(1, tj, ci), PF::sp(a.grav[0])));
                    du = PF::fma(rho, vg, du);
                }
            }
            float2 acc = PF::sp(0.f);
            if constexpr (NPREV > 0) {
#pragma unroll
                for (int q = 0; q < NPREV; ++q) acc = PF::fma(PF::sp(a.wprev[q]), stg[(q * V + v) * NT + tid], acc);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (q < a.nprev)
                        acc = PF::fma(PF::sp(a.wprev[q]), *reinterpret_cast<const float2 *>(a.prev[q] + ob + v * NC), acc);
            }
            U[v] = PF::fma(dte, du, acc);
            *reinterpret_cast<float2 *>(a.out + ob + v * NC) = U[v];
        }
        // complete the row's DRAM sectors: the output's x-ghost cells
        if (tx0 + ci == 0 || tx0 + ci + 1 == N - 1) {
            const int64_t og = ob + (tx0 + ci == 0 ? -NG : 2);
#pragma unroll
            for (int v = 0; v < V; ++v) *reinterpret_cast<float2 *>(a.out + og + v * NC) = PF::sp(0.f);
        }
        if (a.update_dt) {
            const int gi = tx0 + ci, gj = ty0 + tj;
            const int m = info.fixmask;
            const bool rowfix = ((m & 4) && gj == 0) || ((m & 8) && gj == N - 1);
            const bool fx0 = rowfix || ((m & 1) && gi == 0);
            const bool fx1 = rowfix || ((m & 2) && gi + 1 == N - 1);
            float2 w[V];
            pair_prim2d(U, w, gam);
            const float2 c2 = PF::mul(PF::mul(PF::sp(gam), w[3]), PF::rcp(w[0]));
            const float2 c = PF::mul(c2, PF::rsqrt(c2));
            float2 s = PF::mul(PF::add(PF::abs(w[1]), c), i0);
            s = PF::fma(PF::add(PF::abs(w[2]), c), i1, s);
            if (!fx0) vmax = s.x > vmax ? s.x : vmax;
            if (!fx1) vmax = s.y > vmax ? s.y : vmax;
        }
    }
    __syncthreads();   // shared memory is reused by the CTA's next item

    if (a.update_dt) {
        double mx = double(vmax);
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((tid & 31) == 0) atomic_max_nonneg(&a.sc[info.inst].maxspeed_bits, mx);
    }
    if (__syncthreads_or(nonphys) && tid == 0) raise_status(&a.sc[0].status, 7);
}

// CTAs take items with a grid stride; the copies of a CTA's next item are
// issued before it works on the current one.  16 x 16 tiles: six CTAs per SM
// for one previous state (80 registers), five for two (their staging takes
// more shared memory).
template <int N, int TT, int NPREV, int LIM, int FLX>
__global__ void __launch_bounds__(PairShape2D<N, TT>::NT, (TT >= 16 ? (NPREV == 1 ? 6 : 5) : 2)) k_stage_pair2d(StageArgs<float> a, Geom g) {
    int item = blockIdx.x;
    if (item >= a.n_items) return;
    pair2d_issue<N, TT, NPREV>(a, item, 0);
    for (int buf = 0; item < a.n_items; item += gridDim.x, buf ^= 1) {
        const int next = item + int(gridDim.x);
        if (next < a.n_items) {
            pair2d_issue<N, TT, NPREV>(a, next, buf ^ 1);
            cp_async_wait_1();
        } else {
            cp_async_wait_all();
        }
        stage_pair2d_item<N, TT, NPREV, LIM, FLX>(a, g, item, buf);
    }
}

}  // namespace amrb
