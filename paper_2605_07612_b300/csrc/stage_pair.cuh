// FP32 stage kernel for 2 ghost layers: the same computation as k_stage
// (Sec. 3.1-3.5, Eq. 5), organised so that every thread owns two cells that
// are neighbours along x.  All arithmetic on such a pair runs as packed
// two-wide FP32 instructions (add/mul/fma .f32x2 of sm_100-class GPUs), and
// every shared- and global-memory access of a pair is one aligned 8-byte
// access.  The flux is Rusanov's or HLL (template parameter).
//
// One CTA per (block, T x T column tile), T = min(N, 16) or 8 (autotuned),
// T*T/2 threads (128 for T = 16); thread (ip, tj) owns
// cells (2ip, 2ip+1) of row tj.  The CTA marches k with a ring of
// primitive variables in shared memory (4 planes: the z face state of the
// plane above is carried in registers).  Per plane k:
//   [copy of plane k's previous states | fluxes of plane k | commit of plane
//    k+3] barrier [update of plane k] barrier
// The previous states travel by cp.async into per-thread shared slots while
// the fluxes are computed, so the update does not wait on global loads.  Face
// states (MUSCL with minmod) are formed in the flux phase from the ring: an
// x-face pair reads three aligned pairs of a row, a y- or z-face pair four.
// The T x-faces and T y-faces left over at the tile's upper edges are taken
// by the first warp in one flux evaluation (T/2 lanes per normal, the normal
// chosen at run time); the second round of halo loads goes to the last
// warps.
#pragma once

#include "stage.cuh"

namespace amrb {

struct PF {
    __device__ static __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
    __device__ static __forceinline__ float2 sp(float a) { return make_float2(a, a); }
    __device__ static __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
    __device__ static __forceinline__ float2 sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
    __device__ static __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
    __device__ static __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
    __device__ static __forceinline__ float2 rsqrt(float2 a) { return make_float2(rsqrt_ftz(a.x), rsqrt_ftz(a.y)); }
    __device__ static __forceinline__ float2 rcp(float2 a) { return make_float2(rcp_ftz(a.x), rcp_ftz(a.y)); }
    __device__ static __forceinline__ float2 abs(float2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
    // 0.5 minmod(a, b) = qs(a, b) * mabs(a, b): qs = (sign a + sign b) / 4 is
    // +-1/2 when the signs agree and 0 otherwise; mabs = min(|a|, |b|) (a zero
    // gives 0).  The product is exact, so w + 0.5 minmod(a, b) is the single
    // rounding fma(qs, mabs, w).
    __device__ static __forceinline__ float sg(float a) { return __uint_as_float((__float_as_uint(a) & 0x80000000u) | 0x3e800000u); }
    __device__ static __forceinline__ float2 qs(float2 a, float2 b) {
        return add(make_float2(sg(a.x), sg(a.y)), make_float2(sg(b.x), sg(b.y)));
    }
    __device__ static __forceinline__ float2 mabs(float2 a, float2 b) {
        return make_float2(fminf(fabsf(a.x), fabsf(b.x)), fminf(fabsf(a.y), fabsf(b.y)));
    }
    __device__ static __forceinline__ float2 nmabs(float2 a, float2 b) {
        return make_float2(fmaxf(-fabsf(a.x), -fabsf(b.x)), fmaxf(-fabsf(a.y), -fabsf(b.y)));
    }
    __device__ static __forceinline__ bool positive(float2 a) { return a.x > 0.f && a.y > 0.f; }
};

constexpr int kPairV = 5;   // 3D Euler variables

// Bulk prefetch of a contiguous range into L2 by the TMA unit (no registers,
// no shared memory).  Address and size must be multiples of 16 bytes.
__device__ __forceinline__ void l2_prefetch(const void *p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// 8-byte asynchronous global -> shared copy (cp.async, L1-allocating) and
// its group commit / wait.
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    const unsigned d = unsigned(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Rusanov / Einfeldt flux of a pair of faces with the same normal n
// (compile-time NRM >= 0, or runtime n when NRM < 0).
template <int NRM>
__device__ __forceinline__ void pair_flux(const float2 *wL, const float2 *wR, int n, float gam, float gm1i, float2 *F) {
    const int nn = NRM >= 0 ? NRM : n;
    float2 vnL, vnR;
    if (NRM >= 0) {
        vnL = wL[1 + (NRM >= 0 ? NRM : 0)];
        vnR = wR[1 + (NRM >= 0 ? NRM : 0)];
    } else {
        vnL = nn == 0 ? wL[1] : (nn == 1 ? wL[2] : wL[3]);
        vnR = nn == 0 ? wR[1] : (nn == 1 ? wR[2] : wR[3]);
    }
    const float2 rL = wL[0], rR = wR[0], pL = wL[4], pR = wR[4];
    const float2 qL = PF::rsqrt(rL), qR = PF::rsqrt(rR);
    const float2 sL = PF::mul(rL, qL), sR = PF::mul(rR, qR);            // sqrt(rho)
    const float2 iL = PF::mul(qL, qL), iR = PF::mul(qR, qR);            // 1 / rho
    const float2 inv = PF::rcp(PF::add(sL, sR));
    const float2 g2 = PF::sp(gam);
    const float2 c2L = PF::mul(PF::mul(g2, pL), iL), c2R = PF::mul(PF::mul(g2, pR), iR);
    const float2 uroe = PF::mul(PF::fma(sL, vnL, PF::mul(sR, vnR)), inv);
    const float2 du = PF::sub(vnR, vnL);
    const float2 h = PF::mul(PF::mul(PF::mul(sL, sR), PF::mul(inv, inv)), PF::sp(0.5f));
    const float2 d2 = PF::fma(PF::mul(h, du), du, PF::mul(PF::fma(sL, c2L, PF::mul(sR, c2R)), inv));
    const float2 d = PF::mul(d2, PF::rsqrt(d2));
    const float2 a = PF::add(PF::abs(uroe), d);
    float2 v2L = PF::mul(wL[1], wL[1]), v2R = PF::mul(wR[1], wR[1]);
    v2L = PF::fma(wL[2], wL[2], v2L);
    v2R = PF::fma(wR[2], wR[2], v2R);
    v2L = PF::fma(wL[3], wL[3], v2L);
    v2R = PF::fma(wR[3], wR[3], v2R);
    const float2 half = PF::sp(0.5f);
    const float2 EL = PF::fma(pL, PF::sp(gm1i), PF::mul(PF::mul(half, rL), v2L));
    const float2 ER = PF::fma(pR, PF::sp(gm1i), PF::mul(PF::mul(half, rR), v2R));
    const float2 nha = PF::mul(a, PF::sp(-0.5f));
    const float2 mL = PF::mul(rL, vnL), mR = PF::mul(rR, vnR);
    F[0] = PF::fma(nha, PF::sub(rR, rL), PF::mul(half, PF::add(mL, mR)));
#pragma unroll
    for (int d3 = 0; d3 < 3; ++d3) {
        float2 fl = PF::fma(mL, wL[1 + d3], PF::mul(mR, wR[1 + d3]));
        if (d3 == nn) fl = PF::add(fl, PF::add(pL, pR));
        const float2 jump = PF::sub(PF::mul(rR, wR[1 + d3]), PF::mul(rL, wL[1 + d3]));
        F[1 + d3] = PF::fma(nha, jump, PF::mul(half, fl));
    }
    const float2 fe = PF::fma(PF::add(EL, pL), vnL, PF::mul(PF::add(ER, pR), vnR));
    F[4] = PF::fma(nha, PF::sub(ER, EL), PF::mul(half, fe));
}

// HLL flux (Harten, Lax and van Leer) of a pair of faces with the same
// Einfeldt estimates as pair_flux: sL = min(u_roe - d, 0), sR = max(u_roe + d,
// 0), F = (sR F_L - sL F_R + sL sR (U_R - U_L)) / (sR - sL).
template <int NRM>
__device__ __forceinline__ void pair_flux_hll(const float2 *wL, const float2 *wR, int n, float gam, float gm1i, float2 *F) {
    const int nn = NRM >= 0 ? NRM : n;
    float2 vnL, vnR;
    if (NRM >= 0) {
        vnL = wL[1 + (NRM >= 0 ? NRM : 0)];
        vnR = wR[1 + (NRM >= 0 ? NRM : 0)];
    } else {
        vnL = nn == 0 ? wL[1] : (nn == 1 ? wL[2] : wL[3]);
        vnR = nn == 0 ? wR[1] : (nn == 1 ? wR[2] : wR[3]);
    }
    const float2 rL = wL[0], rR = wR[0], pL = wL[4], pR = wR[4];
    const float2 qL = PF::rsqrt(rL), qR = PF::rsqrt(rR);
    const float2 sqL = PF::mul(rL, qL), sqR = PF::mul(rR, qR);
    const float2 iL = PF::mul(qL, qL), iR = PF::mul(qR, qR);
    const float2 inv = PF::rcp(PF::add(sqL, sqR));
    const float2 g2 = PF::sp(gam);
    const float2 c2L = PF::mul(PF::mul(g2, pL), iL), c2R = PF::mul(PF::mul(g2, pR), iR);
    const float2 uroe = PF::mul(PF::fma(sqL, vnL, PF::mul(sqR, vnR)), inv);
    const float2 du = PF::sub(vnR, vnL);
    const float2 h = PF::mul(PF::mul(PF::mul(sqL, sqR), PF::mul(inv, inv)), PF::sp(0.5f));
    const float2 d2 = PF::fma(PF::mul(h, du), du, PF::mul(PF::fma(sqL, c2L, PF::mul(sqR, c2R)), inv));
    const float2 d = PF::mul(d2, PF::rsqrt(d2));
    const float2 lo = PF::sub(uroe, d), hi = PF::add(uroe, d);
    const float2 sL = make_float2(fminf(lo.x, 0.f), fminf(lo.y, 0.f));
    const float2 sR = make_float2(fmaxf(hi.x, 0.f), fmaxf(hi.y, 0.f));
    const float2 iw = PF::rcp(PF::sub(sR, sL)), sLR = PF::mul(sL, sR);
    float2 v2L = PF::mul(wL[1], wL[1]), v2R = PF::mul(wR[1], wR[1]);
    v2L = PF::fma(wL[2], wL[2], v2L);
    v2R = PF::fma(wR[2], wR[2], v2R);
    v2L = PF::fma(wL[3], wL[3], v2L);
    v2R = PF::fma(wR[3], wR[3], v2R);
    const float2 half = PF::sp(0.5f);
    const float2 EL = PF::fma(pL, PF::sp(gm1i), PF::mul(PF::mul(half, rL), v2L));
    const float2 ER = PF::fma(pR, PF::sp(gm1i), PF::mul(PF::mul(half, rR), v2R));
    const float2 mL = PF::mul(rL, vnL), mR = PF::mul(rR, vnR);
    // (sR fL - sL fR + sL sR jump) / (sR - sL)
    auto comb = [&](float2 fL, float2 fR, float2 jump) {
        return PF::mul(PF::fma(sLR, jump, PF::sub(PF::mul(sR, fL), PF::mul(sL, fR))), iw);
    };
    F[0] = comb(mL, mR, PF::sub(rR, rL));
#pragma unroll
    for (int d3 = 0; d3 < 3; ++d3) {
        float2 fL = PF::mul(mL, wL[1 + d3]), fR = PF::mul(mR, wR[1 + d3]);
        if (d3 == nn) {
            fL = PF::add(fL, pL);
            fR = PF::add(fR, pR);
        }
        F[1 + d3] = comb(fL, fR, PF::sub(PF::mul(rR, wR[1 + d3]), PF::mul(rL, wL[1 + d3])));
    }
    F[4] = comb(PF::mul(PF::add(EL, pL), vnL), PF::mul(PF::add(ER, pR), vnR), PF::sub(ER, EL));
}

// the pair flux of the configured scheme (FLX 0 Rusanov, 1 HLL)
template <int FLX, int NRM>
__device__ __forceinline__ void pair_face_flux(const float2 *wL, const float2 *wR, int n, float gam, float gm1i, float2 *F) {
    if constexpr (FLX == 1) pair_flux_hll<NRM>(wL, wR, n, gam, gm1i, F);
    else pair_flux<NRM>(wL, wR, n, gam, gm1i, F);
}

// Half of the limited slope of a pair of cells from their one-sided
// differences a (left) and b (right): LIM 1 monotonized central (Eq. 1 with
// theta = 2: sign min(|a|, |b|, |a + b| / 4) when the signs agree), LIM 2 van
// Leer (ab / (a + b) when ab > 0); zero when the signs differ.  (LIM 0,
// minmod, is fused into the face states below.)
template <int LIM>
__device__ __forceinline__ float2 pair_half_slope(float2 a, float2 b) {
    if constexpr (LIM == 2) {
        const float2 p = PF::mul(a, b);
        const float2 h = PF::mul(p, PF::rcp(PF::add(a, b)));
        return make_float2(p.x > 0.f ? h.x : 0.f, p.y > 0.f ? h.y : 0.f);
    } else {
        const float2 q = PF::qs(a, b);                        // +-1/2 or 0
        const float2 c = PF::mul(PF::add(a, b), PF::sp(0.25f));
        const float2 m = make_float2(fminf(fminf(fabsf(a.x), fabsf(b.x)), fabsf(c.x)),
                                     fminf(fminf(fabsf(a.y), fabsf(b.y)), fabsf(c.y)));
        return PF::mul(PF::add(q, q), m);
    }
}

// face states of a pair of faces from the four pairs of cells around them
// (c-2, c-1, c, c+1 along the face normal)
template <int LIM>
__device__ __forceinline__ void pair_states(float2 w0, float2 w1, float2 w2, float2 w3, float2 &L, float2 &R) {
    const float2 d01 = PF::sub(w1, w0), d12 = PF::sub(w2, w1), d23 = PF::sub(w3, w2);
    if constexpr (LIM == 0) {
        L = PF::fma(PF::qs(d01, d12), PF::mabs(d01, d12), w1);
        R = PF::fma(PF::qs(d12, d23), PF::nmabs(d12, d23), w2);
    } else {
        L = PF::add(w1, pair_half_slope<LIM>(d01, d12));
        R = PF::sub(w2, pair_half_slope<LIM>(d12, d23));
    }
}

// minus and plus states of a pair of cells w1 from its neighbours w0, w2
template <int LIM>
__device__ __forceinline__ void pair_cell_states(float2 w0, float2 w1, float2 w2, float2 &minus, float2 &plus) {
    const float2 d01 = PF::sub(w1, w0), d12 = PF::sub(w2, w1);
    if constexpr (LIM == 0) {
        const float2 q = PF::qs(d01, d12);
        minus = PF::fma(q, PF::nmabs(d01, d12), w1);
        plus = PF::fma(q, PF::mabs(d01, d12), w1);
    } else {
        const float2 h = pair_half_slope<LIM>(d01, d12);
        minus = PF::sub(w1, h);
        plus = PF::add(w1, h);
    }
}

// conservative -> primitive for a pair of cells
__device__ __forceinline__ void pair_prim(const float2 *U, float2 *w, float gam) {
    const float2 ir = PF::rcp(U[0]);
    w[0] = U[0];
    w[1] = PF::mul(U[1], ir);
    w[2] = PF::mul(U[2], ir);
    w[3] = PF::mul(U[3], ir);
    float2 ke = PF::mul(w[1], U[1]);
    ke = PF::fma(w[2], U[2], ke);
    ke = PF::fma(w[3], U[3], ke);
    w[4] = PF::mul(PF::sp(gam - 1.f), PF::fma(ke, PF::sp(-0.5f), U[4]));
}

// T: the staging tile (T x T columns per CTA); 16 by default (N for N = 8),
// 8 as the autotuner's alternative for larger blocks.
template <int N, int T_ = (N < 16 ? N : 16)>
struct PairShape {
    static constexpr int T = T_, NG = 2, S = N + 2 * NG, P = T + 4, PL = P * P, R = 4, V = 5;
    static constexpr int NT = T * T / 2;              // threads: one per cell pair of a plane
    static constexpr int TILES = (N / T) * (N / T);
    // x-flux row pitch (T + 1 faces + pad); for T = 16 it is 20 words, so the
    // rows r and r + 4 that a half-warp touches fall into opposite bank halves
    static constexpr int FXP = T == 16 ? 20 : T + 2;
    static constexpr int NFX = T * FXP;
    static constexpr int NFY = (T + 1) * T;
    static constexpr int FBUF = V * (NFX + NFY);      // one flux buffer
    static constexpr int LOADS = ((T * T + 8 * T) / 2 + NT - 1) / NT;   // halo pairs without corners
    // y-flux row `row` (T + 1 rows of T faces): for T = 16 rows 2m and 2m + 1
    // share a 32-word line, their halves swapped when bit 2 of the row is
    // set, so rows r and r + 4 (one half-warp) use opposite bank halves
    __device__ static __forceinline__ int fy(int row, int c) {
        if constexpr (T == 16) return 32 * (row >> 1) + 16 * ((row ^ (row >> 2)) & 1) + c;
        else return row * T + c;
    }
    // ring, one flux buffer, and (nprev > 0) each thread's previous-state
    // pairs of the plane being updated [nprev][V][NT]
    static constexpr size_t smem_bytes(int nprev) {
        return sizeof(float) * (size_t(R) * V * PL + size_t(FBUF)) + sizeof(float2) * size_t(nprev > 0 ? nprev : 0) * V * NT;
    }
};

// NPREV >= 0: the number of previous states, fixed at compile time (Heun's two
// stages use 1 and 2); -1 reads it from the arguments.  FLX: 0 Rusanov, 1 HLL.
template <int N, int TT, int NPREV, int LIM, int FLX>
__device__ __forceinline__ void stage_pair_item(const StageArgs<float> &a, const Geom &g, int item) {
    using Sh = PairShape<N, TT>;
    constexpr int T = Sh::T, NG = Sh::NG, S = Sh::S, P = Sh::P, PL = Sh::PL, V = Sh::V, NT = Sh::NT;
    constexpr int FXP = Sh::FXP, NFX = Sh::NFX, FBUF = Sh::FBUF;
    constexpr int64_t NC = int64_t(S) * S * S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *ring = reinterpret_cast<float *>(smem_raw);         // [R][V][P*P]
    float *fbuf = ring + Sh::R * V * PL;                        // Fx [V][T][FXP], Fy [V][T+1][T]
    float2 *stg = reinterpret_cast<float2 *>(fbuf + FBUF);      // [NPREV][V][NT] previous states

    const int tid = threadIdx.x;
    const int b = item / Sh::TILES;
    const int tile = item - b * Sh::TILES;
    const int tx0 = (tile % (N / T)) * T, ty0 = (tile / (N / T)) * T;
    // thread -> (row tj, pair ip).  For T = 16 the two 8-lane row groups of a
    // half-warp take rows r and r + 4: 80 words apart in the ring (pitch 20),
    // i.e. opposite halves of the 32 banks, so a half-warp's 8-byte accesses
    // to a ring row never conflict.
    int ip, tj;
    if constexpr (T == 16) {
        const int lane = tid & 31, q = (tid >> 5) * 2 + (lane >> 4);
        ip = lane & 7;
        tj = (q & 3) + (q >> 2) * 8 + ((lane >> 3) & 1) * 4;
    } else {
        ip = tid % (T / 2);
        tj = tid / (T / 2);
    }
    const int ci = 2 * ip;                                      // first cell of the pair
    const BlockInfo info = a.info[b];
    const int gc = info.gclass;
    const float idx0 = float(g.inv_dx[3 * gc]), idx1 = float(g.inv_dx[3 * gc + 1]), idx2 = float(g.inv_dx[3 * gc + 2]);
    const float gam = a.gamma;
    const float gm1i = 1.f / (gam - 1.f);
    const float dt_eff = float(a.w_dt * a.sc_in[info.inst].dt);
    const float *__restrict__ ub = a.deriv + int64_t(b) * V * NC;
    // same-level neighbours (scalars: a runtime-indexed array would live in local memory)
    const int nb0 = a.gather ? info.nbr[0] : -1, nb1 = a.gather ? info.nbr[1] : -1;
    const int nb2 = a.gather ? info.nbr[2] : -1, nb3 = a.gather ? info.nbr[3] : -1;
    const int nb4 = a.gather ? info.nbr[4] : -1, nb5 = a.gather ? info.nbr[5] : -1;

    bool nonphys = false;
    float vmax = 0.f;

    auto slot = [&](int k) -> float * { return ring + ((k + 2) % Sh::R) * V * PL; };
    auto gofs = [&](int i, int j, int k) -> int64_t { return (int64_t(k + NG) * S + (j + NG)) * S + (i + NG); };
    // source of cell (tx0 + ii, ty0 + jj, k): this block, or a same-level
    // neighbour's interior in gather mode
    auto src_of = [&](int ii, int jj, int k, int64_t &o) -> const float * {
        int gi = tx0 + ii, gj = ty0 + jj, gk = k, nb = -1;
        if (gi < 0) { nb = nb0; gi += N; }
        else if (gi >= N) { nb = nb1; gi -= N; }
        else if (gj < 0) { nb = nb2; gj += N; }
        else if (gj >= N) { nb = nb3; gj -= N; }
        else if (gk < 0) { nb = nb4; gk += N; }
        else if (gk >= N) { nb = nb5; gk -= N; }
        if (nb >= 0) {
            o = gofs(gi, gj, gk);
            return a.deriv + int64_t(nb) * V * NC;
        }
        o = gofs(tx0 + ii, ty0 + jj, k);
        return ub;
    };
    // ---- plane loading: conservative pairs into registers, then primitives
    // into the ring.  An interior plane (0 <= k < N) needs the tile and its
    // x/y halo without the corners: NPAIR = (T^2 + 8T) / 2 pairs, numbered row
    // by row.  Every thread takes pair tid; the remaining REST pairs go to the
    // last REST threads (warps 2 and 3 for T = 16, whose first warp
    // computes the tile's edge faces).  The source of a thread's pairs does
    // not change with k, so its address at k = 0 is kept.  The planes k < 0
    // and k >= N need only the tile: thread tid takes its own pair.
    constexpr int HP = T / 2, WP = (T + 4) / 2;
    constexpr int NPAIR = 2 * HP + T * WP + 2 * HP, REST = NPAIR - NT;
    static_assert(Sh::LOADS == 2 && REST > 0 && REST <= NT, "two load rounds per plane");
    auto pair_rc = [&](int p, int &ii, int &jj) {
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
    };
    const float *hsrc[2];
    int hoff[2];
    bool hval[2];
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        const int p = l == 0 ? tid : (tid >= NT - REST ? NT + tid - (NT - REST) : -1);
        hval[l] = p >= 0;
        hsrc[l] = ub;
        hoff[l] = 0;
        if (p >= 0) {
            int ii, jj;
            pair_rc(p, ii, jj);
            int64_t o;
            hsrc[l] = src_of(ii, jj, 0, o) + o;
            hoff[l] = (jj + 2) * P + ii + 2;
        }
    }
    const int own_off = (tid / (T / 2) + 2) * P + 2 * (tid % (T / 2)) + 2;

    float2 pre[Sh::LOADS][V];
    auto prefetch = [&](int k) {
        if (k >= 0 && k < N) {
            const int64_t ko = int64_t(k) * S * S;
#pragma unroll
            for (int l = 0; l < 2; ++l)
                if (hval[l])
#pragma unroll
                    for (int v = 0; v < V; ++v) pre[l][v] = *reinterpret_cast<const float2 *>(hsrc[l] + ko + v * NC);
        } else {
            int64_t o;
            const float *src = src_of(2 * (tid % (T / 2)), tid / (T / 2), k, o);
#pragma unroll
            for (int v = 0; v < V; ++v) pre[0][v] = *reinterpret_cast<const float2 *>(src + v * NC + o);
        }
    };
    auto commit_pair = [&](float *dst, const float2 *U) {
        float2 w[V];
        pair_prim(U, w, gam);
        nonphys |= !PF::positive(w[0]) || !PF::positive(w[4]);
#pragma unroll
        for (int v = 0; v < V; ++v) *reinterpret_cast<float2 *>(dst + v * PL) = w[v];
    };
    auto commit = [&](int k) {
        float *pl = slot(k);
        if (k >= 0 && k < N) {
#pragma unroll
            for (int l = 0; l < 2; ++l)
                if (hval[l]) commit_pair(pl + hoff[l], pre[l]);
        } else {
            commit_pair(pl + own_off, pre[0]);
        }
    };
    auto ld2 = [&](const float *pl, int v, int jj, int ii) -> float2 {
        return *reinterpret_cast<const float2 *>(pl + v * PL + (jj + 2) * P + (ii + 2));
    };

    const int nface_b = N * N;
    auto store_bflux1 = [&](int f, int t, float Fv0, float Fv1, float Fv2, float Fv3, float Fv4) {
        const int sl = info.bslot[f];
        if (sl < 0) return;
        float *dst = a.bflux + int64_t(sl) * V * nface_b + t;
        dst[0] = Fv0;
        dst[nface_b] = Fv1;
        dst[2 * nface_b] = Fv2;
        dst[3 * nface_b] = Fv3;
        dst[4 * nface_b] = Fv4;
    };
    // store both faces of a pair (tangential indices t and t + 1)
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

    // ---- fluxes of plane k into buffer fb
    float2 FzA[V], FzB[V];   // z fluxes below / above the plane being updated
    float2 zP[V];            // plus z state of the pair at the plane whose fluxes come next
    auto fluxes = [&](int k, float *fb, float2 *Fz_new) {
        float *Fx = fb, *Fy = fb + V * NFX;
        const float *pl = slot(k);
        float2 wL[V], wR[V], F[V];
        // x-faces ci, ci+1 of row tj
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const float2 A = ld2(pl, v, tj, ci - 2), B = ld2(pl, v, tj, ci), C2 = ld2(pl, v, tj, ci + 2);
            pair_states<LIM>(A, make_float2(A.y, B.x), B, make_float2(B.y, C2.x), wL[v], wR[v]);
        }
        pair_face_flux<FLX, 0>(wL, wR, 0, gam, gm1i, F);
#pragma unroll
        for (int v = 0; v < V; ++v) *reinterpret_cast<float2 *>(Fx + v * NFX + tj * FXP + ci) = F[v];
        if (ci == 0 && tx0 == 0) store_bflux1(0, ty0 + tj + N * k, F[0].x, F[1].x, F[2].x, F[3].x, F[4].x);
        // y-face tj (between rows tj-1 and tj) of columns ci, ci+1
#pragma unroll
        for (int v = 0; v < V; ++v)
            pair_states<LIM>(ld2(pl, v, tj - 2, ci), ld2(pl, v, tj - 1, ci), ld2(pl, v, tj, ci), ld2(pl, v, tj + 1, ci), wL[v], wR[v]);
        pair_face_flux<FLX, 1>(wL, wR, 1, gam, gm1i, F);
#pragma unroll
        for (int v = 0; v < V; ++v) *reinterpret_cast<float2 *>(Fy + v * (T + 1) * T + Sh::fy(tj, ci)) = F[v];
        if (tj == 0 && ty0 == 0) store_bflux2(2, tx0 + ci + N * k, F);
        // z-face k + 1/2 of cells ci, ci+1: the plus state of plane k is
        // carried from the previous plane, the minus / plus states of plane
        // k+1 come from planes k .. k+2
        {
            const float *p1 = pl, *p2 = slot(k + 1), *p3 = slot(k + 2);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const float2 w1 = ld2(p1, v, tj, ci), w2 = ld2(p2, v, tj, ci), w3 = ld2(p3, v, tj, ci);
                if constexpr (LIM == 0) {
                    const float2 d12 = PF::sub(w2, w1), d23 = PF::sub(w3, w2), q = PF::qs(d12, d23);
                    wR[v] = PF::fma(q, PF::nmabs(d12, d23), w2);
                    wL[v] = zP[v];
                    zP[v] = PF::fma(q, PF::mabs(d12, d23), w2);
                } else {
                    wL[v] = zP[v];
                    pair_cell_states<LIM>(w1, w2, w3, wR[v], zP[v]);
                }
            }
            pair_face_flux<FLX, 2>(wL, wR, 2, gam, gm1i, Fz_new);
            if (k == N - 1) store_bflux2(5, tx0 + ci + N * (ty0 + tj), Fz_new);
        }
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
            pair_face_flux<FLX, -1>(wL, wR, isx ? 0 : 1, gam, gm1i, F);
            if (isx) {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    Fx[v * NFX + (2 * r) * FXP + T] = F[v].x;
                    Fx[v * NFX + (2 * r + 1) * FXP + T] = F[v].y;
                }
                if (tx0 + T == N) {
                    store_bflux1(1, ty0 + 2 * r + N * k, F[0].x, F[1].x, F[2].x, F[3].x, F[4].x);
                    store_bflux1(1, ty0 + 2 * r + 1 + N * k, F[0].y, F[1].y, F[2].y, F[3].y, F[4].y);
                }
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) *reinterpret_cast<float2 *>(Fy + v * (T + 1) * T + Sh::fy(T, 2 * r)) = F[v];
                if (ty0 + T == N) store_bflux2(3, tx0 + 2 * r + N * k, F);
            }
        }
    };

    // ---- L2 prefetch, one plane period ahead: the previous states' plane k
    // (read by the update of plane k in the next iteration) and this block's
    // derivative plane k + 5 (loaded into registers two iterations later)
    // ---- L2 prefetch: the previous states' plane k (copied to shared memory
    // at the start of the next plane period) and this block's derivative
    // plane k + 4 (loaded into registers in the next plane period)
    auto l2_ahead = [&](int k) {
        if (tid != NT - 32) return;   // a thread of the last warp (the first takes the edge faces)
        constexpr unsigned PB = unsigned(S) * S * sizeof(float);
        const int64_t blk = int64_t(b) * V * NC;
        if (k < N) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q < (NPREV >= 0 ? NPREV : a.nprev))
#pragma unroll
                    for (int v = 0; v < V; ++v) l2_prefetch(a.prev[q] + blk + v * NC + int64_t(k + NG) * S * S, PB);
        }
        if (k + 4 <= N + 1)
#pragma unroll
            for (int v = 0; v < V; ++v) l2_prefetch(ub + v * NC + int64_t(k + 4 + NG) * S * S, PB);
    };

    // ---- previous states of plane k: asynchronous copies of this thread's
    // pairs into its staging slots, awaited by the update of plane k
    auto stage_prev = [&](int k) {
        if constexpr (NPREV > 0) {
            const int64_t ob = int64_t(b) * V * NC + gofs(tx0 + ci, ty0 + tj, k);
#pragma unroll
            for (int q = 0; q < NPREV; ++q)
#pragma unroll
                for (int v = 0; v < V; ++v) cp_async8(stg + (q * V + v) * NT + tid, a.prev[q] + ob + v * NC);
            cp_async_commit();
        }
    };

    auto update = [&](int k, const float *fb, const float2 *Fzlo, const float2 *Fzhi) {
        if constexpr (NPREV > 0) cp_async_wait_all();
        const float *Fx = fb, *Fy = fb + V * NFX;
        const int64_t o = gofs(tx0 + ci, ty0 + tj, k);
        const int64_t ob = int64_t(b) * V * NC + o;
        const float2 i0 = PF::sp(idx0), i1 = PF::sp(idx1), i2 = PF::sp(idx2), dte = PF::sp(dt_eff);
        float2 U[V];
        // gravity source S = (0, rho g, rho g.u) of variable v from the
        // primitives of plane k, still in the ring
        auto source = [&](int v) -> float2 {
            const float *pk = slot(k);
            const float2 rho = ld2(pk, 0, tj, ci);
            if (v < 4) return PF::mul(rho, PF::sp(a.grav[v - 1]));
            float2 vg = PF::mul(ld2(pk, 1, tj, ci), PF::sp(a.grav[0]));
            vg = PF::fma(ld2(pk, 2, tj, ci), PF::sp(a.grav[1]), vg);
            vg = PF::fma(ld2(pk, 3, tj, ci), PF::sp(a.grav[2]), vg);
            return PF::mul(rho, vg);
        };
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const float2 x0 = *reinterpret_cast<const float2 *>(Fx + v * NFX + tj * FXP + ci);
            const float2 x1 = *reinterpret_cast<const float2 *>(Fx + v * NFX + tj * FXP + ci + 2);
            const float2 y0 = *reinterpret_cast<const float2 *>(Fy + v * (T + 1) * T + Sh::fy(tj, ci));
            const float2 y1 = *reinterpret_cast<const float2 *>(Fy + v * (T + 1) * T + Sh::fy(tj + 1, ci));
            float2 du = PF::mul(PF::sub(x0, make_float2(x0.y, x1.x)), i0);
            du = PF::fma(PF::sub(y0, y1), i1, du);
            du = PF::fma(PF::sub(Fzlo[v], Fzhi[v]), i2, du);
            if (v > 0 && a.gravity_on) du = PF::add(du, source(v));
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
            // cells next to a coarse-side refinement face are reduced after flux fixing
            const bool rowfix = ((m & 4) && gj == 0) || ((m & 8) && gj == N - 1) || ((m & 16) && k == 0) ||
                                ((m & 32) && k == N - 1);
            const bool fx0 = rowfix || ((m & 1) && gi == 0);
            const bool fx1 = rowfix || ((m & 2) && gi + 1 == N - 1);
            float2 w[V];
            pair_prim(U, w, gam);
            const float2 c2 = PF::mul(PF::mul(PF::sp(gam), w[4]), PF::rcp(w[0]));
            const float2 c = PF::mul(c2, PF::rsqrt(c2));
            float2 s = PF::mul(PF::add(PF::abs(w[1]), c), i0);
            s = PF::fma(PF::add(PF::abs(w[2]), c), i1, s);
            s = PF::fma(PF::add(PF::abs(w[3]), c), i2, s);
            if (!fx0) vmax = s.x > vmax ? s.x : vmax;
            if (!fx1) vmax = s.y > vmax ? s.y : vmax;
        }
    };

    // ---- the march (ring of 4 planes: the fluxes of plane k read planes
    // k .. k+2 while plane k+3 is committed into the slot of plane k-1)
    prefetch(-2);
    commit(-2);
    prefetch(-1);
    commit(-1);
    prefetch(0);
    commit(0);
    prefetch(1);
    commit(1);
    prefetch(2);
    __syncthreads();
    {
        // z flux through the block's lower face (k = -1/2) and the plus
        // state of plane 0
        const float *p0 = slot(-2), *p1 = slot(-1), *p2 = slot(0), *p3 = slot(1);
        float2 wL[V], wR[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const float2 w0 = ld2(p0, v, tj, ci), w1 = ld2(p1, v, tj, ci), w2 = ld2(p2, v, tj, ci), w3 = ld2(p3, v, tj, ci);
            pair_states<LIM>(w0, w1, w2, w3, wL[v], wR[v]);
            if constexpr (LIM == 0) {
                const float2 d12 = PF::sub(w2, w1), d23 = PF::sub(w3, w2);
                zP[v] = PF::fma(PF::qs(d12, d23), PF::mabs(d12, d23), w2);
            } else {
                float2 zm;
                pair_cell_states<LIM>(w1, w2, w3, zm, zP[v]);
            }
        }
        pair_face_flux<FLX, 2>(wL, wR, 2, gam, gm1i, FzA);
        store_bflux2(4, tx0 + ci + N * (ty0 + tj), FzA);
    }
    __syncthreads();
    commit(2);          // into the slot of plane -2
    prefetch(3);
    __syncthreads();
    // plane k: copy its previous states, compute its x/y fluxes and the z flux
    // above it, commit plane k+3 into the slot of plane k-1 and load plane
    // k+4; barrier; update plane k; barrier (flux buffer reused)
    for (int k = 0; k < N; ++k) {
        stage_prev(k);
        l2_ahead(k + 1);
        fluxes(k, fbuf, FzB);
        if (k + 3 <= N + 1) {
            commit(k + 3);
            if (k + 4 <= N + 1) prefetch(k + 4);
        }
        __syncthreads();
        update(k, fbuf, FzA, FzB);
#pragma unroll
        for (int v = 0; v < V; ++v) FzA[v] = FzB[v];
        __syncthreads();
    }

    if (a.update_dt) {
        double m = double(vmax);
        for (int s = 16; s > 0; s >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, s));
        if ((tid & 31) == 0) atomic_max_nonneg(&a.sc[info.inst].maxspeed_bits, m);
    }
    if (__syncthreads_or(nonphys) && tid == 0) raise_status(&a.sc[0].status, 7);
}

template <int N, int TT, int NPREV, int LIM, int FLX>
__global__ void __launch_bounds__(PairShape<N, TT>::NT, (TT >= 16 ? 4 : 1)) k_stage_pair(StageArgs<float> a, Geom g) {
    for (int item = blockIdx.x; item < a.n_items; item += gridDim.x) stage_pair_item<N, TT, NPREV, LIM, FLX>(a, g, item);
}

}  // namespace amrb
