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
//   [copies of previous states | fluxes of plane k | commit of plane k+3]
//   barrier [update of plane k]
// (with two previous states a second barrier opens each plane: their single
// y-face buffer must be read by every update before the next fluxes).  The
// previous states travel by cp.async into per-thread shared slots while the
// fluxes are computed, so the update does not wait on global loads.  Face
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
    // minmod(a, b) (Eq. 1 with theta = 1) as the median of a, b and 0:
    // min(max(a, b), max(min(a, b), 0)) is the argument of smaller magnitude
    // when a and b have the same strict sign and 0 otherwise, so
    // w + 0.5 minmod(a, b) is the single rounding fma(0.5, mm(a, b), w).
    __device__ static __forceinline__ float mm1(float a, float b) { return fminf(fmaxf(a, b), fmaxf(fminf(a, b), 0.f)); }
    __device__ static __forceinline__ float2 mm(float2 a, float2 b) { return make_float2(mm1(a.x, b.x), mm1(a.y, b.y)); }
    // minmod(a, b) and minmod(c, b) with the middle difference b shared:
    // the median of (x, b, 0) is max(min(x, max(b, 0)), min(b, 0)), so the
    // two limited slopes of a face take six min/max per lane instead of eight
    __device__ static __forceinline__ void mm2(float2 a, float2 b, float2 c, float2 &mab, float2 &mcb) {
        const float px = fmaxf(b.x, 0.f), py = fmaxf(b.y, 0.f), nx = fminf(b.x, 0.f), ny = fminf(b.y, 0.f);
        mab = make_float2(fmaxf(fminf(a.x, px), nx), fmaxf(fminf(a.y, py), ny));
        mcb = make_float2(fmaxf(fminf(c.x, px), nx), fmaxf(fminf(c.y, py), ny));
    }
    // qs = (sign a + sign b) / 4 from the sign bits: +-1/2 when the signs
    // agree, 0 otherwise (the monotonized-central limiter builds on it)
    __device__ static __forceinline__ float sg(float a) { return __uint_as_float((__float_as_uint(a) & 0x80000000u) | 0x3e800000u); }
    __device__ static __forceinline__ float2 qs(float2 a, float2 b) {
        return add(make_float2(sg(a.x), sg(a.y)), make_float2(sg(b.x), sg(b.y)));
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
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Rusanov or HLL flux (Sec. 3.2) of a pair of faces with the same normal
// (compile-time NRM >= 0, or the runtime normal n when NRM < 0) from the
// primitive states (rho, v_0 .. v_{D-1}, p) on either side, with Einfeldt's
// signal speeds (Sec. 3.5): u_roe = (sqrt(rL) vnL + sqrt(rR) vnR) / S and
// d^2 = gamma (pL / sqrt(rL) + pR / sqrt(rR)) / S
//       + 1/2 sqrt(rL) sqrt(rR) / S^2 (vnR - vnL)^2,  S = sqrt(rL) + sqrt(rR)
// (the weighted mean of c^2 = gamma p / rho written with p / sqrt(rho)).
//
// Both fluxes are evaluated with the terms of each conserved variable
// grouped by side:
//   F_rho = B_L + B_R,   B = A rho
//   F_m   = B_L v_L + B_R v_R + (pi_L p_L + pi_R p_R) e_n
//   F_E   = p_L (A_L g + pi_L vn_L) + p_R (A_R g + pi_R vn_R)
//           + (B_L |v_L|^2 + B_R |v_R|^2) / 2,          g = 1 / (gamma - 1)
// which is F = (F(wL) + F(wR)) / 2 - a (U_R - U_L) / 2 for Rusanov with
// A_L = (vn_L + a) / 2, A_R = (vn_R - a) / 2, pi = 1/2, a = |u_roe| + d, and
// F = (sR F(wL) - sL F(wR) + sL sR (U_R - U_L)) / (sR - sL) for HLL with
// sL = min(u_roe - d, 0), sR = max(u_roe + d, 0), w = 1 / (sR - sL),
// pi_L = w sR, pi_R = -w sL, A_L = pi_L (vn_L - sL), A_R = pi_R (vn_R - sR)
// (E = p g + rho |v|^2 / 2 expanded).  The grouped form needs neither the
// conservative face states nor both physical fluxes.
template <int D, int FLX, int NRM>
__device__ __forceinline__ void pair_flux_grouped(const float2 *wL, const float2 *wR, int n, float gam, float gm1i, float2 *F) {
    const int nn = NRM >= 0 ? NRM : n;
    float2 vnL, vnR;
    if constexpr (NRM >= 0) {
        vnL = wL[1 + NRM];
        vnR = wR[1 + NRM];
    } else if constexpr (D == 2) {
        vnL = nn == 0 ? wL[1] : wL[2];
        vnR = nn == 0 ? wR[1] : wR[2];
    } else {
        vnL = nn == 0 ? wL[1] : (nn == 1 ? wL[2] : wL[3]);
        vnR = nn == 0 ? wR[1] : (nn == 1 ? wR[2] : wR[3]);
    }
    const float2 rL = wL[0], rR = wR[0], pL = wL[D + 1], pR = wR[D + 1];
    const float2 half = PF::sp(0.5f);
    const float2 qL = PF::rsqrt(rL), qR = PF::rsqrt(rR);
    const float2 sL = PF::mul(rL, qL), sR = PF::mul(rR, qR);               // sqrt(rho)
    const float2 inv = PF::rcp(PF::add(sL, sR));                           // 1 / S
    const float2 uroe = PF::mul(PF::fma(sL, vnL, PF::mul(sR, vnR)), inv);
    const float2 du = PF::sub(vnR, vnL);
    const float2 P = PF::fma(pR, qR, PF::mul(pL, qL));                     // pL / sqrt(rL) + pR / sqrt(rR)
    const float2 x = PF::mul(PF::mul(sL, sR), inv);                        // sqrt(rL rR) / S
    const float2 y = PF::mul(inv, du);                                      // du / S
    const float2 d2 = PF::fma(PF::mul(x, y), PF::mul(half, du), PF::mul(PF::mul(PF::sp(gam), inv), P));
    const float2 d = PF::mul(d2, PF::rsqrt(d2));
    float2 AL, AR, piL, piR;
    if constexpr (FLX == 1) {
        const float2 lo = PF::sub(uroe, d), hi = PF::add(uroe, d);
        const float2 nsl = make_float2(fmaxf(-lo.x, 0.f), fmaxf(-lo.y, 0.f));   // -sL >= 0
        const float2 sr = make_float2(fmaxf(hi.x, 0.f), fmaxf(hi.y, 0.f));     // sR >= 0
        const float2 w = PF::rcp(PF::add(sr, nsl));
        piL = PF::mul(w, sr);
        piR = PF::mul(w, nsl);
        AL = PF::mul(piL, PF::add(vnL, nsl));
        AR = PF::mul(piR, PF::sub(vnR, sr));
    } else {
        const float2 ha = PF::mul(half, PF::add(PF::abs(uroe), d));
        piL = PF::mul(half, vnL);                                          // here: vn / 2
        piR = PF::mul(half, vnR);
        AL = PF::add(piL, ha);
        AR = PF::sub(piR, ha);
    }
    const float2 BL = PF::mul(AL, rL), BR = PF::mul(AR, rR);
    F[0] = PF::add(BL, BR);
    float2 pn;
    if constexpr (FLX == 1) pn = PF::fma(piR, pR, PF::mul(piL, pL));
    else pn = PF::mul(half, PF::add(pL, pR));
#pragma unroll
    for (int c = 0; c < D; ++c) {
        float2 f = PF::fma(BL, wL[1 + c], PF::mul(BR, wR[1 + c]));
        if (c == nn) f = PF::add(f, pn);
        F[1 + c] = f;
    }
    float2 v2L = PF::mul(wL[1], wL[1]), v2R = PF::mul(wR[1], wR[1]);
#pragma unroll
    for (int c = 1; c < D; ++c) {
        v2L = PF::fma(wL[1 + c], wL[1 + c], v2L);
        v2R = PF::fma(wR[1 + c], wR[1 + c], v2R);
    }
    const float2 g1 = PF::sp(gm1i);
    // Rusanov: pi vn = vn^2 / 2 would be wrong -- the pressure work is p vn / 2
    const float2 cL = FLX == 1 ? PF::fma(AL, g1, PF::mul(piL, vnL)) : PF::fma(AL, g1, piL);
    const float2 cR = FLX == 1 ? PF::fma(AR, g1, PF::mul(piR, vnR)) : PF::fma(AR, g1, piR);
    const float2 ke = PF::fma(BR, v2R, PF::mul(BL, v2L));
    F[D + 1] = PF::fma(half, ke, PF::fma(pR, cR, PF::mul(pL, cL)));
}

template <int NRM>
__device__ __forceinline__ void pair_flux(const float2 *wL, const float2 *wR, int n, float gam, float gm1i, float2 *F) {
    pair_flux_grouped<3, 0, NRM>(wL, wR, n, gam, gm1i, F);
}
template <int NRM>
__device__ __forceinline__ void pair_flux_hll(const float2 *wL, const float2 *wR, int n, float gam, float gm1i, float2 *F) {
    pair_flux_grouped<3, 1, NRM>(wL, wR, n, gam, gm1i, F);
}

// the pair flux of the configured scheme (FLX 0 Rusanov, 1 HLL)
template <int FLX, int NRM>
__device__ __forceinline__ void pair_face_flux(const float2 *wL, const float2 *wR, int n, float gam, float gm1i, float2 *F) {
    pair_flux_grouped<3, FLX, NRM>(wL, wR, n, gam, gm1i, F);
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
        float2 m01, m23;
        PF::mm2(d01, d12, d23, m01, m23);
        L = PF::fma(PF::sp(0.5f), m01, w1);
        R = PF::fma(PF::sp(-0.5f), m23, w2);
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
        const float2 m = PF::mm(d01, d12);
        minus = PF::fma(PF::sp(-0.5f), m, w1);
        plus = PF::fma(PF::sp(0.5f), m, w1);
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
    static constexpr int LOADS = ((T * T + 8 * T) / 2 + NT - 1) / NT;   // halo pairs without corners
    // upper y-face of row `row` (T rows of T faces): for T = 16 rows 2m and
    // 2m + 1 share a 32-word line, their halves swapped when bit 2 of the row
    // is set, so rows r and r + 4 (one half-warp) use opposite bank halves
    __device__ static __forceinline__ int fy(int row, int c) {
        if constexpr (T == 16) return 32 * (row >> 1) + 16 * ((row ^ (row >> 2)) & 1) + c;
        else return row * T + c;
    }
    static constexpr int FYB = V * T * T;             // one y-face buffer
    static constexpr int EXB = V * T;                 // one buffer of the tile's upper x-faces
    // y-face buffers: two, alternating with the parity of k, or one for two
    // previous states (a second barrier per plane instead; the shared memory
    // saved goes to the L1 cache)
    static constexpr int fy_bufs(int nprev) { return nprev == 2 ? 1 : 2; }
    // staging slots of a thread's previous-state pairs: one per state, and
    // for two states a second slot for the first state, whose copies of the
    // next plane are issued a plane period ahead
    static constexpr int stg_slots(int nprev) { return nprev == 2 ? 3 : (nprev > 0 ? nprev : 0); }
    // ring, y-face buffers, two upper-x-face buffers and the staging slots [stg_slots][V][NT]
    static constexpr size_t smem_bytes(int nprev) {
        return sizeof(float) * (size_t(R) * V * PL + size_t(fy_bufs(nprev)) * size_t(FYB) + 2 * size_t(EXB)) +
               sizeof(float2) * size_t(stg_slots(nprev)) * V * NT;
    }
};

// One CTA's (block, tile) item.  Per plane k (one barrier):
//   flux phase:  copy plane k's previous states (cp.async); the x-, y- and
//                z-face fluxes of the thread's cell pair; its divergence
//                accumulated in registers except the upper y-face (from
//                the thread of the next row, through shared memory); the
//                first warp computes the tile's upper x-faces of plane k+1
//                and upper y-faces of plane k; commit plane k+3, load k+4
//   barrier
//   update:      subtract the upper y-face, combine with the previous
//                states and store
// The right x-face of a pair comes from the next lane of the row (shuffle),
// or for the last pair of a row from the upper x-faces computed one plane
// ahead; the lower y-face of a row is the thread's own flux.  y- and x-face
// buffers alternate with the parity of k, so the next plane's flux phase can
// overwrite nothing the update still reads (with two previous states there is
// one y-face buffer and a second barrier before each flux phase instead).
// FIX: the mesh has refinement
// faces (flux stores for the flux fix, cells excluded from the CFL maximum);
// without them that code is compiled out.
template <int N, int TT, int NPREV, int LIM, int FLX, bool FIX>
__device__ __forceinline__ void stage_pair_item(const StageArgs<float> &a, const Geom &g, int item) {
    using Sh = PairShape<N, TT>;
    constexpr int T = Sh::T, NG = Sh::NG, S = Sh::S, P = Sh::P, PL = Sh::PL, V = Sh::V, NT = Sh::NT;
    constexpr int FYB = Sh::FYB, EXB = Sh::EXB, HP = T / 2;
    constexpr int64_t NC = int64_t(S) * S * S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *ring = reinterpret_cast<float *>(smem_raw);         // [R][V][P*P]
    float *fyb = ring + Sh::R * V * PL;                         // [fy_bufs][V][T x T] upper y-faces
    constexpr int FYN = Sh::fy_bufs(NPREV);
    float *exb = fyb + FYN * FYB;                               // [2][V][T] upper x-faces
    float2 *stg = reinterpret_cast<float2 *>(exb + 2 * EXB);    // [stg_slots][V][NT] previous states

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
        ip = tid % HP;
        tj = tid / HP;
    }
    const int ci = 2 * ip;                                      // first cell of the pair
    const bool last = ip == HP - 1;                             // the pair at the tile's upper x edge
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
    // refinement-face flux slots this thread stores into (-1: none)
    const int bs_x0 = (FIX && ci == 0 && tx0 == 0) ? info.bslot[0] : -1;
    const int bs_y0 = (FIX && tj == 0 && ty0 == 0) ? info.bslot[2] : -1;
    const int bs_z0 = FIX ? info.bslot[4] : -1, bs_z1 = FIX ? info.bslot[5] : -1;

    bool nonphys = false;
    float vmax = 0.f;

    auto slot = [&](int k) -> float * { return ring + ((k + 2) & (Sh::R - 1)) * V * PL; };
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
    constexpr int WP = (T + 4) / 2;
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
    const int own_off = (tid / HP + 2) * P + 2 * (tid % HP) + 2;

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
            const float *src = src_of(2 * (tid % HP), tid / HP, k, o);
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
    auto store_bflux1 = [&](int sl, int t, float Fv0, float Fv1, float Fv2, float Fv3, float Fv4) {
        float *dst = a.bflux + int64_t(sl) * V * nface_b + t;
        dst[0] = Fv0;
        dst[nface_b] = Fv1;
        dst[2 * nface_b] = Fv2;
        dst[3 * nface_b] = Fv3;
        dst[4 * nface_b] = Fv4;
    };
    // store both faces of a pair (tangential indices t and t + 1)
    auto store_bflux2 = [&](int sl, int t, const float2 *F) {
        float *dst = a.bflux + int64_t(sl) * V * nface_b + t;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            dst[v * nface_b] = F[v].x;
            dst[v * nface_b + 1] = F[v].y;
        }
    };

    // The first warp's edge faces: lanes r < T/2 the upper x-face of rows
    // (2r, 2r+1) of plane kx, lanes T/2 + r the upper y-face of columns
    // (2r, 2r+1) of plane ky; one flux evaluation with a runtime normal.
    // Lane offsets in a ring plane: base + i st (+ po for the second face).
    const int bs_x1 = (FIX && tx0 + T == N) ? info.bslot[1] : -1;
    const int bs_y1 = (FIX && ty0 + T == N) ? info.bslot[3] : -1;
    auto edge_faces = [&](int kx, int ky, bool do_x) {
        const bool e_isx = tid < HP;
        const int e_r = e_isx ? tid : tid - HP;
        const int e_base = e_isx ? (2 * e_r + 2) * P + T : T * P + 2 + 2 * e_r;
        const int e_st = e_isx ? 1 : P, e_po = e_isx ? P : 1;
        if (e_isx && !do_x) return;
        const float *pl = (e_isx ? slot(kx) : slot(ky)) + e_base;
        float2 wL[V], wR[V], F[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const float *b0 = pl + v * PL;
            pair_states<LIM>(make_float2(b0[0], b0[e_po]), make_float2(b0[e_st], b0[e_st + e_po]),
                             make_float2(b0[2 * e_st], b0[2 * e_st + e_po]), make_float2(b0[3 * e_st], b0[3 * e_st + e_po]),
                             wL[v], wR[v]);
        }
        pair_face_flux<FLX, -1>(wL, wR, e_isx ? 0 : 1, gam, gm1i, F);
        if (e_isx) {
            float *ex = exb + (kx & 1) * EXB + 2 * e_r;
#pragma unroll
            for (int v = 0; v < V; ++v) *reinterpret_cast<float2 *>(ex + v * T) = F[v];
            if (bs_x1 >= 0) {
                store_bflux1(bs_x1, ty0 + 2 * e_r + N * kx, F[0].x, F[1].x, F[2].x, F[3].x, F[4].x);
                store_bflux1(bs_x1, ty0 + 2 * e_r + 1 + N * kx, F[0].y, F[1].y, F[2].y, F[3].y, F[4].y);
            }
        } else {
            float *fy = fyb + (FYN == 2 ? (ky & 1) : 0) * FYB;
#pragma unroll
            for (int v = 0; v < V; ++v) *reinterpret_cast<float2 *>(fy + v * T * T + Sh::fy(T - 1, 2 * e_r)) = F[v];
            if (bs_y1 >= 0) store_bflux2(bs_y1, tx0 + 2 * e_r + N * ky, F);
        }
    };

    // ---- flux phase of plane k: the divergence of the pair's fluxes into
    // du (all faces but the upper y-face); Fz holds the z flux below the
    // plane on entry and above it on return
    float2 Fz[V];            // z flux below the plane being updated
    float2 zP[V];            // plus z state of the pair at the plane whose fluxes come next
    float2 du[V];
    const float2 i0 = PF::sp(idx0), i1 = PF::sp(idx1), i2 = PF::sp(idx2);
    auto fluxes = [&](int k) {
        const float *pl = slot(k);
        float2 Bw[V], wL[V], wR[V], F[V];
#pragma unroll
        for (int v = 0; v < V; ++v) Bw[v] = ld2(pl, v, tj, ci);
        // x-faces ci - 1/2, ci + 1/2 of row tj
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const float2 A = ld2(pl, v, tj, ci - 2), C2 = ld2(pl, v, tj, ci + 2);
            pair_states<LIM>(A, make_float2(A.y, Bw[v].x), Bw[v], make_float2(Bw[v].y, C2.x), wL[v], wR[v]);
        }
        pair_face_flux<FLX, 0>(wL, wR, 0, gam, gm1i, F);
        if (bs_x0 >= 0) store_bflux1(bs_x0, ty0 + tj + N * k, F[0].x, F[1].x, F[2].x, F[3].x, F[4].x);
        const float *ex = exb + (k & 1) * EXB + tj;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            // the face right of the pair: the next lane's first face, or the
            // tile's upper x-face for the last pair of the row
            const float nx = __shfl_down_sync(0xffffffffu, F[v].x, 1, HP);
            const float right = last ? ex[v * T] : nx;
            du[v] = PF::mul(PF::sub(F[v], make_float2(F[v].y, right)), i0);
        }
        // y-face tj - 1/2 (between rows tj-1 and tj) of columns ci, ci+1: the
        // lower face of this row, the upper face of row tj - 1
#pragma unroll
        for (int v = 0; v < V; ++v)
            pair_states<LIM>(ld2(pl, v, tj - 2, ci), ld2(pl, v, tj - 1, ci), Bw[v], ld2(pl, v, tj + 1, ci), wL[v], wR[v]);
        pair_face_flux<FLX, 1>(wL, wR, 1, gam, gm1i, F);
        if (tj > 0) {
            float *fy = fyb + (FYN == 2 ? (k & 1) : 0) * FYB + Sh::fy(tj - 1, ci);
#pragma unroll
            for (int v = 0; v < V; ++v) *reinterpret_cast<float2 *>(fy + v * T * T) = F[v];
        }
        if (bs_y0 >= 0) store_bflux2(bs_y0, tx0 + ci + N * k, F);
#pragma unroll
        for (int v = 0; v < V; ++v) du[v] = PF::fma(F[v], i1, du[v]);
        // z-face k + 1/2 of cells ci, ci+1: the plus state of plane k is
        // carried from the previous plane, the minus / plus states of plane
        // k+1 come from planes k .. k+2
        {
            const float *p2 = slot(k + 1), *p3 = slot(k + 2);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const float2 w1 = Bw[v], w2 = ld2(p2, v, tj, ci), w3 = ld2(p3, v, tj, ci);
                if constexpr (LIM == 0) {
                    const float2 d12 = PF::sub(w2, w1), d23 = PF::sub(w3, w2), m = PF::mm(d12, d23);
                    wR[v] = PF::fma(PF::sp(-0.5f), m, w2);
                    wL[v] = zP[v];
                    zP[v] = PF::fma(PF::sp(0.5f), m, w2);
                } else {
                    wL[v] = zP[v];
                    pair_cell_states<LIM>(w1, w2, w3, wR[v], zP[v]);
                }
            }
            pair_face_flux<FLX, 2>(wL, wR, 2, gam, gm1i, F);
            if (k == N - 1 && bs_z1 >= 0) store_bflux2(bs_z1, tx0 + ci + N * (ty0 + tj), F);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                du[v] = PF::fma(PF::sub(Fz[v], F[v]), i2, du[v]);
                Fz[v] = F[v];
            }
        }
        // gravity source S = (0, rho g, rho g.u) of the cells' primitives
        if (a.gravity_on) {
            const float2 rho = Bw[0];
            float2 vg = PF::mul(Bw[1], PF::sp(a.grav[0]));
            vg = PF::fma(Bw[2], PF::sp(a.grav[1]), vg);
            vg = PF::fma(Bw[3], PF::sp(a.grav[2]), vg);
#pragma unroll
            for (int c = 0; c < 3; ++c) du[1 + c] = PF::fma(rho, PF::sp(a.grav[c]), du[1 + c]);
            du[4] = PF::fma(rho, vg, du[4]);
        }
    };

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
    // pairs into its staging slots, awaited by the update of plane k.  The
    // slots are the thread's own, so a copy may be issued as soon as the
    // thread has read the slot's last contents.  With two previous states
    // the first one's copies of plane k + 1 go out a plane period ahead
    // (slot k & 1), the second's at the start of period k (slot 2).
    auto stg_at = [&](int k, int q, int v) -> float2 * {
        return stg + (((NPREV == 2) ? (q == 0 ? (k & 1) : 2) : q) * V + v) * NT + tid;
    };
    auto stage_prev_q = [&](int k, int q) {
        if (k < N) {
            const int64_t ob = int64_t(b) * V * NC + gofs(tx0 + ci, ty0 + tj, k);
#pragma unroll
            for (int v = 0; v < V; ++v) cp_async8(stg_at(k, q, v), a.prev[q] + ob + v * NC);
        }
        cp_async_commit();
    };
    auto stage_prev = [&](int k) {
        if constexpr (NPREV > 0) {
            const int64_t ob = int64_t(b) * V * NC + gofs(tx0 + ci, ty0 + tj, k);
#pragma unroll
            for (int q = 0; q < NPREV; ++q)
#pragma unroll
                for (int v = 0; v < V; ++v) cp_async8(stg_at(k, q, v), a.prev[q] + ob + v * NC);
            cp_async_commit();
        }
    };

    // cells next to a coarse-side refinement face are reduced after flux
    // fixing (the parts of that test that do not depend on k)
    const int fmask = FIX ? info.fixmask : 0;
    const int gi0 = tx0 + ci, gj0 = ty0 + tj;
    const bool rowfix_jk = ((fmask & 4) && gj0 == 0) || ((fmask & 8) && gj0 == N - 1);
    const bool colfix0 = (fmask & 1) && gi0 == 0, colfix1 = (fmask & 2) && gi0 + 1 == N - 1;

    auto update = [&](int k) {
        if constexpr (NPREV == 2) {
            cp_async_wait_one();      // the first state's copies of plane k + 1 may stay in flight
        } else if constexpr (NPREV > 0) {
            cp_async_wait_all();
        }
        const float *fy = fyb + (FYN == 2 ? (k & 1) : 0) * FYB + Sh::fy(tj, ci);
        const int64_t ob = int64_t(b) * V * NC + gofs(tx0 + ci, ty0 + tj, k);
        const float2 dte = PF::sp(dt_eff);
        float2 U[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const float2 up = *reinterpret_cast<const float2 *>(fy + v * T * T);
            const float2 d = PF::fma(up, PF::sp(-idx1), du[v]);
            float2 acc = PF::sp(0.f);
            if constexpr (NPREV > 0) {
#pragma unroll
                for (int q = 0; q < NPREV; ++q) acc = PF::fma(PF::sp(a.wprev[q]), *stg_at(k, q, v), acc);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (q < a.nprev)
                        acc = PF::fma(PF::sp(a.wprev[q]), *reinterpret_cast<const float2 *>(a.prev[q] + ob + v * NC), acc);
            }
            U[v] = PF::fma(dte, d, acc);
            *reinterpret_cast<float2 *>(a.out + ob + v * NC) = U[v];
        }
        // complete the row's DRAM sectors: the output's x-ghost cells
        if (gi0 == 0 || gi0 + 1 == N - 1) {
            const int64_t og = ob + (gi0 == 0 ? -NG : 2);
#pragma unroll
            for (int v = 0; v < V; ++v) *reinterpret_cast<float2 *>(a.out + og + v * NC) = PF::sp(0.f);
        }
        if (a.update_dt) {
            const bool rowfix = rowfix_jk || ((fmask & 16) && k == 0) || ((fmask & 32) && k == N - 1);
            float2 w[V];
            pair_prim(U, w, gam);
            const float2 c2 = PF::mul(PF::mul(PF::sp(gam), w[4]), PF::rcp(w[0]));
            const float2 c = PF::mul(c2, PF::rsqrt(c2));
            float2 s = PF::mul(PF::add(PF::abs(w[1]), c), i0);
            s = PF::fma(PF::add(PF::abs(w[2]), c), i1, s);
            s = PF::fma(PF::add(PF::abs(w[3]), c), i2, s);
            if (!(rowfix || colfix0)) vmax = s.x > vmax ? s.x : vmax;
            if (!(rowfix || colfix1)) vmax = s.y > vmax ? s.y : vmax;
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
        // state of plane 0; the tile's upper x-faces of plane 0
        const float *p0 = slot(-2), *p1 = slot(-1), *p2 = slot(0), *p3 = slot(1);
        float2 wL[V], wR[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const float2 w0 = ld2(p0, v, tj, ci), w1 = ld2(p1, v, tj, ci), w2 = ld2(p2, v, tj, ci), w3 = ld2(p3, v, tj, ci);
            pair_states<LIM>(w0, w1, w2, w3, wL[v], wR[v]);
            if constexpr (LIM == 0) {
                const float2 d12 = PF::sub(w2, w1), d23 = PF::sub(w3, w2);
                zP[v] = PF::fma(PF::sp(0.5f), PF::mm(d12, d23), w2);
            } else {
                float2 zm;
                pair_cell_states<LIM>(w1, w2, w3, zm, zP[v]);
            }
        }
        pair_face_flux<FLX, 2>(wL, wR, 2, gam, gm1i, Fz);
        if (bs_z0 >= 0) store_bflux2(bs_z0, tx0 + ci + N * (ty0 + tj), Fz);
        if (tid < HP) edge_faces(0, 0, true);
    }
    __syncthreads();
    commit(2);          // into the slot of plane -2
    prefetch(3);
    __syncthreads();
    // copy groups of a thread with two previous states, oldest first, at
    // the update of plane k: [state 0, plane k][state 1, plane k][state 0,
    // plane k + 1] (empty beyond the block), so waiting for all but the
    // newest group leaves only the copies of plane k + 1 in flight
    if constexpr (NPREV == 2) stage_prev_q(0, 0);
    for (int k = 0; k < N; ++k) {
        if constexpr (NPREV == 2) {
            if (k > 0) __syncthreads();     // every update of plane k - 1 has read the y-face buffer
            stage_prev_q(k, 1);
            stage_prev_q(k + 1, 0);
        } else {
            stage_prev(k);
        }
        l2_ahead(k + 1);
        fluxes(k);
        if (tid < T) edge_faces(k + 1, k, k + 1 < N);
        if (k + 3 <= N + 1) {
            commit(k + 3);
            if (k + 4 <= N + 1) prefetch(k + 4);
        }
        __syncthreads();
        update(k);
    }
    __syncthreads();   // the next item's prologue overwrites the ring and the face buffers

    if (a.update_dt) {
        double m = double(vmax);
        for (int s = 16; s > 0; s >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, s));
        if ((tid & 31) == 0) atomic_max_nonneg(&a.sc[info.inst].maxspeed_bits, m);
    }
    if (__syncthreads_or(nonphys) && tid == 0) raise_status(&a.sc[0].status, 7);
}

// 16 x 16 tiles: four CTAs per SM (128 registers a thread), or three with
// two previous states (about 160 registers: that stage gains more from
// longer-lived registers and the L1 cache than from resident warps)
template <int N, int TT, int NPREV, int LIM, int FLX, bool FIX>
__global__ void __launch_bounds__(PairShape<N, TT>::NT, (TT >= 16 ? (NPREV == 2 ? 3 : 4) : 1)) k_stage_pair(StageArgs<float> a, Geom g) {
    for (int item = blockIdx.x; item < a.n_items; item += gridDim.x) stage_pair_item<N, TT, NPREV, LIM, FLX, FIX>(a, g, item);
}

}  // namespace amrb
