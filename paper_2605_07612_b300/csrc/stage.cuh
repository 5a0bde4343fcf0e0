// Finite-volume Runge-Kutta stage of the Euler equations (Sec. 3.1-3.5):
//   u_out = w_dt dt F(u_deriv) + sum_i w_i u_prev_i            (Eq. 5)
// F: primitive variables (Eq. 15), MUSCL face values with the configured slope
// limiter (minmod, MC or van Leer), Rusanov or HLL flux with Einfeldt's
// wave-speed estimate, flux divergence.
//
// Work decomposition (ours, not the paper's gang/collapse loops): one CTA per
// (block, T x T column tile).  The CTA marches k through the block keeping a
// ring of 5 planes of primitives (tile plus a 2-cell x/y halo, corners
// excluded) in shared memory, so each cell is converted to primitives once.
// Per plane:
//   phase A  every cell's limited face states along x and y (one limited
//            slope per variable and direction) into shared memory; the z face states of
//            the cell above, in registers;
//   phase B  every face flux once (x, y from the stored states, z in
//            registers); the plane three ahead is converted and committed;
//   phase C  divergence and Runge-Kutta combination, merged with phase A of
//            the next plane.
// Two barriers per plane.  Loads of the next plane are issued one phase
// ahead.  Output rows are written whole (the x-ghost cells of the output
// are overwritten with zeros) so that every DRAM sector is written
// completely.  The kernel also stores the fluxes of refinement faces for
// flux fixing (Sec. 2.7) and, on the last stage of a step, reduces the CFL
// limit of its output (Sec. 3.2).  2D blocks are the single-plane case.
//
// FP32 uses the hardware reciprocal and reciprocal-square-root; FP64 uses
// IEEE division and square root.
#pragma once
#include <type_traits>

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
    const DevScalars *sc_in;     // per instance: dt
    DevScalars *sc;              // per instance: max speed accumulation; status in [0]
    const BlockInfo *info;
    real *bflux;                 // [slot][V][N^(D-1)]
    int update_dt;
    int gather;                  // halo cells across SRL faces from the neighbour's interior
    int n_items;                 // blocks x column tiles; CTAs loop over them with a grid stride
    real gamma;
    int limiter;                 // amr_limiter (the pair kernels: minmod, MC, van Leer)
    int flux;                    // amr_flux (the pair kernels: Rusanov and HLL)
    int gravity_on;              // add the source S = (0, rho g, rho g.u) of u_deriv
    real grav[3];
    real vel[3];                 // advection velocity (scalar advection only)
};

// Constants a numerical flux needs: gamma and 1 / (gamma - 1) for Euler,
// the uniform velocity for scalar advection.
template <class real>
struct PhysCtx {
    real gam, gm1i;
    real vel[3];
};

template <class real>
struct FM;
template <>
struct FM<float> {
    __device__ static __forceinline__ float rcp(float x) { return rcp_ftz(x); }
    // sqrt(x) and 1/x for x > 0
    __device__ static __forceinline__ void sqrt_inv(float x, float &s, float &inv) {
        const float r = rsqrt_ftz(x);
        s = x * r;
        inv = r * r;
    }
    __device__ static __forceinline__ float sqrtp(float x) { return x * rsqrt_ftz(x); }   // x > 0
};
template <>
struct FM<double> {
    __device__ static __forceinline__ double rcp(double x) { return 1.0 / x; }
    __device__ static __forceinline__ void sqrt_inv(double x, double &s, double &inv) {
        s = sqrt(x);
        inv = 1.0 / x;
    }
    __device__ static __forceinline__ double sqrtp(double x) { return sqrt(x); }
};

template <class real, int D>
struct Euler {
    static constexpr int V = D + 2;

    // primitive (rho, v, p) from conservative (rho, rho v, E)
    __device__ static __forceinline__ void prim(const real *U, real *w, real gam) {
        const real rho = U[0];
        const real ir = FM<real>::rcp(rho);
        real ke = real(0);
#pragma unroll
        for (int d = 0; d < D; ++d) {
            w[1 + d] = U[1 + d] * ir;
            ke += w[1 + d] * U[1 + d];
        }
        w[0] = rho;
        w[D + 1] = (gam - real(1)) * (U[D + 1] - real(0.5) * ke);
    }

    // Rusanov flux along normal n with the Einfeldt speed a = |u_roe| + d_roe
    // (Einfeldt 1988, as cited in Sec. 3.5).  NRM >= 0: compile-time normal;
    // NRM < 0: runtime normal n.
    template <int NRM>
    __device__ static __forceinline__ void flux(const real *wL, const real *wR, int n, real gam, real gm1i, real *F) {
        const int nn = NRM >= 0 ? NRM : n;
        real vnL, vnR;
        if (NRM >= 0) {
            vnL = wL[1 + (NRM >= 0 ? NRM : 0)];
            vnR = wR[1 + (NRM >= 0 ? NRM : 0)];
        } else {
            vnL = nn == 0 ? wL[1] : (nn == 1 ? wL[2] : wL[D]);
            vnR = nn == 0 ? wR[1] : (nn == 1 ? wR[2] : wR[D]);
        }
        const real rL = wL[0], rR = wR[0], pL = wL[D + 1], pR = wR[D + 1];
        real sL, iL, sR, iR;
        FM<real>::sqrt_inv(rL, sL, iL);
        FM<real>::sqrt_inv(rR, sR, iR);
        const real inv = FM<real>::rcp(sL + sR);
        const real c2L = gam * pL * iL, c2R = gam * pR * iR;
        const real uroe = (sL * vnL + sR * vnR) * inv;
        const real du = vnR - vnL;
        const real d2 = (sL * c2L + sR * c2R) * inv + real(0.5) * sL * sR * inv * inv * du * du;
        const real a = fabs(uroe) + FM<real>::sqrtp(d2);
        real v2L = real(0), v2R = real(0);
#pragma unroll
        for (int d = 0; d < D; ++d) {
            v2L += wL[1 + d] * wL[1 + d];
            v2R += wR[1 + d] * wR[1 + d];
        }
        const real EL = pL * gm1i + real(0.5) * rL * v2L;
        const real ER = pR * gm1i + real(0.5) * rR * v2R;
        const real ha = real(0.5) * a;
        const real mL = rL * vnL, mR = rR * vnR;
        F[0] = real(0.5) * (mL + mR) - ha * (rR - rL);
#pragma unroll
        for (int d = 0; d < D; ++d) {
            real fl = mL * wL[1 + d] + mR * wR[1 + d];
            if (d == nn) fl += pL + pR;
            F[1 + d] = real(0.5) * fl - ha * (rR * wR[1 + d] - rL * wL[1 + d]);
        }
        F[D + 1] = real(0.5) * ((EL + pL) * vnL + (ER + pR) * vnR) - ha * (ER - EL);
    }

    // HLL flux with the same Einfeldt speeds: sL = min(u_roe - d, 0),
    // sR = max(u_roe + d, 0), F = (sR F_L - sL F_R + sL sR (U_R - U_L)) / (sR - sL)
    template <int NRM>
    __device__ static __forceinline__ void hll(const real *wL, const real *wR, int n, real gam, real gm1i, real *F) {
        const int nn = NRM >= 0 ? NRM : n;
        real vnL, vnR;
        if (NRM >= 0) {
            vnL = wL[1 + (NRM >= 0 ? NRM : 0)];
            vnR = wR[1 + (NRM >= 0 ? NRM : 0)];
        } else {
            vnL = nn == 0 ? wL[1] : (nn == 1 ? wL[2] : wL[D]);
            vnR = nn == 0 ? wR[1] : (nn == 1 ? wR[2] : wR[D]);
        }
        const real rL = wL[0], rR = wR[0], pL = wL[D + 1], pR = wR[D + 1];
        real sqL, iL, sqR, iR;
        FM<real>::sqrt_inv(rL, sqL, iL);
        FM<real>::sqrt_inv(rR, sqR, iR);
        const real inv = FM<real>::rcp(sqL + sqR);
        const real c2L = gam * pL * iL, c2R = gam * pR * iR;
        const real uroe = (sqL * vnL + sqR * vnR) * inv;
        const real du = vnR - vnL;
        const real d = FM<real>::sqrtp((sqL * c2L + sqR * c2R) * inv + real(0.5) * sqL * sqR * inv * inv * du * du);
        const real sL = fmin(uroe - d, real(0)), sR = fmax(uroe + d, real(0));
        const real iw = FM<real>::rcp(sR - sL), sLR = sL * sR;
        real v2L = real(0), v2R = real(0);
#pragma unroll
        for (int dd = 0; dd < D; ++dd) {
            v2L += wL[1 + dd] * wL[1 + dd];
            v2R += wR[1 + dd] * wR[1 + dd];
        }
        const real EL = pL * gm1i + real(0.5) * rL * v2L;
        const real ER = pR * gm1i + real(0.5) * rR * v2R;
        const real mL = rL * vnL, mR = rR * vnR;
        F[0] = (sR * mL - sL * mR + sLR * (rR - rL)) * iw;
#pragma unroll
        for (int dd = 0; dd < D; ++dd) {
            real fL = mL * wL[1 + dd], fR = mR * wR[1 + dd];
            if (dd == nn) {
                fL += pL;
                fR += pR;
            }
            F[1 + dd] = (sR * fL - sL * fR + sLR * (rR * wR[1 + dd] - rL * wL[1 + dd])) * iw;
        }
        F[D + 1] = (sR * (EL + pL) * vnL - sL * (ER + pR) * vnR + sLR * (ER - EL)) * iw;
    }

    // the configured numerical flux
    template <int NRM>
    __device__ static __forceinline__ void face_flux(int kind, const real *wL, const real *wR, int n, real gam, real gm1i,
                                                     real *F) {
        if (kind == 1) hll<NRM>(wL, wR, n, gam, gm1i, F);
        else flux<NRM>(wL, wR, n, gam, gm1i, F);
    }
    template <int NRM>
    __device__ static __forceinline__ void face_flux(int kind, const real *wL, const real *wR, int n, const PhysCtx<real> &c,
                                                     real *F) {
        face_flux<NRM>(kind, wL, wR, n, c.gam, c.gm1i, F);
    }

    static constexpr bool EULER = true;
    // rho <= 0 or p <= 0 (also catches NaN)
    __device__ static __forceinline__ bool nonphys(const real *w) { return !(w[0] > real(0)) || !(w[D + 1] > real(0)); }
    // variables whose face states must stay positive
    __device__ static __forceinline__ constexpr bool positive_var(int v) { return v == 0 || v == D + 1; }
    // sum_d (|v_d| + c) / dx_d of a conservative state (the CFL limit)
    __device__ static __forceinline__ real speed(const real *U, real gam, const real *idx, const PhysCtx<real> &) {
        real w[V];
        prim(U, w, gam);
        const real cs = FM<real>::sqrtp(gam * w[D + 1] * FM<real>::rcp(w[0]));
        real s = real(0);
#pragma unroll
        for (int d = 0; d < D; ++d) s += (fabs(w[1 + d]) + cs) * idx[d];
        return s;
    }
};

// Scalar advection (Sec. 3.4, Eq. 13) with a uniform velocity: one
// variable, primitive = conservative, physical flux rho v_n, wave speeds
// min(v_n, 0) and max(v_n, 0).  Rusanov: a = max of their magnitudes = |v_n|;
// HLL with sL = min(v_n, 0), sR = max(v_n, 0), and no flux where v_n = 0.
template <class real, int D>
struct Advect {
    static constexpr int V = 1;
    static constexpr bool EULER = false;
    __device__ static __forceinline__ void prim(const real *U, real *w, real) { w[0] = U[0]; }
    template <int NRM>
    __device__ static __forceinline__ void face_flux(int kind, const real *wL, const real *wR, int n, const PhysCtx<real> &c,
                                                     real *F) {
        const int nn = NRM >= 0 ? NRM : n;
        const real vn = nn == 0 ? c.vel[0] : (nn == 1 ? c.vel[1] : c.vel[2]);
        const real rL = wL[0], rR = wR[0];
        const real FL = rL * vn, FR = rR * vn;
        const real sL = vn < real(0) ? vn : real(0), sR = vn > real(0) ? vn : real(0);
        if (kind == 1) {
            F[0] = sR - sL == real(0) ? real(0) : (sR * FL - sL * FR + sL * sR * (rR - rL)) / (sR - sL);
        } else {
            const real a = fabs(sL) > fabs(sR) ? fabs(sL) : fabs(sR);
            F[0] = real(0.5) * (FL + FR) - real(0.5) * a * (rR - rL);
        }
    }
    __device__ static __forceinline__ bool nonphys(const real *) { return false; }
    __device__ static __forceinline__ constexpr bool positive_var(int) { return false; }
    __device__ static __forceinline__ real speed(const real *, real, const real *idx, const PhysCtx<real> &c) {
        real s = real(0);
#pragma unroll
        for (int d = 0; d < D; ++d) s += fabs(c.vel[d]) * idx[d];
        return s;
    }
};

// physics by code: 0 Euler, 1 scalar advection (amr_physics)
template <class real, int D, int PH>
using Phys = typename std::conditional<PH == 1, Advect<real, D>, Euler<real, D>>::type;

template <class real, int D, int N, int NG, int T, int PH = 0>
struct StageShape {
    static constexpr int V = Phys<real, D, PH>::V;
    static constexpr int P = T + 4;                  // plane pitch (tile + 2-cell halo each side)
    static constexpr int R = (D == 3) ? 5 : 1;       // ring depth
    static constexpr int S = N + 2 * NG;
    static constexpr int NT = T * T;                 // threads
    static constexpr int TILES = (D == 3) ? (N / T) * (N / T) : (N / T) * (N / T);
    static constexpr int NFX = T * (T + 1);          // faces per direction and plane
    static constexpr int NFS = T * (T + 2);          // cells with face states per direction and plane
    static constexpr bool PAIRS = (NG == 2);         // 2-element vector loads (rows start on even elements)
    static constexpr int HALO_PAIRS = P * P / 2;     // pairs of a halo plane incl. skipped corners
    static constexpr int GHOST_PAIRS = T * T / 2;    // pairs of a z-ghost plane (tile only)
    static constexpr int HALO_CELLS = T * P + 4 * T; // scalar path: cells of a halo plane
    static constexpr int LOADS = PAIRS ? (HALO_PAIRS + NT - 1) / NT : (HALO_CELLS + NT - 1) / NT;
    static constexpr int ITEMS = 2 * NFS;            // face-state work items per plane
    static constexpr size_t smem_bytes() {
        return sizeof(real) * (size_t(R) * V * P * P + 4 * size_t(V) * NFS + 2 * size_t(V) * NFX);
    }
};

// GEN = false: minmod and Rusanov fixed at compile time (the default scheme);
// GEN = true: the limiter and flux named in the arguments.  PH: physics
// (0 Euler, 1 scalar advection).
template <class real, int D, int N, int NG, int T, bool GEN, int PH>
__device__ __forceinline__ void stage_item(const StageArgs<real> &a, const Geom &g, int item) {
    using Sh = StageShape<real, D, N, NG, T, PH>;
    using E = Phys<real, D, PH>;
    using V2 = typename Vec2<real>::type;
    constexpr int V = Sh::V, P = Sh::P, S = Sh::S, NT = Sh::NT, NFX = Sh::NFX, NFS = Sh::NFS;
    constexpr int64_t NC = (D == 3) ? int64_t(S) * S * S : int64_t(S) * S;
    constexpr int PL = P * P;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real *ring = reinterpret_cast<real *>(smem_raw);          // [R][V][P*P]
    real *FSm = ring + Sh::R * V * PL;                         // [2][V][NFS] minus states (x, y)
    real *FSp = FSm + 2 * V * NFS;                             // [2][V][NFS] plus states
    real *Fx = FSp + 2 * V * NFS;                              // [V][T][T+1]
    real *Fy = Fx + V * NFX;                                   // [V][T+1][T]

    const int tid = threadIdx.x;
    const int b = item / Sh::TILES;
    const int tile = item - b * Sh::TILES;
    const int tx0 = (tile % (N / T)) * T, ty0 = (tile / (N / T)) * T;
    const int ti = tid % T, tj = tid / T;
    const BlockInfo info = a.info[b];
    const int gc = info.gclass;
    const real idx0 = real(g.inv_dx[3 * gc + 0]), idx1 = real(g.inv_dx[3 * gc + 1]);
    const real idx2 = (D == 3) ? real(g.inv_dx[3 * gc + 2]) : real(0);
    const real gam = a.gamma;
    const real gm1i = real(1) / (gam - real(1));
    const PhysCtx<real> pc{gam, gm1i, {a.vel[0], a.vel[1], a.vel[2]}};
    const real dt_eff = real(a.w_dt * a.sc_in[info.inst].dt);
    const int lim = GEN ? a.limiter : 0, flx = GEN ? a.flux : 0;
    const real *__restrict__ ub = a.deriv + int64_t(b) * V * NC;
    // halo source: in gather mode a cell outside the block across a face with
    // a same-level neighbour is read from that neighbour's interior
    // same-level neighbours (scalars: a runtime-indexed array would live in local memory)
    const int nb0 = a.gather ? info.nbr[0] : -1, nb1 = a.gather ? info.nbr[1] : -1;
    const int nb2 = a.gather ? info.nbr[2] : -1, nb3 = a.gather ? info.nbr[3] : -1;
    const int nb4 = a.gather ? info.nbr[4] : -1, nb5 = a.gather ? info.nbr[5] : -1;
    auto src_of = [&](int ii, int jj, int k, int64_t &o) -> const real * {
        int gi = tx0 + ii, gj = ty0 + jj, gk = k, nb = -1;
        if (gi < 0) { nb = nb0; gi += N; }
        else if (gi >= N) { nb = nb1; gi -= N; }
        else if (gj < 0) { nb = nb2; gj += N; }
        else if (gj >= N) { nb = nb3; gj -= N; }
        else if (D == 3 && gk < 0) { nb = nb4; gk += N; }
        else if (D == 3 && gk >= N) { nb = nb5; gk -= N; }
        if (nb >= 0) {
            o = (int64_t(D == 3 ? gk + NG : 0) * S + (gj + NG)) * S + (gi + NG);
            return a.deriv + int64_t(nb) * V * NC;
        }
        o = (int64_t(D == 3 ? k + NG : 0) * S + (ty0 + jj + NG)) * S + (tx0 + ii + NG);
        return ub;
    };

    bool nonphys = false;
    real vmax = real(0);

    auto gaddr = [&](int ii, int jj, int k) -> int64_t {
        return (int64_t(D == 3 ? k + NG : 0) * S + (ty0 + jj + NG)) * S + (tx0 + ii + NG);
    };
    auto is_halo_plane = [&](int k) { return D == 2 || (k >= 0 && k < N); };
    auto slot = [&](int k) -> real * { return ring + ((k + 2) % Sh::R) * V * PL; };

    // ------------------------------------------------------ plane loading
    // Pair path (NG = 2): a halo plane is P rows of P/2 pairs minus the 2x2
    // corner regions; a z-ghost plane is the T x T tile.  Every pair starts
    // on an even element, so 8- (float) or 16-byte (double) loads are aligned.
    real pre[Sh::LOADS][2][V];
    auto pair_of = [&](int p, bool halo, int &ii, int &jj) -> bool {
        if (halo) {
            if (p >= Sh::HALO_PAIRS) return false;
            jj = p / (P / 2) - 2;
            ii = 2 * (p % (P / 2)) - 2;
            return !((jj < 0 || jj >= T) && (ii < 0 || ii >= T));
        }
        if (p >= Sh::GHOST_PAIRS) return false;
        jj = p / (T / 2);
        ii = 2 * (p % (T / 2));
        return true;
    };
    auto scalar_cell = [&](int c, bool halo, int &ii, int &jj) -> bool {
        if (!halo) {
            if (c >= T * T) return false;
            ii = c % T;
            jj = c / T;
            return true;
        }
        if (c >= Sh::HALO_CELLS) return false;
        if (c < T * P) {
            jj = c / P;
            ii = c % P - 2;
            return true;
        }
        c -= T * P;
        const int r = c / T;
        ii = c % T;
        jj = (r < 2) ? r - 2 : T + r - 2;
        return true;
    };
    auto prefetch = [&](int k) {
        const bool halo = is_halo_plane(k);
#pragma unroll
        for (int l = 0; l < Sh::LOADS; ++l) {
            int ii, jj;
            if (Sh::PAIRS) {
                if (pair_of(tid + l * NT, halo, ii, jj)) {
                    int64_t o;
                    const real *src = src_of(ii, jj, k, o);
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        const V2 x = *reinterpret_cast<const V2 *>(src + v * NC + o);
                        pre[l][0][v] = x.x;
                        pre[l][1][v] = x.y;
                    }
                }
            } else if (scalar_cell(tid + l * NT, halo, ii, jj)) {
                int64_t o;
                const real *src = src_of(ii, jj, k, o);
#pragma unroll
                for (int v = 0; v < V; ++v) pre[l][0][v] = src[v * NC + o];
            }
        }
    };
    auto commit = [&](int k) {
        real *pl = slot(k);
        const bool halo = is_halo_plane(k);
#pragma unroll
        for (int l = 0; l < Sh::LOADS; ++l) {
            int ii, jj;
            const bool ok = Sh::PAIRS ? pair_of(tid + l * NT, halo, ii, jj) : scalar_cell(tid + l * NT, halo, ii, jj);
            if (!ok) continue;
            const int o = (jj + 2) * P + (ii + 2);
#pragma unroll
            for (int e = 0; e < (Sh::PAIRS ? 2 : 1); ++e) {
                real w[V];
                E::prim(pre[l][e], w, gam);
                nonphys |= E::nonphys(w);
#pragma unroll
                for (int v = 0; v < V; ++v) pl[v * PL + o + e] = w[v];
            }
        }
    };

    // ------------------------------------------------------ phase A: states
    // item q < NFS: x states of cell (q % (T+2) - 1, q / (T+2));
    // item q >= NFS: y states of cell (q' % T, q' / T - 1), q' = q - NFS.
    auto face_states = [&](int k) {
        const real *pl = slot(k);
        for (int q = tid; q < Sh::ITEMS; q += NT) {
            const int dir = q >= NFS;
            const int qq = q - dir * NFS;
            int ii, jj, st;
            if (!dir) {
                jj = qq / (T + 2);
                ii = qq - jj * (T + 2) - 1;
                st = 1;
            } else {
                jj = qq / T - 1;
                ii = qq % T;
                st = P;
            }
            const int c = (jj + 2) * P + (ii + 2);
            bool bad = false;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const real w0 = pl[v * PL + c], wm = pl[v * PL + c - st], wp = pl[v * PL + c + st];
                real lo, hi;
                cell_faces<real>(lim, wm, w0, wp, lo, hi);
                if (E::positive_var(v)) bad |= !(lo > real(0)) || !(hi > real(0));
                FSm[(dir * V + v) * NFS + qq] = lo;
                FSp[(dir * V + v) * NFS + qq] = hi;
            }
            nonphys |= bad;
        }
    };
    // z face states of cell (ti, tj, kz) from planes kz-1, kz, kz+1
    auto z_states = [&](int kz, real *zm, real *zp) {
        const int c = (tj + 2) * P + (ti + 2);
        const real *p0 = slot(kz - 1), *p1 = slot(kz), *p2 = slot(kz + 1);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const real w0 = p1[v * PL + c], wm = p0[v * PL + c], wp = p2[v * PL + c];
            cell_faces<real>(lim, wm, w0, wp, zm[v], zp[v]);
        }
        nonphys |= E::nonphys(zm) || E::nonphys(zp);
    };

    const int nface_b = (D == 3) ? N * N : N;
    auto store_bflux = [&](int f, int t, const real *F) {
        const int sl = info.bslot[f];
        if (sl < 0) return;
        real *dst = a.bflux + int64_t(sl) * V * nface_b + t;
#pragma unroll
        for (int v = 0; v < V; ++v) dst[v * nface_b] = F[v];
    };

    // ------------------------------------------------------ phase B: fluxes
    auto x_face = [&](int q, int k) {
        const int jj = q / (T + 1), fi = q - jj * (T + 1);
        real wL[V], wR[V], F[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            wL[v] = FSp[v * NFS + jj * (T + 2) + fi];
            wR[v] = FSm[v * NFS + jj * (T + 2) + fi + 1];
        }
        E::template face_flux<0>(flx, wL, wR, 0, pc, F);
#pragma unroll
        for (int v = 0; v < V; ++v) Fx[v * NFX + q] = F[v];
        if (fi == 0 && tx0 == 0) store_bflux(0, ty0 + jj + N * k, F);
        if (fi == T && tx0 + T == N) store_bflux(1, ty0 + jj + N * k, F);
    };
    auto y_face = [&](int q, int k) {
        const int fj = q / T, ii = q - fj * T;
        real wL[V], wR[V], F[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            wL[v] = FSp[(V + v) * NFS + fj * T + ii];
            wR[v] = FSm[(V + v) * NFS + (fj + 1) * T + ii];
        }
        E::template face_flux<1>(flx, wL, wR, 1, pc, F);
#pragma unroll
        for (int v = 0; v < V; ++v) Fy[v * NFX + q] = F[v];
        if (fj == 0 && ty0 == 0) store_bflux(2, tx0 + ii + N * k, F);
        if (fj == T && ty0 + T == N) store_bflux(3, tx0 + ii + N * k, F);
    };
    // the 2T faces left over after T*T threads took one x- and one y-face:
    // lanes < T take an x-face, the others a y-face (runtime normal, so the
    // warp does not split into two flux evaluations)
    auto extra_face = [&](int k) {
        const int dir = tid >= T;
        const int q = NT + (dir ? tid - T : tid);
        int iL, iR, fa, fb;
        if (!dir) {
            const int jj = q / (T + 1), fi = q - jj * (T + 1);
            iL = jj * (T + 2) + fi;
            iR = iL + 1;
            fa = fi;
            fb = jj;
        } else {
            const int fj = q / T, ii = q - fj * T;
            iL = fj * T + ii;
            iR = iL + T;
            fa = fj;
            fb = ii;
        }
        real wL[V], wR[V], F[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            wL[v] = FSp[(dir * V + v) * NFS + iL];
            wR[v] = FSm[(dir * V + v) * NFS + iR];
        }
        E::template face_flux<-1>(flx, wL, wR, dir, pc, F);
        real *Fd = dir ? Fy : Fx;
#pragma unroll
        for (int v = 0; v < V; ++v) Fd[v * NFX + q] = F[v];
        // the leftover faces are the last x row / y row of the tile
        if (!dir) {
            if (fa == 0 && tx0 == 0) store_bflux(0, ty0 + fb + N * k, F);
            if (fa == T && tx0 + T == N) store_bflux(1, ty0 + fb + N * k, F);
        } else {
            if (fa == 0 && ty0 == 0) store_bflux(2, tx0 + fb + N * k, F);
            if (fa == T && ty0 + T == N) store_bflux(3, tx0 + fb + N * k, F);
        }
    };

    // ------------------------------------------------------ phase C: update
    real Fz_lo[V], Fz_hi[V];
    auto update = [&](int k) {
        const int64_t o = gaddr(ti, tj, k);
        const int64_t ob = int64_t(b) * V * NC + o;
        real U[V], src[V];
#pragma unroll
        for (int v = 0; v < V; ++v) src[v] = real(0);
        if constexpr (E::EULER) {
            if (a.gravity_on) {
                // S = (0, rho g, rho g.u) from the conservative state of the cell
                const real *uc = a.deriv + ob;
                const real rho = uc[0];
                real sg = real(0);
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    src[1 + d] = rho * a.grav[d];
                    sg += uc[(1 + d) * NC] * a.grav[d];
                }
                src[V - 1] = sg;
            }
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
            real du = (Fx[v * NFX + tj * (T + 1) + ti] - Fx[v * NFX + tj * (T + 1) + ti + 1]) * idx0 +
                      (Fy[v * NFX + tj * T + ti] - Fy[v * NFX + (tj + 1) * T + ti]) * idx1;
            if (D == 3) du += (Fz_lo[v] - Fz_hi[v]) * idx2;
            du += src[v];
            real acc = real(0);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q < a.nprev) acc += a.wprev[q] * a.prev[q][ob + v * NC];
            U[v] = dt_eff * du + acc;
            a.out[ob + v * NC] = U[v];
        }
        // complete the row's DRAM sectors: the output's x-ghost cells
        if (tx0 + ti == 0 || tx0 + ti == N - 1) {
            const int64_t og = ob + (tx0 + ti == 0 ? -NG : 1);
#pragma unroll
            for (int v = 0; v < V; ++v)
#pragma unroll
                for (int e = 0; e < NG; ++e) a.out[og + v * NC + e] = real(0);
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
                const real idx[3] = {idx0, idx1, idx2};
                const real s = E::speed(U, gam, idx, pc);
                vmax = s > vmax ? s : vmax;
            }
        }
    };

    // ------------------------------------------------------ the march
    if (D == 3) {
        for (int k = -2; k <= 2; ++k) {
            prefetch(k);
            commit(k);
        }
        __syncthreads();
        {
            real zm[V], zp[V], pm1[V];
            z_states(-1, zm, pm1);          // plus state of cell -1
            z_states(0, zm, zp);            // minus / plus states of cell 0
            E::template face_flux<2>(flx, pm1, zm, 2, pc, Fz_lo);
            store_bflux(4, tx0 + ti + N * (ty0 + tj), Fz_lo);
#pragma unroll
            for (int v = 0; v < V; ++v) Fz_hi[v] = zp[v];     // carries plus(0) into the loop
        }
        real zplus[V], zm1[V], zp1[V];
#pragma unroll
        for (int v = 0; v < V; ++v) zplus[v] = Fz_hi[v];
        prefetch(3);
        face_states(0);
        z_states(1, zm1, zp1);
        __syncthreads();
        for (int k = 0; k < N; ++k) {
            // phase B
            x_face(tid, k);
            y_face(tid, k);
            if (tid < 2 * T) extra_face(k);
            E::template face_flux<2>(flx, zplus, zm1, 2, pc, Fz_hi);
            if (k == N - 1) store_bflux(5, tx0 + ti + N * (ty0 + tj), Fz_hi);
#pragma unroll
            for (int v = 0; v < V; ++v) zplus[v] = zp1[v];
            if (k + 3 <= N + 1) commit(k + 3);
            __syncthreads();
            // phase C (plane k) + phase A (plane k + 1)
            if (k + 1 < N && k + 4 <= N + 1) prefetch(k + 4);
            update(k);
#pragma unroll
            for (int v = 0; v < V; ++v) Fz_lo[v] = Fz_hi[v];
            if (k + 1 < N) {
                face_states(k + 1);
                z_states(k + 2, zm1, zp1);
            }
            __syncthreads();
        }
    } else {
        prefetch(0);
        commit(0);
        __syncthreads();
        face_states(0);
        __syncthreads();
        x_face(tid, 0);
        y_face(tid, 0);
        if (tid < 2 * T) extra_face(0);
        __syncthreads();
        update(0);
        __syncthreads();   // shared memory is reused by the CTA's next item
    }

    // ---- CTA reductions: max speed and non-physical flag
    if (a.update_dt) {
        double m = double(vmax);
        for (int s = 16; s > 0; s >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, s));
        if ((tid & 31) == 0) atomic_max_nonneg(&a.sc[info.inst].maxspeed_bits, m);
    }
    if (__syncthreads_or(nonphys) && tid == 0) raise_status(&a.sc[0].status, 7);
}

// CTAs take items (block, column tile) with a grid stride: one CTA per item
// when the grid covers them all, a persistent sweep when it is smaller.
template <class real, int D, int N, int NG, int T, bool GEN, int PH>
__global__ void __launch_bounds__(T * T) k_stage(StageArgs<real> a, Geom g) {
    for (int item = blockIdx.x; item < a.n_items; item += gridDim.x) stage_item<real, D, N, NG, T, GEN, PH>(a, g, item);
}

}  // namespace amrb
