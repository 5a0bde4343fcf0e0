// FP32 stage kernel for scalar advection (Sec. 3.4, Eq. 13) with two ghost
// layers and a MUSCL slope limiter (minmod, MC, van Leer): the sub-step of
// Eq. 5 on blocks of one variable.  With one variable a block with its face
// halo is small (20^3 floats = 32 KB for 16^3), so one CTA copies a whole
// block -- in gather mode the halo straight from the same-level neighbours
// -- into shared memory with cp.async, and every thread then updates pairs
// of x-neighbour cells with packed two-wide FP32 arithmetic: its pair's
// x faces from three aligned pairs, y faces from five rows, and in 3D a march
// over a segment of z planes that carries the z states and the lower z flux
// in registers.  With the wave speeds min(v,0), max(v,0) both flux schemes
// are F = max(v,0) rho_L + min(v,0) rho_R (the coefficients are exact in
// either formula).  Blocks of 8^3 and 16^3 (3D) and 8^2..32^2 (2D).
#pragma once

#include "stage_pair.cuh"

namespace amrb {

// 16-byte asynchronous global -> shared copy (both addresses 16-byte aligned)
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    const unsigned d = unsigned(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}

template <int D, int N>
struct AdvShape {
    static constexpr int NG = 2, S = N + 4, PL = S * S;
    static constexpr int ZS = D == 3 ? 2 : 1;               // z segments per pair column (3D)
    static constexpr int KZ = D == 3 ? N / ZS : 1;          // planes per segment
    static constexpr int NT = (N / 2) * N * ZS;             // threads
    static constexpr int ROWS = D == 3 ? N * N : N;         // interior rows (j, k)
    // copies of an interior row: 8-byte pairs at i = -2, 0, N-2, N (the x
    // halo may come from another block) and 16-byte chunks at i = 2, 6, ..,
    // N-6; of a y- or z-halo row: the S/4 16-byte chunks of the whole row
    static constexpr int QC = (N - 4) / 4;                  // 16-byte chunks of an interior row
    static constexpr int IR = 4 + QC;                       // copies per interior row
    static constexpr int HR = S / 4;                        // copies per halo row
    static constexpr int HROWS = D == 3 ? 8 * N : 4;        // y-halo rows (4 per plane) + z-halo rows
    static constexpr int NA = ROWS * IR;
    static constexpr int NCOPY = NA + HROWS * HR;
    static constexpr size_t smem_bytes() { return sizeof(float) * (D == 3 ? size_t(S) * PL : size_t(PL)); }
};

// 3D 16^3: 6 CTAs of 256 threads per SM (32 KB of shared memory each).
// NPREV: previous states fixed at compile time (1 or 2), -1 from the arguments.
template <int D, int N, int LIM, int NPREV>
__global__ void __launch_bounds__(AdvShape<D, N>::NT, (D == 3 && N == 16 ? 6 : 1)) k_adv_pair(StageArgs<float> a, Geom g) {
    using Sh = AdvShape<D, N>;
    constexpr int NG = Sh::NG, S = Sh::S, PL = Sh::PL, NT = Sh::NT, KZ = Sh::KZ;
    constexpr int64_t NCELL = D == 3 ? int64_t(S) * S * S : int64_t(S) * S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *sm = reinterpret_cast<float *>(smem_raw);
    const int tid = threadIdx.x;
    int ip, tj;
    const int zs = tid / ((N / 2) * N);
    if constexpr (N == 16) {
        // the two 8-lane row groups of a half-warp take rows r and r + 4
        // (80 words apart: opposite bank halves, conflict-free 8-byte loads)
        const int lt = tid % 128, lane = lt & 31, q = (lt >> 5) * 2 + (lane >> 4);
        ip = lane & 7;
        tj = (q & 3) + (q >> 2) * 8 + ((lane >> 3) & 1) * 4;
    } else {
        ip = tid % (N / 2);
        tj = (tid / (N / 2)) % N;
    }
    const int ci = 2 * ip;
    const float cl[3] = {fmaxf(a.vel[0], 0.f), fmaxf(a.vel[1], 0.f), fmaxf(a.vel[2], 0.f)};
    const float cr[3] = {fminf(a.vel[0], 0.f), fminf(a.vel[1], 0.f), fminf(a.vel[2], 0.f)};
    auto flux = [&](int n, float2 L, float2 R) -> float2 { return PF::fma(PF::sp(cr[n]), R, PF::mul(PF::sp(cl[n]), L)); };
    auto soff = [&](int i, int j, int k) -> int { return (D == 3 ? (k + NG) * PL : 0) + (j + NG) * S + (i + NG); };
    auto gofs = [&](int i, int j, int k) -> int64_t {
        return (int64_t(D == 3 ? k + NG : 0) * S + (j + NG)) * S + (i + NG);
    };
    auto ld2 = [&](int i, int j, int k) -> float2 { return *reinterpret_cast<const float2 *>(sm + soff(i, j, k)); };
    const int nface = D == 3 ? N * N : N;

    for (int b = blockIdx.x; b < a.n_items; b += gridDim.x) {
        const BlockInfo info = a.info[b];
        const float *ub = a.deriv + int64_t(b) * NCELL;
        const int nb0 = a.gather ? info.nbr[0] : -1, nb1 = a.gather ? info.nbr[1] : -1;
        const int nb2 = a.gather ? info.nbr[2] : -1, nb3 = a.gather ? info.nbr[3] : -1;
        const int nb4 = (D == 3 && a.gather) ? info.nbr[4] : -1, nb5 = (D == 3 && a.gather) ? info.nbr[5] : -1;
        // ---- copies: interior rows with their x halo (from the x neighbours
        // in gather mode), then the y- and z-halo rows (from the neighbours)
        for (int p = tid; p < Sh::NCOPY; p += NT) {
            if (p < Sh::NA) {
                const int row = p / Sh::IR, part = p - row * Sh::IR;
                const int j = row % N, k = D == 3 ? row / N : 0;
                if (part >= 2 && part < 2 + Sh::QC) {
                    const int i = 2 + 4 * (part - 2);
                    cp_async16(sm + soff(i, j, k), ub + gofs(i, j, k));
                } else {
                    const int i = part == 0 ? -2 : (part == 1 ? 0 : (part == 2 + Sh::QC ? N - 2 : N));
                    const float *src = ub + gofs(i, j, k);
                    if (i < 0 && nb0 >= 0) src = a.deriv + int64_t(nb0) * NCELL + gofs(i + N, j, k);
                    if (i >= N && nb1 >= 0) src = a.deriv + int64_t(nb1) * NCELL + gofs(i - N, j, k);
                    cp_async8(sm + soff(i, j, k), src);
                }
            } else {
                const int q = p - Sh::NA, row = q / Sh::HR, c = q - row * Sh::HR;
                int j, k, nb, sj, sk;
                if (row < (D == 3 ? 4 * N : 4)) {        // y halo: 4 rows per plane
                    const int jr = row % 4;
                    k = D == 3 ? row / 4 : 0;
                    j = jr < 2 ? jr - 2 : N + jr - 2;
                    nb = jr < 2 ? nb2 : nb3;
                    sj = jr < 2 ? j + N : j - N;
                    sk = k;
                } else {                                  // z halo: rows of 4 planes
                    const int r2 = row - 4 * N, kr = r2 / N;
                    j = r2 % N;
                    k = kr < 2 ? kr - 2 : N + kr - 2;
                    nb = kr < 2 ? nb4 : nb5;
                    sj = j;
                    sk = kr < 2 ? k + N : k - N;
                }
                const int i = 4 * c - 2;
                const float *src = nb >= 0 ? a.deriv + int64_t(nb) * NCELL + gofs(i, sj, sk) : ub + gofs(i, j, k);
                cp_async16(sm + soff(i, j, k), src);
            }
        }
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();

        const int gc = info.gclass;
        const float idx0 = float(g.inv_dx[3 * gc]), idx1 = float(g.inv_dx[3 * gc + 1]);
        const float idx2 = D == 3 ? float(g.inv_dx[3 * gc + 2]) : 0.f;
        const float dte = float(a.w_dt * a.sc_in[info.inst].dt);
        auto store_b1 = [&](int f, int t, float v) {
            const int sl = info.bslot[f];
            if (sl >= 0) a.bflux[int64_t(sl) * nface + t] = v;
        };
        auto store_b2 = [&](int f, int t, float2 v) {
            const int sl = info.bslot[f];
            if (sl >= 0) {
                a.bflux[int64_t(sl) * nface + t] = v.x;
                a.bflux[int64_t(sl) * nface + t + 1] = v.y;
            }
        };
        const int k0 = D == 3 ? zs * KZ : 0;
        float2 zm_next = PF::sp(0.f), zp_cur = PF::sp(0.f), Fz_lo = PF::sp(0.f);
        if constexpr (D == 3) {
            // states of planes k0 - 1 (plus) and k0 (minus, plus), lower z flux
            const float2 zA = ld2(ci, tj, k0 - 2), zB = ld2(ci, tj, k0 - 1), zC = ld2(ci, tj, k0), zD = ld2(ci, tj, k0 + 1);
            float2 m1, p1, m0, p0;
            pair_cell_states<LIM>(zA, zB, zC, m1, p1);
            pair_cell_states<LIM>(zB, zC, zD, m0, p0);
            Fz_lo = flux(2, p1, m0);
            zp_cur = p0;
            if (k0 == 0) store_b2(4, ci + N * tj, Fz_lo);
        }
        for (int kk = 0; kk < KZ; ++kk) {
            const int k = k0 + kk;
            // x faces ci, ci+1, ci+2 of row (tj, k)
            const float2 A = ld2(ci - 2, tj, k), B = ld2(ci, tj, k), C = ld2(ci + 2, tj, k);
            float2 M, P, Mo, Po;
            pair_cell_states<LIM>(make_float2(A.y, B.x), B, make_float2(B.y, C.x), M, P);          // cells ci, ci+1
            pair_cell_states<LIM>(make_float2(A.x, B.y), make_float2(A.y, C.x), make_float2(B.x, C.y), Mo, Po);  // ci-1, ci+2
            const float2 FxL = flux(0, make_float2(Po.x, P.x), M);
            const float2 FxH = flux(0, P, make_float2(M.y, Mo.y));
            float2 du = PF::mul(PF::sub(FxL, FxH), PF::sp(idx0));
            if (ci == 0) store_b1(0, tj + N * k, FxL.x);
            if (ci == N - 2) store_b1(1, tj + N * k, FxH.y);
            // y faces tj, tj+1 of columns ci, ci+1
            const float2 R0 = ld2(ci, tj - 2, k), R1 = ld2(ci, tj - 1, k), R3 = ld2(ci, tj + 1, k), R4 = ld2(ci, tj + 2, k);
            float2 ym1, yp1, ym0, yp0, ym2, yp2;
            pair_cell_states<LIM>(R0, R1, B, ym1, yp1);
            pair_cell_states<LIM>(R1, B, R3, ym0, yp0);
            pair_cell_states<LIM>(B, R3, R4, ym2, yp2);
            const float2 FyL = flux(1, yp1, ym0), FyH = flux(1, yp0, ym2);
            du = PF::fma(PF::sub(FyL, FyH), PF::sp(idx1), du);
            if (tj == 0) store_b2(2, ci + N * k, FyL);
            if (tj == N - 1) store_b2(3, ci + N * k, FyH);
            if constexpr (D == 3) {
                // z face k + 1/2: plus state of plane k (carried), minus of k+1
                const float2 z2 = ld2(ci, tj, k + 2);
                float2 p_next;
                pair_cell_states<LIM>(B, ld2(ci, tj, k + 1), z2, zm_next, p_next);
                const float2 Fz_hi = flux(2, zp_cur, zm_next);
                du = PF::fma(PF::sub(Fz_lo, Fz_hi), PF::sp(idx2), du);
                if (k == N - 1) store_b2(5, ci + N * tj, Fz_hi);
                Fz_lo = Fz_hi;
                zp_cur = p_next;
            }
            // Eq. 5: u_out = w_dt dt du + sum_q w_q u_q
            const int64_t ob = int64_t(b) * NCELL + gofs(ci, tj, k);
            float2 acc = PF::sp(0.f);
#pragma unroll
            for (int q = 0; q < (NPREV > 0 ? NPREV : 4); ++q)
                if (NPREV > 0 || q < a.nprev)
                    acc = PF::fma(PF::sp(a.wprev[q]), *reinterpret_cast<const float2 *>(a.prev[q] + ob), acc);
            *reinterpret_cast<float2 *>(a.out + ob) = PF::fma(PF::sp(dte), du, acc);
            // complete the row's DRAM sectors: the output's x-ghost cells
            if (ci == 0) *reinterpret_cast<float2 *>(a.out + ob - NG) = PF::sp(0.f);
            if (ci == N - 2) *reinterpret_cast<float2 *>(a.out + ob + 2) = PF::sp(0.f);
        }
        if (a.update_dt && tid == 0) {
            // the CFL speed sum_d |v_d| / dx_d is the same in every cell
            float s = fabsf(a.vel[0]) * idx0;
            s += fabsf(a.vel[1]) * idx1;
            if (D == 3) s += fabsf(a.vel[2]) * idx2;
            atomic_max_nonneg(&a.sc[info.inst].maxspeed_bits, double(s));
        }
        __syncthreads();   // shared memory is reused by the CTA's next block
    }
}

}  // namespace amrb
