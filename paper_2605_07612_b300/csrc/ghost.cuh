// Ghost-pattern executor (Sec. 2.6).  `parts` warps per pattern entry
// ("strip"), each taking every parts-th group of 128 values (32 for edge and
// corner regions), so that a few large strips (a boundary face of 32^3
// blocks) still spread over many warps; the lanes walk the strip's ghost
// cells with x fastest so that both the gather and the scatter are coalesced
// along rows.  Round 1 executes SRL,
// F2C and BC entries (they read interior cells only); round 2 executes C2F
// entries, whose limited prolongation reads round-1 ghosts of the coarse
// block (the tangential neighbours at the face edge and the ghost layer
// facing the fine block).  Face ghost cells only (Sec. 2.1), unless the mesh
// asks for edge and corner cells (DIAG entries: copies and restrictions in
// round 1, prolongations in round 2).
#pragma once

#include "common.cuh"

namespace amrb {

template <class real>
struct GhostArgs {
    real *u;                 // state slot, max_blocks blocks
    const Entry *list;
    int n;
    int parts;               // warps per entry
    const real *bcdata;      // [n_bc][V][N^(D-1)]
    const int32_t *bc_type;  // [instance][6]
    const real *bc_val;      // [instance][6][8]
    const BlockInfo *info;   // per block: instance and geometry class
};

// Restriction (Sec. 2.2): mean of the 2^D fine cells starting at fine index
// (fi, fj, fk), summed x-pairs, then y-pairs, then z-pairs, then scaled.
template <class real, int D>
__device__ __forceinline__ real restrict_at(const real *fb, const Geom &g, int fi, int fj, int fk) {
    const int S = g.S;
    const real *p = fb + cell_index<real>(g, fi, fj, fk);
    real s00 = p[0] + p[1];
    real s10 = p[S] + p[S + 1];
    real s0 = s00 + s10;
    if (D == 3) {
        const real *q = p + int64_t(S) * S;
        real s01 = q[0] + q[1];
        real s11 = q[S] + q[S + 1];
        real s1 = s01 + s11;
        return (s0 + s1) * real(0.125);
    }
    return s0 * real(0.25);
}

// Limited prolongation (Sec. 2.2, Eq. 1 with theta = 1): the fine value at
// sub-position sub_d (0 lower, 1 upper half) of coarse cell (ci, cj, ck) is
// u_c + sum_d (+-1/4) minmod(u_c - u_{c-e_d}, u_{c+e_d} - u_c), the
// corrections summed left to right before being added to u_c.
template <class real, int D>
__device__ __forceinline__ real prolong_at(const real *cb, const Geom &g, int ci, int cj, int ck, int si, int sj, int sk) {
    const int64_t S = g.S;
    const real *p = cb + cell_index<real>(g, ci, cj, ck);
    const real uc = p[0];
    real t = (si ? real(0.25) : real(-0.25)) * minmod<real>(uc - p[-1], p[1] - uc);
    t = t + (sj ? real(0.25) : real(-0.25)) * minmod<real>(uc - p[-S], p[S] - uc);
    if (D == 3) t = t + (sk ? real(0.25) : real(-0.25)) * minmod<real>(uc - p[-S * S], p[S * S] - uc);
    return uc + t;
}

// Same-level copy of one strip with 2-element vectors (Ng even: every row
// segment of the strip starts on an even element, so the vectors are
// aligned).  ND = face-normal dimension.  Each lane keeps 4 independent
// loads in flight before storing.
template <class real, int D, int N, int NG, int ND>
__device__ __forceinline__ void srl_pairs(real *dstb, const real *srcb, int side, int lane, int part, int parts, int V) {
    using V2 = typename Vec2<real>::type;
    constexpr int S = N + 2 * NG;
    constexpr int64_t NCc = (D == 3) ? int64_t(S) * S * S : int64_t(S) * S;
    constexpr int T1 = (D == 3) ? N : 1;
    constexpr int UPV = (ND == 0) ? N * T1 * (NG / 2) : NG * T1 * (N / 2);
    const int TOTAL = V * UPV;
    const int lo = side ? N : -NG, shift = side ? -N : N;
    auto cidx = [](int i, int j, int k) -> int64_t {
        return (int64_t(D == 3 ? k + NG : 0) * S + (j + NG)) * S + (i + NG);
    };
    for (int base = lane + 128 * part; base < TOTAL; base += 128 * parts) {
        V2 val[4];
        int64_t od[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int u = base + 32 * r;
            od[r] = -1;
            if (u < TOTAL) {
                const int v = u / UPV, rem = u - v * UPV;
                int i, j, k;
                if (ND == 0) {
                    const int pp = rem % (NG / 2), row = rem / (NG / 2);
                    j = row % N;
                    k = (D == 3) ? row / N : 0;
                    i = lo + 2 * pp;
                } else if (ND == 1) {
                    const int pp = rem % (N / 2), t = rem / (N / 2);
                    j = lo + t % NG;
                    k = (D == 3) ? t / NG : 0;
                    i = 2 * pp;
                } else {
                    const int pp = rem % (N / 2), t = rem / (N / 2);
                    j = t % N;
                    k = lo + t / N;
                    i = 2 * pp;
                }
                const int is = ND == 0 ? i + shift : i, js = ND == 1 ? j + shift : j, ks = ND == 2 ? k + shift : k;
                val[r] = *reinterpret_cast<const V2 *>(srcb + v * NCc + cidx(is, js, ks));
                od[r] = v * NCc + cidx(i, j, k);
            }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
            if (od[r] >= 0) *reinterpret_cast<V2 *>(dstb + od[r]) = val[r];
    }
}

// Round-2 strip of one fine block's face (C2F), by coarse cell: each coarse
// cell's three limited slopes are taken once and give its 2^D fine ghost
// cells inside the strip (the fine layers nearest the face when Ng is odd),
// each evaluated exactly as prolong_at does.  ND = face-normal dimension.
template <class real, int D, int N, int NG, int ND>
__device__ __forceinline__ void c2f_strip(const Geom &g, const Entry &e, real *dstb, const real *srcb, int lane, int part,
                                          int parts) {
    constexpr int T0 = ND == 0 ? 1 : 0, T1 = ND == 2 ? 1 : 2;
    constexpr int CL = (NG + 1) / 2;                 // coarse layers the strip covers
    constexpr int H = N / 2;
    constexpr int UPV = CL * H * (D == 3 ? H : 1);   // coarse cells per variable
    const int side = e.face & 1;
    int off[3] = {0, 0, 0};                          // the fine block's half of the coarse face
    off[T0] = e.offset & 1;
    if (D == 3) off[T1] = (e.offset >> 1) & 1;
    const int64_t S = g.S;
    const int total = UPV * g.V;
    for (int u = lane + 32 * part; u < total; u += 32 * parts) {
        const int v = u / UPV;
        int r = u - v * UPV;
        const int k = r % CL;
        r /= CL;
        const int c0 = r % H, c1 = (D == 3) ? r / H : 0;
        const int cn = side ? k : -1 - k;            // coarse layer relative to the face
        int y[3] = {0, 0, 0};
        y[T0] = off[T0] * H + c0;
        if (D == 3) y[T1] = off[T1] * H + c1;
        y[ND] = side ? cn : N + cn;
        const real *p = srcb + int64_t(v) * g.ncell + cell_index<real>(g, y[0], y[1], y[2]);
        const real uc = p[0];
        const real m0 = minmod<real>(uc - p[-1], p[1] - uc);
        const real m1 = minmod<real>(uc - p[-S], p[S] - uc);
        const real m2 = D == 3 ? minmod<real>(uc - p[-S * S], p[S * S] - uc) : real(0);
        real *db = dstb + int64_t(v) * g.ncell;
        if constexpr (NG % 2 == 0) {
            // both x children in one aligned 2-element store (Ng even: all
            // children lie in the strip and x + Ng of the lower one is even)
            using V2 = typename Vec2<real>::type;
#pragma unroll
            for (int ch = 0; ch < (1 << D); ch += 2) {
                const int sb1 = (ch >> 1) & 1, sb2 = (ch >> 2) & 1;
                int x[3] = {0, 0, 0};
                if (ND == 0) {
                    x[0] = side ? 2 * cn + N : 2 * cn;
                    x[1] = 2 * c0 + sb1;
                    if (D == 3) x[2] = 2 * c1 + sb2;
                } else {
                    x[0] = 2 * c0;
                    x[ND] = side ? 2 * cn + (ND == 1 ? sb1 : sb2) + N : 2 * cn + (ND == 1 ? sb1 : sb2);
                    if (D == 3) x[ND == 1 ? 2 : 1] = 2 * c1 + (ND == 1 ? sb2 : sb1);
                }
                real t0 = real(-0.25) * m0, t1 = real(0.25) * m0;
                t0 = t0 + (sb1 ? real(0.25) : real(-0.25)) * m1;
                t1 = t1 + (sb1 ? real(0.25) : real(-0.25)) * m1;
                if (D == 3) {
                    t0 = t0 + (sb2 ? real(0.25) : real(-0.25)) * m2;
                    t1 = t1 + (sb2 ? real(0.25) : real(-0.25)) * m2;
                }
                V2 pr;
                pr.x = uc + t0;
                pr.y = uc + t1;
                *reinterpret_cast<V2 *>(db + cell_index<real>(g, x[0], x[1], x[2])) = pr;
            }
            continue;
        }
#pragma unroll
        for (int ch = 0; ch < (1 << D); ++ch) {
            const int sb[3] = {ch & 1, (ch >> 1) & 1, (ch >> 2) & 1};
            const int xn = 2 * cn + sb[ND];          // fine layer relative to the face
            if (side ? xn >= NG : xn < -NG) continue;
            int x[3] = {0, 0, 0};
            x[T0] = 2 * c0 + sb[T0];
            if (D == 3) x[T1] = 2 * c1 + sb[T1];
            x[ND] = side ? xn + N : xn;
            real t = (sb[0] ? real(0.25) : real(-0.25)) * m0;
            t = t + (sb[1] ? real(0.25) : real(-0.25)) * m1;
            if (D == 3) t = t + (sb[2] ? real(0.25) : real(-0.25)) * m2;
            db[cell_index<real>(g, x[0], x[1], x[2])] = uc + t;
        }
    }
}

// One face strip of round 1 (F2C, BC, and SRL when NG is odd),
// ND = face-normal dimension, HALF = the F2C strip of one fine block (half
// the face along each tangential dimension).
template <class real, int D, int N, int NG, int ND, bool HALF>
__device__ __forceinline__ void ghost_strip(const GhostArgs<real> &a, const Geom &g, const Entry &e, real *dstb,
                                            const real *srcb, int lane, int part) {
    constexpr int ng = NG;
    constexpr int nd = ND;
    // tangential dimensions (lower first) and the strip's extents, fixed at
    // compile time so that no division by a runtime extent is left
    constexpr int T0 = ND == 0 ? 1 : 0, T1 = ND == 2 ? 1 : 2;
    constexpr int tdim[2] = {T0, T1};
    constexpr int E0 = ND == 0 ? NG : (HALF ? N / 2 : N);
    constexpr int E1 = ND == 1 ? NG : (HALF ? N / 2 : N);
    constexpr int E2 = D == 3 ? (ND == 2 ? NG : (HALF ? N / 2 : N)) : 1;
    constexpr int ext[3] = {E0, E1, E2};
    const int side = e.face & 1;
    int lo[3] = {0, 0, 0};
    lo[nd] = side ? N : -ng;
    int off[3] = {0, 0, 0};   // tangential position of the fine block (F2C/C2F)
    off[tdim[0]] = e.offset & 1;
    if (D == 3) off[tdim[1]] = (e.offset >> 1) & 1;
    if constexpr (HALF) {
        lo[T0] = off[T0] * (N / 2);
        if (D == 3) lo[T1] = off[T1] * (N / 2);
    }
    constexpr int ncells = E0 * E1 * E2;
    const int total = ncells * g.V;
    // four values per lane per round: all their loads are issued before
    // the first store, so a warp keeps several loads in flight
    for (int base = lane + 128 * part; base < total; base += 128 * a.parts) {
        real vals[4];
        int64_t dsti[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int idx = base + 32 * r;
            dsti[r] = -1;
            vals[r] = real(0);
            if (idx >= total) continue;
            int v = idx / ncells, c = idx - v * ncells;
            int x[3];
            x[0] = lo[0] + c % ext[0];
            c /= ext[0];
            x[1] = lo[1] + c % ext[1];
            x[2] = (D == 3) ? lo[2] + c / ext[1] : 0;
            real val;
            if (e.kind == KIND_SRL) {
                int y[3] = {x[0], x[1], x[2]};
                y[nd] += side ? -N : N;
                val = srcb[int64_t(v) * g.ncell + cell_index<real>(g, y[0], y[1], y[2])];
            } else if (e.kind == KIND_F2C) {
                int y[3] = {0, 0, 0};
                for (int d = 0; d < D; ++d) y[d] = 2 * x[d] - off[d] * N;
                y[nd] = side ? 2 * (x[nd] - N) : 2 * x[nd] + N;
                val = restrict_at<real, D>(srcb + int64_t(v) * g.ncell, g, y[0], y[1], y[2]);
            } else {  // physical boundary (Sec. 2.4)
                const int k = side ? x[nd] - N + 1 : -x[nd];          // layer 1..ng
                int y[3] = {x[0], x[1], x[2]};
                y[nd] = side ? N - k : k - 1;                          // mirror cell
                const real um = dstb[int64_t(v) * g.ncell + cell_index<real>(g, y[0], y[1], y[2])];
                const int inst = a.info[e.dst].inst;
                const int ty = a.bc_type[6 * inst + e.face];
                const real bv = a.bc_val[(6 * inst + e.face) * 8 + v];
                if (ty == 1) {
                    val = real(2) * bv - um;
                } else if (ty == 2) {
                    const real h = mul_rn(real(2 * k - 1), real(g.dx[3 * a.info[e.dst].gclass + nd]));
                    val = add_rn(um, mul_rn(h, bv));
                } else {
                    const int t = x[tdim[0]] + (D == 3 ? N * x[tdim[1]] : 0);
                    const int64_t nface = (D == 3) ? int64_t(N) * N : N;
                    val = real(2) * a.bcdata[(int64_t(e.aux) * g.V + v) * nface + t] - um;
                }
            }
            vals[r] = val;
            dsti[r] = int64_t(v) * g.ncell + cell_index<real>(g, x[0], x[1], x[2]);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
            if (dsti[r] >= 0) dstb[dsti[r]] = vals[r];
    }
}

template <class real, int D, int N, int NG>
__global__ void __launch_bounds__(256) k_ghost(GhostArgs<real> a, Geom g) {
    const int gw = int((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    const int warp = gw / a.parts, part = gw - warp * a.parts;
    if (warp >= a.n) return;
    const Entry e = a.list[warp];
    real *dstb = a.u + int64_t(e.dst) * g.bstride;
    const real *srcb = e.src >= 0 ? a.u + int64_t(e.src) * g.bstride : nullptr;
    if (e.kind == KIND_DIAG || e.kind == KIND_DIAG_F2C || e.kind == KIND_DIAG_C2F || e.kind == KIND_DIAG_BC) {
        // edge / corner region in direction (dx, dy, dz): ghost box of the
        // block, copied from a same-level neighbour's interior, restricted
        // from a finer neighbour (half the box along a 3D edge per neighbour),
        // or prolonged from a coarser one (offset bit d: parity of the
        // same-size box along d, i.e. which half of the coarse block)
        const int dir[3] = {e.face % 3 - 1, (e.face / 3) % 3 - 1, e.face / 9 - 1};
        int lo[3] = {0, 0, 0}, ext[3] = {1, 1, 1};
        for (int d = 0; d < D; ++d) {
            lo[d] = dir[d] < 0 ? -NG : (dir[d] > 0 ? N : 0);
            ext[d] = dir[d] != 0 ? NG : N;
            if (e.kind == KIND_DIAG_F2C && dir[d] == 0) {
                lo[d] = e.offset * (N / 2);
                ext[d] = N / 2;
            }
        }
        const int ncells = ext[0] * ext[1] * ext[2];
        for (int idx = lane + 32 * part; idx < ncells * g.V; idx += 32 * a.parts) {
            const int v = idx / ncells;
            int c = idx - v * ncells;
            int x[3];
            x[0] = lo[0] + c % ext[0];
            c /= ext[0];
            x[1] = lo[1] + c % ext[1];
            x[2] = lo[2] + c / ext[1];
            real val;
            if (e.kind == KIND_DIAG) {
                const int y0 = x[0] - dir[0] * N, y1 = x[1] - dir[1] * N, y2 = D == 3 ? x[2] - dir[2] * N : 0;
                val = srcb[int64_t(v) * g.ncell + cell_index<real>(g, y0, y1, y2)];
            } else if (e.kind == KIND_DIAG_BC) {
                // outside a non-periodic domain: the boundary formula of face
                // e.offset applied to the cell mirrored across it (a face
                // ghost for an edge cell, filled before; an edge cell for a
                // corner, filled by the launch before); per-cell boundary
                // data at the tangential position clamped to the face
                const int fb = e.offset, nb = fb >> 1, sb = fb & 1;
                const int k = sb ? x[nb] - N + 1 : -x[nb];
                int y[3] = {x[0], x[1], x[2]};
                y[nb] = sb ? N - k : k - 1;
                const real um = dstb[int64_t(v) * g.ncell + cell_index<real>(g, y[0], y[1], y[2])];
                const int inst = a.info[e.dst].inst;
                const int ty = a.bc_type[6 * inst + fb];
                const real bv = a.bc_val[(6 * inst + fb) * 8 + v];
                if (ty == 1) {
                    val = real(2) * bv - um;
                } else if (ty == 2) {
                    const real h = mul_rn(real(2 * k - 1), real(g.dx[3 * a.info[e.dst].gclass + nb]));
                    val = add_rn(um, mul_rn(h, bv));
                } else {
                    int t = 0, scale = 1;
                    for (int d = 0; d < D; ++d) {
                        if (d == nb) continue;
                        const int c = x[d] < 0 ? 0 : (x[d] >= N ? N - 1 : x[d]);
                        t += c * scale;
                        scale *= N;
                    }
                    const int64_t nface = (D == 3) ? int64_t(N) * N : N;
                    val = real(2) * a.bcdata[(int64_t(e.aux) * g.V + v) * nface + t] - um;
                }
            } else if (e.kind == KIND_DIAG_F2C) {
                // lower corner of the 2^D fine cells: across the region's
                // faces as for a face restriction, along an edge shifted by
                // the fine block's position
                int y[3] = {0, 0, 0};
                for (int d = 0; d < D; ++d)
                    y[d] = dir[d] < 0 ? 2 * x[d] + N : (dir[d] > 0 ? 2 * (x[d] - N) : 2 * x[d] - e.offset * N);
                val = restrict_at<real, D>(srcb + int64_t(v) * g.ncell, g, y[0], y[1], y[2]);
            } else {
                // the cell's position in the same-size box, then the coarse
                // cell and the sub-cell
                int y[3] = {0, 0, 0}, sb[3] = {0, 0, 0};
                for (int d = 0; d < D; ++d) {
                    const int r = x[d] - dir[d] * N;
                    y[d] = ((e.offset >> d) & 1) * (N / 2) + (r >> 1);
                    sb[d] = r & 1;
                }
                val = prolong_at<real, D>(srcb + int64_t(v) * g.ncell, g, y[0], y[1], y[2], sb[0], sb[1], sb[2]);
            }
            dstb[int64_t(v) * g.ncell + cell_index<real>(g, x[0], x[1], x[2])] = val;
        }
        return;
    }
    const int nd = e.face >> 1, side = e.face & 1;
    if constexpr (NG % 2 == 0) {
        if (e.kind == KIND_SRL) {
            if (nd == 0) srl_pairs<real, D, N, NG, 0>(dstb, srcb, side, lane, part, a.parts, g.V);
            else if (nd == 1 || D == 2) srl_pairs<real, D, N, NG, 1>(dstb, srcb, side, lane, part, a.parts, g.V);
            else srl_pairs<real, D, N, NG, (D == 3 ? 2 : 1)>(dstb, srcb, side, lane, part, a.parts, g.V);
            return;
        }
    }
    if (e.kind == KIND_C2F) {
        if (nd == 0) c2f_strip<real, D, N, NG, 0>(g, e, dstb, srcb, lane, part, a.parts);
        else if (nd == 1 || D == 2) c2f_strip<real, D, N, NG, 1>(g, e, dstb, srcb, lane, part, a.parts);
        else c2f_strip<real, D, N, NG, (D == 3 ? 2 : 1)>(g, e, dstb, srcb, lane, part, a.parts);
        return;
    }
    // the general path, with the strip shape fixed per normal and kind
    const bool half = e.kind == KIND_F2C;
    if (nd == 0) {
        if (half) ghost_strip<real, D, N, NG, 0, true>(a, g, e, dstb, srcb, lane, part);
        else ghost_strip<real, D, N, NG, 0, false>(a, g, e, dstb, srcb, lane, part);
    } else if (nd == 1 || D == 2) {
        if (half) ghost_strip<real, D, N, NG, 1, true>(a, g, e, dstb, srcb, lane, part);
        else ghost_strip<real, D, N, NG, 1, false>(a, g, e, dstb, srcb, lane, part);
    } else {
        if (half) ghost_strip<real, D, N, NG, (D == 3 ? 2 : 1), true>(a, g, e, dstb, srcb, lane, part);
        else ghost_strip<real, D, N, NG, (D == 3 ? 2 : 1), false>(a, g, e, dstb, srcb, lane, part);
    }
}

}  // namespace amrb
