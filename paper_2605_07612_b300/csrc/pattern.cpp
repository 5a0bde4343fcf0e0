// Face-neighbour walk that classifies every block face as SRL / F2C / C2F /
// BC (Sec. 2.6).  For block A at level l and face f the same-size box across
// the face is looked up: a leaf -> SRL; its parent a leaf -> C2F (A is fine);
// otherwise the 2^(d-1) children facing A must be leaves -> F2C (A is coarse,
// one entry per fine source).  Outside a non-periodic domain -> BC.
#include "pattern.hpp"

#include <algorithm>

namespace amrb {

bool build_pattern(const std::vector<const Forest *> &inst, const std::vector<int64_t> &offset, Pattern &P,
                   std::string &err, bool diagonal) {
    P = Pattern();
    int nb = 0;
    for (const Forest *F : inst) nb += int(F->leaves.size());
    P.entries.reserve(size_t(nb) * 6);
    for (size_t ii = 0; ii < inst.size(); ++ii) {
    const Forest &F = *inst[ii];
    const Geometry &G = F.geo;
    const int D = G.ndim;
    const int o0 = int(offset[ii]);
    const int nbi = int(F.leaves.size());
    for (int bl = 0; bl < nbi; ++bl) {
        const int b = o0 + bl;
        const Leaf &A = F.leaves[bl];
        for (int f = 0; f < 2 * D; ++f) {
            const int n = f >> 1, side = f & 1;
            int t0 = -1, t1 = -1;
            for (int d = 0, c = 0; d < D; ++d)
                if (d != n) (c++ == 0 ? t0 : t1) = d;
            int64_t q[3] = {A.g[0], A.g[1], A.g[2]};
            q[n] += side ? 1 : -1;
            if (!F.wrap(n, A.lev, q[n])) {
                P.entries.push_back({KIND_BC, f, b, -1, 0, 0});
                continue;
            }
            int s = F.find(A.lev, q[0], q[1], q[2]);
            if (s >= 0) {
                P.entries.push_back({KIND_SRL, f, b, o0 + s, 0, 0});
                continue;
            }
            if (A.lev > 0) {
                int c = F.find(A.lev - 1, q[0] >> 1, q[1] >> 1, D == 3 ? q[2] >> 1 : 0);
                if (c >= 0) {
                    int off = int(A.g[t0] & 1) | (D == 3 ? int(A.g[t1] & 1) << 1 : 0);
                    P.entries.push_back({KIND_C2F, f, b, o0 + c, off, 0});
                    continue;
                }
            }
            // finer neighbours: children of q adjacent to A
            for (int o = 0; o < (1 << (D - 1)); ++o) {
                int64_t ch[3] = {0, 0, 0};
                ch[n] = 2 * q[n] + (side ? 0 : 1);
                ch[t0] = 2 * q[t0] + (o & 1);
                if (D == 3) ch[t1] = 2 * q[t1] + ((o >> 1) & 1);
                int fs = (A.lev < G.max_level) ? F.find(A.lev + 1, ch[0], ch[1], ch[2]) : -1;
                if (fs < 0) {
                    err = "ghost pattern: block " + std::to_string(b) + " face " + std::to_string(f) +
                          " has no leaf neighbour within one level (2:1 balance broken)";
                    return false;
                }
                P.entries.push_back({KIND_F2C, f, b, o0 + fs, o, 0});
            }
        }
        // edge and corner regions: held by a same-level leaf, part of a
        // coarser leaf, or covered by the finer children that touch A
        if (diagonal)
            for (int dz = (D == 3 ? -1 : 0); dz <= (D == 3 ? 1 : 0); ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int dir[3] = {dx, dy, dz};
                        if ((dx != 0) + (dy != 0) + (dz != 0) < 2) continue;
                        const int code = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
                        // outside a non-periodic domain: the boundary formula
                        // of the face across the lowest such dimension
                        int dout = -1;
                        for (int d = 0; d < D && dout < 0; ++d) {
                            int64_t qd = A.g[d] + dir[d];
                            if (dir[d] != 0 && !F.wrap(d, A.lev, qd)) dout = d;
                        }
                        if (dout >= 0) {
                            P.entries.push_back({KIND_DIAG_BC, code, b, -1, 2 * dout + (dir[dout] > 0 ? 1 : 0), -1});
                            continue;
                        }
                        int64_t q[3] = {A.g[0], A.g[1], A.g[2]};
                        for (int d = 0; d < D; ++d) {
                            q[d] += dir[d];
                            F.wrap(d, A.lev, q[d]);
                        }
                        const int s = F.find(A.lev, q[0], q[1], q[2]);
                        if (s >= 0) {
                            P.entries.push_back({KIND_DIAG, code, b, o0 + s, 0, 0});
                            continue;
                        }
                        if (A.lev > 0) {
                            const int c = F.find(A.lev - 1, q[0] >> 1, q[1] >> 1, D == 3 ? q[2] >> 1 : 0);
                            if (c >= 0) {
                                int par = 0;
                                for (int d = 0; d < D; ++d) par |= int(q[d] & 1) << d;
                                P.entries.push_back({KIND_DIAG_C2F, code, b, o0 + c, par, 0});
                                continue;
                            }
                        }
                        // finer: the children of q touching A (two along a 3D edge)
                        int ed = -1;
                        for (int d = 0; d < D; ++d)
                            if (dir[d] == 0) ed = d;
                        for (int o = 0; o < (ed >= 0 ? 2 : 1); ++o) {
                            int64_t ch[3] = {0, 0, 0};
                            for (int d = 0; d < D; ++d)
                                ch[d] = dir[d] != 0 ? 2 * q[d] + (dir[d] < 0 ? 1 : 0) : 2 * q[d] + o;
                            const int fs = A.lev < G.max_level ? F.find(A.lev + 1, ch[0], ch[1], ch[2]) : -1;
                            if (fs >= 0) P.entries.push_back({KIND_DIAG_F2C, code, b, o0 + fs, o, 0});
                        }
                    }
    }
    }
    std::sort(P.entries.begin(), P.entries.end(), [](const Entry &x, const Entry &y) {
        if (x.kind != y.kind) return x.kind < y.kind;
        if (x.face != y.face) return x.face < y.face;
        if (x.dst != y.dst) return x.dst < y.dst;
        return x.offset < y.offset;
    });
    int32_t ibf = 0;
    std::vector<int32_t> bc_index(size_t(nb) * 6, -1);   // (block, face) -> boundary-face index
    for (Entry &e : P.entries)
        if (e.kind == KIND_BC) {
            bc_index[size_t(e.dst) * 6 + size_t(e.face)] = ibf;
            e.aux = ibf++;
        }
    P.n_bc = ibf;
    for (Entry &e : P.entries)
        if (e.kind == KIND_DIAG_BC) e.aux = bc_index[size_t(e.dst) * 6 + size_t(e.offset)];

    // execution lists and refinement-face flux slots
    P.info.assign(size_t(nb), BlockInfo{});
    for (size_t ii = 0; ii < inst.size(); ++ii)
        for (size_t bl = 0; bl < inst[ii]->leaves.size(); ++bl) {
            const size_t b = size_t(offset[ii]) + bl;
            P.info[b].level = inst[ii]->leaves[bl].lev;
            P.info[b].inst = int32_t(ii);
            P.info[b].gclass = int32_t(ii) * kMaxLevels + P.info[b].level;
        }
    for (int b = 0; b < nb; ++b) {
        P.info[b].fixmask = 0;
        for (int f = 0; f < 6; ++f) P.info[b].bslot[f] = P.info[b].nbr[f] = -1;
    }
    // blocks whose face ghosts a prolongation reads (their same-level face
    // ghosts are filled in gather mode too)
    // (and blocks whose outside edge and corner cells mirror their face ghosts)
    std::vector<char> c2f_src(size_t(nb), 0);
    for (const Entry &e : P.entries) {
        if (e.kind == KIND_C2F || e.kind == KIND_DIAG_C2F) c2f_src[size_t(e.src)] = 1;
        if (e.kind == KIND_DIAG_BC) c2f_src[size_t(e.dst)] = 1;
    }
    std::vector<Entry> corners;
    for (const Entry &e : P.entries) {
        if (e.kind == KIND_DIAG_BC) {
            const bool corner = e.face != 13 && (e.face % 3) != 1 && ((e.face / 3) % 3) != 1 && (e.face / 9) != 1;
            (corner ? corners : P.round3).push_back(e);
            continue;
        }
        const bool r2 = e.kind == KIND_C2F || e.kind == KIND_DIAG_C2F;
        (r2 ? P.round2 : P.round1).push_back(e);
        if (e.kind == KIND_SRL) P.info[e.dst].nbr[e.face] = e.src;
        if (!r2 && (e.kind != KIND_SRL || c2f_src[size_t(e.dst)])) P.round1_gather.push_back(e);
        if (e.kind == KIND_F2C || e.kind == KIND_C2F) {
            int32_t &slot = P.info[e.dst].bslot[e.face];
            if (slot < 0) slot = P.n_slots++;
            if (e.kind == KIND_F2C) P.info[e.dst].fixmask |= 1 << e.face;
        }
    }
    // execution order: by receiving block, so that the strips on both sides
    // of a face (which share the 32-byte sectors of the rows they touch)
    // run close together in time and meet in L2
    for (std::vector<Entry> *l : {&P.round1, &P.round2, &P.round1_gather})
        std::stable_sort(l->begin(), l->end(), [](const Entry &x, const Entry &y) { return x.dst < y.dst; });
    P.n_round3_edges = int32_t(P.round3.size());
    P.round3.insert(P.round3.end(), corners.begin(), corners.end());
    // fix-up faces: every (coarse block, face) with F2C sources
    for (const Entry &e : P.entries) {
        if (e.kind != KIND_F2C) continue;
        if (P.fix.empty() || P.fix.back().block != e.dst || P.fix.back().face != e.face)
            P.fix.push_back({e.dst, e.face, P.info[e.dst].bslot[e.face], {-1, -1, -1, -1}});
        P.fix.back().fslot[e.offset] = P.info[e.src].bslot[e.face ^ 1];
    }
    std::sort(P.fix.begin(), P.fix.end(), [](const FixFace &x, const FixFace &y) {
        return x.block != y.block ? x.block < y.block : x.face < y.face;
    });
    for (size_t i = 0; i < P.fix.size(); ++i)
        if (i == 0 || P.fix[i].block != P.fix[i - 1].block) P.fix_start.push_back(int32_t(i));
    P.fix_start.push_back(int32_t(P.fix.size()));
    return true;
}

}  // namespace amrb
