// Ghost-cell pattern of Sec. 2.6, built on the host from the forest's face
// connectivity and executed on the GPU.  Besides the canonical entry list
// this produces the tables the kernels need: refinement-face flux slots for
// flux fixing (Sec. 2.7) and the per-coarse-block fix-up lists.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "forest.hpp"

namespace amrb {

constexpr int kMaxLevels = 13;   // levels 0..12 per instance

enum : int32_t { KIND_SRL = 0, KIND_F2C = 1, KIND_BC = 2, KIND_C2F = 3, KIND_DIAG = 4, KIND_DIAG_F2C = 5, KIND_DIAG_C2F = 6,
                 KIND_DIAG_BC = 7 };

struct Entry {
    int32_t kind, face, dst, src, offset, aux;
};

// One coarse block face that touches 2^(d-1) finer blocks.
struct FixFace {
    int32_t block, face;
    int32_t cslot;      // flux slot of the coarse side
    int32_t fslot[4];   // flux slots of the fine sides, by offset
};

// Per-block data read by the stage kernel.
struct BlockInfo {
    int32_t level;
    int32_t fixmask;    // bit f: face f is the coarse side of a refinement face
    int32_t bslot[6];   // flux slot of face f, -1 if not a refinement face
    int32_t nbr[6];     // same-level neighbour across face f, -1 if none
    int32_t inst;       // mesh instance of the block
    int32_t gclass;     // inst * kMaxLevels + level: row of the cell-size tables
};

struct Pattern {
    std::vector<Entry> entries;   // canonical order (kind, face, dst, offset)
    std::vector<Entry> round1;    // SRL, F2C, BC (and DIAG)
    std::vector<Entry> round2;    // C2F
    // round 1 when the stage kernel gathers same-level halos itself: every
    // non-SRL entry, plus the SRL entries of blocks that are the coarse
    // source of a C2F entry (their ghosts feed the prolongation)
    std::vector<Entry> round1_gather;
    // edge and corner regions outside a non-periodic domain (KIND_DIAG_BC),
    // after rounds 1 and 2: the edges first (their mirror cells are face
    // ghosts), then the 3D corners (their mirror cells are edge cells)
    std::vector<Entry> round3;
    int32_t n_round3_edges = 0;
    std::vector<BlockInfo> info;  // per block
    std::vector<FixFace> fix;     // sorted by (block, face)
    std::vector<int32_t> fix_start;  // per fix-up block: first index into fix (+ sentinel)
    int32_t n_slots = 0;
    int32_t n_bc = 0;
};

// Builds the pattern of one or more independent mesh instances whose blocks
// are numbered consecutively (instance i owns blocks offset[i] ..
// offset[i] + n_i - 1).  Returns false (with a message) if some face has no
// valid neighbour configuration (2:1 balance broken).
// diagonal: also emit entries for the edge / corner ghost regions (face =
// direction code (dx+1) + 3 (dy+1) + 9 (dz+1)) inside the domain: KIND_DIAG
// (a same-level leaf holds the region: copy, round 1), KIND_DIAG_F2C (finer
// leaves: restriction, round 1, one entry per fine leaf, offset = its
// position along a 3D edge), KIND_DIAG_C2F (a coarser leaf: prolongation,
// round 2, offset bit d = parity of the same-size box along dimension d);
// a region reaching outside a non-periodic domain gets KIND_DIAG_BC (the
// boundary formula of face `offset`, the face across the region's lowest
// dimension that leaves the domain, applied to the mirrored cell; aux = that
// face's boundary-face index; round 3).
bool build_pattern(const std::vector<const Forest *> &inst, const std::vector<int64_t> &offset, Pattern &out,
                   std::string &err, bool diagonal = false);

}  // namespace amrb
