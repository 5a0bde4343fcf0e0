// Host-side forest of the block-AMR library: a linear quadtree/octree over a
// brick of trees (Sec. 2.2), stored as a sorted leaf array plus a hash of
// packed (level, coordinates) keys.  Mesh adaptation follows Sec. 2.2:
// refine, coarsen, then 2:1 balance across faces, edges and corners.
#pragma once

#include <cstdint>
#include <string>
#include <unordered_map>
#include <vector>

namespace amrb {

struct Leaf {
    int lev;
    int64_t g[3];  // block coordinates at level `lev` over the whole brick
};

// Packed key: level in the top 6 bits, 19 bits per coordinate.
inline uint64_t pack_key(int lev, int64_t x, int64_t y, int64_t z) {
    return (uint64_t(lev) << 57) | (uint64_t(z) << 38) | (uint64_t(y) << 19) | uint64_t(x);
}
inline uint64_t pack_key(const Leaf &l) { return pack_key(l.lev, l.g[0], l.g[1], l.g[2]); }

struct Geometry {
    int ndim = 3;
    int ntrees[3] = {1, 1, 1};
    int periodic[3] = {1, 1, 1};
    int max_level = 0;
    int64_t extent(int d, int lev) const { return int64_t(ntrees[d]) << lev; }
};

class Forest {
public:
    Geometry geo;
    std::vector<Leaf> leaves;              // block order
    std::unordered_map<uint64_t, int> index;  // key -> block
    uint64_t revision = 0;

    void init_uniform(const Geometry &g, int level);
    int find(int lev, int64_t x, int64_t y, int64_t z) const {
        auto it = index.find(pack_key(lev, x, y, z));
        return it == index.end() ? -1 : it->second;
    }
    // Applies flags (+1 refine, -1 coarsen, 0 keep); returns the new leaf list
    // without modifying this forest.
    std::vector<Leaf> adapted(const std::vector<int8_t> &flags) const;
    void assign(std::vector<Leaf> &&l);   // sorts, indexes, bumps revision

    // wraps coordinate x of dimension d at level lev; false if outside a
    // non-periodic domain
    bool wrap(int d, int lev, int64_t &x) const {
        int64_t E = geo.extent(d, lev);
        if (x >= 0 && x < E) return true;
        if (!geo.periodic[d]) return false;
        x = ((x % E) + E) % E;
        return true;
    }
};

void sort_leaves(const Geometry &g, std::vector<Leaf> &l);

}  // namespace amrb
