// Forest construction and adaptation (Sec. 2.2 of the paper: brick of trees,
// refine -> coarsen -> 2:1 balance with full connectivity; the n-th leaf in
// tree-then-Morton order is the n-th block).
#include "forest.hpp"

#include <algorithm>
#include <deque>
#include <unordered_set>

namespace amrb {

namespace {

// Spreads the low 21 bits of v so that consecutive bits land `stride` apart.
inline uint64_t spread(uint64_t v, int stride) {
    uint64_t r = 0;
    for (int b = 0; b < 21; ++b) r |= ((v >> b) & 1ull) << (stride * b);
    return r;
}

struct SortKey {
    int64_t tree;
    uint64_t morton;
};

constexpr int kDepth = 20;

SortKey sort_key(const Geometry &g, const Leaf &l) {
    int64_t t[3] = {0, 0, 0};
    uint64_t m = 0;
    for (int d = 0; d < g.ndim; ++d) {
        t[d] = l.g[d] >> l.lev;
        uint64_t loc = uint64_t(l.g[d] - (t[d] << l.lev)) << (kDepth - l.lev);
        m |= spread(loc, g.ndim) << d;
    }
    return {t[0] + int64_t(g.ntrees[0]) * (t[1] + int64_t(g.ntrees[1]) * t[2]), m};
}

}  // namespace

void sort_leaves(const Geometry &g, std::vector<Leaf> &l) {
    std::vector<std::pair<SortKey, int>> k(l.size());
    for (size_t i = 0; i < l.size(); ++i) k[i] = {sort_key(g, l[i]), int(i)};
    std::sort(k.begin(), k.end(), [](const auto &a, const auto &b) {
        if (a.first.tree != b.first.tree) return a.first.tree < b.first.tree;
        return a.first.morton < b.first.morton;
    });
    std::vector<Leaf> out(l.size());
    for (size_t i = 0; i < l.size(); ++i) out[i] = l[k[i].second];
    l.swap(out);
}

void Forest::init_uniform(const Geometry &g, int level) {
    geo = g;
    std::vector<Leaf> l;
    int64_t n[3] = {1, 1, 1};
    for (int d = 0; d < g.ndim; ++d) n[d] = g.extent(d, level);
    l.reserve(size_t(n[0] * n[1] * n[2]));
    for (int64_t z = 0; z < n[2]; ++z)
        for (int64_t y = 0; y < n[1]; ++y)
            for (int64_t x = 0; x < n[0]; ++x) l.push_back({level, {x, y, z}});
    revision = 0;
    assign(std::move(l));
}

void Forest::assign(std::vector<Leaf> &&l) {
    sort_leaves(geo, l);
    leaves = std::move(l);
    index.clear();
    index.reserve(leaves.size() * 2);
    for (size_t i = 0; i < leaves.size(); ++i) index[pack_key(leaves[i])] = int(i);
    ++revision;
}

std::vector<Leaf> Forest::adapted(const std::vector<int8_t> &flags) const {
    const int D = geo.ndim, nch = 1 << D;
    // 1. coarsening candidates: families whose 2^d children are all leaves
    //    flagged -1 (counted per parent)
    std::unordered_map<uint64_t, int> votes;
    for (size_t b = 0; b < leaves.size(); ++b) {
        const Leaf &l = leaves[b];
        if (flags[b] < 0 && l.lev > 0)
            ++votes[pack_key(l.lev - 1, l.g[0] >> 1, l.g[1] >> 1, D == 3 ? l.g[2] >> 1 : 0)];
    }
    // 2. refine flagged leaves below max_level, coarsen complete families
    std::unordered_set<uint64_t> set;   // current leaf keys
    std::vector<Leaf> work;
    auto add = [&](const Leaf &l) {
        set.insert(pack_key(l));
        work.push_back(l);
    };
    std::unordered_set<uint64_t> parents_done;
    for (size_t b = 0; b < leaves.size(); ++b) {
        const Leaf &l = leaves[b];
        if (flags[b] > 0 && l.lev < geo.max_level) {
            for (int c = 0; c < nch; ++c)
                add({l.lev + 1, {2 * l.g[0] + (c & 1), 2 * l.g[1] + ((c >> 1) & 1), D == 3 ? 2 * l.g[2] + ((c >> 2) & 1) : 0}});
            continue;
        }
        if (flags[b] < 0 && l.lev > 0) {
            Leaf p{l.lev - 1, {l.g[0] >> 1, l.g[1] >> 1, D == 3 ? l.g[2] >> 1 : 0}};
            uint64_t pk = pack_key(p);
            auto it = votes.find(pk);
            if (it != votes.end() && it->second == nch) {
                if (parents_done.insert(pk).second) add(p);
                continue;
            }
        }
        add(l);
    }
    // 3. balance (ripple): a leaf whose corner/edge/face neighbourhood holds a
    //    leaf two or more levels coarser forces that leaf to split.  Split
    //    leaves are removed from `set` lazily (work entries checked on pop).
    auto is_leaf = [&](const Leaf &l) { return set.count(pack_key(l)) != 0; };
    std::deque<Leaf> queue(work.begin(), work.end());
    while (!queue.empty()) {
        Leaf l = queue.front();
        queue.pop_front();
        if (!is_leaf(l) || l.lev < 2) continue;
        bool split_any = false;
        for (int dz = (D == 3 ? -1 : 0); dz <= (D == 3 ? 1 : 0); ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if (!dx && !dy && !dz) continue;
                    int64_t q[3] = {l.g[0] + dx, l.g[1] + dy, l.g[2] + dz};
                    bool inside = true;
                    for (int d = 0; d < D; ++d) inside = inside && wrap(d, l.lev, q[d]);
                    if (!inside) continue;
                    // ancestors two or more levels up that are leaves
                    for (int up = 2; up <= l.lev; ++up) {
                        Leaf a{l.lev - up, {q[0] >> up, q[1] >> up, D == 3 ? q[2] >> up : 0}};
                        if (!is_leaf(a)) continue;
                        set.erase(pack_key(a));
                        for (int c = 0; c < nch; ++c) {
                            Leaf ch{a.lev + 1, {2 * a.g[0] + (c & 1), 2 * a.g[1] + ((c >> 1) & 1),
                                                D == 3 ? 2 * a.g[2] + ((c >> 2) & 1) : 0}};
                            set.insert(pack_key(ch));
                            work.push_back(ch);
                            queue.push_back(ch);
                        }
                        split_any = true;
                        break;
                    }
                }
        if (split_any) queue.push_back(l);
    }
    std::vector<Leaf> out;
    out.reserve(set.size());
    std::unordered_set<uint64_t> emitted;
    for (const Leaf &l : work)
        if (set.count(pack_key(l)) && emitted.insert(pack_key(l)).second) out.push_back(l);
    sort_leaves(geo, out);
    return out;
}

}  // namespace amrb
