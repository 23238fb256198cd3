// Row-packing plan of the exact-slice GEMM (host only, no CUDA): problems of fewer rows than a tile that read the
// same B operand share output tiles.
#pragma once
#include <algorithm>
#include <map>
#include <utility>
#include <vector>

namespace osv {

// One packed tile: the B operand key its problems share, and its members as (problem, first row in the tile).
struct OzPackTile {
    int key;
    std::vector<std::pair<int, int>> members;
};

// Problems i with 0 < rows[i] < tile_rows and key[i] >= 0 are grouped by key; within a group they fill tiles of
// tile_rows rows first fit in decreasing row count (ties in problem order).  A group is packed only if that
// needs fewer tiles than it has problems; a problem is in at most one tile, its rows contiguous from its offset.
inline std::vector<OzPackTile> oz_pack_rows(const std::vector<int> &rows, const std::vector<int> &key, int tile_rows) {
    std::map<int, std::vector<int>> groups;
    for (size_t i = 0; i < rows.size(); ++i)
        if (key[i] >= 0 && rows[i] > 0 && rows[i] < tile_rows) groups[key[i]].push_back((int)i);
    std::vector<OzPackTile> out;
    for (auto &kv : groups) {
        std::vector<int> &v = kv.second;
        if (v.size() < 2) continue;
        std::stable_sort(v.begin(), v.end(), [&](int x, int y) { return rows[x] > rows[y]; });
        std::vector<int> fill;                  // rows used per tile
        std::vector<int> bin(v.size()), at(v.size());
        for (size_t u = 0; u < v.size(); ++u) {
            size_t t = 0;
            while (t < fill.size() && fill[t] + rows[v[u]] > tile_rows) ++t;
            if (t == fill.size()) fill.push_back(0);
            bin[u] = (int)t;
            at[u] = fill[t];
            fill[t] += rows[v[u]];
        }
        if (fill.size() >= v.size()) continue;
        const size_t base = out.size();
        for (size_t t = 0; t < fill.size(); ++t) out.push_back(OzPackTile{kv.first, {}});
        for (size_t u = 0; u < v.size(); ++u) out[base + bin[u]].members.emplace_back(v[u], at[u]);
    }
    return out;
}

}  // namespace osv
