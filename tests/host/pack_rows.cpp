// Host check of the exact-slice GEMM's row-packing plan (oz_pack.h): tiles never overflow, members share their
// tile's key, each packed problem sits in one tile on its own contiguous rows, a group is packed only when that
// saves tiles, and problems that are too tall, keyless or empty are never packed.  Known small plans are pinned.
#include <cstdio>
#include <random>
#include <set>

#include "../../paper_2106_06149_gb300/csrc/oz_pack.h"

static int fails = 0;
#define CHECK(c) do { if (!(c)) { ++fails; if (fails < 20) printf("FAIL line %d: %s\n", __LINE__, #c); } } while (0)

static void check_plan(const std::vector<int> &rows, const std::vector<int> &key, int T) {
    const auto plan = osv::oz_pack_rows(rows, key, T);
    std::vector<int> seen(rows.size(), 0);
    std::map<int, int> tiles_of_key, packed_of_key, eligible_of_key;
    for (size_t i = 0; i < rows.size(); ++i)
        if (key[i] >= 0 && rows[i] > 0 && rows[i] < T) ++eligible_of_key[key[i]];
    for (const auto &pt : plan) {
        ++tiles_of_key[pt.key];
        std::vector<char> used(T, 0);
        CHECK(!pt.members.empty());
        for (const auto &m : pt.members) {
            const int p = m.first, off = m.second;
            CHECK(p >= 0 && p < (int)rows.size());
            CHECK(key[p] == pt.key);
            CHECK(rows[p] > 0 && rows[p] < T);
            CHECK(off >= 0 && off + rows[p] <= T);
            for (int r = off; r < off + rows[p] && r < T; ++r) {
                CHECK(!used[r]);
                used[r] = 1;
            }
            ++seen[p];
            ++packed_of_key[pt.key];
        }
    }
    for (size_t i = 0; i < rows.size(); ++i) CHECK(seen[i] <= 1);
    for (const auto &kv : tiles_of_key) {
        CHECK(packed_of_key[kv.first] == eligible_of_key[kv.first]);   // a group is packed whole or not at all
        CHECK(kv.second < packed_of_key[kv.first]);                    // and only when that saves tiles
    }
    for (const auto &kv : eligible_of_key)   // an unpacked group: first fit would not have saved a tile
        if (!tiles_of_key.count(kv.first)) {
            std::vector<int> v;
            for (size_t i = 0; i < rows.size(); ++i)
                if (key[i] == kv.first && rows[i] > 0 && rows[i] < T) v.push_back(rows[i]);
            std::sort(v.rbegin(), v.rend());
            std::vector<int> fill;
            for (int x : v) {
                size_t t = 0;
                while (t < fill.size() && fill[t] + x > T) ++t;
                if (t == fill.size()) fill.push_back(0);
                fill[t] += x;
            }
            CHECK(fill.size() >= v.size());
        }
}

int main() {
    // pinned plans
    {
        const auto p = osv::oz_pack_rows({40, 40, 40}, {7, 7, 7}, 128);   // three 40-row problems: one tile
        CHECK(p.size() == 1 && p[0].key == 7 && p[0].members.size() == 3);
        if (p.size() == 1 && p[0].members.size() == 3) {
            CHECK(p[0].members[0] == std::make_pair(0, 0));
            CHECK(p[0].members[1] == std::make_pair(1, 40));
            CHECK(p[0].members[2] == std::make_pair(2, 80));
        }
    }
    CHECK(osv::oz_pack_rows({100, 100}, {1, 1}, 128).empty());           // no tile saved
    CHECK(osv::oz_pack_rows({40, 40}, {1, 2}, 128).empty());             // different B operands
    CHECK(osv::oz_pack_rows({40, 40}, {-1, -1}, 128).empty());           // no key
    CHECK(osv::oz_pack_rows({128, 40, 40}, {3, 3, 3}, 128).size() == 1); // the full-height problem stays out
    {
        const auto p = osv::oz_pack_rows({90, 40, 30, 60, 20}, {5, 5, 5, 5, 5}, 128);   // 90+30, 60+40+20
        CHECK(p.size() == 2);
        if (p.size() == 2) {
            CHECK(p[0].members.size() == 2 && p[0].members[0].first == 0 && p[0].members[1].first == 2);
            CHECK(p[1].members.size() == 3 && p[1].members[0].first == 3 && p[1].members[1].first == 1 &&
                  p[1].members[2].first == 4);
        }
    }
    // random plans
    std::mt19937 g(11);
    for (int it = 0; it < 3000; ++it) {
        const int n = 1 + g() % 60, nkeys = 1 + g() % 6, T = (g() % 2) ? 128 : 64;
        std::vector<int> rows(n), key(n);
        for (int i = 0; i < n; ++i) {
            const int kind = g() % 10;
            rows[i] = kind == 0 ? 0 : (kind == 1 ? T + (int)(g() % 50) : 1 + (int)(g() % (T - 1)));
            key[i] = (g() % 8 == 0) ? -1 : (int)(g() % nkeys);
        }
        check_plan(rows, key, T);
    }
    printf("fails=%d\n", fails);
    return fails == 0 ? 0 : 1;
}
