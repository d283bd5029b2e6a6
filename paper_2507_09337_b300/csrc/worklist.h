// worklist.h -- host-side work lists of the persistent hydro kernel.
#pragma once

#include <algorithm>
#include <cmath>
#include <vector>

#include "persistent.cuh"

namespace orcha {

// One mesh of a launch: its slot, block grid, block size and column tiles per
// block plane.
struct ColumnSource {
    int slot;
    int nb[3], bs[3];
    int ntile;
};

// Whether a mesh's block columns fit the 15-bit plane fields of Item::zr.
inline bool column_items_fit(const MeshDev& d) { return (long long)d.nb[2] * d.bs[2] < (1 << 15); }

// Work list of a 3D launch: z ranges of block columns. The planes of every
// column tile (each mesh, column and tile in turn) form one stream of W
// planes, cut at the multiples of W / G (G resident CTAs: one segment per
// CTA) and at every column end; a piece shorter than 2 planes joins its
// neighbour. The pieces are queued longest first, so every resident CTA
// takes about one segment, a column tile pays its two-plane z halo about
// once per CTA rather than once per block, and the last items to start are
// the short ones. Same bits as full-block items. (Modelled with the halo at
// 0.55 plane: 128^3 Sedov 39.2 plane-times per CTA against 43.3 for
// full-block items with the last partial wave split in halves; ideal 38.)
inline std::vector<Item> column_items(const std::vector<ColumnSource>& src, long long G) {
    struct Col {
        int slot, blk, tile, depth;
    };
    std::vector<Col> cols;
    long long W = 0;
    for (const ColumnSource& m : src) {
        const int depth = m.nb[2] * m.bs[2];
        for (int by = 0; by < m.nb[1]; ++by)
            for (int bx = 0; bx < m.nb[0]; ++bx)
                for (int t = 0; t < m.ntile; ++t) {
                    cols.push_back({m.slot, bx + m.nb[0] * by, t, depth});
                    W += depth;
                }
    }
    const double seg = (double)W / (double)std::max(1LL, G);
    const int kMinPiece = 2;
    std::vector<Item> items;
    long long base = 0;                        // stream position of the column's first plane
    for (const Col& c : cols) {
        std::vector<int> cuts{0};
        for (long long k = (long long)std::floor((double)base / seg) + 1;; ++k) {
            const long long pos = std::llround((double)k * seg) - base;
            if (pos >= c.depth) break;
            if (pos > cuts.back()) cuts.push_back((int)pos);
        }
        cuts.push_back(c.depth);
        std::vector<int> kept{0};
        for (size_t i = 1; i < cuts.size(); ++i) {
            const bool last = i + 1 == cuts.size();
            if (!last && cuts[i] - kept.back() < kMinPiece) continue;
            if (last && cuts[i] - kept.back() < kMinPiece && kept.size() > 1) kept.pop_back();
            kept.push_back(cuts[i]);
        }
        for (size_t i = 0; i + 1 < kept.size(); ++i) items.push_back({c.slot, c.blk, c.tile, kept[i] | (kept[i + 1] << 16)});
        base += c.depth;
    }
    std::stable_sort(items.begin(), items.end(), [](const Item& x, const Item& y) {
        return (x.zr >> 16) - (x.zr & 0xFFFF) > (y.zr >> 16) - (y.zr & 0xFFFF);
    });
    return items;
}

}  // namespace orcha
