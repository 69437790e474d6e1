// Host-side tiling of the last two depths for k_tail_slots (stream.cuh), and the tile limits the
// kernel's shared-memory stages are sized for.
#pragma once

#include <cstdint>
#include <vector>

#include "layout.hpp"

namespace cfrgb {

constexpr int kSTP = 128;                  // parents per tile, at most (one per consumer thread)
constexpr int kSTC = 384;                  // children per tile, at most
constexpr int kSTSP = 640;                 // parents' slots per tile, at most
constexpr int kSTSC = 1536;                // children's slots (= their terminal children) per tile, at most
constexpr int kSTTP = 384;                 // parents' terminal children per tile, at most

// Tiles over the parents [jb, je) of one depth whose decision children (the next depth) have terminal
// children only: consecutive parents while their slots continue one contiguous range, their decision
// children's slots another, and every staged range fits its array (4 elements of each kept free for
// the 16-byte widening of the copies).  The children's terminals then sit at the offsets of their
// slots, since consecutive nodes of the last depth have consecutive terminal ranges.  Appends 12
// words per tile to *meta: {j0, j1, cs, ce}, {pts, pte, cts, cte}, {qps, qpe, qcs, qce} (parents,
// decision children, the two terminal ranges, the two slot ranges).  False if some parent's own
// children do not have contiguous slots, or if the tiles would hold fewer than kSTP / 2 parents on
// average (too fragmented to stream well).
inline bool cut_slot_tail_tiles(const Layout &Lo, int32_t jb, int32_t je, std::vector<int32_t> *meta) {
    auto qb = [&](int32_t j) { return (int32_t)(Lo.qp[(size_t)j] & 0x1fffffffu); };
    auto na = [&](int32_t j) {
        return (Lo.dfirst[(size_t)j + 1] - Lo.dfirst[(size_t)j]) + (Lo.tfirst[(size_t)j + 1] - Lo.tfirst[(size_t)j]);
    };
    if (je <= jb) return false;
    std::vector<int32_t> tb{jb};
    int32_t n = 0, nc = 0, npt = 0, nct = 0, nsp = 0;
    int32_t pend = -1, cend = -1;            // slot after the tile's last parent / last child so far
    for (int32_t j = jb; j < je; ++j) {
        const int32_t d0 = Lo.dfirst[(size_t)j], d1 = Lo.dfirst[(size_t)j + 1];
        for (int32_t c = d0; c < d1; ++c) {
            if (Lo.dfirst[(size_t)c + 1] != Lo.dfirst[(size_t)c]) return false;   // a child with a decision child
            if (c + 1 < d1 && qb(c + 1) != qb(c) + na(c)) return false;
        }
        const int32_t ndj = d1 - d0, ptj = Lo.tfirst[(size_t)j + 1] - Lo.tfirst[(size_t)j];
        const int32_t ctj = Lo.tfirst[(size_t)d1] - Lo.tfirst[(size_t)d0], naj = na(j);
        const bool cont = qb(j) == pend && (ndj == 0 || cend < 0 || qb(d0) == cend);
        if (n > 0 && (!cont || n + 1 > kSTP || nc + ndj > kSTC - 4 || npt + ptj > kSTTP - 4 ||
                      nct + ctj > kSTSC - 4 || nsp + naj > kSTSP - 4)) {
            tb.push_back(j);
            n = nc = npt = nct = nsp = 0;
            cend = -1;
        }
        if (ndj > kSTC - 4 || ptj > kSTTP - 4 || ctj > kSTSC - 4 || naj > kSTSP - 4) return false;
        ++n; nc += ndj; npt += ptj; nct += ctj; nsp += naj;
        pend = qb(j) + naj;
        if (ndj > 0) cend = qb(d1 - 1) + na(d1 - 1);
    }
    tb.push_back(je);
    const int32_t nt = (int32_t)tb.size() - 1;
    if ((int64_t)nt * (kSTP / 2) > (int64_t)(je - jb)) return false;
    meta->clear();
    meta->reserve((size_t)12 * nt);
    for (int32_t i = 0; i < nt; ++i) {
        const int32_t j0 = tb[(size_t)i], j1 = tb[(size_t)i + 1];
        const int32_t cs = Lo.dfirst[(size_t)j0], ce = Lo.dfirst[(size_t)j1];
        const int32_t qcs = ce > cs ? qb(cs) : 0, qce = ce > cs ? qb(ce - 1) + na(ce - 1) : 0;
        const int32_t v[12] = {j0, j1, cs, ce, Lo.tfirst[(size_t)j0], Lo.tfirst[(size_t)j1], Lo.tfirst[(size_t)cs],
                               Lo.tfirst[(size_t)ce], qb(j0), qb(j1 - 1) + na(j1 - 1), qcs, qce};
        meta->insert(meta->end(), v, v + 12);
    }
    return true;
}

}  // namespace cfrgb
