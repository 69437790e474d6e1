// Host-side validation of a game description and the level-ordered layout the kernels read.
//
// Layout (Section 3.1 replaces the tree by the adjacency matrix G, the level graphs L^(l) and the
// masks M^(Q+,V), M^(H+,Q+), M^(V,I+); here they are implicit):
//   * Decision nodes and terminals get separate internal ids, each in breadth-first order (depth
//     by depth, parents in order, children in action order).  Hence the decision children of a
//     decision node are a contiguous id range and so are its terminal children:
//       decision children of j:  dfirst[j] .. dfirst[j+1]
//       terminal children of j:  tfirst[j] .. tfirst[j+1]
//     and bit a of kmask[j] says whether action a leads to a terminal (interleaving them back into
//     action order).  A node with more than 32 actions instead stores in kmask[j] the offset of
//     its ceil(|A|/32) mask words in the side table wbits.  dlevel[l] .. dlevel[l+1] are the
//     decision nodes of depth l.
//   * Player infosets get internal ids [0, Hp) in order of first appearance in that order, so they
//     are sorted by their shallowest depth; chance infosets follow.  qbase[h] .. qbase[h+1] are
//     infoset h's (infoset, action) slots
//     (the mask M^(H+,Q+)), and the slot of child a of j is qbase[dinfo[j]] + a (M^(Q+,V)).
//   * pseq[h] is the slot of the acting player's last own (infoset, action) above h (-1 if none);
//     under perfect recall it is the same for every node of h and gives the own reach recursion
//     pi_i(h) = pi_i(hp) * sigma(pseq[h]) (Eq. 4 restricted to one player), hp = pseq_h[h].
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "cfr_gb300.h"

namespace cfrgb {

struct Layout {
    int64_t N = 0, Nd = 0, Nt = 0, Q = 0;
    int32_t H = 0;
    int32_t L = 0;               // number of depths holding decision nodes
    int32_t max_depth = 0;
    int32_t max_actions = 0;
    bool single_level = true;    // every infoset's nodes at one depth
    std::vector<int32_t> dfirst, tfirst;   // [Nd + 1]
    std::vector<int32_t> dinfo;            // [Nd] internal infoset
    std::vector<uint32_t> kmask;           // [Nd] terminal-child mask, or offset into wbits
    std::vector<uint32_t> wbits;           // mask words of nodes with > 32 actions
    std::vector<uint32_t> qp;              // [Nd] qbase[dinfo[j]] | (|A| > 32) << 29 | player << 30
    std::vector<int32_t> dlevel;           // [L + 1]
    std::vector<int32_t> hlevel;           // [L + 1]: player infosets whose shallowest depth is l
    int32_t Hp = 0;                        // player infosets: internal ids [0, Hp); chance ones [Hp, H)
    std::vector<int32_t> wide;             // decision nodes with more than 32 actions, by depth
    std::vector<int32_t> wlevel;           // [L + 1]: wide[wlevel[l] .. wlevel[l+1]) are at depth l
    std::vector<double> util;              // [Nt] u(t, 1)
    std::vector<int32_t> qbase;            // [H + 1] internal
    std::vector<int8_t> iplayer;           // [H]
    std::vector<int32_t> pseq;             // [H] internal slot or -1
    std::vector<int32_t> pseq_h;           // [H] internal infoset holding pseq, or -1
    std::vector<double> sigma0;            // [Q] chance slots, internal order
    std::vector<int32_t> q_int2user;       // [Q]
    std::vector<int32_t> h_int2user;       // [H]
    std::vector<int32_t> dnode_user;       // [Nd] internal decision id -> caller node id
    std::vector<int32_t> tnode_user;       // [Nt]
    // Only with infoset_lists: the decision nodes of infoset h are hnode[hnode_start[h] ..
    // hnode_start[h+1]), in depth-first order (the order a recursive walk reaches them).
    std::vector<int32_t> hnode_start;      // [H + 1]
    std::vector<int32_t> hnode;            // [Nd]
};

// Validates g; if layout != nullptr also builds the layout (with the per-infoset node lists when
// infoset_lists).  forest: g may have several roots (independent games side by side, all at depth 0,
// taken in node-id order; each depth then lists its nodes game by game).  Returns CFR_OK or an error
// code and writes the reason into *err.
cfr_status build_layout(const cfr_game_desc *g, Layout *layout, std::string *err, bool infoset_lists = false,
                        bool forest = false);

// The two builders build_layout chooses between (by size): one thread, and several host threads from
// kParallelLayoutNodes nodes on.  Same results, same errors.
constexpr int64_t kParallelLayoutNodes = 1 << 20;
cfr_status build_layout_serial(const cfr_game_desc *g, Layout *layout, std::string *err, bool infoset_lists, bool forest);
cfr_status build_layout_parallel(const cfr_game_desc *g, Layout *layout, std::string *err, bool infoset_lists,
                                 bool forest);

}  // namespace cfrgb
