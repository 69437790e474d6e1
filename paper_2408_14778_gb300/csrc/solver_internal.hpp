// Internal entry points of the single-game solver used by the batched solver (not part of the C ABI).
#pragma once

#include "cfr_gb300.h"

namespace cfrgb {

// cfr_load_tree; with forest, g may hold several independent games (one root each, all at depth 0).
cfr_status load_tree_impl(const cfr_game_desc *g, const cfr_config *c, bool forest, cfr_solver **out);

// NashConv of each root's game of a forest (per_root[k] for the k-th decision node of depth 0).
cfr_status root_nash_conv(cfr_solver *s, double *per_root, int32_t n);

}  // namespace cfrgb
