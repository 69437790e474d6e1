/*
 * cfr_gb300.h - C ABI of a GB300-native (sm_103a) counterfactual regret minimization solver.
 *
 * One solver holds one finite extensive-form game <T, H, f_h, A, f_a, I, f_i, sigma_0, u>
 * (Definition in Section 2.1) on the GPU and runs full-tree CFR iterations (Section 2.3; the
 * matrix form of Section 3, Eq. 11-15) as hand-written CUDA kernels over a level-ordered layout of
 * the tree.  Two-player zero-sum games only (u_2 = -u_1).
 *
 * Conventions shared by every entry point
 *   - Node ids, infoset ids and action indices are the caller's.  "Q arrays" are infoset-major
 *     over ALL infosets (chance infosets included), actions 0..|A(h)|-1 in order; their length is
 *     num_q = sum_h |A(h)|.  Regret and strategy-sum entries of chance infosets are 0; strategy
 *     entries of chance infosets hold sigma_0.
 *   - Host pointers only.  The library copies every input before returning; outputs go to
 *     caller-owned host buffers whose length is passed and checked (too short -> CFR_ERR_INVALID).
 *   - The library owns its device memory.  It allocates through cfr_config.dev_alloc/dev_free when
 *     given (e.g. a framework's caching allocator), otherwise through cudaMalloc/cudaFree.
 *   - Work is queued on cfr_config.cuda_stream (borrowed, never destroyed).  Entry points that
 *     return data to host buffers synchronise that stream first.
 *   - Nothing throws across the ABI.  Every call returns a cfr_status; cfr_last_error() gives a
 *     message.  A CUDA error poisons the solver: later calls return CFR_ERR_STATE; free it.
 *   - One solver must not be used from two threads at once.
 */
#ifndef CFR_GB300_H
#define CFR_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CFR_OK = 0,
    CFR_ERR_INVALID = 1,     /* malformed arguments or game description */
    CFR_ERR_CUDA = 2,        /* a CUDA runtime call failed */
    CFR_ERR_OOM = 3,         /* device allocation failed */
    CFR_ERR_TIMEOUT = 4,     /* a bounded device-side wait expired */
    CFR_ERR_STATE = 5,       /* solver poisoned by an earlier error, or called out of order */
    CFR_ERR_UNSUPPORTED = 6  /* valid game the solver does not handle (see each call) */
} cfr_status;

/* Variants.  CFR+ is named in Section 1 without formulas; it is read as regret-matching+
 * (cumulative regrets clipped at 0 after every iteration) with linear averaging.  Linear and
 * discounted CFR are reweightings of Eq. 8 and Eq. 10 (Section 5 calls such variants direct in the
 * matrix form): linear CFR weights iteration T's instantaneous regret and average contribution by T;
 * discounted CFR (Brown and Sandholm, 2019) scales the accumulated regret, after adding iteration T's,
 * by T^alpha / (T^alpha + 1) where positive and T^beta / (T^beta + 1) elsewhere, and weights the
 * average contribution by T^gamma (cfr_config.dcfr_*). */
enum { CFR_VANILLA = 0, CFR_PLUS = 1, CFR_LINEAR = 2, CFR_DISCOUNTED = 3 };
/* Precision (Section 4.1 runs FP32 and FP64).  CFR_FP32: reach, node values and instantaneous
 * regrets in FP32, cumulative regrets and strategy sums in FP64.  CFR_FP64: everything FP64. */
enum { CFR_FP32 = 0, CFR_FP64 = 1 };
/* Simultaneous: both players update from the same iteration (the paper's vector form, Section 3.2).
 * Alternating: player 1's pass and update, then player 2's pass under player 1's new strategy (both
 * weighted as iteration T). */
enum { CFR_SIMULTANEOUS = 0, CFR_ALTERNATING = 1 };
/* Weight of iteration T in the average strategy: 1 (Eq. 10) or T.  DEFAULT = UNIFORM for vanilla
 * and LINEAR for CFR+.  Linear and discounted CFR fix their own weights (T, T^gamma). */
enum { CFR_AVG_DEFAULT = -1, CFR_AVG_UNIFORM = 0, CFR_AVG_LINEAR = 1 };
/* Phases of one iteration reported by cfr_phase_times. */
enum { CFR_PHASE_TOPDOWN = 0, CFR_PHASE_BOTTOMUP = 1, CFR_PHASE_FUSED = 2, CFR_PHASE_UPDATE = 3, CFR_PHASE_OWN = 4,
       CFR_PHASE_TOPDOWN_PAIR = 5, CFR_PHASE_BOTTOMUP_PAIR = 6 };

typedef struct cfr_solver cfr_solver;   /* opaque; owned by the library */

/* The game of the Definition in Section 2.1, as flat arrays in any node order. */
typedef struct {
    int64_t num_nodes;                  /* |V| >= 1; must be < 2^31 - 1 */
    const int32_t *parent;              /* [num_nodes] f_Pa; exactly one -1 (the root v_0) */
    const int32_t *action;              /* [num_nodes] f_a: index in [0, |A(f_h(parent))|); ignored at the root */
    const int32_t *infoset;             /* [num_nodes] f_h for decision nodes, -1 for terminals */
    int32_t num_infosets;               /* |H|, chance infosets included */
    const int8_t *infoset_player;       /* [num_infosets] f_i: 0 = chance (i_0), 1, 2 */
    const int32_t *infoset_num_actions; /* [num_infosets] |A(h)| >= 1 */
    const double *chance_prob;          /* sigma_0: chance infosets in id order, actions in order */
    int64_t num_chance_prob;            /* length of chance_prob = sum of |A(h)| over chance infosets */
    const double *utility;              /* [num_nodes x 2] u(t, 1), u(t, 2) row-major; read at terminals */
} cfr_game_desc;

/* Returns NULL on failure, else memory aligned to 256 bytes as cudaMalloc's is (the kernels' bulk copies
 * need 16-byte aligned arrays; a block that is not 256-byte aligned fails the call with CFR_ERR_INVALID). */
typedef void *(*cfr_alloc_fn)(size_t bytes, void *ctx);
typedef void (*cfr_free_fn)(void *ptr, void *ctx);

typedef struct {
    int32_t variant;        /* CFR_VANILLA | CFR_PLUS */
    int32_t precision;      /* CFR_FP32 | CFR_FP64 */
    int32_t update_mode;    /* CFR_SIMULTANEOUS | CFR_ALTERNATING */
    int32_t avg_weight;     /* CFR_AVG_DEFAULT | CFR_AVG_UNIFORM | CFR_AVG_LINEAR */
    int32_t device;         /* CUDA device ordinal; -1 = the calling thread's current device */
    void *cuda_stream;      /* cudaStream_t to run on (borrowed); NULL = the legacy default stream */
    cfr_alloc_fn dev_alloc; /* optional device allocator (both or neither) */
    cfr_free_fn dev_free;
    void *alloc_ctx;
    int32_t fuse_levels;    /* FP32 mode: the deepest depths run as one kernel, tile by tile in shared
                               memory, with their reaches and values kept on chip.  -1 = automatic
                               (default): the last two depths in one streamed pass, and the two depths
                               above them as a pair (one top-down and one bottom-up launch for both, see
                               cfr_info.pair_depth) where they lie below the head launches, hold no node
                               of more than 32 actions and the upper one has at least 8192 decision
                               nodes; 0 or 1 = none (one kernel per depth and pass); k >= 2 = at most k
                               depths (fewer where a subtree exceeds a tile or a node has more than 32
                               actions), no pair.  The forest part of a batch (cfr_batch_load) is
                               loaded with this setting too.  Ignored in FP64 mode. */
    int32_t record_nodes;   /* 1: fused depths also write every node's value and reaches to device
                               memory, so that cfr_get_nodes can return them; 0 (default): they do
                               not, and cfr_get_nodes returns CFR_ERR_STATE when depths are fused. */
    double dcfr_alpha;      /* CFR_DISCOUNTED: alpha, beta, gamma (defaults 1.5, 0, 2); finite */
    double dcfr_beta;
    double dcfr_gamma;
    int32_t head_levels;    /* FP32 mode: the shallowest depths of a tree whose root has decision children
                               only run in one launch per direction instead of one launch per depth, each
                               block walking the subtrees of a range of root children: the root and the
                               next k depths (each at most 2^19 nodes, none with more than 32 actions).
                               The forest part of a batch (cfr_batch_load) does the same with blocks
                               walking ranges of its games' roots (no root of more than 32 actions).
                               -1 (default) = as many as qualify, 0 = none, k >= 1 = at most k.
                               Ignored in FP64 mode. */
    int64_t batch_split_nodes;  /* cfr_batch_load: games of at least this many nodes run as one forest
                                   through the per-depth kernels, the rest in the persistent kernel if
                                   their image fits shared memory (0 = default 4096; negative = no split) */
    int32_t tail_slots;     /* FP32 mode, last two depths fused and streamed: 0 (default) = per-slot
                               strategy loads and regret atomics; where the tree's tiles are slot-dense
                               (consecutive nodes of a depth in consecutive infosets, as below one deal of
                               a public tree): 1 = the tiles' strategy entries staged in shared memory by
                               bulk copies, regrets by per-slot atomics; 2 = the same with the regrets
                               added to r~ by bulk reductions.  Elsewhere 1 and 2 act as 0. */
} cfr_config;

/* Sizes and accounting of a loaded solver. */
typedef struct {
    int64_t num_nodes, num_decision, num_terminal;
    int64_t num_q;
    int32_t num_infosets;
    int32_t num_levels;           /* depth levels holding decision nodes */
    int32_t max_depth;            /* deepest node (root at depth 0) */
    int32_t max_actions;
    int32_t single_level_infosets;/* 1 if every infoset's nodes share one depth (needed by cfr_exploitability) */
    int32_t variant, precision, update_mode, avg_weight;
    int64_t iteration;            /* completed iterations T */
    int64_t device_bytes;         /* device memory held by the solver */
    int64_t bytes_per_iteration;  /* algorithmic bytes of one iteration, the sum over cfr_phase_times'
                                     phases; with nothing fused 56 Nd + 4 Nt + 44 Q + 13 Hp - 12 - 20 Ndl
                                     (FP32 mode) or 96 Nd + 8 Nt + 56 Q + 17 Hp - 24 - 32 Ndl (FP64 mode),
                                     Hp the player infosets, Ndl the decision nodes of the last depth */
    int32_t kernels_per_iteration;/* kernel launches of one iteration */
    int64_t kernel_launches;      /* kernel launches made by cfr_iterate so far */
    int32_t fused_from_depth;     /* first depth run by the fused kernel (num_levels: none) */
    int32_t fused_tiles;          /* thread blocks of the fused kernel that process nodes */
    int32_t head_depths;          /* FP32 mode: leading depths run by the head launches (the root and the
                                     depths below it; cfr_config.head_levels), 0 if none */
    int32_t tail_kernel;          /* the last two depths: 0 per-depth kernels, 1 one thread per node (small
                                     trees), 2 streamed tiles with per-slot strategy loads and regret
                                     atomics, 3 streamed slot-dense tiles with staged strategy entries,
                                     4 the same with bulk-reduced regrets (cfr_config.tail_slots) */
    int32_t pair_depth;           /* FP32 mode: m when depths m and m+1 (just above the fused last two
                                     depths) run as a pair, one top-down and one bottom-up launch for both
                                     with depth m+1's reaches and values kept on chip; -1 if not */
} cfr_info;

/* Fills *c with defaults: vanilla, FP32, simultaneous, default averaging, current device,
 * legacy default stream, cudaMalloc. */
void cfr_config_init(cfr_config *c);

/* Checks a game description without touching the GPU.  CFR_OK, CFR_ERR_INVALID (malformed: bad
 * sizes or ids, not a single rooted tree, children not a bijection onto 0..|A(h)|-1, sigma_0
 * negative or not summing to 1 +- 1e-9 per chance infoset, non-finite utility, imperfect recall:
 * two nodes of one infoset whose acting player's own (infoset, action) history differs), or
 * CFR_ERR_UNSUPPORTED (valid but not two-player zero-sum, or sizes beyond 32-bit ids).  If msg is
 * non-NULL, a NUL-terminated reason of at most msg_len bytes is written. */
cfr_status cfr_validate(const cfr_game_desc *g, char *msg, size_t msg_len);

/* Test hook: builds the host layout of g with the one-thread builder (builder 0) or the multi-threaded
 * one (builder 1; cfr_load_tree uses it from 2^20 nodes on) and returns a 64-bit hash of every layout
 * array, so that the two can be compared; forest != 0 accepts several roots.  Errors as cfr_validate. */
cfr_status cfr_layout_digest(const cfr_game_desc *g, int32_t builder, int32_t forest, uint64_t *digest);

/* Validates the game (as cfr_validate), builds the level-ordered layout on the host (nodes sorted
 * by depth, children of a node contiguous and in action order - the level graphs L^(l) of
 * Section 3.1 made implicit), uploads it once and sets sigma^(1) to uniform (Section 3.1).
 * On success *out owns the solver; on failure *out is NULL and cfr_last_error(NULL) explains.
 * c may be NULL (defaults). */
cfr_status cfr_load_tree(const cfr_game_desc *g, const cfr_config *c, cfr_solver **out);

/* Queues n >= 0 full-tree CFR iterations (Section 3.2): top-down reach (Eq. 2, 4, 13), bottom-up
 * node values with the instantaneous-regret scatter (Eq. 1, 7, 11), then per infoset the
 * cumulative regret (Eq. 8/15, CFR+ clipping), strategy sum (Eq. 10/14) and regret matching
 * (Eq. 9).  Asynchronous on the solver's stream. */
cfr_status cfr_iterate(cfr_solver *s, int32_t n);

/* Waits for all queued work of the solver. */
cfr_status cfr_synchronize(cfr_solver *s);

/* Average strategy sigma-bar^(T) (Eq. 10, normalised; uniform where the strategy sum is 0) into
 * out[num_q]. */
cfr_status cfr_average_strategy(cfr_solver *s, double *out, int64_t len);

/* Current strategy sigma^(T+1) (Eq. 9) into out[num_q]. */
cfr_status cfr_current_strategy(cfr_solver *s, double *out, int64_t len);

/* NashConv = sum_i max_{sigma'_i} u_i(sigma'_i, sigma-bar_-i) - u_i(sigma-bar) of the average
 * strategy (Section 2.2, epsilon-Nash; used for sanity testing in Appendix A), computed on the GPU
 * in FP64 by one top-down and one bottom-up best-response pass per player; exploitability =
 * NashConv / 2.  Either pointer may be NULL.  CFR_ERR_UNSUPPORTED if some infoset spans two depths. */
cfr_status cfr_exploitability(cfr_solver *s, double *nash_conv, double *exploitability);

/* Size of the fixed working region used by cfr_exploitability_static, per GPU. */
#define CFR_STATIC_SCRATCH_BYTES ((size_t)32 << 20)

/* cfr_exploitability without any device allocation.  The paper has no counterpart; this entry
 * point exists for callers that may not allocate GPU memory while they run (a host application
 * that gives the library a fixed memory budget at set-up, or a real-time loop where cudaMalloc and
 * cudaFree, and the synchronisation they bring, are not allowed).  It runs the same best-response
 * kernels, but keeps all of their working memory in one region compiled into this library,
 * CFR_STATIC_SCRATCH_BYTES per GPU, which every GPU that loads the library holds until the process
 * exits.  A game needing more - 16 (num_decision + num_q) + 4 num_infosets bytes, rounded up -
 * returns CFR_ERR_UNSUPPORTED and leaves cfr_exploitability as the way to evaluate it.
 * The first call on a device looks up the region's device address (set-up, once per device); make
 * that first call before any stream capture.  All calls share the region and leave their contents
 * in it (each call resets what must start at zero), so calls that overlap on the GPU - from two
 * streams or two threads - race and give wrong results.  Results agree with cfr_exploitability's
 * to 1e-6 (the per-player kernels sum in another order than the two-player pass). */
cfr_status cfr_exploitability_static(cfr_solver *s, double *nash_conv, double *exploitability);

/* Copies the FP64 cumulative regrets R (R = T * r-bar of Eq. 8), strategy sums S (numerator of
 * Eq. 10 with one node's own reach per infoset), the last iteration's instantaneous regrets (Eq. 7)
 * into [len_q] buffers, the last iteration's own reach per infoset (Eq. 4) into own_reach[len_h],
 * and T into *iteration.  Any pointer may be NULL.  Checkpoint and test hook. */
cfr_status cfr_get_state(cfr_solver *s, double *cum_regret, double *strat_sum, double *inst_regret,
                         int64_t len_q, double *own_reach, int64_t len_h, int64_t *iteration);

/* Replaces R, S (each [len_q], len_q == num_q) and T, then sets the current strategy to the regret
 * matching of R (Eq. 9).  Entries of chance infosets are ignored.  Checkpoint restore / test hook. */
cfr_status cfr_set_state(cfr_solver *s, const double *cum_regret, const double *strat_sum, int64_t len_q,
                         int64_t iteration);

/* Per node of the last iteration, in caller node order ([len] each, len == num_nodes; any pointer
 * may be NULL): u1 = u-check(v, 1) (Eq. 1; the utility at terminals), cf_reach1 = pi-check(v, 1)
 * and cf_reach2 = pi-check(v, 2) (Eq. 2) at decision nodes, NaN at terminals.  CFR_ERR_STATE when
 * depths are fused and the solver was loaded without cfr_config.record_nodes.  Test hook. */
cfr_status cfr_get_nodes(cfr_solver *s, double *u1, double *cf_reach1, double *cf_reach2, int64_t len);

/* ---- depth-limited solving: leaves whose utility is refreshed between iterations -------------------
 * A depth-limited game ends in "leaves": terminals standing for the subtrees cut below them, whose
 * player-1 utility is set from outside (a value network) as the strategies change.  These calls keep
 * the refresh on the device: cfr_gather_ranges writes both players' ranges at the cut (products of
 * strategy probabilities along each public path, Eq. 4) into the network's input, and
 * cfr_set_leaf_values copies the network's output into the leaves' utilities.  Both are queued on the
 * solver's stream and take effect from the next iteration. */

/* Registers the range program: segment k (a range vector: one player at one cut public node) has
 * entries seg_entries[k] .. seg_entries[k + 1] - 1, written to out[seg_dst[k] + 0, 1, ...] by
 * cfr_gather_ranges; entry e is the product of the current strategy over the caller slots
 * slots[entry_prod[e] .. entry_prod[e + 1] - 1] (empty: 1), and each segment is divided by its sum
 * (uniform if 0).  seg_entries and entry_prod start at 0 and do not decrease.  Host arrays, copied. */
cfr_status cfr_set_range_program(cfr_solver *s, int64_t num_segments, const int64_t *seg_dst, const int64_t *seg_entries,
                                 const int64_t *entry_prod, const int32_t *slots);

/* Runs the range program on the current strategy sigma^(T+1) (CFR_CURRENT_STRATEGY) or on the average
 * strategy (CFR_AVERAGE_STRATEGY, Eq. 15); out is a DEVICE FP32 array. */
#define CFR_CURRENT_STRATEGY 0
#define CFR_AVERAGE_STRATEGY 1
cfr_status cfr_gather_ranges(cfr_solver *s, float *out, int32_t strategy);

/* Registers num_leaves terminal nodes (caller ids) and, per leaf, the index of its value in the array
 * cfr_set_leaf_values reads.  Host arrays, copied.  CFR_ERR_INVALID if a node is not a terminal. */
cfr_status cfr_set_leaves(cfr_solver *s, const int32_t *nodes, const int64_t *src_index, int64_t num_leaves);

/* Sets each registered leaf's player-1 utility to scale * src[src_index] (src: DEVICE FP32 array);
 * player 2's is its negation. */
cfr_status cfr_set_leaf_values(cfr_solver *s, const float *src, double scale);

/* Expected payoff of player 1 under the last iteration's profile sigma^(T): u-check(sigma^(T), v_0, 1)
 * of Eq. 1 at the root, which equals u-hat(sigma^(T), 1) of Section 2.2.  One scalar; synchronises
 * the stream (a per-iteration progress read).  0 before the first iteration. */
cfr_status cfr_root_value(cfr_solver *s, double *u1);

/* cfr_root_value without waiting: enqueues on the solver's stream, after the work queued so far, the
 * write of that value (as an FP64 number) to *u1, and returns.  u1 is caller-owned PAGE-LOCKED host
 * memory (cudaHostAlloc or cudaHostRegister; PyTorch's pin_memory) that the GPU can address; it holds
 * the value once the stream has passed this point (cfr_synchronize, or an event recorded on the stream
 * after this call).  For a loop that reads each iteration's value while the next one runs.
 * CFR_ERR_INVALID if u1 is NULL or not page-locked. */
cfr_status cfr_root_value_async(cfr_solver *s, double *u1);

/* Runs ONE iteration (it counts: T advances by 1) as individually launched kernels on the solver's
 * stream with CUDA events between its phases, and returns per phase the elapsed time in
 * microseconds (us), the phase's algorithmic bytes (bytes), its kind (CFR_PHASE_*) and depth (depth;
 * the first fused depth for CFR_PHASE_FUSED, the upper depth m for CFR_PHASE_TOPDOWN_PAIR and
 * CFR_PHASE_BOTTOMUP_PAIR, -1 for the own reaches and the update).  Phases in order: the own reaches of
 * all infosets (Eq. 4; if there are player infosets - cfr_iterate runs them beside the node passes),
 * top-down from depth 0, 1, ..., f-1 (depths m and m+1 in one CFR_PHASE_TOPDOWN_PAIR phase when
 * cfr_info.pair_depth = m >= 0), the fused depths f .. num_levels-1 (if any; f =
 * cfr_info.fused_from_depth), bottom-up at depth f-1, ..., 0 (depths m+1 and m in one
 * CFR_PHASE_BOTTOMUP_PAIR phase), then the per-infoset update (no phase at all for a game without
 * decision nodes).  The bytes add up to cfr_info.bytes_per_iteration.
 * *nphases receives the count; with us, bytes, kind and depth all NULL only the count is returned (no
 * iteration runs), otherwise len must be at least the count (NULL arrays are skipped).  Tracing hook. */
cfr_status cfr_phase_times(cfr_solver *s, double *us, double *bytes, int32_t *kind, int32_t *depth, int32_t len,
                           int32_t *nphases);

cfr_status cfr_get_info(const cfr_solver *s, cfr_info *info);

/* Message of the last failed call on s, or of the calling thread's last failed cfr_load_tree /
 * cfr_validate when s is NULL.  Valid until the next call on the same solver / thread. */
const char *cfr_last_error(const cfr_solver *s);

/* Releases the solver and its device memory (waits for its queued work).  NULL is a no-op. */
void cfr_free(cfr_solver *s);

/* ---- batched solving (many independent games; no counterpart in the paper) -------------------------
 * Many independent games solved side by side; every cfr_batch_iterate call advances all of them by n
 * iterations.  A game below the size split (cfr_config.batch_split_nodes) whose image fits in shared
 * memory (its structure, reaches, values, r~, sigma, R and S; at most 200 KB, about 5000 nodes) runs in
 * ONE persistent kernel launch (a CUDA graph of the launch and two bookkeeping nodes): a thread block
 * takes a game from a work queue (largest first), copies it into its shared memory, runs its n
 * iterations there depth by depth (Section 3.2's steps, as cfr_iterate's kernels compute them per node
 * and infoset), writes R, S and sigma back and takes the next game.  Every other game (larger, or with
 * a node of more than 32 actions) runs in one forest (one root per game) through cfr_iterate's
 * per-depth kernels on a second stream, concurrently.  FP32 mode with FP64 accumulators, simultaneous or
 * alternating updates, every variant.  Game g's arrays use its own caller numbering. */
typedef struct cfr_batch cfr_batch;   /* opaque; owned by the library */

typedef struct {
    int32_t threads_per_block;  /* multiple of 32 in [32, 256] */
    int32_t blocks_per_sm;      /* 0 = as many as fit */
} cfr_batch_tuning;

typedef struct {
    int32_t num_games;
    int64_t num_nodes, num_decision, num_q;
    int64_t iteration;          /* iterations every game has run */
    int64_t device_bytes;
    int32_t threads_per_block, blocks_per_sm, grid;   /* the launch shape in use */
    int32_t tuned;              /* 1 once set by cfr_batch_set_tuning or cfr_batch_autotune */
    int64_t kernel_launches;    /* kernels launched by cfr_batch_iterate so far */
    int32_t forest_games;       /* games run as one forest (at or above the split, too large or too wide) */
    int64_t forest_nodes;
    int64_t split_nodes;
    int64_t smem_bytes;         /* dynamic shared memory of a persistent block (its largest game's image) */
    int64_t forest_bytes_per_iteration;   /* algorithmic bytes of one iteration of the forest part
                                             (cfr_info.bytes_per_iteration of its solver) */
    int32_t forest_head_depths; /* cfr_info.head_depths of the forest part's solver */
} cfr_batch_info;

/* Validates and lays out num_games >= 1 games (each as cfr_load_tree would; the combined size must stay
 * below 2^31 - 1 nodes).  CFR_ERR_UNSUPPORTED for FP64 mode.  c may be NULL (defaults: vanilla; pass
 * variant CFR_PLUS for CFR+). */
cfr_status cfr_batch_load(const cfr_game_desc *games, int32_t num_games, const cfr_config *c, cfr_batch **out);

/* Queues n >= 0 iterations of every game (one persistent launch).  Asynchronous on the batch's stream. */
cfr_status cfr_batch_iterate(cfr_batch *b, int32_t n);

/* Sets the launch shape. */
cfr_status cfr_batch_set_tuning(cfr_batch *b, const cfr_batch_tuning *t);

/* Measures trial_iterations of every game for each block size in {64, 128, 256} and each
 * blocks-per-SM count in {1, 2, 4, 8, 16} that fits, on a copy of the state that is restored
 * afterwards (the iteration count does not move), and keeps the fastest.  *chosen and *best_us (time
 * per iteration of the whole batch) may be NULL.  Synchronises. */
cfr_status cfr_batch_autotune(cfr_batch *b, int32_t trial_iterations, cfr_batch_tuning *chosen, double *best_us);

/* Per game [len >= num_games]: the microseconds per iteration of its part of the last cfr_batch_iterate
 * call (from its first iteration's start to its last iteration's end, divided by n).  Synchronises. */
cfr_status cfr_batch_game_times(cfr_batch *b, double *us_per_iteration, int32_t len);

/* Per game [len >= num_games]: NashConv of its average strategy (Section 2.2; exploitability =
 * NashConv / 2).  CFR_ERR_UNSUPPORTED when an infoset spans depths.  Synchronises. */
cfr_status cfr_batch_exploitability(cfr_batch *b, double *nash_conv, int32_t len);

/* Game `game`'s cumulative regrets and strategy sums (either may be NULL; len >= its num_q) and the
 * iteration count.  Synchronises. */
cfr_status cfr_batch_get_state(cfr_batch *b, int32_t game, double *cum_regret, double *strat_sum, int64_t len,
                               int64_t *iteration);

/* Game `game`'s average strategy (Eq. 10 normalised; len >= its num_q).  Synchronises. */
cfr_status cfr_batch_average_strategy(cfr_batch *b, int32_t game, double *out, int64_t len);

cfr_status cfr_batch_get_info(const cfr_batch *b, cfr_batch_info *info);
const char *cfr_batch_last_error(const cfr_batch *b);   /* thread-local message if b == NULL */
void cfr_batch_free(cfr_batch *b);

/* ---- learned leaf values: a BF16 multilayer perceptron (no counterpart in the paper) ---------------
 * Depth-limited solving replaces the subtrees below a depth cutoff by a value network: a multilayer
 * perceptron of num_layers linear layers with ReLU between them, y = W_L(...ReLU(W_1 x + b_1)...) + b_L,
 * mapping (public-state embedding, both players' ranges) to both players' counterfactual values.  The
 * matrix products run on the tensor cores with BF16 operands and FP32 accumulation; the parameters are
 * kept in FP32 (the master copy, updated by Adam) with a BF16 copy for the products; hidden activations
 * and backpropagated gradients are BF16 between layers.  Loss: mean squared error over the batch and
 * the outputs, L = (1 / (B n_out)) sum (y - t)^2.
 * Parameter layout (host arrays of cfr_mlp_num_params floats): layer by layer, W_l row-major
 * [dims[l + 1]][dims[l]], then b_l [dims[l + 1]].
 * Device arrays (x, y, target, loss) belong to the caller and must stay valid until the queued work is
 * done; every call is asynchronous on the network's stream unless it says it synchronises. */
typedef struct cfr_mlp cfr_mlp;   /* opaque; owned by the library */

/* dims[0 .. num_layers]: input width, hidden widths, output width (each in [1, 8192]); 1 <= num_layers
 * <= 8.  Parameters start at zero (set them with cfr_mlp_set_params). */
cfr_status cfr_mlp_create(const int32_t *dims, int32_t num_layers, int32_t device, void *cuda_stream, cfr_mlp **out);
int64_t cfr_mlp_num_params(const cfr_mlp *m);

/* Host copies of the FP32 parameters / of the gradients of the last cfr_mlp_backward (layout above).
 * Synchronise. */
cfr_status cfr_mlp_set_params(cfr_mlp *m, const float *params, int64_t len);
cfr_status cfr_mlp_get_params(cfr_mlp *m, float *params, int64_t len);
cfr_status cfr_mlp_get_grads(cfr_mlp *m, float *grads, int64_t len);

/* y [batch][dims[L]] = the network at x [batch][dims[0]] (device, FP32, row-major); batch >= 1. */
cfr_status cfr_mlp_forward(cfr_mlp *m, const float *x, int32_t batch, float *y);

/* Forward and backward pass at (x, target [batch][dims[L]]): leaves dL/dparams in the network's
 * gradient buffer and, if loss != NULL, writes L to *loss (device, one double). */
cfr_status cfr_mlp_backward(cfr_mlp *m, const float *x, const float *target, int32_t batch, double *loss);

/* Test hook: a host copy (as FP32) of one intermediate of the last cfr_mlp_forward or
 * cfr_mlp_backward call, rows [0, batch) of that call and the real columns, row-major:
 *   CFR_MLP_ACT  layer `layer`'s input as its product read it (BF16): the rounded input x for
 *                layer 0, bf16(ReLU(Z)) of layer - 1 otherwise; [batch][dims[layer]];
 *   CFR_MLP_DZ   dL/dZ of layer `layer` (BF16), after cfr_mlp_backward only; [batch][dims[layer + 1]];
 *   CFR_MLP_OUT  the network output y (FP32); [batch][dims[num_layers]] (layer ignored).
 * Synchronises.  CFR_ERR_INVALID for a bad selector or layer or a short buffer (len entries),
 * CFR_ERR_STATE before the first pass or for CFR_MLP_DZ after a forward pass. */
#define CFR_MLP_ACT 0
#define CFR_MLP_DZ 1
#define CFR_MLP_OUT 2
cfr_status cfr_mlp_get_intermediate(cfr_mlp *m, int32_t which, int32_t layer, float *out, int64_t len);

/* One Adam step (Kingma and Ba, 2015, bias-corrected) on the gradients of the last cfr_mlp_backward:
 * m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2, p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps). */
cfr_status cfr_mlp_adam(cfr_mlp *m, float lr, float beta1, float beta2, float eps);

/* The time of one pass of each of the last cfr_mlp_forward and cfr_mlp_backward calls' matrix
 * products (microseconds, summed over layers) and their FLOPs (2 M N K over the padded shapes); NULLs
 * skip.  Synchronises. */
cfr_status cfr_mlp_gemm_stats(cfr_mlp *m, double *fwd_us, double *fwd_flops, double *bwd_us, double *bwd_flops);

/* The instructions the products run on: 2 (default) every product on tcgen05.mma (accumulator in tensor
 * memory, TMA-loaded operands; the data gradients read a transposed BF16 copy of the weights, the weight
 * gradients transposed copies of the layer inputs and output gradients written by the training pass, their
 * batch reduction split over blocks); 0 mma.sync for every product; 1 tcgen05.mma for every product with
 * per-thread operand copies.  Results agree within the rounding of FP32 accumulation.  Takes effect for
 * later calls. */
cfr_status cfr_mlp_set_tensor_path(cfr_mlp *m, int32_t path);

/* Waits for the network's queued work; CFR_ERR_TIMEOUT if a tensor-core kernel gave up waiting for its
 * operands (the network is then unusable). */
cfr_status cfr_mlp_synchronize(cfr_mlp *m);

const char *cfr_mlp_last_error(const cfr_mlp *m);   /* thread-local message if m == NULL */
void cfr_mlp_free(cfr_mlp *m);

#ifdef __cplusplus
}
#endif
#endif /* CFR_GB300_H */
