// C ABI of the solver (include/cfr_gb300.h): device memory, uploads, the per-iteration launch
// sequence captured once into a CUDA graph, getters and the GPU best response.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "cfr_gb300.h"
#include "kernels.cuh"
#include "layout.hpp"
#include "solver_internal.hpp"
#include "stream.cuh"

using namespace cfrgb;

namespace {

thread_local std::string g_thread_err;

constexpr int kBlock = 256;
constexpr int kGraphIters = 4;   // iterations captured in the solver's second graph (cfr_iterate replays it first)
constexpr int kWideBlock = 1024;   // nodes and infosets with more than 32 actions: one block each
constexpr int32_t kFuseAuto = 2;   // fused depths when cfr_config.fuse_levels < 0
constexpr int32_t kPairMinNodes = 8192;      // FP32: fewest decision nodes at the upper depth of a pair
constexpr int32_t kStreamMinNodes = 32768;   // FP32 bottom-up depths this large use k_bottomup_stream
constexpr int32_t kHeadMaxNodes = 1 << 19;   // FP32: leading depths at most this large run in the head launches
constexpr int32_t kHeadMaxSmem = 96 << 10;   // shared memory of a head block, at most

inline int32_t nblocks(int64_t n) { return (int32_t)((n + kBlock - 1) / kBlock); }

// Restores the caller's current device when an entry point returns.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; prev = -1; return; }
        if (dev >= 0 && dev != prev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

struct cfr_solver {
    cfr_config cfg{};
    int device = 0;
    cudaStream_t stream = nullptr;   // borrowed
    cudaStream_t cap = nullptr;      // private, for graph capture
    cudaStream_t side = nullptr;     // private: the own-reach branch of the captured iteration
    cudaEvent_t fork[2] = {nullptr, nullptr}, join[2] = {nullptr, nullptr};   // per pass of an iteration
    cudaEvent_t deep[2] = {nullptr, nullptr};             // split update: the deep infosets' regrets are complete
    cudaEvent_t upd[2] = {nullptr, nullptr};              // split update: the deep infosets' update is done
    int prio_least = 0, prio_greatest = 0;                // the device's stream priority range
    double *wts = nullptr;                                // linear / discounted CFR weights (k_weights)
    // sizes
    int64_t N = 0, Nd = 0, Nt = 0, Q = 0;
    int32_t H = 0, L = 0, max_depth = 0, max_actions = 0;
    bool single_level = true;
    std::vector<int32_t> dlevel, hlevel, dnode_user, tnode_user, h_int2user;
    // device arrays
    int32_t *dfirst = nullptr, *tfirst = nullptr, *dinfo = nullptr, *qbase = nullptr, *pseq = nullptr,
            *pseq_h = nullptr, *q_int2user = nullptr, *astar = nullptr;
    int8_t *iplayer = nullptr;
    uint32_t *kmask = nullptr, *wbits = nullptr, *qp = nullptr;
    void *util = nullptr, *sigma = nullptr, *inst = nullptr, *reach1 = nullptr, *reach2 = nullptr,
         *u = nullptr, *own = nullptr;
    double *util64 = nullptr, *sigma064 = nullptr, *R = nullptr, *S = nullptr, *stage = nullptr;
    double *br_reach = nullptr, *br_val = nullptr, *br_cfv = nullptr, *avg = nullptr, *br_out = nullptr;
    double *br_reach2 = nullptr, *br_val2 = nullptr;   // player 2's, beside player 1's in br_reach / br_val
    cudaGraphExec_t br_exec = nullptr;                   // the average strategy and both best responses
    int64_t *d_iter = nullptr;
    int *d_err = nullptr;                                 // set by a device-side wait that expired
    int32_t sb_grid[3] = {0, 0, 0}, td_grid[3] = {0, 0, 0};   // streamed kernels: resident blocks, per
                                                                // unrolled action count (kStreamNA)
    std::vector<int32_t> level_na;                        // per depth: index into kStreamNA
    int32_t hp_na = 0;                                    // FP32 update: largest action count of at most 32
    int32_t nwide_h = 0;                                  // player infosets with more than 32 actions
    int32_t *wide_h = nullptr;
    void *contrib = nullptr;                              // FP64 mode: per-edge regret contributions
    int32_t *hnode_start = nullptr, *hnode = nullptr;     // FP64 mode: nodes of each infoset, depth-first
    int32_t *wide = nullptr;                              // nodes with more than 32 actions, by depth
    std::vector<int32_t> wlevel;
    std::vector<char> ddepth_children;                    // depth l has a node with a decision child
    std::vector<int64_t> level_children;                  // children of the decision nodes of depth l
    std::vector<int64_t> level_terminals;                 // terminal children of the decision nodes of depth l
    // FP32 mode: depths fuse_r .. L-1 run in k_fused (fuse_r == L: none), in fuse_ntiles tiles whose
    // node ranges per fused depth are fuse_bounds[k][0 .. fuse_ntiles]
    int32_t fuse_r = 0, fuse_ntiles = 0;
    int32_t *fuse_bounds = nullptr;
    bool fuse_tail = false;                               // the last two depths by k_tail / k_tail_stream /
                                                          // k_tail_slots
    bool tail_slots = false;                              // k_tail_slots (slot-dense tiles) for them
    int32_t *tail_tiles = nullptr;                        // 8 words per tile (TailTiles::tm), or 12
                                                          // (SlotTailTiles::tm)
    int32_t ntail_tiles = 0, tl_grid[3] = {0, 0, 0}, ts_grid[3] = {0, 0, 0};
    // FP32 mode: depths pair_m and pair_m + 1 (just above the fused tail) in one top-down and one bottom-up
    // launch (k_pair_*), over npair_tiles tiles of 12 words (PairTopDownTiles::tm); pair_m < 0: none
    int32_t pair_m = -1, npair_tiles = 0, pt_grid[3] = {0, 0, 0}, pb_grid[3] = {0, 0, 0};
    int32_t *pair_tiles = nullptr;
    int32_t Hp = 0;                                       // player infosets: internal ids [0, Hp)
    // FP32 mode: depths 0 .. head_n - 1 run in one launch per direction (k_head_*), head_per_block root
    // children per block; head_n == 0: per-depth launches
    int32_t head_n = 0, head_per_block = 0, head_cap = 0, head_na = 0;   // head_na: index into kStreamNA
    int32_t *head_done = nullptr;
    int32_t *head_rng = nullptr;                          // per head block kHeadRangeWords words (head_ranges)
    // depth-limited solving (cfr_set_range_program, cfr_set_leaves)
    int64_t rp_nseg = 0, nleaves = 0;
    int64_t *rp_dst = nullptr, *rp_ent = nullptr, *rp_prod = nullptr, *leaf_src = nullptr;
    int32_t *rp_slots = nullptr, *leaf_t = nullptr;
    int64_t kernel_launches = 0;
    int64_t iteration = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    cudaGraph_t graph2 = nullptr;                         // kGraphIters iterations back to back: no graph-launch
    cudaGraphExec_t graph_exec2 = nullptr;                // gap between them
    std::vector<std::pair<void *, size_t>> blocks;
    int64_t device_bytes = 0;
    std::string err;
    bool poisoned = false;

    size_t real_size() const { return cfg.precision == CFR_FP64 ? sizeof(double) : sizeof(float); }
};

namespace {

cfr_status set_err(cfr_solver *s, cfr_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (s) s->err = buf;
    else g_thread_err = buf;
    return st;
}

#define CK(call)                                                                                        \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess) {                                                                        \
            s->poisoned = true;                                                                         \
            return set_err(s, e_ == cudaErrorMemoryAllocation ? CFR_ERR_OOM : CFR_ERR_CUDA, "%s: %s (%s:%d)", \
                           #call, cudaGetErrorString(e_), __FILE__, __LINE__);                           \
        }                                                                                               \
    } while (0)

#define CK_LAUNCH() CK(cudaGetLastError())

cfr_status dev_alloc(cfr_solver *s, void **p, size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes == 0) bytes = 256;
    void *ptr = nullptr;
    if (s->cfg.dev_alloc) {
        ptr = s->cfg.dev_alloc(bytes, s->cfg.alloc_ctx);
        if (!ptr) return set_err(s, CFR_ERR_OOM, "device allocator returned NULL for %zu bytes", bytes);
        if (reinterpret_cast<uintptr_t>(ptr) & 255u) {
            s->cfg.dev_free(ptr, s->cfg.alloc_ctx);
            return set_err(s, CFR_ERR_INVALID, "device allocator returned %p: not 256-byte aligned", ptr);
        }
    } else {
        cudaError_t e = cudaMalloc(&ptr, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_err(s, CFR_ERR_OOM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
        }
    }
    s->blocks.emplace_back(ptr, bytes);
    s->device_bytes += (int64_t)bytes;
    *p = ptr;
    return CFR_OK;
}

template <typename T>
cfr_status alloc_n(cfr_solver *s, T **p, int64_t n) {
    return dev_alloc(s, reinterpret_cast<void **>(p), sizeof(T) * (size_t)(n > 0 ? n : 1));
}

template <typename T>
cfr_status upload(cfr_solver *s, T *dst, const std::vector<T> &src) {
    if (src.empty()) return CFR_OK;
    CK(cudaMemcpyAsync(dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, s->stream));
    return CFR_OK;
}

#define TRY(x)                                \
    do {                                      \
        cfr_status st_ = (x);                 \
        if (st_ != CFR_OK) return st_;        \
    } while (0)

template <typename real>
DevTree<real> dev_tree(cfr_solver *s) {
    DevTree<real> t;
    t.dfirst = s->dfirst; t.tfirst = s->tfirst; t.dinfo = s->dinfo;
    t.kmask = s->kmask; t.wbits = s->wbits; t.qp = s->qp;
    t.util = static_cast<const real *>(s->util);
    t.qbase = s->qbase; t.iplayer = s->iplayer; t.pseq = s->pseq; t.pseq_h = s->pseq_h;
    t.sigma = static_cast<real *>(s->sigma); t.inst = static_cast<real *>(s->inst);
    t.reach1 = static_cast<real *>(s->reach1); t.reach2 = static_cast<real *>(s->reach2);
    t.u = static_cast<real *>(s->u); t.own = static_cast<real *>(s->own);
    t.R = s->R; t.S = s->S; t.iter = s->d_iter;
    t.contrib = static_cast<real *>(s->contrib); t.hnode_start = s->hnode_start; t.hnode = s->hnode;
    t.pmask = 6;
    t.wts = s->wts;
    return t;
}

// Kernel launches of one queued iteration.  In the captured graph (pdl) a kernel that directly follows
// another kernel on its stream is a programmatic dependent launch: its blocks may be scheduled while
// the previous kernel drains, and it waits for that kernel in grid_dependency_wait.  Any other
// operation on the stream (a memset, an event) ends the chain (`cut`).
struct Launcher {
    bool pdl = false;
    int prio = 0;                                        // launch priority (cudaLaunchAttributePriority) if nonzero
    cudaStream_t chained[2] = {nullptr, nullptr};   // streams whose last operation was a kernel
    int nchained = 0;
    bool follows_kernel(cudaStream_t st) const {
        for (int i = 0; i < nchained; ++i)
            if (chained[i] == st) return true;
        return false;
    }
    void cut(cudaStream_t st) {
        for (int i = 0; i < nchained; ++i)
            if (chained[i] == st) chained[i] = chained[--nchained];
    }
    template <typename... P, typename... A>
    cudaError_t operator()(void (*k)(P...), int grid, int block, size_t smem, cudaStream_t st, A... args) {
        cudaLaunchConfig_t c = {};
        c.gridDim = dim3((unsigned)grid);
        c.blockDim = dim3((unsigned)block);
        c.dynamicSmemBytes = smem;
        c.stream = st;
        cudaLaunchAttribute at[2];
        unsigned n = 0;
        if (pdl && follows_kernel(st)) {
            at[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            at[n++].val.programmaticStreamSerializationAllowed = 1;
        }
        if (prio != 0) {
            at[n].id = cudaLaunchAttributePriority;
            at[n++].val.priority = prio;
        }
        c.attrs = at;
        c.numAttrs = n;
        const cudaError_t e = cudaLaunchKernelEx(&c, k, args...);
        if (!follows_kernel(st) && nchained < 2) chained[nchained++] = st;
        return e;
    }
    // One thread-block cluster of `ctas` blocks.
    template <typename... P, typename... A>
    cudaError_t cluster(void (*k)(P...), int ctas, int block, cudaStream_t st, A... args) {
        cudaLaunchConfig_t c = {};
        c.gridDim = dim3((unsigned)ctas);
        c.blockDim = dim3((unsigned)block);
        c.stream = st;
        cudaLaunchAttribute at[2];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)ctas;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[1].val.programmaticStreamSerializationAllowed = 1;
        c.attrs = at;
        c.numAttrs = pdl && follows_kernel(st) ? 2 : 1;
        const cudaError_t e = cudaLaunchKernelEx(&c, k, args...);
        if (!follows_kernel(st) && nchained < 2) chained[nchained++] = st;
        return e;
    }
};

HeadArgs head_args(const cfr_solver *s, bool bump) {
    HeadArgs a{};
    a.n = s->head_n - 1;
    a.bump = bump;
    a.forest = s->dlevel[1] > 1;
    a.d1 = a.forest ? 0 : s->dlevel[1];
    a.nroot = a.forest ? s->dlevel[1] : s->dlevel[2] - s->dlevel[1];
    a.per_block = s->head_per_block;
    a.nblk = (a.nroot + a.per_block - 1) / a.per_block;
    a.cap = s->head_cap;
    a.nown = s->hlevel[(size_t)s->head_n];
    a.done = s->head_done;
    a.rng = s->head_rng;
    return a;
}

// Whether the head top-down of this pass clears r~ (instead of the memset before it): simultaneous
// updates, in the graph's iteration.
bool head_clears(const cfr_solver *s, bool timed_phases, bool alt) { return s->head_n > 0 && !timed_phases && !alt; }

// Whether the top-down step from depth l launches anything: a depth whose nodes have no decision
// children (the last one) has none, except depth 0, whose first thread counts the iteration, and
// FP32 mode's wide nodes, whose kernel runs regardless.
bool topdown_launches(const cfr_solver *s, int32_t l) {
    return s->ddepth_children[l] || l == 0 ||
           (s->cfg.precision == CFR_FP32 && s->wlevel[l + 1] > s->wlevel[l]);
}

// Streamed top-down (bottom_up false) or bottom-up step of depth l = [j0, j1) in the instantiation
// for the depth's largest action count.  False when the kernels could not be set up (then the caller
// launches the per-depth kernel).
template <int NA>
cudaError_t launch_stream_na(Launcher &go, const cfr_solver *s, const DevTree<float> &t, cudaStream_t st,
                             bool bottom_up, int32_t l, int32_t j0, int32_t j1, int gi, bool first) {
    const int32_t tiles = (j1 - j0 + kSBN - 1) / kSBN;
    if (bottom_up)
        return go(k_bottomup_stream<NA>, std::min(s->sb_grid[gi], tiles), kSBThreads, sizeof(SBStage) * kSBStages, st,
                  t, j0, j1, s->d_err);
    return go(k_topdown_stream<NA>, std::min(s->td_grid[gi], tiles), kSBThreads,
              sizeof(TDStage) * TopDownTiles<NA>::kStages, st, t, j0, j1, (int32_t)(first && l == 0), s->d_err);
}

bool launch_stream(Launcher &go, const cfr_solver *s, const DevTree<float> &t, cudaStream_t st, bool bottom_up,
                   int32_t l, int32_t j0, int32_t j1, bool first) {
    const int gi = s->level_na[(size_t)l];
    if ((bottom_up ? s->sb_grid[gi] : s->td_grid[gi]) <= 0) return false;
    if (gi == 0) launch_stream_na<kStreamNA[0]>(go, s, t, st, bottom_up, l, j0, j1, gi, first);
    else if (gi == 1) launch_stream_na<kStreamNA[1]>(go, s, t, st, bottom_up, l, j0, j1, gi, first);
    else launch_stream_na<kStreamNA[2]>(go, s, t, st, bottom_up, l, j0, j1, gi, first);
    return true;
}

// Shared-memory limits and resident blocks of the streamed kernels built for NA actions.
template <int NA>
cfr_status setup_stream_na(cfr_solver *s, int gi, int sms) {
    int per_sm = 0;
    const int bsmem = (int)(sizeof(SBStage) * kSBStages);
    CK(cudaFuncSetAttribute(k_bottomup_stream<NA>, cudaFuncAttributeMaxDynamicSharedMemorySize, bsmem));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bottomup_stream<NA>, kSBThreads, bsmem));
    s->sb_grid[gi] = per_sm * sms;
    const int tsmem = (int)(sizeof(TDStage) * TopDownTiles<NA>::kStages);
    CK(cudaFuncSetAttribute(k_topdown_stream<NA>, cudaFuncAttributeMaxDynamicSharedMemorySize, tsmem));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_topdown_stream<NA>, kSBThreads, tsmem));
    s->td_grid[gi] = per_sm * sms;
    const int lsmem = (int)(sizeof(TLStage) * TailTiles<NA>::kStages);
    CK(cudaFuncSetAttribute(k_tail_stream<NA>, cudaFuncAttributeMaxDynamicSharedMemorySize, lsmem));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tail_stream<NA>, kSBThreads, lsmem));
    s->tl_grid[gi] = per_sm * sms;
    const int ssmem = (int)(sizeof(STStage) * SlotTailTiles<NA, false>::kStages);
    for (auto k : {k_tail_slots<NA, false>, k_tail_slots<NA, true>})
        CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, ssmem));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tail_slots<NA, false>, 32 * (kSTWarps + 1), ssmem));
    s->ts_grid[gi] = per_sm * sms;
    const int ptsmem = (int)(sizeof(PTStage) * PairTopDownTiles<NA>::kStages);
    CK(cudaFuncSetAttribute(k_pair_topdown<NA>, cudaFuncAttributeMaxDynamicSharedMemorySize, ptsmem));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pair_topdown<NA>, kSBThreads, ptsmem));
    s->pt_grid[gi] = per_sm * sms;
    const int pbsmem = (int)(sizeof(PBStage) * PairBottomUpTiles<NA>::kStages);
    CK(cudaFuncSetAttribute(k_pair_bottomup<NA>, cudaFuncAttributeMaxDynamicSharedMemorySize, pbsmem));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pair_bottomup<NA>, kSBThreads, pbsmem));
    s->pb_grid[gi] = per_sm * sms;
    return CFR_OK;
}

// Whether depths l and l + 1 run as the pair (k_pair_topdown / k_pair_bottomup) in a pass whose first
// per-depth launch is at depth head.
bool pair_at(const cfr_solver *s, int32_t l, int32_t head) {
    return s->pair_m >= head && l == s->pair_m && s->npair_tiles > 0;
}

// The paired launches of depths pair_m and pair_m + 1, in the instantiation for their largest action
// count; bump: depth pair_m is the root's (the top-down launch counts the iteration).
cfr_status launch_pair(Launcher &go, cfr_solver *s, const DevTree<float> &t, cudaStream_t st, bool bottom_up,
                       int32_t bump) {
    const int32_t m = s->pair_m;
    const int gi = std::max(s->level_na[(size_t)m], s->level_na[(size_t)m + 1]);
    const int4 *tb = reinterpret_cast<const int4 *>(s->pair_tiles);
    const int32_t rec = s->cfg.record_nodes != 0, nt = s->npair_tiles;
    if (bottom_up) {
        const int grid = std::min(s->pb_grid[gi], nt);
        const size_t smem = sizeof(PBStage) * PairBottomUpTiles<3>::kStages;
        if (gi == 0) CK(go(k_pair_bottomup<kStreamNA[0]>, grid, kSBThreads, smem, st, t, tb, nt, rec, s->d_err));
        else if (gi == 1) CK(go(k_pair_bottomup<kStreamNA[1]>, grid, kSBThreads, smem, st, t, tb, nt, rec, s->d_err));
        else CK(go(k_pair_bottomup<kStreamNA[2]>, grid, kSBThreads, smem, st, t, tb, nt, rec, s->d_err));
    } else {
        const int grid = std::min(s->pt_grid[gi], nt);
        const size_t smem = sizeof(PTStage) * PairTopDownTiles<3>::kStages;
        if (gi == 0) CK(go(k_pair_topdown<kStreamNA[0]>, grid, kSBThreads, smem, st, t, tb, nt, rec, bump, s->d_err));
        else if (gi == 1) CK(go(k_pair_topdown<kStreamNA[1]>, grid, kSBThreads, smem, st, t, tb, nt, rec, bump, s->d_err));
        else CK(go(k_pair_topdown<kStreamNA[2]>, grid, kSBThreads, smem, st, t, tb, nt, rec, bump, s->d_err));
    }
    return CFR_OK;
}

// FP32 update of variant V: one thread per infoset (k_update_rows, instantiated for the largest action
// count) and one block per infoset of more than 32 actions.
// The update of the player infosets [h0, h1) (up to 32 actions) and, with wide, of the wider ones.
template <int V>
cfr_status launch_update(Launcher &go, cfr_solver *s, const DevTree<float> &t, cudaStream_t st, int32_t linear,
                         int32_t h0, int32_t h1, bool wide) {
    if (h1 > h0) {
        const int g = nblocks(h1 - h0);
        if (s->hp_na <= 3) CK(go(k_update_rows<3, V>, g, kBlock, 0, st, t, h0, h1, linear));
        else if (s->hp_na <= 5) CK(go(k_update_rows<5, V>, g, kBlock, 0, st, t, h0, h1, linear));
        else CK(go(k_update_rows<8, V>, g, kBlock, 0, st, t, h0, h1, linear));
    }
    if (wide && s->nwide_h > 0)
        CK(go(k_update_list<V>, s->nwide_h, kWideBlock, 0, st, t, (const int32_t *)s->wide_h, linear));
    return CFR_OK;
}
cfr_status launch_update_any(Launcher &go, cfr_solver *s, const DevTree<float> &t, cudaStream_t st, int32_t linear,
                             int32_t h0, int32_t h1, bool wide) {
    switch (s->cfg.variant) {
    case CFR_VANILLA: return launch_update<CFRV_VANILLA>(go, s, t, st, linear, h0, h1, wide);
    case CFR_PLUS: return launch_update<CFRV_PLUS>(go, s, t, st, linear, h0, h1, wide);
    case CFR_LINEAR: return launch_update<CFRV_LINEAR>(go, s, t, st, linear, h0, h1, wide);
    default: return launch_update<CFRV_DISCOUNTED>(go, s, t, st, linear, h0, h1, wide);
    }
}

// One full-tree iteration, queued on `st` (captured into the solver's graph).  FP64 mode reduces
// the instantaneous regrets deterministically (k_update sums per-edge contributions in depth-first
// node order); FP32 mode adds them with atomics, streams large depths through shared memory, and
// runs the depths fuse_r .. L-1 in one kernel when fusion is on.  The own reaches (k_own, one launch
// per depth) depend only on sigma and on shallower own reaches: in the graph they run on a branch
// forked from `st` that joins before the update.  With `ev` (one more than the phases), everything
// runs on `st` and an event is recorded before the first phase and after each phase: own reaches,
// top-down from depth 0 .. fuse_r - 1, the fused depths (if any), bottom-up at depth fuse_r - 1 .. 0,
// update.
template <typename real>
cfr_status enqueue_pass(cfr_solver *s, cudaStream_t st, cudaEvent_t *ev, int32_t pmask, bool first) {
    constexpr bool det = sizeof(real) == sizeof(double);
    DevTree<real> t = dev_tree<real>(s);
    t.pmask = pmask;
    const bool alt = pmask != 6;
    const int pi = pmask == 4;                                   // which fork/join events
    const int32_t r = det ? s->L : s->fuse_r;
    Launcher go;
    go.pdl = ev == nullptr;
    int ne = 0;
    auto mark = [&]() -> cfr_status {
        if (ev) {
            CK(cudaEventRecord(ev[ne++], st));
            go.cut(st);
        }
        return CFR_OK;
    };
    if (!det && !alt && !head_clears(s, ev != nullptr, alt)) CK(cudaMemsetAsync(s->inst, 0, sizeof(real) * (size_t)s->Q, st));
    if (!det && alt && s->Hp > 0) CK(go(k_zero_inst<real>, nblocks(s->Hp), kBlock, 0, st, t, s->Hp));
    TRY(mark());
    // the shallowest depths in one launch per direction (the graph's iteration only: the phase timer
    // keeps one launch per depth); the top-down launch also forms their infosets' own reaches
    const int32_t head = (!det && ev == nullptr) ? s->head_n : 0;
    if constexpr (!det) {
        if (head > 0) {
            HeadArgs ha = head_args(s, first);
            if (head_clears(s, ev != nullptr, alt)) {
                ha.zero = reinterpret_cast<float *>(s->inst);
                ha.nzero = s->Q;
            }
            auto k = s->head_na == 0 ? k_head_topdown<kStreamNA[0]>
                   : s->head_na == 1 ? k_head_topdown<kStreamNA[1]> : k_head_topdown<kStreamNA[2]>;
            CK(go(k, ha.nblk + (ha.nown + kHeadThreads - 1) / kHeadThreads, kHeadThreads, head_smem_topdown(ha.cap), st,
                  t, ha));
        }
    }
    // the other own reaches, depth by depth; in the graph on a branch beside the node passes that forks
    // after the head (whose own reaches they extend) and joins before the update
    const bool branch = ev == nullptr;
    // Split update (the graph's simultaneous pass with a head): the regrets of the infosets first seen
    // below the head are complete when the deep bottom-up passes end, so their update runs on the branch
    // beside the head's bottom-up launch (latency-bound: few bytes, block barriers); the head's infosets'
    // update follows it.  (Starting the fused depths' infosets right after the fused kernel, beside the
    // bandwidth-bound bottom-up passes, measured slower.)
    const bool split = branch && head > 0 && !alt && s->Hp > 0;
    const int32_t hsplit = split ? s->hlevel[(size_t)head] : 0;
    const int32_t linear = s->cfg.avg_weight == CFR_AVG_LINEAR, variant = s->cfg.variant;
    // the deep infosets' update on the branch, after its own reaches and the event below
    auto deep_update = [&]() -> cfr_status {
        if (first && variant == CFR_DISCOUNTED)
            CK(go(k_weights, 1, 1, 0, st, (const int64_t *)s->d_iter, s->wts, s->cfg.dcfr_alpha, s->cfg.dcfr_beta,
                  s->cfg.dcfr_gamma));
        CK(cudaEventRecord(s->deep[pi], st));
        CK(cudaStreamWaitEvent(s->side, s->deep[pi], 0));
        go.cut(s->side);
        if constexpr (!det) TRY(launch_update_any(go, s, t, s->side, linear, hsplit, s->Hp, false));
        CK(cudaEventRecord(s->upd[pi], s->side));
        go.cut(s->side);
        go.prio = s->prio_greatest;                      // the head's blocks go ahead of its blocks
        return CFR_OK;
    };
    cudaStream_t os = st;
    if (branch) {
        os = s->side;
        CK(cudaEventRecord(s->fork[pi], st));
        CK(cudaStreamWaitEvent(os, s->fork[pi], 0));
    }
    for (int32_t l = head; l < s->L; ++l) {
        const int32_t h0 = s->hlevel[l], h1 = s->hlevel[l + 1];
        if (h1 > h0) CK(go(k_own<real>, nblocks(h1 - h0), kBlock, 0, os, t, h0, h1));
    }
    if (branch) {
        CK(cudaEventRecord(s->join[pi], os));
        go.cut(os);
    }
    if (s->Hp > 0) TRY(mark());
    for (int32_t l = head; l < r; ++l) {
        if constexpr (!det) {
            if (pair_at(s, l, head)) {                   // the top-down steps of depths l and l + 1
                TRY(launch_pair(go, s, t, st, false, (int32_t)(first && l == 0)));
                TRY(mark());
                ++l;
                continue;
            }
        }
        if (!topdown_launches(s, l)) continue;
        const int32_t j0 = s->dlevel[l], j1 = s->dlevel[l + 1];
        if (s->ddepth_children[l] || l == 0) {
            bool streamed = false;
            if constexpr (!det) {
                if (j1 - j0 >= kStreamMinNodes) streamed = launch_stream(go, s, t, st, false, l, j0, j1, first);
            }
            if (!streamed)
                CK(go(k_topdown<real, !det>, nblocks(j1 - j0), kBlock, 0, st, t, j0, j1, (int32_t)(first && l == 0)));
            CK_LAUNCH();
        }
        const int32_t nw = s->wlevel[l + 1] - s->wlevel[l];
        if (!det && nw > 0) CK(go(k_topdown_wide<real>, nw, kWideBlock, 0, st, t, (const int32_t *)s->wide, s->wlevel[l]));
        TRY(mark());
    }
    if constexpr (!det) {
        if (r < s->L && s->fuse_tail) {
            const int32_t j0 = s->dlevel[r], j1 = s->dlevel[r + 1];
            const int32_t rec = s->cfg.record_nodes != 0, bump = first && r == 0;
            const int gi = std::max(s->level_na[(size_t)r], s->level_na[(size_t)r + 1]);
            if (s->tail_slots && s->ntail_tiles > 0 && s->ts_grid[gi] > 0) {
                const int grid = std::min(s->ts_grid[gi], s->ntail_tiles);
                const size_t smem = sizeof(STStage) * SlotTailTiles<3, false>::kStages;
                const int4 *tb = reinterpret_cast<const int4 *>(s->tail_tiles);
                const int nth = 32 * (kSTWarps + 1);
                const bool bulk = s->cfg.tail_slots == 2;
                auto kern = gi == 0 ? (bulk ? k_tail_slots<kStreamNA[0], true> : k_tail_slots<kStreamNA[0], false>)
                          : gi == 1 ? (bulk ? k_tail_slots<kStreamNA[1], true> : k_tail_slots<kStreamNA[1], false>)
                                    : (bulk ? k_tail_slots<kStreamNA[2], true> : k_tail_slots<kStreamNA[2], false>);
                CK(go(kern, grid, nth, smem, st, t, tb, s->ntail_tiles, rec, bump, s->d_err));
            } else if (s->ntail_tiles > 0 && s->tl_grid[gi] > 0) {
                const int grid = std::min(s->tl_grid[gi], s->ntail_tiles);
                const size_t smem = sizeof(TLStage) * TailTiles<3>::kStages;
                const int4 *tb = reinterpret_cast<const int4 *>(s->tail_tiles);
                if (gi == 0) CK(go(k_tail_stream<kStreamNA[0]>, grid, kSBThreads, smem, st, t, tb, s->ntail_tiles, rec, bump, s->d_err));
                else if (gi == 1) CK(go(k_tail_stream<kStreamNA[1]>, grid, kSBThreads, smem, st, t, tb, s->ntail_tiles, rec, bump, s->d_err));
                else CK(go(k_tail_stream<kStreamNA[2]>, grid, kSBThreads, smem, st, t, tb, s->ntail_tiles, rec, bump, s->d_err));
            } else {
                CK(go(k_tail, nblocks(j1 - j0), kBlock, 0, st, t, j0, j1, rec, bump));
            }
            TRY(mark());
        } else if (r < s->L) {
            FuseArgs fa;
            fa.bounds = s->fuse_bounds;
            fa.ntiles = s->fuse_ntiles;
            fa.levels = s->L - r;
            fa.record = s->cfg.record_nodes != 0;
            fa.bump = first && r == 0;
            CK(go(k_fused, s->fuse_ntiles, kBlock, 0, st, t, fa));
            TRY(mark());
        }
    }
    for (int32_t l = r - 1; l >= head; --l) {
        if constexpr (!det) {
            if (l >= 1 && pair_at(s, l - 1, head)) {     // the bottom-up steps of depths l and l - 1
                TRY(launch_pair(go, s, t, st, true, 0));
                TRY(mark());
                --l;
                continue;
            }
        }
        const int32_t j0 = s->dlevel[l], j1 = s->dlevel[l + 1];
        bool streamed = false;
        if constexpr (!det) {
            if (j1 - j0 >= kStreamMinNodes) streamed = launch_stream(go, s, t, st, true, l, j0, j1, first);
        }
        if (!streamed) CK(go(k_bottomup<real, det>, nblocks(j1 - j0), kBlock, 0, st, t, j0, j1));
        CK_LAUNCH();
        const int32_t nw = s->wlevel[l + 1] - s->wlevel[l];
        if (!det && nw > 0) CK(go(k_bottomup_wide<real>, nw, kWideBlock, 0, st, t, (const int32_t *)s->wide, s->wlevel[l]));
        TRY(mark());
    }
    if constexpr (!det) {
        if (split) TRY(deep_update());
        if (head > 0) {
            const HeadArgs ha = head_args(s, false);
            auto k = s->head_na == 0 ? k_head_bottomup<kStreamNA[0]>
                   : s->head_na == 1 ? k_head_bottomup<kStreamNA[1]> : k_head_bottomup<kStreamNA[2]>;
            CK(go(k, ha.nblk, kHeadThreads, head_smem_bottomup(ha.cap), st, t, ha));
        }
    }
    if (branch) {
        CK(cudaStreamWaitEvent(st, s->join[pi], 0));
        go.cut(st);
    }
    if (first && variant == CFR_DISCOUNTED && !split)
        CK(go(k_weights, 1, 1, 0, st, (const int64_t *)s->d_iter, s->wts, s->cfg.dcfr_alpha, s->cfg.dcfr_beta,
              s->cfg.dcfr_gamma));
    if constexpr (det) {
        if (s->Hp > 0) CK(go(k_update<real, det>, nblocks(s->Hp), kBlock, 0, st, t, s->Hp, variant, linear));
    } else {
        go.prio = 0;
        TRY(launch_update_any(go, s, t, st, linear, 0, split ? hsplit : s->Hp, true));
        if (split) {
            CK(cudaStreamWaitEvent(st, s->upd[pi], 0));
            go.cut(st);
        }
    }
    TRY(mark());
    return CFR_OK;
}

// One full-tree iteration: one pass over both players (simultaneous updates), or a pass for player 1
// and then one for player 2 under player 1's new strategy (alternating updates); the phase events
// (ev) are for simultaneous updates only.
template <typename real>
cfr_status enqueue_iteration(cfr_solver *s, cudaStream_t st, cudaEvent_t *ev = nullptr) {
    if (s->cfg.update_mode != CFR_ALTERNATING) return enqueue_pass<real>(s, st, ev, 6, true);
    TRY(enqueue_pass<real>(s, st, nullptr, 2, true));
    return enqueue_pass<real>(s, st, nullptr, 4, false);
}

// First fused depth (L when nothing is fused).
int32_t fused_from(const cfr_solver *s) { return s->cfg.precision == CFR_FP64 ? s->L : s->fuse_r; }

// Phases of one iteration, in the order of enqueue_iteration's events: kind (CFR_PHASE_*) and depth.
std::vector<std::pair<int32_t, int32_t>> phases(const cfr_solver *s) {
    std::vector<std::pair<int32_t, int32_t>> p;
    if (s->L == 0) return p;
    const int32_t r = fused_from(s);
    if (s->Hp > 0) p.push_back({CFR_PHASE_OWN, -1});
    for (int32_t l = 0; l < r; ++l) {
        if (r < s->L && pair_at(s, l, 0)) {
            p.push_back({CFR_PHASE_TOPDOWN_PAIR, l++});
            continue;
        }
        if (topdown_launches(s, l)) p.push_back({CFR_PHASE_TOPDOWN, l});
    }
    if (r < s->L) p.push_back({CFR_PHASE_FUSED, r});
    for (int32_t l = r - 1; l >= 0; --l) {
        if (r < s->L && l >= 1 && pair_at(s, l - 1, 0)) {
            p.push_back({CFR_PHASE_BOTTOMUP_PAIR, --l});
            continue;
        }
        p.push_back({CFR_PHASE_BOTTOMUP, l});
    }
    p.push_back({CFR_PHASE_UPDATE, -1});
    return p;
}

// Algorithmic bytes of each phase, in the order of phases() (FP32 mode; FP64 mode doubles the value
// bytes: 17 Hp, 32 Nd(l) + 16 Nd(l+1), 40 Nd(l) + 8 C(l), 56 Q):
//   own reaches:            13 Hp                  pseq, pseq_h, player read, own written
//   top-down from depth l:  20 Nd(l) + 8 Nd(l+1)   node fields and reaches read, child reaches written
//   bottom-up at depth l:   24 Nd(l) + 4 C(l)      node fields, reach, value write; one value per child
//   last two depths (k_tail, r = L-2):
//                           28 Nd(r) + 12 Nd(r+1)  node fields and reaches of depth r, value written;
//                                                  node fields of depth r+1 (k_tail_slots: 4 Nd(r+1),
//                                                  the packed word alone)
//                         + 4 T(r) + 4 T(r+1)      one utility per terminal child
//   depths m, m+1 paired (k_pair_topdown, k_pair_bottomup; m = r-2 below the fused tail):
//     top-down              20 Nd(m) + 12 Nd(m+1)  fields and reaches of depth m, fields of depth m+1
//                         + 8 Nd(m+2)             the reaches of depth m+2 written
//     bottom-up             28 Nd(m) + 16 Nd(m+1)  as k_tail's, with the children's first decision child
//                         + 4 T(m) + 4 T(m+1)     one utility per terminal child
//                         + 4 Nd(m+2)             one value per decision grandchild
//   fused depths r..L-1 (k_fused tiles):
//                           16 Nd(>=r) + 4 T(>=r)  node fields; one utility per terminal child
//                         + 12 Nd(r)               the tile roots' reaches read and values written
//   update:                 44 Q                   r~ read and zeroed, R and S read+written, sigma written
// With nothing fused they add up to 56 Nd + 4 Nt + 44 Q + 13 Hp - 12 - 20 Nd(L-1) (96 Nd + 8 Nt + 56 Q
// + 17 Hp - 24 - 32 Nd(L-1) in FP64 mode): every node but the root is a child once, and the last depth
// has no top-down step (topdown_launches).  Hp counts the player infosets, C(l) all children of depth
// l's nodes, T(l) their terminal children.
std::vector<double> phase_bytes(const cfr_solver *s) {
    const bool f64 = s->cfg.precision == CFR_FP64;
    std::vector<double> b;
    auto nd = [&](int32_t l) -> double { return l < s->L ? (double)(s->dlevel[l + 1] - s->dlevel[l]) : 0.0; };
    for (const auto &ph : phases(s)) {
        const int32_t l = ph.second;
        if (ph.first == CFR_PHASE_OWN) {
            b.push_back((f64 ? 17.0 : 13.0) * (double)s->Hp);
        } else if (ph.first == CFR_PHASE_TOPDOWN) {
            b.push_back(f64 ? 32 * nd(l) + 16 * nd(l + 1) : 20 * nd(l) + 8 * nd(l + 1));
        } else if (ph.first == CFR_PHASE_BOTTOMUP) {
            const double children = (double)s->level_children[l];
            b.push_back(f64 ? 40 * nd(l) + 8 * children : 24 * nd(l) + 4 * children);
        } else if (ph.first == CFR_PHASE_TOPDOWN_PAIR) {
            b.push_back(20 * nd(l) + 12 * nd(l + 1) + 8 * nd(l + 2));
        } else if (ph.first == CFR_PHASE_BOTTOMUP_PAIR) {
            b.push_back(28 * nd(l) + 16 * nd(l + 1) + 4 * nd(l + 2) +
                        4 * (double)(s->level_terminals[l] + s->level_terminals[l + 1]));
        } else if (ph.first == CFR_PHASE_FUSED && s->fuse_tail) {
            b.push_back(28 * nd(l) + (s->tail_slots ? 4 : 12) * nd(l + 1) +
                        4 * (double)(s->level_terminals[l] + s->level_terminals[l + 1]));
        } else if (ph.first == CFR_PHASE_FUSED) {
            double x = 12 * nd(l);
            for (int32_t k = l; k < s->L; ++k) x += 16 * nd(k) + 4 * (double)s->level_terminals[k];
            b.push_back(x);
        } else {
            b.push_back((f64 ? 56.0 : 44.0) * (double)s->Q);
        }
    }
    return b;
}

// Kernel launches of one iteration (for cfr_info and the benchmark's launch count).
int32_t launches_per_pass(const cfr_solver *s);
int32_t launches_per_iteration(const cfr_solver *s) {
    if (s->L == 0) return 0;
    const bool alt = s->cfg.update_mode == CFR_ALTERNATING;
    const int32_t zero = alt && s->cfg.precision == CFR_FP32 && s->Hp > 0;   // k_zero_inst per pass
    return (alt ? 2 * (launches_per_pass(s) + zero) : launches_per_pass(s)) + (s->cfg.variant == CFR_DISCOUNTED);
}

int32_t launches_per_pass(const cfr_solver *s) {
    const bool det = s->cfg.precision == CFR_FP64;
    const int32_t r = fused_from(s);
    const int32_t head = det ? 0 : s->head_n;
    int32_t n = (r - head) + 1 + (r < s->L);                  // bottom-up depths, fused, update
    for (int32_t l = head; l < s->L; ++l) n += s->hlevel[l + 1] > s->hlevel[l];   // own reaches
    if (head > 0) n += 2;                                     // the head's two launches
    if (head > 0 && s->cfg.update_mode != CFR_ALTERNATING && s->hlevel[(size_t)head] > 0 &&
        s->hlevel[(size_t)head] < s->Hp)
        n += 1;                                               // the update split in two (enqueue_pass)
    for (int32_t l = head; l < r; ++l) {
        n += s->ddepth_children[l] || l == 0;                 // top-down
        if (!det) n += 2 * (s->wlevel[l + 1] > s->wlevel[l]);
    }
    if (!det && r < s->L && s->pair_m >= head && s->npair_tiles > 0) n -= 2;   // two depths per launch
    return n;
}

// FP32 mode: the leading depths run by k_head_topdown / k_head_bottomup: depths 0 .. n (head_n = n + 1)
// for a single root whose children are all decision nodes, or for a forest whose roots have at most 32
// actions, n >= 1 the deepest depth below the fused ones
// such that every depth 1 .. n holds at most kHeadMaxNodes nodes and no node of more than 32 actions,
// and the largest block's nodes of depths 1 .. n fit kHeadMaxSmem bytes of shared memory (at most
// cfg.head_levels depths below the root when that is positive; 0: none).  About two blocks per SM walk
// the root children's subtrees.
// Tiles of the depth-m parents [jb, je) for k_pair_topdown / k_pair_bottomup: consecutive parents while
// every staged range (their decision children, both terminal ranges, the decision grandchildren) fits
// its array, 4 elements of each kept free for the 16-byte widening of the copies.  Appends 12 words per
// tile: {j0, j1, cs, ce}, {pts, pte, cts, cte}, {gs, ge, 0, 0}.  False if one parent alone exceeds a range.
bool cut_pair_tiles(const Layout &Lo, int32_t jb, int32_t je, std::vector<int32_t> *meta) {
    const auto df = [&](int32_t j) { return Lo.dfirst[(size_t)j]; };
    const auto tf = [&](int32_t j) { return Lo.tfirst[(size_t)j]; };
    std::vector<int32_t> tb{jb};
    int32_t n = 0, nc = 0, npt = 0, nct = 0, ng = 0;
    for (int32_t j = jb; j < je; ++j) {
        const int32_t d0 = df(j), d1 = df(j + 1);
        const int32_t ndj = d1 - d0, ptj = tf(j + 1) - tf(j), ctj = tf(d1) - tf(d0), gj = df(d1) - df(d0);
        if (ndj > kPC - 4 || ptj > kPPT - 4 || ctj > kPCT - 4 || gj > kPG - 4) return false;
        if (n + 1 > kPP || nc + ndj > kPC - 4 || npt + ptj > kPPT - 4 || nct + ctj > kPCT - 4 || ng + gj > kPG - 4) {
            tb.push_back(j);
            n = nc = npt = nct = ng = 0;
        }
        ++n; nc += ndj; npt += ptj; nct += ctj; ng += gj;
    }
    tb.push_back(je);
    meta->clear();
    meta->reserve((size_t)12 * (tb.size() - 1));
    for (size_t i = 0; i + 1 < tb.size(); ++i) {
        const int32_t j0 = tb[i], j1 = tb[i + 1], cs = df(j0), ce = df(j1);
        const int32_t v[12] = {j0, j1, cs, ce, tf(j0), tf(j1), tf(cs), tf(ce), df(cs), df(ce), 0, 0};
        meta->insert(meta->end(), v, v + 12);
    }
    return true;
}

// FP32 mode with automatic fusion, after plan_fusion and plan_head: the two depths m = fuse_r - 2 and
// m + 1 above the streamed tail run as a pair (one top-down and one bottom-up launch) when both lie below
// the head, hold decision children and no node of more than 32 actions, and depth m holds at least
// kPairMinNodes decision nodes.
cfr_status plan_pair(cfr_solver *s, const Layout &Lo) {
    s->pair_m = -1;
    s->npair_tiles = 0;
    if (s->cfg.fuse_levels >= 0 || !s->fuse_tail || s->ntail_tiles == 0) return CFR_OK;
    const int32_t m = s->fuse_r - 2;
    if (m < 0 || m < s->head_n || s->dlevel[m + 1] - s->dlevel[m] < kPairMinNodes) return CFR_OK;
    if (s->wlevel[(size_t)m + 2] > s->wlevel[(size_t)m] || !s->ddepth_children[m] || !s->ddepth_children[m + 1])
        return CFR_OK;
    std::vector<int32_t> meta;
    if (!cut_pair_tiles(Lo, s->dlevel[m], s->dlevel[m + 1], &meta)) return CFR_OK;
    TRY(alloc_n(s, &s->pair_tiles, (int64_t)meta.size()));
    TRY(upload(s, s->pair_tiles, meta));
    CK(cudaStreamSynchronize(s->stream));
    s->npair_tiles = (int32_t)(meta.size() / 12);
    s->pair_m = m;
    return CFR_OK;
}

cfr_status plan_head(cfr_solver *s, const Layout &Lo, int sms) {
    s->head_n = 0;
    if (s->cfg.head_levels == 0 || s->L < 2) return CFR_OK;
    const bool forest = s->dlevel[1] > 1;
    // the nodes blocks take ranges of: the roots of a forest (none of more than 32 actions), else the root's
    // children (all decision nodes)
    const int32_t first = forest ? 0 : 1;
    const int32_t nroot = forest ? s->dlevel[1] : s->dlevel[2] - s->dlevel[1];
    if (forest ? s->wlevel[1] > s->wlevel[0] : (nroot < 1 || s->level_children[0] != nroot)) return CFR_OK;
    const int32_t r = fused_from(s);
    const int32_t cap = s->cfg.head_levels < 0 ? kHeadMaxDepths : std::min(s->cfg.head_levels, (int32_t)kHeadMaxDepths);
    int32_t n = 0;
    while (n + 1 <= cap && n + 1 < r && n + 1 < s->L && s->dlevel[(size_t)n + 2] - s->dlevel[(size_t)n + 1] <= kHeadMaxNodes &&
           s->wlevel[(size_t)n + 2] == s->wlevel[(size_t)n + 1])
        ++n;
    const int32_t nblk = std::min(nroot, kHeadBlocksPerSM * std::max(sms, 1));
    const int32_t per = (nroot + nblk - 1) / nblk;
    // the largest block's nodes of depths 1 .. n, as head_ranges cuts them; fewer depths until they fit
    int32_t most = 0;
    for (; n >= 1; --n) {
        most = 0;
        for (int32_t lo1 = s->dlevel[(size_t)first]; lo1 < s->dlevel[(size_t)first] + nroot; lo1 += per) {
            int32_t lo = lo1, hi = std::min(lo1 + per, s->dlevel[(size_t)first] + nroot), tot = 0;
            for (int32_t l = first; l <= n; ++l) {
                tot += hi - lo;
                lo = Lo.dfirst[(size_t)lo];
                hi = Lo.dfirst[(size_t)hi];
            }
            most = std::max(most, tot);
        }
        if (head_smem_bottomup(most) <= (size_t)kHeadMaxSmem && head_smem_topdown(most) <= (size_t)kHeadMaxSmem) break;
    }
    if (n < 1) return CFR_OK;
    for (const void *k : {(const void *)k_head_topdown<kStreamNA[0]>, (const void *)k_head_bottomup<kStreamNA[0]>,
                          (const void *)k_head_topdown<kStreamNA[1]>, (const void *)k_head_bottomup<kStreamNA[1]>,
                          (const void *)k_head_topdown<kStreamNA[2]>, (const void *)k_head_bottomup<kStreamNA[2]>})
        CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kHeadMaxSmem));
    if (!s->head_done) {
        TRY(alloc_n(s, &s->head_done, 1));
        CK(cudaMemsetAsync(s->head_done, 0, sizeof(int32_t), s->stream));
    }
    // each block's node ranges per depth (head_ranges in kernels.cuh): lo, hi and shared-memory offsets
    {
        constexpr int K = kHeadMaxDepths + 2;
        const int32_t d1 = s->dlevel[(size_t)first];
        const int32_t nblocks_head = (nroot + per - 1) / per;
        std::vector<int32_t> rng((size_t)nblocks_head * kHeadRangeWords, 0);
        for (int32_t b = 0; b < nblocks_head; ++b) {
            int32_t *lo = rng.data() + (size_t)b * kHeadRangeWords, *hi = lo + K, *off = hi + K;
            lo[first] = d1 + b * per;
            hi[first] = std::min(lo[first] + per, d1 + nroot);
            off[first] = 0;
            for (int32_t l = first; l <= n; ++l) {
                lo[l + 1] = Lo.dfirst[(size_t)lo[l]];
                hi[l + 1] = Lo.dfirst[(size_t)hi[l]];
                off[l + 1] = off[l] + (hi[l] - lo[l]);
            }
        }
        TRY(alloc_n(s, &s->head_rng, (int64_t)rng.size()));
        TRY(upload(s, s->head_rng, rng));
        CK(cudaStreamSynchronize(s->stream));
    }
    s->head_n = n + 1;
    s->head_per_block = per;
    s->head_cap = std::max(most, 1);
    s->head_na = 0;
    for (int32_t l = first; l <= n; ++l) s->head_na = std::max(s->head_na, s->level_na[(size_t)l]);
    return CFR_OK;
}

cfr_status build_graph(cfr_solver *s) {
    if (s->L == 0) return CFR_OK;
    CK(cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal));
    cfr_status st = s->cfg.precision == CFR_FP64 ? enqueue_iteration<double>(s, s->cap)
                                                 : enqueue_iteration<float>(s, s->cap);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s->cap, &g);
    if (st != CFR_OK) { if (g) cudaGraphDestroy(g); return st; }
    if (e != cudaSuccess) { s->poisoned = true; return set_err(s, CFR_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e)); }
    s->graph = g;
    CK(cudaGraphInstantiate(&s->graph_exec, g, 0));
    CK(cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < kGraphIters && st == CFR_OK; ++i)
        st = s->cfg.precision == CFR_FP64 ? enqueue_iteration<double>(s, s->cap) : enqueue_iteration<float>(s, s->cap);
    g = nullptr;
    e = cudaStreamEndCapture(s->cap, &g);
    if (st != CFR_OK) { if (g) cudaGraphDestroy(g); return st; }
    if (e != cudaSuccess) { s->poisoned = true; return set_err(s, CFR_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e)); }
    s->graph2 = g;
    CK(cudaGraphInstantiate(&s->graph_exec2, g, 0));
    return CFR_OK;
}

template <typename real>
void regret_match_all(cfr_solver *s) {
    k_regret_match_all<real><<<nblocks(s->H), kBlock, 0, s->stream>>>(static_cast<real *>(s->sigma), s->R, s->qbase,
                                                                        s->iplayer, s->H);
}

cfr_status check_usable(cfr_solver *s) {
    if (!s) return set_err(nullptr, CFR_ERR_INVALID, "solver is NULL");
    if (s->poisoned) return set_err(s, CFR_ERR_STATE, "solver is unusable after an earlier CUDA error: %s", s->err.c_str());
    return CFR_OK;
}

// Waits for the solver's stream; a device-side wait that expired poisons the solver.
cfr_status sync_and_check(cfr_solver *s) {
    CK(cudaStreamSynchronize(s->stream));
    if (s->d_err) {
        int e = 0;
        CK(cudaMemcpy(&e, s->d_err, sizeof e, cudaMemcpyDeviceToHost));
        if (e) {
            s->poisoned = true;
            return set_err(s, CFR_ERR_TIMEOUT, "a bounded device-side wait expired (TMA copy not completed)");
        }
    }
    return CFR_OK;
}

// k_tail_slots' tiles (cut_slot_tail_tiles) uploaded for depth r; false (nothing set) where the tree's
// tiles are not slot-dense.
bool slot_tail_tiles(cfr_solver *s, const Layout &Lo, int32_t r) {
    std::vector<int32_t> meta;
    if (!cut_slot_tail_tiles(Lo, s->dlevel[r], s->dlevel[r + 1], &meta)) return false;
    if (alloc_n(s, &s->tail_tiles, (int64_t)meta.size()) != CFR_OK || upload(s, s->tail_tiles, meta) != CFR_OK ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return false;
    s->ntail_tiles = (int32_t)(meta.size() / 12);
    s->tail_slots = true;
    return true;
}

// FP32 mode: picks the fused depths r .. L-1 and cuts them into tiles for k_fused.  At most
// cfg.fuse_levels depths (kFuseAuto when negative; none below 2) are fused, fewer where a depth-r
// node's decision subtree exceeds kFuseCap or a depth >= r holds a node with more than 32 actions.
// Tiles take consecutive depth-r nodes while their subtrees fit kFuseCap together.
cfr_status plan_fusion(cfr_solver *s, const Layout &Lo) {
    s->fuse_r = s->L;
    s->fuse_ntiles = 0;
    int32_t want = s->cfg.fuse_levels < 0 ? kFuseAuto : s->cfg.fuse_levels;
    want = std::min(std::min(want, (int32_t)kFuseMaxLevels), s->L);
    if (want < 2) return CFR_OK;
    int32_t wdeep = -1;                                        // deepest depth holding a wide node
    for (int32_t l = 0; l < s->L; ++l)
        if (s->wlevel[l + 1] > s->wlevel[l]) wdeep = l;
    const int32_t rmin = std::max(s->L - want, wdeep + 1);
    if (s->L - rmin < 2) return CFR_OK;
    if (want == 2) {                                           // the last two depths in one pass
        const int32_t r = s->L - 2;
        s->fuse_r = r;
        s->fuse_tail = true;
        if (s->dlevel[r + 1] - s->dlevel[r] >= kStreamMinNodes && s->cfg.tail_slots > 0 && slot_tail_tiles(s, Lo, r))
            return CFR_OK;
        if (s->dlevel[r + 1] - s->dlevel[r] >= kStreamMinNodes) {
            // tiles for k_tail_stream: consecutive parents while every staged range fits its array
            // (4 elements of each kept free for the 16-byte widening of the copies)
            std::vector<int32_t> tb{s->dlevel[r]};
            int32_t n = 0, nc = 0, npt = 0, nct = 0;
            for (int32_t j = s->dlevel[r]; j < s->dlevel[r + 1]; ++j) {
                const int32_t d0 = Lo.dfirst[(size_t)j], d1 = Lo.dfirst[(size_t)j + 1];
                const int32_t ndj = d1 - d0, ptj = Lo.tfirst[(size_t)j + 1] - Lo.tfirst[(size_t)j];
                const int32_t ctj = Lo.tfirst[(size_t)d1] - Lo.tfirst[(size_t)d0];
                if (n + 1 > kTP || nc + ndj > kTC - 4 || npt + ptj > kTPT - 4 || nct + ctj > kTCT - 4) {
                    tb.push_back(j);
                    n = nc = npt = nct = 0;
                }
                ++n; nc += ndj; npt += ptj; nct += ctj;
            }
            tb.push_back(s->dlevel[r + 1]);
            s->ntail_tiles = (int32_t)tb.size() - 1;
            // per tile: {j0, j1, cs, ce}, {pts, pte, cts, cte} (k_tail_stream's TailTiles::tm)
            std::vector<int32_t> meta;
            meta.reserve((size_t)8 * s->ntail_tiles);
            for (int32_t i = 0; i < s->ntail_tiles; ++i) {
                const int32_t j0 = tb[(size_t)i], j1 = tb[(size_t)i + 1];
                const int32_t cs = Lo.dfirst[(size_t)j0], ce = Lo.dfirst[(size_t)j1];
                const int32_t v[8] = {j0, j1, cs, ce, Lo.tfirst[(size_t)j0], Lo.tfirst[(size_t)j1], Lo.tfirst[(size_t)cs],
                                      Lo.tfirst[(size_t)ce]};
                meta.insert(meta.end(), v, v + 8);
            }
            TRY(alloc_n(s, &s->tail_tiles, (int64_t)meta.size()));
            TRY(upload(s, s->tail_tiles, meta));
            CK(cudaStreamSynchronize(s->stream));
        }
        return CFR_OK;
    }
    // decision nodes in the subtree of each node of depth >= rmin (children have larger ids)
    const int32_t jmin = s->dlevel[rmin];
    std::vector<int32_t> cnt((size_t)(s->Nd - jmin), 0);
    for (int64_t j = s->Nd - 1; j >= jmin; --j) {
        int64_t c = 1;
        for (int32_t d = Lo.dfirst[j]; d < Lo.dfirst[j + 1]; ++d) c += cnt[(size_t)(d - jmin)];
        cnt[(size_t)(j - jmin)] = (int32_t)std::min<int64_t>(c, INT32_MAX);
    }
    int32_t r = rmin;
    for (; s->L - r >= 2; ++r) {
        bool fits = true;
        for (int32_t j = s->dlevel[r]; j < s->dlevel[r + 1] && fits; ++j) fits = cnt[(size_t)(j - jmin)] <= kFuseCap;
        if (fits) break;
    }
    if (s->L - r < 2) return CFR_OK;
    std::vector<int32_t> roots;
    int64_t acc = 0;
    for (int32_t j = s->dlevel[r]; j < s->dlevel[r + 1]; ++j) {
        const int32_t c = cnt[(size_t)(j - jmin)];
        if (roots.empty() || acc + c > kFuseCap) { roots.push_back(j); acc = 0; }
        acc += c;
    }
    roots.push_back(s->dlevel[r + 1]);
    const int32_t K = s->L - r, nt = (int32_t)roots.size() - 1;
    std::vector<int32_t> bounds((size_t)K * (nt + 1));
    for (int32_t i = 0; i <= nt; ++i) {
        int32_t j = roots[(size_t)i];
        for (int32_t k = 0; k < K; ++k) {
            bounds[(size_t)k * (nt + 1) + i] = j;
            j = Lo.dfirst[(size_t)j];
        }
    }
    TRY(alloc_n(s, &s->fuse_bounds, (int64_t)bounds.size()));
    TRY(upload(s, s->fuse_bounds, bounds));
    CK(cudaStreamSynchronize(s->stream));
    s->fuse_r = r;
    s->fuse_ntiles = nt;
    return CFR_OK;
}

cfr_status load(cfr_solver *s, Layout &Lo) {
    s->N = Lo.N; s->Nd = Lo.Nd; s->Nt = Lo.Nt; s->Q = Lo.Q; s->H = Lo.H; s->L = Lo.L;
    s->max_depth = Lo.max_depth; s->max_actions = Lo.max_actions; s->single_level = Lo.single_level;
    s->dlevel = Lo.dlevel; s->hlevel = Lo.hlevel; s->wlevel = Lo.wlevel; s->Hp = Lo.Hp;
    s->ddepth_children.assign((size_t)s->L, 0);
    s->level_children.assign((size_t)s->L, 0);
    s->level_terminals.assign((size_t)s->L, 0);
    for (int32_t l = 0; l < s->L; ++l) {
        const size_t a = (size_t)s->dlevel[l], b = (size_t)s->dlevel[l + 1];
        s->ddepth_children[l] = Lo.dfirst[b] > Lo.dfirst[a];
        s->level_children[l] = (int64_t)(Lo.dfirst[b] - Lo.dfirst[a]) + (Lo.tfirst[b] - Lo.tfirst[a]);
        s->level_terminals[l] = (int64_t)(Lo.tfirst[b] - Lo.tfirst[a]);
    }
    s->dnode_user.swap(Lo.dnode_user); s->tnode_user.swap(Lo.tnode_user); s->h_int2user.swap(Lo.h_int2user);
    const bool fp64 = s->cfg.precision == CFR_FP64;
    const size_t rs = s->real_size();

    TRY(alloc_n(s, &s->dfirst, s->Nd + 1));
    TRY(alloc_n(s, &s->tfirst, s->Nd + 1));
    TRY(alloc_n(s, &s->dinfo, s->Nd));
    TRY(alloc_n(s, &s->kmask, s->Nd));
    TRY(alloc_n(s, &s->qp, s->Nd));
    TRY(alloc_n(s, &s->wbits, (int64_t)Lo.wbits.size()));
    TRY(alloc_n(s, &s->sigma064, s->Q));
    TRY(alloc_n(s, &s->util64, s->Nt));
    if (fp64) s->util = s->util64;
    else TRY(dev_alloc(s, &s->util, rs * (size_t)std::max<int64_t>(s->Nt, 1)));
    TRY(alloc_n(s, &s->qbase, (int64_t)s->H + 1));
    TRY(alloc_n(s, &s->iplayer, s->H));
    TRY(alloc_n(s, &s->pseq, s->H));
    TRY(alloc_n(s, &s->pseq_h, s->H));
    TRY(alloc_n(s, &s->q_int2user, s->Q));
    TRY(dev_alloc(s, &s->sigma, rs * (size_t)std::max<int64_t>(s->Q, 1)));
    TRY(dev_alloc(s, &s->inst, rs * (size_t)std::max<int64_t>(s->Q, 1)));
    TRY(dev_alloc(s, &s->reach1, rs * (size_t)std::max<int64_t>(s->Nd, 1)));
    TRY(dev_alloc(s, &s->reach2, rs * (size_t)std::max<int64_t>(s->Nd, 1)));
    TRY(dev_alloc(s, &s->u, rs * (size_t)std::max<int64_t>(s->Nd, 1)));
    TRY(dev_alloc(s, &s->own, rs * (size_t)std::max<int32_t>(s->H, 1)));
    TRY(alloc_n(s, &s->R, s->Q));
    TRY(alloc_n(s, &s->S, s->Q));
    TRY(alloc_n(s, &s->stage, s->Q));
    TRY(alloc_n(s, &s->d_iter, 1));
    TRY(alloc_n(s, &s->d_err, 1));
    TRY(alloc_n(s, &s->wts, 4));
    if (fp64) {
        TRY(dev_alloc(s, &s->contrib, sizeof(double) * (size_t)std::max<int64_t>(s->N - 1, 1)));
        TRY(alloc_n(s, &s->hnode_start, (int64_t)s->H + 1));
        TRY(alloc_n(s, &s->hnode, s->Nd));
        TRY(upload(s, s->hnode_start, Lo.hnode_start));
        TRY(upload(s, s->hnode, Lo.hnode));
    }
    TRY(alloc_n(s, &s->wide, (int64_t)Lo.wide.size()));
    TRY(upload(s, s->wide, Lo.wide));
    if (!fp64) {
        // per depth, the smallest unrolled action count covering its largest node of at most 32 actions
        s->level_na.assign((size_t)s->L, 2);
        for (int32_t l = 0; l < s->L; ++l) {
            int32_t maxa = 0;
            for (int32_t j = s->dlevel[l]; j < s->dlevel[l + 1]; ++j) {
                if ((Lo.qp[(size_t)j] >> 29) & 1u) continue;
                maxa = std::max<int32_t>(maxa, (Lo.dfirst[(size_t)j + 1] - Lo.dfirst[j]) + __builtin_popcount(Lo.kmask[j]));
            }
            s->level_na[(size_t)l] = maxa <= kStreamNA[0] ? 0 : maxa <= kStreamNA[1] ? 1 : 2;
        }
        TRY(plan_fusion(s, Lo));
        int sms = 0;
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device));
        TRY(plan_head(s, Lo, sms));
        TRY(plan_pair(s, Lo));
        {
            std::vector<int32_t> wh;
            for (int32_t h = 0; h < s->Hp; ++h) {
                const int32_t na = Lo.qbase[(size_t)h + 1] - Lo.qbase[h];
                if (na > 32) wh.push_back(h); else s->hp_na = std::max(s->hp_na, na);
            }
            s->nwide_h = (int32_t)wh.size();
            TRY(alloc_n(s, &s->wide_h, (int64_t)wh.size()));
            TRY(upload(s, s->wide_h, wh));
            CK(cudaStreamSynchronize(s->stream));
        }
    }

    TRY(upload(s, s->dfirst, Lo.dfirst));
    TRY(upload(s, s->tfirst, Lo.tfirst));
    TRY(upload(s, s->dinfo, Lo.dinfo));
    TRY(upload(s, s->kmask, Lo.kmask));
    TRY(upload(s, s->qp, Lo.qp));
    TRY(upload(s, s->wbits, Lo.wbits));
    TRY(upload(s, s->sigma064, Lo.sigma0));
    TRY(upload(s, s->util64, Lo.util));
    std::vector<float> tmpf;
    if (!fp64) {
        tmpf.assign(Lo.util.begin(), Lo.util.end());
        CK(cudaMemcpyAsync(s->util, tmpf.data(), sizeof(float) * tmpf.size(), cudaMemcpyHostToDevice, s->stream));
    }
    TRY(upload(s, s->qbase, Lo.qbase));
    TRY(upload(s, s->iplayer, Lo.iplayer));
    TRY(upload(s, s->pseq, Lo.pseq));
    TRY(upload(s, s->pseq_h, Lo.pseq_h));
    TRY(upload(s, s->q_int2user, Lo.q_int2user));
    // sigma_0 at chance slots, zero elsewhere; then regret matching of R = 0 gives sigma^(1).
    if (fp64) {
        TRY(upload(s, static_cast<double *>(s->sigma), Lo.sigma0));
    } else {
        std::vector<float> s0(Lo.sigma0.begin(), Lo.sigma0.end());
        CK(cudaMemcpyAsync(s->sigma, s0.data(), sizeof(float) * s0.size(), cudaMemcpyHostToDevice, s->stream));
        CK(cudaStreamSynchronize(s->stream));
    }
    CK(cudaMemsetAsync(s->inst, 0, rs * (size_t)std::max<int64_t>(s->Q, 1), s->stream));
    CK(cudaMemsetAsync(s->R, 0, sizeof(double) * (size_t)std::max<int64_t>(s->Q, 1), s->stream));
    CK(cudaMemsetAsync(s->S, 0, sizeof(double) * (size_t)std::max<int64_t>(s->Q, 1), s->stream));
    CK(cudaMemsetAsync(s->own, 0, rs * (size_t)std::max<int32_t>(s->H, 1), s->stream));
    CK(cudaMemsetAsync(s->u, 0, rs * (size_t)std::max<int64_t>(s->Nd, 1), s->stream));
    CK(cudaMemsetAsync(s->d_iter, 0, sizeof(int64_t), s->stream));
    CK(cudaMemsetAsync(s->d_err, 0, sizeof(int), s->stream));
    if (!fp64) {
        int sms = 0;
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device));
        TRY(setup_stream_na<kStreamNA[0]>(s, 0, sms));
        TRY(setup_stream_na<kStreamNA[1]>(s, 1, sms));
        TRY(setup_stream_na<kStreamNA[2]>(s, 2, sms));
    }
    // The root's counterfactual reaches are 1 (Eq. 2, v = v_0) and never change (every root's, for a
    // forest of independent games).
    if (s->Nd > 0) {
        const size_t nroots = (size_t)s->dlevel[1];
        std::vector<double> one64(nroots, 1.0);
        std::vector<float> one32(nroots, 1.0f);
        const void *one = fp64 ? (const void *)one64.data() : (const void *)one32.data();
        CK(cudaMemcpyAsync(s->reach1, one, rs * nroots, cudaMemcpyHostToDevice, s->stream));
        CK(cudaMemcpyAsync(s->reach2, one, rs * nroots, cudaMemcpyHostToDevice, s->stream));
        CK(cudaStreamSynchronize(s->stream));
    }
    if (s->H > 0) {
        if (fp64) regret_match_all<double>(s); else regret_match_all<float>(s);
        CK_LAUNCH();
    }
    CK(cudaStreamSynchronize(s->stream));
    return build_graph(s);
}

int64_t bytes_model(const cfr_solver *s) {
    double b = 0;
    for (double x : phase_bytes(s)) b += x;
    if (s->cfg.update_mode == CFR_ALTERNATING) b *= 2;       // two passes (the zeroing of r~ aside)
    return (int64_t)b;
}

template <typename T>
cfr_status gather_q_to_host(cfr_solver *s, const T *src, double *out) {
    if (s->Q == 0) return CFR_OK;
    k_gather_q<T><<<nblocks(s->Q), kBlock, 0, s->stream>>>(src, s->q_int2user, s->stage, (int32_t)s->Q);
    CK_LAUNCH();
    CK(cudaMemcpyAsync(out, s->stage, sizeof(double) * (size_t)s->Q, cudaMemcpyDeviceToHost, s->stream));
    return sync_and_check(s);
}

// The average strategy (Eq. 10 normalised) and both players' best responses against it in one pass
// (k_br2_*, one launch per step and depth), captured once into a graph; afterwards br_val[0 .. roots)
// and br_val2[0 .. roots) hold each responder's value at every root.
cfr_status enqueue_best_responses(cfr_solver *s, cudaStream_t st) {
    DevBR b1;
    b1.dfirst = s->dfirst; b1.tfirst = s->tfirst; b1.dinfo = s->dinfo;
    b1.kmask = s->kmask; b1.wbits = s->wbits;
    b1.util = s->util64; b1.qbase = s->qbase; b1.iplayer = s->iplayer; b1.avg = s->avg;
    b1.preach = s->br_reach; b1.val = s->br_val; b1.cfv = s->br_cfv; b1.astar = s->astar;
    DevBR b2 = b1;
    b2.preach = s->br_reach2;
    b2.val = s->br_val2;
    Launcher go;
    go.pdl = false;          // the set-up kernels do not wait on a predecessor: plain ordering
    if (s->H > 0) CK(go(k_average, nblocks(s->H), kBlock, 0, st, (const double *)s->S, (const double *)s->sigma064,
                        (const int32_t *)s->qbase, (const int8_t *)s->iplayer, s->avg, s->H));
    const int32_t nr = s->dlevel[1];
    CK(go(k_fill, nblocks(nr), kBlock, 0, st, s->br_reach, nr, 1.0));
    CK(go(k_fill, nblocks(nr), kBlock, 0, st, s->br_reach2, nr, 1.0));
    CK(cudaMemsetAsync(s->br_cfv, 0, sizeof(double) * (size_t)std::max<int64_t>(s->Q, 1), st));
    go.cut(st);
    go.pdl = true;           // the k_br2_* kernels wait (griddepcontrol.wait) before touching memory
    for (int32_t l = 0; l + 1 < s->L; ++l) {
        const int32_t j0 = s->dlevel[l], j1 = s->dlevel[l + 1];
        CK(go(k_br2_topdown, nblocks(j1 - j0), kBlock, 0, st, b1, b2, j0, j1));
    }
    for (int32_t l = s->L - 1; l >= 0; --l) {
        const int32_t j0 = s->dlevel[l], j1 = s->dlevel[l + 1];
        const int32_t h0 = s->hlevel[l], h1 = s->hlevel[l + 1];
        CK(go(k_br2_nodes, nblocks(j1 - j0), kBlock, 0, st, b1, b2, j0, j1));
        if (h1 > h0) CK(go(k_br2_choose, nblocks(h1 - h0), kBlock, 0, st, b1, b2, h0, h1));
        CK(go(k_br2_pick, nblocks(j1 - j0), kBlock, 0, st, b1, b2, j0, j1));
    }
    return CFR_OK;
}

// Runs the captured best-response pass; the per-root values are then read from br_val / br_val2.
cfr_status best_responses(cfr_solver *s) {
    if (!s->avg) TRY(alloc_n(s, &s->avg, s->Q));
    if (!s->br_reach2) {
        if (!s->br_reach) {
            TRY(alloc_n(s, &s->br_reach, s->Nd));
            TRY(alloc_n(s, &s->br_val, s->Nd));
            TRY(alloc_n(s, &s->br_cfv, s->Q));
            TRY(alloc_n(s, &s->astar, s->H));
        }
        TRY(alloc_n(s, &s->br_reach2, s->Nd));
        TRY(alloc_n(s, &s->br_val2, s->Nd));
        CK(cudaStreamSynchronize(s->stream));
    }
    if (!s->br_exec) {
        CK(cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal));
        const cfr_status st = enqueue_best_responses(s, s->cap);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(s->cap, &g);
        if (st != CFR_OK) { if (g) cudaGraphDestroy(g); return st; }
        if (e != cudaSuccess) { s->poisoned = true; return set_err(s, CFR_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e)); }
        const cudaError_t ie = cudaGraphInstantiate(&s->br_exec, g, 0);
        cudaGraphDestroy(g);
        CK(ie);
    }
    CK(cudaGraphLaunch(s->br_exec, s->stream));
    return CFR_OK;
}

}  // namespace

// ================================================================================================
extern "C" {

void cfr_config_init(cfr_config *c) {
    if (!c) return;
    std::memset(c, 0, sizeof *c);
    c->variant = CFR_VANILLA;
    c->precision = CFR_FP32;
    c->update_mode = CFR_SIMULTANEOUS;
    c->avg_weight = CFR_AVG_DEFAULT;
    c->device = -1;
    c->fuse_levels = -1;
    c->head_levels = -1;
    c->dcfr_alpha = 1.5;
    c->dcfr_beta = 0.0;
    c->dcfr_gamma = 2.0;
    c->batch_split_nodes = 0;
    c->tail_slots = 0;
}

cfr_status cfr_validate(const cfr_game_desc *g, char *msg, size_t msg_len) {
    std::string err;
    cfr_status st = build_layout(g, nullptr, &err);
    if (st != CFR_OK) g_thread_err = err;
    if (msg && msg_len > 0) std::snprintf(msg, msg_len, "%s", st == CFR_OK ? "" : err.c_str());
    return st;
}

cfr_status cfr_load_tree(const cfr_game_desc *g, const cfr_config *c, cfr_solver **out) {
    return cfrgb::load_tree_impl(g, c, false, out);
}

cfr_status cfr_layout_digest(const cfr_game_desc *g, int32_t builder, int32_t forest, uint64_t *digest) {
    if (!digest || (builder != 0 && builder != 1)) return set_err(nullptr, CFR_ERR_INVALID, "digest is NULL or builder not 0/1");
    Layout Lo;
    std::string err;
    const cfr_status st = builder == 0 ? build_layout_serial(g, &Lo, &err, true, forest != 0)
                                       : build_layout_parallel(g, &Lo, &err, true, forest != 0);
    if (st != CFR_OK) {
        g_thread_err = err;
        return st;
    }
    uint64_t h = 1469598103934665603ull;   // FNV-1a over every field, in declaration order
    auto mix = [&](const void *p, size_t bytes) {
        const unsigned char *c = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < bytes; ++i) { h ^= c[i]; h *= 1099511628211ull; }
    };
    auto vec = [&](const auto &v) {
        const uint64_t n = v.size();
        mix(&n, sizeof n);
        if (n) mix(v.data(), sizeof(v[0]) * v.size());
    };
    const int64_t sizes[] = {Lo.N, Lo.Nd, Lo.Nt, Lo.Q, Lo.H, Lo.L, Lo.max_depth, Lo.max_actions, Lo.single_level, Lo.Hp};
    mix(sizes, sizeof sizes);
    vec(Lo.dfirst); vec(Lo.tfirst); vec(Lo.dinfo); vec(Lo.kmask); vec(Lo.wbits); vec(Lo.qp); vec(Lo.dlevel);
    vec(Lo.hlevel); vec(Lo.wide); vec(Lo.wlevel); vec(Lo.util); vec(Lo.qbase); vec(Lo.iplayer); vec(Lo.pseq);
    vec(Lo.pseq_h); vec(Lo.sigma0); vec(Lo.q_int2user); vec(Lo.h_int2user); vec(Lo.dnode_user); vec(Lo.tnode_user);
    vec(Lo.hnode_start); vec(Lo.hnode);
    *digest = h;
    return CFR_OK;
}

}  // extern "C"

// cfr_load_tree, or (forest) several independent games side by side: one root per game at depth 0.
cfr_status cfrgb::load_tree_impl(const cfr_game_desc *g, const cfr_config *c, bool forest, cfr_solver **out) {
    if (!out) return set_err(nullptr, CFR_ERR_INVALID, "out is NULL");
    *out = nullptr;
    cfr_config cfg;
    if (c) cfg = *c; else cfr_config_init(&cfg);
    if (cfg.variant < CFR_VANILLA || cfg.variant > CFR_DISCOUNTED)
        return set_err(nullptr, CFR_ERR_INVALID, "variant %d unknown", cfg.variant);
    if (cfg.variant == CFR_DISCOUNTED &&
        !(std::isfinite(cfg.dcfr_alpha) && std::isfinite(cfg.dcfr_beta) && std::isfinite(cfg.dcfr_gamma)))
        return set_err(nullptr, CFR_ERR_INVALID, "discounted CFR needs finite alpha, beta, gamma");
    if (cfg.precision != CFR_FP32 && cfg.precision != CFR_FP64)
        return set_err(nullptr, CFR_ERR_INVALID, "precision %d unknown", cfg.precision);
    if (cfg.update_mode != CFR_SIMULTANEOUS && cfg.update_mode != CFR_ALTERNATING)
        return set_err(nullptr, CFR_ERR_INVALID, "update_mode %d unknown", cfg.update_mode);
    if (cfg.avg_weight == CFR_AVG_DEFAULT) cfg.avg_weight = cfg.variant == CFR_VANILLA ? CFR_AVG_UNIFORM : CFR_AVG_LINEAR;
    if (cfg.avg_weight != CFR_AVG_UNIFORM && cfg.avg_weight != CFR_AVG_LINEAR)
        return set_err(nullptr, CFR_ERR_INVALID, "avg_weight %d unknown", cfg.avg_weight);
    if ((cfg.dev_alloc == nullptr) != (cfg.dev_free == nullptr))
        return set_err(nullptr, CFR_ERR_INVALID, "dev_alloc and dev_free must both be set or both NULL");

    std::unique_ptr<Layout> Lo(new Layout());
    std::string err;
    cfr_status st = build_layout(g, Lo.get(), &err, cfg.precision == CFR_FP64, forest);
    if (st != CFR_OK) return set_err(nullptr, st, "%s", err.c_str());

    DeviceGuard dg(cfg.device);
    if (!dg.ok) return set_err(nullptr, CFR_ERR_CUDA, "cannot select CUDA device %d", cfg.device);
    std::unique_ptr<cfr_solver> s(new cfr_solver());
    s->cfg = cfg;
    cudaGetDevice(&s->device);
    s->stream = static_cast<cudaStream_t>(cfg.cuda_stream);
    cudaError_t e = cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&s->prio_least, &s->prio_greatest);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = cudaEventCreateWithFlags(&s->fork[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->join[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->deep[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->upd[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        std::string msg = cudaGetErrorString(e);
        cfr_free(s.release());
        return set_err(nullptr, CFR_ERR_CUDA, "stream/event creation: %s", msg.c_str());
    }
    st = load(s.get(), *Lo);
    if (st != CFR_OK) {
        std::string msg = s->err;
        cfr_free(s.release());
        return set_err(nullptr, st, "%s", msg.c_str());
    }
    *out = s.release();
    return CFR_OK;
}

// NashConv of every root's game (a forest; single-depth infosets): both best responses, each root's
// value read after each.  per_root[k] for the k-th decision root (decision nodes of depth 0 in order).
cfr_status cfrgb::root_nash_conv(cfr_solver *s, double *per_root, int32_t n) {
    TRY(check_usable(s));
    if (!s->single_level)
        return set_err(s, CFR_ERR_UNSUPPORTED, "the GPU best response needs every infoset at a single depth");
    if (s->Nd == 0 || n < s->dlevel[1]) return set_err(s, CFR_ERR_INVALID, "need %d root entries", s->Nd ? s->dlevel[1] : 0);
    DeviceGuard dg(s->device);
    const int32_t nr = s->dlevel[1];
    TRY(best_responses(s));
    std::vector<double> v1((size_t)nr), v2((size_t)nr);
    CK(cudaMemcpyAsync(v1.data(), s->br_val, sizeof(double) * nr, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(v2.data(), s->br_val2, sizeof(double) * nr, cudaMemcpyDeviceToHost, s->stream));
    TRY(sync_and_check(s));
    for (int32_t k = 0; k < nr; ++k) per_root[k] = v1[(size_t)k] + v2[(size_t)k];   // zero-sum
    return CFR_OK;
}

extern "C" {

cfr_status cfr_iterate(cfr_solver *s, int32_t n) {
    TRY(check_usable(s));
    if (n < 0) return set_err(s, CFR_ERR_INVALID, "n must be >= 0");
    DeviceGuard dg(s->device);
    for (int32_t i = 0; i < n && s->graph_exec;) {
        const bool many = i + kGraphIters <= n && s->graph_exec2;
        CK(cudaGraphLaunch(many ? s->graph_exec2 : s->graph_exec, s->stream));
        s->kernel_launches += (many ? kGraphIters : 1) * launches_per_iteration(s);
        i += many ? kGraphIters : 1;
    }
    s->iteration += n;
    return CFR_OK;
}

cfr_status cfr_synchronize(cfr_solver *s) {
    TRY(check_usable(s));
    DeviceGuard dg(s->device);
    return sync_and_check(s);
}

cfr_status cfr_average_strategy(cfr_solver *s, double *out, int64_t len) {
    TRY(check_usable(s));
    if (!out || len < s->Q) return set_err(s, CFR_ERR_INVALID, "output needs %lld entries", (long long)s->Q);
    DeviceGuard dg(s->device);
    if (!s->avg) TRY(alloc_n(s, &s->avg, s->Q));
    if (s->H > 0) {
        k_average<<<nblocks(s->H), kBlock, 0, s->stream>>>(s->S, s->sigma064, s->qbase, s->iplayer, s->avg, s->H);
        CK_LAUNCH();
    }
    return gather_q_to_host(s, s->avg, out);
}

cfr_status cfr_current_strategy(cfr_solver *s, double *out, int64_t len) {
    TRY(check_usable(s));
    if (!out || len < s->Q) return set_err(s, CFR_ERR_INVALID, "output needs %lld entries", (long long)s->Q);
    DeviceGuard dg(s->device);
    if (s->cfg.precision == CFR_FP64) return gather_q_to_host(s, static_cast<double *>(s->sigma), out);
    return gather_q_to_host(s, static_cast<float *>(s->sigma), out);
}

cfr_status cfr_exploitability(cfr_solver *s, double *nash_conv, double *exploitability) {
    TRY(check_usable(s));
    if (!s->single_level)
        return set_err(s, CFR_ERR_UNSUPPORTED, "the GPU best response needs every infoset at a single depth");
    DeviceGuard dg(s->device);
    double nc = 0.0;
    if (s->Nd > 0) {
        TRY(best_responses(s));
        double v[2] = {0.0, 0.0};
        CK(cudaMemcpyAsync(&v[0], s->br_val, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
        CK(cudaMemcpyAsync(&v[1], s->br_val2, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
        TRY(sync_and_check(s));
        nc = v[0] + v[1];   // zero-sum: u_1(avg) + u_2(avg) = 0
    }
    if (nash_conv) *nash_conv = nc;
    if (exploitability) *exploitability = nc / 2.0;
    return CFR_OK;
}

cfr_status cfr_get_state(cfr_solver *s, double *cum_regret, double *strat_sum, double *inst_regret, int64_t len_q,
                         double *own_reach, int64_t len_h, int64_t *iteration) {
    TRY(check_usable(s));
    if ((cum_regret || strat_sum || inst_regret) && len_q < s->Q)
        return set_err(s, CFR_ERR_INVALID, "Q buffers need %lld entries", (long long)s->Q);
    if (own_reach && len_h < s->H) return set_err(s, CFR_ERR_INVALID, "own_reach needs %d entries", s->H);
    DeviceGuard dg(s->device);
    if (cum_regret) TRY(gather_q_to_host(s, s->R, cum_regret));
    if (strat_sum) TRY(gather_q_to_host(s, s->S, strat_sum));
    if (inst_regret) {
        if (s->cfg.precision == CFR_FP64) TRY(gather_q_to_host(s, static_cast<double *>(s->inst), inst_regret));
        else TRY(gather_q_to_host(s, static_cast<float *>(s->inst), inst_regret));
    }
    if (own_reach && s->H > 0) {
        std::vector<double> tmp((size_t)s->H);
        CK(cudaStreamSynchronize(s->stream));
        if (s->cfg.precision == CFR_FP64) {
            CK(cudaMemcpy(tmp.data(), s->own, sizeof(double) * s->H, cudaMemcpyDeviceToHost));
        } else {
            std::vector<float> f((size_t)s->H);
            CK(cudaStreamSynchronize(s->stream));
            CK(cudaMemcpy(f.data(), s->own, sizeof(float) * s->H, cudaMemcpyDeviceToHost));
            for (int32_t h = 0; h < s->H; ++h) tmp[h] = f[h];
        }
        for (int32_t h = 0; h < s->H; ++h) own_reach[s->h_int2user[h]] = tmp[h];
    }
    if (iteration) *iteration = s->iteration;
    return CFR_OK;
}

cfr_status cfr_set_state(cfr_solver *s, const double *cum_regret, const double *strat_sum, int64_t len_q,
                         int64_t iteration) {
    TRY(check_usable(s));
    if (!cum_regret || !strat_sum || len_q != s->Q)
        return set_err(s, CFR_ERR_INVALID, "cum_regret and strat_sum need exactly %lld entries", (long long)s->Q);
    if (iteration < 0) return set_err(s, CFR_ERR_INVALID, "iteration must be >= 0");
    DeviceGuard dg(s->device);
    CK(cudaStreamSynchronize(s->stream));
    if (s->Q > 0) {
        CK(cudaMemcpy(s->stage, cum_regret, sizeof(double) * s->Q, cudaMemcpyHostToDevice));
        k_scatter_player_q<<<nblocks(s->H), kBlock, 0, s->stream>>>(s->stage, s->q_int2user, s->qbase, s->iplayer, s->R, s->H);
        CK_LAUNCH();
        CK(cudaStreamSynchronize(s->stream));
        CK(cudaMemcpy(s->stage, strat_sum, sizeof(double) * s->Q, cudaMemcpyHostToDevice));
        k_scatter_player_q<<<nblocks(s->H), kBlock, 0, s->stream>>>(s->stage, s->q_int2user, s->qbase, s->iplayer, s->S, s->H);
        CK_LAUNCH();
        if (s->cfg.precision == CFR_FP64) regret_match_all<double>(s); else regret_match_all<float>(s);
        CK_LAUNCH();
    }
    CK(cudaMemcpyAsync(s->d_iter, &iteration, sizeof(int64_t), cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    s->iteration = iteration;
    return CFR_OK;
}

cfr_status cfr_get_nodes(cfr_solver *s, double *u1, double *cf_reach1, double *cf_reach2, int64_t len) {
    TRY(check_usable(s));
    if ((u1 || cf_reach1 || cf_reach2) && len < s->N)
        return set_err(s, CFR_ERR_INVALID, "node buffers need %lld entries", (long long)s->N);
    if (fused_from(s) < s->L && !s->cfg.record_nodes)
        return set_err(s, CFR_ERR_STATE, "node values of fused depths are not kept: load with record_nodes = 1");
    DeviceGuard dg(s->device);
    CK(cudaStreamSynchronize(s->stream));
    const bool fp64 = s->cfg.precision == CFR_FP64;
    auto fetch = [&](const void *src, int64_t n, std::vector<double> &dst) -> cfr_status {
        dst.assign((size_t)n, 0.0);
        if (n == 0) return CFR_OK;
        if (fp64) {
            CK(cudaMemcpy(dst.data(), src, sizeof(double) * n, cudaMemcpyDeviceToHost));
        } else {
            std::vector<float> f((size_t)n);
            CK(cudaMemcpy(f.data(), src, sizeof(float) * n, cudaMemcpyDeviceToHost));
            for (int64_t i = 0; i < n; ++i) dst[i] = f[i];
        }
        return CFR_OK;
    };
    std::vector<double> tmp;
    const double nan = std::numeric_limits<double>::quiet_NaN();
    if (u1) {
        TRY(fetch(s->u, s->Nd, tmp));
        for (int64_t j = 0; j < s->Nd; ++j) u1[s->dnode_user[j]] = tmp[j];
        tmp.assign((size_t)s->Nt, 0.0);
        if (s->Nt > 0) CK(cudaMemcpy(tmp.data(), s->util64, sizeof(double) * s->Nt, cudaMemcpyDeviceToHost));
        for (int64_t k = 0; k < s->Nt; ++k) u1[s->tnode_user[k]] = tmp[k];
    }
    double *outs[2] = {cf_reach1, cf_reach2};
    void *srcs[2] = {s->reach1, s->reach2};
    for (int i = 0; i < 2; ++i) {
        if (!outs[i]) continue;
        TRY(fetch(srcs[i], s->Nd, tmp));
        for (int64_t j = 0; j < s->Nd; ++j) outs[i][s->dnode_user[j]] = tmp[j];
        for (int64_t k = 0; k < s->Nt; ++k) outs[i][s->tnode_user[k]] = nan;
    }
    return CFR_OK;
}

static bool nondecreasing_from_zero(const int64_t *a, int64_t n) {
    if (a[0] != 0) return false;
    for (int64_t i = 0; i < n; ++i)
        if (a[i + 1] < a[i]) return false;
    return true;
}

cfr_status cfr_set_range_program(cfr_solver *s, int64_t num_segments, const int64_t *seg_dst, const int64_t *seg_entries,
                                 const int64_t *entry_prod, const int32_t *slots) {
    TRY(check_usable(s));
    if (num_segments < 0 || (num_segments > 0 && (!seg_dst || !seg_entries || !entry_prod)))
        return set_err(s, CFR_ERR_INVALID, "range program: malformed arrays");
    if (num_segments == 0) { s->rp_nseg = 0; return CFR_OK; }
    if (!nondecreasing_from_zero(seg_entries, num_segments))
        return set_err(s, CFR_ERR_INVALID, "range program: seg_entries must start at 0 and not decrease");
    const int64_t E = seg_entries[num_segments];
    if (!nondecreasing_from_zero(entry_prod, E))
        return set_err(s, CFR_ERR_INVALID, "range program: entry_prod must start at 0 and not decrease");
    const int64_t nslots = entry_prod[E];
    if (nslots > 0 && !slots) return set_err(s, CFR_ERR_INVALID, "range program: slots is NULL");
    for (int64_t k = 0; k < num_segments; ++k)
        if (seg_dst[k] < 0) return set_err(s, CFR_ERR_INVALID, "range program: seg_dst[%lld] < 0", (long long)k);
    DeviceGuard dg(s->device);
    std::vector<int32_t> q2u((size_t)std::max<int64_t>(s->Q, 1)), u2q((size_t)std::max<int64_t>(s->Q, 1), -1);
    CK(cudaMemcpyAsync(q2u.data(), s->q_int2user, sizeof(int32_t) * (size_t)s->Q, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    for (int64_t q = 0; q < s->Q; ++q) u2q[(size_t)q2u[(size_t)q]] = (int32_t)q;
    std::vector<int32_t> sl((size_t)nslots);
    for (int64_t i = 0; i < nslots; ++i) {
        if (slots[i] < 0 || slots[i] >= s->Q) return set_err(s, CFR_ERR_INVALID, "range program: slot %d out of range", slots[i]);
        sl[(size_t)i] = u2q[(size_t)slots[i]];
    }
    TRY(alloc_n(s, &s->rp_dst, num_segments)); TRY(alloc_n(s, &s->rp_ent, num_segments + 1));
    TRY(alloc_n(s, &s->rp_prod, E + 1)); TRY(alloc_n(s, &s->rp_slots, nslots));
    TRY(upload(s, s->rp_dst, std::vector<int64_t>(seg_dst, seg_dst + num_segments)));
    TRY(upload(s, s->rp_ent, std::vector<int64_t>(seg_entries, seg_entries + num_segments + 1)));
    TRY(upload(s, s->rp_prod, std::vector<int64_t>(entry_prod, entry_prod + E + 1)));
    TRY(upload(s, s->rp_slots, sl));
    CK(cudaStreamSynchronize(s->stream));
    s->rp_nseg = num_segments;
    return CFR_OK;
}

cfr_status cfr_gather_ranges(cfr_solver *s, float *out, int32_t strategy) {
    TRY(check_usable(s));
    if (strategy != CFR_CURRENT_STRATEGY && strategy != CFR_AVERAGE_STRATEGY)
        return set_err(s, CFR_ERR_INVALID, "strategy must be CFR_CURRENT_STRATEGY or CFR_AVERAGE_STRATEGY");
    if (s->rp_nseg == 0) return CFR_OK;
    if (!out) return set_err(s, CFR_ERR_INVALID, "out is NULL");
    DeviceGuard dg(s->device);
    const int grid = (int)std::min<int64_t>((s->rp_nseg + 127) / 128, 4096);
    if (strategy == CFR_AVERAGE_STRATEGY) {
        if (!s->avg) TRY(alloc_n(s, &s->avg, s->Q));
        if (s->H > 0) {
            k_average<<<nblocks(s->H), kBlock, 0, s->stream>>>(s->S, s->sigma064, s->qbase, s->iplayer, s->avg, s->H);
            CK_LAUNCH();
        }
        k_ranges<double><<<grid, 128, 0, s->stream>>>(s->avg, s->rp_dst, s->rp_ent, s->rp_prod, s->rp_slots, s->rp_nseg, out);
        CK_LAUNCH();
        s->kernel_launches += 2;
        return CFR_OK;
    }
    if (s->cfg.precision == CFR_FP64)
        k_ranges<double><<<grid, 128, 0, s->stream>>>(static_cast<const double *>(s->sigma), s->rp_dst, s->rp_ent, s->rp_prod,
                                                      s->rp_slots, s->rp_nseg, out);
    else
        k_ranges<float><<<grid, 128, 0, s->stream>>>(static_cast<const float *>(s->sigma), s->rp_dst, s->rp_ent, s->rp_prod,
                                                     s->rp_slots, s->rp_nseg, out);
    CK_LAUNCH();
    s->kernel_launches += 1;
    return CFR_OK;
}

cfr_status cfr_set_leaves(cfr_solver *s, const int32_t *nodes, const int64_t *src_index, int64_t num_leaves) {
    TRY(check_usable(s));
    if (num_leaves < 0 || (num_leaves > 0 && (!nodes || !src_index)))
        return set_err(s, CFR_ERR_INVALID, "leaves: malformed arrays");
    std::vector<int32_t> node2t((size_t)std::max<int64_t>(s->N, 1), -1);
    for (int64_t k = 0; k < s->Nt; ++k) node2t[(size_t)s->tnode_user[(size_t)k]] = (int32_t)k;
    std::vector<int32_t> t((size_t)num_leaves);
    for (int64_t i = 0; i < num_leaves; ++i) {
        if (nodes[i] < 0 || nodes[i] >= s->N || node2t[(size_t)nodes[i]] < 0)
            return set_err(s, CFR_ERR_INVALID, "leaves: node %d is not a terminal", nodes[i]);
        if (src_index[i] < 0) return set_err(s, CFR_ERR_INVALID, "leaves: src_index[%lld] < 0", (long long)i);
        t[(size_t)i] = node2t[(size_t)nodes[i]];
    }
    DeviceGuard dg(s->device);
    s->nleaves = 0;
    if (num_leaves == 0) return CFR_OK;
    TRY(alloc_n(s, &s->leaf_t, num_leaves));
    TRY(alloc_n(s, &s->leaf_src, num_leaves));
    TRY(upload(s, s->leaf_t, t));
    TRY(upload(s, s->leaf_src, std::vector<int64_t>(src_index, src_index + num_leaves)));
    CK(cudaStreamSynchronize(s->stream));
    s->nleaves = num_leaves;
    return CFR_OK;
}

cfr_status cfr_set_leaf_values(cfr_solver *s, const float *src, double scale) {
    TRY(check_usable(s));
    if (s->nleaves == 0) return CFR_OK;
    if (!src) return set_err(s, CFR_ERR_INVALID, "src is NULL");
    DeviceGuard dg(s->device);
    const int grid = (int)std::min<int64_t>((s->nleaves + 255) / 256, 4096);
    if (s->cfg.precision == CFR_FP64)
        k_set_leaves<double><<<grid, 256, 0, s->stream>>>(static_cast<double *>(s->util), s->util64, s->leaf_t, s->leaf_src,
                                                          src, scale, s->nleaves);
    else
        k_set_leaves<float><<<grid, 256, 0, s->stream>>>(static_cast<float *>(s->util), s->util64, s->leaf_t, s->leaf_src,
                                                         src, scale, s->nleaves);
    CK_LAUNCH();
    s->kernel_launches += 1;
    return CFR_OK;
}

cfr_status cfr_root_value(cfr_solver *s, double *u1) {
    TRY(check_usable(s));
    if (!u1) return set_err(s, CFR_ERR_INVALID, "u1 is NULL");
    DeviceGuard dg(s->device);
    if (s->Nd == 0) {
        CK(cudaMemcpy(u1, s->util64, sizeof(double), cudaMemcpyDeviceToHost));
        return CFR_OK;
    }
    if (s->cfg.precision == CFR_FP64) {
        CK(cudaMemcpyAsync(u1, s->u, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
    } else {
        float f = 0.0f;
        CK(cudaMemcpyAsync(&f, s->u, sizeof(float), cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        *u1 = f;
    }
    return CFR_OK;
}

cfr_status cfr_root_value_async(cfr_solver *s, double *u1) {
    TRY(check_usable(s));
    if (!u1) return set_err(s, CFR_ERR_INVALID, "u1 is NULL");
    DeviceGuard dg(s->device);
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, u1) != cudaSuccess || a.type != cudaMemoryTypeHost || !a.devicePointer) {
        cudaGetLastError();
        return set_err(s, CFR_ERR_INVALID, "u1 is not page-locked host memory");
    }
    double *dst = static_cast<double *>(a.devicePointer);
    if (s->Nd == 0) k_root_out<double><<<1, 1, 0, s->stream>>>(static_cast<const double *>(s->util64), dst);
    else if (s->cfg.precision == CFR_FP64) k_root_out<double><<<1, 1, 0, s->stream>>>(static_cast<const double *>(s->u), dst);
    else k_root_out<float><<<1, 1, 0, s->stream>>>(static_cast<const float *>(s->u), dst);
    CK_LAUNCH();
    return CFR_OK;
}

cfr_status cfr_phase_times(cfr_solver *s, double *us, double *bytes, int32_t *kind, int32_t *depth, int32_t len,
                           int32_t *nphases) {
    TRY(check_usable(s));
    if (s->cfg.update_mode == CFR_ALTERNATING)
        return set_err(s, CFR_ERR_UNSUPPORTED, "phase timing covers simultaneous updates only");
    const auto ph = phases(s);
    const int32_t n = (int32_t)ph.size();
    if (nphases) *nphases = n;
    if (!us && !bytes && !kind && !depth) return CFR_OK;
    if (len < n) return set_err(s, CFR_ERR_INVALID, "phase buffers need %d entries", n);
    if (n == 0) return CFR_OK;
    DeviceGuard dg(s->device);
    std::vector<cudaEvent_t> ev((size_t)n + 1, nullptr);
    for (auto &e : ev) CK(cudaEventCreate(&e));
    cfr_status st = s->cfg.precision == CFR_FP64 ? enqueue_iteration<double>(s, s->stream, ev.data())
                                                 : enqueue_iteration<float>(s, s->stream, ev.data());
    if (st == CFR_OK) {
        s->iteration += 1;
        s->kernel_launches += launches_per_iteration(s);
        cudaError_t e = cudaEventSynchronize(ev[(size_t)n]);
        for (int32_t k = 0; k < n && e == cudaSuccess; ++k) {
            float ms = 0.f;
            e = cudaEventElapsedTime(&ms, ev[(size_t)k], ev[(size_t)k + 1]);
            if (us) us[k] = 1e3 * (double)ms;
        }
        if (e != cudaSuccess) { s->poisoned = true; st = set_err(s, CFR_ERR_CUDA, "phase timing: %s", cudaGetErrorString(e)); }
    }
    for (auto &e : ev) cudaEventDestroy(e);
    if (st == CFR_OK) {
        const std::vector<double> b = phase_bytes(s);
        for (int32_t k = 0; k < n; ++k) {
            if (bytes) bytes[k] = b[(size_t)k];
            if (kind) kind[k] = ph[(size_t)k].first;
            if (depth) depth[k] = ph[(size_t)k].second;
        }
    }
    return st;
}

cfr_status cfr_get_info(const cfr_solver *s, cfr_info *info) {
    if (!s || !info) return set_err(nullptr, CFR_ERR_INVALID, "solver or info is NULL");
    std::memset(info, 0, sizeof *info);
    info->num_nodes = s->N; info->num_decision = s->Nd; info->num_terminal = s->Nt; info->num_q = s->Q;
    info->num_infosets = s->H; info->num_levels = s->L; info->max_depth = s->max_depth;
    info->max_actions = s->max_actions; info->single_level_infosets = s->single_level;
    info->variant = s->cfg.variant; info->precision = s->cfg.precision; info->update_mode = s->cfg.update_mode;
    info->avg_weight = s->cfg.avg_weight; info->iteration = s->iteration; info->device_bytes = s->device_bytes;
    info->bytes_per_iteration = bytes_model(s);
    info->kernels_per_iteration = launches_per_iteration(s);
    info->kernel_launches = s->kernel_launches;
    info->fused_from_depth = fused_from(s);
    info->head_depths = s->cfg.precision == CFR_FP64 ? 0 : s->head_n;
    info->tail_kernel = fused_from(s) == s->L || !s->fuse_tail ? 0
                        : s->ntail_tiles == 0 ? 1
                        : !s->tail_slots ? 2 : s->cfg.tail_slots == 2 ? 4 : 3;
    info->pair_depth = fused_from(s) < s->L && s->npair_tiles > 0 ? s->pair_m : -1;
    info->fused_tiles = fused_from(s) == s->L ? 0
                        : !s->fuse_tail ? s->fuse_ntiles
                        : s->ntail_tiles > 0 ? s->ntail_tiles : nblocks(s->dlevel[s->fuse_r + 1] - s->dlevel[s->fuse_r]);
    return CFR_OK;
}

const char *cfr_last_error(const cfr_solver *s) { return s ? s->err.c_str() : g_thread_err.c_str(); }

void cfr_free(cfr_solver *s) {
    if (!s) return;
    DeviceGuard dg(s->device);
    if (s->stream || s->cap) cudaStreamSynchronize(s->stream);
    if (s->graph_exec) cudaGraphExecDestroy(s->graph_exec);
    if (s->br_exec) cudaGraphExecDestroy(s->br_exec);
    if (s->graph) cudaGraphDestroy(s->graph);
    if (s->graph_exec2) cudaGraphExecDestroy(s->graph_exec2);
    if (s->graph2) cudaGraphDestroy(s->graph2);
    for (auto &b : s->blocks) {
        if (s->cfg.dev_free) s->cfg.dev_free(b.first, s->cfg.alloc_ctx);
        else cudaFree(b.first);
    }
    if (s->side) cudaStreamSynchronize(s->side);
    if (s->cap) cudaStreamDestroy(s->cap);
    if (s->side) cudaStreamDestroy(s->side);
    for (int i = 0; i < 2; ++i) {
        if (s->fork[i]) cudaEventDestroy(s->fork[i]);
        if (s->join[i]) cudaEventDestroy(s->join[i]);
        if (s->deep[i]) cudaEventDestroy(s->deep[i]);
        if (s->upd[i]) cudaEventDestroy(s->upd[i]);
    }
    delete s;
}

}  // extern "C"

// ================================================================================================
// Exploitability without device allocation (cfr_exploitability_static).
//
// Some callers may not allocate GPU memory once they are running: a host application that hands
// the library a fixed memory budget up front, or a real-time loop in which an allocation (and the
// synchronisation cudaMalloc/cudaFree imply) is not allowed.  For them this variant runs the same
// best-response kernels as cfr_exploitability with all of its working memory - the average
// strategy, the opponent reaches, the node values, the per-action sums and the chosen actions - in
// one fixed region compiled into this library, kStaticScratchBytes per GPU, which every GPU that
// loads the library holds until the process exits.  Calls share the region and leave their
// contents in it; calls that overlap on the GPU (two streams, or two threads) race on it.
namespace {

constexpr size_t kStaticScratchBytes = CFR_STATIC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxStaticDevices = 64;
std::mutex g_static_mu;
void *g_static_ptr[kMaxStaticDevices] = {};

// The region's device address on the current device; looked up once per device.  Host code must
// not use the symbol itself: on the host it names a host-side stand-in, not device memory.
cudaError_t static_scratch(int dev, unsigned char **out) {
    if (dev < 0 || dev >= kMaxStaticDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_static_ptr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_static_ptr[dev]);
    return cudaSuccess;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" cfr_status cfr_exploitability_static(cfr_solver *s, double *nash_conv, double *exploitability) {
    TRY(check_usable(s));
    if (!s->single_level)
        return set_err(s, CFR_ERR_UNSUPPORTED, "the GPU best response needs every infoset at a single depth");
    const size_t need = align256(sizeof(double) * (size_t)s->Q) * 2 + align256(sizeof(double) * (size_t)s->Nd) * 2 +
                        align256(sizeof(int32_t) * (size_t)s->H) + 256;
    if (need > kStaticScratchBytes)
        return set_err(s, CFR_ERR_UNSUPPORTED,
                       "cfr_exploitability_static needs %zu bytes of working memory for this game; its fixed region "
                       "holds %zu (use cfr_exploitability)", need, kStaticScratchBytes);
    DeviceGuard dg(s->device);
    unsigned char *base = nullptr;
    CK(static_scratch(s->device, &base));
    double nc = 0.0;
    if (s->Nd > 0) {
        unsigned char *p = base;
        double *avg = reinterpret_cast<double *>(p);        p += align256(sizeof(double) * (size_t)s->Q);
        double *cfv = reinterpret_cast<double *>(p);        p += align256(sizeof(double) * (size_t)s->Q);
        double *preach = reinterpret_cast<double *>(p);     p += align256(sizeof(double) * (size_t)s->Nd);
        double *val = reinterpret_cast<double *>(p);        p += align256(sizeof(double) * (size_t)s->Nd);
        int32_t *astar = reinterpret_cast<int32_t *>(p);
        cudaStream_t st = s->stream;
        k_average<<<nblocks(s->H), kBlock, 0, st>>>(s->S, s->sigma064, s->qbase, s->iplayer, avg, s->H);
        CK_LAUNCH();
        DevBR b;
        b.dfirst = s->dfirst; b.tfirst = s->tfirst; b.dinfo = s->dinfo;
        b.kmask = s->kmask; b.wbits = s->wbits;
        b.util = s->util64; b.qbase = s->qbase; b.iplayer = s->iplayer; b.avg = avg;
        b.preach = preach; b.val = val; b.cfv = cfv; b.astar = astar;
        const int32_t nr = s->dlevel[1];   // every depth-0 root, as the allocating path fills them
        for (int player = 1; player <= 2; ++player) {
            // the region keeps the previous call's contents: the root reaches and the sums restart here
            k_fill<<<nblocks(nr), kBlock, 0, st>>>(preach, nr, 1.0);
            CK_LAUNCH();
            CK(cudaMemsetAsync(cfv, 0, sizeof(double) * (size_t)std::max<int64_t>(s->Q, 1), st));
            for (int32_t l = 0; l + 1 < s->L; ++l) {
                const int32_t j0 = s->dlevel[l], j1 = s->dlevel[l + 1];
                k_br_topdown<<<nblocks(j1 - j0), kBlock, 0, st>>>(b, j0, j1, player);
                CK_LAUNCH();
            }
            for (int32_t l = s->L - 1; l >= 0; --l) {
                const int32_t j0 = s->dlevel[l], j1 = s->dlevel[l + 1];
                const int32_t h0 = s->hlevel[l], h1 = s->hlevel[l + 1];
                k_br_nodes<<<nblocks(j1 - j0), kBlock, 0, st>>>(b, j0, j1, player);
                CK_LAUNCH();
                if (h1 > h0) {
                    k_br_choose<<<nblocks(h1 - h0), kBlock, 0, st>>>(b, h0, h1, player);
                    CK_LAUNCH();
                }
                k_br_pick<<<nblocks(j1 - j0), kBlock, 0, st>>>(b, j0, j1, player);
                CK_LAUNCH();
            }
            double v = 0.0;
            CK(cudaMemcpyAsync(&v, val, sizeof(double), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            nc += v;   // zero-sum: u_1(avg) + u_2(avg) = 0
        }
    }
    if (nash_conv) *nash_conv = nc;
    if (exploitability) *exploitability = nc / 2.0;
    return CFR_OK;
}
