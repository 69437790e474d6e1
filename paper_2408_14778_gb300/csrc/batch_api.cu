// C ABI of batched solving (include/cfr_gb300.h, cfr_batch_*): many independent games advanced together.
// Games below a size split whose image fits shared memory run in one persistent launch per call, each
// solved by one block in its shared memory (batch.cuh), the launch shape picked by a measured sweep
// (cfr_batch_autotune); the others as one forest through the single-game solver's per-depth kernels on
// a second stream, concurrently.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "batch.cuh"
#include "cfr_gb300.h"
#include "layout.hpp"
#include "solver_internal.hpp"

using namespace cfrgb;

namespace {

thread_local std::string g_batch_err;

constexpr int64_t kBatchSplitDefault = 4096;    // games of at least this many nodes run as one forest
constexpr int64_t kSmemCap = 200 * 1024;        // shared memory a resident game may take, at most
// Resident games are launched in classes by footprint, each with the shared memory of its largest
// game, so that a few large games do not lower every block's occupancy.
constexpr int kClasses = 4;
constexpr int64_t kClassCap[kClasses] = {24 * 1024, 48 * 1024, 100 * 1024, kSmemCap};

// A game's shared-memory image (batch.cuh) from its own single-game layout; the slot map is filled
// once the batch's layout is known.  False when the game cannot be resident (a node with more than 32
// actions, or more than kSmemCap bytes); *err explains an invalid game.
struct GameImage {
    std::vector<int32_t> w;
    std::vector<int32_t> q_int2user, qplayer;   // per local slot: the game's caller slot, its player
    int64_t bytes = 0;
};

cfr_status make_image(const cfr_game_desc &g, GameImage &img, bool *fits, std::string *err) {
    Layout Lg;
    const cfr_status st = build_layout(&g, &Lg, err);
    if (st != CFR_OK) return st;
    *fits = Lg.wide.empty();
    if (!*fits) return CFR_OK;
    std::vector<int32_t> &w = img.w;
    w.assign(kImgHeader, 0);
    auto put = [&](const void *data, size_t bytes) -> int32_t {
        while (w.size() % 4) w.push_back(0);
        const int32_t off = (int32_t)w.size();
        const size_t nw = (bytes + 3) / 4;
        w.resize(w.size() + nw, 0);
        if (data && bytes) std::memcpy(w.data() + off, data, bytes);
        return off;
    };
    const std::vector<float> util(Lg.util.begin(), Lg.util.end()), sigma0(Lg.sigma0.begin(), Lg.sigma0.end());
    w[kImgNd] = (int32_t)Lg.Nd; w[kImgNt] = (int32_t)Lg.Nt; w[kImgH] = Lg.H; w[kImgHp] = Lg.Hp;
    w[kImgQ] = (int32_t)Lg.Q; w[kImgL] = Lg.L;
    w[kImgDlevel] = put(Lg.dlevel.data(), 4 * Lg.dlevel.size());
    w[kImgHlevel] = put(Lg.hlevel.data(), 4 * Lg.hlevel.size());
    w[kImgDfirst] = put(Lg.dfirst.data(), 4 * Lg.dfirst.size());
    w[kImgTfirst] = put(Lg.tfirst.data(), 4 * Lg.tfirst.size());
    w[kImgKmask] = put(Lg.kmask.data(), 4 * Lg.kmask.size());
    w[kImgQp] = put(Lg.qp.data(), 4 * Lg.qp.size());
    w[kImgUtil] = put(util.data(), 4 * util.size());
    w[kImgQbase] = put(Lg.qbase.data(), 4 * Lg.qbase.size());
    w[kImgPseq] = put(Lg.pseq.data(), 4 * Lg.pseq.size());
    w[kImgPseqH] = put(Lg.pseq_h.data(), 4 * Lg.pseq_h.size());
    w[kImgIplayer] = put(Lg.iplayer.data(), Lg.iplayer.size());
    w[kImgSigma0] = put(sigma0.data(), 4 * sigma0.size());
    w[kImgQmap] = put(nullptr, 4 * (size_t)Lg.Q);
    while (w.size() % 4) w.push_back(0);
    w[kImgWords] = (int32_t)w.size();
    img.q_int2user = Lg.q_int2user;
    img.qplayer.assign((size_t)Lg.Q, 0);
    for (int32_t h = 0; h < Lg.H; ++h)
        for (int32_t q = Lg.qbase[(size_t)h]; q < Lg.qbase[(size_t)h + 1]; ++q) img.qplayer[(size_t)q] = Lg.iplayer[(size_t)h];
    img.bytes = smem_game_bytes((int64_t)w.size(), Lg.Nd, Lg.H, Lg.Q);
    *fits = img.bytes <= kSmemCap;
    return CFR_OK;
}

struct BDeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit BDeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; prev = -1; return; }
        if (dev >= 0 && dev != prev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~BDeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

struct cfr_batch {
    cfr_config cfg{};
    int device = 0, sms = 0;
    cudaStream_t stream = nullptr;   // borrowed
    cudaStream_t cap = nullptr;      // private, for graph capture
    // The games split by size: the small ones run in the persistent kernel (the fields below), those of
    // at least split_nodes nodes as one forest through the single-game solver's per-depth kernels
    // (`big`, on `side`), concurrently.
    int32_t n_games = 0;
    int64_t split_nodes = 0;
    std::vector<int8_t> part;            // per game: 0 persistent, 1 forest
    std::vector<int32_t> idx;            // per game: its index within its part
    std::vector<int64_t> big_q_off;      // forest part: per game, its first slot in the forest's numbering
    std::vector<int64_t> big_nodes;
    cfr_solver *big = nullptr;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_b0 = nullptr, ev_b1 = nullptr;
    bool big_timed = false;
    int32_t G = 0, stride = 0, Hp = 0, H = 0, hp_na = 0;   // the persistent part
    int32_t *images = nullptr;           // per game of the persistent part, its shared-memory image
    int64_t *img_off = nullptr;          // word offset of each image
    int64_t smem_bytes = 0;              // dynamic shared memory of a block (the largest game's need)
    // footprint classes: class c's games are order[cls_off[c] .. cls_off[c + 1]), launched with
    // cls_smem[c] bytes per block, each class but the first on its own stream (graph branch)
    std::vector<int32_t> cls_off;
    std::vector<int64_t> cls_smem;
    cudaStream_t aux[kClasses] = {};
    cudaEvent_t cls_fork = nullptr, cls_join[kClasses] = {};
    int64_t N = 0, Nd = 0, Nt = 0, Q = 0;
    bool single_level = true;
    // host: per game, its first node / infoset / infoset-action slot in the caller's numbering (+ total)
    std::vector<int64_t> node_off, h_off, q_off;
    std::vector<int32_t> q_int2user;     // internal slot -> caller slot of the combined game
    std::vector<int64_t> game_nodes;
    // device
    // (the forest's structure serves the best response; the iterations run on the images)
    int32_t *dfirst = nullptr, *tfirst = nullptr, *dinfo = nullptr, *qbase = nullptr, *astar = nullptr;
    int8_t *iplayer = nullptr;
    uint32_t *kmask = nullptr;
    float *sigma = nullptr;
    double *util64 = nullptr, *sigma064 = nullptr, *R = nullptr, *S = nullptr, *avg = nullptr, *cfv = nullptr,
           *preach = nullptr, *val = nullptr, *br_out = nullptr, *snapR = nullptr, *snapS = nullptr;
    float *snapSigma = nullptr;
    int32_t *order = nullptr, *dlo = nullptr, *dhi = nullptr, *hlo = nullptr, *hhi = nullptr, *nlev = nullptr,
            *next = nullptr;
    unsigned long long *t_start = nullptr, *t_end = nullptr;
    int64_t *d_iter = nullptr;
    // launch shape and its graph (one per K)
    int32_t threads = 256, blocks_per_sm = 0;
    bool tuned = false;
    cudaGraphExec_t graph_exec = nullptr;
    int32_t graph_K = -1;
    int64_t iteration = 0, kernel_launches = 0;
    int32_t last_K = 0;
    std::vector<void *> blocks;
    int64_t device_bytes = 0;
    std::string err;
    bool poisoned = false;
};

namespace {

cfr_status berr(cfr_batch *b, cfr_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    else g_batch_err = buf;
    return st;
}

#define BCK(call)                                                                                       \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess) {                                                                        \
            b->poisoned = true;                                                                         \
            return berr(b, e_ == cudaErrorMemoryAllocation ? CFR_ERR_OOM : CFR_ERR_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                             \
        }                                                                                               \
    } while (0)

#define BTRY(x)                                \
    do {                                       \
        cfr_status st_ = (x);                  \
        if (st_ != CFR_OK) return st_;         \
    } while (0)

template <typename T>
cfr_status balloc(cfr_batch *b, T **p, int64_t n) {
    size_t bytes = (sizeof(T) * (size_t)std::max<int64_t>(n, 1) + 255) & ~(size_t)255;
    void *ptr = nullptr;
    if (b->cfg.dev_alloc) {
        ptr = b->cfg.dev_alloc(bytes, b->cfg.alloc_ctx);
        if (!ptr) return berr(b, CFR_ERR_OOM, "device allocator returned NULL for %zu bytes", bytes);
    } else {
        cudaError_t e = cudaMalloc(&ptr, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return berr(b, CFR_ERR_OOM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
        }
    }
    b->blocks.push_back(ptr);
    b->device_bytes += (int64_t)bytes;
    *p = static_cast<T *>(ptr);
    return CFR_OK;
}

template <typename T>
cfr_status bupload(cfr_batch *b, T *dst, const std::vector<T> &src) {
    if (src.empty()) return CFR_OK;
    BCK(cudaMemcpyAsync(dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    return CFR_OK;
}

BatchDesc batch_desc(const cfr_batch *b) {
    BatchDesc d;
    d.order = b->order; d.dlo = b->dlo; d.dhi = b->dhi; d.hlo = b->hlo; d.hhi = b->hhi; d.nlev = b->nlev;
    d.G = b->G; d.stride = b->stride; d.next = b->next; d.t_start = b->t_start; d.t_end = b->t_end;
    return d;
}

// The persistent launch of K iterations (games resident in shared memory) for the batch's variant and
// action count.
template <int NA, int V>
void *smem_kernel() { return reinterpret_cast<void *>(k_batch_smem<NA, V>); }

void *smem_kernel_for(const cfr_batch *b) {
    const int na = b->hp_na <= 3 ? 0 : b->hp_na <= 5 ? 1 : 2;
    switch (b->cfg.variant * 3 + na) {
    case 0: return smem_kernel<3, CFRV_VANILLA>();
    case 1: return smem_kernel<5, CFRV_VANILLA>();
    case 2: return smem_kernel<8, CFRV_VANILLA>();
    case 3: return smem_kernel<3, CFRV_PLUS>();
    case 4: return smem_kernel<5, CFRV_PLUS>();
    case 5: return smem_kernel<8, CFRV_PLUS>();
    case 6: return smem_kernel<3, CFRV_LINEAR>();
    case 7: return smem_kernel<5, CFRV_LINEAR>();
    case 8: return smem_kernel<8, CFRV_LINEAR>();
    case 9: return smem_kernel<3, CFRV_DISCOUNTED>();
    case 10: return smem_kernel<5, CFRV_DISCOUNTED>();
    default: return smem_kernel<8, CFRV_DISCOUNTED>();
    }
}

int32_t class_games(const cfr_batch *b, int c) { return b->cls_off[(size_t)c + 1] - b->cls_off[(size_t)c]; }

cudaError_t launch_class(cfr_batch *b, cudaStream_t st, int c, int32_t K, int grid, int threads) {
    const int32_t linear = b->cfg.avg_weight == CFR_AVG_LINEAR;
    const double3 dc = make_double3(b->cfg.dcfr_alpha, b->cfg.dcfr_beta, b->cfg.dcfr_gamma);
    const int32_t *images = b->images;
    const int64_t *img_off = b->img_off;
    const int32_t *order = b->order + b->cls_off[(size_t)c];
    int32_t G = class_games(b, c);
    int32_t *next = b->next + c;
    double *gR = b->R, *gS = b->S;
    float *gs = b->sigma;
    const int64_t *T0 = b->d_iter;
    unsigned long long *t0 = b->t_start, *t1 = b->t_end;
    int32_t alternating = b->cfg.update_mode == CFR_ALTERNATING;
    void *args[] = {&images, &img_off, &order, &G, &next, &gR, &gS, &gs, &T0, &K, (void *)&linear, (void *)&dc,
                    &alternating, &t0, &t1};
    return cudaLaunchKernel(smem_kernel_for(b), dim3((unsigned)grid), dim3((unsigned)threads), args,
                            (size_t)b->cls_smem[(size_t)c], st);
}

// Resident blocks per SM of class c's launch at a block size.
int occupancy(const cfr_batch *b, int c, int threads) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, smem_kernel_for(b), threads,
                                                      (size_t)b->cls_smem[(size_t)c]) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm;
}

// The most blocks per SM any non-empty class can hold, and the fewest (0: no class fits).
int occupancy_max(const cfr_batch *b, int threads) {
    int m = 0;
    for (int c = 0; c < kClasses; ++c)
        if (class_games(b, c) > 0) m = std::max(m, occupancy(b, c, threads));
    return m;
}
int occupancy_min(const cfr_batch *b, int threads) {
    int m = 1 << 30;
    for (int c = 0; c < kClasses; ++c)
        if (class_games(b, c) > 0) m = std::min(m, occupancy(b, c, threads));
    return m == 1 << 30 ? 0 : m;
}

int grid_of(const cfr_batch *b, int c, int threads, int bps) {
    const int occ = occupancy(b, c, threads);
    const int per_sm = std::max(1, bps > 0 ? std::min(bps, occ) : occ);
    return std::max(1, std::min(class_games(b, c), per_sm * b->sms));
}

// Queues K iterations: the work counter reset, the persistent launch, the iteration count advanced.
// Class 0 (or the first non-empty class) runs on st, the others on their own streams forked from and
// joined back to it.
cfr_status enqueue_batch(cfr_batch *b, cudaStream_t st, int32_t K, int threads, int bps) {
    BCK(cudaMemsetAsync(b->next, 0, sizeof(int32_t) * kClasses, st));
    int first = -1;
    for (int c = 0; c < kClasses; ++c) {
        if (class_games(b, c) == 0) continue;
        if (first < 0) { first = c; BCK(cudaEventRecord(b->cls_fork, st)); continue; }
        BCK(cudaStreamWaitEvent(b->aux[c], b->cls_fork, 0));
        BCK(launch_class(b, b->aux[c], c, K, grid_of(b, c, threads, bps), threads));
        BCK(cudaEventRecord(b->cls_join[c], b->aux[c]));
    }
    if (first >= 0) BCK(launch_class(b, st, first, K, grid_of(b, first, threads, bps), threads));
    for (int c = first + 1; c < kClasses && first >= 0; ++c)
        if (class_games(b, c) > 0) BCK(cudaStreamWaitEvent(st, b->cls_join[c], 0));
    k_batch_advance<<<1, 1, 0, st>>>(b->d_iter, K);
    BCK(cudaGetLastError());
    return CFR_OK;
}

cfr_status build_batch_graph(cfr_batch *b, int32_t K) {
    if (b->graph_exec) { cudaGraphExecDestroy(b->graph_exec); b->graph_exec = nullptr; }
    BCK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    cfr_status st = enqueue_batch(b, b->cap, K, b->threads, b->blocks_per_sm);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap, &g);
    if (st != CFR_OK) { if (g) cudaGraphDestroy(g); return st; }
    if (e != cudaSuccess) { b->poisoned = true; return berr(b, CFR_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e)); }
    e = cudaGraphInstantiate(&b->graph_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { b->poisoned = true; return berr(b, CFR_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e)); }
    b->graph_K = K;
    return CFR_OK;
}

cfr_status small_exploitability(cfr_batch *b, double *nash_conv);

cfr_status bsync(cfr_batch *b) {
    BCK(cudaStreamSynchronize(b->stream));
    return CFR_OK;
}

cfr_status busable(cfr_batch *b) {
    if (!b) return berr(nullptr, CFR_ERR_INVALID, "batch is NULL");
    if (b->poisoned) return berr(b, CFR_ERR_STATE, "batch is unusable after an earlier CUDA error: %s", b->err.c_str());
    return CFR_OK;
}

// Concatenates the games into one forest description (caller numbering: game g's nodes, infosets and
// slots follow game g - 1's).
cfr_status combine(const cfr_game_desc *games, int32_t n, cfr_batch *b, std::vector<int32_t> &parent,
                   std::vector<int32_t> &action, std::vector<int32_t> &infoset, std::vector<int8_t> &player,
                   std::vector<int32_t> &nact, std::vector<double> &cprob, std::vector<double> &util) {
    b->node_off.assign((size_t)n + 1, 0);
    b->h_off.assign((size_t)n + 1, 0);
    b->q_off.assign((size_t)n + 1, 0);
    for (int32_t i = 0; i < n; ++i) {
        const cfr_game_desc &g = games[i];
        if (g.num_nodes < 1 || !g.parent || !g.action || !g.infoset || !g.utility || g.num_infosets < 0 ||
            (g.num_infosets > 0 && (!g.infoset_player || !g.infoset_num_actions)))
            return berr(nullptr, CFR_ERR_INVALID, "game %d: malformed description", i);
        int64_t q = 0;
        for (int32_t h = 0; h < g.num_infosets; ++h) q += g.infoset_num_actions[h];
        b->node_off[(size_t)i + 1] = b->node_off[(size_t)i] + g.num_nodes;
        b->h_off[(size_t)i + 1] = b->h_off[(size_t)i] + g.num_infosets;
        b->q_off[(size_t)i + 1] = b->q_off[(size_t)i] + q;
    }
    const int64_t N = b->node_off[(size_t)n];
    if (N >= (int64_t)INT32_MAX || b->h_off[(size_t)n] >= (int64_t)INT32_MAX)
        return berr(nullptr, CFR_ERR_UNSUPPORTED, "the batch has %lld nodes (at most 2^31 - 2)", (long long)N);
    parent.resize((size_t)N); action.resize((size_t)N); infoset.resize((size_t)N); util.resize((size_t)N * 2);
    player.resize((size_t)b->h_off[(size_t)n]); nact.resize((size_t)b->h_off[(size_t)n]);
    b->game_nodes.assign((size_t)n, 0);
    for (int32_t i = 0; i < n; ++i) {
        const cfr_game_desc &g = games[i];
        const int64_t no = b->node_off[(size_t)i], ho = b->h_off[(size_t)i];
        b->game_nodes[(size_t)i] = g.num_nodes;
        for (int64_t v = 0; v < g.num_nodes; ++v) {
            const int32_t p = g.parent[v];
            if (p < -1 || p >= g.num_nodes) return berr(nullptr, CFR_ERR_INVALID, "game %d node %lld: parent %d", i, (long long)v, p);
            parent[(size_t)(no + v)] = p < 0 ? -1 : (int32_t)(no + p);
            action[(size_t)(no + v)] = g.action[v];
            const int32_t h = g.infoset[v];
            if (h < -1 || h >= g.num_infosets) return berr(nullptr, CFR_ERR_INVALID, "game %d node %lld: infoset %d", i, (long long)v, h);
            infoset[(size_t)(no + v)] = h < 0 ? -1 : (int32_t)(ho + h);
            util[(size_t)(no + v) * 2] = g.utility[2 * v];
            util[(size_t)(no + v) * 2 + 1] = g.utility[2 * v + 1];
        }
        int64_t nc = 0;
        for (int32_t h = 0; h < g.num_infosets; ++h) {
            player[(size_t)(ho + h)] = g.infoset_player[h];
            nact[(size_t)(ho + h)] = g.infoset_num_actions[h];
            if (g.infoset_player[h] == 0) nc += g.infoset_num_actions[h];
        }
        if (nc > 0 && (!g.chance_prob || g.num_chance_prob < nc))
            return berr(nullptr, CFR_ERR_INVALID, "game %d: chance_prob needs %lld entries", i, (long long)nc);
        cprob.insert(cprob.end(), g.chance_prob, g.chance_prob + nc);
    }
    return CFR_OK;
}

cfr_status load_batch(cfr_batch *b, Layout &Lo) {
    b->N = Lo.N; b->Nd = Lo.Nd; b->Nt = Lo.Nt; b->Q = Lo.Q; b->H = Lo.H; b->Hp = Lo.Hp;
    b->single_level = Lo.single_level;
    b->q_int2user = Lo.q_int2user;
    // per game and depth: its decision nodes and the player infosets first seen there (each depth lists
    // its nodes, and its newly seen infosets, game by game)
    const int32_t G = b->G, L = Lo.L;
    b->stride = std::max(L, 1);
    std::vector<int32_t> dlo((size_t)G * b->stride, 0), dhi((size_t)G * b->stride, 0), hlo((size_t)G * b->stride, 0),
        hhi((size_t)G * b->stride, 0), nlev((size_t)G, 0);
    auto game_of_node = [&](int32_t v) {
        return (int32_t)(std::upper_bound(b->node_off.begin(), b->node_off.end(), (int64_t)v) - b->node_off.begin() - 1);
    };
    auto game_of_infoset = [&](int32_t h) {
        return (int32_t)(std::upper_bound(b->h_off.begin(), b->h_off.end(), (int64_t)h) - b->h_off.begin() - 1);
    };
    for (int32_t l = 0; l < L; ++l) {
        for (int32_t j = Lo.dlevel[(size_t)l]; j < Lo.dlevel[(size_t)l + 1]; ++j) {
            const int32_t g = game_of_node(Lo.dnode_user[(size_t)j]);
            const size_t k = (size_t)g * b->stride + l;
            if (dhi[k] == 0) dlo[k] = j;
            else if (dhi[k] != j) return berr(nullptr, CFR_ERR_INVALID, "internal: game %d's nodes at depth %d are not contiguous", g, l);
            dhi[k] = j + 1;
            nlev[(size_t)g] = std::max(nlev[(size_t)g], l + 1);
        }
        for (int32_t h = Lo.hlevel[(size_t)l]; h < Lo.hlevel[(size_t)l + 1]; ++h) {
            const int32_t g = game_of_infoset(Lo.h_int2user[(size_t)h]);
            const size_t k = (size_t)g * b->stride + l;
            if (hhi[k] == 0) hlo[k] = h;
            else if (hhi[k] != h) return berr(nullptr, CFR_ERR_INVALID, "internal: game %d's infosets at depth %d are not contiguous", g, l);
            hhi[k] = h + 1;
        }
    }
    // largest games first, so the long ones start early
    std::vector<int32_t> order((size_t)G);
    for (int32_t g = 0; g < G; ++g) order[(size_t)g] = g;
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return b->game_nodes[(size_t)x] > b->game_nodes[(size_t)y]; });
    for (int32_t h = 0; h < b->Hp; ++h) {
        const int32_t na = Lo.qbase[(size_t)h + 1] - Lo.qbase[(size_t)h];
        if (na > 32) return berr(nullptr, CFR_ERR_UNSUPPORTED, "batched solving handles at most 32 actions per infoset");
        b->hp_na = std::max(b->hp_na, na);
    }
    if (!Lo.wide.empty()) return berr(nullptr, CFR_ERR_UNSUPPORTED, "batched solving handles at most 32 actions per node");

    BTRY(balloc(b, &b->dfirst, b->Nd + 1)); BTRY(balloc(b, &b->tfirst, b->Nd + 1)); BTRY(balloc(b, &b->dinfo, b->Nd));
    BTRY(balloc(b, &b->kmask, b->Nd)); BTRY(balloc(b, &b->util64, b->Nt));
    BTRY(balloc(b, &b->qbase, (int64_t)b->H + 1)); BTRY(balloc(b, &b->iplayer, b->H));
    BTRY(balloc(b, &b->sigma, b->Q)); BTRY(balloc(b, &b->sigma064, b->Q));
    BTRY(balloc(b, &b->R, b->Q)); BTRY(balloc(b, &b->S, b->Q));
    BTRY(balloc(b, &b->order, G)); BTRY(balloc(b, &b->dlo, (int64_t)dlo.size())); BTRY(balloc(b, &b->dhi, (int64_t)dhi.size()));
    BTRY(balloc(b, &b->hlo, (int64_t)hlo.size())); BTRY(balloc(b, &b->hhi, (int64_t)hhi.size()));
    BTRY(balloc(b, &b->nlev, G)); BTRY(balloc(b, &b->next, kClasses));
    BTRY(balloc(b, &b->t_start, G)); BTRY(balloc(b, &b->t_end, G)); BTRY(balloc(b, &b->d_iter, 1));

    BTRY(bupload(b, b->dfirst, Lo.dfirst)); BTRY(bupload(b, b->tfirst, Lo.tfirst)); BTRY(bupload(b, b->dinfo, Lo.dinfo));
    BTRY(bupload(b, b->kmask, Lo.kmask));
    BTRY(bupload(b, b->util64, Lo.util));
    BTRY(bupload(b, b->qbase, Lo.qbase)); BTRY(bupload(b, b->iplayer, Lo.iplayer));
    BTRY(bupload(b, b->sigma064, Lo.sigma0));
    BTRY(bupload(b, b->sigma, std::vector<float>(Lo.sigma0.begin(), Lo.sigma0.end())));
    BTRY(bupload(b, b->order, order)); BTRY(bupload(b, b->dlo, dlo)); BTRY(bupload(b, b->dhi, dhi));
    BTRY(bupload(b, b->hlo, hlo)); BTRY(bupload(b, b->hhi, hhi)); BTRY(bupload(b, b->nlev, nlev));
    BCK(cudaMemsetAsync(b->R, 0, sizeof(double) * (size_t)std::max<int64_t>(b->Q, 1), b->stream));
    BCK(cudaMemsetAsync(b->S, 0, sizeof(double) * (size_t)std::max<int64_t>(b->Q, 1), b->stream));
    BCK(cudaMemsetAsync(b->d_iter, 0, sizeof(int64_t), b->stream));
    if (b->H > 0) {
        k_regret_match_all<float><<<(b->H + 255) / 256, 256, 0, b->stream>>>(b->sigma, b->R, b->qbase, b->iplayer, b->H);
        BCK(cudaGetLastError());
    }
    BCK(cudaStreamSynchronize(b->stream));
    BCK(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device));
    b->blocks_per_sm = 0;
    return CFR_OK;
}

// The resident games' images with their slot maps (local slot -> the batch layout's slot, -1 for
// chance), uploaded; the games ordered by footprint class, then largest first, each class's shared
// memory sized for its largest game; the classes' streams and events.
cfr_status load_images(cfr_batch *b, std::vector<GameImage> &imgs) {
    std::vector<int64_t> user2int((size_t)std::max<int64_t>(b->Q, 1), -1);
    for (int64_t qi = 0; qi < b->Q; ++qi) user2int[(size_t)b->q_int2user[(size_t)qi]] = qi;
    std::vector<int32_t> all, cls((size_t)b->G);
    std::vector<int64_t> off((size_t)b->G, 0), bytes((size_t)b->G);
    b->smem_bytes = 0;
    b->cls_smem.assign(kClasses, 0);
    for (int32_t k = 0; k < b->G; ++k) {
        GameImage &img = imgs[(size_t)k];
        int32_t *qmap = img.w.data() + img.w[kImgQmap];
        for (size_t q = 0; q < img.q_int2user.size(); ++q)
            qmap[q] = img.qplayer[q] > 0 ? (int32_t)user2int[(size_t)(b->q_off[(size_t)k] + img.q_int2user[q])] : -1;
        off[(size_t)k] = (int64_t)all.size();
        all.insert(all.end(), img.w.begin(), img.w.end());
        bytes[(size_t)k] = img.bytes;
        int c = 0;
        while (img.bytes > kClassCap[c]) ++c;
        cls[(size_t)k] = c;
        b->cls_smem[(size_t)c] = std::max(b->cls_smem[(size_t)c], img.bytes);
        b->smem_bytes = std::max(b->smem_bytes, img.bytes);
        img = GameImage();
    }
    std::vector<int32_t> order((size_t)b->G);
    for (int32_t g = 0; g < b->G; ++g) order[(size_t)g] = g;
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
        return cls[(size_t)x] != cls[(size_t)y] ? cls[(size_t)x] < cls[(size_t)y] : bytes[(size_t)x] > bytes[(size_t)y];
    });
    b->cls_off.assign(kClasses + 1, 0);
    for (int32_t g = 0; g < b->G; ++g) ++b->cls_off[(size_t)cls[(size_t)g] + 1];
    for (int c = 0; c < kClasses; ++c) b->cls_off[(size_t)c + 1] += b->cls_off[(size_t)c];
    BTRY(balloc(b, &b->images, (int64_t)all.size()));
    BTRY(balloc(b, &b->img_off, (int64_t)b->G));
    BTRY(bupload(b, b->images, all));
    BTRY(bupload(b, b->img_off, off));
    BTRY(bupload(b, b->order, order));
    // the kernel's limit is every batch's cap (a batch of smaller games must not lower it for another)
    BCK(cudaFuncSetAttribute(smem_kernel_for(b), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap));
    BCK(cudaEventCreateWithFlags(&b->cls_fork, cudaEventDisableTiming));
    for (int c = 0; c < kClasses; ++c) {
        BCK(cudaStreamCreateWithFlags(&b->aux[c], cudaStreamNonBlocking));
        BCK(cudaEventCreateWithFlags(&b->cls_join[c], cudaEventDisableTiming));
    }
    b->threads = 128;
    return CFR_OK;
}

}  // namespace

extern "C" {

cfr_status cfr_batch_load(const cfr_game_desc *games, int32_t num_games, const cfr_config *c, cfr_batch **out) {
    if (!out) return berr(nullptr, CFR_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!games || num_games < 1) return berr(nullptr, CFR_ERR_INVALID, "need at least one game");
    cfr_config cfg;
    if (c) cfg = *c; else cfr_config_init(&cfg);
    if (cfg.variant < CFR_VANILLA || cfg.variant > CFR_DISCOUNTED)
        return berr(nullptr, CFR_ERR_INVALID, "variant %d unknown", cfg.variant);
    if (cfg.precision != CFR_FP32)
        return berr(nullptr, CFR_ERR_UNSUPPORTED, "batched solving runs in FP32 mode (FP64 accumulators)");
    if (cfg.update_mode != CFR_SIMULTANEOUS && cfg.update_mode != CFR_ALTERNATING)
        return berr(nullptr, CFR_ERR_INVALID, "update_mode %d unknown", cfg.update_mode);
    if (cfg.avg_weight == CFR_AVG_DEFAULT) cfg.avg_weight = cfg.variant == CFR_VANILLA ? CFR_AVG_UNIFORM : CFR_AVG_LINEAR;
    if (cfg.avg_weight != CFR_AVG_UNIFORM && cfg.avg_weight != CFR_AVG_LINEAR)
        return berr(nullptr, CFR_ERR_INVALID, "avg_weight %d unknown", cfg.avg_weight);
    if ((cfg.dev_alloc == nullptr) != (cfg.dev_free == nullptr))
        return berr(nullptr, CFR_ERR_INVALID, "dev_alloc and dev_free must both be set or both NULL");

    std::unique_ptr<cfr_batch> b(new cfr_batch());
    b->cfg = cfg;
    b->n_games = num_games;
    b->split_nodes = cfg.batch_split_nodes == 0 ? kBatchSplitDefault : cfg.batch_split_nodes;
    std::vector<cfr_game_desc> small, large;
    std::vector<GameImage> imgs;
    b->part.assign((size_t)num_games, 0);
    b->idx.assign((size_t)num_games, 0);
    for (int32_t i = 0; i < num_games; ++i) {
        bool big = b->split_nodes > 0 && games[i].num_nodes >= b->split_nodes;
        GameImage img;
        if (!big) {                                    // resident in shared memory if its image fits
            bool fits = false;
            std::string err;
            const cfr_status st = make_image(games[i], img, &fits, &err);
            if (st != CFR_OK) return berr(nullptr, st, "game %d: %s", i, err.c_str());
            big = !fits;
        }
        b->part[(size_t)i] = big;
        b->idx[(size_t)i] = (int32_t)(big ? large.size() : small.size());
        (big ? large : small).push_back(games[i]);
        if (!big) imgs.push_back(std::move(img));
    }
    b->G = (int32_t)small.size();
    std::vector<int32_t> parent, action, infoset, nact;
    std::vector<int8_t> player;
    std::vector<double> cprob, util;
    cfr_status st = CFR_OK;
    if (!large.empty()) {
        // the forest part: the large games combined in order, loaded by the single-game solver
        cfr_batch tmp;
        st = combine(large.data(), (int32_t)large.size(), &tmp, parent, action, infoset, player, nact, cprob, util);
        if (st != CFR_OK) return st;
        b->big_q_off = tmp.q_off;
        b->big_nodes = tmp.game_nodes;
        cfr_game_desc all{};
        all.num_nodes = tmp.node_off.back();
        all.parent = parent.data(); all.action = action.data(); all.infoset = infoset.data();
        all.num_infosets = (int32_t)tmp.h_off.back();
        all.infoset_player = player.data(); all.infoset_num_actions = nact.data();
        all.chance_prob = cprob.data(); all.num_chance_prob = (int64_t)cprob.size(); all.utility = util.data();
        BDeviceGuard dg0(cfg.device);
        if (!dg0.ok) return berr(nullptr, CFR_ERR_CUDA, "cannot select CUDA device %d", cfg.device);
        cudaError_t e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);
        for (cudaEvent_t *ev : {&b->ev_fork, &b->ev_join})
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
        for (cudaEvent_t *ev : {&b->ev_b0, &b->ev_b1})
            if (e == cudaSuccess) e = cudaEventCreate(ev);
        if (e != cudaSuccess) {
            cudaGetLastError();
            cfr_batch_free(b.release());
            return berr(nullptr, CFR_ERR_CUDA, "stream/event creation: %s", cudaGetErrorString(e));
        }
        cfr_config fc = cfg;
        fc.cuda_stream = b->side;
        st = cfrgb::load_tree_impl(&all, &fc, true, &b->big);
        if (st != CFR_OK) {
            std::string msg = cfr_last_error(nullptr);
            cfr_batch_free(b.release());
            return berr(nullptr, st, "%s", msg.c_str());
        }
        parent.clear(); action.clear(); infoset.clear(); player.clear(); nact.clear(); cprob.clear(); util.clear();
    }
    if (b->G == 0) {
        BDeviceGuard dg1(cfg.device);
        cudaGetDevice(&b->device);
        b->stream = static_cast<cudaStream_t>(cfg.cuda_stream);
        *out = b.release();
        return CFR_OK;
    }
    st = combine(small.data(), b->G, b.get(), parent, action, infoset, player, nact, cprob, util);
    if (st != CFR_OK) { cfr_batch_free(b.release()); return st; }
    cfr_game_desc all{};
    all.num_nodes = b->node_off.back();
    all.parent = parent.data(); all.action = action.data(); all.infoset = infoset.data();
    all.num_infosets = (int32_t)b->h_off.back();
    all.infoset_player = player.data(); all.infoset_num_actions = nact.data();
    all.chance_prob = cprob.data(); all.num_chance_prob = (int64_t)cprob.size(); all.utility = util.data();
    std::unique_ptr<Layout> Lo(new Layout());
    std::string err;
    st = build_layout(&all, Lo.get(), &err, false, true);
    if (st != CFR_OK) { cfr_batch_free(b.release()); return berr(nullptr, st, "%s", err.c_str()); }
    parent.clear(); parent.shrink_to_fit(); action.clear(); action.shrink_to_fit();
    infoset.clear(); infoset.shrink_to_fit(); util.clear(); util.shrink_to_fit();

    BDeviceGuard dg(cfg.device);
    if (!dg.ok) { cfr_batch_free(b.release()); return berr(nullptr, CFR_ERR_CUDA, "cannot select CUDA device %d", cfg.device); }
    cudaGetDevice(&b->device);
    b->stream = static_cast<cudaStream_t>(cfg.cuda_stream);
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cfr_batch_free(b.release());
        return berr(nullptr, CFR_ERR_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
    }
    st = load_batch(b.get(), *Lo);
    if (st == CFR_OK) st = load_images(b.get(), imgs);
    if (st != CFR_OK) {
        std::string msg = b->err.empty() ? g_batch_err : b->err;
        cfr_batch_free(b.release());
        return berr(nullptr, st, "%s", msg.c_str());
    }
    *out = b.release();
    return CFR_OK;
}

cfr_status cfr_batch_iterate(cfr_batch *b, int32_t n) {
    BTRY(busable(b));
    if (n < 0) return berr(b, CFR_ERR_INVALID, "n must be >= 0");
    if (n == 0) return CFR_OK;
    BDeviceGuard dg(b->device);
    if (b->big) {                                      // the forest part, on its stream, after earlier work
        BCK(cudaEventRecord(b->ev_fork, b->stream));
        BCK(cudaStreamWaitEvent(b->side, b->ev_fork, 0));
        BCK(cudaEventRecord(b->ev_b0, b->side));
        if (cfr_iterate(b->big, n) != CFR_OK) return berr(b, CFR_ERR_CUDA, "forest part: %s", cfr_last_error(b->big));
        BCK(cudaEventRecord(b->ev_b1, b->side));
        BCK(cudaEventRecord(b->ev_join, b->side));
        b->big_timed = true;
    }
    if (b->G > 0) {
        if (!b->graph_exec || b->graph_K != n) BTRY(build_batch_graph(b, n));
        BCK(cudaGraphLaunch(b->graph_exec, b->stream));
        b->kernel_launches += 2;
    }
    if (b->big) BCK(cudaStreamWaitEvent(b->stream, b->ev_join, 0));
    b->iteration += n;
    b->last_K = n;
    return CFR_OK;
}

cfr_status cfr_batch_set_tuning(cfr_batch *b, const cfr_batch_tuning *t) {
    BTRY(busable(b));
    if (!t || t->threads_per_block < 32 || t->threads_per_block > 256 || t->threads_per_block % 32 || t->blocks_per_sm < 0)
        return berr(b, CFR_ERR_INVALID, "threads_per_block must be a multiple of 32 in [32, 256], blocks_per_sm >= 0");
    BDeviceGuard dg(b->device);
    if (b->G > 0 && occupancy_min(b, t->threads_per_block) < 1)
        return berr(b, CFR_ERR_INVALID, "no block of %d threads fits an SM", t->threads_per_block);
    b->threads = t->threads_per_block;
    b->blocks_per_sm = t->blocks_per_sm;
    b->tuned = true;
    if (b->graph_exec) { cudaGraphExecDestroy(b->graph_exec); b->graph_exec = nullptr; b->graph_K = -1; }
    return CFR_OK;
}

cfr_status cfr_batch_autotune(cfr_batch *b, int32_t trial_iterations, cfr_batch_tuning *chosen, double *best_us) {
    BTRY(busable(b));
    if (trial_iterations < 1) return berr(b, CFR_ERR_INVALID, "trial_iterations must be >= 1");
    if (b->G == 0) {                                   // only the forest part: nothing to tune
        if (chosen) { chosen->threads_per_block = b->threads; chosen->blocks_per_sm = b->blocks_per_sm; }
        if (best_us) *best_us = 0.0;
        return CFR_OK;
    }
    BDeviceGuard dg(b->device);
    // the trials run real iterations on a snapshot of the state, restored afterwards
    if (!b->snapR) {
        BTRY(balloc(b, &b->snapR, b->Q));
        BTRY(balloc(b, &b->snapS, b->Q));
        BTRY(balloc(b, &b->snapSigma, b->Q));
    }
    const size_t q8 = sizeof(double) * (size_t)std::max<int64_t>(b->Q, 1), q4 = sizeof(float) * (size_t)std::max<int64_t>(b->Q, 1);
    int64_t T0 = 0;
    BCK(cudaStreamSynchronize(b->stream));
    BCK(cudaMemcpy(&T0, b->d_iter, sizeof T0, cudaMemcpyDeviceToHost));
    BCK(cudaMemcpy(b->snapR, b->R, q8, cudaMemcpyDeviceToDevice));
    BCK(cudaMemcpy(b->snapS, b->S, q8, cudaMemcpyDeviceToDevice));
    BCK(cudaMemcpy(b->snapSigma, b->sigma, q4, cudaMemcpyDeviceToDevice));
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    double best = 1e300;
    int best_threads = b->threads, best_bps = b->blocks_per_sm;
    for (int threads : {64, 128, 256}) {
        if (occupancy_min(b, threads) < 1) continue;
        const int occ = occupancy_max(b, threads);
        for (int bps : {1, 2, 4, 8, 16}) {
            if (bps > occ) break;
            BCK(cudaMemcpy(b->d_iter, &T0, sizeof T0, cudaMemcpyHostToDevice));
            BCK(cudaEventRecord(e0, b->stream));
            BTRY(enqueue_batch(b, b->stream, trial_iterations, threads, bps));
            BCK(cudaEventRecord(e1, b->stream));
            BCK(cudaEventSynchronize(e1));
            float ms = 0.f;
            BCK(cudaEventElapsedTime(&ms, e0, e1));
            const double us = 1e3 * ms / trial_iterations;
            if (us < best) { best = us; best_threads = threads; best_bps = bps; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    BCK(cudaMemcpy(b->R, b->snapR, q8, cudaMemcpyDeviceToDevice));
    BCK(cudaMemcpy(b->S, b->snapS, q8, cudaMemcpyDeviceToDevice));
    BCK(cudaMemcpy(b->sigma, b->snapSigma, q4, cudaMemcpyDeviceToDevice));
    BCK(cudaMemcpy(b->d_iter, &T0, sizeof T0, cudaMemcpyHostToDevice));
    b->threads = best_threads;
    b->blocks_per_sm = best_bps;
    b->tuned = true;
    if (b->graph_exec) { cudaGraphExecDestroy(b->graph_exec); b->graph_exec = nullptr; b->graph_K = -1; }
    if (chosen) { chosen->threads_per_block = best_threads; chosen->blocks_per_sm = best_bps; }
    if (best_us) *best_us = best;
    return CFR_OK;
}

cfr_status cfr_batch_game_times(cfr_batch *b, double *us_per_iteration, int32_t len) {
    BTRY(busable(b));
    if (!us_per_iteration || len < b->n_games) return berr(b, CFR_ERR_INVALID, "output needs %d entries", b->n_games);
    if (b->last_K <= 0) return berr(b, CFR_ERR_STATE, "no cfr_batch_iterate call yet");
    BDeviceGuard dg(b->device);
    BTRY(bsync(b));
    std::vector<unsigned long long> t0((size_t)std::max(b->G, 1)), t1((size_t)std::max(b->G, 1));
    if (b->G > 0) {
        BCK(cudaMemcpy(t0.data(), b->t_start, sizeof(unsigned long long) * (size_t)b->G, cudaMemcpyDeviceToHost));
        BCK(cudaMemcpy(t1.data(), b->t_end, sizeof(unsigned long long) * (size_t)b->G, cudaMemcpyDeviceToHost));
    }
    float big_ms = 0.f;
    if (b->big && b->big_timed) BCK(cudaEventElapsedTime(&big_ms, b->ev_b0, b->ev_b1));
    for (int32_t g = 0; g < b->n_games; ++g) {
        const size_t k = (size_t)b->idx[(size_t)g];
        us_per_iteration[g] = b->part[(size_t)g] ? 1e3 * (double)big_ms / b->last_K     // the forest advances together
                                                 : (double)(t1[k] - t0[k]) * 1e-3 / b->last_K;
    }
    return CFR_OK;
}

cfr_status cfr_batch_exploitability(cfr_batch *b, double *nash_conv, int32_t len) {
    BTRY(busable(b));
    if (!nash_conv || len < b->n_games) return berr(b, CFR_ERR_INVALID, "output needs %d entries", b->n_games);
    if (!b->single_level)
        return berr(b, CFR_ERR_UNSUPPORTED, "the GPU best response needs every infoset at a single depth");
    BDeviceGuard dg(b->device);
    std::vector<double> big_nc(b->big_nodes.size());
    if (b->big) {
        BTRY(bsync(b));
        if (cfrgb::root_nash_conv(b->big, big_nc.data(), (int32_t)big_nc.size()) != CFR_OK)
            return berr(b, CFR_ERR_CUDA, "forest part: %s", cfr_last_error(b->big));
    }
    std::vector<double> small_nc((size_t)b->G);
    BTRY(small_exploitability(b, small_nc.data()));
    for (int32_t g = 0; g < b->n_games; ++g)
        nash_conv[g] = b->part[(size_t)g] ? big_nc[(size_t)b->idx[(size_t)g]] : small_nc[(size_t)b->idx[(size_t)g]];
    return CFR_OK;
}

}  // extern "C"

namespace {

// NashConv of every game of the persistent part.
cfr_status small_exploitability(cfr_batch *b, double *nash_conv) {
    if (b->G == 0) return CFR_OK;
    if (!b->avg) {
        BTRY(balloc(b, &b->avg, b->Q)); BTRY(balloc(b, &b->cfv, b->Q)); BTRY(balloc(b, &b->preach, b->Nd));
        BTRY(balloc(b, &b->val, b->Nd)); BTRY(balloc(b, &b->astar, b->H)); BTRY(balloc(b, &b->br_out, 2 * (int64_t)b->G));
    }
    if (b->H > 0) {
        k_average<<<(b->H + 255) / 256, 256, 0, b->stream>>>(b->S, b->sigma064, b->qbase, b->iplayer, b->avg, b->H);
        BCK(cudaGetLastError());
    }
    BCK(cudaMemsetAsync(b->cfv, 0, sizeof(double) * (size_t)std::max<int64_t>(b->Q, 1), b->stream));
    BCK(cudaMemsetAsync(b->next, 0, sizeof(int32_t), b->stream));
    DevBR br;
    br.dfirst = b->dfirst; br.tfirst = b->tfirst; br.dinfo = b->dinfo; br.kmask = b->kmask; br.wbits = nullptr;
    br.util = b->util64; br.qbase = b->qbase; br.iplayer = b->iplayer; br.avg = b->avg;
    br.preach = b->preach; br.val = b->val; br.cfv = b->cfv; br.astar = b->astar;
    const int grid = std::max(1, std::min(b->G, 8 * b->sms));
    k_batch_br<<<grid, 256, 0, b->stream>>>(br, batch_desc(b), b->br_out);
    BCK(cudaGetLastError());
    std::vector<double> v((size_t)2 * b->G);
    BCK(cudaMemcpyAsync(v.data(), b->br_out, sizeof(double) * v.size(), cudaMemcpyDeviceToHost, b->stream));
    BTRY(bsync(b));
    for (int32_t g = 0; g < b->G; ++g) nash_conv[g] = v[(size_t)2 * g] + v[(size_t)2 * g + 1];
    return CFR_OK;
}

}  // namespace

extern "C" {

// Per game of the persistent part: R and S (and the average strategy) in the game's own infoset-major
// order.
static cfr_status small_slots(cfr_batch *b, int32_t game, const double *dev, double *out, int64_t len) {
    const int64_t q0 = b->q_off[(size_t)game], q1 = b->q_off[(size_t)game + 1];
    if (!out || len < q1 - q0) return berr(b, CFR_ERR_INVALID, "output needs %lld entries", (long long)(q1 - q0));
    std::vector<double> all((size_t)std::max<int64_t>(b->Q, 1));
    BCK(cudaMemcpy(all.data(), dev, sizeof(double) * (size_t)b->Q, cudaMemcpyDeviceToHost));
    for (int64_t qi = 0; qi < b->Q; ++qi) {
        const int64_t qu = b->q_int2user[(size_t)qi];
        if (qu >= q0 && qu < q1) out[qu - q0] = all[(size_t)qi];
    }
    return CFR_OK;
}

// A forest-part game's slice of a whole-forest array (the forest's own caller numbering).
static cfr_status big_slice(cfr_batch *b, int32_t k, const std::vector<double> &all, double *out, int64_t len) {
    const int64_t q0 = b->big_q_off[(size_t)k], q1 = b->big_q_off[(size_t)k + 1];
    if (!out || len < q1 - q0) return berr(b, CFR_ERR_INVALID, "output needs %lld entries", (long long)(q1 - q0));
    std::copy(all.begin() + q0, all.begin() + q1, out);
    return CFR_OK;
}

cfr_status cfr_batch_get_state(cfr_batch *b, int32_t game, double *cum_regret, double *strat_sum, int64_t len,
                               int64_t *iteration) {
    BTRY(busable(b));
    if (game < 0 || game >= b->n_games) return berr(b, CFR_ERR_INVALID, "game %d out of range", game);
    BDeviceGuard dg(b->device);
    BTRY(bsync(b));
    const int32_t k = b->idx[(size_t)game];
    if (b->part[(size_t)game]) {
        const int64_t Qb = b->big_q_off.back();
        std::vector<double> R((size_t)std::max<int64_t>(Qb, 1)), S((size_t)std::max<int64_t>(Qb, 1));
        if (cfr_get_state(b->big, R.data(), S.data(), nullptr, std::max<int64_t>(Qb, 1), nullptr, 0, nullptr) != CFR_OK)
            return berr(b, CFR_ERR_CUDA, "forest part: %s", cfr_last_error(b->big));
        if (cum_regret) BTRY(big_slice(b, k, R, cum_regret, len));
        if (strat_sum) BTRY(big_slice(b, k, S, strat_sum, len));
    } else {
        if (cum_regret) BTRY(small_slots(b, k, b->R, cum_regret, len));
        if (strat_sum) BTRY(small_slots(b, k, b->S, strat_sum, len));
    }
    if (iteration) *iteration = b->iteration;
    return CFR_OK;
}

cfr_status cfr_batch_average_strategy(cfr_batch *b, int32_t game, double *out, int64_t len) {
    BTRY(busable(b));
    if (game < 0 || game >= b->n_games) return berr(b, CFR_ERR_INVALID, "game %d out of range", game);
    BDeviceGuard dg(b->device);
    BTRY(bsync(b));
    const int32_t k = b->idx[(size_t)game];
    if (b->part[(size_t)game]) {
        const int64_t Qb = b->big_q_off.back();
        std::vector<double> A((size_t)std::max<int64_t>(Qb, 1));
        if (cfr_average_strategy(b->big, A.data(), std::max<int64_t>(Qb, 1)) != CFR_OK)
            return berr(b, CFR_ERR_CUDA, "forest part: %s", cfr_last_error(b->big));
        return big_slice(b, k, A, out, len);
    }
    if (!b->avg) BTRY(balloc(b, &b->avg, b->Q));
    if (b->H > 0) {
        k_average<<<(b->H + 255) / 256, 256, 0, b->stream>>>(b->S, b->sigma064, b->qbase, b->iplayer, b->avg, b->H);
        BCK(cudaGetLastError());
    }
    BTRY(bsync(b));
    return small_slots(b, k, b->avg, out, len);
}

cfr_status cfr_batch_get_info(const cfr_batch *b, cfr_batch_info *info) {
    if (!b || !info) return berr(nullptr, CFR_ERR_INVALID, "batch or info is NULL");
    std::memset(info, 0, sizeof *info);
    info->num_games = b->n_games;
    cfr_info fi{};
    if (b->big) cfr_get_info(b->big, &fi);
    info->num_nodes = b->N + fi.num_nodes;
    info->num_decision = b->Nd + fi.num_decision;
    info->num_q = b->Q + fi.num_q;
    info->forest_games = (int32_t)b->big_nodes.size();
    info->forest_nodes = fi.num_nodes;
    info->split_nodes = b->split_nodes;
    info->smem_bytes = b->smem_bytes;
    info->forest_bytes_per_iteration = fi.bytes_per_iteration;
    info->forest_head_depths = fi.head_depths;
    info->device_bytes = b->device_bytes + fi.device_bytes;
    info->iteration = b->iteration;
    info->threads_per_block = b->threads;
    info->blocks_per_sm = b->blocks_per_sm;
    info->grid = 0;
    for (int c = 0; c < kClasses && b->G > 0; ++c)
        if (class_games(b, c) > 0) info->grid += grid_of(b, c, b->threads, b->blocks_per_sm);
    info->tuned = b->tuned;
    info->kernel_launches = b->kernel_launches + fi.kernel_launches;
    return CFR_OK;
}

const char *cfr_batch_last_error(const cfr_batch *b) { return b ? b->err.c_str() : g_batch_err.c_str(); }

void cfr_batch_free(cfr_batch *b) {
    if (!b) return;
    BDeviceGuard dg(b->device);
    if (b->stream || b->cap) cudaStreamSynchronize(b->stream);
    if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
    if (b->side) cudaStreamSynchronize(b->side);
    if (b->big) cfr_free(b->big);
    for (void *p : b->blocks) {
        if (b->cfg.dev_free) b->cfg.dev_free(p, b->cfg.alloc_ctx);
        else cudaFree(p);
    }
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->side) cudaStreamDestroy(b->side);
    for (cudaEvent_t ev : {b->ev_fork, b->ev_join, b->ev_b0, b->ev_b1, b->cls_fork})
        if (ev) cudaEventDestroy(ev);
    for (int c = 0; c < kClasses; ++c) {
        if (b->aux[c]) { cudaStreamSynchronize(b->aux[c]); cudaStreamDestroy(b->aux[c]); }
        if (b->cls_join[c]) cudaEventDestroy(b->cls_join[c]);
    }
    delete b;
}

}  // extern "C"
