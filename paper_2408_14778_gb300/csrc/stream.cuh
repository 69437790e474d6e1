// Bottom-up step of a large depth (FP32 mode) with its inputs streamed into shared memory by TMA.
//
// The per-depth kernel k_bottomup gives each thread a chain of dependent global loads (node fields,
// then child values and strategy entries), so the bytes in flight per SM - and with them the HBM
// bandwidth - are capped by occupancy.  Here one producer warp per block moves tiles of kSBN
// consecutive nodes into a ring of shared-memory stages with bulk copies (cp.async.bulk, completion
// counted in bytes on a "full" mbarrier per stage): the node fields (qp, kmask, dfirst, tfirst), both
// counterfactual reaches, and the contiguous ranges of the tile's child values - the terminal
// utilities and the decision children's values.  Eight consumer warps wait for a stage, handle two
// nodes per thread exactly as bu_node does (strategy entries are gathered from global memory, mostly
// L2 hits), and release the stage on its "empty" mbarrier.  A tile whose child ranges exceed the stage
// reads its child values from global memory instead.  Nodes with more than 32 actions are left to
// k_bottomup_wide.
//
// Every wait is bounded by kWaitNs of %globaltimer (and a poll count).  A wait that expires sets *err,
// raises the block's abort flag (which ends the other waits), and the producer waits - bounded again -
// for the copies it issued before the block exits; the host turns *err into CFR_ERR_TIMEOUT.
#pragma once

#include <cstdint>

#include "kernels.cuh"
#include "tail_tiles.hpp"

namespace cfrgb {
namespace {   // device code: internal to each translation unit that includes it

constexpr int kSBN = 512;                  // nodes per tile
constexpr int kSBT = 3072;                 // staged terminal-child values per tile
constexpr int kSBD = 2048;                 // staged decision-child values per tile
constexpr int kSBStages = 2;
constexpr int kSBConsumerWarps = 8;        // 256 consumer threads, two nodes each
constexpr int kSBThreads = 32 * (kSBConsumerWarps + 1);
constexpr uint64_t kWaitNs = 1000000000ull;   // 1 s
constexpr uint32_t kWaitPolls = 1u << 26;

struct SBStage {                           // element 0 of each array is the 16-byte-aligned copy start
    uint32_t qp[kSBN + 4], km[kSBN + 4];
    int32_t df[kSBN + 8], tf[kSBN + 8];
    float r1[kSBN + 4], r2[kSBN + 4];
    float tval[kSBT + 4], dval[kSBD + 4];
};

struct SBTile {
    int32_t j0, n, o;                      // first node, node count, offset of node j0 in the field arrays
    int32_t tal, dal;                      // global index of tval[0] / dval[0]
    int32_t staged;                        // child values in tval/dval (else global memory)
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits until the phase with the given parity has completed.  False when the wait expired or the
// block is aborting (abort != nullptr and *abort set).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort) {
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t i = 0; i < kWaitPolls; ++i) {
        if (mbar_test(bar, parity)) return true;
        if (abort && *abort) return false;
        if ((i & 255u) == 255u && globaltimer_ns() - t0 > kWaitNs) return false;
    }
    return false;
}

// 1-D bulk copy global -> shared: addresses 16-byte aligned, bytes a multiple of 16.  The streamed node
// fields, reaches and utilities are read once per pass: they go into L2 marked evict-first, so that the
// strategy entries and r~ that the kernels gather and scatter meanwhile stay resident.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
                 : "memory");
}

// Elements [a, b) of a 4-byte array widened to 16-byte boundaries: first index, and the bytes.  The
// solver's arrays are allocated in multiples of 256 bytes, so the widened end stays inside them.
__device__ __forceinline__ int32_t widen16(int32_t a, int32_t b, uint32_t *bytes) {
    const int32_t a0 = a & ~3, b0 = (b + 3) & ~3;
    *bytes = (uint32_t)(b0 - a0) * 4u;
    return a0;
}

// Producer: the copies of nodes [j0, j0 + n) into stage st; r = {tfirst[j0], tfirst[j0 + n],
// dfirst[j0], dfirst[j0 + n]} (loaded a tile ahead).
__device__ __forceinline__ void sb_issue(const DevTree<float> &t, int32_t j0, int32_t n, const int32_t *r, SBStage *st,
                                         SBTile *ti, uint64_t *full) {
    uint32_t bf, bd, btv = 0, bdv = 0;
    const int32_t jal = widen16(j0, j0 + n, &bf);
    widen16(j0, j0 + n + 1, &bd);
    const int32_t ts = r[0], te = r[1], ds = r[2], de = r[3];
    const int32_t tal = widen16(ts, te, &btv);
    const int32_t dal = widen16(ds, de, &bdv);
    const bool staged = btv <= 4u * (kSBT + 4) && bdv <= 4u * (kSBD + 4);
    ti->j0 = j0; ti->n = n; ti->o = j0 - jal;
    ti->tal = tal; ti->dal = dal; ti->staged = staged;
    uint32_t total = 4 * bf + 2 * bd;
    if (staged) total += btv + bdv;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive_expect_tx(full, total);
    bulk_g2s(st->qp, t.qp + jal, bf, full);
    bulk_g2s(st->km, t.kmask + jal, bf, full);
    bulk_g2s(st->df, t.dfirst + jal, bd, full);
    bulk_g2s(st->tf, t.tfirst + jal, bd, full);
    bulk_g2s(st->r1, t.reach1 + jal, bf, full);
    bulk_g2s(st->r2, t.reach2 + jal, bf, full);
    if (staged) {
        if (btv) bulk_g2s(st->tval, t.util + tal, btv, full);
        if (bdv) bulk_g2s(st->dval, t.u + dal, bdv, full);
    }
}

// Consumer: bottom-up step of nodes i and i2 (i2 may be past the tile) of a staged tile, with the loads
// of both nodes issued before either is used.  Per node the operations and their order are bu_node's.
// NA: the unrolled action count (at least the depth's largest action count for full unrolling; nodes
// with more actions take bu_node's loop).
template <int NA>
__device__ __forceinline__ void sb_nodes(const DevTree<float> &t, const SBStage &st, const SBTile &ti, int32_t i,
                                         int32_t i2) {
    const int32_t ii[2] = {i, i2};
    float v[2][NA], s[2][NA];
    int na[2], pl[2];
    int32_t qb[2], c0[2], t0[2];
    uint32_t m[2];
    bool go[2], allterm[2];
#pragma unroll
    for (int x = 0; x < 2; ++x) {
        go[x] = false;
        na[x] = 0;
        if (ii[x] >= ti.n) continue;
        const int32_t k = ti.o + ii[x];
        const uint32_t w = st.qp[k];
        if (qp_wide(w)) continue;
        go[x] = true;
        qb[x] = qp_base(w);
        pl[x] = qp_player(w);
        m[x] = st.km[k];
        c0[x] = st.df[k];
        t0[x] = st.tf[k];
        const int32_t nd = st.df[k + 1] - c0[x];
        allterm[x] = nd == 0;
        na[x] = nd + __popc(m[x]);
    }
    // general path (more than NA actions): one node at a time, as bu_node's loop
#pragma unroll
    for (int x = 0; x < 2; ++x) {
        if (!go[x] || na[x] <= NA) continue;
        const int32_t k = ti.o + ii[x];
        const float *tv = ti.staged ? st.tval + (t0[x] - ti.tal) : t.util + t0[x];
        const float *dv = ti.staged ? st.dval + (c0[x] - ti.dal) : t.u + c0[x];
        float ud = 0.f;
        int kt = 0, kd = 0;
        for (int a = 0; a < na[x]; ++a) {
            const float val = ((m[x] >> a) & 1u) ? tv[kt++] : dv[kd++];
            ud = madd(ud, __ldg(t.sigma + qb[x] + a), val);
        }
        t.u[ti.j0 + ii[x]] = ud;
        go[x] = false;
        if (!collects(t, pl[x])) continue;
        const float wr = pl[x] == 1 ? st.r1[k] : -st.r2[k];
        if (wr == 0.f) continue;
        kt = kd = 0;
        for (int a = 0; a < na[x]; ++a) {
            const float val = ((m[x] >> a) & 1u) ? tv[kt++] : dv[kd++];
            atomicAdd(&t.inst[qb[x] + a], wr * (val - ud));
        }
    }
#pragma unroll
    for (int x = 0; x < 2; ++x) {
        if (!go[x]) continue;
        const float *tv = ti.staged ? st.tval + (t0[x] - ti.tal) : t.util + t0[x];
        if (allterm[x]) {                              // terminal children only (the deepest depth)
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                if (a < na[x]) {
                    v[x][a] = tv[a];
                    s[x][a] = __ldg(t.sigma + qb[x] + a);
                }
            }
        } else {
            const float *dv = ti.staged ? st.dval + (c0[x] - ti.dal) : t.u + c0[x];
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                if (a < na[x]) {
                    const int kt = __popc(m[x] & ((1u << a) - 1u));   // terminal children before action a
                    const float *src = ((m[x] >> a) & 1u) ? tv + kt : dv + (a - kt);
                    v[x][a] = *src;
                    s[x][a] = __ldg(t.sigma + qb[x] + a);
                }
            }
        }
    }
#pragma unroll
    for (int x = 0; x < 2; ++x) {
        if (!go[x]) continue;
        const int32_t k = ti.o + ii[x];
        float ud = 0.f;
#pragma unroll
        for (int a = 0; a < NA; ++a)
            if (a < na[x]) ud = madd(ud, s[x][a], v[x][a]);
        t.u[ti.j0 + ii[x]] = ud;
        if (!collects(t, pl[x])) continue;
        const float wr = pl[x] == 1 ? st.r1[k] : -st.r2[k];
        if (wr == 0.f) continue;
#pragma unroll
        for (int a = 0; a < NA; ++a)
            if (a < na[x]) atomicAdd(&t.inst[qb[x] + a], wr * (v[x][a] - ud));
    }
}

// Named barrier 1 over the NT consumer threads (the producer warp does not take part).
template <int NT = kSBConsumerWarps * 32>
__device__ __forceinline__ void consumers_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
}

// Named barrier 1 over the NT consumer threads that also returns, to every one of them, whether any
// passed true.
template <int NT = kSBConsumerWarps * 32>
__device__ __forceinline__ bool consumers_any(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred p, 1, %2, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(NT)
        : "memory");
    return r != 0;
}

// ---- the producer/consumer pipeline --------------------------------------------------------------
// P supplies the tile work: P::Stage and P::Tile (shared-memory stage and its description),
// P::kStages, P::kConsumerWarps, ntiles(), prefetch(tile, meta) (loads P::kMetaWords words of P::Meta
// describing a tile, one tile ahead), issue(tile, meta, stage, tile info, full barrier) run by one
// producer thread (the first lane of warp P::kConsumerWarps), and consume(stage, tile info, consumer
// thread index) run by each of the P::kConsumerWarps * 32 consumer threads.  P::kConsumerSync: consume() synchronises the consumer threads, so they agree (one
// barrier with an OR) on whether to take each tile or stop.  Block b takes tiles b, b + gridDim.x, ...  Returns true in consumer threads once their
// tiles are done (false in the producer warp), so a kernel may continue with other consumer work.
template <class P>
__device__ __forceinline__ bool run_pipeline(const P &p, int *err) {
    using Stage = typename P::Stage;
    constexpr int S = P::kStages;
    extern __shared__ __align__(128) unsigned char pipe_smem[];
    Stage *stage = reinterpret_cast<Stage *>(pipe_smem);
    __shared__ __align__(8) uint64_t full[S], empty[S];
    __shared__ typename P::Tile tinfo[S];
    __shared__ int abort_flag;
    constexpr int CW = P::kConsumerWarps;
    const int32_t ntiles = p.ntiles();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], CW);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    volatile int *abort = &abort_flag;
    if (warp == CW) {                                                 // producer warp
        if (lane != 0) return false;
        int32_t issued = 0;
        typename P::Meta meta[2][P::kMetaWords];
        if ((int32_t)blockIdx.x < ntiles) p.prefetch(blockIdx.x, meta[0]);
        for (int32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++issued) {
            const int s = issued % S;
            // the next tile's description is loaded while this one waits for its stage
            if (tile + (int32_t)gridDim.x < ntiles) p.prefetch(tile + gridDim.x, meta[(issued + 1) & 1]);
            if (issued >= S && !mbar_wait(&empty[s], (uint32_t)((issued / S - 1) & 1), abort)) {
                if (!*abort) { atomicExch(err, 1); *abort = 1; }
                break;
            }
            p.issue(tile, meta[issued & 1], &stage[s], &tinfo[s], &full[s]);
        }
        // the block must not exit with copies in flight: wait for the last use of each stage
        for (int s = 0; s < S && s < issued; ++s) {
            const int32_t last = s + ((issued - 1 - s) / S) * S;
            if (!mbar_wait(&full[s], (uint32_t)((last / S) & 1), nullptr)) atomicExch(err, 1);
        }
        return false;
    }
    int32_t k = 0;
    for (int32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++k) {
        const int s = k % S;
        const bool ok = mbar_wait(&full[s], (uint32_t)((k / S) & 1), abort);
        if (!ok && !*abort) { atomicExch(err, 1); *abort = 1; }
        if constexpr (P::kConsumerSync) {
            // consume() synchronises the consumer threads: they must all take the tile or all stop
            if (consumers_any<CW * 32>(!ok || *abort)) break;
        } else if (!ok) {
            break;
        }
        p.consume(stage[s], tinfo[s], (int)threadIdx.x);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
    return true;
}

// Bottom-up at depth [jb, je): the stages of SBStage described above.
template <int NA>
struct BottomUpTiles {
    using Stage = SBStage;
    using Tile = SBTile;
    static constexpr int kConsumerWarps = kSBConsumerWarps;
    static constexpr int kStages = kSBStages;
    static constexpr bool kConsumerSync = false;
    DevTree<float> t;
    int32_t jb, je;
    __device__ int32_t ntiles() const { return (je - jb + kSBN - 1) / kSBN; }
    using Meta = int32_t;
    static constexpr int kMetaWords = 4;
    __device__ void prefetch(int32_t tile, int32_t *r) const {        // the tile's child ranges
        const int32_t j0 = jb + tile * kSBN, j1 = min(je, j0 + kSBN);
        r[0] = __ldg(t.tfirst + j0);
        r[1] = __ldg(t.tfirst + j1);
        r[2] = __ldg(t.dfirst + j0);
        r[3] = __ldg(t.dfirst + j1);
    }
    __device__ void issue(int32_t tile, const int32_t *r, Stage *st, Tile *ti, uint64_t *full) const {
        const int32_t j0 = jb + tile * kSBN;
        sb_issue(t, j0, min(kSBN, je - j0), r, st, ti, full);
    }
    __device__ void consume(const Stage &st, const Tile &ti, int c) const {
        const Tile tl = ti;
        sb_nodes<NA>(t, st, tl, c, c + kSBConsumerWarps * 32);
    }
};

template <int NA>
__global__ void __launch_bounds__(kSBThreads) k_bottomup_stream(DevTree<float> t, int32_t jb, int32_t je, int *err) {
    grid_dependency_wait();
    run_pipeline(BottomUpTiles<NA>{t, jb, je}, err);
}

// Top-down from depth [jb, je): tiles of kSBN nodes stage qp, kmask, dfirst and both reaches.  The
// consumers compute the decision children's reaches as td_node does into a shared-memory buffer, then
// store the tile's contiguous child range [dfirst[j0], dfirst[j0 + n]) with coalesced writes (a tile
// with more than kTDOut children writes them directly instead).  Nodes with more than 32 actions are
// left to k_topdown_wide.
constexpr int kTDOut = 4096;

struct TDStage {
    uint32_t qp[kSBN + 4], km[kSBN + 4];
    int32_t df[kSBN + 8];
    float r1[kSBN + 4], r2[kSBN + 4];
};

struct TDTile {
    int32_t j0, n, o;
};

template <int NA>
struct TopDownTiles {
    using Stage = TDStage;
    using Tile = TDTile;
    static constexpr int kConsumerWarps = kSBConsumerWarps;
    static constexpr int kStages = 3;
    static constexpr bool kConsumerSync = true;
    DevTree<float> t;
    int32_t jb, je;
    float *o1, *o2;                                  // shared-memory output buffers, kTDOut each
    __device__ int32_t ntiles() const { return (je - jb + kSBN - 1) / kSBN; }
    using Meta = int32_t;
    static constexpr int kMetaWords = 1;
    __device__ void prefetch(int32_t, int32_t *) const {}
    __device__ void issue(int32_t tile, const int32_t *, Stage *st, Tile *ti, uint64_t *full) const {
        const int32_t j0 = jb + tile * kSBN, n = min(kSBN, je - j0);
        uint32_t bf, bd;
        const int32_t jal = widen16(j0, j0 + n, &bf);
        widen16(j0, j0 + n + 1, &bd);
        ti->j0 = j0; ti->n = n; ti->o = j0 - jal;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(full, 4 * bf + bd);
        bulk_g2s(st->qp, t.qp + jal, bf, full);
        bulk_g2s(st->km, t.kmask + jal, bf, full);
        bulk_g2s(st->df, t.dfirst + jal, bd, full);
        bulk_g2s(st->r1, t.reach1 + jal, bf, full);
        bulk_g2s(st->r2, t.reach2 + jal, bf, full);
    }
    // Nodes c and c + 256 of the tile: strategy loads of both issued before the stores.
    __device__ void consume(const Stage &st, const Tile &ti, int c) const {
        const int32_t ds = st.df[ti.o], nc = st.df[ti.o + ti.n] - ds;
        const bool buffered = nc <= kTDOut;            // uniform over the block
        float *w1 = buffered ? o1 - ds : t.reach1;     // child reach destinations, by global child index
        float *w2 = buffered ? o2 - ds : t.reach2;
        const int32_t ii[2] = {c, c + kSBConsumerWarps * 32};
        float s[2][NA];
        int na[2], pl[2];
        int32_t c0[2];
        uint32_t m[2];
        float r1[2], r2[2];
        bool go[2];
#pragma unroll
        for (int x = 0; x < 2; ++x) {
            go[x] = false;
            na[x] = 0;
            if (ii[x] >= ti.n) continue;
            const int32_t k = ti.o + ii[x];
            const uint32_t w = st.qp[k];
            c0[x] = st.df[k];
            const int32_t nd = st.df[k + 1] - c0[x];
            if (nd == 0 || qp_wide(w)) continue;
            go[x] = true;
            m[x] = st.km[k];
            na[x] = nd + __popc(m[x]);
            pl[x] = qp_player(w);
            r1[x] = st.r1[k];
            r2[x] = st.r2[k];
            const int32_t qb = qp_base(w);
            if (na[x] <= NA) {
#pragma unroll
                for (int a = 0; a < NA; ++a) s[x][a] = a < na[x] ? __ldg(t.sigma + qb + a) : 0.f;
            } else {                                       // more than NA actions: td_node's loop
                int32_t cc = c0[x];
                for (int a = 0; a < na[x]; ++a) {
                    if ((m[x] >> a) & 1u) continue;
                    const float sv = __ldg(t.sigma + qb + a);
                    w1[cc] = pl[x] == 1 ? r1[x] : r1[x] * sv;
                    w2[cc] = pl[x] == 2 ? r2[x] : r2[x] * sv;
                    ++cc;
                }
                go[x] = false;
            }
        }
#pragma unroll
        for (int x = 0; x < 2; ++x) {
            if (!go[x]) continue;
            int32_t cc = c0[x];
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                if (a < na[x] && !((m[x] >> a) & 1u)) {
                    w1[cc] = pl[x] == 1 ? r1[x] : r1[x] * s[x][a];
                    w2[cc] = pl[x] == 2 ? r2[x] : r2[x] * s[x][a];
                    ++cc;
                }
            }
        }
        if (!buffered) return;
        consumers_sync();                              // the tile's child reaches are in o1/o2
        for (int32_t i = c; i < nc; i += kSBConsumerWarps * 32) {
            t.reach1[ds + i] = o1[i];
            t.reach2[ds + i] = o2[i];
        }
        consumers_sync();                              // o1/o2 free for the next tile
    }
};

template <int NA>
__global__ void __launch_bounds__(kSBThreads) k_topdown_stream(DevTree<float> t, int32_t jb, int32_t je, int32_t bump,
                                                               int *err) {
    grid_dependency_wait();
    __shared__ float out1[kTDOut], out2[kTDOut];
    if (bump && blockIdx.x == 0 && threadIdx.x == 0) *t.iter += 1;
    run_pipeline(TopDownTiles<NA>{t, jb, je, out1, out2}, err);
}

// ---- the last two depths, streamed (FP32 mode) -------------------------------------------------------
// One pass over the depths L-2 and L-1 (the nodes of L-1 have terminal children only) in tiles of
// consecutive depth-(L-2) nodes ("parents"), cut on the host so that every range below fits its stage
// array (tail_tiles in the host code).  The producer stages the parents' fields and reaches, their
// decision children's fields (qp, kmask, tfirst) and the two contiguous utility ranges: the parents'
// terminal children and the children's terminal children.  The consumers then run
//   phase 0, one thread per parent: the top-down step (td_node's arithmetic) with the children's
//            reaches written to shared memory, the parent's strategy entries kept in registers;
//   phase 1, one thread per child: its bottom-up step (bu_node's arithmetic), value to shared memory;
//   phase 2, one thread per parent: its bottom-up step.
// Global memory sees the staged inputs once, the parents' values (written), the strategy gathers and
// the regret scatter; the children's reaches and values stay on chip unless record is set.  Nodes with
// more than 32 actions are not handled (the host keeps such trees off this kernel).
constexpr int kTP = 256;                   // parents per tile, at most (one per consumer thread)
constexpr int kTC = 768;                   // children per tile, at most
constexpr int kTPT = 768;                  // parents' terminal children per tile, at most
constexpr int kTCT = 3072;                 // children's terminal children per tile, at most

struct TLStage {                           // + 4 / + 8: room for widening the copies to 16 bytes
    uint32_t qp[kTP + 4], km[kTP + 4];
    float r1[kTP + 4], r2[kTP + 4];
    int32_t df[kTP + 8], tf[kTP + 8];
    uint32_t cqp[kTC + 4], ckm[kTC + 4];
    int32_t ctf[kTC + 8];
    float pu[kTPT + 4], cu[kTCT + 4];
};

struct TLTile {
    int32_t j0, n, o;                      // parents [j0, j0 + n); node j0 at index o of the parent arrays
    int32_t cs, nc, co;                    // children [cs, cs + nc); child cs at index co of the child arrays
    int32_t pal, cal;                      // global terminal index of pu[0] / cu[0]
};

template <int NA>
struct TailTiles {
    using Stage = TLStage;
    using Tile = TLTile;
    static constexpr int kConsumerWarps = kSBConsumerWarps;
    static constexpr int kStages = 2;
    static constexpr bool kConsumerSync = true;
    DevTree<float> t;
    const int4 *tm;                        // per tile two int4: {j0, j1, cs, ce}, {pts, pte, cts, cte}: its
                                           // parents, their decision children, and the two terminal ranges
    int32_t nt, record;
    float *q1, *q2, *cu;                   // shared memory, kTC each: children's reaches and values
    __device__ int32_t ntiles() const { return nt; }
    using Meta = int4;
    static constexpr int kMetaWords = 2;
    __device__ void prefetch(int32_t tile, int4 *meta) const {
        meta[0] = __ldg(tm + 2 * tile);
        meta[1] = __ldg(tm + 2 * tile + 1);
    }
    __device__ void issue(int32_t, const int4 *meta, Stage *st, Tile *ti, uint64_t *full) const {
        const int32_t j0 = meta[0].x, n = meta[0].y - j0, cs = meta[0].z, ce = meta[0].w;
        const int32_t pts = meta[1].x, pte = meta[1].y, cts = meta[1].z, cte = meta[1].w;
        uint32_t bf, bd, bc, bct, bpu, bcu;
        const int32_t jal = widen16(j0, j0 + n, &bf);
        widen16(j0, j0 + n + 1, &bd);
        const int32_t cal_n = widen16(cs, ce, &bc);
        widen16(cs, ce + 1, &bct);
        const int32_t pal = widen16(pts, pte, &bpu);
        const int32_t cal = widen16(cts, cte, &bcu);
        ti->j0 = j0; ti->n = n; ti->o = j0 - jal;
        ti->cs = cs; ti->nc = ce - cs; ti->co = cs - cal_n;
        ti->pal = pal; ti->cal = cal;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(full, 4 * bf + 2 * bd + 2 * bc + bct + bpu + bcu);
        bulk_g2s(st->qp, t.qp + jal, bf, full);
        bulk_g2s(st->km, t.kmask + jal, bf, full);
        bulk_g2s(st->r1, t.reach1 + jal, bf, full);
        bulk_g2s(st->r2, t.reach2 + jal, bf, full);
        bulk_g2s(st->df, t.dfirst + jal, bd, full);
        bulk_g2s(st->tf, t.tfirst + jal, bd, full);
        if (bc) {
            bulk_g2s(st->cqp, t.qp + cal_n, bc, full);
            bulk_g2s(st->ckm, t.kmask + cal_n, bc, full);
        }
        bulk_g2s(st->ctf, t.tfirst + cal_n, bct, full);
        if (bpu) bulk_g2s(st->pu, t.util + pal, bpu, full);
        if (bcu) bulk_g2s(st->cu, t.util + cal, bcu, full);
    }
    // Thread c takes parent c and children c, c + 256, c + 512 (kTCPer of them); the strategy entries of
    // all of them are loaded in one round before phase 0.
    static constexpr int kTCPer = (kTC + kSBConsumerWarps * 32 - 1) / (kSBConsumerWarps * 32);
    __device__ void consume(const Stage &st, const Tile &ti, int c) const {
        constexpr int kC = kSBConsumerWarps * 32;
        const bool act = c < ti.n;
        const int32_t k = ti.o + c;
        uint32_t m = 0;
        int32_t c0 = 0, t0 = 0, qb = 0;
        int na = 0, p = 0;
        float r1 = 0.f, r2 = 0.f;
        float s[NA];
        if (act) {
            const uint32_t w = st.qp[k];
            m = st.km[k];
            c0 = st.df[k];
            na = (st.df[k + 1] - c0) + __popc(m);
            t0 = st.tf[k];
            r1 = st.r1[k];
            r2 = st.r2[k];
            qb = qp_base(w);
            p = qp_player(w);
#pragma unroll
            for (int a = 0; a < NA; ++a) s[a] = a < na ? __ldg(t.sigma + qb + a) : 0.f;
        }
        uint32_t cm[kTCPer];
        int32_t cqb[kTCPer];
        float sc[kTCPer][NA];
#pragma unroll
        for (int r = 0; r < kTCPer; ++r) {
            const int32_t ci = c + r * kC;
            cm[r] = 0;
            cqb[r] = 0;
            if (ci < ti.nc) {
                const uint32_t cw = st.cqp[ti.co + ci];
                cm[r] = st.ckm[ti.co + ci];
                cqb[r] = (int32_t)cw;                      // qp word; base and player taken below
                const int cna = __popc(cm[r]);
#pragma unroll
                for (int b = 0; b < NA; ++b) sc[r][b] = b < cna ? __ldg(t.sigma + qp_base(cw) + b) : 0.f;
            }
        }
        // phase 0: parent c's top-down step, the children's reaches to shared memory
        if (act) {
            int32_t y = c0 - ti.cs;
            if (na <= NA) {
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    if (a < na && !((m >> a) & 1u)) {
                        q1[y] = p == 1 ? r1 : r1 * s[a];
                        q2[y] = p == 2 ? r2 : r2 * s[a];
                        ++y;
                    }
                }
            } else {
                for (int a = 0; a < na; ++a) {
                    if ((m >> a) & 1u) continue;
                    const float sv = __ldg(t.sigma + qb + a);
                    q1[y] = p == 1 ? r1 : r1 * sv;
                    q2[y] = p == 2 ? r2 : r2 * sv;
                    ++y;
                }
            }
        }
        consumers_sync();
        // phase 1: the children's bottom-up steps (terminal children only)
#pragma unroll
        for (int r = 0; r < kTCPer; ++r) {
            const int32_t ci = c + r * kC;
            if (ci >= ti.nc) continue;
            const uint32_t cw = (uint32_t)cqb[r];
            const int32_t cq = qp_base(cw);
            const int cp = qp_player(cw);
            const int cna = __popc(cm[r]);
            const float *tv = st.cu + (st.ctf[ti.co + ci] - ti.cal);
            float ud = 0.f;
            float v[NA];
            if (cna <= NA) {
#pragma unroll
                for (int b = 0; b < NA; ++b) {
                    if (b < cna) {
                        v[b] = tv[b];
                        ud = madd(ud, sc[r][b], v[b]);
                    }
                }
            } else {
                for (int b = 0; b < cna; ++b) ud = madd(ud, __ldg(t.sigma + cq + b), tv[b]);
            }
            cu[ci] = ud;
            const float cq1 = q1[ci], cq2 = q2[ci];
            if (record) {
                const int32_t cg = ti.cs + ci;
                t.u[cg] = ud;
                t.reach1[cg] = cq1;
                t.reach2[cg] = cq2;
            }
            if (!collects(t, cp)) continue;
            const float wr = cp == 1 ? cq1 : -cq2;
            if (wr == 0.f) continue;
            if (cna <= NA) {
#pragma unroll
                for (int b = 0; b < NA; ++b)
                    if (b < cna) atomicAdd(&t.inst[cq + b], wr * (v[b] - ud));
            } else {
                for (int b = 0; b < cna; ++b) atomicAdd(&t.inst[cq + b], wr * (tv[b] - ud));
            }
        }
        consumers_sync();
        // phase 2: parent c's bottom-up step
        if (!act) return;
        const float *pv = st.pu + (t0 - ti.pal);
        const float *dv = cu + (c0 - ti.cs);
        float ud = 0.f;
        if (na <= NA) {
            float v[NA];
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                if (a < na) {
                    const int kt = __popc(m & ((1u << a) - 1u));   // terminal children before action a
                    const float *src = ((m >> a) & 1u) ? pv + kt : dv + (a - kt);
                    v[a] = *src;
                }
            }
#pragma unroll
            for (int a = 0; a < NA; ++a)
                if (a < na) ud = madd(ud, s[a], v[a]);
            t.u[ti.j0 + c] = ud;
            if (!collects(t, p)) return;
            const float wr = p == 1 ? r1 : -r2;
            if (wr == 0.f) return;
#pragma unroll
            for (int a = 0; a < NA; ++a)
                if (a < na) atomicAdd(&t.inst[qb + a], wr * (v[a] - ud));
            return;
        }
        int kt = 0, kd = 0;
        for (int a = 0; a < na; ++a) {
            const float val = ((m >> a) & 1u) ? pv[kt++] : dv[kd++];
            ud = madd(ud, __ldg(t.sigma + qb + a), val);
        }
        t.u[ti.j0 + c] = ud;
        if (!collects(t, p)) return;
        const float wr = p == 1 ? r1 : -r2;
        if (wr == 0.f) return;
        kt = kd = 0;
        for (int a = 0; a < na; ++a) {
            const float val = ((m >> a) & 1u) ? pv[kt++] : dv[kd++];
            atomicAdd(&t.inst[qb + a], wr * (val - ud));
        }
    }
};

// bump: depth L-2 is the root's, so no top-down launch precedes this one; count the iteration.
template <int NA>
__global__ void __launch_bounds__(kSBThreads) k_tail_stream(DevTree<float> t, const int4 *tm, int32_t nt,
                                                            int32_t record, int32_t bump, int *err) {
    grid_dependency_wait();
    __shared__ float q1[kTC], q2[kTC], cu[kTC];
    if (bump && blockIdx.x == 0 && threadIdx.x == 0) *t.iter += 1;
    run_pipeline(TailTiles<NA>{t, tm, nt, record, q1, q2, cu}, err);
}

// ---- the last two depths with their strategy and regret slots staged (FP32 mode) ----------------------
// k_tail_slots computes what k_tail_stream does (top-down of depth L-2, bottom-up of L-1 and L-2), for
// trees whose tiles are slot-dense: the infoset slots of a tile's parents form one contiguous range,
// those of its children another, and each child's terminal children sit at the same offset in the
// terminal range as its slots in the slot range.  Breadth-first ids give this wherever consecutive
// nodes of a depth belong to consecutive infosets - the public tree below one root outcome (deal),
// whose nodes meet their infosets in the same order for every deal - so the host cuts tiles at every
// break of contiguity and uses this kernel when no single parent breaks it (plan_fusion).
// Per tile the producer bulk-copies, besides the parents' fields and reaches, the strategy entries of
// both slot ranges and both utility ranges; a child needs only its packed word (slot base, player),
// its action count being the distance to the next child's base.  The consumers (one thread per
// parent) read every strategy entry from shared memory, write each slot's instantaneous regret into
// the place of its strategy entry, and one thread adds both regret ranges to r~ with two bulk
// reductions (cp.reduce.async.bulk .add.f32, element-wise atomic), so no per-slot atomics remain.
// The widened ends of the ranges (16-byte copies) belong to neighbouring tiles and are zeroed before
// the reduction.
constexpr int kSTWarps = kSTP / 32;        // tile limits kSTP .. kSTTP: tail_tiles.hpp

struct STStage {                           // + 4 / + 8: room for widening the copies to 16 bytes
    uint32_t qp[kSTP + 4], km[kSTP + 4];
    float r1[kSTP + 4], r2[kSTP + 4];
    int32_t df[kSTP + 8], tf[kSTP + 8];
    uint32_t cqp[kSTC + 4];
    float sp[kSTSP + 4], sc[kSTSC + 4];    // strategy entries of the two slot ranges, then their regrets
    float pu[kSTTP + 4], cu[kSTSC + 4];    // the two utility ranges
};

struct STTile {
    int32_t j0, n, o;                      // parents [j0, j0 + n); node j0 at index o of the parent arrays
    int32_t cs, nc, co;                    // children [cs, cs + nc); child cs at index co of cqp
    int32_t pal;                           // global terminal index of pu[0]
    int32_t spal, spn, scal, scn;          // global slot of sp[0] / sc[0] and their widened lengths
    int32_t qps, qpe, qcs, qce;            // the exact slot ranges of the parents and the children
    int32_t ushift;                        // cu index of a child's first terminal = its slot base + ushift
};

// Bulk reduction shared -> global of `bytes` (a multiple of 16, both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_add_s2g(float *dst, const float *src, uint32_t bytes) {
    asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f32 [%0], [%1], %2;" ::"l"(dst),
                 "r"(smem_u32(src)), "r"(bytes)
                 : "memory");
}

// BULK: the regrets replace the strategy entries in shared memory and are added to r~ by two bulk
// reductions per tile (one thread waits for the copy engine to read them before the stage is
// released); otherwise each nonzero contribution is added with a per-slot atomic, as in
// k_tail_stream, and contributions of zero counterfactual reach are skipped.
template <int NA, bool BULK>
struct SlotTailTiles {
    using Stage = STStage;
    using Tile = STTile;
    static constexpr int kStages = 2;
    static constexpr int kConsumerWarps = kSTWarps;
    static constexpr bool kConsumerSync = true;
    static constexpr int kN = kSTP;        // consumer threads
    DevTree<float> t;
    const int4 *tm;                        // per tile three int4: {j0, j1, cs, ce}, {pts, pte, cts, cte},
                                           // {qps, qpe, qcs, qce}
    int32_t nt, record;
    float *q1, *q2, *cv;                   // shared memory, kSTC each: children's reaches and values
    __device__ int32_t ntiles() const { return nt; }
    using Meta = int4;
    static constexpr int kMetaWords = 3;
    __device__ void prefetch(int32_t tile, int4 *meta) const {
        meta[0] = __ldg(tm + 3 * tile);
        meta[1] = __ldg(tm + 3 * tile + 1);
        meta[2] = __ldg(tm + 3 * tile + 2);
    }
    __device__ void issue(int32_t, const int4 *meta, Stage *st, Tile *ti, uint64_t *full) const {
        const int32_t j0 = meta[0].x, n = meta[0].y - j0, cs = meta[0].z, ce = meta[0].w;
        const int32_t pts = meta[1].x, pte = meta[1].y, cts = meta[1].z, cte = meta[1].w;
        const int32_t qps = meta[2].x, qpe = meta[2].y, qcs = meta[2].z, qce = meta[2].w;
        uint32_t bf, bd, bc, bpu, bcu, bsp, bsc;
        const int32_t jal = widen16(j0, j0 + n, &bf);
        widen16(j0, j0 + n + 1, &bd);
        const int32_t cal_n = widen16(cs, ce, &bc);
        const int32_t pal = widen16(pts, pte, &bpu);
        const int32_t cual = widen16(cts, cte, &bcu);
        const int32_t spal = widen16(qps, qpe, &bsp);
        const int32_t scal = widen16(qcs, qce, &bsc);
        ti->j0 = j0; ti->n = n; ti->o = j0 - jal;
        ti->cs = cs; ti->nc = ce - cs; ti->co = cs - cal_n;
        ti->pal = pal;
        ti->spal = spal; ti->spn = (int32_t)(bsp / 4u); ti->scal = scal; ti->scn = (int32_t)(bsc / 4u);
        ti->qps = qps; ti->qpe = qpe; ti->qcs = qcs; ti->qce = qce;
        ti->ushift = cts - cual - qcs;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(full, 4 * bf + 2 * bd + bc + bpu + bcu + bsp + bsc);
        bulk_g2s(st->qp, t.qp + jal, bf, full);
        bulk_g2s(st->km, t.kmask + jal, bf, full);
        bulk_g2s(st->r1, t.reach1 + jal, bf, full);
        bulk_g2s(st->r2, t.reach2 + jal, bf, full);
        bulk_g2s(st->df, t.dfirst + jal, bd, full);
        bulk_g2s(st->tf, t.tfirst + jal, bd, full);
        if (bc) bulk_g2s(st->cqp, t.qp + cal_n, bc, full);
        if (bpu) bulk_g2s(st->pu, t.util + pal, bpu, full);
        if (bcu) bulk_g2s(st->cu, t.util + cual, bcu, full);
        if (bsp) bulk_g2s(st->sp, t.sigma + spal, bsp, full);
        if (bsc) bulk_g2s(st->sc, t.sigma + scal, bsc, full);
    }
    // Thread c takes parent c (phases 0 and 2) and children c, c + kN, ... (phase 1).
    __device__ void consume(Stage &st, const Tile &tref, int c) const {
        const Tile ti = tref;              // the tile's description in registers
        const bool act = c < ti.n;
        uint32_t m = 0;
        int32_t c0 = 0, t0 = 0, e0 = 0;
        int na = 0, p = 0;
        float r1 = 0.f, r2 = 0.f;
        float s[NA];
        if (act) {
            const int32_t k = ti.o + c;
            const uint32_t w = st.qp[k];
            m = st.km[k];
            c0 = st.df[k];
            t0 = st.tf[k];
            na = (st.df[k + 1] - c0) + __popc(m);
            p = qp_player(w);
            e0 = qp_base(w) - ti.spal;
            r1 = st.r1[k];
            r2 = st.r2[k];
#pragma unroll
            for (int a = 0; a < NA; ++a) s[a] = a < na ? st.sp[e0 + a] : 0.f;
            // phase 0: the top-down step, the children's reaches to shared memory
            int32_t y = c0 - ti.cs;
            if (na <= NA) {
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    if (a < na && !((m >> a) & 1u)) {
                        q1[y] = p == 1 ? r1 : r1 * s[a];
                        q2[y] = p == 2 ? r2 : r2 * s[a];
                        ++y;
                    }
                }
            } else {
                for (int a = 0; a < na; ++a) {
                    if ((m >> a) & 1u) continue;
                    const float sv = st.sp[e0 + a];
                    q1[y] = p == 1 ? r1 : r1 * sv;
                    q2[y] = p == 2 ? r2 : r2 * sv;
                    ++y;
                }
            }
        }
        if constexpr (BULK) {
            // the widened ends of both slot ranges belong to other tiles' infosets: nothing is added there
            if (c < 4) {
                if (ti.spal + c < ti.qps) st.sp[c] = 0.f;
                if (ti.spn > c && ti.spal + ti.spn - 1 - c >= ti.qpe) st.sp[ti.spn - 1 - c] = 0.f;
                if (ti.scn > c && ti.scal + c < ti.qcs) st.sc[c] = 0.f;
                if (ti.scn > c && ti.scal + ti.scn - 1 - c >= ti.qce) st.sc[ti.scn - 1 - c] = 0.f;
            }
        }
        consumers_sync<kN>();
        // phase 1: the children's bottom-up steps (terminal children only)
        for (int32_t ci = c; ci < ti.nc; ci += kN) {
            const uint32_t cw = st.cqp[ti.co + ci];
            const int32_t cq = qp_base(cw);
            const int cp = qp_player(cw);
            const int32_t nx = ci + 1 < ti.nc ? qp_base(st.cqp[ti.co + ci + 1]) : ti.qce;
            const int cna = nx - cq;
            float *sv = st.sc + (cq - ti.scal);
            const float *tv = st.cu + (cq + ti.ushift);
            float ud = 0.f;
            float v[NA];
            if (cna <= NA) {
#pragma unroll
                for (int b = 0; b < NA; ++b) {
                    if (b < cna) {
                        v[b] = tv[b];
                        ud = madd(ud, sv[b], v[b]);
                    }
                }
            } else {
                for (int b = 0; b < cna; ++b) ud = madd(ud, sv[b], tv[b]);
            }
            cv[ci] = ud;
            const float cq1 = q1[ci], cq2 = q2[ci];
            if (record) {
                const int32_t cg = ti.cs + ci;
                t.u[cg] = ud;
                t.reach1[cg] = cq1;
                t.reach2[cg] = cq2;
            }
            const float wr = !collects(t, cp) ? 0.f : cp == 1 ? cq1 : -cq2;
            if constexpr (BULK) {
                if (cna <= NA) {
#pragma unroll
                    for (int b = 0; b < NA; ++b)
                        if (b < cna) sv[b] = wr * (v[b] - ud);
                } else {
                    for (int b = 0; b < cna; ++b) sv[b] = wr * (tv[b] - ud);
                }
            } else {
                if (wr == 0.f) continue;
                if (cna <= NA) {
#pragma unroll
                    for (int b = 0; b < NA; ++b)
                        if (b < cna) atomicAdd(&t.inst[cq + b], wr * (v[b] - ud));
                } else {
                    for (int b = 0; b < cna; ++b) atomicAdd(&t.inst[cq + b], wr * (tv[b] - ud));
                }
            }
        }
        consumers_sync<kN>();
        // phase 2: parent c's bottom-up step
        if (act) {
            const float *pv = st.pu + (t0 - ti.pal);
            const float *dv = cv + (c0 - ti.cs);
            float *sv = st.sp + e0;
            const int32_t qb = e0 + ti.spal;
            const float wr = !collects(t, p) ? 0.f : p == 1 ? r1 : -r2;
            float ud = 0.f;
            if (na <= NA) {
                float v[NA];
                int kt = 0, kd = 0;
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    if (a < na) {
                        const bool term = (m >> a) & 1u;
                        v[a] = *(term ? pv + kt : dv + kd);
                        kt += term;
                        kd += !term;
                    }
                }
#pragma unroll
                for (int a = 0; a < NA; ++a)
                    if (a < na) ud = madd(ud, s[a], v[a]);
                t.u[ti.j0 + c] = ud;
                if constexpr (BULK) {
#pragma unroll
                    for (int a = 0; a < NA; ++a)
                        if (a < na) sv[a] = wr * (v[a] - ud);
                } else if (wr != 0.f) {
#pragma unroll
                    for (int a = 0; a < NA; ++a)
                        if (a < na) atomicAdd(&t.inst[qb + a], wr * (v[a] - ud));
                }
            } else {
                int kt = 0, kd = 0;
                for (int a = 0; a < na; ++a) {
                    const float val = ((m >> a) & 1u) ? pv[kt++] : dv[kd++];
                    ud = madd(ud, sv[a], val);
                }
                t.u[ti.j0 + c] = ud;
                kt = kd = 0;
                for (int a = 0; a < na; ++a) {
                    const float val = ((m >> a) & 1u) ? pv[kt++] : dv[kd++];
                    if constexpr (BULK) sv[a] = wr * (val - ud);
                    else if (wr != 0.f) atomicAdd(&t.inst[qb + a], wr * (val - ud));
                }
            }
        }
        if constexpr (BULK) {
            // the regrets of both ranges into r~: visible to the bulk copy engine, then two reductions; the
            // stage is released only after the engine has read them
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            consumers_sync<kN>();
            if (c == 0) {
                if (ti.spn) bulk_add_s2g(t.inst + ti.spal, st.sp, 4u * (uint32_t)ti.spn);
                if (ti.scn) bulk_add_s2g(t.inst + ti.scal, st.sc, 4u * (uint32_t)ti.scn);
                asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
            }
        }
    }
};

// bump: depth L-2 is the root's, so no top-down launch precedes this one; count the iteration.
template <int NA, bool BULK>
__global__ void __launch_bounds__(32 * (kSTWarps + 1)) k_tail_slots(DevTree<float> t, const int4 *tm, int32_t nt,
                                                                     int32_t record, int32_t bump, int *err) {
    grid_dependency_wait();
    __shared__ float q1[kSTC], q2[kSTC], cv[kSTC];
    if (bump && blockIdx.x == 0 && threadIdx.x == 0) *t.iter += 1;
    run_pipeline(SlotTailTiles<NA, BULK>{t, tm, nt, record, q1, q2, cv}, err);
}

// ---- two depths above the fused tail, paired (FP32 mode) ----------------------------------------------
// The top-down steps of depths m and m+1 in one launch, and their bottom-up steps in another, over
// tiles of consecutive depth-m nodes ("parents") cut on the host so that every range below fits its
// stage array (cut_pair_tiles in the host code).  A tile's decision children (depth m+1, "children")
// and their decision children (depth m+2, "grandchildren") are contiguous ranges in breadth-first
// order.  Depth m+1's reaches and values stay on chip:
//   top-down:  phase 0, one thread per parent: td_node's arithmetic, the children's reaches to shared
//              memory; phase 1, one thread per child: the same for the child, the grandchildren's
//              reaches to a shared-memory buffer, stored afterwards as one coalesced range;
//   bottom-up: phase 0 as above (the same products, so the children's reaches are those the top-down
//              launch formed); phase 1, one thread per child: bu_node's arithmetic on the staged
//              grandchildren's values and terminal utilities, value to shared memory; phase 2, one
//              thread per parent: its bottom-up step.
// With record set both launches also store depth m+1's reaches and values.  Nodes with more than 32
// actions are not handled (the host keeps such depths off these kernels).
constexpr int kPP = 256;                   // parents per tile, at most (one per consumer thread)
constexpr int kPC = 640;                   // children per tile, at most
constexpr int kPPT = 640;                  // parents' terminal children per tile, at most
constexpr int kPCT = 1344;                 // children's terminal children per tile, at most
constexpr int kPG = 1664;                  // grandchildren per tile, at most
constexpr int kPCPer = (kPC + kSBConsumerWarps * 32 - 1) / (kSBConsumerWarps * 32);

struct PTStage {                           // top-down stage; + 4 / + 8: room for widening the copies
    uint32_t qp[kPP + 4], km[kPP + 4];
    float r1[kPP + 4], r2[kPP + 4];
    int32_t df[kPP + 8];
    uint32_t cqp[kPC + 4], ckm[kPC + 4];
    int32_t cdf[kPC + 8];
};

struct PBStage {                           // bottom-up stage
    uint32_t qp[kPP + 4], km[kPP + 4];
    float r1[kPP + 4], r2[kPP + 4];
    int32_t df[kPP + 8], tf[kPP + 8];
    uint32_t cqp[kPC + 4], ckm[kPC + 4];
    int32_t cdf[kPC + 8], ctf[kPC + 8];
    float pu[kPPT + 4], cu[kPCT + 4], gu[kPG + 4];
};

struct PRTile {
    int32_t j0, n, o;                      // parents [j0, j0 + n); node j0 at index o of the parent arrays
    int32_t cs, nc, co;                    // children [cs, cs + nc); child cs at index co of the child arrays
    int32_t gs, ng, gal;                   // grandchildren [gs, gs + ng); global index of gu[0]
    int32_t pal, cal;                      // global terminal index of pu[0] / cu[0]
};

// Phase 0 of both launches: parent c's decision children's reaches into q1/q2 (indexed from the tile's
// first child), as td_node forms them; s: the parent's strategy entries (its first NA).
template <int NA>
__device__ __forceinline__ void pair_parent_topdown(const DevTree<float> &t, int32_t c0, int na, uint32_t m, int p,
                                                    float r1, float r2, int32_t qb, const float (&s)[NA], float *q1,
                                                    float *q2) {
    int32_t y = c0;
    if (na <= NA) {
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            if (a < na && !((m >> a) & 1u)) {
                q1[y] = p == 1 ? r1 : r1 * s[a];
                q2[y] = p == 2 ? r2 : r2 * s[a];
                ++y;
            }
        }
    } else {
        for (int a = 0; a < na; ++a) {
            if ((m >> a) & 1u) continue;
            const float sv = __ldg(t.sigma + qb + a);
            q1[y] = p == 1 ? r1 : r1 * sv;
            q2[y] = p == 2 ? r2 : r2 * sv;
            ++y;
        }
    }
}

template <int NA>
struct PairTopDownTiles {
    using Stage = PTStage;
    using Tile = PRTile;
    static constexpr int kConsumerWarps = kSBConsumerWarps;
    static constexpr int kStages = 2;
    static constexpr bool kConsumerSync = true;
    DevTree<float> t;
    const int4 *tm;                        // per tile three int4: {j0, j1, cs, ce}, {pts, pte, cts, cte}, {gs, ge, -, -}
    int32_t nt, record;
    float *q1, *q2;                        // shared memory, kPC each: the children's reaches
    float *o1, *o2;                        // shared memory, kPG each: the grandchildren's reaches
    __device__ int32_t ntiles() const { return nt; }
    using Meta = int4;
    static constexpr int kMetaWords = 3;
    __device__ void prefetch(int32_t tile, int4 *meta) const {
        meta[0] = __ldg(tm + 3 * tile);
        meta[1] = __ldg(tm + 3 * tile + 1);
        meta[2] = __ldg(tm + 3 * tile + 2);
    }
    __device__ void issue(int32_t, const int4 *meta, Stage *st, Tile *ti, uint64_t *full) const {
        const int32_t j0 = meta[0].x, n = meta[0].y - j0, cs = meta[0].z, ce = meta[0].w;
        uint32_t bf, bd, bc, bcd;
        const int32_t jal = widen16(j0, j0 + n, &bf);
        widen16(j0, j0 + n + 1, &bd);
        const int32_t cal_n = widen16(cs, ce, &bc);
        widen16(cs, ce + 1, &bcd);
        ti->j0 = j0; ti->n = n; ti->o = j0 - jal;
        ti->cs = cs; ti->nc = ce - cs; ti->co = cs - cal_n;
        ti->gs = meta[2].x; ti->ng = meta[2].y - meta[2].x; ti->gal = 0;
        ti->pal = 0; ti->cal = 0;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(full, 4 * bf + bd + 2 * bc + bcd);
        bulk_g2s(st->qp, t.qp + jal, bf, full);
        bulk_g2s(st->km, t.kmask + jal, bf, full);
        bulk_g2s(st->r1, t.reach1 + jal, bf, full);
        bulk_g2s(st->r2, t.reach2 + jal, bf, full);
        bulk_g2s(st->df, t.dfirst + jal, bd, full);
        if (bc) {
            bulk_g2s(st->cqp, t.qp + cal_n, bc, full);
            bulk_g2s(st->ckm, t.kmask + cal_n, bc, full);
        }
        bulk_g2s(st->cdf, t.dfirst + cal_n, bcd, full);
    }
    // Thread c takes parent c and children c, c + 256, c + 512; the strategy entries of all of them are
    // loaded in one round before phase 0.
    __device__ void consume(const Stage &st, const Tile &ti, int c) const {
        constexpr int kC = kSBConsumerWarps * 32;
        const int32_t k = ti.o + c;
        uint32_t m = 0;
        int32_t c0 = 0, qb = 0;
        int na = 0, p = 0;
        float r1 = 0.f, r2 = 0.f;
        float s[NA];
        bool act = false;
        if (c < ti.n) {
            c0 = st.df[k];
            const int32_t nd = st.df[k + 1] - c0;
            act = nd > 0;
            if (act) {
                const uint32_t w = st.qp[k];
                m = st.km[k];
                na = nd + __popc(m);
                r1 = st.r1[k];
                r2 = st.r2[k];
                qb = qp_base(w);
                p = qp_player(w);
#pragma unroll
                for (int a = 0; a < NA; ++a) s[a] = a < na ? __ldg(t.sigma + qb + a) : 0.f;
            }
        }
        uint32_t cm[kPCPer];
        int32_t cw[kPCPer], cd0[kPCPer];
        float sc[kPCPer][NA];
#pragma unroll
        for (int r = 0; r < kPCPer; ++r) {               // cd0 < 0: no child, or one without decision children
            const int32_t ci = c + r * kC;
            cm[r] = 0;
            cw[r] = 0;
            cd0[r] = -1;
            if (ci < ti.nc) {
                const int32_t cd = st.cdf[ti.co + ci], cnd = st.cdf[ti.co + ci + 1] - cd;
                if (cnd > 0) {
                    cw[r] = (int32_t)st.cqp[ti.co + ci];
                    cm[r] = st.ckm[ti.co + ci];
                    cd0[r] = cd;
                    const int cna = cnd + __popc(cm[r]);
                    const int32_t cq = qp_base((uint32_t)cw[r]);
#pragma unroll
                    for (int b = 0; b < NA; ++b) sc[r][b] = b < cna ? __ldg(t.sigma + cq + b) : 0.f;
                }
            }
        }
        // phase 0: parent c's top-down step, the children's reaches to shared memory
        if (act) pair_parent_topdown<NA>(t, c0 - ti.cs, na, m, p, r1, r2, qb, s, q1, q2);
        consumers_sync();
        // phase 1: the children's top-down steps, the grandchildren's reaches to the output buffers
#pragma unroll
        for (int r = 0; r < kPCPer; ++r) {
            const int32_t ci = c + r * kC;
            if (ci >= ti.nc) continue;
            const float cr1 = q1[ci], cr2 = q2[ci];
            if (record) {
                t.reach1[ti.cs + ci] = cr1;
                t.reach2[ti.cs + ci] = cr2;
            }
            if (cd0[r] < 0) continue;
            const int32_t cnd = st.cdf[ti.co + ci + 1] - cd0[r];
            const int cna = cnd + __popc(cm[r]);
            pair_parent_topdown<NA>(t, cd0[r] - ti.gs, cna, cm[r], qp_player((uint32_t)cw[r]), cr1, cr2,
                                    qp_base((uint32_t)cw[r]), sc[r], o1, o2);
        }
        consumers_sync();                              // the tile's grandchildren's reaches are in o1/o2
        for (int32_t i = c; i < ti.ng; i += kC) {
            t.reach1[ti.gs + i] = o1[i];
            t.reach2[ti.gs + i] = o2[i];
        }
    }
};

// bump: depth m is the root's, so no top-down launch precedes this one; count the iteration.
template <int NA>
__global__ void __launch_bounds__(kSBThreads) k_pair_topdown(DevTree<float> t, const int4 *tm, int32_t nt,
                                                             int32_t record, int32_t bump, int *err) {
    grid_dependency_wait();
    __shared__ float q1[kPC], q2[kPC], o1[kPG], o2[kPG];
    if (bump && blockIdx.x == 0 && threadIdx.x == 0) *t.iter += 1;
    run_pipeline(PairTopDownTiles<NA>{t, tm, nt, record, q1, q2, o1, o2}, err);
}

template <int NA>
struct PairBottomUpTiles {
    using Stage = PBStage;
    using Tile = PRTile;
    static constexpr int kConsumerWarps = kSBConsumerWarps;
    static constexpr int kStages = 2;
    static constexpr bool kConsumerSync = true;
    DevTree<float> t;
    const int4 *tm;
    int32_t nt, record;
    float *q1, *q2, *cv;                   // shared memory, kPC each: the children's reaches and values
    __device__ int32_t ntiles() const { return nt; }
    using Meta = int4;
    static constexpr int kMetaWords = 3;
    __device__ void prefetch(int32_t tile, int4 *meta) const {
        meta[0] = __ldg(tm + 3 * tile);
        meta[1] = __ldg(tm + 3 * tile + 1);
        meta[2] = __ldg(tm + 3 * tile + 2);
    }
    __device__ void issue(int32_t, const int4 *meta, Stage *st, Tile *ti, uint64_t *full) const {
        const int32_t j0 = meta[0].x, n = meta[0].y - j0, cs = meta[0].z, ce = meta[0].w;
        const int32_t pts = meta[1].x, pte = meta[1].y, cts = meta[1].z, cte = meta[1].w;
        const int32_t gs = meta[2].x, ge = meta[2].y;
        uint32_t bf, bd, bc, bcd, bpu, bcu, bgu;
        const int32_t jal = widen16(j0, j0 + n, &bf);
        widen16(j0, j0 + n + 1, &bd);
        const int32_t cal_n = widen16(cs, ce, &bc);
        widen16(cs, ce + 1, &bcd);
        const int32_t pal = widen16(pts, pte, &bpu);
        const int32_t cal = widen16(cts, cte, &bcu);
        const int32_t gal = widen16(gs, ge, &bgu);
        ti->j0 = j0; ti->n = n; ti->o = j0 - jal;
        ti->cs = cs; ti->nc = ce - cs; ti->co = cs - cal_n;
        ti->gs = gs; ti->ng = ge - gs; ti->gal = gal;
        ti->pal = pal; ti->cal = cal;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(full, 4 * bf + 2 * bd + 2 * bc + 2 * bcd + bpu + bcu + bgu);
        bulk_g2s(st->qp, t.qp + jal, bf, full);
        bulk_g2s(st->km, t.kmask + jal, bf, full);
        bulk_g2s(st->r1, t.reach1 + jal, bf, full);
        bulk_g2s(st->r2, t.reach2 + jal, bf, full);
        bulk_g2s(st->df, t.dfirst + jal, bd, full);
        bulk_g2s(st->tf, t.tfirst + jal, bd, full);
        if (bc) {
            bulk_g2s(st->cqp, t.qp + cal_n, bc, full);
            bulk_g2s(st->ckm, t.kmask + cal_n, bc, full);
        }
        bulk_g2s(st->cdf, t.dfirst + cal_n, bcd, full);
        bulk_g2s(st->ctf, t.tfirst + cal_n, bcd, full);
        if (bpu) bulk_g2s(st->pu, t.util + pal, bpu, full);
        if (bcu) bulk_g2s(st->cu, t.util + cal, bcu, full);
        if (bgu) bulk_g2s(st->gu, t.u + gal, bgu, full);
    }
    // Thread c takes parent c and children c, c + 256, c + 512; the strategy entries of all of them are
    // loaded in one round before phase 0.
    __device__ void consume(const Stage &st, const Tile &ti, int c) const {
        constexpr int kC = kSBConsumerWarps * 32;
        const bool act = c < ti.n;
        const int32_t k = ti.o + c;
        uint32_t m = 0;
        int32_t c0 = 0, t0 = 0, qb = 0;
        int na = 0, p = 0;
        float r1 = 0.f, r2 = 0.f;
        float s[NA];
        if (act) {
            const uint32_t w = st.qp[k];
            m = st.km[k];
            c0 = st.df[k];
            na = (st.df[k + 1] - c0) + __popc(m);
            t0 = st.tf[k];
            r1 = st.r1[k];
            r2 = st.r2[k];
            qb = qp_base(w);
            p = qp_player(w);
#pragma unroll
            for (int a = 0; a < NA; ++a) s[a] = a < na ? __ldg(t.sigma + qb + a) : 0.f;
        }
        uint32_t cm[kPCPer];
        int32_t cw[kPCPer];
        float sc[kPCPer][NA];
#pragma unroll
        for (int r = 0; r < kPCPer; ++r) {
            const int32_t ci = c + r * kC;
            cm[r] = 0;
            cw[r] = 0;
            if (ci < ti.nc) {
                cw[r] = (int32_t)st.cqp[ti.co + ci];
                cm[r] = st.ckm[ti.co + ci];
                const int cna = (st.cdf[ti.co + ci + 1] - st.cdf[ti.co + ci]) + __popc(cm[r]);
                const int32_t cq = qp_base((uint32_t)cw[r]);
#pragma unroll
                for (int b = 0; b < NA; ++b) sc[r][b] = b < cna ? __ldg(t.sigma + cq + b) : 0.f;
            }
        }
        // phase 0: parent c's top-down step, the children's reaches to shared memory
        if (act) pair_parent_topdown<NA>(t, c0 - ti.cs, na, m, p, r1, r2, qb, s, q1, q2);
        consumers_sync();
        // phase 1: the children's bottom-up steps (grandchildren's values and terminal utilities staged)
#pragma unroll
        for (int r = 0; r < kPCPer; ++r) {
            const int32_t ci = c + r * kC;
            if (ci >= ti.nc) continue;
            const uint32_t w = (uint32_t)cw[r];
            const int32_t cq = qp_base(w);
            const int cp = qp_player(w);
            const int32_t cd = st.cdf[ti.co + ci];
            const int cna = (st.cdf[ti.co + ci + 1] - cd) + __popc(cm[r]);
            const float *tv = st.cu + (st.ctf[ti.co + ci] - ti.cal);
            const float *dv = st.gu + (cd - ti.gal);
            const uint32_t mm = cm[r];
            float ud = 0.f;
            float v[NA];
            if (cna <= NA) {
#pragma unroll
                for (int b = 0; b < NA; ++b) {
                    if (b < cna) {
                        const int kt = __popc(mm & ((1u << b) - 1u));
                        const float *src = ((mm >> b) & 1u) ? tv + kt : dv + (b - kt);
                        v[b] = *src;
                        ud = madd(ud, sc[r][b], v[b]);
                    }
                }
            } else {
                int kt = 0, kd = 0;
                for (int b = 0; b < cna; ++b) {
                    const float val = ((mm >> b) & 1u) ? tv[kt++] : dv[kd++];
                    ud = madd(ud, __ldg(t.sigma + cq + b), val);
                }
            }
            cv[ci] = ud;
            const float cq1 = q1[ci], cq2 = q2[ci];
            if (record) {
                const int32_t cg = ti.cs + ci;
                t.u[cg] = ud;
                t.reach1[cg] = cq1;
                t.reach2[cg] = cq2;
            }
            if (!collects(t, cp)) continue;
            const float wr = cp == 1 ? cq1 : -cq2;
            if (wr == 0.f) continue;
            if (cna <= NA) {
#pragma unroll
                for (int b = 0; b < NA; ++b)
                    if (b < cna) atomicAdd(&t.inst[cq + b], wr * (v[b] - ud));
            } else {
                int kt = 0, kd = 0;
                for (int b = 0; b < cna; ++b) {
                    const float val = ((mm >> b) & 1u) ? tv[kt++] : dv[kd++];
                    atomicAdd(&t.inst[cq + b], wr * (val - ud));
                }
            }
        }
        consumers_sync();
        // phase 2: parent c's bottom-up step
        if (!act) return;
        const float *pv = st.pu + (t0 - ti.pal);
        const float *dv = cv + (c0 - ti.cs);
        float ud = 0.f;
        if (na <= NA) {
            float v[NA];
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                if (a < na) {
                    const int kt = __popc(m & ((1u << a) - 1u));   // terminal children before action a
                    const float *src = ((m >> a) & 1u) ? pv + kt : dv + (a - kt);
                    v[a] = *src;
                }
            }
#pragma unroll
            for (int a = 0; a < NA; ++a)
                if (a < na) ud = madd(ud, s[a], v[a]);
            t.u[ti.j0 + c] = ud;
            if (!collects(t, p)) return;
            const float wr = p == 1 ? r1 : -r2;
            if (wr == 0.f) return;
#pragma unroll
            for (int a = 0; a < NA; ++a)
                if (a < na) atomicAdd(&t.inst[qb + a], wr * (v[a] - ud));
            return;
        }
        int kt = 0, kd = 0;
        for (int a = 0; a < na; ++a) {
            const float val = ((m >> a) & 1u) ? pv[kt++] : dv[kd++];
            ud = madd(ud, __ldg(t.sigma + qb + a), val);
        }
        t.u[ti.j0 + c] = ud;
        if (!collects(t, p)) return;
        const float wr = p == 1 ? r1 : -r2;
        if (wr == 0.f) return;
        kt = kd = 0;
        for (int a = 0; a < na; ++a) {
            const float val = ((m >> a) & 1u) ? pv[kt++] : dv[kd++];
            atomicAdd(&t.inst[qb + a], wr * (val - ud));
        }
    }
};

template <int NA>
__global__ void __launch_bounds__(kSBThreads) k_pair_bottomup(DevTree<float> t, const int4 *tm, int32_t nt,
                                                              int32_t record, int *err) {
    grid_dependency_wait();
    __shared__ float q1[kPC], q2[kPC], cv[kPC];
    run_pipeline(PairBottomUpTiles<NA>{t, tm, nt, record, q1, q2, cv}, err);
}

// Unrolled action counts the streamed kernels are built for; a depth takes the smallest one that
// covers its largest (non-wide) node.
constexpr int kStreamNA[3] = {3, 5, 8};

}  // namespace
}  // namespace cfrgb
