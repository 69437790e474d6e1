// Batched solving of many independent games in one persistent launch (FP32 mode).
//
// The games are laid out as one forest (layout.hpp, forest = true): every depth lists its nodes game by
// game, so game g's decision nodes at depth l are one range dlo[g][l] .. dhi[g][l] - 1 and its player
// infosets first seen at depth l one range hlo[g][l] .. hhi[g][l] - 1.  A block takes a game from a
// work counter (largest games first), runs all K iterations of it depth by depth with block barriers
// between the depths - the same per-node and per-infoset steps as the single-game kernels (td_node,
// bu_node, own_infoset, update_row), with loads through L2 since the block wrote the data earlier in
// the launch - and takes the next game.  Per game, the global timer is read when its first iteration
// starts and when its last ends.
#pragma once

#include <cstdint>

#include "kernels.cuh"

namespace cfrgb {
namespace {   // device code: internal to each translation unit that includes it

struct BatchDesc {
    const int32_t *order;          // games, largest first
    const int32_t *dlo, *dhi;      // [G][stride]: per game and depth, its decision nodes [dlo, dhi)
    const int32_t *hlo, *hhi;      // [G][stride]: per game and depth, its player infosets first seen there
    const int32_t *nlev;           // [G]: depths holding decision nodes
    int32_t G, stride;
    int32_t *next;                 // work counter (zeroed before the launch)
    unsigned long long *t_start, *t_end;   // [G] global timer (ns)
};

__device__ __forceinline__ unsigned long long batch_clock() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// The next game of this block (every thread gets it), or -1.
__device__ __forceinline__ int32_t batch_take(const BatchDesc &d, int32_t *slot) {
    __syncthreads();                                   // the previous game's last reads of *slot are done
    if (threadIdx.x == 0) *slot = atomicAdd(d.next, 1);
    __syncthreads();
    const int32_t i = *slot;
    return i < d.G ? d.order[i] : -1;
}

// K iterations of every game, T0 + 1 .. T0 + K (T0 = *T0p, the iterations already run).  V: variant
// (CFRV_*); NA: unrolled action count of the update (the batch's largest); linear: linear averaging for
// vanilla / CFR+.
template <int NA, int V>
__global__ void __launch_bounds__(1024) k_batch_iterate(DevTree<float> t, BatchDesc d, const int64_t *T0p, int32_t K,
                                                        int32_t linear, double3 dcfr) {
    grid_dependency_wait();
    __shared__ int32_t slot;
    const int32_t tid = (int32_t)threadIdx.x, bs = (int32_t)blockDim.x;
    const int64_t T0 = *T0p;
    for (int32_t g = batch_take(d, &slot); g >= 0; g = batch_take(d, &slot)) {
        const size_t o = (size_t)g * d.stride;
        const int32_t *dlo = d.dlo + o, *dhi = d.dhi + o, *hlo = d.hlo + o, *hhi = d.hhi + o;
        const int L = d.nlev[g];
        if (tid == 0) d.t_start[g] = batch_clock();
        for (int32_t it = 1; it <= K; ++it) {
            const double T = (double)(T0 + it);
            UpdWeights u;
            u.T = T;
            u.fpos = u.fneg = 1.0;
            u.w = linear ? (float)T : 1.f;
            if (V == CFRV_LINEAR) u.w = (float)T;
            if (V == CFRV_DISCOUNTED) {
                const double ta = pow(T, dcfr.x), tb = pow(T, dcfr.y);
                u.fpos = ta / (ta + 1.0);
                u.fneg = tb / (tb + 1.0);
                u.w = (float)pow(T, dcfr.z);
            }
            // depth by depth: r~ zeroed and own reaches of the infosets first seen at depth l, and the
            // top-down step from depth l
            for (int l = 0; l < L; ++l) {
                for (int32_t h = hlo[l] + tid; h < hhi[l]; h += bs) {
                    for (int32_t q = t.qbase[h]; q < t.qbase[h + 1]; ++q) t.inst[q] = 0.f;
                    own_infoset<float, true>(t, h);
                }
                if (l + 1 < L)
                    for (int32_t j = dlo[l] + tid; j < dhi[l]; j += bs) td_node<float, true, true>(t, j);
                __syncthreads();
            }
            for (int l = L - 1; l >= 0; --l) {
                for (int32_t j = dlo[l] + tid; j < dhi[l]; j += bs) bu_node<float, false, true>(t, j);
                __syncthreads();
            }
            for (int l = 0; l < L; ++l)
                for (int32_t h = hlo[l] + tid; h < hhi[l]; h += bs) update_row<NA, V, true>(t, h, u);
            __syncthreads();
        }
        if (tid == 0) d.t_end[g] = batch_clock();
    }
}

// Best responses of both players against every game's average strategy (b.avg, filled beforehand):
// out[2 g + p - 1] = the value of player p's best response in game g.  b.cfv must be zero on entry.
__global__ void __launch_bounds__(256) k_batch_br(DevBR b, BatchDesc d, double *out) {
    __shared__ int32_t slot;
    const int32_t tid = (int32_t)threadIdx.x, bs = (int32_t)blockDim.x;
    for (int32_t g = batch_take(d, &slot); g >= 0; g = batch_take(d, &slot)) {
        const size_t o = (size_t)g * d.stride;
        const int32_t *dlo = d.dlo + o, *dhi = d.dhi + o, *hlo = d.hlo + o, *hhi = d.hhi + o;
        const int L = d.nlev[g];
        for (int32_t player = 1; player <= 2; ++player) {
            if (L == 0) {
                if (tid == 0) out[2 * g + player - 1] = 0.0;   // a terminal root: nothing to respond to
                continue;
            }
            if (tid == 0) b.preach[dlo[0]] = 1.0;
            __syncthreads();
            for (int l = 0; l + 1 < L; ++l) {
                for (int32_t j = dlo[l] + tid; j < dhi[l]; j += bs) br_topdown_node<true>(b, j, player);
                __syncthreads();
            }
            for (int l = L - 1; l >= 0; --l) {
                for (int32_t j = dlo[l] + tid; j < dhi[l]; j += bs) br_node<true>(b, j, player);
                __syncthreads();
                for (int32_t h = hlo[l] + tid; h < hhi[l]; h += bs) br_choose<true>(b, h, player);
                __syncthreads();
                for (int32_t j = dlo[l] + tid; j < dhi[l]; j += bs) br_pick<true>(b, j, player);
                __syncthreads();
            }
            if (tid == 0) out[2 * g + player - 1] = __ldcg(b.val + dlo[0]);
            // clear the game's cfv for the other player's pass
            for (int l = 0; l < L; ++l)
                for (int32_t h = hlo[l] + tid; h < hhi[l]; h += bs)
                    for (int32_t q = b.qbase[h]; q < b.qbase[h + 1]; ++q) b.cfv[q] = 0.0;
            __syncthreads();
        }
    }
}

// The iteration count after a batched launch of K iterations.
__global__ void k_batch_advance(int64_t *T, int32_t K) { *T += K; }

}  // namespace
}  // namespace cfrgb

