// Batched solving of many independent games in one persistent launch (FP32 mode).
//
// The games' state (R, S, sigma) lives in one forest layout (layout.hpp, forest = true): every depth
// lists its nodes game by game, so game g's decision nodes at depth l are one range dlo[g][l] ..
// dhi[g][l] - 1 and its player infosets first seen at depth l one range hlo[g][l] .. hhi[g][l] - 1; the
// best response walks that layout, a block per game.  The iterations run on per-game images in shared
// memory (k_batch_smem below): a block takes a game from a work counter (largest games first), runs all
// K iterations of it, and takes the next.  Per game, the global timer is read when its first iteration
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

// ---- games resident in shared memory -----------------------------------------------------------------
// A game small enough is solved entirely in shared memory: its image - its own single-game layout with
// local indices (layout.hpp), built on the host - is copied in, R, S and sigma are gathered from the
// batch's arrays through the image's slot map, all K iterations run with block barriers only, and the
// state is written back.  The per-node and per-infoset steps are the single-game kernels' (td_node,
// bu_node, own_infoset, update_row) on generic pointers into shared memory.
//
// Image layout (32-bit words; every section starts on a 16-byte boundary):
//   [0, 20)  header: Nd, Nt, H, Hp, Q, L, the word offsets of dlevel, hlevel, dfirst, tfirst, kmask, qp,
//            util (float, Nt), qbase, pseq, pseq_h, iplayer (int8), sigma0 (float, Q) and qmap (int32, Q:
//            local slot -> batch slot, -1 for a chance slot), then the image's length in words (a
//            multiple of 4)
//   then     those sections, in that order
// and after the image, in shared memory, the work arrays: reach1, reach2, u (Nd), inst, sigma (Q),
// own (H) as float, R and S (Q) as double.
enum {
    kImgNd = 0, kImgNt, kImgH, kImgHp, kImgQ, kImgL, kImgDlevel, kImgHlevel, kImgDfirst, kImgTfirst, kImgKmask,
    kImgQp, kImgUtil, kImgQbase, kImgPseq, kImgPseqH, kImgIplayer, kImgSigma0, kImgQmap, kImgWords, kImgHeader = 20
};

__host__ __device__ inline int64_t smem_align16(int64_t bytes) { return (bytes + 15) & ~(int64_t)15; }

// Bytes of shared memory a game needs: its image (words) plus the work arrays.
__host__ __device__ inline int64_t smem_game_bytes(int64_t words, int64_t Nd, int64_t H, int64_t Q) {
    return smem_align16(4 * words) + smem_align16(12 * Nd) + smem_align16(8 * Q) + smem_align16(4 * H) +
           smem_align16(16 * Q);
}

template <int NA, int V>
__global__ void __launch_bounds__(256) k_batch_smem(const int32_t *images, const int64_t *img_off, const int32_t *order,
                                                    int32_t G, int32_t *next, double *gR, double *gS, float *gsigma,
                                                    const int64_t *T0p, int32_t K, int32_t linear, double3 dcfr,
                                                    int32_t alternating, unsigned long long *t_start,
                                                    unsigned long long *t_end) {
    grid_dependency_wait();
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int32_t slot;
    const int32_t tid = (int32_t)threadIdx.x, bs = (int32_t)blockDim.x;
    const int64_t T0 = *T0p;
    for (;;) {
        __syncthreads();
        if (tid == 0) slot = atomicAdd(next, 1);
        __syncthreads();
        if (slot >= G) return;
        const int32_t g = order[slot];
        const int32_t *img = images + img_off[g];
        const int32_t words = img[kImgWords];
        {   // the image, 16 bytes at a time (words is a multiple of 4)
            const int4 *src = reinterpret_cast<const int4 *>(img);
            int4 *dst = reinterpret_cast<int4 *>(smem);
            for (int32_t i = tid; i < words / 4; i += bs) dst[i] = __ldg(src + i);
        }
        __syncthreads();
        const int32_t *w = reinterpret_cast<const int32_t *>(smem);
        const int32_t Nd = w[kImgNd], H = w[kImgH], Hp = w[kImgHp], Q = w[kImgQ], L = w[kImgL];
        unsigned char *p = smem + smem_align16(4 * (int64_t)words);
        DevTree<float> t{};
        t.reach1 = reinterpret_cast<float *>(p);
        t.reach2 = t.reach1 + Nd;
        t.u = t.reach2 + Nd;
        p += smem_align16(12 * (int64_t)Nd);
        t.inst = reinterpret_cast<float *>(p);
        t.sigma = t.inst + Q;
        p += smem_align16(8 * (int64_t)Q);
        t.own = reinterpret_cast<float *>(p);
        p += smem_align16(4 * (int64_t)H);
        t.R = reinterpret_cast<double *>(p);
        t.S = t.R + Q;
        t.dfirst = w + w[kImgDfirst];
        t.tfirst = w + w[kImgTfirst];
        t.kmask = reinterpret_cast<const uint32_t *>(w + w[kImgKmask]);
        t.qp = reinterpret_cast<const uint32_t *>(w + w[kImgQp]);
        t.util = reinterpret_cast<const float *>(w + w[kImgUtil]);
        t.qbase = w + w[kImgQbase];
        t.pseq = w + w[kImgPseq];
        t.pseq_h = w + w[kImgPseqH];
        t.iplayer = reinterpret_cast<const int8_t *>(w + w[kImgIplayer]);
        t.wbits = nullptr;
        t.pmask = 6;
        const float *sigma0 = reinterpret_cast<const float *>(w + w[kImgSigma0]);
        const int32_t *qmap = w + w[kImgQmap];
        const int32_t *dlevel = w + w[kImgDlevel], *hlevel = w + w[kImgHlevel];
        // the state: player slots from the batch's arrays, chance slots sigma_0; the root's reaches 1
        for (int32_t q = tid; q < Q; q += bs) {
            const int32_t bq = qmap[q];
            if (bq >= 0) {
                t.R[q] = gR[bq];
                t.S[q] = gS[bq];
                t.sigma[q] = gsigma[bq];
            } else {
                t.R[q] = t.S[q] = 0.0;
                t.sigma[q] = sigma0[q];
            }
        }
        if (tid == 0 && Nd > 0) { t.reach1[0] = 1.f; t.reach2[0] = 1.f; }
        if (tid == 0) t_start[g] = batch_clock();
        __syncthreads();
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
            // one pass for both players, or (alternating updates) player 1's and then player 2's under
            // player 1's new strategy, with the same iteration weights
            for (int pass = 0; pass < (alternating ? 2 : 1); ++pass) {
                t.pmask = alternating ? (pass == 0 ? 2 : 4) : 6;
                for (int l = 0; l < L; ++l) {
                    for (int32_t h = hlevel[l] + tid; h < hlevel[l + 1]; h += bs) {
                        for (int32_t q = t.qbase[h]; q < t.qbase[h + 1]; ++q) t.inst[q] = 0.f;
                        own_infoset<float, false>(t, h);
                    }
                    if (l + 1 < L)
                        for (int32_t j = dlevel[l] + tid; j < dlevel[l + 1]; j += bs) td_node<float, true, false>(t, j);
                    __syncthreads();
                }
                for (int l = L - 1; l >= 0; --l) {
                    for (int32_t j = dlevel[l] + tid; j < dlevel[l + 1]; j += bs) bu_node<float, false, false>(t, j);
                    __syncthreads();
                }
                for (int32_t h = tid; h < Hp; h += bs)
                    if (collects(t, t.iplayer[h])) update_row<NA, V, false>(t, h, u);
                __syncthreads();
            }
        }
        if (tid == 0) t_end[g] = batch_clock();
        for (int32_t q = tid; q < Q; q += bs) {
            const int32_t bq = qmap[q];
            if (bq >= 0) {
                gR[bq] = t.R[q];
                gS[bq] = t.S[q];
                gsigma[bq] = t.sigma[q];
            }
        }
    }
}

// The iteration count after a batched launch of K iterations.
__global__ void k_batch_advance(int64_t *T, int32_t K) { *T += K; }

}  // namespace
}  // namespace cfrgb

