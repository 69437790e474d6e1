// Device kernels of one full-tree CFR iteration over the level-ordered layout (layout.hpp).
//
//   k_topdown   depth l -> l+1: counterfactual reaches of the decision children (Eq. 2 / Eq. 13,
//               the top-down recurrence for Pi-check) and, for the infosets whose shallowest depth
//               is l, the own reach pi_i(h) (Eq. 4 restricted to the acting player).
//   k_bottomup  depth l: node values u(d) = sum_a sigma(h,a) u(child_a) (Eq. 1 / Eq. 11) and the
//               instantaneous regret scatter r~(h,a) += pi-check(d) (u_p(child_a) - u_p(d)) (Eq. 7,
//               summed over the nodes of h as in Eq. 3 and Eq. 6; the vector form of Section 3.2.3).
//   k_update    per infoset: R += r~ (Eq. 8 / Eq. 15 as a cumulative sum; CFR+ clips at 0),
//               S += w_T pi_i(h) sigma (Eq. 10 / Eq. 14 numerator), sigma' = regret matching (Eq. 9).
//
// Per decision node the tree layout costs dfirst/tfirst/dinfo/kmask (4 B each);
// the infoset tables (qbase, iplayer) and the strategy sigma are small and stay L2-resident.
#pragma once

#include <cstdint>

namespace cfrgb {

// Whether action a of a node with na actions leads to a terminal (see layout.hpp).
__device__ __forceinline__ bool is_terminal(uint32_t m, const uint32_t *wbits, int na, int a) {
    return na > 32 ? ((wbits[m + (a >> 5)] >> (a & 31)) & 1u) : ((m >> a) & 1u);
}

// acc + a * b.  FP64 rounds the product and the sum separately (no fused multiply-add), so the
// FP64 path performs exactly the operations of a plain sequential evaluation; FP32 fuses.
__device__ __forceinline__ double madd(double acc, double a, double b) { return __dadd_rn(acc, __dmul_rn(a, b)); }
__device__ __forceinline__ float madd(float acc, float a, float b) { return fmaf(a, b, acc); }

template <typename real>
struct DevTree {
    const int32_t *dfirst, *tfirst, *dinfo;
    const uint32_t *kmask;     // terminal-child mask, or offset into wbits when |A| > 32
    const uint32_t *wbits;
    const real *util;          // u(t, 1) per terminal
    const int32_t *qbase;      // [H + 1]
    const int8_t *iplayer;     // [H]
    const int32_t *pseq, *pseq_h;
    real *sigma, *inst;        // [Q]
    real *reach1, *reach2;     // [Nd] pi-check(d, 1) = r_c r_2, pi-check(d, 2) = r_c r_1
    real *u;                   // [Nd] u(d, 1)
    real *own;                 // [H]
    double *R, *S;             // [Q]
    int64_t *iter;             // completed iterations (device copy)
    // deterministic mode: per-edge regret contributions and the nodes of each infoset in
    // depth-first order (edge offset of node j's children: dfirst[j] + tfirst[j] - 1)
    real *contrib;             // [N - 1]
    const int32_t *hnode_start, *hnode;
};

template <typename real>
__global__ void __launch_bounds__(256) k_topdown(DevTree<real> t, int32_t j0, int32_t j1, int32_t nblk_nodes,
                                                 int32_t h0, int32_t h1, int32_t bump) {
    if (bump && blockIdx.x == 0 && threadIdx.x == 0) *t.iter += 1;
    if ((int32_t)blockIdx.x < nblk_nodes) {
        const int32_t j = j0 + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
        if (j >= j1) return;
        int32_t c = t.dfirst[j];
        if (c == t.dfirst[j + 1]) return;                 // no decision children
        const int32_t h = t.dinfo[j];
        const int p = t.iplayer[h];
        const int32_t qb = t.qbase[h];
        const int na = t.qbase[h + 1] - qb;
        const uint32_t m = t.kmask[j];
        const real r1 = t.reach1[j], r2 = t.reach2[j];
        for (int a = 0; a < na; ++a) {
            if (is_terminal(m, t.wbits, na, a)) continue;
            const real s = t.sigma[qb + a];
            t.reach1[c] = p == 1 ? r1 : r1 * s;
            t.reach2[c] = p == 2 ? r2 : r2 * s;
            ++c;
        }
    } else {
        const int32_t h = h0 + (int32_t)((blockIdx.x - nblk_nodes) * blockDim.x + threadIdx.x);
        if (h >= h1 || t.iplayer[h] == 0) return;
        const int32_t ps = t.pseq[h];
        t.own[h] = ps < 0 ? real(1) : t.own[t.pseq_h[h]] * t.sigma[ps];
    }
}

// kDet = false: the regret contributions are added to inst with atomics (order unspecified).
// kDet = true: they are stored per edge and k_update sums them per infoset in depth-first node
// order, which makes the result independent of scheduling.
template <typename real, bool kDet>
__global__ void __launch_bounds__(256) k_bottomup(DevTree<real> t, int32_t j0, int32_t j1) {
    const int32_t j = j0 + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (j >= j1) return;
    const int32_t h = t.dinfo[j];
    const int p = t.iplayer[h];
    const int32_t qb = t.qbase[h];
    const int na = t.qbase[h + 1] - qb;
    const uint32_t m = t.kmask[j];
    const int32_t c0 = t.dfirst[j], t0 = t.tfirst[j];
    real ud = 0;
    int32_t c = c0, tt = t0;
    for (int a = 0; a < na; ++a) {
        const real v = is_terminal(m, t.wbits, na, a) ? t.util[tt++] : t.u[c++];
        ud = madd(ud, t.sigma[qb + a], v);
    }
    t.u[j] = ud;
    if (p == 0) return;
    const real w = p == 1 ? t.reach1[j] : -t.reach2[j];   // u_2 = -u_1
    if (!kDet && w == real(0)) return;
    c = c0; tt = t0;
    real *out = kDet ? t.contrib + (c0 + t0 - 1) : nullptr;
    for (int a = 0; a < na; ++a) {
        const real v = is_terminal(m, t.wbits, na, a) ? t.util[tt++] : t.u[c++];
        if (kDet) out[a] = w * (v - ud);
        else atomicAdd(&t.inst[qb + a], w * (v - ud));
    }
}

template <typename real>
__device__ __forceinline__ void regret_match(real *sigma, const double *R, int32_t qb, int na) {
    double pos = 0.0;
    for (int a = 0; a < na; ++a) pos += R[qb + a] > 0.0 ? R[qb + a] : 0.0;
    for (int a = 0; a < na; ++a) {
        const double r = R[qb + a];
        sigma[qb + a] = (real)(pos > 0.0 ? (r > 0.0 ? r : 0.0) / pos : 1.0 / na);
    }
}

template <typename real, bool kDet>
__global__ void __launch_bounds__(256) k_update(DevTree<real> t, int32_t H, int32_t plus, int32_t linear) {
    const int32_t h = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (h >= H || t.iplayer[h] == 0) return;
    const int32_t qb = t.qbase[h];
    const int na = t.qbase[h + 1] - qb;
    if (kDet) {
        for (int a = 0; a < na; ++a) t.inst[qb + a] = real(0);
        for (int32_t i = t.hnode_start[h]; i < t.hnode_start[h + 1]; ++i) {
            const int32_t j = t.hnode[i];
            const real *src = t.contrib + (t.dfirst[j] + t.tfirst[j] - 1);
            for (int a = 0; a < na; ++a) t.inst[qb + a] += src[a];
        }
    }
    const double w = linear ? (double)*t.iter : 1.0;
    const double wo = __dmul_rn(w, (double)t.own[h]);
    for (int a = 0; a < na; ++a) {
        double r = t.R[qb + a] + (double)t.inst[qb + a];
        if (plus) r = r > 0.0 ? r : 0.0;
        t.R[qb + a] = r;
        t.S[qb + a] = madd(t.S[qb + a], wo, (double)t.sigma[qb + a]);
    }
    regret_match(t.sigma, t.R, qb, na);
}

// sigma := regret matching of R for every player infoset (uniform when R = 0: sigma^(1)).
template <typename real>
__global__ void k_regret_match_all(real *sigma, const double *R, const int32_t *qbase, const int8_t *iplayer, int32_t H) {
    const int32_t h = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (h >= H || iplayer[h] == 0) return;
    regret_match(sigma, R, qbase[h], qbase[h + 1] - qbase[h]);
}

// out[user slot] = src[internal slot], widened to double.
template <typename T>
__global__ void k_gather_q(const T *src, const int32_t *q_int2user, double *out, int32_t Q) {
    const int32_t q = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (q < Q) out[q_int2user[q]] = (double)src[q];
}

// dst[internal slot] = src[user slot] for player infosets, 0 for chance infosets.
__global__ void k_scatter_player_q(const double *src, const int32_t *q_int2user, const int32_t *qbase,
                                   const int8_t *iplayer, double *dst, int32_t H) {
    const int32_t h = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (h >= H) return;
    for (int32_t q = qbase[h]; q < qbase[h + 1]; ++q) dst[q] = iplayer[h] == 0 ? 0.0 : src[q_int2user[q]];
}

// Average strategy (Eq. 10 normalised) in internal order: S / sum S, uniform if the sum is 0;
// chance infosets copy sigma_0 (FP64).
__global__ void k_average(const double *S, const double *sigma0, const int32_t *qbase, const int8_t *iplayer,
                          double *avg, int32_t H) {
    const int32_t h = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (h >= H) return;
    const int32_t qb = qbase[h];
    const int na = qbase[h + 1] - qb;
    if (iplayer[h] == 0) {
        for (int a = 0; a < na; ++a) avg[qb + a] = sigma0[qb + a];
        return;
    }
    double s = 0.0;
    for (int a = 0; a < na; ++a) s += S[qb + a];
    for (int a = 0; a < na; ++a) avg[qb + a] = s > 0.0 ? S[qb + a] / s : 1.0 / na;
}

// ---- best response (FP64), used by cfr_exploitability -------------------------------------------
// Player i's best response against a fixed profile (the average strategy): top-down the reach of
// chance and the opponent, pi_-i(d); bottom-up per depth, values v(d) = sum_a avg(h,a) v(child_a) at
// nodes of chance/the opponent, and at i's nodes v(d) = v(child_{a*(h)}) with
// a*(h) = argmax_a sum_{d in h} pi_-i(d) v(child_a(d)).  Needs every infoset at a single depth.

struct DevBR {
    const int32_t *dfirst, *tfirst, *dinfo;
    const uint32_t *kmask, *wbits;
    const double *util;        // u(t, 1) in FP64
    const int32_t *qbase;
    const int8_t *iplayer;
    const double *avg;         // [Q] internal
    double *preach, *val;      // [Nd]
    double *cfv;               // [Q]
    int32_t *astar;            // [H]
};

__global__ void __launch_bounds__(256) k_br_topdown(DevBR b, int32_t j0, int32_t j1, int32_t player) {
    const int32_t j = j0 + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (j >= j1) return;
    int32_t c = b.dfirst[j];
    if (c == b.dfirst[j + 1]) return;
    const int32_t h = b.dinfo[j];
    const bool mine = b.iplayer[h] == player;
    const int32_t qb = b.qbase[h];
    const int na = b.qbase[h + 1] - qb;
    const uint32_t m = b.kmask[j];
    const double r = b.preach[j];
    for (int a = 0; a < na; ++a) {
        if (is_terminal(m, b.wbits, na, a)) continue;
        b.preach[c++] = mine ? r : r * b.avg[qb + a];
    }
}

__device__ __forceinline__ double br_child(const DevBR &b, uint32_t m, int na, int a, int32_t &c, int32_t &tt,
                                           double sign) {
    return is_terminal(m, b.wbits, na, a) ? sign * b.util[tt++] : b.val[c++];
}

__global__ void __launch_bounds__(256) k_br_nodes(DevBR b, int32_t j0, int32_t j1, int32_t player) {
    const int32_t j = j0 + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (j >= j1) return;
    const int32_t h = b.dinfo[j];
    const int32_t qb = b.qbase[h];
    const int na = b.qbase[h + 1] - qb;
    const uint32_t m = b.kmask[j];
    const double sign = player == 1 ? 1.0 : -1.0;
    int32_t c = b.dfirst[j], tt = b.tfirst[j];
    if (b.iplayer[h] != player) {
        double v = 0.0;
        for (int a = 0; a < na; ++a) v += b.avg[qb + a] * br_child(b, m, na, a, c, tt, sign);
        b.val[j] = v;
    } else {
        const double r = b.preach[j];
        if (r == 0.0) return;
        for (int a = 0; a < na; ++a) {
            const double v = br_child(b, m, na, a, c, tt, sign);
            atomicAdd(&b.cfv[qb + a], r * v);
        }
    }
}

__global__ void k_br_choose(DevBR b, int32_t h0, int32_t h1, int32_t player) {
    const int32_t h = h0 + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (h >= h1 || b.iplayer[h] != player) return;
    const int32_t qb = b.qbase[h];
    const int na = b.qbase[h + 1] - qb;
    int best = 0;
    for (int a = 1; a < na; ++a)
        if (b.cfv[qb + a] > b.cfv[qb + best]) best = a;
    b.astar[h] = best;
}

__global__ void __launch_bounds__(256) k_br_pick(DevBR b, int32_t j0, int32_t j1, int32_t player) {
    const int32_t j = j0 + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (j >= j1) return;
    const int32_t h = b.dinfo[j];
    if (b.iplayer[h] != player) return;
    const uint32_t m = b.kmask[j];
    const int na = b.qbase[h + 1] - b.qbase[h];
    const int as = b.astar[h];
    int32_t c = b.dfirst[j], tt = b.tfirst[j];
    double v = 0.0;
    for (int a = 0; a <= as; ++a) v = br_child(b, m, na, a, c, tt, player == 1 ? 1.0 : -1.0);
    b.val[j] = v;
}

}  // namespace cfrgb
