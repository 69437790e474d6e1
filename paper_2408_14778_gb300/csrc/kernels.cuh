// Device kernels of one full-tree CFR iteration over the level-ordered layout (layout.hpp).
//
//   own reach   per depth l, for the infosets whose shallowest depth is l: pi_i(h) (Eq. 4 restricted
//               to the acting player), from the parent sequence's own reach; independent of the node
//               passes, so it runs on a parallel branch of the iteration's graph.
//   top-down    depth l -> l+1: counterfactual reaches of the decision children (Eq. 2 / Eq. 13,
//               the top-down recurrence for Pi-check).
//   bottom-up   depth l: node values u(d) = sum_a sigma(h,a) u(child_a) (Eq. 1 / Eq. 11) and the
//               instantaneous regret scatter r~(h,a) += pi-check(d) (u_p(child_a) - u_p(d)) (Eq. 7,
//               summed over the nodes of h as in Eq. 3 and Eq. 6; the vector form of Section 3.2.3).
//   update      per infoset: R += r~ (Eq. 8 / Eq. 15 as a cumulative sum; CFR+ clips at 0),
//               S += w_T pi_i(h) sigma (Eq. 10 / Eq. 14 numerator), sigma' = regret matching (Eq. 9).
//
// One kernel per depth and step; one iteration's launches are captured into a CUDA graph.  The step
// bodies are __device__ functions; their template flag C selects L1-bypassing loads for callers that
// read data written earlier in the same launch (the kernels here read with ordinary cached loads).
// Per decision node the layout costs dfirst/tfirst/kmask/qp (4 B each); the infoset tables and the
// strategy sigma are small and mostly L2-resident.
#pragma once

#include <cstdint>

namespace cfrgb {
namespace {   // device code: internal to each translation unit that includes it

// Whether action a of a node with na actions leads to a terminal (see layout.hpp).
__device__ __forceinline__ bool is_terminal(uint32_t m, const uint32_t *wbits, int na, int a) {
    return na > 32 ? ((wbits[m + (a >> 5)] >> (a & 31)) & 1u) : ((m >> a) & 1u);
}

// acc + a * b.  FP64 rounds the product and the sum separately (no fused multiply-add), so the
// FP64 path performs exactly the operations of a plain sequential evaluation; FP32 fuses.
__device__ __forceinline__ double madd(double acc, double a, double b) { return __dadd_rn(acc, __dmul_rn(a, b)); }
__device__ __forceinline__ float madd(float acc, float a, float b) { return fmaf(a, b, acc); }

// Load of data written during the current launch (C = true: through L2, bypassing a possibly
// stale L1 line of this SM).
template <bool C, typename T>
__device__ __forceinline__ T ldm(const T *p) {
    if constexpr (C) return __ldcg(p);
    else return *p;
}

// Waits until the kernels this launch depends on have completed and their writes are visible.  The
// iteration's kernels are launched as programmatic dependent launches (their blocks may be scheduled
// while the previous kernel drains), so each calls this before touching memory; for an ordinary
// launch it returns at once.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Per-node word qp (layout.hpp): the infoset's first slot, a wide flag and the acting player.
__device__ __forceinline__ int32_t qp_base(uint32_t w) { return (int32_t)(w & 0x1fffffffu); }
__device__ __forceinline__ bool qp_wide(uint32_t w) { return (w >> 29) & 1u; }
__device__ __forceinline__ int qp_player(uint32_t w) { return (int)(w >> 30); }

// Number of terminal children among actions 0..a-1 of a node whose mask words are wb.
__device__ __forceinline__ int terminals_before(const uint32_t *wb, int a) {
    int n = __popc(wb[a >> 5] & ((1u << (a & 31)) - 1u));
    for (int w = 0; w < (a >> 5); ++w) n += __popc(wb[w]);
    return n;
}

// Exact float -> double by bit manipulation (integer pipe); zero keeps its sign, and subnormal,
// infinite or NaN inputs take the hardware conversion.  GB300's FP64 pipe is narrow (ncu: the row update
// had it 80% busy with two additions and a conversion per slot); with narrow and add_nonneg below, the
// update's only FP64 operation per slot is the regret addition.
__device__ __forceinline__ double widen(float x) {
    const uint32_t b = __float_as_uint(x);
    if ((b << 1) == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
    const uint32_t e = (b >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) return (double)x;
    const uint32_t hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)(b << 29));
}

// double -> float rounded to nearest, ties to even, by integer operations where the result is a normal
// FP32 number (biased double exponent 897 .. 1150): the top 23 of the 52 fraction bits are kept and the
// 29 dropped bits round them (above half, or exactly half with an odd kept part, adds one; a carry out of
// the fraction moves into the exponent, and past the largest finite value gives infinity, as the
// rounding rule does).  Zero, subnormal results, overflow of the exponent range, infinities and NaN take
// the hardware conversion, which would otherwise occupy the FP64 pipe once per slot.
__device__ __forceinline__ float narrow(double x) {
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const uint32_t e = (hi >> 20) & 0x7ffu;
    if (e - 897u > 253u) return __double2float_rn(x);
    const uint32_t m = (((hi & 0x7fffffffu) - (896u << 20)) << 3) | (lo >> 29);
    const uint32_t up = ((lo & 0x1fffffffu) + (m & 1u)) > 0x10000000u;
    return __uint_as_float((hi & 0x80000000u) | (m + up));
}

// a + b for a, b >= 0, rounded to nearest, ties to even, by integer operations (the average-strategy
// sum S and its increment are never negative).  With A >= B as bit patterns, B's significand is shifted
// right by the exponent gap, the bits shifted out kept as a sticky bit below the two guard bits; the
// sum is normalised by at most one place (a carry), then rounded on the three low bits, a carry out of
// the significand moving into the exponent and past the largest finite value giving infinity.  A zero
// or subnormal smaller operand, and any infinity, NaN or negative input, take the FP64 addition.
__device__ __forceinline__ double add_nonneg(double a, double b) {
    uint64_t A = (uint64_t)__double_as_longlong(a), B = (uint64_t)__double_as_longlong(b);
    if (A < B) { const uint64_t t = A; A = B; B = t; }
    const uint32_t ea = (uint32_t)(A >> 52), eb = (uint32_t)(B >> 52);
    if (eb == 0u || ea >= 0x7ffu) return a + b;
    const uint64_t F = (1ull << 52) - 1ull, H = 1ull << 52;
    const uint64_t ma = ((A & F) | H) << 3;
    uint64_t mb = ((B & F) | H) << 3;
    const uint32_t d = ea - eb;
    mb = d >= 56u ? 1ull : (mb >> d) | (uint64_t)((mb & ((1ull << d) - 1ull)) != 0ull);
    uint64_t sum = ma + mb;
    uint32_t e = ea;
    if (sum >> 56) { sum = (sum >> 1) | (sum & 1ull); ++e; }
    const uint32_t low = (uint32_t)sum & 7u;
    uint64_t sig = sum >> 3;
    sig += (low > 4u) || (low == 4u && (sig & 1ull));
    if (sig >> 53) { sig >>= 1; ++e; }
    return __longlong_as_double((long long)(e >= 0x7ffu ? 0x7ff0000000000000ull : ((uint64_t)e << 52) | (sig & F)));
}

// Sum over the block (every thread gets it); scratch32 holds one value per warp.
template <typename real>
__device__ __forceinline__ real block_sum(real v, real *scratch32) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) scratch32[threadIdx.x >> 5] = v;
    __syncthreads();
    real s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += scratch32[w];
    __syncthreads();
    return s;
}

template <typename real>
struct DevTree {
    const int32_t *dfirst, *tfirst, *dinfo;
    const uint32_t *kmask;     // terminal-child mask, or offset into wbits when |A| > 32
    const uint32_t *wbits;
    const uint32_t *qp;        // per node: infoset's first slot | wide << 29 | player << 30
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
    int32_t pmask;             // bit p set: player p collects regrets and is updated in this pass (6: both)
    const double *wts;         // linear / discounted CFR: this iteration's weights (k_weights)
};

// Variants (the values of cfr_gb300.h's CFR_VANILLA .. CFR_DISCOUNTED).
constexpr int CFRV_VANILLA = 0, CFRV_PLUS = 1, CFRV_LINEAR = 2, CFRV_DISCOUNTED = 3;

// Whether the acting player p (0 = chance) collects regrets in this pass.
template <typename real>
__device__ __forceinline__ bool collects(const DevTree<real> &t, int p) { return (t.pmask >> p) & 1; }

// Nodes with up to kUnroll actions take a fully unrolled path in which every child-value and strategy
// load is issued before any is used.  The operations and their order are those of the general loop.
constexpr int kUnroll = 8;

// ---- step bodies ---------------------------------------------------------------------------------

// Own reach of infoset h (Eq. 4 for its acting player): the parent sequence's own reach times sigma.
template <typename real, bool C>
__device__ __forceinline__ void own_infoset(const DevTree<real> &t, int32_t h) {
    const int p = t.iplayer[h];
    if (p == 0 || !collects(t, p)) return;
    const int32_t ps = t.pseq[h];
    t.own[h] = ps < 0 ? real(1) : ldm<C>(t.own + t.pseq_h[h]) * ldm<C>(t.sigma + ps);
}

// Top-down step of decision node j: reaches of its decision children.
// kSkipWide: nodes with more than 32 actions are left to td_wide.
// The node's fields are all loaded before any is used (one memory round trip; the kernels that call
// this on small depths are latency-bound).
template <typename real, bool kSkipWide, bool C>
__device__ __forceinline__ void td_node(const DevTree<real> &t, int32_t j) {
    int32_t c = t.dfirst[j];
    const int32_t c1 = t.dfirst[j + 1];
    const uint32_t w = t.qp[j];
    const uint32_t m = t.kmask[j];
    const real r1 = ldm<C>(t.reach1 + j), r2 = ldm<C>(t.reach2 + j);
    const int32_t nd = c1 - c;
    if (nd == 0) return;                                  // no decision children
    if (kSkipWide && qp_wide(w)) return;
    const int32_t qb = qp_base(w);
    const int p = qp_player(w);
    if (!qp_wide(w)) {
        const int na = nd + __popc(m);
        if (na <= kUnroll) {
            real s[kUnroll];
#pragma unroll
            for (int a = 0; a < kUnroll; ++a) s[a] = a < na ? ldm<C>(t.sigma + qb + a) : real(0);
#pragma unroll
            for (int a = 0; a < kUnroll; ++a) {
                if (a < na && !((m >> a) & 1u)) {
                    t.reach1[c] = p == 1 ? r1 : r1 * s[a];
                    t.reach2[c] = p == 2 ? r2 : r2 * s[a];
                    ++c;
                }
            }
            return;
        }
    }
    const int na = nd + (t.tfirst[j + 1] - t.tfirst[j]);
    for (int a = 0; a < na; ++a) {
        if (is_terminal(m, t.wbits, na, a)) continue;
        const real s = ldm<C>(t.sigma + qb + a);
        t.reach1[c] = p == 1 ? r1 : r1 * s;
        t.reach2[c] = p == 2 ? r2 : r2 * s;
        ++c;
    }
}

// Bottom-up step of decision node j.
// kDet = false: the regret contributions are added to inst with atomics (order unspecified), and
// nodes with more than 32 actions are left to bu_wide.
// kDet = true: they are stored per edge and k_update sums them per infoset in depth-first node
// order, which makes the result independent of scheduling; every node is summed sequentially.
// The node's fields, both reaches included, are loaded before any is used (one memory round trip
// before the child values; the kernels that call this on small depths are latency-bound).
template <typename real, bool kDet, bool C>
__device__ __forceinline__ void bu_node(const DevTree<real> &t, int32_t j) {
    const uint32_t w = t.qp[j];
    const uint32_t m = t.kmask[j];
    const int32_t c0 = t.dfirst[j], c1 = t.dfirst[j + 1], t0 = t.tfirst[j], t1 = t.tfirst[j + 1];
    const real rr1 = ldm<C>(t.reach1 + j), rr2 = ldm<C>(t.reach2 + j);
    if (!kDet && qp_wide(w)) return;
    const int32_t qb = qp_base(w);
    const int p = qp_player(w);
    const int32_t nd = c1 - c0;
    const int na = qp_wide(w) ? nd + (t1 - t0) : nd + __popc(m);
    real *out = kDet ? t.contrib + (c0 + t0 - 1) : nullptr;
    if (na <= kUnroll) {
        real v[kUnroll], s[kUnroll];
        int kt = 0, kd = 0;
#pragma unroll
        for (int a = 0; a < kUnroll; ++a) {
            if (a < na) {
                const bool term = (m >> a) & 1u;
                v[a] = term ? t.util[t0 + kt] : ldm<C>(t.u + c0 + kd);
                kt += term;
                kd += !term;
                s[a] = ldm<C>(t.sigma + qb + a);
            }
        }
        real ud = 0;
#pragma unroll
        for (int a = 0; a < kUnroll; ++a)
            if (a < na) ud = madd(ud, s[a], v[a]);
        t.u[j] = ud;
        if (!collects(t, p)) return;
        const real wr = p == 1 ? rr1 : -rr2;   // u_2 = -u_1
        if (!kDet && wr == real(0)) return;
#pragma unroll
        for (int a = 0; a < kUnroll; ++a) {
            if (a < na) {
                if (kDet) out[a] = wr * (v[a] - ud);
                else atomicAdd(&t.inst[qb + a], wr * (v[a] - ud));
            }
        }
        return;
    }
    real ud = 0;
    int32_t c = c0, tt = t0;
    for (int a = 0; a < na; ++a) {
        const real v = is_terminal(m, t.wbits, na, a) ? t.util[tt++] : ldm<C>(t.u + c++);
        ud = madd(ud, ldm<C>(t.sigma + qb + a), v);
    }
    t.u[j] = ud;
    if (!collects(t, p)) return;
    const real wr = p == 1 ? rr1 : -rr2;
    if (!kDet && wr == real(0)) return;
    c = c0; tt = t0;
    for (int a = 0; a < na; ++a) {
        const real v = is_terminal(m, t.wbits, na, a) ? t.util[tt++] : ldm<C>(t.u + c++);
        if (kDet) out[a] = wr * (v - ud);
        else atomicAdd(&t.inst[qb + a], wr * (v - ud));
    }
}

// Top-down step of a node with more than 32 actions, shared by the threads of a block.
template <typename real, bool C>
__device__ __forceinline__ void td_wide(const DevTree<real> &t, int32_t j) {
    const uint32_t w = t.qp[j];
    const int32_t qb = qp_base(w);
    const int p = qp_player(w);
    const uint32_t *wb = t.wbits + t.kmask[j];
    const int32_t d0 = t.dfirst[j];
    const int na = (t.dfirst[j + 1] - d0) + (t.tfirst[j + 1] - t.tfirst[j]);
    const real r1 = ldm<C>(t.reach1 + j), r2 = ldm<C>(t.reach2 + j);
    for (int a = threadIdx.x; a < na; a += blockDim.x) {
        if ((wb[a >> 5] >> (a & 31)) & 1u) continue;
        const int32_t c = d0 + (a - terminals_before(wb, a));
        const real s = ldm<C>(t.sigma + qb + a);
        t.reach1[c] = p == 1 ? r1 : r1 * s;
        t.reach2[c] = p == 2 ? r2 : r2 * s;
    }
}

template <typename real, bool C>
__device__ __forceinline__ real wide_child_value(const DevTree<real> &t, const uint32_t *wb, int32_t d0, int32_t t0,
                                                 int a) {
    const int tb = terminals_before(wb, a);
    return ((wb[a >> 5] >> (a & 31)) & 1u) ? t.util[t0 + tb] : ldm<C>(t.u + d0 + (a - tb));
}

// Bottom-up step of a node with more than 32 actions, shared by the threads of a block (all of which
// must call it).
template <typename real, bool C>
__device__ __forceinline__ void bu_wide(const DevTree<real> &t, int32_t j, real *scratch32) {
    const uint32_t w = t.qp[j];
    const int32_t qb = qp_base(w);
    const int p = qp_player(w);
    const uint32_t *wb = t.wbits + t.kmask[j];
    const int32_t d0 = t.dfirst[j], t0 = t.tfirst[j];
    const int na = (t.dfirst[j + 1] - d0) + (t.tfirst[j + 1] - t0);
    real part = 0;
    for (int a = threadIdx.x; a < na; a += blockDim.x)
        part = madd(part, ldm<C>(t.sigma + qb + a), wide_child_value<real, C>(t, wb, d0, t0, a));
    const real ud = block_sum(part, scratch32);
    if (threadIdx.x == 0) t.u[j] = ud;
    if (!collects(t, p)) return;
    const real wr = p == 1 ? ldm<C>(t.reach1 + j) : -ldm<C>(t.reach2 + j);
    if (wr == real(0)) return;
    for (int a = threadIdx.x; a < na; a += blockDim.x)
        atomicAdd(&t.inst[qb + a], wr * (wide_child_value<real, C>(t, wb, d0, t0, a) - ud));
}

// ---- per-infoset update, FP32 mode: one thread per infoset ---------------------------------------
// The arithmetic of update_wide, per infoset, with no block-wide barriers: a thread loads all of its
// infoset's R, r~ and sigma entries at once, then S where something accrues.  Infosets with more than
// 32 actions are skipped (k_update_list takes them, one block each).

// Iteration weights of the FP32 update: T, the average weight w, and the discounted-CFR regret factors.
struct UpdWeights {
    double T, fpos, fneg;
    float w;
};

template <typename real>
__device__ __forceinline__ UpdWeights update_weights(const DevTree<real> &t, int variant, bool linear) {
    UpdWeights u;
    u.T = (double)*t.iter;
    u.fpos = u.fneg = 1.0;
    u.w = linear ? (float)u.T : 1.f;
    if (variant == CFRV_LINEAR) u.w = (float)u.T;
    if (variant == CFRV_DISCOUNTED) {
        u.w = (float)t.wts[0];
        u.fpos = t.wts[1];
        u.fneg = t.wts[2];
    }
    return u;
}

// R += r~ (CFR+: clipped at 0; linear CFR: R += T r~; discounted CFR: R = (R + r~) times the factor
// for its sign) for one slot; returns the slot's positive regret as a float.  V is the variant: a
// compile-time choice, so that vanilla and CFR+ spend no FP64 operation beyond the one addition.
template <int V>
__device__ __forceinline__ float update_regret(double *R, double rr, float in, const UpdWeights &u) {
    double r0;
    if constexpr (V == CFRV_LINEAR) r0 = rr + u.T * widen(in);
    else r0 = rr + widen(in);
    const bool positive = __double_as_longlong(r0) > 0;      // r0 > 0 without an FP64 compare
    if constexpr (V == CFRV_DISCOUNTED) r0 *= positive ? u.fpos : u.fneg;
    const double r = V == CFRV_PLUS && !positive ? 0.0 : r0;
    *R = r;
    return positive ? narrow(r) : 0.f;
}

// sigma' of an infoset whose positive regrets sum to `sum` below FP32's normal range: FP64 division.
__device__ __forceinline__ void regret_match_tiny(const DevTree<float> &t, int32_t qs, int na) {
    double p = 0.0;
    for (int a = 0; a < na; ++a) p += fmax(t.R[qs + a], 0.0);
    for (int a = 0; a < na; ++a) t.sigma[qs + a] = (float)(fmax(t.R[qs + a], 0.0) / p);
}

// ---- per-infoset update of a wide infoset (more than 32 actions), FP32 mode ----------------------
// The block shares the infoset's actions; the two FP64 accumulations stay FP64 (R += r~,
// S += w pi_i sigma) and regret matching runs in FP32, the strategy's precision, with the positive
// regrets summed over the block.  All threads of the block must call it.
template <int V>
__device__ __forceinline__ void update_wide(const DevTree<float> &t, int32_t h, const UpdWeights &u, float *s_red) {
    const int32_t qs = t.qbase[h];
    const int32_t nq = t.qbase[h + 1] - qs;
    const float wo = u.w * t.own[h];
    float part = 0.f;
    for (int32_t i = threadIdx.x; i < nq; i += blockDim.x) {
        const int32_t q = qs + i;
        part += update_regret<V>(t.R + q, t.R[q], t.inst[q], u);
        t.S[q] = t.S[q] + widen(wo * t.sigma[q]);
    }
    const float sum = block_sum(part, s_red);   // (its barriers also order the R writes above)
    if (sum >= 1e-30f || sum == 0.f) {
        for (int32_t i = threadIdx.x; i < nq; i += blockDim.x) {
            const double r = t.R[qs + i];
            t.sigma[qs + i] = sum > 0.f ? (r > 0.0 ? (float)r : 0.f) * (1.f / sum) : 1.f / (float)nq;
        }
    } else {                          // sums below FP32 range: normalise in FP64
        double pos = 0.0;
        for (int32_t i = 0; i < nq; ++i) pos += fmax(t.R[qs + i], 0.0);
        for (int32_t i = threadIdx.x; i < nq; i += blockDim.x) t.sigma[qs + i] = (float)(fmax(t.R[qs + i], 0.0) / pos);
    }
}

// The update of player infoset h (at most 32 actions) with the iteration's weights u.  C: loads
// through L2 (the caller wrote R, S, sigma or r~ earlier in the same launch).
template <int NA, int V, bool C>
__device__ __forceinline__ void update_row(const DevTree<float> &t, int32_t h, const UpdWeights &u) {
    const int32_t qs = t.qbase[h];
    const int na = t.qbase[h + 1] - qs;
    const float wo = u.w * ldm<C>(t.own + h);
    if (na <= NA) {
        double rr[NA];
        float in[NA], sg[NA], pos[NA];
#pragma unroll
        for (int a = 0; a < NA; ++a)
            if (a < na) { rr[a] = ldm<C>(t.R + qs + a); in[a] = ldm<C>(t.inst + qs + a); sg[a] = ldm<C>(t.sigma + qs + a); }
        float sum = 0.f;
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            if (a < na) {
                pos[a] = update_regret<V>(t.R + qs + a, rr[a], in[a], u);
                sg[a] = wo * sg[a];                            // the strategy-sum increment
            }
        }
#pragma unroll
        for (int a = 0; a < NA; ++a)                            // nothing accrues where own reach or sigma is 0
            if (a < na && sg[a] != 0.f) rr[a] = ldm<C>(t.S + qs + a);
#pragma unroll
        for (int a = 0; a < NA; ++a)
            if (a < na && sg[a] != 0.f) t.S[qs + a] = add_nonneg(rr[a], widen(sg[a]));
#pragma unroll
        for (int a = 0; a < NA; ++a)
            if (a < na) sum += pos[a];
        if (sum >= 1e-30f) {
            const float f = 1.f / sum;
#pragma unroll
            for (int a = 0; a < NA; ++a)
                if (a < na) t.sigma[qs + a] = pos[a] * f;
        } else if (sum > 0.f) {
            regret_match_tiny(t, qs, na);
        } else {
            const float un = 1.f / (float)na;                  // no positive regret: uniform (Eq. 9)
#pragma unroll
            for (int a = 0; a < NA; ++a)
                if (a < na) t.sigma[qs + a] = un;
        }
        return;
    }
    float pos[32];
    float sum = 0.f;
    for (int a = 0; a < na; ++a) {
        pos[a] = update_regret<V>(t.R + qs + a, ldm<C>(t.R + qs + a), ldm<C>(t.inst + qs + a), u);
        const float inc = wo * ldm<C>(t.sigma + qs + a);
        if (inc != 0.f) t.S[qs + a] = add_nonneg(ldm<C>(t.S + qs + a), widen(inc));
    }
    for (int a = 0; a < na; ++a) sum += pos[a];
    if (sum >= 1e-30f) {
        const float f = 1.f / sum;
        for (int a = 0; a < na; ++a) t.sigma[qs + a] = pos[a] * f;
    } else if (sum > 0.f) {
        regret_match_tiny(t, qs, na);
    } else {
        for (int a = 0; a < na; ++a) t.sigma[qs + a] = 1.f / (float)na;
    }
}

template <int NA, int V>
__global__ void __launch_bounds__(256) k_update_rows(DevTree<float> t, int32_t h0, int32_t h1, int32_t linear) {
    grid_dependency_wait();
    const int32_t h = h0 + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (h >= h1) return;
    if (t.pmask != 6 && !collects(t, t.iplayer[h])) return;      // alternating: the other player's pass
    if (t.qbase[h + 1] - t.qbase[h] > 32) return;
    update_row<NA, V, false>(t, h, update_weights(t, V, linear != 0));
}

// The infosets hs[0 .. gridDim.x) (more than 32 actions), one block each (up to 1024 threads).
template <int V>
__global__ void __launch_bounds__(1024) k_update_list(DevTree<float> t, const int32_t *hs, int32_t linear) {
    grid_dependency_wait();
    __shared__ float s_red[32];
    const int32_t h = hs[blockIdx.x];
    if (!collects(t, t.iplayer[h])) return;                      // alternating: the other player's pass
    update_wide<V>(t, h, update_weights(t, V, linear != 0), s_red);
}

// ---- one kernel per depth and step ----------------------------------------------------------------

// Own reaches of the player infosets [h0, h1) (those whose shallowest depth is one given depth).
template <typename real>
__global__ void __launch_bounds__(256) k_own(DevTree<real> t, int32_t h0, int32_t h1) {
    grid_dependency_wait();
    const int32_t h = h0 + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (h < h1) own_infoset<real, false>(t, h);
}

// Top-down from depth l: one thread per decision node of depth l.  bump: count the iteration.
template <typename real, bool kSkipWide>
__global__ void __launch_bounds__(256) k_topdown(DevTree<real> t, int32_t j0, int32_t j1, int32_t bump) {
    grid_dependency_wait();
    if (bump && blockIdx.x == 0 && threadIdx.x == 0) *t.iter += 1;
    const int32_t j = j0 + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (j < j1) td_node<real, kSkipWide, false>(t, j);
}

template <typename real, bool kDet>
__global__ void __launch_bounds__(256) k_bottomup(DevTree<real> t, int32_t j0, int32_t j1) {
    grid_dependency_wait();
    const int32_t j = j0 + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (j < j1) bu_node<real, kDet, false>(t, j);
}

template <typename real>
__global__ void __launch_bounds__(1024) k_topdown_wide(DevTree<real> t, const int32_t *wide, int32_t w0) {
    grid_dependency_wait();
    td_wide<real, false>(t, wide[w0 + blockIdx.x]);
}

template <typename real>
__global__ void __launch_bounds__(1024) k_bottomup_wide(DevTree<real> t, const int32_t *wide, int32_t w0) {
    grid_dependency_wait();
    __shared__ real s_red[32];
    bu_wide<real, false>(t, wide[w0 + blockIdx.x], s_red);
}

// ---- the shallowest depths in one launch per direction, FP32 mode ---------------------------------------
// Depths 0 .. n of a large tree hold few nodes (the deal, its first actions): one launch per depth
// spends its time in launch and dependency latency, not in memory traffic.  Below the root, the
// subtrees of consecutive root children are consecutive at every depth (breadth-first ids), and no
// node's step needs another subtree's, so k_head_topdown gives each block a range of root children
// and walks their subtrees down depth by depth with block barriers only; k_head_bottomup walks them
// back up, and the block that finishes last (a global counter, with fences) takes the root.  A block
// first stages the node fields of all its depths in shared memory (one round of independent loads)
// and keeps the reaches and values of its nodes there, so a depth costs one round of strategy and
// utility loads.  The arithmetic per node and its order are td_node's and bu_node's.  The top-down
// launch also computes the own reaches (Eq. 4) of the infosets first seen at depths 0 .. n, each as
// the product of the strategy entries of its player's own sequence, multiplied from the first action
// on - the same products in the same order as k_own's depth-by-depth recursion.  The host uses these
// kernels for a single root whose children are all decision nodes, with no node of more than 32
// actions in depths 1 .. n, or for a forest of independent games (blocks then take ranges of roots,
// and no node of depths 0 .. n may have more than 32 actions), and sizes the shared memory for the
// largest block (HeadArgs::cap nodes).
// NA: the unrolled action count (at least the largest of depths 1 .. n for full unrolling; nodes with more
// actions take the general loop).
constexpr int kHeadMaxDepths = 16;
constexpr int kHeadThreads = 512;
constexpr int kHeadBlocksPerSM = 3;

struct HeadArgs {
    int32_t n;                 // the top-down steps of depths 0 .. n (reaches of depths 1 .. n + 1) and the
                               // bottom-up steps of depths n .. 0
    int32_t bump;              // count the iteration (first pass of an iteration)
    int32_t forest;            // several roots (independent games): blocks take ranges of roots, and depth 0
                               // is a level like the others; else blocks take ranges of the root's children
    int32_t d1, nroot;         // the nodes blocks take ranges of: d1 .. d1 + nroot - 1 (the root's children at
                               // depth 1, or the roots at depth 0)
    int32_t per_block, nblk;   // root children per block; blocks walking subtrees
    int32_t cap;               // nodes of depths 1 .. n in a block, at most (shared-memory arrays)
    int32_t nown;              // infosets 0 .. nown - 1 are first seen at depths 0 .. n (own reaches)
    int32_t *done;             // k_head_bottomup: blocks that have finished (reset by the last)
    const int32_t *rng;        // per block kHeadRangeWords words: lo, hi, off of head_ranges (set at load)
    float *zero;               // k_head_topdown: r~ to clear (nzero floats; nullptr: cleared elsewhere),
    int64_t nzero;             // in slices by the subtree blocks - no kernel before the bottom-up reads it
};

// This block's slice of r~ (zero[0 .. nzero)) cleared with 16-byte stores where the slice allows.
__device__ __forceinline__ void head_clear(const HeadArgs &a) {
    if (!a.zero) return;
    const int64_t per = ((a.nzero + a.nblk - 1) / a.nblk + 3) & ~(int64_t)3;   // a multiple of 4 floats
    const int64_t b0 = per * blockIdx.x, b1 = min(b0 + per, a.nzero);
    if (b0 >= b1) return;
    const bool aligned = (reinterpret_cast<uintptr_t>(a.zero) & 15u) == 0;
    const int64_t v1 = aligned ? b0 + ((b1 - b0) & ~(int64_t)3) : b0;   // b0 is a multiple of 4
    float4 *z4 = reinterpret_cast<float4 *>(a.zero + b0);
    for (int64_t i = threadIdx.x; i < (v1 - b0) / 4; i += blockDim.x) z4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t i = v1 + threadIdx.x; i < b1; i += blockDim.x) a.zero[i] = 0.f;
}

// Own reach of infoset h from the strategy entries along its player's own sequence.
__device__ __forceinline__ void own_path(const DevTree<float> &t, int32_t h) {
    const int p = t.iplayer[h];
    if (p == 0 || !collects(t, p)) return;
    int32_t q[kHeadMaxDepths + 1];
    int k = 0;
    for (int32_t x = h; x >= 0 && t.pseq[x] >= 0 && k <= kHeadMaxDepths; x = t.pseq_h[x]) q[k++] = t.pseq[x];
    float own = 1.f;
    for (int i = k - 1; i >= 0; --i) own = own * t.sigma[q[i]];
    t.own[h] = own;
}

// The block's node ranges per depth: nodes lo[l] .. hi[l] - 1 of depth l (l = f .. n + 1, f the first
// depth the blocks split: 0 for a forest, else 1), at offset off[l] of the shared-memory arrays (l <= n).
// The host computes them once at load (head_block_ranges: lo[f] = d1 + block * per_block, hi[f] = lo[f] +
// per_block capped at d1 + nroot, lo[l + 1] = dfirst[lo[l]], hi[l + 1] = dfirst[hi[l]], off[f] = 0,
// off[l + 1] = off[l] + hi[l] - lo[l]), so a block reads them in one round instead of a chain of dependent
// loads per depth.  rng: the three arrays, kHeadMaxDepths + 2 words each; its threads load them.
constexpr int kHeadRangeWords = 3 * (kHeadMaxDepths + 2);
__device__ __forceinline__ void head_ranges(const HeadArgs &a, int32_t (*rng)[kHeadMaxDepths + 2]) {
    const int32_t *src = a.rng + (size_t)blockIdx.x * kHeadRangeWords;
    for (int i = (int)threadIdx.x; i < kHeadRangeWords; i += (int)blockDim.x)
        rng[i / (kHeadMaxDepths + 2)][i % (kHeadMaxDepths + 2)] = src[i];
}

// Stages the fields of the block's nodes of depths 1 .. n: local index off[l] + (j - lo[l]).
__device__ __forceinline__ void head_stage(const DevTree<float> &t, const HeadArgs &a, const int32_t *lo,
                                           const int32_t *off, uint32_t *qp_s, uint32_t *km_s, int32_t *df_s,
                                           int32_t *tf_s) {
    const int32_t total = off[a.n + 1];
    for (int32_t i = (int32_t)threadIdx.x; i < total; i += (int32_t)blockDim.x) {
        int l = a.forest ? 0 : 1;
        while (l < a.n && i >= off[l + 1]) ++l;
        const int32_t j = lo[l] + (i - off[l]);
        qp_s[i] = t.qp[j];
        km_s[i] = t.kmask[j];
        df_s[i] = t.dfirst[j];
        if (tf_s) tf_s[i] = t.tfirst[j];
    }
}

template <int NA>
__global__ void __launch_bounds__(kHeadThreads, kHeadBlocksPerSM) k_head_topdown(DevTree<float> t, HeadArgs a) {
    grid_dependency_wait();
    if (a.bump && blockIdx.x == 0 && threadIdx.x == 0) *t.iter += 1;
    const int32_t tid = (int32_t)threadIdx.x, bs = (int32_t)blockDim.x;
    if ((int32_t)blockIdx.x >= a.nblk) {                       // own reaches of the shallow infosets
        const int32_t h = ((int32_t)blockIdx.x - a.nblk) * bs + tid;
        if (h < a.nown) own_path(t, h);
        return;
    }
    extern __shared__ __align__(16) unsigned char head_smem[];
    uint32_t *qp_s = reinterpret_cast<uint32_t *>(head_smem);
    uint32_t *km_s = qp_s + a.cap;
    int32_t *df_s = reinterpret_cast<int32_t *>(km_s + a.cap);
    float *r1_s = reinterpret_cast<float *>(df_s + a.cap);
    float *r2_s = r1_s + a.cap;
    __shared__ int32_t rng[3][kHeadMaxDepths + 2];
    const int32_t *lo = rng[0], *hi = rng[1], *off = rng[2];
    head_ranges(a, rng);
    __syncthreads();
    head_stage(t, a, lo, off, qp_s, km_s, df_s, nullptr);
    head_clear(a);
    const int f = a.forest ? 0 : 1;
    if (a.forest) {   // depth 0: the roots' reaches (1, set at load)
        for (int32_t j = lo[0] + tid; j < hi[0]; j += bs) {
            r1_s[j - lo[0]] = t.reach1[j];
            r2_s[j - lo[0]] = t.reach2[j];
        }
    } else {          // depth 0: the root's step for this block's children (all decision nodes: child d1 + a is action a)
        const uint32_t w = t.qp[0];
        const int32_t qb = qp_base(w);
        const int p = qp_player(w);
        const float r1 = t.reach1[0], r2 = t.reach2[0];
        for (int32_t c = lo[1] + tid; c < hi[1]; c += bs) {
            const float sv = t.sigma[qb + (c - a.d1)];
            r1_s[c - lo[1]] = p == 1 ? r1 : r1 * sv;
            r2_s[c - lo[1]] = p == 2 ? r2 : r2 * sv;
        }
    }
    __syncthreads();
    for (int l = f; l <= a.n; ++l) {
        const int32_t cnt = hi[l] - lo[l];
        const bool deep = l == a.n;                             // children outside the block's arrays
        for (int32_t i = tid; i < cnt; i += bs) {
            const int32_t k = off[l] + i, j = lo[l] + i;
            const float r1 = r1_s[k], r2 = r2_s[k];
            t.reach1[j] = r1;
            t.reach2[j] = r2;
            const uint32_t w = qp_s[k], m = km_s[k];
            const int32_t c0 = df_s[k], c1 = i + 1 < cnt ? df_s[k + 1] : hi[l + 1];
            const int32_t nd = c1 - c0;
            if (nd == 0) continue;
            const int32_t qb = qp_base(w);
            const int p = qp_player(w);
            const int na = nd + __popc(m);
            float *w1 = deep ? t.reach1 + c0 : r1_s + off[l + 1] + (c0 - lo[l + 1]);
            float *w2 = deep ? t.reach2 + c0 : r2_s + off[l + 1] + (c0 - lo[l + 1]);
            if (na <= NA) {
                float s[NA];
#pragma unroll
                for (int b = 0; b < NA; ++b) s[b] = b < na ? t.sigma[qb + b] : 0.f;
                int y = 0;
#pragma unroll
                for (int b = 0; b < NA; ++b) {
                    if (b < na && !((m >> b) & 1u)) {
                        w1[y] = p == 1 ? r1 : r1 * s[b];
                        w2[y] = p == 2 ? r2 : r2 * s[b];
                        ++y;
                    }
                }
            } else {
                int y = 0;
                for (int b = 0; b < na; ++b) {
                    if ((m >> b) & 1u) continue;
                    const float sv = t.sigma[qb + b];
                    w1[y] = p == 1 ? r1 : r1 * sv;
                    w2[y] = p == 2 ? r2 : r2 * sv;
                    ++y;
                }
            }
        }
        __syncthreads();
    }
}

template <int NA>
__global__ void __launch_bounds__(kHeadThreads, kHeadBlocksPerSM) k_head_bottomup(DevTree<float> t, HeadArgs a) {
    grid_dependency_wait();
    extern __shared__ __align__(16) unsigned char head_smem[];
    uint32_t *qp_s = reinterpret_cast<uint32_t *>(head_smem);
    uint32_t *km_s = qp_s + a.cap;
    int32_t *df_s = reinterpret_cast<int32_t *>(km_s + a.cap);
    int32_t *tf_s = df_s + a.cap;
    float *u_s = reinterpret_cast<float *>(tf_s + a.cap);
    __shared__ int32_t rng[3][kHeadMaxDepths + 2];
    const int32_t *lo = rng[0], *hi = rng[1], *off = rng[2];
    __shared__ int32_t last;
    __shared__ float red[kHeadThreads / 32];
    const int32_t tid = (int32_t)threadIdx.x, bs = (int32_t)blockDim.x;
    head_ranges(a, rng);
    __syncthreads();
    head_stage(t, a, lo, off, qp_s, km_s, df_s, tf_s);
    __syncthreads();
    for (int l = a.n; l >= (a.forest ? 0 : 1); --l) {
        const int32_t cnt = hi[l] - lo[l];
        const bool deep = l == a.n;                             // children's values in global memory
        for (int32_t i = tid; i < cnt; i += bs) {
            const int32_t k = off[l] + i, j = lo[l] + i;
            const uint32_t w = qp_s[k], m = km_s[k];
            const int32_t c0 = df_s[k], c1 = i + 1 < cnt ? df_s[k + 1] : hi[l + 1], t0 = tf_s[k];
            const float rr1 = t.reach1[j], rr2 = t.reach2[j];
            const int32_t qb = qp_base(w);
            const int p = qp_player(w);
            const int na = (c1 - c0) + __popc(m);
            const float *dv = deep ? t.u + c0 : u_s + off[l + 1] + (c0 - lo[l + 1]);
            float ud = 0.f;
            const float wr = !collects(t, p) ? 0.f : p == 1 ? rr1 : -rr2;   // u_2 = -u_1
            if (na <= NA) {
                float v[NA], s[NA];
                int kt = 0, kd = 0;
#pragma unroll
                for (int b = 0; b < NA; ++b) {
                    if (b < na) {
                        const bool term = (m >> b) & 1u;
                        v[b] = term ? t.util[t0 + kt] : dv[kd];
                        kt += term;
                        kd += !term;
                        s[b] = t.sigma[qb + b];
                    }
                }
#pragma unroll
                for (int b = 0; b < NA; ++b)
                    if (b < na) ud = madd(ud, s[b], v[b]);
                u_s[k] = ud;
                t.u[j] = ud;
                if (wr != 0.f) {
#pragma unroll
                    for (int b = 0; b < NA; ++b)
                        if (b < na) atomicAdd(&t.inst[qb + b], wr * (v[b] - ud));
                }
            } else {
                int kt = 0, kd = 0;
                for (int b = 0; b < na; ++b) {
                    const float v = ((m >> b) & 1u) ? t.util[t0 + kt++] : dv[kd++];
                    ud = madd(ud, t.sigma[qb + b], v);
                }
                u_s[k] = ud;
                t.u[j] = ud;
                if (wr != 0.f) {
                    kt = kd = 0;
                    for (int b = 0; b < na; ++b) {
                        const float v = ((m >> b) & 1u) ? t.util[t0 + kt++] : dv[kd++];
                        atomicAdd(&t.inst[qb + b], wr * (v - ud));
                    }
                }
            }
        }
        __syncthreads();
    }
    if (a.forest) return;                                       // every root is its own game's
    // this block's depth-1 values are written; the last block to finish takes the root
    if (tid == 0) {
        __threadfence();
        last = atomicAdd(a.done, 1) == a.nblk - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const uint32_t w = t.qp[0];
    const int32_t qb = qp_base(w);
    const int p = qp_player(w);
    float part = 0.f;
    for (int32_t c = tid; c < a.nroot; c += bs) part = madd(part, t.sigma[qb + c], __ldcg(t.u + a.d1 + c));
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((tid & 31) == 0) red[tid >> 5] = part;
    __syncthreads();
    float ud = 0.f;
    for (int i = 0; i < bs / 32; ++i) ud += red[i];
    if (tid == 0) {
        t.u[0] = ud;
        *a.done = 0;                                           // ready for the next launch
    }
    if (!collects(t, p)) return;
    const float wr = p == 1 ? t.reach1[0] : -t.reach2[0];
    if (wr == 0.f) return;
    for (int32_t c = tid; c < a.nroot; c += bs) atomicAdd(&t.inst[qb + c], wr * (__ldcg(t.u + a.d1 + c) - ud));
}

// Shared memory of the head kernels for blocks of at most cap nodes.
inline size_t head_smem_topdown(int32_t cap) { return (size_t)cap * 20; }
inline size_t head_smem_bottomup(int32_t cap) { return (size_t)cap * 20; }

// ---- fused deepest depths, FP32 mode ----------------------------------------------------------------
// The depths r .. L-1, which hold most of the nodes, in one launch.  Block b takes a tile of
// consecutive depth-r nodes with all their decision descendants - consecutive at every depth, since
// the children of consecutive nodes are consecutive - and stages the tile's node fields in shared
// memory.  It then runs the top-down step depth by depth with the reaches kept in shared memory, and
// the bottom-up step from the deepest depth up with the values kept in shared memory.  Global memory
// sees the node fields once, the tile roots' reaches (read) and values (written), the terminal
// utilities, the strategy gathers and the regret scatter; the reaches and values of the deeper
// nodes never leave the SM unless the solver records them for cfr_get_nodes.  The arithmetic per
// node, and its order, is that of td_node and bu_node.  Nodes with more than 32 actions are not
// fused (the host keeps such depths out of the fused range).
constexpr int kFuseCap = 1024;       // decision nodes of one tile, all fused depths together
constexpr int kFuseMaxLevels = 8;
constexpr int kFuseBatch = 4;        // staging loads in flight per thread

struct FuseArgs {
    const int32_t *bounds;   // [levels][ntiles + 1]: tile i holds nodes bounds[k][i] .. bounds[k][i+1] - 1
                             // at fused depth r + k
    int32_t ntiles, levels;
    int32_t record;          // also write the values and reaches of every fused node
    int32_t bump;            // the fused depths start at the root: count the iteration
};

struct FuseShared {
    uint32_t qp[kFuseCap], km[kFuseCap];
    int32_t df[kFuseCap + kFuseMaxLevels], tf[kFuseCap + kFuseMaxLevels];   // n_k + 1 entries per depth
    float r1[kFuseCap], r2[kFuseCap], u[kFuseCap];
    int32_t lo[kFuseMaxLevels + 1], off[kFuseMaxLevels + 1];
};

// Top-down step of node i of fused depth k (as td_node, reaches from and to shared memory).
__device__ __forceinline__ void fused_td(const DevTree<float> &t, FuseShared &sh, int k, int32_t i, bool record) {
    const int32_t x = sh.off[k] + i, e = x + k;
    int32_t c = sh.df[e];
    const int32_t nd = sh.df[e + 1] - c;
    if (nd == 0) return;
    const uint32_t w = sh.qp[x];
    const int32_t qb = qp_base(w);
    const int p = qp_player(w);
    const uint32_t m = sh.km[x];
    const float r1 = sh.r1[x], r2 = sh.r2[x];
    int32_t y = sh.off[k + 1] + (c - sh.lo[k + 1]);
    const int na = nd + __popc(m);
    if (na <= kUnroll) {
        float s[kUnroll];
#pragma unroll
        for (int a = 0; a < kUnroll; ++a) s[a] = a < na ? __ldg(t.sigma + qb + a) : 0.f;
#pragma unroll
        for (int a = 0; a < kUnroll; ++a) {
            if (a < na && !((m >> a) & 1u)) {
                const float c1 = p == 1 ? r1 : r1 * s[a], c2 = p == 2 ? r2 : r2 * s[a];
                sh.r1[y] = c1;
                sh.r2[y] = c2;
                if (record) { t.reach1[c] = c1; t.reach2[c] = c2; }
                ++y;
                ++c;
            }
        }
        return;
    }
    for (int a = 0; a < na; ++a) {
        if ((m >> a) & 1u) continue;
        const float s = __ldg(t.sigma + qb + a);
        const float c1 = p == 1 ? r1 : r1 * s, c2 = p == 2 ? r2 : r2 * s;
        sh.r1[y] = c1;
        sh.r2[y] = c2;
        if (record) { t.reach1[c] = c1; t.reach2[c] = c2; }
        ++y;
        ++c;
    }
}

// Bottom-up step of node i of fused depth k (as bu_node with atomics; child values of decision
// children from shared memory).
__device__ __forceinline__ void fused_bu(const DevTree<float> &t, FuseShared &sh, int k, int32_t i, bool record) {
    const int32_t x = sh.off[k] + i, e = x + k;
    const uint32_t w = sh.qp[x];
    const int32_t qb = qp_base(w);
    const int p = qp_player(w);
    const uint32_t m = sh.km[x];
    const int32_t c0 = sh.df[e], t0 = sh.tf[e];
    const int32_t nd = sh.df[e + 1] - c0;
    const int na = nd + __popc(m);
    const float *dv = sh.u + (sh.off[k + 1] + (c0 - sh.lo[k + 1]));   // read only when nd > 0 (k + 1 fused)
    const float *tv = t.util + t0;
    float ud = 0.f;
    if (na <= kUnroll) {
        float v[kUnroll], s[kUnroll];
        int kt = 0, kd = 0;
#pragma unroll
        for (int a = 0; a < kUnroll; ++a) {
            if (a < na) {
                const bool term = (m >> a) & 1u;
                v[a] = term ? __ldg(tv + kt) : dv[kd];
                kt += term;
                kd += !term;
                s[a] = __ldg(t.sigma + qb + a);
            }
        }
#pragma unroll
        for (int a = 0; a < kUnroll; ++a)
            if (a < na) ud = madd(ud, s[a], v[a]);
        sh.u[x] = ud;
        if (k == 0 || record) t.u[sh.lo[k] + i] = ud;
        if (!collects(t, p)) return;
        const float wr = p == 1 ? sh.r1[x] : -sh.r2[x];
        if (wr == 0.f) return;
#pragma unroll
        for (int a = 0; a < kUnroll; ++a)
            if (a < na) atomicAdd(&t.inst[qb + a], wr * (v[a] - ud));
        return;
    }
    int kt = 0, kd = 0;
    for (int a = 0; a < na; ++a) {
        const float v = ((m >> a) & 1u) ? __ldg(tv + kt++) : dv[kd++];
        ud = madd(ud, __ldg(t.sigma + qb + a), v);
    }
    sh.u[x] = ud;
    if (k == 0 || record) t.u[sh.lo[k] + i] = ud;
    if (!collects(t, p)) return;
    const float wr = p == 1 ? sh.r1[x] : -sh.r2[x];
    if (wr == 0.f) return;
    kt = kd = 0;
    for (int a = 0; a < na; ++a) {
        const float v = ((m >> a) & 1u) ? __ldg(tv + kt++) : dv[kd++];
        atomicAdd(&t.inst[qb + a], wr * (v - ud));
    }
}

__global__ void __launch_bounds__(256) k_fused(DevTree<float> t, FuseArgs a) {
    grid_dependency_wait();
    __shared__ FuseShared sh;
    if (a.bump && blockIdx.x == 0 && threadIdx.x == 0) *t.iter += 1;
    const int K = a.levels;
    if (threadIdx.x == 0) {
        int32_t off = 0;
        for (int k = 0; k < K; ++k) {
            const int32_t *b = a.bounds + (size_t)k * (a.ntiles + 1) + blockIdx.x;
            sh.lo[k] = b[0];
            sh.off[k] = off;
            off += b[1] - b[0];
        }
        sh.off[K] = off;
        sh.lo[K] = 0;
    }
    __syncthreads();
    // Stage the node fields: entry f of depth k's run [off_k + k, off_{k+1} + k + 1) is node lo_k + f - (off_k + k)
    // (dfirst and tfirst take one entry more per depth, for the last node's end).
    const int32_t nent = sh.off[K] + K;
    for (int32_t f0 = threadIdx.x; f0 < nent; f0 += kFuseBatch * blockDim.x) {
        int32_t vd[kFuseBatch], vt[kFuseBatch];
        uint32_t vq[kFuseBatch], vk[kFuseBatch];
        float v1[kFuseBatch], v2[kFuseBatch];
        int kk[kFuseBatch];
        int32_t ii[kFuseBatch];
#pragma unroll
        for (int b = 0; b < kFuseBatch; ++b) {
            const int32_t f = f0 + b * (int32_t)blockDim.x;
            kk[b] = -1;
            if (f < nent) {
                int k = 0;
                while (k + 1 < K && f >= sh.off[k + 1] + k + 1) ++k;
                const int32_t i = f - (sh.off[k] + k);
                const int32_t j = sh.lo[k] + i;
                kk[b] = k;
                ii[b] = i;
                vd[b] = __ldg(t.dfirst + j);
                vt[b] = __ldg(t.tfirst + j);
                if (i < sh.off[k + 1] - sh.off[k]) {
                    vq[b] = __ldg(t.qp + j);
                    vk[b] = __ldg(t.kmask + j);
                    if (k == 0) { v1[b] = __ldg(t.reach1 + j); v2[b] = __ldg(t.reach2 + j); }
                }
            }
        }
#pragma unroll
        for (int b = 0; b < kFuseBatch; ++b) {
            const int k = kk[b];
            if (k < 0) continue;
            const int32_t f = f0 + b * (int32_t)blockDim.x, i = ii[b];
            sh.df[f] = vd[b];
            sh.tf[f] = vt[b];
            if (i < sh.off[k + 1] - sh.off[k]) {
                sh.qp[sh.off[k] + i] = vq[b];
                sh.km[sh.off[k] + i] = vk[b];
                if (k == 0) { sh.r1[i] = v1[b]; sh.r2[i] = v2[b]; }
            }
        }
    }
    __syncthreads();
    const bool record = a.record != 0;
    for (int k = 0; k + 1 < K; ++k) {
        const int32_t n = sh.off[k + 1] - sh.off[k];
        for (int32_t i = threadIdx.x; i < n; i += blockDim.x) fused_td(t, sh, k, i, record);
        __syncthreads();
    }
    for (int k = K - 1; k >= 0; --k) {
        const int32_t n = sh.off[k + 1] - sh.off[k];
        for (int32_t i = threadIdx.x; i < n; i += blockDim.x) fused_bu(t, sh, k, i, record);
        __syncthreads();
    }
}

// ---- the last two depths in one pass, FP32 mode -----------------------------------------------------
// One thread per node j of depth L-2 runs the top-down step of j (its children's reaches stay in
// registers), the bottom-up step of each decision child c (depth L-1, terminal children only) and then
// the bottom-up step of j.  The reaches and values of depth L-1 never go through memory unless the
// solver records them.  Per node the arithmetic and its order are those of td_node and bu_node.
// Nodes with more than 32 actions are not handled here (the host keeps such trees on the per-depth
// kernels).

// Bottom-up step of a node of the last depth (terminal children only) with the given reaches; returns
// its value.
__device__ __forceinline__ float tail_leaf(const DevTree<float> &t, int32_t c, float q1, float q2, bool record) {
    const uint32_t w = __ldg(t.qp + c);
    const int32_t qb = qp_base(w);
    const int p = qp_player(w);
    const int na = __popc(__ldg(t.kmask + c));
    const float *tv = t.util + __ldg(t.tfirst + c);
    float ud = 0.f;
    float v[kUnroll], s[kUnroll];
    if (na <= kUnroll) {
#pragma unroll
        for (int b = 0; b < kUnroll; ++b) {
            if (b < na) {
                v[b] = __ldg(tv + b);
                s[b] = __ldg(t.sigma + qb + b);
            }
        }
#pragma unroll
        for (int b = 0; b < kUnroll; ++b)
            if (b < na) ud = madd(ud, s[b], v[b]);
    } else {
        for (int b = 0; b < na; ++b) ud = madd(ud, __ldg(t.sigma + qb + b), __ldg(tv + b));
    }
    if (record) {
        t.u[c] = ud;
        t.reach1[c] = q1;
        t.reach2[c] = q2;
    }
    if (!collects(t, p)) return ud;
    const float wr = p == 1 ? q1 : -q2;
    if (wr == 0.f) return ud;
    if (na <= kUnroll) {
#pragma unroll
        for (int b = 0; b < kUnroll; ++b)
            if (b < na) atomicAdd(&t.inst[qb + b], wr * (v[b] - ud));
    } else {
        for (int b = 0; b < na; ++b) atomicAdd(&t.inst[qb + b], wr * (__ldg(tv + b) - ud));
    }
    return ud;
}

// bump: depth L-2 is the root's, so no top-down launch precedes this one; count the iteration.
__global__ void __launch_bounds__(256) k_tail(DevTree<float> t, int32_t j0, int32_t j1, int32_t record,
                                              int32_t bump) {
    grid_dependency_wait();
    if (bump && blockIdx.x == 0 && threadIdx.x == 0) *t.iter += 1;
    const int32_t j = j0 + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (j >= j1) return;
    const bool rec = record != 0;
    const uint32_t w = __ldg(t.qp + j);
    const int32_t qb = qp_base(w);
    const int p = qp_player(w);
    const uint32_t m = __ldg(t.kmask + j);
    const int32_t c0 = __ldg(t.dfirst + j);
    const int32_t nd = __ldg(t.dfirst + j + 1) - c0;
    const int32_t t0 = __ldg(t.tfirst + j);
    const float r1 = __ldg(t.reach1 + j), r2 = __ldg(t.reach2 + j);
    const int na = nd + __popc(m);
    float ud = 0.f;
    if (na <= kUnroll) {
        float s[kUnroll], v[kUnroll];
        int kt = 0;
#pragma unroll
        for (int a = 0; a < kUnroll; ++a) {
            if (a < na) {
                s[a] = __ldg(t.sigma + qb + a);
                if ((m >> a) & 1u) v[a] = __ldg(t.util + t0 + kt++);
            }
        }
        int kd = 0;
#pragma unroll
        for (int a = 0; a < kUnroll; ++a) {
            if (a < na && !((m >> a) & 1u)) {
                const float q1 = p == 1 ? r1 : r1 * s[a], q2 = p == 2 ? r2 : r2 * s[a];
                v[a] = tail_leaf(t, c0 + kd++, q1, q2, rec);
            }
        }
#pragma unroll
        for (int a = 0; a < kUnroll; ++a)
            if (a < na) ud = madd(ud, s[a], v[a]);
        t.u[j] = ud;
        if (!collects(t, p)) return;
        const float wr = p == 1 ? r1 : -r2;
        if (wr == 0.f) return;
#pragma unroll
        for (int a = 0; a < kUnroll; ++a)
            if (a < na) atomicAdd(&t.inst[qb + a], wr * (v[a] - ud));
        return;
    }
    // more than kUnroll actions (at most 32): child values are recomputed from memory in the second
    // loop only for terminals; decision children's values are kept in a per-thread array
    float vd[32];
    int kt = 0, kd = 0;
    for (int a = 0; a < na; ++a) {
        const float s = __ldg(t.sigma + qb + a);
        float v;
        if ((m >> a) & 1u) {
            v = __ldg(t.util + t0 + kt++);
        } else {
            const float q1 = p == 1 ? r1 : r1 * s, q2 = p == 2 ? r2 : r2 * s;
            v = tail_leaf(t, c0 + kd++, q1, q2, rec);
        }
        vd[a] = v;
        ud = madd(ud, s, v);
    }
    t.u[j] = ud;
    if (!collects(t, p)) return;
    const float wr = p == 1 ? r1 : -r2;
    if (wr == 0.f) return;
    for (int a = 0; a < na; ++a) atomicAdd(&t.inst[qb + a], wr * (vd[a] - ud));
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

// Per-infoset update, one thread per infoset, FP64 operations in the oracle's order (FP64 mode).
template <typename real, bool kDet>
__global__ void __launch_bounds__(256) k_update(DevTree<real> t, int32_t H, int32_t variant, int32_t linear) {
    grid_dependency_wait();
    const int32_t h = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (h >= H || t.iplayer[h] == 0 || !collects(t, t.iplayer[h])) return;
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
    const double T = (double)*t.iter;
    double w = linear ? T : 1.0;
    if (variant == CFRV_LINEAR) w = T;
    if (variant == CFRV_DISCOUNTED) w = t.wts[0];
    const double wo = __dmul_rn(w, (double)t.own[h]);
    for (int a = 0; a < na; ++a) {
        const double in = (double)t.inst[qb + a];
        double r;
        if (variant == CFRV_LINEAR) {
            r = __dadd_rn(t.R[qb + a], __dmul_rn(T, in));
        } else if (variant == CFRV_DISCOUNTED) {
            const double x = __dadd_rn(t.R[qb + a], in);
            r = __dmul_rn(x, x > 0.0 ? t.wts[1] : t.wts[2]);
        } else {
            r = t.R[qb + a] + in;
            if (variant == CFRV_PLUS) r = r > 0.0 ? r : 0.0;
        }
        t.R[qb + a] = r;
        t.S[qb + a] = madd(t.S[qb + a], wo, (double)t.sigma[qb + a]);
    }
    regret_match(t.sigma, t.R, qb, na);
}

// Linear / discounted CFR: iteration T's weights, once per iteration (T is the already counted
// iteration): wts[0] = T^gamma, wts[1] = T^alpha / (T^alpha + 1), wts[2] = T^beta / (T^beta + 1).
__global__ void k_weights(const int64_t *iter, double *wts, double alpha, double beta, double gamma) {
    grid_dependency_wait();
    const double T = (double)*iter;
    const double ta = pow(T, alpha), tb = pow(T, beta);
    wts[0] = pow(T, gamma);
    wts[1] = ta / (ta + 1.0);
    wts[2] = tb / (tb + 1.0);
}

// Alternating updates: zeroes the instantaneous regrets of the infosets [0, Hp) whose player takes
// this pass (the other player's keep their last pass's values).
template <typename real>
__global__ void __launch_bounds__(256) k_zero_inst(DevTree<real> t, int32_t Hp) {
    grid_dependency_wait();
    const int32_t h = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (h >= Hp || !collects(t, t.iplayer[h])) return;
    for (int32_t q = t.qbase[h]; q < t.qbase[h + 1]; ++q) t.inst[q] = real(0);
}

// ---- state access -----------------------------------------------------------------------------------

// sigma := regret matching of R for every player infoset (uniform when R = 0: sigma^(1)).
template <typename real>
__global__ void k_regret_match_all(real *sigma, const double *R, const int32_t *qbase, const int8_t *iplayer, int32_t H) {
    const int32_t h = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (h >= H || iplayer[h] == 0) return;
    regret_match(sigma, R, qbase[h], qbase[h + 1] - qbase[h]);
}

// ---- depth-limited solving: leaf refresh ----------------------------------------------------------
// Range program: segment s writes its entries e in [ent[s], ent[s + 1]) to out[dst[s] + e - ent[s]],
// each the product of sigma over the internal slots slots[prod[e] .. prod[e + 1]) (a player's own
// reach of one private state at one public node, Eq. 4), then divides the segment by its sum (uniform
// when the sum is 0).  One thread per segment.
template <typename real>
__global__ void k_ranges(const real *sigma, const int64_t *dst, const int64_t *ent, const int64_t *prod,
                         const int32_t *slots, int64_t nseg, float *out) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nseg; s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e0 = ent[s], e1 = ent[s + 1];
        double sum = 0.0;
        for (int64_t e = e0; e < e1; ++e) {
            double p = 1.0;
            for (int64_t i = prod[e]; i < prod[e + 1]; ++i) p *= (double)sigma[slots[i]];
            sum += p;
        }
        for (int64_t e = e0; e < e1; ++e) {
            double p = 1.0;
            for (int64_t i = prod[e]; i < prod[e + 1]; ++i) p *= (double)sigma[slots[i]];
            out[dst[s] + (e - e0)] = sum > 0.0 ? (float)(p / sum) : (float)(1.0 / (double)(e1 - e0));
        }
    }
}

// Leaf refresh: the utility of registered terminal t[i] becomes scale * src[src_index[i]] (both the
// working-precision copy and the FP64 one the best response reads).
template <typename real>
__global__ void k_set_leaves(real *util, double *util64, const int32_t *t, const int64_t *src_index, const float *src,
                             double scale, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = scale * (double)src[src_index[i]];
        util[t[i]] = (real)v;
        util64[t[i]] = v;
    }
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

// Best-response steps (one node or infoset each).  C: loads through L2 of the values this launch wrote.
// Top-down: the reach of node j's decision children that excludes the best responder's own actions.
template <bool C>
__device__ __forceinline__ void br_topdown_node(const DevBR &b, int32_t j, int32_t player) {
    int32_t c = b.dfirst[j];
    if (c == b.dfirst[j + 1]) return;
    const int32_t h = b.dinfo[j];
    const bool mine = b.iplayer[h] == player;
    const int32_t qb = b.qbase[h];
    const int na = b.qbase[h + 1] - qb;
    const uint32_t m = b.kmask[j];
    const double r = ldm<C>(b.preach + j);
    for (int a = 0; a < na; ++a) {
        if (is_terminal(m, b.wbits, na, a)) continue;
        b.preach[c++] = mine ? r : r * b.avg[qb + a];
    }
}

template <bool C>
__device__ __forceinline__ double br_child(const DevBR &b, uint32_t m, int na, int a, int32_t &c, int32_t &tt,
                                           double sign) {
    return is_terminal(m, b.wbits, na, a) ? sign * b.util[tt++] : ldm<C>(b.val + c++);
}

// Bottom-up: the value of an opponent (or chance) node under the average strategy; at the best
// responder's nodes, the reach-weighted action values summed per infoset (cfv).
template <bool C>
__device__ __forceinline__ void br_node(const DevBR &b, int32_t j, int32_t player) {
    const int32_t h = b.dinfo[j];
    const int32_t qb = b.qbase[h];
    const int na = b.qbase[h + 1] - qb;
    const uint32_t m = b.kmask[j];
    const double sign = player == 1 ? 1.0 : -1.0;
    int32_t c = b.dfirst[j], tt = b.tfirst[j];
    if (b.iplayer[h] != player) {
        double v = 0.0;
        for (int a = 0; a < na; ++a) v += b.avg[qb + a] * br_child<C>(b, m, na, a, c, tt, sign);
        b.val[j] = v;
    } else {
        const double r = ldm<C>(b.preach + j);
        if (r == 0.0) return;
        for (int a = 0; a < na; ++a) {
            const double v = br_child<C>(b, m, na, a, c, tt, sign);
            atomicAdd(&b.cfv[qb + a], r * v);
        }
    }
}

// The best action of the responder's infoset h (lowest index among ties).
template <bool C>
__device__ __forceinline__ void br_choose(const DevBR &b, int32_t h, int32_t player) {
    if (b.iplayer[h] != player) return;
    const int32_t qb = b.qbase[h];
    const int na = b.qbase[h + 1] - qb;
    int best = 0;
    double bv = ldm<C>(b.cfv + qb);
    for (int a = 1; a < na; ++a) {
        const double v = ldm<C>(b.cfv + qb + a);
        if (v > bv) { best = a; bv = v; }
    }
    b.astar[h] = best;
}

// The value of a responder's node: that of its infoset's best action.
template <bool C>
__device__ __forceinline__ void br_pick(const DevBR &b, int32_t j, int32_t player) {
    const int32_t h = b.dinfo[j];
    if (b.iplayer[h] != player) return;
    const uint32_t m = b.kmask[j];
    const int na = b.qbase[h + 1] - b.qbase[h];
    const int as = ldm<C>(b.astar + h);
    int32_t c = b.dfirst[j], tt = b.tfirst[j];
    double v = 0.0;
    for (int a = 0; a <= as; ++a) v = br_child<C>(b, m, na, a, c, tt, player == 1 ? 1.0 : -1.0);
    b.val[j] = v;
}

__global__ void __launch_bounds__(256) k_br_topdown(DevBR b, int32_t j0, int32_t j1, int32_t player) {
    const int32_t j = j0 + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (j < j1) br_topdown_node<false>(b, j, player);
}

__global__ void __launch_bounds__(256) k_br_nodes(DevBR b, int32_t j0, int32_t j1, int32_t player) {
    const int32_t j = j0 + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (j < j1) br_node<false>(b, j, player);
}

__global__ void k_br_choose(DevBR b, int32_t h0, int32_t h1, int32_t player) {
    const int32_t h = h0 + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (h < h1) br_choose<false>(b, h, player);
}

__global__ void __launch_bounds__(256) k_br_pick(DevBR b, int32_t j0, int32_t j1, int32_t player) {
    const int32_t j = j0 + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (j < j1) br_pick<false>(b, j, player);
}

// Both players' best responses in one pass: b1 and b2 hold each responder's reaches and values and
// share cfv and astar, which each responder writes at its own infosets only.
__global__ void __launch_bounds__(256) k_br2_topdown(DevBR b1, DevBR b2, int32_t j0, int32_t j1) {
    grid_dependency_wait();
    const int32_t j = j0 + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (j >= j1) return;
    br_topdown_node<false>(b1, j, 1);
    br_topdown_node<false>(b2, j, 2);
}

__global__ void __launch_bounds__(256) k_br2_nodes(DevBR b1, DevBR b2, int32_t j0, int32_t j1) {
    grid_dependency_wait();
    const int32_t j = j0 + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (j >= j1) return;
    br_node<false>(b1, j, 1);
    br_node<false>(b2, j, 2);
}

__global__ void __launch_bounds__(256) k_br2_choose(DevBR b1, DevBR b2, int32_t h0, int32_t h1) {
    grid_dependency_wait();
    const int32_t h = h0 + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (h >= h1) return;
    if (b1.iplayer[h] == 1) br_choose<false>(b1, h, 1);
    else br_choose<false>(b2, h, 2);
}

__global__ void __launch_bounds__(256) k_br2_pick(DevBR b1, DevBR b2, int32_t j0, int32_t j1) {
    grid_dependency_wait();
    const int32_t j = j0 + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (j >= j1) return;
    br_pick<false>(b1, j, 1);
    br_pick<false>(b2, j, 2);
}

// The root's value u(v_0) (or the terminal root's utility) as FP64 into page-locked host memory.
template <typename real>
__global__ void k_root_out(const real *u, double *out) { out[0] = (double)u[0]; }

__global__ void k_fill(double *p, int32_t n, double v) {
    const int32_t i = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (i < n) p[i] = v;
}

}  // namespace
}  // namespace cfrgb
