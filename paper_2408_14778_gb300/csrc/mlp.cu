// Learned leaf values: the BF16 multilayer perceptron of include/cfr_gb300.h (cfr_mlp_*), trained and
// evaluated with this file's kernels.
//
// Matrix products: C[M][N] = sum_k A(m, k) B(k, n), BF16 operands and FP32 accumulation, by three
// kernels (cfr_mlp_set_tensor_path chooses):
//   k_gemm_tma  the 5th-generation tensor cores (tcgen05.mma, accumulator in tensor memory) with
//               TMA-loaded, 128-byte-swizzled, K-major operands and warp-specialised copy / MMA issue;
//   k_gemm      the warp-level kernel (mma.sync m16n8k16, 128 x 128 x 32 block tiles staged through
//               shared memory by cp.async in a three-stage pipeline, eight warps of 64 x 32), any
//               operand orientation;
//   k_gemm_tc   tcgen05.mma with operands copied by every thread with cp.async into the canonical
//               no-swizzle layout, any orientation.
// The three products of a layer:
//   forward        Z[b][o]  = sum_i X[b][i] W[o][i]      A K-major, B K-major ([o][i])
//   weight grad    dW[o][i] = sum_b dZ[b][o] X[b][i]     A and B with the output index contiguous
//   data grad      dX[b][i] = sum_o dZ[b][o] W[o][i]     A K-major, B with the output index contiguous
// The default (path 2) runs all three on k_gemm_tma, whose TMA boxes need K-major operands: the data
// gradient reads a transposed BF16 copy of the weights (kept by cfr_mlp_set_params and Adam), and the
// weight gradient reads transposed copies of the layer input and of the output gradient [feature][batch],
// which a training pass writes beside the row-major ones (the input packing, the loss gradient and the
// products' epilogues); its reduction over the batch is split over blocks that add their partial tiles
// with FP32 vector atomics.  Paths 0 and 1 read every operand in its stored orientation (ldmatrix with
// .trans, or the tcgen05 descriptor's major bits) and need no transposed copies.
// Every dimension is padded to a multiple of 128 (the batch too): padded weights and inputs are zero and
// padded rows of the output gradient are zero, so padding never reaches a real result.
#include <cuda.h>   // CUtensorMap and its enums; the encoder is fetched through the runtime's entry point
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "cfr_gb300.h"

namespace {

constexpr int kBM = 128, kBN = 128, kBK = 32, kStages = 3, kThreads = 256;
constexpr int kTileBytes = kBM * kBK * 2;   // one operand tile of one stage (both orientations)
constexpr int kPad = 128;

__host__ __device__ inline int64_t pad_to(int64_t x, int64_t q) { return (x + q - 1) / q * q; }

// ---- shared-memory tile addressing (16-byte chunks XOR-swizzled so ldmatrix rows hit distinct banks)
// K-major tile: 128 rows x 32 bf16 (64 bytes, 4 chunks per row).
__device__ __forceinline__ uint32_t km_off(int row, int chunk) { return (uint32_t)(row * 64 + ((chunk ^ ((row >> 1) & 3)) << 4)); }
// Output-index-contiguous tile: 32 rows (reduction) x 128 bf16 (256 bytes, 16 chunks per row).
__device__ __forceinline__ uint32_t mm_off(int row, int chunk) { return (uint32_t)(row * 256 + ((chunk ^ (row & 7)) << 4)); }

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void *g) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}
__device__ __forceinline__ void mma_bf16(float *d, const uint32_t *a, uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                 "{%8, %9}, {%0, %1, %2, %3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One operand tile (rows r0.., reduction k0..) of stage buffer `s` from global memory.  K-major: tile
// rows are 128 output rows of 32 reduction values at &G[(r0 + r) ld + k0]; otherwise 32 reduction rows
// of 128 output values at &G[(k0 + r) ld + r0].
template <bool KM>
__device__ __forceinline__ void load_tile(uint32_t s, const __nv_bfloat16 *G, int64_t ld, int64_t r0, int64_t k0) {
#pragma unroll
    for (int it = 0; it < (kBM * kBK / 8) / kThreads; ++it) {
        const int i = (int)threadIdx.x + it * kThreads;
        if (KM) {
            const int r = i >> 2, c = i & 3;
            cp_async16(s + km_off(r, c), G + (r0 + r) * ld + k0 + c * 8);
        } else {
            const int r = i >> 4, c = i & 15;
            cp_async16(s + mm_off(r, c), G + (k0 + r) * ld + r0 + c * 8);
        }
    }
}

enum Epi { kEpiHidden = 0, kEpiOut = 1, kEpiStore = 2, kEpiMask = 3, kEpiAdd = 4 };

// C = A B over M x N (multiples of 128), reduction K (multiple of 32).  AKM / BKM: whether A / B is
// stored K-major.  Epilogues: kEpiHidden bf16(ReLU(acc + bias[n])); kEpiOut acc + bias[n] (FP32);
// kEpiStore acc (FP32); kEpiMask bf16(acc if mask[m][n] > 0 else 0); kEpiAdd C += acc (FP32 atomics).
// Split reduction: block z of gridDim.z takes the reduction steps [z ksteps, (z + 1) ksteps) of kBK
// (ksteps <= 0: all of them), its partial sum added with kEpiAdd.
template <bool AKM, bool BKM, int EPI>
__global__ void __launch_bounds__(kThreads) k_gemm(const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B,
                                                   int64_t ldb, void *C, int64_t ldc, int32_t K, const float *bias,
                                                   const __nv_bfloat16 *mask, int32_t ksteps) {
    __shared__ __align__(128) unsigned char smem[kStages * 2 * kTileBytes];
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
    const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
    const int wm = (warp >> 2) * 64, wn = (warp & 3) * 32;
    const int64_t m0 = (int64_t)blockIdx.y * kBM, n0 = (int64_t)blockIdx.x * kBN;
    const int kall = K / kBK;
    const int kz = ksteps > 0 ? (int)blockIdx.z * ksteps : 0;
    const int nk = ksteps > 0 ? min(ksteps, kall - kz) : kall;
    const int64_t koff = (int64_t)kz * kBK;
    float acc[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

    auto sa = [&](int st) { return sbase + (uint32_t)(st * 2 * kTileBytes); };
    auto sb = [&](int st) { return sbase + (uint32_t)(st * 2 * kTileBytes + kTileBytes); };
#pragma unroll
    for (int st = 0; st < kStages - 1; ++st) {
        if (st < nk) {
            load_tile<AKM>(sa(st), A, lda, m0, koff + (int64_t)st * kBK);
            load_tile<BKM>(sb(st), B, ldb, n0, koff + (int64_t)st * kBK);
        }
        cp_commit();
    }
    for (int kt = 0; kt < nk; ++kt) {
        cp_wait<kStages - 2>();
        __syncthreads();
        {   // prefetch kStages - 1 tiles ahead into the buffer computed on in the previous step
            const int kn = kt + kStages - 1;
            if (kn < nk) {
                load_tile<AKM>(sa(kn % kStages), A, lda, m0, koff + (int64_t)kn * kBK);
                load_tile<BKM>(sb(kn % kStages), B, ldb, n0, koff + (int64_t)kn * kBK);
            }
            cp_commit();
        }
        const uint32_t ta = sa(kt % kStages), tb = sb(kt % kStages);
#pragma unroll
        for (int kk = 0; kk < kBK; kk += 16) {
            uint32_t af[4][4], bf[4][2];
#pragma unroll
            for (int mi = 0; mi < 4; ++mi) {
                if (AKM) {
                    const int row = wm + mi * 16 + (lane & 15), chunk = (kk >> 3) + (lane >> 4);
                    ldsm_x4(ta + km_off(row, chunk), af[mi][0], af[mi][1], af[mi][2], af[mi][3]);
                } else {
                    const int i = lane >> 3;
                    const int row = kk + (i >> 1) * 8 + (lane & 7), chunk = (wm + mi * 16 + (i & 1) * 8) >> 3;
                    ldsm_x4_t(ta + mm_off(row, chunk), af[mi][0], af[mi][1], af[mi][2], af[mi][3]);
                }
            }
#pragma unroll
            for (int nj = 0; nj < 2; ++nj) {
                const int i = lane >> 3;
                if (BKM) {
                    const int row = wn + nj * 16 + (i >> 1) * 8 + (lane & 7), chunk = (kk >> 3) + (i & 1);
                    ldsm_x4(tb + km_off(row, chunk), bf[2 * nj][0], bf[2 * nj][1], bf[2 * nj + 1][0], bf[2 * nj + 1][1]);
                } else {
                    const int row = kk + (i & 1) * 8 + (lane & 7), chunk = (wn + nj * 16 + (i >> 1) * 8) >> 3;
                    ldsm_x4_t(tb + mm_off(row, chunk), bf[2 * nj][0], bf[2 * nj][1], bf[2 * nj + 1][0], bf[2 * nj + 1][1]);
                }
            }
#pragma unroll
            for (int mi = 0; mi < 4; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], af[mi], bf[ni][0], bf[ni][1]);
        }
    }
    cp_wait<0>();
    // epilogue: thread holds rows g, g + 8 and columns 2 t, 2 t + 1 of each 16 x 8 tile
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t m = m0 + wm + mi * 16 + g + h * 8, n = n0 + wn + ni * 8 + 2 * t;
                float v0 = acc[mi][ni][2 * h], v1 = acc[mi][ni][2 * h + 1];
                if (EPI == kEpiHidden || EPI == kEpiOut) { v0 += bias[n]; v1 += bias[n + 1]; }
                if (EPI == kEpiHidden) { v0 = fmaxf(v0, 0.f); v1 = fmaxf(v1, 0.f); }
                if (EPI == kEpiMask) {
                    const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162 *>(mask + m * ldc + n);
                    if (!(__bfloat162float(mk.x) > 0.f)) v0 = 0.f;
                    if (!(__bfloat162float(mk.y) > 0.f)) v1 = 0.f;
                }
                if (EPI == kEpiHidden || EPI == kEpiMask) {
                    *reinterpret_cast<__nv_bfloat162 *>(static_cast<__nv_bfloat16 *>(C) + m * ldc + n) =
                        __floats2bfloat162_rn(v0, v1);
                } else if (EPI == kEpiAdd) {
                    atomicAdd(static_cast<float *>(C) + m * ldc + n, v0);
                    atomicAdd(static_cast<float *>(C) + m * ldc + n + 1, v1);
                } else {
                    *reinterpret_cast<float2 *>(static_cast<float *>(C) + m * ldc + n) = make_float2(v0, v1);
                }
            }
}

// ---- the same products on the 5th-generation tensor cores (tcgen05, accumulator in tensor memory) ---
// One CTA of 128 threads computes a 128 x 128 tile of C.  Per 32-wide reduction step all threads copy the
// A and B tiles into shared memory with cp.async, four steps ahead of the one multiplied (six stages),
// in the tensor core's canonical no-swizzle layout: 8 x 16-byte core matrices, each an 8-row x 8-element
// block stored contiguously (128 bytes); core (r, k) of an operand tile sits at r * 512 + k * 128 bytes
// (4 cores along the reduction, 16 along the rows).  A
// K-major operand's core rows are its rows (8 reduction values each); an operand whose output index is
// contiguous in memory is stored the same way with the roles of the 8 x 8 block transposed (each core
// row holds 8 output-index values at one reduction index) and the instruction's major bit set.  In both
// cases the descriptor's leading offset (128 bytes) steps along the reduction and its stride offset
// (512 bytes) along the rows.  One elected thread issues two tcgen05.mma (M = 128, N = 128, K = 16) per
// step and commits them to the stage's mbarrier, which the refill of that stage waits for two steps
// later.  The FP32 accumulator lives in 128 columns of tensor memory; the epilogue reads it with
// tcgen05.ld (warp w owns lanes 32 w .. 32 w + 31, one output row per thread).  Every mbarrier wait is
// bounded; a wait that gives up sets *err and the CTA still releases its tensor memory.
constexpr int kTcK = 32, kTcStages = 6, kTcThreads = 128;
constexpr int kTcDist = kTcStages - 2;                        // tiles loaded ahead of the one multiplied
constexpr int kTcTileBytes = 128 * kTcK * 2;                  // 8 KB per operand per stage
constexpr int kTcRowCore = (kTcK / 8) * 128;                  // bytes between core matrices along the rows
constexpr int kTcSmem = kTcStages * 2 * kTcTileBytes + 64;     // + mbarriers and the TMEM address
constexpr uint32_t kTcCols = 128;
constexpr uint32_t kTcWaitPolls = 1u << 26;

__device__ __forceinline__ uint32_t tc_smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool tc_mbar_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t i = 0; i < kTcWaitPolls; ++i) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

// Shared-memory matrix descriptor: start address, leading (reduction) and stride (row) byte offsets, the
// descriptor version of this architecture (1), no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// Byte offset of element (row, k) of an operand tile in the layout above.  KM: the element's 16-byte
// core row runs along k; otherwise along the rows.
template <bool KM>
__device__ __forceinline__ uint32_t tc_off(int row, int k) {
    const uint32_t core = (uint32_t)((row >> 3) * kTcRowCore + (k >> 3) * 128);
    return KM ? core + (uint32_t)((row & 7) * 16 + (k & 7) * 2) : core + (uint32_t)((k & 7) * 16 + (row & 7) * 2);
}

// Copies one operand tile (rows r0 .. r0 + 127, reduction k0 .. k0 + kTcK - 1) into stage buffer s.
template <bool KM>
__device__ __forceinline__ void tc_load(uint32_t s, const __nv_bfloat16 *G, int64_t ld, int64_t r0, int64_t k0) {
#pragma unroll
    for (int it = 0; it < (128 * kTcK / 8) / kTcThreads; ++it) {
        const int i = (int)threadIdx.x + it * kTcThreads;
        if (KM) {                                  // row r, reduction chunk c (8 values)
            const int r = i / (kTcK / 8), c = i % (kTcK / 8);
            cp_async16(s + tc_off<true>(r, c * 8), G + (r0 + r) * ld + k0 + c * 8);
        } else {                                   // reduction index k, row chunk c (8 rows)
            const int k = i >> 4, c = i & 15;      // 16 chunks of 8 rows per reduction index
            cp_async16(s + tc_off<false>(c * 8, k), G + (k0 + k) * ld + r0 + c * 8);
        }
    }
}

template <bool AKM, bool BKM, int EPI>
__global__ void __launch_bounds__(kTcThreads) k_gemm_tc(const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B,
                                                        int64_t ldb, void *C, int64_t ldc, int32_t K, const float *bias,
                                                        const __nv_bfloat16 *mask, int *err) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    const uint32_t sbase = tc_smem_u32(tsm);
    uint64_t *bars = reinterpret_cast<uint64_t *>(tsm + kTcStages * 2 * kTcTileBytes);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + kTcStages);
    const int tid = (int)threadIdx.x, warp = tid >> 5;
    const int64_t m0 = (int64_t)blockIdx.y * 128, n0 = (int64_t)blockIdx.x * 128;
    const int nk = K / kTcK;
    auto sa = [&](int st) { return sbase + (uint32_t)(st * 2 * kTcTileBytes); };
    auto sb = [&](int st) { return sbase + (uint32_t)(st * 2 * kTcTileBytes + kTcTileBytes); };
    auto bar = [&](int st) { return tc_smem_u32(bars + st); };

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem_u32(tslot)),
                     "r"(kTcCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0)
        for (int st = 0; st < kTcStages; ++st)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar(st)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    // instruction descriptor: FP32 accumulator, BF16 A and B, their majors, N = 128, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((AKM ? 0u : 1u) << 15) | ((BKM ? 0u : 1u) << 16) |
                           ((128u >> 3) << 17) | ((128u >> 4) << 24);
    bool ok = true;
#pragma unroll
    for (int st = 0; st < kTcDist; ++st) {
        if (st < nk) {
            tc_load<AKM>(sa(st), A, lda, m0, (int64_t)st * kTcK);
            tc_load<BKM>(sb(st), B, ldb, n0, (int64_t)st * kTcK);
        }
        cp_commit();
    }
    for (int kt = 0; kt < nk; ++kt) {
        // tile kt's copies (committed kTcDist groups ago) have landed
        cp_wait<kTcDist - 1>();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (!__syncthreads_and(ok)) { ok = false; break; }
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int st = kt % kTcStages;
#pragma unroll
            for (int kk = 0; kk < kTcK / 16; ++kk) {
                const uint64_t ad = tc_desc(sa(st) + kk * 256, 128, kTcRowCore);
                const uint64_t bd = tc_desc(sb(st) + kk * 256, 128, kTcRowCore);
                const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                             ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar(st))
                         : "memory");
        }
        // with tile kt's products queued, refill the stage of tile kt - 2 (its products issued two steps
        // ago) with tile kt + kTcDist
        const int kn = kt + kTcDist;
        if (kn < nk) {
            if (kt >= 2 && !tc_mbar_wait(bar((kt - 2) % kTcStages), (uint32_t)(((kt - 2) / kTcStages) & 1))) ok = false;
            if (ok) {
                tc_load<AKM>(sa(kn % kTcStages), A, lda, m0, (int64_t)kn * kTcK);
                tc_load<BKM>(sb(kn % kTcStages), B, ldb, n0, (int64_t)kn * kTcK);
            }
        }
        cp_commit();
    }
    cp_wait<0>();
    // the last step's commit covers every product issued before it
    if (nk > 0 && ok && !tc_mbar_wait(bar((nk - 1) % kTcStages), (uint32_t)(((nk - 1) / kTcStages) & 1))) ok = false;
    if (ok) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int64_t m = m0 + warp * 32 + (tid & 31);
#pragma unroll 1
        for (int c0 = 0; c0 < 128; c0 += 16) {
            uint32_t r[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                         "%12, %13, %14, %15}, [%16];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                           "=r"(r[14]), "=r"(r[15])
                         : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const int64_t n = n0 + c0;
#pragma unroll
            for (int j = 0; j < 16; j += 2) {
                float v0 = __uint_as_float(r[j]), v1 = __uint_as_float(r[j + 1]);
                if (EPI == kEpiHidden || EPI == kEpiOut) { v0 += bias[n + j]; v1 += bias[n + j + 1]; }
                if (EPI == kEpiHidden) { v0 = fmaxf(v0, 0.f); v1 = fmaxf(v1, 0.f); }
                if (EPI == kEpiMask) {
                    const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162 *>(mask + m * ldc + n + j);
                    if (!(__bfloat162float(mk.x) > 0.f)) v0 = 0.f;
                    if (!(__bfloat162float(mk.y) > 0.f)) v1 = 0.f;
                }
                if (EPI == kEpiHidden || EPI == kEpiMask)
                    *reinterpret_cast<__nv_bfloat162 *>(static_cast<__nv_bfloat16 *>(C) + m * ldc + n + j) =
                        __floats2bfloat162_rn(v0, v1);
                else
                    *reinterpret_cast<float2 *>(static_cast<float *>(C) + m * ldc + n + j) = make_float2(v0, v1);
            }
        }
    } else if (tid == 0) {
        atomicExch(err, 1);
        // give the products in flight a bounded chance to finish before the memory is released
        if (nk > 0) tc_mbar_wait(bar((nk - 1) % kTcStages), (uint32_t)(((nk - 1) / kTcStages) & 1));
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
}

// ---- forward products on tcgen05 with TMA-fed, 128-byte-swizzled operands -------------------------
// Both operands of the forward product are K-major (activations [batch][in], weights [out][in]), so
// each stage's tiles are two TMA boxes: 128 rows x 64 reduction values of A and BN x 64 of B, written
// by the copy engine in the 128-byte swizzled layout that the tensor core's descriptor names (8-row
// groups 1024 bytes apart; a 16-wide reduction step is a 32-byte advance inside the swizzle row).
// Warp 0's first lane issues the copies into two (BN = 256) or three (BN = 128) stages, warp 1's first lane issues four tcgen05.mma
// (M = 128, N = BN, K = 16) per stage and commits each stage back to the copier and, at the end, to the
// epilogue; all four warps then read the FP32 accumulator (BN tensor-memory columns) and write the
// result.  Every mbarrier wait is bounded; one that gives up sets *err.
constexpr int kTmK = 64, kTmThreads = 128;

// Two blocks per SM (one's epilogue overlaps the other's products): 96 KB of stages each.
template <int BN>
struct TmShape {
    static constexpr int kStages = BN == 256 ? 2 : 3;
    static constexpr int kA = 128 * kTmK * 2, kB = BN * kTmK * 2, kStage = kA + kB;
    static constexpr int kBias = BN * 4;                          // the tile's bias values
    static constexpr int kSmem = kStages * kStage + 1024 + 128 + kBias;   // + alignment slack, barriers
};

__device__ __forceinline__ uint64_t tm_desc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void tm_load(uint32_t dst, const CUtensorMap *map, int32_t x, int32_t y, uint32_t bar) {
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
                 "[%4];" ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar) : "memory");
}

template <int BN, int EPI>
__global__ void __launch_bounds__(kTmThreads, 2) k_gemm_tma(const __grid_constant__ CUtensorMap ta,
                                                            const __grid_constant__ CUtensorMap tb, void *C, int64_t ldc,
                                                            int32_t K, const float *bias, const __nv_bfloat16 *mask,
                                                            __nv_bfloat16 *Ct, int64_t ldt, int32_t ksteps, int *err) {
    using S = TmShape<BN>;
    extern __shared__ unsigned char raw[];
    const uint32_t raw_s = tc_smem_u32(raw);
    const uint32_t base = (raw_s + 1023u) & ~1023u;              // swizzled tiles: 1024-byte aligned
    const uint32_t bars = base + S::kStages * S::kStage;           // full[stages], empty[stages], acc
    uint32_t *tslot = reinterpret_cast<uint32_t *>(raw + (bars - raw_s) + (2 * S::kStages + 1) * 8);
    float *bias_s = reinterpret_cast<float *>(raw + (bars - raw_s) + 128);   // after the barriers and tslot
    auto full = [&](int st) { return bars + 8u * st; };
    auto empty = [&](int st) { return bars + 8u * (S::kStages + st); };
    const uint32_t accb = bars + 8u * (2 * S::kStages);
    const int tid = (int)threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int32_t m0 = (int32_t)blockIdx.y * 128, n0 = (int32_t)blockIdx.x * BN;
    // reduction steps kt0 .. kt0 + nk - 1: all of them, or (ksteps > 0) block z's share of a split reduction
    const int kt0 = ksteps > 0 ? (int)blockIdx.z * ksteps : 0;
    const int nk = ksteps > 0 ? min(ksteps, K / kTmK - kt0) : K / kTmK;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem_u32(tslot)),
                     "r"((uint32_t)BN) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int st = 0; st < 2 * S::kStages + 1; ++st)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bars + 8u * st) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&ta)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tb)) : "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((128u >> 4) << 24);
    // Launched as a programmatic dependent of the previous product (the host sets the attribute only
    // there): the set-up above overlaps that kernel's end; nothing global is touched before it completes.
    // The next product may launch as soon as this one's blocks are all running.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");

    if (warp == 0 && lane == 0) {                       // the copier
        int issued = 0;
        bool ok = true;
        for (int kt = 0; kt < nk; ++kt) {
            const int st = kt % S::kStages;
            if (kt >= S::kStages && !tc_mbar_wait(empty(st), (uint32_t)((kt / S::kStages - 1) & 1))) { ok = false; break; }
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(full(st)), "r"((uint32_t)S::kStage)
                         : "memory");
            const uint32_t sa = base + (uint32_t)(st * S::kStage);
            tm_load(sa, &ta, (kt0 + kt) * kTmK, m0, full(st));
            tm_load(sa + S::kA, &tb, (kt0 + kt) * kTmK, n0, full(st));
            ++issued;
        }
        // no copy may still be landing when the block exits
        for (int j = issued > S::kStages ? issued - S::kStages : 0; j < issued; ++j)
            if (!tc_mbar_wait(full(j % S::kStages), (uint32_t)((j / S::kStages) & 1))) ok = false;
        if (!ok) atomicExch(err, 1);
    } else if (warp == 1 && lane == 0) {                // the tensor-core issuer
        bool ok = true;
        for (int kt = 0; kt < nk; ++kt) {
            const int st = kt % S::kStages;
            if (!tc_mbar_wait(full(st), (uint32_t)((kt / S::kStages) & 1))) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = base + (uint32_t)(st * S::kStage);
#pragma unroll
            for (int kk = 0; kk < kTmK / 16; ++kk) {
                const uint64_t ad = tm_desc_sw128(sa + kk * 32), bd = tm_desc_sw128(sa + S::kA + kk * 32);
                const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                             ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(empty(st))
                         : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(accb) : "memory");
        if (!ok) atomicExch(err, 1);
    }
    // While the products run: warps 2 and 3 stage the tile's bias values in shared memory, and every
    // thread loads the ReLU mask of its accumulator row (kEpiMask), so that the epilogue waits on no
    // global load.  (The copy and MMA lanes get here once their loops are done.)
    if constexpr (EPI == kEpiHidden || EPI == kEpiOut) {
        if (warp >= 2)
            for (int c = tid - 64; c < BN; c += kTmThreads - 64) bias_s[c] = __ldg(bias + n0 + c);
    }
    constexpr int kMaskHalf = BN / 16 > 8 ? 8 : BN / 16;                 // chunks of 16 columns held at once
    int4 mreg[kMaskHalf][2];
    const int64_t mrow = (int64_t)(m0 + warp * 32 + lane) * ldc + n0;
    if constexpr (EPI == kEpiMask) {
#pragma unroll
        for (int q = 0; q < kMaskHalf; ++q) {
            mreg[q][0] = __ldg(reinterpret_cast<const int4 *>(mask + mrow + 16 * q));
            mreg[q][1] = __ldg(reinterpret_cast<const int4 *>(mask + mrow + 16 * q + 8));
        }
    }
    __syncwarp();
    const bool done = tc_mbar_wait(accb, 0);
    if (!done && lane == 0) atomicExch(err, 1);
    // Epilogue: every product has completed (so the stages' shared memory is free), and the tile goes
    // through it: each thread writes its row (the accumulator's lane) in 16-column pieces to a padded
    // row-major tile, then the block stores whole rows to global memory with coalesced 16-byte stores.
    constexpr bool kBf16 = EPI == kEpiHidden || EPI == kEpiMask;
    using OutT = typename std::conditional<kBf16, __nv_bfloat16, float>::type;
    constexpr int kPadE = 16 / (int)sizeof(OutT);                       // one 16-byte chunk per row
    constexpr int kLd = BN + kPadE;                                      // row stride in elements
    static_assert(128 * kLd * (int)sizeof(OutT) <= S::kStages * S::kStage, "output tile exceeds the stages");
    OutT *tile = reinterpret_cast<OutT *>(raw + (base - raw_s));
    const bool all_done = __syncthreads_and(done);
    if (all_done) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int row = warp * 32 + lane;
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 16) {                            // unrolled: the mask chunks stay in registers
            if constexpr (EPI == kEpiMask) {
                if (c0 > 0 && (c0 / 16) % kMaskHalf == 0) {                 // BN = 256: the second half
#pragma unroll
                    for (int q = 0; q < kMaskHalf; ++q) {
                        mreg[q][0] = __ldg(reinterpret_cast<const int4 *>(mask + mrow + c0 + 16 * q));
                        mreg[q][1] = __ldg(reinterpret_cast<const int4 *>(mask + mrow + c0 + 16 * q + 8));
                    }
                }
            }
            uint32_t r[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                         "%12, %13, %14, %15}, [%16];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                           "=r"(r[14]), "=r"(r[15])
                         : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            uint32_t o[16];                                              // the 16 results, packed
            uint32_t mk[8] = {};                                         // this chunk's 16 mask values
            if constexpr (EPI == kEpiMask) {
                const int q = (c0 / 16) % kMaskHalf;
                const int4 a = mreg[q][0], b = mreg[q][1];
                mk[0] = (uint32_t)a.x; mk[1] = (uint32_t)a.y; mk[2] = (uint32_t)a.z; mk[3] = (uint32_t)a.w;
                mk[4] = (uint32_t)b.x; mk[5] = (uint32_t)b.y; mk[6] = (uint32_t)b.z; mk[7] = (uint32_t)b.w;
            }
#pragma unroll
            for (int j = 0; j < 16; j += 2) {
                float v0 = __uint_as_float(r[j]), v1 = __uint_as_float(r[j + 1]);
                if constexpr (EPI == kEpiHidden || EPI == kEpiOut) {
                    v0 += bias_s[c0 + j];
                    v1 += bias_s[c0 + j + 1];
                }
                if constexpr (EPI == kEpiMask) {                             // zero where the ReLU output was 0
                    const __nv_bfloat162 mw = *reinterpret_cast<const __nv_bfloat162 *>(&mk[j / 2]);
                    if (!(__bfloat162float(mw.x) > 0.f)) v0 = 0.f;
                    if (!(__bfloat162float(mw.y) > 0.f)) v1 = 0.f;
                }
                if constexpr (EPI == kEpiHidden) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                }
                if constexpr (kBf16) {
                    const __nv_bfloat162 b = __floats2bfloat162_rn(v0, v1);
                    o[j / 2] = *reinterpret_cast<const uint32_t *>(&b);
                } else {
                    o[j] = __float_as_uint(v0);
                    o[j + 1] = __float_as_uint(v1);
                }
            }
            if constexpr (kBf16) {
                if (Ct) {                                                // the transposed copy: Ct[n][m]
                    uint16_t *ct = reinterpret_cast<uint16_t *>(Ct) + (int64_t)(n0 + c0) * ldt + m0 + row;
#pragma unroll
                    for (int j = 0; j < 16; ++j) ct[j * ldt] = (uint16_t)((j & 1) ? (o[j / 2] >> 16) : (o[j / 2] & 0xFFFFu));
                }
            }
            int4 *dst = reinterpret_cast<int4 *>(tile + row * kLd + c0);
            constexpr int kVec = kBf16 ? 2 : 4;                          // 16-byte pieces of 16 results
#pragma unroll
            for (int q = 0; q < kVec; ++q) dst[q] = make_int4((int)o[4 * q], (int)o[4 * q + 1], (int)o[4 * q + 2], (int)o[4 * q + 3]);
        }
    }
    __syncthreads();
    if (all_done) {
        constexpr int kChunks = BN * (int)sizeof(OutT) / 16;             // 16-byte pieces of a row
        for (int i = tid; i < 128 * kChunks; i += kTmThreads) {
            const int row = i / kChunks, ch = i % kChunks;
            int4 v = *reinterpret_cast<const int4 *>(tile + row * kLd + ch * (16 / (int)sizeof(OutT)));
            const int64_t at = (m0 + row) * ldc + n0 + ch * (16 / (int)sizeof(OutT));
            if constexpr (EPI == kEpiAdd)                                // a split reduction's partial sum
                atomicAdd(reinterpret_cast<float4 *>(static_cast<float *>(C) + at),
                          make_float4(__int_as_float(v.x), __int_as_float(v.y), __int_as_float(v.z), __int_as_float(v.w)));
            else
                *reinterpret_cast<int4 *>(static_cast<OutT *>(C) + at) = v;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)BN) : "memory");
}

// x [B][n] FP32 -> xp [Bp][np] BF16, zero outside (and its transpose xpt [np][Bp] unless NULL).
__global__ void k_pack_input(const float *x, int32_t B, int32_t n, __nv_bfloat16 *xp, int64_t Bp, int64_t np,
                             __nv_bfloat16 *xpt) {
    const int64_t total = Bp * np;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / np, c = i % np;
        xp[i] = __float2bfloat16_rn(r < B && c < n ? x[r * n + c] : 0.f);
        if (xpt) xpt[c * Bp + r] = xp[i];
    }
}

// yp [Bp][np] -> y [B][n].
__global__ void k_unpack_output(const float *yp, int64_t np, int32_t B, int32_t n, float *y) {
    const int64_t total = (int64_t)B * n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = yp[(i / n) * np + i % n];
}

// Mean squared error: dY = bf16(2 (y - t) / (B n)) on the real entries, 0 elsewhere; *loss += sum (y - t)^2
// / (B n) (zeroed beforehand).
__global__ void k_mse(const float *yp, int64_t np, const float *t, int32_t B, int32_t n, int64_t Bp,
                      __nv_bfloat16 *dy, __nv_bfloat16 *dyt, double *loss) {
    __shared__ double red[32];
    const int64_t total = Bp * np;
    const double scale = 1.0 / ((double)B * n);
    double part = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / np, c = i % np;
        float d = 0.f;
        if (r < B && c < n) {
            d = yp[i] - t[r * n + c];
            part += (double)d * d;
        }
        dy[i] = __float2bfloat16_rn((float)(2.0 * scale) * d);
        if (dyt) dyt[c * Bp + r] = dy[i];                     // the transpose [np][Bp], unless NULL
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x < 32) {
        part = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (threadIdx.x == 0 && loss) atomicAdd(loss, part * scale);
    }
}

// db[c] += sum over rows [blockIdx.y * kBiasRows, + kBiasRows) of dz[r][c] (db zeroed beforehand): 32
// columns per block, the rows strided over blockDim.y = 8, the partial sums added with FP32 atomics.
constexpr int kBiasRows = 256;
__global__ void k_bias_grad(const __nv_bfloat16 *dz, int64_t Bp, int64_t np, float *db) {
    __shared__ float red[8][32];
    const int64_t c = (int64_t)blockIdx.x * 32 + threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.y * kBiasRows, r1 = r0 + kBiasRows < Bp ? r0 + kBiasRows : Bp;
    float s = 0.f;
    for (int64_t r = r0 + threadIdx.y; r < r1; r += blockDim.y) s += __bfloat162float(dz[r * np + c]);
    red[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0) {
        for (int k = 1; k < (int)blockDim.y; ++k) s += red[k][threadIdx.x];
        atomicAdd(db + c, s);
    }
}

// Adam over the flat (padded) parameter array; the BF16 mirror follows the FP32 parameters.
__global__ void k_adam(float *p, const float *g, float *m1, float *m2, __nv_bfloat16 *pb, int64_t n, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float a = b1 * m1[i] + (1.f - b1) * gi;
        const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
        m1[i] = a;
        m2[i] = b;
        const float q = p[i] - lr * (a / c1) / (sqrtf(b / c2) + eps);
        p[i] = q;
        pb[i] = __float2bfloat16_rn(q);
    }
}

// wt [cols][rows] = w [rows][cols] (BF16, both dimensions multiples of 32), through 32 x 32 tiles.
__global__ void k_transpose_w(const __nv_bfloat16 *w, int64_t rows, int64_t cols, __nv_bfloat16 *wt) {
    __shared__ __nv_bfloat16 t[32][34];
    const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    for (int i = (int)threadIdx.y; i < 32; i += (int)blockDim.y) t[i][threadIdx.x] = w[(r0 + i) * cols + c0 + threadIdx.x];
    __syncthreads();
    for (int i = (int)threadIdx.y; i < 32; i += (int)blockDim.y) wt[(c0 + i) * rows + r0 + threadIdx.x] = t[threadIdx.x][i];
}

__global__ void k_to_bf16(const float *p, __nv_bfloat16 *pb, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        pb[i] = __float2bfloat16_rn(p[i]);
}

thread_local std::string g_mlp_err;

}  // namespace

struct cfr_mlp {
    int L = 0;
    std::vector<int32_t> dims;       // real widths
    std::vector<int64_t> pdims;      // padded widths
    std::vector<int64_t> w_off, b_off;   // per layer: offsets of W [pdims[l+1]][pdims[l]] and b in the flat arrays
    int64_t P = 0, num_params = 0;   // flat padded size, real parameter count
    int device = 0, sms = 152;
    cudaStream_t stream = nullptr;
    float *p = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr;
    __nv_bfloat16 *pb = nullptr;
    __nv_bfloat16 *pbt = nullptr;    // each layer's BF16 weights transposed ([in][out] at w_off): the K-major
                                     // operand of the data-gradient products on the TMA path
    int64_t steps = 0;
    // activations for the largest batch seen: acts[0] input, acts[l] hidden output of layer l - 1
    int64_t cap = 0;
    std::vector<__nv_bfloat16 *> acts, grads;   // grads[l]: dL/dZ of layer l (BF16, [cap][pdims[l + 1]])
    // their transposes ([pdims[l]][Bp] and [pdims[l + 1]][Bp], row length the padded batch of the pass),
    // written in training passes on the TMA path: the K-major operands of the weight gradients
    std::vector<__nv_bfloat16 *> acts_t, grads_t;
    float *yp = nullptr;
    int64_t last_batch = 0;          // real rows of the last forward or backward pass
    bool have_dz = false;            // grads[] hold the last backward pass's output gradients
    cudaEvent_t ev[4] = {};
    double fwd_flops = 0, bwd_flops = 0;
    bool fwd_timed = false, bwd_timed = false;
    int32_t path = 2;                // cfr_mlp_set_tensor_path: 0 mma.sync, 1 tcgen05, 2 (default) mixed
    mutable bool pdl_next = false;   // the last operation queued by a pass was a product kernel
    int *d_err = nullptr;            // set by a tcgen05 kernel whose mbarrier wait gave up
    std::string err;
    bool poisoned = false;
    // The products of a forward pass and of a backward pass (after the loss gradient), replayed from a
    // CUDA graph: the host's per-launch work (tensor-map encoding, launch) then no longer sits between the
    // kernels.  A graph is captured (on cap_stream, a stream of its own) the second time a pass runs with the same
    // key; the first run of a key is launched directly.
    cudaStream_t cap_stream = nullptr;
    // Path 2's backward pass runs each layer's weight gradient on side (forked from the pass's stream once
    // that layer's output gradient exists, joined at the end) beside the data-gradient chain.
    cudaStream_t side = nullptr;
    std::vector<cudaEvent_t> fork_ev;
    cudaEvent_t join_ev = nullptr;
    struct PassGraph {
        cudaGraphExec_t exec = nullptr;
        int64_t bp = 0, cap = 0;     // the key: padded batch, buffer capacity, tensor path
        int32_t path = -1;
        bool seen = false;           // the key has run once directly
        double flops = 0;            // the pass's multiply-add work, times two
    } gfwd, gfwd_train, gbwd;
};

namespace {

cfr_status merr(cfr_mlp *m, cfr_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (m) m->err = buf;
    else g_mlp_err = buf;
    return st;
}

#define MCK(call)                                                                                         \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess) {                                                                          \
            m->poisoned = true;                                                                           \
            return merr(m, e_ == cudaErrorMemoryAllocation ? CFR_ERR_OOM : CFR_ERR_CUDA, "%s: %s (%s:%d)", #call, \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                                      \
        }                                                                                                 \
    } while (0)

struct MDeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit MDeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; prev = -1; return; }
        if (dev >= 0 && dev != prev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~MDeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

cfr_status usable(cfr_mlp *m) {
    if (!m) return merr(nullptr, CFR_ERR_INVALID, "network is NULL");
    if (m->poisoned) return merr(m, CFR_ERR_STATE, "network is unusable after an earlier CUDA error: %s", m->err.c_str());
    return CFR_OK;
}

int grid_for(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 152 * 16); }

cfr_status ensure_batch(cfr_mlp *m, int64_t Bp) {
    if (Bp <= m->cap) return CFR_OK;
    for (auto *v : {&m->acts, &m->grads, &m->acts_t, &m->grads_t})
        for (auto *a : *v) cudaFree(a);
    cudaFree(m->yp);
    for (auto *v : {&m->acts, &m->grads, &m->acts_t, &m->grads_t}) v->assign((size_t)m->L, nullptr);
    m->yp = nullptr;
    m->cap = 0;
    for (int l = 0; l < m->L; ++l) {
        MCK(cudaMalloc(&m->acts[(size_t)l], sizeof(__nv_bfloat16) * (size_t)(Bp * m->pdims[(size_t)l])));
        MCK(cudaMalloc(&m->grads[(size_t)l], sizeof(__nv_bfloat16) * (size_t)(Bp * m->pdims[(size_t)l + 1])));
        MCK(cudaMalloc(&m->acts_t[(size_t)l], sizeof(__nv_bfloat16) * (size_t)(Bp * m->pdims[(size_t)l])));
        MCK(cudaMalloc(&m->grads_t[(size_t)l], sizeof(__nv_bfloat16) * (size_t)(Bp * m->pdims[(size_t)l + 1])));
    }
    MCK(cudaMalloc(&m->yp, sizeof(float) * (size_t)(Bp * m->pdims[(size_t)m->L])));
    m->cap = Bp;
    return CFR_OK;
}

template <bool AKM, bool BKM, int EPI>
cudaError_t gemm_tc(cudaStream_t st, int *err, const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B, int64_t ldb,
                    void *C, int64_t ldc, int64_t M, int64_t N, int64_t K, const float *bias, const __nv_bfloat16 *mask) {
    static bool attr = false;   // per instantiation; the attribute is per device function
    if (!attr) {
        const cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<AKM, BKM, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const dim3 grid((unsigned)(N / 128), (unsigned)(M / 128));
    k_gemm_tc<AKM, BKM, EPI><<<grid, kTcThreads, kTcSmem, st>>>(A, lda, B, ldb, C, ldc, (int32_t)K, bias, mask, err);
    return cudaGetLastError();
}

// C = A B on the network's tensor path (tcgen05 or mma.sync); shapes are multiples of 128.  On the
// warp-level path a product with fewer output tiles than two per SM and a long reduction (kEpiStore:
// the weight gradients, reduced over the batch) splits its reduction over more blocks, which add their
// partial sums into C (zeroed first) with FP32 atomics.
template <bool AKM, bool BKM, int EPI>
cudaError_t gemm(const cfr_mlp *m, const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B, int64_t ldb, void *C,
                 int64_t ldc, int64_t M, int64_t N, int64_t K, const float *bias, const __nv_bfloat16 *mask) {
    if (m->path == 1) {
        m->pdl_next = true;
        return gemm_tc<AKM, BKM, EPI>(m->stream, m->d_err, A, lda, B, ldb, C, ldc, M, N, K, bias, mask);
    }
    const int64_t tiles = (N / kBN) * (M / kBM), steps = K / kBK;
    int64_t split = 1;
    if constexpr (EPI == kEpiStore) split = std::min<int64_t>((2 * m->sms + tiles - 1) / tiles, steps / 8);
    if (split > 1) {
        const int32_t ksteps = (int32_t)((steps + split - 1) / split);
        split = (steps + ksteps - 1) / ksteps;
        m->pdl_next = false;                // a memset comes next: the product after it waits in full
        for (int64_t r = 0; r < M; ++r) {   // C's rows are ldc apart: zero them (one call when contiguous)
            if (ldc == N) {
                const cudaError_t e = cudaMemsetAsync(C, 0, sizeof(float) * (size_t)(M * N), m->stream);
                if (e != cudaSuccess) return e;
                break;
            }
            const cudaError_t e = cudaMemsetAsync(static_cast<float *>(C) + r * ldc, 0, sizeof(float) * (size_t)N, m->stream);
            if (e != cudaSuccess) return e;
        }
        const dim3 grid((unsigned)(N / kBN), (unsigned)(M / kBM), (unsigned)split);
        k_gemm<AKM, BKM, kEpiAdd><<<grid, kThreads, 0, m->stream>>>(A, lda, B, ldb, C, ldc, (int32_t)K, bias, mask, ksteps);
        m->pdl_next = true;
        return cudaGetLastError();
    }
    const dim3 grid((unsigned)(N / kBN), (unsigned)(M / kBM));
    k_gemm<AKM, BKM, EPI><<<grid, kThreads, 0, m->stream>>>(A, lda, B, ldb, C, ldc, (int32_t)K, bias, mask, 0);
    m->pdl_next = true;
    return cudaGetLastError();
}

// The driver's tensor-map encoder, fetched once through the runtime.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// A 2-D K-major BF16 operand [rows][K] (row stride K elements) in boxes of box_rows x 64, 128-byte swizzle.
bool encode_operand(CUtensorMap *map, const __nv_bfloat16 *g, int64_t rows, int64_t K, int box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kTmK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(g), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// k_gemm_tma launched on m->stream, as a programmatic dependent of the previous launch when that was a
// product kernel of the same pass (m->pdl_next).
template <int BN, int EPI>
cudaError_t launch_tma(const cfr_mlp *m, dim3 grid, const CUtensorMap &ta, const CUtensorMap &tb, void *C, int64_t ldc,
                       int32_t K, const float *bias, const __nv_bfloat16 *mask, __nv_bfloat16 *Ct = nullptr,
                       int64_t ldt = 0, int32_t ksteps = 0) {
    cudaLaunchConfig_t c = {};
    c.gridDim = grid;
    c.blockDim = dim3(kTmThreads);
    c.dynamicSmemBytes = TmShape<BN>::kSmem;
    c.stream = m->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    c.attrs = at;
    c.numAttrs = m->pdl_next ? 1 : 0;
    const cudaError_t e = cudaLaunchKernelEx(&c, k_gemm_tma<BN, EPI>, ta, tb, C, ldc, K, bias, mask, Ct, ldt, ksteps, m->d_err);
    m->pdl_next = true;
    return e;
}

// The forward product on tcgen05 with TMA operands: BN = 256 where N allows, else 128.
template <int EPI>
cudaError_t gemm_fwd_tma(const cfr_mlp *m, const __nv_bfloat16 *A, const __nv_bfloat16 *W, void *C, int64_t M, int64_t N,
                         int64_t K, const float *bias, const __nv_bfloat16 *mask = nullptr, __nv_bfloat16 *Ct = nullptr) {
    CUtensorMap ta, tb;
    // 256-wide tiles where they still give two blocks per SM, else 128-wide (the FP32 output tile of the
    // last layer takes the 128-wide shape, whose stages can hold it for the epilogue)
    const int bn = (EPI != kEpiOut && N % 256 == 0 && (N / 256) * (M / 128) >= 2 * 152) ? 256 : 128;
    if (!encode_operand(&ta, A, M, K, 128) || !encode_operand(&tb, W, N, K, bn)) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)(N / bn), (unsigned)(M / 128));
    if constexpr (EPI == kEpiOut) {
        static bool attr = false;
        if (!attr) {
            const cudaError_t e = cudaFuncSetAttribute(k_gemm_tma<128, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       TmShape<128>::kSmem);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        return launch_tma<128, EPI>(m, grid, ta, tb, C, N, (int32_t)K, bias, mask, Ct, M);
    } else if (bn == 256) {
        static bool attr = false;
        if (!attr) {
            const cudaError_t e = cudaFuncSetAttribute(k_gemm_tma<256, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       TmShape<256>::kSmem);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        return launch_tma<256, EPI>(m, grid, ta, tb, C, N, (int32_t)K, bias, mask, Ct, M);
    } else {
        static bool attr = false;
        if (!attr) {
            const cudaError_t e = cudaFuncSetAttribute(k_gemm_tma<128, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       TmShape<128>::kSmem);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        return launch_tma<128, EPI>(m, grid, ta, tb, C, N, (int32_t)K, bias, mask, Ct, M);
    }
}

// A weight gradient on tcgen05 with TMA operands: C [M][N] (FP32) = A [M][K] B [N][K]^T with both operands
// K-major (the transposed output gradient [out][batch] and the transposed layer input [in][batch]), the
// reduction over the batch split over enough blocks for two per SM, each adding its partial tile into C
// (zeroed first) with FP32 vector atomics.
cudaError_t gemm_dw_tma(const cfr_mlp *m, const __nv_bfloat16 *A, const __nv_bfloat16 *B, float *C, int64_t M, int64_t N,
                        int64_t K) {
    CUtensorMap ta, tb;
    if (!encode_operand(&ta, A, M, K, 128) || !encode_operand(&tb, B, N, K, 128)) return cudaErrorInvalidValue;
    const int64_t tiles = (N / 128) * (M / 128), steps = K / kTmK;
    // at most two blocks per SM in all (one wave of the two that fit): a block more starts a second wave
    int64_t split = std::max<int64_t>(1, std::min<int64_t>((2 * m->sms) / tiles, steps));
    const int64_t ksteps = (steps + split - 1) / split;
    split = (steps + ksteps - 1) / ksteps;
    static bool attr = false;
    if (!attr) {
        const cudaError_t e = cudaFuncSetAttribute(k_gemm_tma<128, kEpiAdd>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   TmShape<128>::kSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    cudaError_t e = cudaMemsetAsync(C, 0, sizeof(float) * (size_t)(M * N), m->stream);
    if (e != cudaSuccess) return e;
    m->pdl_next = false;
    const dim3 grid((unsigned)(N / 128), (unsigned)(M / 128), (unsigned)split);
    return launch_tma<128, kEpiAdd>(m, grid, ta, tb, C, N, (int32_t)K, nullptr, nullptr, nullptr, 0, (int32_t)ksteps);
}

// The transposed BF16 weights of every layer from the BF16 mirror.
cudaError_t refresh_transposes(const cfr_mlp *m) {
    for (int l = 0; l < m->L; ++l) {
        const int64_t out = m->pdims[(size_t)l + 1], in = m->pdims[(size_t)l];
        k_transpose_w<<<dim3((unsigned)(in / 32), (unsigned)(out / 32)), dim3(32, 8), 0, m->stream>>>(
            m->pb + m->w_off[(size_t)l], out, in, m->pbt + m->w_off[(size_t)l]);
    }
    return cudaGetLastError();
}

// CFR_ERR_TIMEOUT if a tensor-core kernel gave up waiting (synchronises).
cfr_status check_err(cfr_mlp *m) {
    int e = 0;
    MCK(cudaMemcpyAsync(&e, m->d_err, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    MCK(cudaStreamSynchronize(m->stream));
    if (e) {
        m->poisoned = true;
        return merr(m, CFR_ERR_TIMEOUT, "a tensor-core product gave up waiting for its operands");
    }
    return CFR_OK;
}

// The forward pass over Bp padded rows (input already packed into acts[0]); output in yp.  Launches on
// m->stream.  train (TMA path): the hidden outputs' transposes too.
cfr_status forward_impl(cfr_mlp *m, int64_t Bp, double *flops, bool train) {
    double f = 0;
    m->pdl_next = false;
    for (int l = 0; l < m->L; ++l) {
        const int64_t K = m->pdims[(size_t)l], N = m->pdims[(size_t)l + 1];
        const __nv_bfloat16 *W = m->pb + m->w_off[(size_t)l];
        const float *b = m->p + m->b_off[(size_t)l];
        if (m->path != 0) {   // tcgen05 with TMA operands
            if (l + 1 < m->L)
                MCK(gemm_fwd_tma<kEpiHidden>(m, m->acts[(size_t)l], W, m->acts[(size_t)l + 1], Bp, N, K, b, nullptr,
                                             train && m->path == 2 ? m->acts_t[(size_t)l + 1] : nullptr));
            else MCK(gemm_fwd_tma<kEpiOut>(m, m->acts[(size_t)l], W, m->yp, Bp, N, K, b));
        } else if (l + 1 < m->L) {
            MCK((gemm<true, true, kEpiHidden>(m, m->acts[(size_t)l], K, W, K, m->acts[(size_t)l + 1], N, Bp, N, K, b, nullptr)));
        } else {
            MCK((gemm<true, true, kEpiOut>(m, m->acts[(size_t)l], K, W, K, m->yp, N, Bp, N, K, b, nullptr)));
        }
        f += 2.0 * (double)Bp * N * K;
    }
    *flops = f;
    return CFR_OK;
}
cfr_status forward_padded(cfr_mlp *m, int64_t Bp, double *flops) { return forward_impl(m, Bp, flops, false); }
cfr_status forward_train(cfr_mlp *m, int64_t Bp, double *flops) { return forward_impl(m, Bp, flops, true); }

// The backward products over Bp padded rows (the output gradient already in grads[L - 1]): every weight
// gradient and every masked data gradient.  Launches on m->stream.
cfr_status backward_products(cfr_mlp *m, int64_t Bp, double *flops) {
    double fb = 0;
    m->pdl_next = false;
    for (int l = m->L - 1; l >= 0; --l) {
        const int64_t K = m->pdims[(size_t)l], N = m->pdims[(size_t)l + 1];
        const __nv_bfloat16 *dz = m->grads[(size_t)l];
        // dW[o][i] = sum_b dZ[b][o] X[b][i]
        if (m->path == 2) {  // tcgen05 with TMA operands: the transposes dZ^T [out][batch] and X^T [in][batch]
            // on the side stream, beside the data gradients, once this layer's output gradient is written
            MCK(cudaEventRecord(m->fork_ev[(size_t)l], m->stream));
            MCK(cudaStreamWaitEvent(m->side, m->fork_ev[(size_t)l], 0));
            cudaStream_t main = m->stream;
            const bool pdl = m->pdl_next;
            m->stream = m->side;
            const cudaError_t e = gemm_dw_tma(m, m->grads_t[(size_t)l], m->acts_t[(size_t)l], m->g + m->w_off[(size_t)l],
                                              N, K, Bp);
            m->stream = main;
            m->pdl_next = pdl;
            MCK(e);
        } else
            MCK((gemm<false, false, kEpiStore>(m, dz, N, m->acts[(size_t)l], K, m->g + m->w_off[(size_t)l], K, N, K, Bp,
                                               nullptr, nullptr)));
        fb += 2.0 * (double)N * K * Bp;
        if (l > 0) {   // dZ of layer l - 1 = (dZ W) masked where its ReLU output was 0
            if (m->path == 2)   // tcgen05 with TMA operands: dZ [batch][out] and W^T [in][out], both K-major
                MCK(gemm_fwd_tma<kEpiMask>(m, dz, m->pbt + m->w_off[(size_t)l], m->grads[(size_t)l - 1], Bp, K, N, nullptr,
                                           m->acts[(size_t)l], m->grads_t[(size_t)l - 1]));
            else
                MCK((gemm<true, false, kEpiMask>(m, dz, N, m->pb + m->w_off[(size_t)l], K, m->grads[(size_t)l - 1], K, Bp,
                                                 K, N, nullptr, m->acts[(size_t)l])));
            fb += 2.0 * (double)Bp * K * N;
        }
    }
    if (m->path == 2) {              // the weight gradients are done before the pass ends
        MCK(cudaEventRecord(m->join_ev, m->side));
        MCK(cudaStreamWaitEvent(m->stream, m->join_ev, 0));
        m->pdl_next = false;
    }
    *flops = fb;
    return CFR_OK;
}

// Runs pass (forward_padded or backward_products) for Bp rows on m->stream: directly the first time a key
// (Bp, buffers, tensor path) is seen, from the pass's graph after that.
cfr_status run_pass(cfr_mlp *m, cfr_mlp::PassGraph *g, cfr_status (*pass)(cfr_mlp *, int64_t, double *), int64_t Bp,
                    double *flops) {
    const bool same = g->bp == Bp && g->cap == m->cap && g->path == m->path;
    if (!same) {                         // a new key: run directly first (this also sets kernel attributes)
        if (g->exec) cudaGraphExecDestroy(g->exec);
        g->exec = nullptr;
        g->bp = Bp;
        g->cap = m->cap;
        g->path = m->path;
        g->seen = false;
    }
    if (!g->exec && g->seen && m->cap_stream) {
        MCK(cudaStreamBeginCapture(m->cap_stream, cudaStreamCaptureModeThreadLocal));
        cudaStream_t user = m->stream;
        m->stream = m->cap_stream;
        const cfr_status st = pass(m, Bp, &g->flops);
        m->stream = user;
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(m->cap_stream, &graph);
        if (st != CFR_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        MCK(e);
        const cudaError_t ei = cudaGraphInstantiate(&g->exec, graph, 0);
        cudaGraphDestroy(graph);
        MCK(ei);
    }
    if (g->exec) {
        MCK(cudaGraphLaunch(g->exec, m->stream));
        *flops = g->flops;
        return CFR_OK;
    }
    g->seen = true;
    const cfr_status st = pass(m, Bp, &g->flops);
    *flops = g->flops;
    return st;
}

}  // namespace

extern "C" {

cfr_status cfr_mlp_create(const int32_t *dims, int32_t num_layers, int32_t device, void *cuda_stream, cfr_mlp **out) {
    if (!out) return merr(nullptr, CFR_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!dims || num_layers < 1 || num_layers > 8) return merr(nullptr, CFR_ERR_INVALID, "num_layers must be in [1, 8]");
    for (int l = 0; l <= num_layers; ++l)
        if (dims[l] < 1 || dims[l] > 8192) return merr(nullptr, CFR_ERR_INVALID, "dims[%d] = %d is outside [1, 8192]", l, dims[l]);
    MDeviceGuard dg(device);
    if (!dg.ok) return merr(nullptr, CFR_ERR_CUDA, "cannot select CUDA device %d", device);
    cfr_mlp *m = new cfr_mlp();
    cudaGetDevice(&m->device);
    if (cudaDeviceGetAttribute(&m->sms, cudaDevAttrMultiProcessorCount, m->device) != cudaSuccess) {
        cudaGetLastError();
        m->sms = 152;
    }
    m->stream = static_cast<cudaStream_t>(cuda_stream);
    m->L = num_layers;
    m->dims.assign(dims, dims + num_layers + 1);
    for (int l = 0; l <= num_layers; ++l) m->pdims.push_back(pad_to(dims[l], kPad));
    for (int l = 0; l < num_layers; ++l) {
        m->w_off.push_back(m->P);
        m->P += m->pdims[(size_t)l + 1] * m->pdims[(size_t)l];
        m->b_off.push_back(m->P);
        m->P += m->pdims[(size_t)l + 1];
        m->num_params += (int64_t)dims[l + 1] * dims[l] + dims[l + 1];
    }
    auto fail = [&](cudaError_t e) {
        std::string msg = cudaGetErrorString(e);
        cudaGetLastError();
        cfr_mlp_free(m);
        return merr(nullptr, e == cudaErrorMemoryAllocation ? CFR_ERR_OOM : CFR_ERR_CUDA, "network allocation: %s", msg.c_str());
    };
    cudaError_t e = cudaMalloc(&m->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(m->d_err, 0, sizeof(int), m->stream);
    for (float **a : {&m->p, &m->g, &m->m1, &m->m2})
        if (e == cudaSuccess) e = cudaMalloc(a, sizeof(float) * (size_t)m->P);
    if (e == cudaSuccess) e = cudaMalloc(&m->pb, sizeof(__nv_bfloat16) * (size_t)m->P);
    if (e == cudaSuccess) e = cudaMalloc(&m->pbt, sizeof(__nv_bfloat16) * (size_t)m->P);
    for (float *a : {m->p, m->g, m->m1, m->m2})
        if (e == cudaSuccess) e = cudaMemsetAsync(a, 0, sizeof(float) * (size_t)m->P, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->pb, 0, sizeof(__nv_bfloat16) * (size_t)m->P, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->pbt, 0, sizeof(__nv_bfloat16) * (size_t)m->P, m->stream);
    for (cudaEvent_t &ev : m->ev)
        if (e == cudaSuccess) e = cudaEventCreate(&ev);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&m->side, cudaStreamNonBlocking);
    m->fork_ev.assign((size_t)m->L, nullptr);
    for (cudaEvent_t &ev : m->fork_ev)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->join_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return fail(e);
    *out = m;
    return CFR_OK;
}

int64_t cfr_mlp_num_params(const cfr_mlp *m) { return m ? m->num_params : 0; }

cfr_status cfr_mlp_set_params(cfr_mlp *m, const float *params, int64_t len) {
    cfr_status st = usable(m);
    if (st != CFR_OK) return st;
    if (!params || len < m->num_params) return merr(m, CFR_ERR_INVALID, "params needs %lld entries", (long long)m->num_params);
    MDeviceGuard dg(m->device);
    std::vector<float> flat((size_t)m->P, 0.f);
    int64_t k = 0;
    for (int l = 0; l < m->L; ++l) {
        const int64_t in = m->dims[(size_t)l], o = m->dims[(size_t)l + 1], ld = m->pdims[(size_t)l];
        for (int64_t r = 0; r < o; ++r)
            for (int64_t c = 0; c < in; ++c) flat[(size_t)(m->w_off[(size_t)l] + r * ld + c)] = params[k++];
        for (int64_t r = 0; r < o; ++r) flat[(size_t)(m->b_off[(size_t)l] + r)] = params[k++];
    }
    MCK(cudaMemcpyAsync(m->p, flat.data(), sizeof(float) * flat.size(), cudaMemcpyHostToDevice, m->stream));
    k_to_bf16<<<grid_for(m->P), 256, 0, m->stream>>>(m->p, m->pb, m->P);
    MCK(cudaGetLastError());
    MCK(refresh_transposes(m));
    for (float *a : {m->m1, m->m2}) MCK(cudaMemsetAsync(a, 0, sizeof(float) * (size_t)m->P, m->stream));
    m->steps = 0;
    MCK(cudaStreamSynchronize(m->stream));
    return CFR_OK;
}

static cfr_status get_flat(cfr_mlp *m, const float *dev, float *out, int64_t len) {
    cfr_status st = usable(m);
    if (st != CFR_OK) return st;
    if (!out || len < m->num_params) return merr(m, CFR_ERR_INVALID, "output needs %lld entries", (long long)m->num_params);
    MDeviceGuard dg(m->device);
    if ((st = check_err(m)) != CFR_OK) return st;
    std::vector<float> flat((size_t)m->P);
    MCK(cudaMemcpyAsync(flat.data(), dev, sizeof(float) * flat.size(), cudaMemcpyDeviceToHost, m->stream));
    MCK(cudaStreamSynchronize(m->stream));
    int64_t k = 0;
    for (int l = 0; l < m->L; ++l) {
        const int64_t in = m->dims[(size_t)l], o = m->dims[(size_t)l + 1], ld = m->pdims[(size_t)l];
        for (int64_t r = 0; r < o; ++r)
            for (int64_t c = 0; c < in; ++c) out[k++] = flat[(size_t)(m->w_off[(size_t)l] + r * ld + c)];
        for (int64_t r = 0; r < o; ++r) out[k++] = flat[(size_t)(m->b_off[(size_t)l] + r)];
    }
    return CFR_OK;
}

cfr_status cfr_mlp_get_params(cfr_mlp *m, float *params, int64_t len) { return get_flat(m, m ? m->p : nullptr, params, len); }
cfr_status cfr_mlp_get_grads(cfr_mlp *m, float *grads, int64_t len) { return get_flat(m, m ? m->g : nullptr, grads, len); }

cfr_status cfr_mlp_forward(cfr_mlp *m, const float *x, int32_t batch, float *y) {
    cfr_status st = usable(m);
    if (st != CFR_OK) return st;
    if (!x || !y || batch < 1) return merr(m, CFR_ERR_INVALID, "x and y must be device arrays and batch >= 1");
    MDeviceGuard dg(m->device);
    const int64_t Bp = pad_to(batch, kPad);
    if ((st = ensure_batch(m, Bp)) != CFR_OK) return st;
    k_pack_input<<<grid_for(Bp * m->pdims[0]), 256, 0, m->stream>>>(x, batch, m->dims[0], m->acts[0], Bp, m->pdims[0],
                                                                   nullptr);
    MCK(cudaGetLastError());
    MCK(cudaEventRecord(m->ev[0], m->stream));
    if ((st = run_pass(m, &m->gfwd, forward_padded, Bp, &m->fwd_flops)) != CFR_OK) return st;
    MCK(cudaEventRecord(m->ev[1], m->stream));
    m->fwd_timed = true;
    m->last_batch = batch;
    m->have_dz = false;
    k_unpack_output<<<grid_for((int64_t)batch * m->dims[(size_t)m->L]), 256, 0, m->stream>>>(
        m->yp, m->pdims[(size_t)m->L], batch, m->dims[(size_t)m->L], y);
    MCK(cudaGetLastError());
    return CFR_OK;
}

cfr_status cfr_mlp_backward(cfr_mlp *m, const float *x, const float *target, int32_t batch, double *loss) {
    cfr_status st = usable(m);
    if (st != CFR_OK) return st;
    if (!x || !target || batch < 1) return merr(m, CFR_ERR_INVALID, "x and target must be device arrays and batch >= 1");
    MDeviceGuard dg(m->device);
    const int64_t Bp = pad_to(batch, kPad);
    if ((st = ensure_batch(m, Bp)) != CFR_OK) return st;
    const int L = m->L;
    const bool tr = m->path == 2;                         // the weight gradients read transposed operands
    k_pack_input<<<grid_for(Bp * m->pdims[0]), 256, 0, m->stream>>>(x, batch, m->dims[0], m->acts[0], Bp, m->pdims[0],
                                                                   tr ? m->acts_t[0] : nullptr);
    MCK(cudaGetLastError());
    double f = 0;
    if ((st = run_pass(m, &m->gfwd_train, forward_train, Bp, &f)) != CFR_OK) return st;
    if (loss) MCK(cudaMemsetAsync(loss, 0, sizeof(double), m->stream));
    const int64_t nL = m->pdims[(size_t)L];
    // few blocks: each adds its part of the loss with one FP64 atomic
    k_mse<<<std::min(grid_for(Bp * nL), 2 * m->sms), 256, 0, m->stream>>>(m->yp, nL, target, batch, m->dims[(size_t)L], Bp,
                                                    m->grads[(size_t)L - 1], tr ? m->grads_t[(size_t)L - 1] : nullptr, loss);
    MCK(cudaGetLastError());
    MCK(cudaEventRecord(m->ev[2], m->stream));
    double fb = 0;
    if ((st = run_pass(m, &m->gbwd, backward_products, Bp, &fb)) != CFR_OK) return st;
    MCK(cudaEventRecord(m->ev[3], m->stream));
    m->bwd_flops = fb;
    m->bwd_timed = true;
    m->last_batch = batch;
    m->have_dz = true;
    for (int l = 0; l < L; ++l) {
        const int64_t N = m->pdims[(size_t)l + 1];
        MCK(cudaMemsetAsync(m->g + m->b_off[(size_t)l], 0, sizeof(float) * (size_t)N, m->stream));
        k_bias_grad<<<dim3((unsigned)(N / 32), (unsigned)((Bp + kBiasRows - 1) / kBiasRows)), dim3(32, 8), 0, m->stream>>>(
            m->grads[(size_t)l], Bp, N, m->g + m->b_off[(size_t)l]);
        MCK(cudaGetLastError());
    }
    return CFR_OK;
}

cfr_status cfr_mlp_get_intermediate(cfr_mlp *m, int32_t which, int32_t layer, float *out, int64_t len) {
    cfr_status st = usable(m);
    if (st != CFR_OK) return st;
    if (!out) return merr(m, CFR_ERR_INVALID, "out is NULL");
    if (m->last_batch < 1) return merr(m, CFR_ERR_STATE, "no forward or backward pass has run yet");
    if (which == CFR_MLP_DZ && !m->have_dz) return merr(m, CFR_ERR_STATE, "the last pass was not a backward pass");
    if (which != CFR_MLP_OUT && (layer < 0 || layer >= m->L))
        return merr(m, CFR_ERR_INVALID, "layer %d is outside [0, %d)", layer, m->L);
    int64_t cols = 0, ld = 0;
    const void *src = nullptr;
    bool bf16 = true;
    switch (which) {
    case CFR_MLP_ACT: cols = m->dims[(size_t)layer]; ld = m->pdims[(size_t)layer]; src = m->acts[(size_t)layer]; break;
    case CFR_MLP_DZ: cols = m->dims[(size_t)layer + 1]; ld = m->pdims[(size_t)layer + 1]; src = m->grads[(size_t)layer]; break;
    case CFR_MLP_OUT: cols = m->dims[(size_t)m->L]; ld = m->pdims[(size_t)m->L]; src = m->yp; bf16 = false; break;
    default: return merr(m, CFR_ERR_INVALID, "which must be CFR_MLP_ACT, CFR_MLP_DZ or CFR_MLP_OUT");
    }
    const int64_t B = m->last_batch;
    if (len < B * cols) return merr(m, CFR_ERR_INVALID, "out needs %lld entries", (long long)(B * cols));
    MDeviceGuard dg(m->device);
    if ((st = check_err(m)) != CFR_OK) return st;
    const size_t esz = bf16 ? sizeof(__nv_bfloat16) : sizeof(float);
    std::vector<unsigned char> host((size_t)(B * ld) * esz);
    MCK(cudaMemcpyAsync(host.data(), src, host.size(), cudaMemcpyDeviceToHost, m->stream));
    MCK(cudaStreamSynchronize(m->stream));
    for (int64_t r = 0; r < B; ++r)
        for (int64_t c = 0; c < cols; ++c) {
            const size_t i = (size_t)(r * ld + c);
            if (bf16) {
                uint16_t h;
                std::memcpy(&h, host.data() + 2 * i, 2);
                const uint32_t w = (uint32_t)h << 16;   // a BF16 value is the top half of an FP32 one
                std::memcpy(&out[r * cols + c], &w, 4);
            } else {
                std::memcpy(&out[r * cols + c], host.data() + 4 * i, 4);
            }
        }
    return CFR_OK;
}

cfr_status cfr_mlp_adam(cfr_mlp *m, float lr, float beta1, float beta2, float eps) {
    cfr_status st = usable(m);
    if (st != CFR_OK) return st;
    if (!(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
        return merr(m, CFR_ERR_INVALID, "need lr >= 0, beta1 and beta2 in [0, 1), eps > 0");
    MDeviceGuard dg(m->device);
    m->steps += 1;
    const float c1 = (float)(1.0 - std::pow((double)beta1, (double)m->steps));
    const float c2 = (float)(1.0 - std::pow((double)beta2, (double)m->steps));
    k_adam<<<grid_for(m->P), 256, 0, m->stream>>>(m->p, m->g, m->m1, m->m2, m->pb, m->P, lr, beta1, beta2, eps, c1, c2);
    MCK(cudaGetLastError());
    MCK(refresh_transposes(m));
    return CFR_OK;
}

cfr_status cfr_mlp_gemm_stats(cfr_mlp *m, double *fwd_us, double *fwd_flops, double *bwd_us, double *bwd_flops) {
    cfr_status st = usable(m);
    if (st != CFR_OK) return st;
    MDeviceGuard dg(m->device);
    if ((st = check_err(m)) != CFR_OK) return st;
    float a = 0.f, b = 0.f;
    if (m->fwd_timed) MCK(cudaEventElapsedTime(&a, m->ev[0], m->ev[1]));
    if (m->bwd_timed) MCK(cudaEventElapsedTime(&b, m->ev[2], m->ev[3]));
    if (fwd_us) *fwd_us = 1e3 * a;
    if (fwd_flops) *fwd_flops = m->fwd_timed ? m->fwd_flops : 0.0;
    if (bwd_us) *bwd_us = 1e3 * b;
    if (bwd_flops) *bwd_flops = m->bwd_timed ? m->bwd_flops : 0.0;
    return CFR_OK;
}

cfr_status cfr_mlp_set_tensor_path(cfr_mlp *m, int32_t path) {
    cfr_status st = usable(m);
    if (st != CFR_OK) return st;
    if (path < 0 || path > 2) return merr(m, CFR_ERR_INVALID, "path must be 0, 1 or 2");
    m->path = path;
    return CFR_OK;
}

cfr_status cfr_mlp_synchronize(cfr_mlp *m) {
    cfr_status st = usable(m);
    if (st != CFR_OK) return st;
    MDeviceGuard dg(m->device);
    return check_err(m);
}

const char *cfr_mlp_last_error(const cfr_mlp *m) { return m ? m->err.c_str() : g_mlp_err.c_str(); }

void cfr_mlp_free(cfr_mlp *m) {
    if (!m) return;
    MDeviceGuard dg(m->device);
    cudaStreamSynchronize(m->stream);
    for (void *a : {(void *)m->p, (void *)m->g, (void *)m->m1, (void *)m->m2, (void *)m->pb, (void *)m->pbt, (void *)m->yp,
                    (void *)m->d_err})
        if (a) cudaFree(a);
    for (auto *v : {&m->acts, &m->grads, &m->acts_t, &m->grads_t})
        for (auto *a : *v) if (a) cudaFree(a);
    for (cudaEvent_t ev : m->ev)
        if (ev) cudaEventDestroy(ev);
    for (cfr_mlp::PassGraph *g : {&m->gfwd, &m->gfwd_train, &m->gbwd})
        if (g->exec) cudaGraphExecDestroy(g->exec);
    if (m->cap_stream) cudaStreamDestroy(m->cap_stream);
    if (m->side) cudaStreamDestroy(m->side);
    for (cudaEvent_t ev : m->fork_ev)
        if (ev) cudaEventDestroy(ev);
    if (m->join_ev) cudaEventDestroy(m->join_ev);
    delete m;
}

}  // extern "C"
