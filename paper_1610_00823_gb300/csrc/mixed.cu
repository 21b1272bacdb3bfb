// Split-BF16 tensor-core near field (VFMM_MIXED), tcgen05 on sm_103a.
//
// The near-field sum of Section 3.1, out[t][r] = sum_{(cfg, s) in U(t)} sum_k T_cfg[r][k] f_s[k],
// is an exact-enough FP64 contraction computed from BF16 tensor-core products:
//
//  * f is normalised by a global power of two (|a| < 1) and each table row r by its own power
//    of two shared by all 33 configurations; each normalised value is written as 8 balanced
//    base-128 digits a = sum_i m_i 2^(-7 i) (integers |m_1| <= 128, |m_i| <= 64 for i >= 2, exact
//    in BF16), of which a contraction takes the first S (6 by default: 42 bits; up to 8).
//  * Products (i, j) with i + j <= S + 1 are kept (the dropped terms are below 2^(-7 S - 7)). Per K
//    value the products of one diagonal d = i + j - 2 sum to at most 2 * 128 * 64 + (d - 1) * 64^2
//    integer units of 2^(-7(d+2)) (28672 for d = 4), so over a drain group of at most 512 K values
//    diagonals 0..4 stay below 2^24 units and the FP32 tensor-core accumulator holds them exactly.
//    Diagonals 0..4 get one TMEM accumulator each; diagonals 5 and up share a sixth, where the
//    tensor core's truncating accumulation of terms much smaller than the running sum (it does not
//    round to nearest) costs about 2^-51 of the result (2^-46 was measured with base-64 digits,
//    whose diagonal 5 weighs 2^5 more).
//  * After every drain group (one or more configurations, at most 512 K values) the epilogue warps
//    drain the six accumulators into a running double-float sum (FP32 pairs, exact two-sums) in
//    registers; at the end of an item they store (hi, lo). The leaf pass scales by
//    2^(E_f + E_r) and by h^2 (potential) or h (gradient) in FP64.
//
// Tile: 128 rows on the M side (TMEM lanes) x 80 on the N side; which side holds the table rows
// (by TMA) and which the gathered operand rows (by cp.async) depends on the contraction
// (near_transposed). For every table of a group and every K block of 32 values the S slices of
// both go into a 64-byte-swizzled K-major stage (two stages); one thread issues the
// S(S+1)/2 x 2 UMMAs (128 x N x 16) into the six TMEM accumulators; tcgen05.commit frees the
// stage and, after the last K block of a drain group, hands the accumulators to the epilogue.
// Every mbarrier wait is bounded and reports a timeout through an error word.
#include <cuda_bf16.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "mixed.cuh"
#include "ops.cuh"
#include "tc_ptx.cuh"
#include "vfmm_internal.cuh"

namespace vfmm {

using bf16 = __nv_bfloat16;

// ---------------------------------------------------------------- slicing
// Operand layout: [row][K block of 32][slice][32 values]; one row's slices of one K block are 512
// contiguous bytes (one warp-wide cp.async). Offset of (row, slice 0, k):
__device__ __forceinline__ size_t slice_off(size_t row, int Kp, int k) {
    return ((row * (Kp / kKBlock) + k / kKBlock) * kSlices) * kKBlock + (k % kKBlock);
}

// E_r[r] = exponent e with max_{cfg,k} |T_cfg[r][k]| < 2^e (0 for all-zero rows).
__global__ void table_row_exp_kernel(const double* __restrict__ T, int R, int kk, int* __restrict__ Er) {
    __shared__ double red[256];
    const int r = blockIdx.x;
    double m = 0.0;
    for (int q = threadIdx.x; q < kNearCfg * kk; q += blockDim.x) {
        int c = q / kk, k = q % kk;
        m = fmax(m, fabs(T[((size_t)c * R + r) * kk + k]));
    }
    red[threadIdx.x] = m;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        int e = 0;
        if (red[0] > 0.0) frexp(red[0], &e);
        Er[r] = e;
    }
}

// tsl[cfg][r][i][k] (rows r >= R and columns k >= kk are zero)
__global__ void table_slice_kernel(const double* __restrict__ T, int R, int kk, int Rp, int Kp,
                                   const int* __restrict__ Er, bf16* __restrict__ tsl) {
    const int cfg = blockIdx.y, r = blockIdx.x;
    for (int k = threadIdx.x; k < Kp; k += blockDim.x) {
        double v = (r < R && k < kk) ? T[((size_t)cfg * R + r) * kk + k] : 0.0;
        slice_fixed(v, r < R ? Er[r] : 0, tsl + slice_off((size_t)cfg * Rp + r, Kp, k), kKBlock);
    }
}

// out[r] = max |f| of right-hand side r (bits of the double; grid.y = r). Warp and CTA maxima first,
// then one atomic per CTA (the atomics on one address serialise in L2).
__global__ void __launch_bounds__(256) fmax_abs_kernel(const double* __restrict__ f, int64_t n,
                                                       unsigned long long* __restrict__ out) {
    __shared__ double red[8];
    const double* fr = f + (size_t)blockIdx.y * n;
    double m = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, fabs(fr[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
        atomicMax(out + blockIdx.y, (unsigned long long)__double_as_longlong(m));
    }
}

// fsl[leaf * R + r][i][k] from f_r[leaf][k] / 2^E_f[r]; also stores E_f[r]. One thread per 8
// consecutive values of a row (one 16-byte store per slice).
__global__ void f_slice_kernel(const double* __restrict__ f, int nleaf, int kk, int Kp, int R,
                               const unsigned long long* __restrict__ fmax_bits, int* __restrict__ Ef,
                               bf16* __restrict__ fsl) {
    const unsigned cpr = (unsigned)Kp / 8;  // chunks per row
    const unsigned g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (unsigned)nleaf * (unsigned)R * cpr) return;
    const unsigned row = g / cpr, c = g - row * cpr;
    const unsigned leaf = row / (unsigned)R, r = row - leaf * (unsigned)R;
    const int e = exp_bound(__longlong_as_double((long long)fmax_bits[r]));
    const double* fr = f + ((size_t)r * nleaf + leaf) * kk;
    double v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int k = 8 * (int)c + j;
        v[j] = k < kk ? fr[k] : 0.0;
    }
    slice8_fixed(v, e, fsl + slice_off(row, Kp, 8 * (int)c), kKBlock);
    if (leaf == 0 && c == 0) Ef[r] = e;
}

// ---------------------------------------------------------------- the tcgen05 kernel
// Barrier among `count` threads (a multiple of 32) that use the same id; id 0 is __syncthreads.
__device__ __forceinline__ void named_bar_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}


struct SplitArgs {
    const bf16* asl;      // A rows [rows][Kp / 32][kSlices][32]; the tables come through the tensor map
    const int32_t* gptr;  // [n_groups + 1] into gcfg
    const int32_t* gcfg;  // table of each (group, table) entry
    const int32_t* gsrc;  // [entries][128] A row or -1
    const int32_t* gtgt;  // [n_groups][128] output row or -1
    float2* out;          // [n_out_rows][Rp], or partial sums [split][n_out_rows][Rp] when split > 1
    int* err;
    int Kp, Rp, nchunks;
    int split;            // CTAs sharing one group's tables (split-K over tables)
    int drain_every;      // configurations accumulated in TMEM between two drains (exactness bound)
    int transposed;       // table rows on the M side (see near_transposed)
    int slices;           // slices of each operand taken, kMinSlices .. kSlices (products i + j <= slices + 1)
    int n_items;          // work items (n_groups * split * nchunks); the grid may be smaller (persistent CTAs)
    size_t part_stride;   // n_out_rows * Rp
};

// Accumulator of slice product (i, j): its diagonal i + j - 2; diagonals >= kNumAcc - 1 share the last.
__host__ __device__ constexpr int acc_of(int i, int j) { return (i + j - 2) < (kNumAcc - 1) ? (i + j - 2) : (kNumAcc - 1); }

// All slice products (i, j), i + j <= S + 1, of one K block: accumulator acc_of(i, j); on the
// first K block of a configuration the first product into each accumulator overwrites it (with
// S >= kMinSlices every accumulator gets a product).
template <bool kFirst, int S, int N>
__device__ __forceinline__ void issue_unit(uint32_t tmem, uint64_t ad0, uint64_t bd0) {
    constexpr uint32_t idesc = tc::idesc_bf16_f32(kTileM, N);
    constexpr uint32_t A_SLICE = kTileM * 64, B_SLICE = N * 64;
    static_assert(S >= kMinSlices && S <= kSlices, "slice count");
#pragma unroll
    for (int i = 1; i <= S; ++i)
#pragma unroll
        for (int j = 1; j <= S; ++j) {
            if (i + j > S + 1) continue;
            const int acc = acc_of(i, j);
            // first product of accumulator acc in (i, j) order: i == 1 for acc < kNumAcc - 1, else (1, kNumAcc)
            const bool first_of_acc = (acc < kNumAcc - 1) ? (i == 1) : (i == 1 && j == kNumAcc);
#pragma unroll
            for (int ks = 0; ks < kKBlock / 16; ++ks) {
                const uint64_t ad = ad0 + (((i - 1) * A_SLICE + ks * 32) >> 4);
                const uint64_t bd = bd0 + (((j - 1) * B_SLICE + ks * 32) >> 4);
                const uint32_t accum = (kFirst && first_of_acc && ks == 0) ? 0u : 1u;
                tc::umma_bf16(tmem + acc * N, ad, bd, idesc, accum);
            }
        }
}

// Warps 0..7: epilogue (lane quadrant w % 4, column half w / 4); warps 8..10: producers;
// warp 11: TMEM allocation and the MMA issuer (lane 0). Twelve warps keep three warps per SM
// sub-partition, which leaves each thread up to 168 registers.
// N: the MMA's N (TMEM columns per accumulator): 80, or 48 for the 48-row tables of small
// expansions (targets on M only).
template <int N>
__global__ void __launch_bounds__(kThreads, 1) split_gemm_kernel(SplitArgs a, const __grid_constant__ CUtensorMap tmB) {
    extern __shared__ unsigned char dsm[];
    __shared__ __align__(8) uint64_t bars[2 * kStages + 3];
    __shared__ uint32_t tmem_holder;
    __shared__ volatile int abort_flag;
    __shared__ int32_t s_src[kTileM];
    __shared__ volatile int p_abort;  // written by producers only, read after a producer barrier
    static_assert(N % 16 == 0 && (N / 2) % 8 == 0 && kNumAcc * N <= kTmemCols, "tile N");
    constexpr uint32_t A_SLICE = kTileM * 64;
    constexpr uint32_t B_SLICE = N * 64;
    constexpr uint32_t STAGE = kSlices * (A_SLICE + B_SLICE);
    constexpr int HALF = N / 2;  // columns per epilogue warp
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool tr = a.transposed != 0;     // table rows on M (TMA into the A region), targets on N
    const int G = tr ? kTileN : kTileM;    // gathered rows (targets) per group
    const uint32_t base = tc::smem_u32(dsm);
    const uint32_t sbase = (base + 1023u) & ~1023u;
    const uint32_t full0 = tc::smem_u32(&bars[0]);
    const uint32_t empty0 = tc::smem_u32(&bars[kStages]);
    const uint32_t acc_full = tc::smem_u32(&bars[2 * kStages]);
    const uint32_t acc_empty = tc::smem_u32(&bars[2 * kStages + 1]);
    const uint32_t mma_done = tc::smem_u32(&bars[2 * kStages + 2]);  // used only after an abort
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            tc::mbar_init(full0 + 8 * s, kProducerThreads + 1);  // cp.async producers + the TMA issuer
            tc::mbar_init(empty0 + 8 * s, 1);
        }
        tc::mbar_init(acc_full, 1);
        tc::mbar_init(acc_empty, kEpilogueThreads);
        tc::mbar_init(mma_done, 1);
        abort_flag = 0;
        p_abort = 0;
        tc::mbar_fence_init();
    }
    if (warp == kMmaWarp) {
        tc::tmem_alloc(tc::smem_u32(&tmem_holder), kTmemCols);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tmem_holder;
    // Work items (group g, split share sp, row chunk rc), item = (g * split + sp) * nchunks + rc; this
    // CTA takes items blockIdx.x, blockIdx.x + gridDim.x, ... (one item per CTA unless the launch
    // caps the grid). Within an item, units = (table, K block) pairs of the group in table order;
    // share sp of the split takes a contiguous range of them, which may begin or end inside a table
    // (split-K over tables and K blocks). The stage ring and the accumulator hand-offs run on
    // CTA-wide counters (gu: units, dg: drain groups), so one item's loads start while the previous
    // item's accumulators drain.
    const int n_items = a.n_items;
    const int nkb = a.Kp / kKBlock;
    const int DU = a.drain_every * nkb;  // units summed in TMEM between two drains
    struct Item {
        int g, sp, rc, gbeg, ubeg, U;
    };
    auto item = [&](int it) {
        Item x;
        const int qq = it / a.nchunks;
        x.rc = it - qq * a.nchunks;
        x.g = qq / a.split;
        x.sp = qq - x.g * a.split;
        x.gbeg = a.gptr[x.g];
        const long long Ug = (long long)(a.gptr[x.g + 1] - x.gbeg) * nkb;
        x.ubeg = (int)((Ug * x.sp) / a.split);
        x.U = (int)((Ug * (x.sp + 1)) / a.split) - x.ubeg;
        return x;
    };
    int issued = 0;  // producers: units (CTA-wide count) whose copies were started

    if (warp >= kEpilogueWarps && warp < kMmaWarp) {
        // ------------------------------------------------ producers: table tile by TMA (one thread),
        // gathered source rows by cp.async (all producer threads)
        const int ptid = tid - kEpilogueThreads;
        if (ptid == 0) tc::tma_prefetch_desc(&tmB);
        int gu = 0;
        for (int it = blockIdx.x; it < n_items && !p_abort; it += gridDim.x) {
            const Item x = item(it);
            const int r0 = x.rc * (tr ? kTileM : N);  // first table row of this item's tile
            for (int u = 0; u < x.U; ++u, ++gu) {
                const int s = gu & 1;
                if (gu >= 2 && !tc::mbar_wait(empty0 + 8 * s, ((gu >> 1) - 1) & 1, &abort_flag)) p_abort = 1;
                // every producer passes this barrier once per unit, so the exit decision below is uniform
                // and nobody rewrites s_src while another producer still reads it
                named_bar_sync(1, kProducerThreads);
                if (p_abort) {
                    abort_flag = 1;
                    atomicExch(a.err, 1);
                    break;
                }
                const int ci = x.gbeg + (x.ubeg + u) / nkb, kb = (x.ubeg + u) % nkb;
                const int cfg = a.gcfg[ci];
                if (kb == 0 || u == 0) {
                    // gather rows of this table for the group's targets, once per table
                    for (int m = ptid; m < G; m += kProducerThreads) s_src[m] = a.gsrc[(size_t)ci * G + m];
                    named_bar_sync(1, kProducerThreads);
                }
                const uint32_t sA = sbase + s * STAGE, sB = sA + kSlices * A_SLICE;
                // table tile by TMA into the region of its side, gathered rows into the other
                const uint32_t sT = tr ? sA : sB, sG = tr ? sB : sA;
                const uint32_t T_SLICE = tr ? A_SLICE : B_SLICE, G_SLICE = tr ? B_SLICE : A_SLICE;
                if (ptid == 0) {
                    // boxes of (128 or 80) table rows x 64 bytes (one per slice), SW64-swizzled by TMA
                    tc::mbar_arrive_expect_tx(full0 + 8 * s, a.slices * T_SLICE);
                    for (int sl_i = 0; sl_i < a.slices; ++sl_i)
                        tc::tma_load_3d(sT + sl_i * T_SLICE, &tmB, 0, kb * kSlices + sl_i, cfg * a.Rp + r0,
                                        full0 + 8 * s);
                }
                // a warp instruction covers 8 rows x 64 bytes of one slice: 512 contiguous bytes of
                // shared memory (no bank conflicts) from eight 64-byte pieces of global memory
                const int lrow = (ptid & 31) >> 2, ch = ptid & 3, pw = ptid >> 5;
#pragma unroll 4
                for (int q = pw; q < a.slices * (G / 8); q += kProducerThreads / 32) {
                    const int sl_i = q / (G / 8), m = (q % (G / 8)) * 8 + lrow;
                    const int src = s_src[m];
                    const bf16* gp =
                        a.asl + (((size_t)(src < 0 ? 0 : src) * nkb + kb) * kSlices + sl_i) * kKBlock + ch * 8;
                    const uint32_t dst = sG + sl_i * G_SLICE + m * 64 + ((ch ^ ((m >> 1) & 3)) << 4);
                    tc::cp_async16(dst, gp, src < 0 ? 0u : 16u);
                }
                // the stage's full barrier gets this thread's arrival when its copies have landed
                tc::cp_async_mbar_arrive(full0 + 8 * s);
                issued = gu + 1;
            }
        }
        tc::cp_async_wait_all();
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------ MMA issuer: one unit at a time
        if (lane == 0) {
            const uint64_t adesc_base = tc::smem_desc(sbase, 16, 512, tc::kLayoutSwizzle64B);
            int gu = 0, dg = 0;  // units and drain groups of this CTA so far
            bool stop = false;
            for (int it = blockIdx.x; it < n_items && !stop; it += gridDim.x) {
                const Item x = item(it);
                for (int u = 0; u < x.U; ++u, ++gu) {
                    // a drain group = DU consecutive units of an item summed in the same accumulators;
                    // before one starts, the epilogue must have drained the previous one
                    if (u % DU == 0 && dg > 0 && !tc::mbar_wait(acc_empty, (dg - 1) & 1, &abort_flag)) {
                        abort_flag = 1;
                        atomicExch(a.err, 4);
                        stop = true;
                        break;
                    }
                    const int s = gu & 1;
                    if (!tc::mbar_wait(full0 + 8 * s, (gu >> 1) & 1, &abort_flag)) {
                        abort_flag = 1;
                        atomicExch(a.err, 2);
                        stop = true;
                        break;
                    }
                    tc::tc_fence_after();
                    // the gathered rows were written by cp.async (generic proxy): make them visible to
                    // the tensor core's reads (async proxy) before the MMAs
                    tc::fence_proxy_async();
                    // descriptors differ only in the 14-bit start-address field (address >> 4), so
                    // offsets within the stage are added to a base descriptor
                    const uint64_t ad0 = adesc_base + ((s * STAGE) >> 4);
                    const uint64_t bd0 = adesc_base + ((s * STAGE + kSlices * A_SLICE) >> 4);
                    const bool first = u % DU == 0;
                    switch (a.slices) {
                        case 6: first ? issue_unit<true, 6, N>(tmem, ad0, bd0) : issue_unit<false, 6, N>(tmem, ad0, bd0); break;
                        case 7: first ? issue_unit<true, 7, N>(tmem, ad0, bd0) : issue_unit<false, 7, N>(tmem, ad0, bd0); break;
                        default: first ? issue_unit<true, 8, N>(tmem, ad0, bd0) : issue_unit<false, 8, N>(tmem, ad0, bd0); break;
                    }
                    tc::umma_commit(empty0 + 8 * s);
                    if (u % DU == DU - 1 || u == x.U - 1) {
                        tc::umma_commit(acc_full);
                        ++dg;
                    }
                }
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------ epilogue: drain each drain group, write each item
        const int quad = warp & 3, half = warp >> 2;
        const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16) + half * HALF;
        bool ok = true;
        int dg = 0;
        for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
            const Item x = item(it);
            float hi[HALF], lo[HALF];
#pragma unroll
            for (int j = 0; j < HALF; ++j) hi[j] = lo[j] = 0.0f;
            const int ngroups = (x.U + DU - 1) / DU;
            for (int grp = 0; grp < ngroups; ++grp, ++dg) {
                ok = ok && tc::mbar_wait(acc_full, dg & 1, &abort_flag);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) {
                    if (lane == 0) atomicExch(a.err, 3);
                    abort_flag = 1;
                    break;
                }
                tc::tc_fence_after();
                // per 8-column chunk: the 6 accumulators loaded together, one wait, then summed in
                // accumulator order into the double-FP32 (hi, lo) pairs
#pragma unroll
                for (int ch = 0; ch < HALF / 8; ++ch) {
                    uint32_t r[kNumAcc][8];
#pragma unroll
                    for (int acc = 0; acc < kNumAcc; ++acc) tc::tmem_ld8_nowait(lane_base + acc * N + ch * 8, r[acc]);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int acc = 0; acc < kNumAcc; ++acc)
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            float s2, e2;
                            two_sum(hi[ch * 8 + j], __uint_as_float(r[acc][j]), s2, e2);
                            hi[ch * 8 + j] = s2;
                            lo[ch * 8 + j] = __fadd_rn(lo[ch * 8 + j], e2);
                        }
                }
                tc::tc_fence_before();
                tc::mbar_arrive(acc_empty);
            }
            if (!ok) break;
            float2* outp = a.split > 1 ? a.out + (size_t)x.sp * a.part_stride : a.out;
            const int m = quad * 32 + lane;  // TMEM lane
            const int r0 = x.rc * (tr ? kTileM : N);
            if (tr) {
                // lane = table row r0 + m, columns = targets half * HALF + j of the group
                const int row = r0 + m;
#pragma unroll
                for (int j = 0; j < HALF; ++j) {
                    const int tgt = a.gtgt[(size_t)x.g * G + half * HALF + j];
                    if (tgt < 0) continue;
                    const float h = __fadd_rn(hi[j], lo[j]);
                    const float l = __fsub_rn(lo[j], __fsub_rn(h, hi[j]));
                    outp[(size_t)tgt * a.Rp + row] = make_float2(h, l);
                }
            } else {
                // lane = target m of the group, columns = table rows r0 + half * HALF + j
                const int tgt = a.gtgt[(size_t)x.g * G + m];
                if (tgt >= 0) {
                    float4* o = reinterpret_cast<float4*>(outp + (size_t)tgt * a.Rp + r0 + half * HALF);
#pragma unroll
                    for (int j = 0; j < HALF / 2; ++j) {
                        float h0 = __fadd_rn(hi[2 * j], lo[2 * j]);
                        float l0 = __fsub_rn(lo[2 * j], __fsub_rn(h0, hi[2 * j]));
                        float h1 = __fadd_rn(hi[2 * j + 1], lo[2 * j + 1]);
                        float l1 = __fsub_rn(lo[2 * j + 1], __fsub_rn(h1, hi[2 * j + 1]));
                        o[j] = make_float4(h0, l0, h1, l1);
                    }
                }
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (abort_flag) {
        // after an abort (a bounded wait ran out somewhere): wait, with a longer bound, for the work
        // still in flight, so that no copy writes this CTA's shared memory and no MMA its
        // accumulators once they are released. Units may have been started that no MMA consumed
        // (their table tiles come by TMA; the cp.async rows are complete after cp.async.wait_all),
        // and MMAs issued before the abort may still run.
        const volatile int never = 0;
        if (tid == kEpilogueThreads)
            for (int u = issued - 2; u < issued; ++u)
                if (u >= 0) tc::mbar_wait(full0 + 8 * (u & 1), (u >> 1) & 1, &never, 1ll << 27);
        if (warp == kMmaWarp && lane == 0) {
            tc::umma_commit(mma_done);
            tc::mbar_wait(mma_done, 0, &never, 1ll << 27);
        }
        __syncthreads();
    }
    if (warp == kMmaWarp) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, kTmemCols);
    }
}

// ---------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int make_table_map(const void* base, int64_t rows, int Kp, int box_rows, CUtensorMap* out) {
    static EncodeTiledFn encode = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            encode = (EncodeTiledFn)fn;
    });
    if (!encode) return fail(VFMM_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    if (Kp % kKBlock || rows < box_rows || rows > (int64_t)INT32_MAX || ((uintptr_t)base & 15) || box_rows < 1 ||
        box_rows > 256)
        return fail(VFMM_ERR_INTERNAL, "table shape not suitable for a tensor map");
    // [rows][Kp / 32 K blocks][8 slices][32 values]: dim 0 = 32 values (64 bytes, one swizzle row),
    // dim 1 = (K block, slice) segments, dim 2 = rows
    const cuuint64_t nseg = (cuuint64_t)(Kp / kKBlock) * kSlices;
    const cuuint64_t dims[3] = {(cuuint64_t)kKBlock, nseg, (cuuint64_t)rows};
    const cuuint64_t strides[2] = {(cuuint64_t)kKBlock * 2, nseg * kKBlock * 2};
    const cuuint32_t box[3] = {(cuuint32_t)kKBlock, 1, (cuuint32_t)box_rows};
    const cuuint32_t es[3] = {1, 1, 1};
    CUresult r = encode(out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(VFMM_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return VFMM_OK;
}

int mixed_prepare(vfmm_ops* o, cudaStream_t st) {
    if (o->k * o->k * 3 > 4096) return fail(VFMM_ERR_INVALID_ARG, "mixed precision supports k <= 16");
    MixedOps* mo = new MixedOps();
    o->mixed = mo;
    const int kk = o->k * o->k;
    const int R = 3 * kk;
    mo->N = kTileN;
    const int tile_rows = table_rows_per_tile(near_transposed(o->k));
    mo->Rp = (R + tile_rows - 1) / tile_rows * tile_rows;
    mo->Kp = (kk + kKBlock - 1) / kKBlock * kKBlock;
    VFMM_CUDA(cudaMalloc(&mo->Er, mo->Rp * sizeof(int)));
    VFMM_CUDA(cudaMemsetAsync(mo->Er, 0, mo->Rp * sizeof(int), st));
    VFMM_CUDA(cudaMalloc(&mo->tsl, (size_t)kNearCfg * mo->Rp * kSlices * mo->Kp * sizeof(bf16)));
    table_row_exp_kernel<<<R, 256, 0, st>>>(o->near, R, kk, mo->Er);
    table_slice_kernel<<<dim3(mo->Rp, kNearCfg), 128, 0, st>>>(o->near, R, kk, mo->Rp, mo->Kp, mo->Er, (bf16*)mo->tsl);
    VFMM_CUDA(cudaGetLastError());
    VFMM_CUDA(cudaStreamSynchronize(st));
    VFMM_CHECK(make_table_map(mo->tsl, (int64_t)kNearCfg * mo->Rp, mo->Kp, tile_rows, &mo->tm_near));
    return far_prepare(o, st);
}

void mixed_free(vfmm_ops* o) {
    MixedOps* mo = (MixedOps*)o->mixed;
    if (!mo) return;
    far_free(mo);
    if (mo->tsl) cudaFree(mo->tsl);
    if (mo->Er) cudaFree(mo->Er);
    delete mo;
    o->mixed = nullptr;
}

int build_split_plan(const PlanItems& I, const std::vector<int32_t>& order, int n_tables, int n_chunks, int R,
                     bool transposed, int nkb, PlanArena& A, SplitPlan* P) {
    const int G = transposed ? kTileN : kTileM;  // targets per group
    // target t stands for the R consecutive virtual targets t * R + r, whose gathered rows are
    // src * R + r: the right-hand sides of one target share its set of tables
    const int nt0 = (int)I.tgt.size();
    const int64_t nt = (int64_t)nt0 * R;
    if (nt > (int64_t)INT32_MAX / 2) return fail(VFMM_ERR_INVALID_ARG, "too many rows for one split contraction");
    const int ng = (int)((nt + G - 1) / G);
    std::vector<int32_t> gtgt((size_t)std::max(ng, 1) * G, -1), gptr(ng + 1, 0), gcfg, gsrc;
    std::vector<int32_t> slot(n_tables, -1);
    std::vector<char> present(n_tables, 0);
    for (int g = 0; g < ng; ++g) {
        std::fill(present.begin(), present.end(), 0);
        const int m_end = (int)std::min<int64_t>(G, nt - (int64_t)g * G);
        for (int m = 0; m < m_end; ++m) {
            const int64_t v = (int64_t)g * G + m;
            const int t = order[v / R], r = (int)(v % R);
            gtgt[(size_t)g * G + m] = I.tgt[t] * R + r;
            for (int e = I.ptr[t]; e < I.ptr[t + 1]; ++e) present[I.tab[e]] = 1;
        }
        for (int c = 0; c < n_tables; ++c) {
            if (!present[c]) continue;
            slot[c] = (int32_t)gcfg.size();
            gcfg.push_back(c);
        }
        gsrc.resize(gcfg.size() * G, -1);
        for (int m = 0; m < m_end; ++m) {
            const int64_t v = (int64_t)g * G + m;
            const int t = order[v / R], r = (int)(v % R);
            for (int e = I.ptr[t]; e < I.ptr[t + 1]; ++e) gsrc[(size_t)slot[I.tab[e]] * G + m] = I.src[e] * R + r;
        }
        gptr[g + 1] = (int32_t)gcfg.size();
    }
    P->n_groups = ng;
    P->entries = (int64_t)gcfg.size();
    P->transposed = transposed;
    P->group = G;
    {
        int dev = 0, sms = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int64_t ctas = (int64_t)std::max(ng, 1) * n_chunks;
        // units of work per group: (table, K block) pairs
        const double avg_units = ng ? (double)P->entries * nkb / ng : 1.0;
        // split-K over the units only for small contractions (fewer than two CTAs per SM): default =
        // the split minimising (CTAs / SMs, at least 1) x (units per CTA + about one table of fixed
        // cost); vfmm_tune replaces it by timing
        int split = 1;
        P->may_split = ctas < 2 * sms && avg_units >= 2.0;
        if (P->may_split) {
            double best = 1e300;
            for (int sp = 1; sp <= kMaxSplit && sp <= std::max(1.0, avg_units); sp *= 2) {
                const double waves = std::max(1.0, (double)(ctas * sp) / sms);
                const double est = waves * (avg_units / sp + nkb);
                if (est < best - 1e-9) {
                    best = est;
                    split = sp;
                }
            }
        }
        P->split = split;
    }
    P->off[0] = A.put(gtgt);
    P->off[1] = A.put(gptr);
    P->off[2] = A.put(gcfg);
    P->off[3] = A.put(gsrc);
    return VFMM_OK;
}

int commit_plan_arena(PlanArena& A, PlanSet* PS, cudaStream_t st) {
    void* base = nullptr;
    VFMM_CHECK(tree_malloc(&base, A.data.size() * sizeof(int32_t), st));
    PS->arena = base;
    if (!A.data.empty())
        VFMM_CUDA(cudaMemcpyAsync(base, A.data.data(), A.data.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    VFMM_CUDA(cudaStreamSynchronize(st));
    int32_t* b = static_cast<int32_t*>(base);
    for (SplitPlan* top : {&PS->near, &PS->s2m, &PS->m2l, &PS->far, &PS->s2l})
        for (SplitPlan* P = top; P; P = P->alt) {
            int32_t** field[6] = {&P->tgt, &P->ptr, &P->cfg, &P->src, &P->seg, &P->seg_out};
            for (int i = 0; i < 6; ++i) *field[i] = P->off[i] >= 0 ? b + P->off[i] : nullptr;
        }
    return VFMM_OK;
}

// Targets in the order of their keys.
static std::vector<int32_t> key_order(const PlanItems& I) {
    std::vector<int32_t> order(I.tgt.size());
    for (size_t t = 0; t < order.size(); ++t) order[t] = (int32_t)t;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return I.key[x] < I.key[y]; });
    return order;
}

int build_contraction_plan(const PlanItems& I, int n_tables, int n_chunks, int R, bool transposed, int nkb,
                           double slab_overhead, size_t slab_row_bytes, PlanArena& A, SplitPlan* P) {
    constexpr size_t kMaxSlabBytes = size_t(256) << 20;
    VFMM_CHECK(build_split_plan(I, key_order(I), n_tables, n_chunks, R, transposed, nkb, A, P));
    const int nt = (int)I.tgt.size();
    const int64_t G = P->group;
    const int64_t n_entries = (int64_t)I.tab.size();
    std::vector<int64_t> per_table(n_tables + 1, 0);
    for (int64_t e = 0; e < n_entries; ++e) ++per_table[I.tab[e] + 1];
    int64_t entry_cols = 0;
    for (int c = 0; c < n_tables; ++c) entry_cols += (per_table[c + 1] * R + G - 1) / G * G;
    const double grouped_cols = (double)P->entries * G;
    const size_t slab_bytes = (size_t)n_entries * R * slab_row_bytes;
    if (n_entries == 0 || slab_bytes > kMaxSlabBytes || (double)n_entries * R > (double)INT32_MAX / 2)
        return VFMM_OK;
    const bool prefer_entry = (double)entry_cols * (1.0 + slab_overhead) < 0.85 * grouped_cols;
    if (!prefer_entry && !P->may_split) return VFMM_OK;  // large grouped contraction: no alternative
    // entry q (targets in order, their items in order): a target of its own with the one item, in
    // the order of (table, q) (a counting sort by table)
    PlanItems E;
    E.tgt.resize(n_entries);
    E.ptr.resize(n_entries + 1);
    E.tab = I.tab;
    E.src = I.src;
    for (int64_t q = 0; q <= n_entries; ++q) {
        if (q < n_entries) E.tgt[q] = (int32_t)q;
        E.ptr[q] = (int32_t)q;
    }
    for (int c = 0; c < n_tables; ++c) per_table[c + 1] += per_table[c];
    std::vector<int32_t> e_order(n_entries);
    for (int64_t q = 0; q < n_entries; ++q) e_order[per_table[I.tab[q]]++] = (int32_t)q;
    std::vector<int32_t> seg(nt + 1), seg_out(nt);
    for (int t = 0; t < nt; ++t) {
        seg[t] = I.ptr[t];
        seg_out[t] = I.tgt[t];
    }
    seg[nt] = (int32_t)n_entries;
    SplitPlan* E_plan = new SplitPlan();
    int rc = build_split_plan(E, e_order, n_tables, n_chunks, R, transposed, nkb, A, E_plan);
    if (rc == VFMM_OK) {
        E_plan->entry = true;  // the slab occupies the partial-sum buffer: no split-K
        E_plan->may_split = false;
        E_plan->split = 1;
        E_plan->R = R;
        E_plan->n_seg = nt;
        E_plan->slab_rows = n_entries * R;
        E_plan->off[4] = A.put(seg);
        E_plan->off[5] = A.put(seg_out);
    }
    SplitPlan* E_ = E_plan;
    if (rc != VFMM_OK) {
        free_split_plan(E_);
        delete E_;
        return rc;
    }
    if (prefer_entry) {
        // the entry-major form runs; the grouped one stays as the alternative
        SplitPlan* Gp = new SplitPlan(*P);
        *P = *E_;
        *E_ = SplitPlan();
        delete E_;
        P->alt = Gp;
    } else {
        P->alt = E_;
    }
    return VFMM_OK;
}

// The index arrays live in the plan set's arena: a plan owns only its alternative form.
void free_split_plan(SplitPlan* P) {
    if (P->alt) {
        free_split_plan(P->alt);
        delete P->alt;
        P->alt = nullptr;
    }
    *P = SplitPlan();
}

void free_plan_set(PlanSet* ps) {
    free_split_plan(&ps->near);
    free_split_plan(&ps->s2m);
    free_split_plan(&ps->m2l);
    free_split_plan(&ps->far);
    free_split_plan(&ps->s2l);
    tree_free(ps->arena);
    ps->arena = nullptr;
}

static size_t smem_bytes(int N) { return (size_t)kStages * kSlices * (kTileM * 64 + N * 64) + 1024; }

template <int N>
static int launch_split(const SplitArgs& a, const CUtensorMap& bmap, int grid, cudaStream_t st) {
    static thread_local int attr_dev = -1;  // the attribute is per device
    int dev = 0;
    VFMM_CUDA(cudaGetDevice(&dev));
    if (attr_dev != dev) {
        VFMM_CUDA(cudaFuncSetAttribute(split_gemm_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_bytes(N)));
        attr_dev = dev;
    }
    split_gemm_kernel<N><<<(unsigned)grid, kThreads, smem_bytes(N), st>>>(a, bmap);
    VFMM_CUDA(cudaGetLastError());
    return VFMM_OK;
}

static int launch_split_n(int n, const SplitArgs& a, const CUtensorMap& bmap, int grid, cudaStream_t st) {
    return n == kTileNSmall ? launch_split<kTileNSmall>(a, bmap, grid, st) : launch_split<kTileN>(a, bmap, grid, st);
}


// Entry-major contraction: output row of target t (right-hand side r) = sum of the slab rows of
// its entries, in entry order (double-float); one thread per (target, r, row).
__global__ void segment_reduce_kernel(const float2* __restrict__ slab, const int32_t* __restrict__ seg,
                                      const int32_t* __restrict__ seg_out, int n_seg, int R, int Rp,
                                      float2* __restrict__ out) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)n_seg * R * Rp) return;
    const int row = (int)(q % Rp);
    const int64_t vt = q / Rp;
    const int t = (int)(vt / R), r = (int)(vt % R);
    float hi = 0.0f, lo = 0.0f;
    for (int e = seg[t]; e < seg[t + 1]; ++e) df_add(hi, lo, slab[((size_t)e * R + r) * Rp + row]);
    out[((size_t)seg_out[t] * R + r) * Rp + row] = df_final(hi, lo);
}

// out[row][r] = sum over the partial sums (double-float, exact two-sums).
__global__ void split_reduce_kernel(const float2* __restrict__ part, size_t stride, int split, const int32_t* __restrict__ tgt,
                                    int n_tgt, int Rp, float2* __restrict__ out) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)n_tgt * Rp) return;
    const int t = tgt[q / Rp];
    if (t < 0) return;
    const size_t o = (size_t)t * Rp + q % Rp;
    float hi = 0.0f, lo = 0.0f;
    for (int s = 0; s < split; ++s) df_add(hi, lo, part[(size_t)s * stride + o]);
    out[o] = df_final(hi, lo);
}

int split_gemm(const SplitPlan& P, const void* asl, const CUtensorMap& bmap, int Kp, int Rp, float2* out, int* err,
               float2* part, size_t n_out_rows, int slices, cudaStream_t st, cudaEvent_t* ev, int defer) {
    if (slices < kMinSlices || slices > kSlices) return fail(VFMM_ERR_INTERNAL, "slice count out of range");
    if (ev) VFMM_CUDA(cudaEventRecord(ev[0], st));
    if (P.n_groups == 0) {
        if (ev) VFMM_CUDA(cudaEventRecord(ev[1], st));
        return VFMM_OK;
    }
    const int tile_rows = table_rows_per_tile(P.transposed, Rp);
    if (Kp % kKBlock || Rp % tile_rows) return fail(VFMM_ERR_INTERNAL, "split GEMM shape not tiled");
    const int n_mma = mma_n(P.transposed, Rp);
    SplitArgs a;
    a.asl = (const bf16*)asl;
    a.gptr = P.ptr;
    a.gcfg = P.cfg;
    a.gsrc = P.src;
    a.gtgt = P.tgt;
    a.err = err;
    a.Kp = Kp;
    a.Rp = Rp;
    a.nchunks = Rp / tile_rows;
    a.transposed = P.transposed ? 1 : 0;
    a.slices = slices;
    // Per K value the slice products of an exact diagonal (d <= 4) sum to at most
    // 2 * 128 * 64 + 3 * 64^2 = 28672 units (balanced digits), so those accumulators stay exact while
    // 28672 * Kp * configurations < 2^24. The shared accumulator of diagonals 5 and up truncates as
    // it grows, so a drain group also holds at most 512 K values.
    a.drain_every = std::max(1, std::min((int)((1 << 24) / (28672ll * Kp)), 512 / Kp));
    if (P.entry) {
        // one slab row per entry in the partial-sum buffer, then the per-target sums
        if (!part) return fail(VFMM_ERR_INTERNAL, "entry-major contraction without a slab buffer");
        a.split = 1;
        a.part_stride = 0;
        a.out = part;
        a.n_items = P.n_groups * a.nchunks;
        VFMM_CHECK(launch_split_n(n_mma, a, bmap, P.ctas > 0 ? std::min(P.ctas, a.n_items) : a.n_items, st));
        // deferred: the consumer sums each target's slab rows itself (same order)
        const int64_t n = (defer & kDeferSegments) ? 0 : (int64_t)P.n_seg * P.R * Rp;
        if (n > 0)
            segment_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(part, P.seg, P.seg_out, P.n_seg, P.R,
                                                                                Rp, out);
        VFMM_CUDA(cudaGetLastError());
        if (ev) VFMM_CUDA(cudaEventRecord(ev[1], st));
        return VFMM_OK;
    }
    a.split = part ? P.split : 1;
    a.part_stride = n_out_rows * (size_t)Rp;
    a.out = a.split > 1 ? part : out;
    a.n_items = P.n_groups * a.split * a.nchunks;
    VFMM_CHECK(launch_split_n(n_mma, a, bmap, P.ctas > 0 ? std::min(P.ctas, a.n_items) : a.n_items, st));
    if (a.split > 1 && !(defer & kDeferSplits)) {
        const int64_t n = (int64_t)P.n_groups * P.group * Rp;
        split_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(part, a.part_stride, a.split, P.tgt,
                                                                          P.n_groups * P.group, Rp, out);
        VFMM_CUDA(cudaGetLastError());
    }
    if (ev) VFMM_CUDA(cudaEventRecord(ev[1], st));
    return VFMM_OK;
}

// Near field: targets are leaves; tables are the 33 configurations; A rows are leaves.
// The near-field plan (U list: leaves as targets, 33 configurations, gathered row = source leaf).
static int build_near_plan(const DeviceTree& T, int R, const HostLists& H, PlanArena& A, PlanSet* PS) {
    const int nl = T.n_leaves;
    const std::vector<int32_t>& ptr = H.ptr[VFMM_LIST_U];
    const std::vector<int32_t>& idx = H.idx[VFMM_LIST_U];
    const std::vector<int32_t>& cfg = H.cfg[VFMM_LIST_U];
    const std::vector<int32_t>& bol = H.bol;
    const std::vector<int32_t>& lob = H.lob;
    PlanItems I;
    I.tab.reserve(idx.size());
    I.src.reserve(idx.size());
    for (int t = 0; t < nl; ++t) {
        const int b = bol[t];
        uint64_t sig = 0;
        for (int e = ptr[b]; e < ptr[b + 1]; ++e) {
            I.add(cfg[e], lob[idx[e]]);
            sig |= 1ull << cfg[e];
        }
        I.close(t, sig, (uint64_t)t);
    }
    const int rows = 3 * T.k * T.k;
    const bool tr = near_transposed(T.k);
    const int tile_rows = table_rows_per_tile(tr);
    const int Kp = (T.k * T.k + kKBlock - 1) / kKBlock * kKBlock;
    return build_contraction_plan(I, kNearCfg, (rows + tile_rows - 1) / tile_rows, R, tr, Kp / kKBlock, 48.0 / Kp,
                                  (size_t)rows * sizeof(float2), A, &PS->near);
}

// All five plans of R folded right-hand sides. The contractions are independent: each is built on a
// host thread of its own into its own arena; the arenas are then joined (offsets shifted) and
// copied to the device at once.
static int build_plans(const DeviceTree& T, int R, const HostLists& H, PlanSet* PS, cudaStream_t st) {
    PS->R = R;
    int dev = 0;
    VFMM_CUDA(cudaGetDevice(&dev));
    PlanArena A[kNumCtr];
    int rc[kNumCtr];
    auto task = [&](int c) {
        cudaSetDevice(dev);  // the split-K heuristic reads the device's SM count
        rc[c] = c == kCtrNear ? build_near_plan(T, R, H, A[c], PS) : build_far_plan(c, T, R, H, A[c], PS);
    };
    std::vector<std::thread> workers;
    for (int c = 1; c < kNumCtr; ++c) workers.emplace_back(task, c);
    task(kCtrNear);
    for (auto& w : workers) w.join();
    for (int c = 0; c < kNumCtr; ++c)
        if (rc[c] != VFMM_OK) return fail(rc[c], "split-contraction plan " + std::to_string(c) + " failed");
    SplitPlan* top[kNumCtr];
    top[kCtrNear] = &PS->near;
    top[kCtrS2M] = &PS->s2m;
    top[kCtrM2L] = &PS->m2l;
    top[kCtrS2L] = &PS->s2l;
    top[kCtrFar] = &PS->far;
    PlanArena all;
    size_t total = 0;
    for (int c = 0; c < kNumCtr; ++c) total += A[c].data.size();
    all.data.reserve(total);
    for (int c = 0; c < kNumCtr; ++c) {
        const int64_t base = (int64_t)all.data.size();
        for (SplitPlan* P = top[c]; P; P = P->alt)
            for (int i = 0; i < 6; ++i)
                if (P->off[i] >= 0) P->off[i] += base;
        all.data.insert(all.data.end(), A[c].data.begin(), A[c].data.end());
    }
    return commit_plan_arena(all, PS, st);
}

int build_mixed_plan(DeviceTree* T, cudaStream_t st) {
    HostLists H;
    VFMM_CHECK(fetch_host_lists(*T, &H));
    VFMM_CHECK(build_far_slots(T, H, st));
    VFMM_CHECK(build_near_tiles(T, H, st));  // the FP64 form's GEMM tiles
    T->plans_r = new std::map<int, PlanSet*>();
    T->plans_mu = new std::mutex();
    return build_plans(*T, 1, H, &T->plans, st);
}

int plans_for(const DeviceTree& T, int R, const PlanSet** out) {
    if (R == 1) {
        *out = &T.plans;
        return VFMM_OK;
    }
    if (!T.plans_mu || !T.plans_r) return fail(VFMM_ERR_INTERNAL, "tree has no plan cache");
    std::lock_guard<std::mutex> lock(*T.plans_mu);
    auto it = T.plans_r->find(R);
    if (it != T.plans_r->end()) {
        *out = it->second;
        return VFMM_OK;
    }
    PlanSet* ps = new PlanSet();
    HostLists H;
    int rc = fetch_host_lists(T, &H);
    if (rc == VFMM_OK) rc = build_plans(T, R, H, ps, cudaStreamPerThread);
    if (rc != VFMM_OK) {
        free_plan_set(ps);
        delete ps;
        return rc;
    }
    (*T.plans_r)[R] = ps;
    *out = ps;
    return VFMM_OK;
}

static int fmax_sms() {
    static thread_local int dev = -1, n = 0;
    int d = 0;
    cudaGetDevice(&d);
    if (d != dev) {
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d);
        dev = d;
    }
    return n > 0 ? n : 1;
}

int near_slices(const DeviceTree& T, const PlanSet& PS, const vfmm_ops& o, const double* f, const MixedWork& w,
                cudaStream_t st) {
    const MixedOps* mo = (const MixedOps*)o.mixed;
    const int kk = o.k * o.k, R = PS.R;
    VFMM_CUDA(cudaMemsetAsync(w.fmax, 0, (size_t)R * sizeof(unsigned long long), st));
    const int64_t n = (int64_t)T.n_leaves * kk;
    // two CTAs per SM, each thread a few values: a few hundred atomics instead of one per warp
    const int64_t fm_ctas = std::min<int64_t>(2 * (int64_t)fmax_sms(), (n + 255) / 256);
    fmax_abs_kernel<<<dim3((unsigned)std::max<int64_t>(1, fm_ctas), R), 256, 0, st>>>(f, n, w.fmax);
    const int64_t nchunk = (int64_t)T.n_leaves * R * (mo->Kp / 8);
    f_slice_kernel<<<(unsigned)((nchunk + 255) / 256), 256, 0, st>>>(f, T.n_leaves, kk, mo->Kp, R, w.fmax, w.Ef,
                                                                     (bf16*)w.fsl);
    VFMM_CUDA(cudaGetLastError());
    return VFMM_OK;
}

int near_contract(const DeviceTree& T, const PlanSet& PS, const vfmm_ops& o, const MixedWork& w, cudaStream_t st) {
    const MixedOps* mo = (const MixedOps*)o.mixed;
    return split_gemm(PS.near, w.fsl, mo->tm_near, mo->Kp, mo->Rp, w.out, w.err, w.part_side,
                      (size_t)T.n_leaves * PS.R, mo->slices[kCtrNear], st, w.cev ? w.cev + 0 : nullptr);
}

}  // namespace vfmm
