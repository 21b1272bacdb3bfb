// Split-BF16 near field: constants and device buffers.
#pragma once

#include <cuda.h>  // CUtensorMap (the encoder is fetched through the runtime's driver entry point)
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <climits>

#include <utility>
#include <vector>

#include "ops.cuh"
#include "vfmm_internal.cuh"

namespace vfmm {

constexpr int kSlices = 8;   // BF16 slice slots per operand (balanced base-128 digits, 56 bits)
constexpr int kMinSlices = 6;  // fewest slices a contraction may take (every accumulator gets a product)
// contractions of the mixed form, in the order of vfmm_ops_set_slices
enum { kCtrNear = 0, kCtrS2M = 1, kCtrM2L = 2, kCtrS2L = 3, kCtrFar = 4, kNumCtr = 5 };
constexpr int kTileM = 128;  // target leaves per tile (TMEM lanes)
constexpr int kKBlock = 32;  // K values per pipeline stage (64-byte rows)
constexpr int kStages = 2;   // shared-memory stages
constexpr int kTileN = 80;   // table rows per tile
constexpr int kTileNSmall = 48;  // table rows per tile when 2p <= 48 (S2M, M2L, S2L at p <= 24)
constexpr int kNumAcc = 6;   // TMEM accumulators (diagonals 0..4 exact, 5+ shared)
constexpr int kTmemCols = 512;                  // allocation (power of two >= kNumAcc * kTileN)
constexpr int kEpilogueWarps = 8;
constexpr int kEpilogueThreads = 32 * kEpilogueWarps;
constexpr int kProducerThreads = 96;
constexpr int kMmaWarp = kEpilogueWarps + kProducerThreads / 32;  // 11
constexpr int kThreads = 32 * (kMmaWarp + 1);                     // 384: 3 warps per SM sub-partition
constexpr int kMaxSplit = 16;  // largest split-K factor (partial sums held for small contractions only)
static_assert(kNumAcc * kTileN <= kTmemCols, "TMEM budget");

// Orientation of the near-field and leaf far-field contractions: with 3k^2 a multiple of 128
// (k = 16) the table rows are the M side (128 per tile, TMA) and the targets the N side (80 per
// group, gathered), which gathers 40 % fewer bytes; otherwise targets are the M side (128 per group)
// and table rows the N side (80 per tile). M2L, S2L and S2M (2p rows) always use the latter.
__host__ __device__ constexpr bool near_transposed(int k) { return (3 * k * k) % kTileM == 0; }
// Table rows per tile of a contraction whose tables have Rp rows: 128 (transposed), else 80, or 48
// for the 48-row tables of small expansions.
__host__ __device__ constexpr int table_rows_per_tile(bool transposed, int Rp = kTileN) {
    return transposed ? kTileM : (Rp % kTileN == 0 ? kTileN : kTileNSmall);
}
// N of the MMAs (TMEM columns per accumulator): the gathered targets (80) when transposed, else the
// table rows per tile.
__host__ __device__ constexpr int mma_n(bool transposed, int Rp) {
    return transposed ? kTileN : table_rows_per_tile(false, Rp);
}

// Splits v / 2^E (|v| < 2^E) into kSlices balanced base-128 digits, out[(i - 1) * stride] =
// d_i 2^(-7 i), with v / 2^E = sum_i d_i 2^(-7 i) + (|v| 2^(56 - E) - floor(|v| 2^(56 - E))) 2^-56:
// q = floor(|v| 2^(56 - E)) is written in base 128 from its low end, a digit of 64 or more becoming
// d - 128 with a carry into the next higher one, so d_2..d_8 lie in [-64, 63] and d_1 in [0, 128];
// a negative v negates every digit. Each is an integer of at most 8 significant bits (exact in
// BF16), the products of two are below 2^14, and the first S digits are v / 2^E rounded to the
// nearest multiple of 2^(-7 S) (error at most 2^(-7 S - 1) of the scale 2^E). Integer work on the
// bits of v (its significand shifted to 56 fractional bits).
__device__ __forceinline__ void slice_fixed(double v, int E, __nv_bfloat16* out, int stride) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    int ev = (int)((bits >> 52) & 0x7FF);
    unsigned long long mant = bits & ((1ull << 52) - 1);
    if (ev) mant |= 1ull << 52;
    else ev = 1;
    // |v| 2^(56 - E) = mant 2^(ev - 1075 + 56 - E): a right shift by 1019 - ev + E (>= -3 when |v| < 2^E)
    const int shift = 1019 - ev + E;
    const unsigned long long q = shift >= 64 ? 0ull : (shift >= 0 ? mant >> shift : mant << (-shift));
    const bool neg = (bits >> 63) != 0;
    int carry = 0;
#pragma unroll
    for (int i = kSlices; i >= 1; --i) {
        int d = (int)((q >> (7 * (kSlices - i))) & 127ull) + carry;
        carry = (i > 1 && d >= 64) ? 1 : 0;
        d -= carry << 7;
        const float s = (float)(neg ? -d : d) * __int_as_float((127 - 7 * i) << 23);
        out[(i - 1) * stride] = __float2bfloat16_rn(s);
    }
}

// 2^e as a double built from its exponent bits (e clamped to the normal range).
__device__ __forceinline__ double pow2(int e) {
    e = max(-1022, min(1023, e));
    return __longlong_as_double((long long)(e + 1023) << 52);
}

// (double)x * 2^e for a float x from the bits, with integer operations only (the FP64 units are
// the scarce ones): sign and mantissa move over, the exponent is rebiased and shifted by e. A zero
// or subnormal x gives (signed) zero: the (hi, lo) outputs of the split contractions are
// normalised, so a part below 2^-126 is far below the rounding of the sum it belongs to. The
// result must lie in the normal double range.
__device__ __forceinline__ double f2d_scaled(float x, int e) {
    const unsigned int u = __float_as_uint(x);
    const int ex = (int)((u >> 23) & 0xFF);
    const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
    const unsigned long long mag = ((unsigned long long)(ex - 127 + 1023 + e) << 52) |
                                   ((unsigned long long)(u & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)(sign | (ex == 0 ? 0ull : mag)));
}

// Binary exponent e with |m| < 2^e (frexp convention), from the bits; 0 for m = 0.
__device__ __forceinline__ int exp_bound(double m) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(m);
    if ((bits << 1) == 0) return 0;
    const int ev = (int)((bits >> 52) & 0x7FF);
    return (ev ? ev : 1) - 1022;
}

// Offset of (row, slice 0, k) in a sliced operand [row][K block of 32][slice][32 values].
__device__ __forceinline__ size_t slice_at(size_t row, int Kp, int k) {
    return ((row * (Kp / kKBlock) + k / kKBlock) * kSlices) * kKBlock + (k % kKBlock);
}

// Level exponents of the M2L operand: G(l, r) = max over the boxes b of level l and the parts k
// (Re, Im of coefficient k / 2) of multipole row b of part_exp(value, k), kept as G + kGexpBias in
// an unsigned array that starts at zero, so that every producer of a multipole can take the maximum
// with atomicMax as it writes (order-independent, hence deterministic).
constexpr unsigned kGexpBias = 1u << 20;

// frexp exponent of |v| (from the bits, integer work) plus floor(k / 4); INT_MIN for +-0.
__device__ __forceinline__ int part_exp(double v, int k) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    if ((bits << 1) == 0) return INT_MIN;
    const int ev = (int)((bits >> 52) & 0x7FF);
    return (ev ? ev : 1) - 1022 + (k >> 2);
}

// Warp-wide maximum of e, then one atomicMax into the biased level exponent (lanes with INT_MIN
// contribute nothing).
__device__ __forceinline__ void level_exp_max(int e, unsigned* slot) {
    for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
    if ((threadIdx.x & 31) == 0 && e != INT_MIN) atomicMax(slot, (unsigned)(e + (int)kGexpBias));
}

// Block-wide maximum of e, then one atomicMax by thread 0 (every thread of the block must call it;
// at most 32 warps).
__device__ __forceinline__ void level_exp_max_block(int e, unsigned* slot) {
    __shared__ int wmax[32];
    for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)((blockDim.x + 31) >> 5); ++w) e = max(e, wmax[w]);
        if (e != INT_MIN) atomicMax(slot, (unsigned)(e + (int)kGexpBias));
    }
}

// Level exponent from its biased form.
__device__ __forceinline__ int level_exp_value(unsigned g) { return g ? (int)g - (int)kGexpBias : 0; }

// slice_fixed of 8 consecutive values (one exponent bound E) with each slice's 8 BF16 written
// by one 16-byte store: out + i * stride for slice i (16-byte aligned).
__device__ __forceinline__ void slice8_fixed(const double* v, int E, __nv_bfloat16* out, int stride) {
    __align__(16) __nv_bfloat16 tmp[kSlices][8];
#pragma unroll
    for (int j = 0; j < 8; ++j) slice_fixed(v[j], E, &tmp[0][j], 8);
#pragma unroll
    for (int i = 0; i < kSlices; ++i) *reinterpret_cast<uint4*>(out + (size_t)i * stride) = *reinterpret_cast<uint4*>(tmp[i]);
}

struct MixedOps {
    int N = kTileN; // table rows per tile
    int Rp = 0;     // 3k^2 rounded up to N
    int Kp = 0;     // k^2 rounded up to kKBlock
    void* tsl = nullptr;  // bf16 [33][Rp][kSlices][Kp]
    int* Er = nullptr;    // [Rp] row exponents
    // TMA descriptors of the sliced tables (box = 80 rows x 64 bytes of one slice and K block)
    CUtensorMap tm_near, tm_s2m, tm_m2l, tm_far, tm_s2l;
    // far field: expansion coefficients as reals (Re, Im of 0..p), Kx = 2(p+1) padded
    int Kx = 0;           // 2(p+1) rounded up to kKBlock
    int Rx = 0;           // 2p rounded up to 48 (2p <= 48) or to kTileN (rows of S2M and M2L without coefficient 0)
    void* s2m_sl = nullptr;   // bf16 [1][Rx][kSlices][Kp]: S2M rows 2..2p+1
    int* s2m_E = nullptr;     // [Rx]
    // M2L rows 2..2p+1 over input columns 0..2p+1, column k scaled by 2^-floor(k/4) (the decay
    // bound of multipole coefficient k/2), then per row by 2^-m2l_E[r]
    void* m2l_sl = nullptr;   // bf16 [40][Rx][kSlices][Kx]
    int* m2l_E = nullptr;     // [Rx]
    void* far_sl = nullptr;   // bf16 [21][Rp][kSlices][Kx]: L2T (0) and M2T per W configuration
    int* far_E = nullptr;     // [Rp]
    void* s2l_sl = nullptr;   // bf16 [20][Rx][kSlices][Kp]: S2L rows of coefficients 1..p
    int* s2l_E = nullptr;     // [Rx]
    double* s2l_r0 = nullptr; // [20][kk] FP64: Re of S2L row 0
    double* m2l_r0 = nullptr; // [40][p+1] complex FP64: M2L row 0 (output coefficient 0) per offset
    // slices taken per contraction (kCtr*): the first S of the 8 stored slices of each operand and
    // the S(S+1)/2 products i + j <= S + 1. Default 6 for all (42 bits, 21 products): the error
    // against the FP64 form is then at most 6e-12 on the 20-Gaussian, kinked and uniform k = 16
    // workloads, 17x below 1e-10 (7 for all: 6e-14)
    int slices[kNumCtr] = {6, 6, 6, 6, 6};
};

// s + e = a + b exactly (FP32, round to nearest).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (hi, lo) += v in double-float with exact two-sums; df_final renormalises.
__device__ __forceinline__ void df_add(float& hi, float& lo, float2 v) {
    float s1, e1, s2, e2;
    two_sum(hi, v.x, s1, e1);
    two_sum(s1, v.y, s2, e2);
    hi = s2;
    lo = __fadd_rn(lo, __fadd_rn(e1, e2));
}

__device__ __forceinline__ float2 df_final(float hi, float lo) {
    const float h = __fadd_rn(hi, lo);
    return make_float2(h, __fsub_rn(lo, __fsub_rn(h, hi)));
}

struct MixedWork {
    void* fsl = nullptr;                  // bf16 [n_leaves][kSlices][Kp]
    float2* out = nullptr;                // [n_leaves][Rp] (hi, lo), scaled by 2^-(E_f + E_r)
    unsigned long long* fmax = nullptr;   // [R] max |f| per right-hand side (bits)
    int* Ef = nullptr;                    // [R] exponent of f per right-hand side
    int* err = nullptr;                   // non-zero after a bounded wait expired
    // far field
    float2* s2m_out = nullptr;            // [n_leaves][Rx]
    unsigned* glev = nullptr;             // [(depth + 1) * R] G(l, r) + kGexpBias (0: level all zero):
                                          // |multipole part k| 2^floor(k/4) < 2^G for parts k = 0 .. 2p+1
    void* msl = nullptr;                  // bf16 [n_boxes][kSlices][Kx]
    float2* m2l_out = nullptr;            // [n_boxes][Rx]
    double* m2l_c0 = nullptr;             // [n_boxes] Re local coefficient 0 from the V and X lists
    float2* s2l_out = nullptr;            // [n_boxes][Rx]
    void* aprep = nullptr;                // bf16 [n_far_slots][kSlices][Kx]
    int* Et = nullptr;                    // [n_leaves]
    float2* far_out = nullptr;            // [n_leaves][Rp]
    float2* part = nullptr;               // partial sums or slab of S2M, M2L and the leaf far field
    float2* part_side = nullptr;          // partial sums or slab of the near field
    float2* part_s2l = nullptr;           // partial sums or slab of S2L
    cudaEvent_t* cev = nullptr;           // optional (start, stop) pairs: near, S2M, M2L, S2L, far
};

// Host staging of the index arrays of one plan set: put() appends an array and returns its offset
// (int32 elements; pieces start on 256-byte boundaries); commit_plan_arena() makes one device
// allocation, copies everything once and points every plan of the set (and its alternative form)
// into it.
struct PlanArena {
    std::vector<int32_t> data;
    int64_t put(const std::vector<int32_t>& v) {
        const int64_t off = (int64_t)data.size();
        const size_t len = std::max<size_t>(64, (v.size() + 63) / 64 * 64);
        data.resize(off + len, 0);
        std::copy(v.begin(), v.end(), data.begin() + off);
        return off;
    }
};
int commit_plan_arena(PlanArena& A, PlanSet* PS, cudaStream_t st);

// Targets of one split contraction in flat form: target t (output row tgt[t]) holds the items
// (tab[e], src[e]) = (table, gathered operand row), e in [ptr[t], ptr[t + 1]), and sorts by key[t].
struct PlanItems {
    std::vector<int32_t> tgt, ptr{0}, tab, src;
    std::vector<std::pair<uint64_t, uint64_t>> key;
    void add(int32_t table, int32_t row) {
        tab.push_back(table);
        src.push_back(row);
    }
    void close(int32_t id, uint64_t k0, uint64_t k1) {  // ends the target whose items were just added
        tgt.push_back(id);
        ptr.push_back((int32_t)tab.size());
        key.push_back({k0, k1});
    }
};
// Groups of 128 (80 when transposed) targets taken in the given order; per group the tables present
// and, per table, the gathered row of each target (-1 when the target has no entry for that table).
int build_split_plan(const PlanItems& I, const std::vector<int32_t>& order, int n_tables, int n_chunks, int R,
                     bool transposed, int nkb, PlanArena& A, SplitPlan* P);
// build_split_plan, or its entry-major form when that executes enough fewer columns: chosen when
// (entry-major columns) x (1 + slab_overhead) < 0.85 x (grouped columns, padding included) and the
// slab (entries x R x slab_row_bytes) stays within 256 MB. slab_overhead = the slab's write and read
// time per column relative to its tensor time. A small contraction (fewer CTAs than two per SM)
// whose slab fits keeps the form not chosen in P->alt.
int build_contraction_plan(const PlanItems& I, int n_tables, int n_chunks, int R, bool transposed, int nkb,
                           double slab_overhead, size_t slab_row_bytes, PlanArena& A, SplitPlan* P);
// Tensor map of a sliced table [rows][Kp / 32][kSlices][32] BF16 for the table operand of split_gemm
// (box = box_rows rows x 64 bytes of one slice and K block).
int make_table_map(const void* base, int64_t rows, int Kp, int box_rows, CUtensorMap* out);
// ev (optional): a (start, stop) event pair recorded around the contraction and its reduction.
int split_gemm(const SplitPlan& P, const void* asl, const CUtensorMap& bmap, int Kp, int Rp, float2* out, int* err,
               float2* part, size_t n_out_rows, int slices, cudaStream_t st, cudaEvent_t* ev = nullptr,
               int defer = 0);
// split_gemm's `defer` bits: the consumer of the output sums the entry-major slab rows of each
// target (kDeferSegments) or the split-K partial sums (kDeferSplits) itself, in the same order and
// arithmetic as the reduction kernels, which are then not launched
constexpr int kDeferSegments = 1;
constexpr int kDeferSplits = 2;
// Partial-sum elements (float2) of the three buffers whose contractions may run at the same time:
// [0] S2M, M2L and the leaf far field (one after another), [1] the near field, [2] S2L.
void split_part_elems(const DeviceTree& T, const PlanSet& PS, const vfmm_ops& o, size_t elems[3]);
int build_mixed_plan(DeviceTree* T, cudaStream_t st);
// Host copies of the tree arrays the plan builders read (fetched once per plan set).
struct HostLists {
    std::vector<int32_t> bol, lob, ptr[4], idx[4], cfg[4];
};
int fetch_host_lists(const DeviceTree& T, HostLists* H);
int build_far_slots(DeviceTree* T, const HostLists& H, cudaStream_t st);
// Plan of one far-field contraction (kCtrS2M, kCtrM2L, kCtrS2L or kCtrFar) into PS.
int build_far_plan(int which, const DeviceTree& T, int R, const HostLists& H, PlanArena& A, PlanSet* PS);
// Near field in two parts: max |f| and the f slices (also the operand of S2M and S2L), then the
// split contraction.
int near_slices(const DeviceTree& T, const PlanSet& PS, const vfmm_ops& o, const double* f, const MixedWork& w,
                cudaStream_t st);
int near_contract(const DeviceTree& T, const PlanSet& PS, const vfmm_ops& o, const MixedWork& w, cudaStream_t st);
int far_prepare(vfmm_ops* o, cudaStream_t st);
void far_free(MixedOps* mo);
// Stages of the split-precision far field (see mixed_far.cu). Multipoles and locals are stored per
// virtual box (box * R + r); f is [R][n_leaves][k^2].
int s2m_mixed(const DeviceTree& T, const PlanSet& PS, const vfmm_ops& o, const double* f, double* Mexp,
              const MixedWork& w, cudaStream_t st);
// exps_done: the level exponents of the non-leaf multipoles were already taken (persistent upward
// pass); leaf multipoles always take theirs in S2M.
int m2l_mixed(const DeviceTree& T, const PlanSet& PS, const vfmm_ops& o, const double* Mexp, const MixedWork& w,
              bool exps_done, cudaStream_t st);
int s2l_mixed(const DeviceTree& T, const PlanSet& PS, const vfmm_ops& o, const MixedWork& w, cudaStream_t st);
int far_leaf_mixed(const DeviceTree& T, const PlanSet& PS, const vfmm_ops& o, const double* Mexp, const double* Lexp,
                   const MixedWork& w, cudaStream_t st);

}  // namespace vfmm
