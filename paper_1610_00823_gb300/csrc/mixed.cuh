// Split-BF16 near field: constants and device buffers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ops.cuh"
#include "vfmm_internal.cuh"

namespace vfmm {

constexpr int kSlices = 8;   // BF16 slices per operand (6-bit magnitudes, 48 bits)
constexpr int kTileM = 128;  // target leaves per tile (TMEM lanes)
constexpr int kKBlock = 32;  // K values per pipeline stage (64-byte rows)
constexpr int kStages = 2;   // shared-memory stages
constexpr int kTileN = 80;   // table rows per tile
constexpr int kNumAcc = 6;   // TMEM accumulators (diagonals 0..4 exact, 5+ shared)
constexpr int kTmemCols = 512;                  // allocation (power of two >= kNumAcc * kTileN)
constexpr int kEpilogueWarps = 8;
constexpr int kEpilogueThreads = 32 * kEpilogueWarps;
constexpr int kProducerThreads = 96;
constexpr int kMmaWarp = kEpilogueWarps + kProducerThreads / 32;  // 11
constexpr int kThreads = 32 * (kMmaWarp + 1);                     // 384: 3 warps per SM sub-partition
static_assert(kNumAcc * kTileN <= kTmemCols, "TMEM budget");

struct MixedOps {
    int N = kTileN; // table rows per tile
    int Rp = 0;     // 3k^2 rounded up to N
    int Kp = 0;     // k^2 rounded up to kKBlock
    void* tsl = nullptr;  // bf16 [33][Rp][kSlices][Kp]
    int* Er = nullptr;    // [Rp] row exponents
};

struct MixedWork {
    void* fsl;                  // bf16 [n_leaves][kSlices][Kp]
    float2* out;                // [n_leaves][Rp] (hi, lo), scaled by 2^-(E_f + E_r)
    unsigned long long* fmax;   // max |f| (bits)
    int* Ef;                    // exponent of f
    int* err;                   // non-zero after a bounded wait expired
};

int build_mixed_plan(DeviceTree* T);
int near_mixed(const DeviceTree& T, const vfmm_ops& o, const double* f, const MixedWork& w, cudaStream_t st);

}  // namespace vfmm
