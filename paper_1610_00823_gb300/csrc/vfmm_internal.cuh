// Internal declarations of the vfmm library (device code for sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "vfmm.h"

namespace vfmm {

constexpr int kMaxDepth = 16;
constexpr int kNearCfg = 33;  // same level 9 + coarser 12 + finer 12
constexpr int kVCfg = 40;     // offsets in [-3,3]^2 outside [-1,1]^2
constexpr int kFarCfg = 20;   // W and X configurations

// ---------------------------------------------------------------- error plumbing
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define VFMM_CUDA(call)                                                  \
    do {                                                                 \
        cudaError_t _e = (call);                                         \
        if (_e != cudaSuccess) return ::vfmm::cuda_fail(_e, #call);      \
    } while (0)

#define VFMM_CHECK(call)                  \
    do {                                  \
        int _r = (call);                  \
        if (_r != VFMM_OK) return _r;     \
    } while (0)

// ---------------------------------------------------------------- geometry
// Morton key of a box: bit b of ix -> bit 2b, bit b of iy -> bit 2b+1.
__host__ __device__ inline uint32_t morton_encode(uint32_t ix, uint32_t iy) {
    uint32_t key = 0;
    for (int b = 0; b < 16; ++b) {
        key |= ((ix >> b) & 1u) << (2 * b);
        key |= ((iy >> b) & 1u) << (2 * b + 1);
    }
    return key;
}
__host__ __device__ inline void morton_decode(uint32_t key, int* ix, int* iy) {
    uint32_t x = 0, y = 0;
    for (int b = 0; b < 16; ++b) {
        x |= ((key >> (2 * b)) & 1u) << b;
        y |= ((key >> (2 * b + 1)) & 1u) << b;
    }
    *ix = (int)x;
    *iy = (int)y;
}

// Closed boxes (la, ax, ay) and (lb, bx, by) touch but their interiors are disjoint.
__host__ __device__ inline bool boxes_adjacent(int la, int ax, int ay, int lb, int bx, int by) {
    int top = la > lb ? la : lb;
    long long sa = 1ll << (top - la), sb = 1ll << (top - lb);
    long long a0 = ax * sa, a1 = a0 + sa, b0 = bx * sb, b1 = b0 + sb;
    long long c0 = ay * sa, c1 = c0 + sa, d0 = by * sb, d1 = d0 + sb;
    bool touch = a0 <= b1 && b0 <= a1 && c0 <= d1 && d0 <= c1;
    bool inter = a0 < b1 && b0 < a1 && c0 < d1 && d0 < c1;
    return touch && !inter;
}

// 4 * (centre_c - centre_b) / h_b, exact integers for |level_c - level_b| <= 1.
__host__ __device__ inline void centre_offset4(int lb, int bx, int by, int lc, int cx, int cy, int* dx4, int* dy4) {
    // centre in units of h_20 / 2: (2i + 1) << (20 - l)
    long long pbx = (long long)(2 * bx + 1) << (20 - lb), pby = (long long)(2 * by + 1) << (20 - lb);
    long long pcx = (long long)(2 * cx + 1) << (20 - lc), pcy = (long long)(2 * cy + 1) << (20 - lc);
    long long div = 1ll << (20 - lb - 1);
    *dx4 = (int)((pcx - pbx) / div);
    *dy4 = (int)((pcy - pby) / div);
}

// The 12 offsets of the coarse/fine near configurations (in units of 2D resp. 4D)
// and the 20 of the W/X configurations (4D resp. 2D), each sorted by (y, x).
__host__ __device__ inline int near_pattern_index(int px, int py) {
    const int P[12][2] = {{-3, -3}, {-1, -3}, {1, -3}, {3, -3}, {-3, -1}, {3, -1},
                          {-3, 1},  {3, 1},   {-3, 3}, {-1, 3}, {1, 3},   {3, 3}};
    for (int i = 0; i < 12; ++i)
        if (P[i][0] == px && P[i][1] == py) return i;
    return -1;
}
__host__ __device__ inline void near_pattern(int i, int* px, int* py) {
    const int P[12][2] = {{-3, -3}, {-1, -3}, {1, -3}, {3, -3}, {-3, -1}, {3, -1},
                          {-3, 1},  {3, 1},   {-3, 3}, {-1, 3}, {1, 3},   {3, 3}};
    *px = P[i][0];
    *py = P[i][1];
}
__host__ __device__ inline int far_pattern_index(int px, int py) {
    const int P[20][2] = {{-5, -5}, {-3, -5}, {-1, -5}, {1, -5}, {3, -5}, {5, -5}, {-5, -3},
                          {5, -3},  {-5, -1}, {5, -1},  {-5, 1}, {5, 1},  {-5, 3}, {5, 3},
                          {-5, 5},  {-3, 5},  {-1, 5},  {1, 5},  {3, 5},  {5, 5}};
    for (int i = 0; i < 20; ++i)
        if (P[i][0] == px && P[i][1] == py) return i;
    return -1;
}
__host__ __device__ inline void far_pattern(int i, int* px, int* py) {
    const int P[20][2] = {{-5, -5}, {-3, -5}, {-1, -5}, {1, -5}, {3, -5}, {5, -5}, {-5, -3},
                          {5, -3},  {-5, -1}, {5, -1},  {-5, 1}, {5, 1},  {-5, 3}, {5, 3},
                          {-5, 5},  {-3, 5},  {-1, 5},  {1, 5},  {3, 5},  {5, 5}};
    *px = P[i][0];
    *py = P[i][1];
}
// V offsets: row-major over dy, dx in [-3, 3], skipping max(|dx|,|dy|) <= 1.
__host__ __device__ inline int v_offset_index(int dx, int dy) {
    int idx = 0;
    for (int y = -3; y <= 3; ++y)
        for (int x = -3; x <= 3; ++x) {
            int ax = x < 0 ? -x : x, ay = y < 0 ? -y : y;
            if ((ax > ay ? ax : ay) < 2) continue;
            if (x == dx && y == dy) return idx;
            ++idx;
        }
    return -1;
}
__host__ __device__ inline void v_offset(int i, int* dx, int* dy) {
    int idx = 0;
    for (int y = -3; y <= 3; ++y)
        for (int x = -3; x <= 3; ++x) {
            int ax = x < 0 ? -x : x, ay = y < 0 ? -y : y;
            if ((ax > ay ? ax : ay) < 2) continue;
            if (idx == i) {
                *dx = x;
                *dy = y;
                return;
            }
            ++idx;
        }
}
// Near configuration geometry: source width / target width and centre offset (target widths).
__host__ __device__ inline void near_config_geometry(int cfg, double* rho, double* dx, double* dy) {
    if (cfg < 9) {
        *rho = 1.0;
        *dx = (double)(cfg % 3 - 1);
        *dy = (double)(cfg / 3 - 1);
    } else if (cfg < 21) {
        int px, py;
        near_pattern(cfg - 9, &px, &py);
        *rho = 2.0;
        *dx = px / 2.0;
        *dy = py / 2.0;
    } else {
        int px, py;
        near_pattern(cfg - 21, &px, &py);
        *rho = 0.5;
        *dx = px / 4.0;
        *dy = py / 4.0;
    }
}

// ---------------------------------------------------------------- tree handle
// Schedule of one split-precision contraction: groups of 128 targets, the tables present
// in each group and the A row of every target for every table (-1: none).
struct SplitPlan {
    int32_t n_groups = 0;
    int64_t entries = 0;
    int32_t* tgt = nullptr;  // [n_groups][group] output row or -1
    int32_t* ptr = nullptr;  // [n_groups + 1]
    int32_t* cfg = nullptr;  // [entries] table index
    int32_t* src = nullptr;  // [entries][group] gathered operand row or -1
    int32_t split = 1;       // CTAs per group (each takes a share of the group's tables)
    int32_t ctas = 0;        // CTA cap of the launch (persistent CTAs walk several work items); 0: one CTA per item
    bool may_split = false;  // small contraction (fewer CTAs than two per SM): split-K allowed
    bool transposed = false; // table rows on the M side (128 per tile), targets on the N side
    int32_t group = 128;     // targets per group: 128, or 80 when transposed
    // Entry-major form: every (target, table) entry is a column of its own, grouped by table, so
    // no column is empty; the contraction writes one slab row per entry (in the partial-sum
    // buffer) and a segmented reduction sums each target's entries into its output row.
    bool entry = false;
    int32_t R = 1;             // folded right-hand sides (slab row of entry q: q * R + r)
    int32_t n_seg = 0;         // targets
    int64_t slab_rows = 0;     // entries * R
    int32_t* seg = nullptr;    // [n_seg + 1] first entry of each target
    int32_t* seg_out = nullptr;  // [n_seg] output row (before the R fold) of each target
    // the other form of a small contraction (grouped or entry-major), for vfmm_tune to time
    SplitPlan* alt = nullptr;
    // offsets (int32 elements) of tgt, ptr, cfg, src, seg, seg_out in the plan set's arena while it
    // is being built (-1: absent); the pointers above point into the arena once it is committed
    int64_t off[6] = {-1, -1, -1, -1, -1, -1};
};

// The split contractions of the mixed form with R right-hand sides folded into the rows: the
// virtual row of box or leaf x for right-hand side r is x * R + r (R consecutive rows per box).
struct PlanSet {
    int R = 1;
    SplitPlan near;  // U list: targets leaves, tables 33 configurations, A rows leaves
    SplitPlan s2m;   // targets leaves, one table, A rows leaves
    SplitPlan m2l;   // V list: targets boxes, tables the 40 offsets, A rows boxes
    SplitPlan far;   // L2T + W list: targets leaves, tables 0 (L2T) and 1 + W configuration, A rows far slots
    SplitPlan s2l;   // X list: targets boxes, tables 20 configurations, A rows leaves
    // grid cap of the persistent tree passes (0: one CTA per box of the widest level, at most one per
    // SM); with a capped near field the passes then fit on the SMs the near field leaves free
    int32_t pass_ctas = 0;
    void* arena = nullptr;  // one device allocation holding every index array of the plans above
};

struct DeviceTree {
    // box table, canonical order
    int32_t n_boxes = 0, n_leaves = 0, depth = 0, k = 0;
    double cx = 0, cy = 0, width = 0;
    double f_scale = 0, min_margin = 0;
    int64_t n_capped = 0;  // leaves at max_depth still failing the split test (-1: not tested)
    std::vector<int32_t> level_start;  // host copy, depth + 2 entries
    uint32_t* key = nullptr;           // Morton key per box
    int32_t* level = nullptr;
    int32_t* ix = nullptr;
    int32_t* iy = nullptr;
    int32_t* parent = nullptr;
    int32_t* child0 = nullptr;  // first of the 4 consecutive children, -1 for leaves
    int32_t* leaf_of_box = nullptr;  // leaf rank or -1
    int32_t* box_of_leaf = nullptr;
    int32_t* level_start_dev = nullptr;
    // lists (CSR by box)
    int32_t* lptr[4] = {nullptr, nullptr, nullptr, nullptr};
    int32_t* lidx[4] = {nullptr, nullptr, nullptr, nullptr};
    int32_t* lcfg[4] = {nullptr, nullptr, nullptr, nullptr};
    int64_t llen[4] = {0, 0, 0, 0};
    // U entries grouped by near configuration (stable within a configuration)
    int32_t* u_by_cfg = nullptr;       // [llen[U]] U-entry indices
    int32_t* u_tgt = nullptr;          // [llen[U]] target leaf box of each U entry
    std::vector<int64_t> u_cfg_start;  // host, 34 entries
    // GEMM tile schedule for the near field: per tile (cfg, first column)
    int32_t* near_tiles = nullptr;
    int32_t n_near_tiles = 0;
    // V and X entries grouped by configuration, with GEMM tiles (configuration, first, end) over
    // the grouped order and each entry's target box (FP64 form's M2L and S2L)
    int32_t* v_by_cfg = nullptr;
    int32_t* v_tiles = nullptr;
    int32_t n_v_tiles = 0;
    int32_t* x_by_cfg = nullptr;
    int32_t* x_tiles = nullptr;
    int32_t* x_tgt = nullptr;
    int32_t n_x_tiles = 0;
    // split-precision schedules (VFMM_MIXED): one right-hand side built with the tree, others on
    // first use (plans_for), guarded by plans_mu
    PlanSet plans;
    std::map<int, PlanSet*>* plans_r = nullptr;
    std::mutex* plans_mu = nullptr;
    int32_t* nonleaf = nullptr;           // non-leaf boxes in canonical order (grouped by level)
    std::vector<int32_t> nonleaf_start;   // host, depth + 2: first entry of each level
    int32_t* nonleaf_start_dev = nullptr; // device copy
    int32_t* far_slot = nullptr;  // [n_leaves + 1] first A row of each leaf in the far operand
    int64_t n_far_slots = 0;
};

void free_tree(DeviceTree* t);
void free_split_plan(SplitPlan* p);
void free_plan_set(PlanSet* ps);
// Plans for R folded right-hand sides (R = 1: the tree's own set); builds and caches on first use.
int plans_for(const DeviceTree& T, int R, const PlanSet** out);
struct HostLists;
int build_near_tiles(DeviceTree* t, const HostLists& h, cudaStream_t st);
// Device arrays a tree keeps (boxes, lists, schedules) come from a per-device stream-ordered pool:
// tree_malloc allocates in the order of stream st (the tree build synchronises st before it
// returns, after which the arrays are valid on every stream); tree_free returns one to the pool
// and is called once the device has finished with it (free_tree synchronises the device first).
int tree_malloc(void** p, size_t bytes, cudaStream_t st);
void tree_free(void* p);
// vfmm_volume_potential with flags: fork = false keeps every launch on `st` (no second stream);
// reset = false leaves the workspace's status word as it is (a caller solving several right-hand
// sides one after another clears it once, so that a timeout in an early one is not lost).
int volume_potential(const vfmm_tree* tree, const vfmm_ops* ops, const double* f_dev, int32_t nrhs, double* u_dev,
                     double* ux_dev, double* uy_dev, void* workspace_dev, size_t workspace_bytes, cudaStream_t st,
                     bool fork, bool reset = true);
// Reads a status word (device address) after the solve that wrote it has finished: VFMM_OK, or
// VFMM_ERR_TIMEOUT naming the bounded wait that ran out.
int read_status_word(const int* word);
// Device address of the allocation-free scratch's status word on the current device.
int noalloc_status_word(const int** word);
// Multipole and local expansions ([n_boxes][2(p+1)] scaled, complex interleaved) that a
// one-right-hand-side solve with this tree and ops left in its workspace.
int solve_expansions(const vfmm_tree* tree, const vfmm_ops* ops, const void* workspace_dev, size_t workspace_bytes,
                     const double** Mexp, const double** Lexp, int* R);

}  // namespace vfmm

struct vfmm_tree {
    vfmm::DeviceTree t;
};

// A captured, instantiated CUDA graph (one solve, or one batch of solves).
struct vfmm_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};
