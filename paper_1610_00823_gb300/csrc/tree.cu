// Quadtree build, level restriction and interaction lists on the device (Section 3.1).
//
// Build plan (host-driven loop over levels, device work per level):
//   1. F = max |f| over the nodes of the uniform level-min(5, max_depth) tree.
//   2. Refinement, level by level: one CTA per candidate box samples f at its k*k
//      nodes, forms the 2-D Chebyshev coefficients, and flags the box when the
//      largest trailing coefficient exceeds tol * F. A scan of the flags places the
//      children; children of a Morton-sorted level are again Morton-sorted.
//   3. Level restriction, finest level first: every box at level l requires the
//      level-(l-1) cells adjacent to it; their parents are marked in a bitmap over
//      the level-(l-2) grid (together with the parents of the existing level-(l-1)
//      boxes), the bitmap is compacted in Morton order, and level l-1 is rebuilt as
//      the children of the marked boxes. Every added box is forced, so the result is
//      the minimal balanced refinement.
//   4. Canonical numbering (level, Morton), parent/child links, leaf ranks.
//   5. U/V/W/X lists: one thread per box, neighbour lookups by binary search in the
//      Morton-sorted key array of a level, a count pass and a fill pass.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <atomic>
#include <set>
#include <tuple>
#include <unordered_map>

#include "mixed.cuh"
#include "source.cuh"
#include "vfmm_internal.cuh"

namespace vfmm {

// Stream-ordered pool of the tree build's temporaries on the current device (created once, kept
// for the life of the process; up to 256 MB of freed blocks stay reserved for the next build).
static int build_pool(cudaMemPool_t* out) {
    constexpr int kMaxDevices = 16;
    static std::mutex mu;
    static cudaMemPool_t pools[kMaxDevices] = {};
    int dev = 0;
    VFMM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(VFMM_ERR_INTERNAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        VFMM_CUDA(cudaMemPoolCreate(&pools[dev], &props));
        uint64_t keep = uint64_t(256) << 20;
        VFMM_CUDA(cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep));
    }
    *out = pools[dev];
    return VFMM_OK;
}

int tree_malloc(void** p, size_t bytes, cudaStream_t st) {
    cudaMemPool_t pool;
    VFMM_CHECK(build_pool(&pool));
    cudaError_t e = cudaMallocFromPoolAsync(p, std::max<size_t>(bytes, 256), pool, st);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(VFMM_ERR_OOM, "stream-ordered allocation failed for a tree array");
    }
    return VFMM_OK;
}

void tree_free(void* p) {
    if (p) cudaFreeAsync(p, cudaStreamPerThread);
}

// Device buffer of the tree build. alloc(count, st): a temporary from the build pool, allocated
// and freed in the order of stream st (no free waits for the device; the stream must outlive the
// buffer); alloc_keep(count): an array the tree or a builder keeps (cudaMalloc), which release()
// hands over.
template <class T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
    cudaStream_t st = nullptr;
    bool pooled = false;
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    DBuf(DBuf&& o) noexcept : p(o.p), n(o.n), st(o.st), pooled(o.pooled) {
        o.p = nullptr;
        o.n = 0;
    }
    DBuf& operator=(DBuf&& o) noexcept {
        if (this != &o) {
            reset();
            p = o.p;
            n = o.n;
            st = o.st;
            pooled = o.pooled;
            o.p = nullptr;
            o.n = 0;
        }
        return *this;
    }
    ~DBuf() { reset(); }
    void reset() {
        if (p) {
            if (pooled) cudaFreeAsync(p, st);
            else cudaFree(p);
        }
        p = nullptr;
        n = 0;
    }
    int alloc(size_t count, cudaStream_t s) {
        reset();
        n = count;
        if (count == 0) return VFMM_OK;
        cudaMemPool_t pool;
        VFMM_CHECK(build_pool(&pool));
        cudaError_t e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&p), count * sizeof(T), pool, s);
        if (e != cudaSuccess) {
            p = nullptr;
            return fail(VFMM_ERR_OOM, "stream-ordered allocation failed in tree build");
        }
        st = s;
        pooled = true;
        return VFMM_OK;
    }
    // an array the tree keeps, from the build pool in the order of stream s (release() hands it to
    // the tree, whose free_tree returns it with tree_free)
    int alloc_tree(size_t count, cudaStream_t s) { return alloc(count, s); }
    int alloc_keep(size_t count) {
        reset();
        n = count;
        if (count == 0) return VFMM_OK;
        cudaError_t e = cudaMalloc(&p, count * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            return fail(VFMM_ERR_OOM, "cudaMalloc failed in tree build");
        }
        pooled = false;
        return VFMM_OK;
    }
    T* release() {
        T* q = p;
        p = nullptr;
        n = 0;
        return q;
    }
};

// ---------------------------------------------------------------- scan (exclusive, int32)
constexpr int kScanItems = 1024;

__global__ void scan_blocks_kernel(const int32_t* __restrict__ in, int32_t* __restrict__ out,
                                   int32_t* __restrict__ sums, int64_t n) {
    __shared__ int32_t s[256];
    const int64_t base = (int64_t)blockIdx.x * kScanItems;
    const int t = threadIdx.x;
    int32_t v[4];
    int32_t local = 0;
    for (int i = 0; i < 4; ++i) {
        int64_t g = base + t * 4 + i;
        v[i] = g < n ? in[g] : 0;
        local += v[i];
    }
    s[t] = local;
    __syncthreads();
    for (int off = 1; off < 256; off <<= 1) {
        int32_t x = t >= off ? s[t - off] : 0;
        __syncthreads();
        s[t] += x;
        __syncthreads();
    }
    int32_t run = s[t] - local;
    for (int i = 0; i < 4; ++i) {
        int64_t g = base + t * 4 + i;
        if (g < n) out[g] = run;
        run += v[i];
    }
    if (t == 255) sums[blockIdx.x] = s[255];
}

__global__ void scan_add_kernel(int32_t* __restrict__ out, const int32_t* __restrict__ offs, int64_t n) {
    const int64_t base = (int64_t)blockIdx.x * kScanItems;
    const int32_t o = offs[blockIdx.x];
    for (int i = threadIdx.x; i < kScanItems; i += blockDim.x) {
        int64_t g = base + i;
        if (g < n) out[g] += o;
    }
}

// out[i] = sum_{j < i} in[j]; *total = sum of all (host). `in` and `out` may alias.
static int exclusive_scan(const int32_t* in, int32_t* out, int64_t n, int64_t* total, cudaStream_t st) {
    if (n <= 0) {
        *total = 0;
        return VFMM_OK;
    }
    int64_t nb = (n + kScanItems - 1) / kScanItems;
    DBuf<int32_t> sums, sums_x;
    VFMM_CHECK(sums.alloc(nb, st));
    scan_blocks_kernel<<<(unsigned)nb, 256, 0, st>>>(in, out, sums.p, n);
    VFMM_CUDA(cudaGetLastError());
    if (nb == 1) {
        int32_t h = 0;
        VFMM_CUDA(cudaMemcpyAsync(&h, sums.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        VFMM_CUDA(cudaStreamSynchronize(st));
        *total = h;
        return VFMM_OK;
    }
    VFMM_CHECK(sums_x.alloc(nb, st));
    VFMM_CHECK(exclusive_scan(sums.p, sums_x.p, nb, total, st));
    scan_add_kernel<<<(unsigned)nb, 256, 0, st>>>(out, sums_x.p, n);
    VFMM_CUDA(cudaGetLastError());
    return VFMM_OK;
}

// ---------------------------------------------------------------- leaf geometry
struct NodeGeom {
    double lox, loy, width;
    int k;
    const double* xhat;  // [k] device
};

// x = lo + ((i_box + 0.5) + xhat) * h, rounded step by step (no contraction).
__device__ inline double node_coord(double lo, int ib, double xh, double h) {
    return __dadd_rn(lo, __dmul_rn(__dadd_rn(__dadd_rn((double)ib, 0.5), xh), h));
}

// ---------------------------------------------------------------- refinement
__device__ inline void atomic_max_nonneg(double* addr, double v) {
    atomicMax((unsigned long long*)addr, (unsigned long long)__double_as_longlong(v));
}
__device__ inline void atomic_min_nonneg(double* addr, double v) {
    atomicMin((unsigned long long*)addr, (unsigned long long)__double_as_longlong(v));
}

__global__ void fscale_kernel(NodeGeom g, SourceDev src, int level, double* fmax_out, double* vals) {
    const int side = 1 << level;
    const int b = blockIdx.x;
    const int ix = b % side, iy = b / side;
    const double h = ldexp(g.width, -level);
    double m = 0.0;
    for (int t = threadIdx.x; t < g.k * g.k; t += blockDim.x) {
        int i = t % g.k, j = t / g.k;
        double x = node_coord(g.lox, ix, g.xhat[i], h);
        double y = node_coord(g.loy, iy, g.xhat[j], h);
        const double f = source_eval(src, x, y);
        if (vals) vals[(size_t)b * g.k * g.k + t] = f;  // kept for the refinement of this level
        m = fmax(m, fabs(f));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(fmax_out, m);
}

// f at the k^2 nodes of each of n boxes, one thread per node, out[b * k^2 + t] (node t = j k + i):
// the source evaluations of a level spread over every SM (FP64 is the scarce unit, and one CTA per
// box would leave most SMs idle on the coarse levels). lev: per-box levels, or null for `level`.
__global__ void __launch_bounds__(64) node_values_kernel(NodeGeom g, SourceDev src, int level,
                                                        const int32_t* __restrict__ lev,
                                                        const uint32_t* __restrict__ keys, int n,
                                                        double* __restrict__ out) {
    const int kk = g.k * g.k;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)n * kk) return;
    const int b = (int)(q / kk), t = (int)(q - (int64_t)b * kk);
    const int l = lev ? lev[b] : level;
    int ix, iy;
    morton_decode(keys[b], &ix, &iy);
    const double h = ldexp(g.width, -l);
    out[q] = source_eval(src, node_coord(g.lox, ix, g.xhat[t % g.k], h), node_coord(g.loy, iy, g.xhat[t / g.k], h));
}

// The values of n boxes of the f-scale level from that level's full grid of node values (box
// (ix, iy) at row-major position iy 2^level + ix): the same evaluations, not repeated.
__global__ void grid_values_kernel(const double* __restrict__ grid, int level, int kk, const uint32_t* __restrict__ keys,
                                   int n, double* __restrict__ out) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)n * kk) return;
    const int b = (int)(q / kk), t = (int)(q - (int64_t)b * kk);
    int ix, iy;
    morton_decode(keys[b], &ix, &iy);
    out[q] = grid[((size_t)iy * (1u << level) + ix) * kk + t];
}

// Largest trailing Chebyshev coefficient (last two rows and columns) of the k x k interpolant of
// f on the box (level, key): values -> coefficients as c = C V C^T with
// C[m*k + i] = (2 - delta_m0)/k T_m(t_i). Called by a whole CTA (blockDim = k*k rounded up to
// a multiple of 32); the result is valid in thread 0. V and Tm hold k*k doubles, red 8.
__device__ double box_tail(const NodeGeom& g, const SourceDev& src, int level, uint32_t key,
                           const double* __restrict__ C, double* V, double* Tm, double* red,
                           const double* __restrict__ fv = nullptr) {
    const int k = g.k;
    const int t = threadIdx.x;
    const bool active = t < k * k;
    int ix, iy;
    morton_decode(key, &ix, &iy);
    const double h = ldexp(g.width, -level);
    const int i = t % k, j = t / k;
    // f at the box's nodes: the caller's values (pull protocol) or the built-in source
    if (active)
        V[j * k + i] = fv ? fv[t]
                          : source_eval(src, node_coord(g.lox, ix, g.xhat[i], h), node_coord(g.loy, iy, g.xhat[j], h));
    __syncthreads();
    // Tm[m][i] = sum_q C[m][q] V[q][i], thread (m = j, i)
    if (active) {
        double acc = 0.0;
        for (int q = 0; q < k; ++q) acc += C[j * k + q] * V[q * k + i];
        Tm[j * k + i] = acc;
    }
    __syncthreads();
    // c[m][nn] = sum_q Tm[m][q] C[nn][q], thread (m = j, nn = i); trailing entries only
    double tail = 0.0;
    if (active && (j >= k - 2 || i >= k - 2)) {
        double acc = 0.0;
        for (int q = 0; q < k; ++q) acc += Tm[j * k + q] * C[i * k + q];
        tail = fabs(acc);
    }
    for (int o = 16; o > 0; o >>= 1) tail = fmax(tail, __shfl_xor_sync(0xffffffffu, tail, o));
    const int nw = blockDim.x / 32;
    if ((t & 31) == 0) red[t >> 5] = tail;
    __syncthreads();
    double mx = 0.0;
    if (t == 0)
        for (int w = 0; w < nw; ++w) mx = fmax(mx, red[w]);
    return mx;
}

// One CTA per candidate box of one level: split flag = tail > thresh. fv (optional): the caller's
// f values, k^2 per candidate box in candidate order.
__global__ void refine_kernel(NodeGeom g, SourceDev src, int level, const uint32_t* __restrict__ keys, int n,
                              const double* __restrict__ C, double thresh, int32_t* __restrict__ flags,
                              double* __restrict__ min_margin, const double* __restrict__ fv = nullptr) {
    __shared__ double V[16 * 16];
    __shared__ double Tm[16 * 16];
    __shared__ double red[8];
    const int b = blockIdx.x;
    const double mx = box_tail(g, src, level, keys[b], C, V, Tm, red, fv ? fv + (size_t)b * g.k * g.k : nullptr);
    if (threadIdx.x == 0 && b < n) {
        flags[b] = mx > thresh ? 1 : 0;
        if (thresh > 0.0) atomic_min_nonneg(min_margin, fabs(mx / thresh - 1.0));
    }
}

// The a-priori rules of Section 6.1: one CTA (4k^2 threads) per candidate box. e = max |f - p| over
// the nodes of the box's four children, p the interpolant of f on the box's own nodes
// (L: [2k][k] Lagrange basis of the own nodes at the children's node positions); weighted by 1
// (rule 1), (h/W)^2 (rule 2), or (h/W)^2 where the source's boundary level set takes both signs on
// those nodes and h/W elsewhere (rule 3); split flag = weighted e > thresh.
__global__ void __launch_bounds__(1024) interp_rule_kernel(NodeGeom g, SourceDev src, int level,
                                                           const uint32_t* __restrict__ keys, int n,
                                                           const double* __restrict__ L, int rule, double thresh,
                                                           int32_t* __restrict__ flags,
                                                           double* __restrict__ min_margin) {
    __shared__ double V[16 * 16];
    __shared__ double R[16 * 32];
    __shared__ double Ls[32 * 16];
    __shared__ double red[32];
    __shared__ int pos, nonpos;
    const int k = g.k, K2 = 2 * k, t = threadIdx.x;
    const int b = blockIdx.x;
    int ix, iy;
    morton_decode(keys[b], &ix, &iy);
    const double h = ldexp(g.width, -level), hc = ldexp(g.width, -(level + 1));
    if (t == 0) {
        pos = 0;
        nonpos = 0;
    }
    bool p_pos = false, p_non = false;
    if (t < k * k) {
        const double x = node_coord(g.lox, ix, g.xhat[t % k], h), y = node_coord(g.loy, iy, g.xhat[t / k], h);
        V[t] = source_eval(src, x, y);
        const double ph = source_phi(src, x, y);
        p_pos = ph > 0.0;
        p_non = !(ph > 0.0);
    }
    if (t < K2 * k) Ls[t] = L[t];
    double fc = 0.0;
    const bool active = t < K2 * K2;
    const int J = t / K2, I = t % K2;
    if (active) {
        const int c = I / k, i = I % k, d = J / k, j = J % k;
        const double x = node_coord(g.lox, 2 * ix + c, g.xhat[i], hc), y = node_coord(g.loy, 2 * iy + d, g.xhat[j], hc);
        fc = source_eval(src, x, y);
        const double ph = source_phi(src, x, y);
        p_pos = p_pos || ph > 0.0;
        p_non = p_non || !(ph > 0.0);
    }
    __syncthreads();
    if (p_pos) pos = 1;
    if (p_non) nonpos = 1;
    if (t < k * K2) {  // R[j][I] = sum_i V[j][i] L[I][i]
        const int j = t / K2, Ii = t % K2;
        double acc = 0.0;
        for (int i = 0; i < k; ++i) acc += V[j * k + i] * Ls[Ii * k + i];
        R[t] = acc;
    }
    __syncthreads();
    double e = 0.0;
    if (active) {
        double p = 0.0;
        for (int j = 0; j < k; ++j) p += Ls[J * k + j] * R[j * K2 + I];
        e = fabs(fc - p);
    }
    for (int o = 16; o > 0; o >>= 1) e = fmax(e, __shfl_xor_sync(0xffffffffu, e, o));
    if ((t & 31) == 0) red[t >> 5] = e;
    __syncthreads();
    if (t == 0 && b < n) {
        double mx = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
        const double side = ldexp(1.0, -level);
        double ind = mx;
        if (rule == 2 || (rule == 3 && pos && nonpos)) ind = mx * side * side;
        else if (rule == 3) ind = mx * side;
        flags[b] = ind > thresh ? 1 : 0;
        if (thresh > 0.0) atomic_min_nonneg(min_margin, fabs(ind / thresh - 1.0));
    }
}

// One CTA per box of a list with per-box levels: tails[b] = box_tail.
__global__ void tail_kernel(NodeGeom g, SourceDev src, const int32_t* __restrict__ lev,
                            const uint32_t* __restrict__ keys, int n, const double* __restrict__ C,
                            double* __restrict__ tails, const double* __restrict__ fv) {
    __shared__ double V[16 * 16];
    __shared__ double Tm[16 * 16];
    __shared__ double red[8];
    const int b = blockIdx.x;
    const double mx = box_tail(g, src, lev[b], keys[b], C, V, Tm, red, fv + (size_t)b * g.k * g.k);
    if (threadIdx.x == 0 && b < n) tails[b] = mx;
}

__global__ void fill_kernel(int32_t* a, int64_t n, int32_t v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

__global__ void emit_children_kernel(const uint32_t* __restrict__ keys, const int32_t* __restrict__ flags,
                                     const int32_t* __restrict__ offs, int n, uint32_t* __restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !flags[i]) return;
    uint32_t base = keys[i] << 2;
    int o = offs[i] * 4;
    for (int c = 0; c < 4; ++c) out[o + c] = base | (uint32_t)c;
}

__global__ void children_of_kernel(const uint32_t* __restrict__ parents, int n, uint32_t* __restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t base = parents[i] << 2;
    for (int c = 0; c < 4; ++c) out[4 * i + c] = base | (uint32_t)c;
}

// ---------------------------------------------------------------- level restriction
// Marks in the level-(l-2) bitmap: parents of every level-(l-1) box, and the
// parents of every level-(l-1) cell adjacent to a level-l box (and of its parent).
__global__ void balance_mark_kernel(const uint32_t* __restrict__ keys_l, int n_l,
                                    const uint32_t* __restrict__ keys_lm1, int n_lm1, int l,
                                    uint32_t* __restrict__ bitmap) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_lm1) {
        uint32_t pk = keys_lm1[i] >> 2;
        atomicOr(&bitmap[pk >> 5], 1u << (pk & 31));
    }
    if (i < n_l) {
        int bx, by;
        morton_decode(keys_l[i], &bx, &by);
        int px = bx >> 1, py = by >> 1;
        int side = 1 << (l - 1);
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int qx = px + dx, qy = py + dy;
                if (qx < 0 || qy < 0 || qx >= side || qy >= side) continue;
                if ((dx || dy) && !boxes_adjacent(l - 1, qx, qy, l, bx, by)) continue;
                uint32_t pk = morton_encode((uint32_t)qx, (uint32_t)qy) >> 2;
                atomicOr(&bitmap[pk >> 5], 1u << (pk & 31));
            }
    }
}

__global__ void popc_kernel(const uint32_t* __restrict__ bm, int64_t nw, int32_t* __restrict__ cnt) {
    int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w < nw) cnt[w] = __popc(bm[w]);
}

__global__ void bitmap_emit_kernel(const uint32_t* __restrict__ bm, int64_t nw, const int32_t* __restrict__ offs,
                                   uint32_t* __restrict__ out) {
    int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nw) return;
    uint32_t bits = bm[w];
    int pos = offs[w];
    while (bits) {
        int b = __ffs(bits) - 1;
        out[pos++] = (uint32_t)(w * 32 + b);
        bits &= bits - 1;
    }
}

// ---------------------------------------------------------------- finalisation
__device__ inline int lower_bound_key(const uint32_t* key, int lo, int hi, uint32_t k) {
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (key[mid] < k) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ inline int find_box(const uint32_t* key, const int32_t* lstart, int depth, int l, int x, int y) {
    if (l < 0 || l > depth) return -1;
    int side = 1 << l;
    if (x < 0 || y < 0 || x >= side || y >= side) return -1;
    uint32_t k = morton_encode((uint32_t)x, (uint32_t)y);
    int lo = lstart[l], hi = lstart[l + 1];
    int p = lower_bound_key(key, lo, hi, k);
    return (p < hi && key[p] == k) ? p : -1;
}

__global__ void box_setup_kernel(const uint32_t* __restrict__ key, const int32_t* __restrict__ lstart, int depth,
                                 int n, int32_t* level, int32_t* ix, int32_t* iy, int32_t* parent, int32_t* child0,
                                 int32_t* is_leaf) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    int l = 0;
    while (l < depth && b >= lstart[l + 1]) ++l;
    int x, y;
    morton_decode(key[b], &x, &y);
    level[b] = l;
    ix[b] = x;
    iy[b] = y;
    parent[b] = l > 0 ? find_box(key, lstart, depth, l - 1, x >> 1, y >> 1) : -1;
    int c = l < depth ? find_box(key, lstart, depth, l + 1, 2 * x, 2 * y) : -1;
    child0[b] = c;
    is_leaf[b] = c < 0 ? 1 : 0;
}

__global__ void leaf_rank_kernel(const int32_t* __restrict__ is_leaf, const int32_t* __restrict__ rank, int n,
                                 int32_t* __restrict__ leaf_of_box, int32_t* __restrict__ box_of_leaf) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    if (is_leaf[b]) {
        leaf_of_box[b] = rank[b];
        box_of_leaf[rank[b]] = b;
    } else {
        leaf_of_box[b] = -1;
    }
}

// ---------------------------------------------------------------- lists
struct TreeView {
    const uint32_t* key;
    const int32_t* lstart;
    const int32_t* level;
    const int32_t* ix;
    const int32_t* iy;
    const int32_t* parent;
    const int32_t* child0;
    int depth;
};

struct Entries {
    int n[4];
    int idx[4][27];
    int cfg[4][27];
    __device__ void add(int list, int box, int c) {
        idx[list][n[list]] = box;
        cfg[list][n[list]] = c;
        ++n[list];
    }
};

__device__ inline void collect_lists(const TreeView& T, int b, Entries& E) {
    E.n[0] = E.n[1] = E.n[2] = E.n[3] = 0;
    const int l = T.level[b], a = T.ix[b], c = T.iy[b];
    const bool leaf = T.child0[b] < 0;
    int dx4, dy4;
    if (leaf) {
        E.add(VFMM_LIST_U, b, 4);
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (!dx && !dy) continue;
                int q = find_box(T.key, T.lstart, T.depth, l, a + dx, c + dy);
                if (q < 0) continue;
                if (T.child0[q] < 0) {
                    E.add(VFMM_LIST_U, q, (dy + 1) * 3 + (dx + 1));
                } else {
                    for (int s = 0; s < 4; ++s) {
                        int ch = T.child0[q] + s;
                        centre_offset4(l, a, c, l + 1, T.ix[ch], T.iy[ch], &dx4, &dy4);
                        if (boxes_adjacent(l, a, c, l + 1, T.ix[ch], T.iy[ch]))
                            E.add(VFMM_LIST_U, ch, 21 + near_pattern_index(dx4, dy4));
                        else
                            E.add(VFMM_LIST_W, ch, far_pattern_index(dx4, dy4));
                    }
                }
            }
        if (l >= 1) {
            int pa = a >> 1, pc = c >> 1;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if (!dx && !dy) continue;
                    int q = find_box(T.key, T.lstart, T.depth, l - 1, pa + dx, pc + dy);
                    if (q < 0 || T.child0[q] >= 0) continue;
                    if (!boxes_adjacent(l, a, c, l - 1, pa + dx, pc + dy)) continue;
                    centre_offset4(l, a, c, l - 1, pa + dx, pc + dy, &dx4, &dy4);
                    E.add(VFMM_LIST_U, q, 9 + near_pattern_index(dx4 / 2, dy4 / 2));
                }
        }
    }
    if (l >= 2) {
        int pa = a >> 1, pc = c >> 1;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int q = find_box(T.key, T.lstart, T.depth, l - 1, pa + dx, pc + dy);
                if (q < 0) continue;
                if (T.child0[q] < 0) {
                    if ((dx || dy) && !boxes_adjacent(l, a, c, l - 1, pa + dx, pc + dy)) {
                        centre_offset4(l, a, c, l - 1, pa + dx, pc + dy, &dx4, &dy4);
                        E.add(VFMM_LIST_X, q, far_pattern_index(dx4 / 2, dy4 / 2));
                    }
                    continue;
                }
                for (int s = 0; s < 4; ++s) {
                    int ch = T.child0[q] + s;
                    if (ch == b || boxes_adjacent(l, a, c, l, T.ix[ch], T.iy[ch])) continue;
                    E.add(VFMM_LIST_V, ch, v_offset_index(T.ix[ch] - a, T.iy[ch] - c));
                }
            }
    }
}

__global__ void list_count_kernel(TreeView T, int n, int32_t* __restrict__ cnt) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    Entries E;
    collect_lists(T, b, E);
    for (int q = 0; q < 4; ++q) cnt[(int64_t)q * n + b] = E.n[q];
}

__global__ void list_fill_kernel(TreeView T, int n, const int32_t* __restrict__ off, int32_t* __restrict__ idxU,
                                 int32_t* __restrict__ cfgU, int32_t* __restrict__ idxV, int32_t* __restrict__ cfgV,
                                 int32_t* __restrict__ idxW, int32_t* __restrict__ cfgW, int32_t* __restrict__ idxX,
                                 int32_t* __restrict__ cfgX) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    Entries E;
    collect_lists(T, b, E);
    int32_t* idxs[4] = {idxU, idxV, idxW, idxX};
    int32_t* cfgs[4] = {cfgU, cfgV, cfgW, cfgX};
    for (int q = 0; q < 4; ++q) {
        // insertion sort by box index
        for (int i = 1; i < E.n[q]; ++i) {
            int vi = E.idx[q][i], vc = E.cfg[q][i], j = i - 1;
            while (j >= 0 && E.idx[q][j] > vi) {
                E.idx[q][j + 1] = E.idx[q][j];
                E.cfg[q][j + 1] = E.cfg[q][j];
                --j;
            }
            E.idx[q][j + 1] = vi;
            E.cfg[q][j + 1] = vc;
        }
        int o = off[(int64_t)q * n + b];
        for (int i = 0; i < E.n[q]; ++i) {
            idxs[q][o + i] = E.idx[q][i];
            cfgs[q][o + i] = E.cfg[q][i];
        }
    }
}

__global__ void ptr_from_offsets_kernel(const int32_t* __restrict__ off, int n, int64_t total, int32_t* __restrict__ ptr) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < n) ptr[b] = off[b];
    if (b == n) ptr[n] = (int32_t)total;
}

__global__ void shift_kernel(int32_t* a, int64_t n, int32_t s) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] -= s;
}

__global__ void cfg_flags_kernel(const int32_t* __restrict__ cfg, int64_t n, int ncfg, int32_t* __restrict__ flags) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    int c = cfg[e];
    for (int j = 0; j < ncfg; ++j) flags[(int64_t)j * n + e] = (j == c) ? 1 : 0;
}

__global__ void cfg_scatter_kernel(const int32_t* __restrict__ cfg, const int32_t* __restrict__ pos, int64_t n,
                                   int32_t* __restrict__ out) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    out[pos[(int64_t)cfg[e] * n + e]] = (int32_t)e;
}

__global__ void entry_target_kernel(const int32_t* __restrict__ ptr, int n, int32_t* __restrict__ tgt) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    for (int e = ptr[b]; e < ptr[b + 1]; ++e) tgt[e] = b;
}

static inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// ---------------------------------------------------------------- host orchestration
struct BuildCtx {
    cudaStream_t st;
    bool keep = false;  // tables outlive the call (a builder): cudaMalloc instead of the build pool
    NodeGeom g;
    DBuf<double> xhat;
    DBuf<double> C;
    DBuf<double> L;  // [2k][k] Lagrange basis of a box's nodes at its children's nodes (Section 6.1 rules)
};

static int upload_node_tables(int k, BuildCtx& B) {
    std::vector<double> xh(k), C(k * k);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < k; ++i) xh[i] = -std::cos(pi * (2.0 * i + 1.0) / (2.0 * k)) / 2.0;
    for (int m = 0; m < k; ++m)
        for (int i = 0; i < k; ++i) {
            double t = 2.0 * xh[i];
            double v = std::cos(m * std::acos(std::min(1.0, std::max(-1.0, t))));
            C[m * k + i] = (m == 0 ? 1.0 : 2.0) / k * v;
        }
    VFMM_CHECK(B.keep ? B.xhat.alloc_keep(k) : B.xhat.alloc(k, B.st));
    VFMM_CHECK(B.keep ? B.C.alloc_keep(k * k) : B.C.alloc(k * k, B.st));
    VFMM_CUDA(cudaMemcpyAsync(B.xhat.p, xh.data(), k * sizeof(double), cudaMemcpyHostToDevice, B.st));
    VFMM_CUDA(cudaMemcpyAsync(B.C.p, C.data(), k * k * sizeof(double), cudaMemcpyHostToDevice, B.st));
    return VFMM_OK;
}

// L[I][i] = l_i(u_I): the Lagrange basis of the k nodes x_i on [-1/2, 1/2] at the positions
// u_I = -1/4 + x_I / 2 (I < k) and 1/4 + x_{I-k} / 2 of the children's nodes, product formula.
static int upload_child_basis(int k, BuildCtx& B) {
    std::vector<double> x(k), L(2 * k * k);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < k; ++i) x[i] = -std::cos(pi * (2.0 * i + 1.0) / (2.0 * k)) / 2.0;
    for (int I = 0; I < 2 * k; ++I) {
        const double u = (I < k ? -0.25 : 0.25) + x[I % k] / 2.0;
        for (int i = 0; i < k; ++i) {
            double num = 1.0, den = 1.0;
            for (int m = 0; m < k; ++m)
                if (m != i) {
                    num *= u - x[m];
                    den *= x[i] - x[m];
                }
            L[I * k + i] = num / den;
        }
    }
    VFMM_CHECK(B.keep ? B.L.alloc_keep(2 * k * k) : B.L.alloc(2 * k * k, B.st));
    VFMM_CUDA(cudaMemcpyAsync(B.L.p, L.data(), L.size() * sizeof(double), cudaMemcpyHostToDevice, B.st));
    return VFMM_OK;
}

// out[c] = in[c * stride], c < n.
__global__ void strided_gather_kernel(const int32_t* __restrict__ in, int64_t stride, int n, int32_t* __restrict__ out) {
    for (int c = threadIdx.x; c < n; c += blockDim.x) out[c] = in[(int64_t)c * stride];
}

static int compute_lists(DeviceTree* T, cudaStream_t st) {
    const int n = T->n_boxes;
    TreeView V{T->key, T->level_start_dev, T->level, T->ix, T->iy, T->parent, T->child0, T->depth};
    DBuf<int32_t> cnt;
    VFMM_CHECK(cnt.alloc((size_t)4 * n, st));
    // 32 threads per CTA: each thread keeps its box's candidate entries (about 1 KB) in local memory,
    // which then stays in L1, and the boxes spread over more SMs
    list_count_kernel<<<nblk(n, 32), 32, 0, st>>>(V, n, cnt.p);
    VFMM_CUDA(cudaGetLastError());
    // one scan over the 4 concatenated count arrays; row q starts at total of rows < q
    int64_t total = 0;
    VFMM_CHECK(exclusive_scan(cnt.p, cnt.p, (int64_t)4 * n, &total, st));
    int32_t starts[5];
    for (int q = 0; q < 4; ++q)
        VFMM_CUDA(cudaMemcpyAsync(&starts[q], cnt.p + (int64_t)q * n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    VFMM_CUDA(cudaStreamSynchronize(st));
    starts[4] = (int32_t)total;
    DBuf<int32_t> idx[4], cfg[4], ptr[4];
    for (int q = 0; q < 4; ++q) {
        T->llen[q] = starts[q + 1] - starts[q];
        VFMM_CHECK(idx[q].alloc_tree(std::max<int64_t>(1, T->llen[q]), st));
        VFMM_CHECK(cfg[q].alloc_tree(std::max<int64_t>(1, T->llen[q]), st));
        VFMM_CHECK(ptr[q].alloc_tree(n + 1, st));
    }
    // offsets within each list: subtract the row start
    for (int q = 0; q < 4; ++q) {
        shift_kernel<<<nblk(n), 256, 0, st>>>(cnt.p + (int64_t)q * n, n, starts[q]);
        ptr_from_offsets_kernel<<<nblk(n + 1), 256, 0, st>>>(cnt.p + (int64_t)q * n, n, T->llen[q], ptr[q].p);
    }
    list_fill_kernel<<<nblk(n, 32), 32, 0, st>>>(V, n, cnt.p, idx[0].p, cfg[0].p, idx[1].p, cfg[1].p, idx[2].p,
                                                   cfg[2].p, idx[3].p, cfg[3].p);
    VFMM_CUDA(cudaGetLastError());
    for (int q = 0; q < 4; ++q) {
        T->lidx[q] = idx[q].release();
        T->lcfg[q] = cfg[q].release();
        T->lptr[q] = ptr[q].release();
    }
    // U entries grouped by configuration, stable (flattened config-major scan)
    const int64_t nU = T->llen[VFMM_LIST_U];
    DBuf<int32_t> flags, byc, tgt;
    VFMM_CHECK(flags.alloc((size_t)kNearCfg * nU, st));
    VFMM_CHECK(byc.alloc_tree(std::max<int64_t>(1, nU), st));
    VFMM_CHECK(tgt.alloc_tree(std::max<int64_t>(1, nU), st));
    cfg_flags_kernel<<<nblk(nU), 256, 0, st>>>(T->lcfg[0], nU, kNearCfg, flags.p);
    VFMM_CUDA(cudaGetLastError());
    int64_t tot = 0;
    VFMM_CHECK(exclusive_scan(flags.p, flags.p, (int64_t)kNearCfg * nU, &tot, st));
    cfg_scatter_kernel<<<nblk(nU), 256, 0, st>>>(T->lcfg[0], flags.p, nU, byc.p);
    entry_target_kernel<<<nblk(n), 256, 0, st>>>(T->lptr[0], n, tgt.p);
    VFMM_CUDA(cudaGetLastError());
    // first entry of each configuration: flags[c * nU], gathered and read back once
    T->u_cfg_start.assign(kNearCfg + 1, 0);
    if (nU > 0) {
        DBuf<int32_t> starts_dev;
        VFMM_CHECK(starts_dev.alloc(kNearCfg, st));
        strided_gather_kernel<<<1, 64, 0, st>>>(flags.p, nU, kNearCfg, starts_dev.p);
        VFMM_CUDA(cudaGetLastError());
        int32_t h[kNearCfg];
        VFMM_CUDA(cudaMemcpyAsync(h, starts_dev.p, kNearCfg * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        VFMM_CUDA(cudaStreamSynchronize(st));
        for (int c = 0; c < kNearCfg; ++c) T->u_cfg_start[c] = h[c];
    }
    T->u_cfg_start[kNearCfg] = nU;
    T->u_by_cfg = byc.release();
    T->u_tgt = tgt.release();
    return VFMM_OK;
}

// Greedy refinement to a leaf count (no counterpart in the paper, which refines to a
// tolerance): starting from the root, the leaf of highest priority is split, one at a time,
// until there are at least n_target leaves (before balancing) or no leaf above max_depth is
// left. Priority = the binary exponent e of the leaf's tail (tail in [2^(e-1), 2^e)), raised to
// at least e_F - 30 (F = 2^e_F m, m in [0.5, 1)) so that tails near rounding level all tie; ties
// go to the coarser leaf, then the smaller Morton key. The host keeps the priority queue and
// asks the device for the tails of the children of the leaves most likely to be split next,
// in batches, so the order of splits is exactly the one-at-a-time order.
// lv[l] = sorted keys of every box of level l; *min_margin = smallest relative distance of a
// tail that decided a priority to the nearest power of two.
static int greedy_refine(const BuildCtx& B, const SourceDev& src, int max_depth, int64_t n_target, double F,
                         std::vector<std::vector<uint32_t>>& lv, double* min_margin) {
    typedef std::tuple<int, int, uint32_t> Item;  // (-priority, level, key): std::set begins with the next split
    int eF = 0;
    if (F > 0.0) std::frexp(F, &eF);
    const int e_floor = eF - 30;
    auto priority = [&](double t, double* margin) {
        int e = e_floor;
        if (t > 0.0) {
            std::frexp(t, &e);
            if (e >= e_floor) {
                const double lo = std::ldexp(1.0, e - 1), hi = std::ldexp(1.0, e);
                *margin = std::min(*margin, std::min(t / lo - 1.0, 1.0 - t / hi));
            }
        }
        return std::max(e, e_floor);
    };
    auto id = [](int level, uint32_t key) { return ((uint64_t)level << 32) | key; };
    std::unordered_map<uint64_t, std::array<double, 4>> kid_tails;
    const int threads = ((B.g.k * B.g.k + 31) / 32) * 32;
    auto compute = [&](const std::vector<int32_t>& lev, const std::vector<uint32_t>& key, std::vector<double>& out) {
        const int n = (int)key.size();
        DBuf<int32_t> dl;
        DBuf<uint32_t> dk;
        DBuf<double> dt;
        DBuf<double> fv;
        const int64_t nv = (int64_t)n * B.g.k * B.g.k;
        VFMM_CHECK(dl.alloc(n, B.st));
        VFMM_CHECK(dk.alloc(n, B.st));
        VFMM_CHECK(dt.alloc(n, B.st));
        VFMM_CHECK(fv.alloc(nv, B.st));
        VFMM_CUDA(cudaMemcpyAsync(dl.p, lev.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, B.st));
        VFMM_CUDA(cudaMemcpyAsync(dk.p, key.data(), n * sizeof(uint32_t), cudaMemcpyHostToDevice, B.st));
        node_values_kernel<<<(unsigned)((nv + 63) / 64), 64, 0, B.st>>>(B.g, src, 0, dl.p, dk.p, n, fv.p);
        tail_kernel<<<(unsigned)n, threads, 0, B.st>>>(B.g, src, dl.p, dk.p, n, B.C.p, dt.p, fv.p);
        VFMM_CUDA(cudaGetLastError());
        out.resize(n);
        VFMM_CUDA(cudaMemcpyAsync(out.data(), dt.p, n * sizeof(double), cudaMemcpyDeviceToHost, B.st));
        VFMM_CUDA(cudaStreamSynchronize(B.st));
        return VFMM_OK;
    };
    lv.assign(1, std::vector<uint32_t>{0u});
    std::vector<double> tails;
    VFMM_CHECK(compute({0}, {0u}, tails));
    std::set<Item> frontier;
    if (max_depth > 0) frontier.insert(Item(-priority(tails[0], min_margin), 0, 0u));
    int64_t n_leaves = 1;
    while (n_leaves < n_target && !frontier.empty()) {
        const Item top = *frontier.begin();
        if (!kid_tails.count(id(std::get<1>(top), std::get<2>(top)))) {
            // children of the next leaves in queue order whose children are not known yet
            const int64_t want = std::max<int64_t>(64, (n_target - n_leaves + 2) / 3);
            std::vector<int32_t> lev;
            std::vector<uint32_t> key;
            std::vector<uint64_t> parents;
            for (auto it = frontier.begin(); it != frontier.end() && (int64_t)parents.size() < want; ++it) {
                const int l = std::get<1>(*it);
                const uint32_t kp = std::get<2>(*it);
                if (kid_tails.count(id(l, kp))) continue;
                parents.push_back(id(l, kp));
                for (uint32_t c = 0; c < 4; ++c) {
                    lev.push_back(l + 1);
                    key.push_back((kp << 2) | c);
                }
            }
            VFMM_CHECK(compute(lev, key, tails));
            for (size_t q = 0; q < parents.size(); ++q)
                kid_tails[parents[q]] = {tails[4 * q], tails[4 * q + 1], tails[4 * q + 2], tails[4 * q + 3]};
        }
        frontier.erase(frontier.begin());
        const int l = std::get<1>(top);
        const uint32_t kp = std::get<2>(top);
        const std::array<double, 4> kt = kid_tails[id(l, kp)];
        if ((int)lv.size() < l + 2) lv.emplace_back();
        for (uint32_t c = 0; c < 4; ++c) {
            const uint32_t kc = (kp << 2) | c;
            lv[l + 1].push_back(kc);
            const int pr = priority(kt[c], min_margin);
            if (l + 1 < max_depth) frontier.insert(Item(-pr, l + 1, kc));
        }
        n_leaves += 3;
    }
    for (auto& v : lv) std::sort(v.begin(), v.end());
    return VFMM_OK;
}

static int finalize(std::vector<DBuf<uint32_t>>& keys, std::vector<int64_t>& cnt, int depth, cudaStream_t st,
                    DeviceTree* T);

// Builds the tree. src == nullptr means a uniform tree of depth `uniform_depth`; leaf_target > 0
// selects the greedy leaf-count refinement instead of the tolerance test.
static int build(const vfmm_tree_params* prm, const SourceDev* src, int uniform_depth, int64_t leaf_target,
                 cudaStream_t st, DeviceTree* T, int rule = VFMM_REFINE_TAIL) {
    const int k = prm->k;
    BuildCtx B;
    B.st = st;
    VFMM_CHECK(upload_node_tables(k, B));
    B.g = NodeGeom{prm->cx - prm->width / 2.0, prm->cy - prm->width / 2.0, prm->width, k, B.xhat.p};
    const bool uniform = src == nullptr;
    const int max_depth = uniform ? uniform_depth : prm->max_depth;
    const int min_depth = uniform ? uniform_depth : prm->min_depth;

    T->k = k;
    T->cx = prm->cx;
    T->cy = prm->cy;
    T->width = prm->width;

    DBuf<double> scal;  // [0] = F, [1] = min margin, [2] = margin sink of the depth-cap test
    VFMM_CHECK(scal.alloc(3, st));
    double init[3] = {0.0, INFINITY, INFINITY};
    VFMM_CUDA(cudaMemcpyAsync(scal.p, init, sizeof(init), cudaMemcpyHostToDevice, st));
    double thresh = 0.0;
    int m0 = -1;              // level of the f-scale grid
    DBuf<double> grid_m0;     // f at every node of that level (tail refinement only)
    if (!uniform) {
        m0 = std::min(5, max_depth);
        if (rule == VFMM_REFINE_TAIL && leaf_target <= 0) VFMM_CHECK(grid_m0.alloc((size_t)k * k << (2 * m0), st));
        fscale_kernel<<<1u << (2 * m0), 128, 0, st>>>(B.g, *src, m0, scal.p, grid_m0.p);
        VFMM_CUDA(cudaGetLastError());
        VFMM_CUDA(cudaMemcpyAsync(&T->f_scale, scal.p, sizeof(double), cudaMemcpyDeviceToHost, st));
        VFMM_CUDA(cudaStreamSynchronize(st));
        thresh = prm->tol * T->f_scale;
    }

    std::vector<DBuf<uint32_t>> keys(max_depth + 1);
    std::vector<int64_t> cnt(max_depth + 1, 0);
    int depth = 0;
    if (leaf_target > 0) {
        std::vector<std::vector<uint32_t>> lv;
        double mm = INFINITY;
        VFMM_CHECK(greedy_refine(B, *src, max_depth, leaf_target, T->f_scale, lv, &mm));
        depth = (int)lv.size() - 1;
        for (int l = 0; l <= depth; ++l) {
            cnt[l] = (int64_t)lv[l].size();
            VFMM_CHECK(keys[l].alloc(cnt[l], st));
            VFMM_CUDA(cudaMemcpy(keys[l].p, lv[l].data(), cnt[l] * sizeof(uint32_t), cudaMemcpyHostToDevice));
        }
        T->min_margin = mm;
        T->n_capped = -1;  // refined to a leaf count, not to the test
    } else {
        VFMM_CHECK(keys[0].alloc(1, st));
        uint32_t zero = 0;
        VFMM_CUDA(cudaMemcpyAsync(keys[0].p, &zero, sizeof(uint32_t), cudaMemcpyHostToDevice, st));
        cnt[0] = 1;
        for (int l = 0; l < max_depth; ++l) {
            const int64_t n = cnt[l];
            DBuf<int32_t> flags, offs;
            DBuf<double> vals;
            VFMM_CHECK(flags.alloc(n, st));
            VFMM_CHECK(offs.alloc(n, st));
            if (l < min_depth) {
                fill_kernel<<<nblk(n), 256, 0, st>>>(flags.p, n, 1);
            } else if (rule == VFMM_REFINE_TAIL) {
                VFMM_CHECK(vals.alloc(n * k * k, st));
                if (l == m0 && grid_m0.p)
                    grid_values_kernel<<<(unsigned)((n * k * k + 255) / 256), 256, 0, st>>>(grid_m0.p, l, k * k,
                                                                                           keys[l].p, (int)n, vals.p);
                else
                    node_values_kernel<<<(unsigned)((n * k * k + 63) / 64), 64, 0, st>>>(B.g, *src, l, nullptr,
                                                                                        keys[l].p, (int)n, vals.p);
                refine_kernel<<<(unsigned)n, ((k * k + 31) / 32) * 32, 0, st>>>(B.g, *src, l, keys[l].p, (int)n, B.C.p,
                                                                                 thresh, flags.p, scal.p + 1, vals.p);
            } else {
                if (!B.L.p) VFMM_CHECK(upload_child_basis(k, B));
                interp_rule_kernel<<<(unsigned)n, ((4 * k * k + 31) / 32) * 32, 0, st>>>(
                    B.g, *src, l, keys[l].p, (int)n, B.L.p, rule, thresh, flags.p, scal.p + 1);
            }
            VFMM_CUDA(cudaGetLastError());
            int64_t m = 0;
            VFMM_CHECK(exclusive_scan(flags.p, offs.p, n, &m, st));
            if (m == 0) break;
            VFMM_CHECK(keys[l + 1].alloc(4 * m, st));
            emit_children_kernel<<<nblk(n), 256, 0, st>>>(keys[l].p, flags.p, offs.p, (int)n, keys[l + 1].p);
            VFMM_CUDA(cudaGetLastError());
            cnt[l + 1] = 4 * m;
            depth = l + 1;
        }
        if (!uniform) {
            double mm = 0;
            VFMM_CUDA(cudaMemcpyAsync(&mm, scal.p + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
            VFMM_CUDA(cudaStreamSynchronize(st));
            T->min_margin = mm;
            // leaves the depth cap stopped: the split test on the boxes of level max_depth
            const int64_t nc = cnt[max_depth];
            T->n_capped = 0;
            if (nc > 0) {
                DBuf<int32_t> cf, co;
                VFMM_CHECK(cf.alloc(nc, st));
                VFMM_CHECK(co.alloc(nc, st));
                if (rule == VFMM_REFINE_TAIL) {
                    DBuf<double> vals;
                    VFMM_CHECK(vals.alloc(nc * k * k, st));
                    node_values_kernel<<<(unsigned)((nc * k * k + 63) / 64), 64, 0, st>>>(
                        B.g, *src, max_depth, nullptr, keys[max_depth].p, (int)nc, vals.p);
                    refine_kernel<<<(unsigned)nc, ((k * k + 31) / 32) * 32, 0, st>>>(
                        B.g, *src, max_depth, keys[max_depth].p, (int)nc, B.C.p, thresh, cf.p, scal.p + 2, vals.p);
                } else {
                    if (!B.L.p) VFMM_CHECK(upload_child_basis(k, B));
                    interp_rule_kernel<<<(unsigned)nc, ((4 * k * k + 31) / 32) * 32, 0, st>>>(
                        B.g, *src, max_depth, keys[max_depth].p, (int)nc, B.L.p, rule, thresh, cf.p, scal.p + 2);
                }
                VFMM_CUDA(cudaGetLastError());
                VFMM_CHECK(exclusive_scan(cf.p, co.p, nc, &T->n_capped, st));
            }
        }
    }

    return finalize(keys, cnt, depth, st, T);
}

// Balance (2:1, finest level first), canonical numbering, lists and schedules of a refined tree
// given its boxes per level (T's root geometry, k, f scale and margin already set).
static int finalize(std::vector<DBuf<uint32_t>>& keys, std::vector<int64_t>& cnt, int depth, cudaStream_t st,
                    DeviceTree* T) {
    // level restriction, finest level first
    for (int l = depth; l >= 2; --l) {
        const int m = l - 2;
        const int64_t nbits = 1ll << (2 * m);
        const int64_t nw = std::max<int64_t>(1, nbits / 32);
        DBuf<uint32_t> bm;
        DBuf<int32_t> wc;
        VFMM_CHECK(bm.alloc(nw, st));
        VFMM_CHECK(wc.alloc(nw, st));
        VFMM_CUDA(cudaMemsetAsync(bm.p, 0, nw * sizeof(uint32_t), st));
        int64_t nmax = std::max(cnt[l], cnt[l - 1]);
        balance_mark_kernel<<<nblk(nmax), 256, 0, st>>>(keys[l].p, (int)cnt[l], keys[l - 1].p, (int)cnt[l - 1], l,
                                                        bm.p);
        popc_kernel<<<nblk(nw), 256, 0, st>>>(bm.p, nw, wc.p);
        VFMM_CUDA(cudaGetLastError());
        int64_t ns = 0;
        VFMM_CHECK(exclusive_scan(wc.p, wc.p, nw, &ns, st));
        DBuf<uint32_t> split;
        VFMM_CHECK(split.alloc(ns, st));
        bitmap_emit_kernel<<<nblk(nw), 256, 0, st>>>(bm.p, nw, wc.p, split.p);
        VFMM_CHECK(keys[l - 1].alloc(4 * ns, st));
        children_of_kernel<<<nblk(ns), 256, 0, st>>>(split.p, (int)ns, keys[l - 1].p);
        VFMM_CUDA(cudaGetLastError());
        cnt[l - 1] = 4 * ns;
    }

    // canonical numbering
    T->depth = depth;
    T->level_start.assign(depth + 2, 0);
    for (int l = 0; l <= depth; ++l) T->level_start[l + 1] = T->level_start[l] + (int32_t)cnt[l];
    const int n = T->level_start[depth + 1];
    T->n_boxes = n;
    DBuf<uint32_t> key;
    DBuf<int32_t> level, ix, iy, parent, child0, isleaf, rank, lob, bol, lsd;
    VFMM_CHECK(key.alloc_tree(n, st));
    VFMM_CHECK(level.alloc_tree(n, st));
    VFMM_CHECK(ix.alloc_tree(n, st));
    VFMM_CHECK(iy.alloc_tree(n, st));
    VFMM_CHECK(parent.alloc_tree(n, st));
    VFMM_CHECK(child0.alloc_tree(n, st));
    VFMM_CHECK(isleaf.alloc(n, st));
    VFMM_CHECK(rank.alloc(n, st));
    VFMM_CHECK(lob.alloc_tree(n, st));
    VFMM_CHECK(lsd.alloc_tree(depth + 2, st));
    for (int l = 0; l <= depth; ++l)
        VFMM_CUDA(cudaMemcpyAsync(key.p + T->level_start[l], keys[l].p, cnt[l] * sizeof(uint32_t),
                                  cudaMemcpyDeviceToDevice, st));
    VFMM_CUDA(cudaMemcpyAsync(lsd.p, T->level_start.data(), (depth + 2) * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    box_setup_kernel<<<nblk(n), 256, 0, st>>>(key.p, lsd.p, depth, n, level.p, ix.p, iy.p, parent.p, child0.p,
                                              isleaf.p);
    VFMM_CUDA(cudaGetLastError());
    int64_t nleaf = 0;
    VFMM_CHECK(exclusive_scan(isleaf.p, rank.p, n, &nleaf, st));
    VFMM_CHECK(bol.alloc_tree(nleaf, st));
    leaf_rank_kernel<<<nblk(n), 256, 0, st>>>(isleaf.p, rank.p, n, lob.p, bol.p);
    VFMM_CUDA(cudaGetLastError());
    T->n_leaves = (int32_t)nleaf;
    T->key = key.release();
    T->level = level.release();
    T->ix = ix.release();
    T->iy = iy.release();
    T->parent = parent.release();
    T->child0 = child0.release();
    T->leaf_of_box = lob.release();
    T->box_of_leaf = bol.release();
    T->level_start_dev = lsd.release();
    VFMM_CHECK(compute_lists(T, st));
    VFMM_CUDA(cudaStreamSynchronize(st));
    {
        // non-leaf boxes per level (for the per-level M2M and L2L GEMMs)
        std::vector<int32_t> c0(n);
        VFMM_CUDA(cudaMemcpy(c0.data(), T->child0, n * sizeof(int32_t), cudaMemcpyDeviceToHost));
        std::vector<int32_t> nl;
        T->nonleaf_start.assign(depth + 2, 0);
        for (int l = 0; l <= depth; ++l) {
            T->nonleaf_start[l] = (int32_t)nl.size();
            for (int b = T->level_start[l]; b < T->level_start[l + 1]; ++b)
                if (c0[b] >= 0) nl.push_back(b);
        }
        T->nonleaf_start[depth + 1] = (int32_t)nl.size();
        VFMM_CHECK(tree_malloc(reinterpret_cast<void**>(&T->nonleaf), std::max<size_t>(1, nl.size()) * sizeof(int32_t),
                               st));
        if (!nl.empty())
            VFMM_CUDA(cudaMemcpyAsync(T->nonleaf, nl.data(), nl.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        VFMM_CHECK(tree_malloc(reinterpret_cast<void**>(&T->nonleaf_start_dev), (depth + 2) * sizeof(int32_t), st));
        VFMM_CUDA(cudaMemcpyAsync(T->nonleaf_start_dev, T->nonleaf_start.data(), (depth + 2) * sizeof(int32_t),
                                  cudaMemcpyHostToDevice, st));
        VFMM_CUDA(cudaStreamSynchronize(st));  // nl leaves scope; later readers use other streams
    }
    VFMM_CHECK(build_mixed_plan(T, st));
    return VFMM_OK;
}

void free_tree(DeviceTree* t) {
    // work queued on any stream may still read the tree
    cudaDeviceSynchronize();
    // v_by_cfg, x_by_cfg and x_tgt point into the v_tiles and x_tiles allocations
    void* ps[] = {t->key,         t->level,       t->ix,       t->iy,           t->parent,     t->child0,
                  t->leaf_of_box, t->box_of_leaf, t->level_start_dev, t->u_by_cfg, t->u_tgt, t->near_tiles,
                  t->far_slot,    t->nonleaf,     t->nonleaf_start_dev, t->v_tiles, t->x_tiles};
    free_plan_set(&t->plans);
    if (t->plans_r) {
        for (auto& kv : *t->plans_r) {
            free_plan_set(kv.second);
            delete kv.second;
        }
        delete t->plans_r;
    }
    delete t->plans_mu;
    for (void* p : ps) tree_free(p);
    for (int q = 0; q < 4; ++q) {
        tree_free(t->lptr[q]);
        tree_free(t->lidx[q]);
        tree_free(t->lcfg[q]);
    }
    *t = DeviceTree();
}

static int check_params(const vfmm_tree_params* prm) {
    if (!prm) return fail(VFMM_ERR_INVALID_ARG, "null params");
    if (prm->k < 4 || prm->k > 16) return fail(VFMM_ERR_INVALID_ARG, "k must be in [4, 16]");
    if (!(prm->width > 0.0) || !std::isfinite(prm->width)) return fail(VFMM_ERR_INVALID_ARG, "width must be > 0");
    if (!std::isfinite(prm->cx) || !std::isfinite(prm->cy)) return fail(VFMM_ERR_INVALID_ARG, "bad centre");
    return VFMM_OK;
}

int make_source(const vfmm_source* s, DBuf<double>& buf, SourceDev* out, cudaStream_t st) {
    if (!s || !s->params) return fail(VFMM_ERR_INVALID_ARG, "null source");
    int len = 0;
    if (s->kind == VFMM_SRC_CONSTANT) len = 1;
    else if (s->kind == VFMM_SRC_GAUSS_SUM) {
        if (s->n < 1 || s->n > 4096) return fail(VFMM_ERR_INVALID_ARG, "gauss sum needs 1..4096 rows");
        len = 4 * s->n;
    } else if (s->kind == VFMM_SRC_KINKED) len = 54;
    else return fail(VFMM_ERR_INVALID_ARG, "unknown source kind");
    VFMM_CHECK(buf.alloc(len, st));
    VFMM_CUDA(cudaMemcpyAsync(buf.p, s->params, len * sizeof(double), cudaMemcpyHostToDevice, st));
    out->kind = s->kind;
    out->n = s->n;
    out->params = buf.p;
    return VFMM_OK;
}

__global__ void leaf_nodes_kernel(NodeGeom g, const int32_t* __restrict__ box_of_leaf, const int32_t* __restrict__ level,
                                  const int32_t* __restrict__ ix, const int32_t* __restrict__ iy, int nleaf,
                                  SourceDev src, int mode, double* __restrict__ out0, double* __restrict__ out1) {
    const int64_t kk = (int64_t)g.k * g.k;
    int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (int64_t)nleaf * kk) return;
    int leaf = (int)(gid / kk);
    int t = (int)(gid % kk);
    int b = box_of_leaf[leaf];
    int l = level[b];
    double h = ldexp(g.width, -l);
    double x = node_coord(g.lox, ix[b], g.xhat[t % g.k], h);
    double y = node_coord(g.loy, iy[b], g.xhat[t / g.k], h);
    if (mode == 0) {
        out0[gid] = x;
        out1[gid] = y;
    } else {
        out0[gid] = source_eval(src, x, y);
    }
}

static int leaf_nodes_impl(const DeviceTree* T, const vfmm_source* s, double* o0, double* o1, cudaStream_t st) {
    BuildCtx B;
    B.st = st;
    VFMM_CHECK(upload_node_tables(T->k, B));
    NodeGeom g{T->cx - T->width / 2.0, T->cy - T->width / 2.0, T->width, T->k, B.xhat.p};
    SourceDev sd;
    DBuf<double> pbuf;
    if (s) VFMM_CHECK(make_source(s, pbuf, &sd, st));
    int64_t total = (int64_t)T->n_leaves * T->k * T->k;
    leaf_nodes_kernel<<<nblk(total), 256, 0, st>>>(g, T->box_of_leaf, T->level, T->ix, T->iy, T->n_leaves, sd,
                                                   s ? 1 : 0, o0, o1);
    VFMM_CUDA(cudaGetLastError());
    // temporaries are freed on return; make sure the kernel has consumed them
    VFMM_CUDA(cudaStreamSynchronize(st));
    return VFMM_OK;
}

// ---------------------------------------------------------------- caller-evaluated f (pull protocol)
// Nodes where the caller evaluates f: box b of `level` (Morton key keys[b], or the full grid
// b = iy 2^level + ix when keys is null), node t = j k + i, the same coordinates the built-in
// sources are evaluated at.
__global__ void pending_nodes_kernel(NodeGeom g, int level, const uint32_t* __restrict__ keys, int64_t nbox,
                                     double* __restrict__ x, double* __restrict__ y) {
    const int kk = g.k * g.k;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nbox * kk) return;
    const int64_t b = q / kk;
    const int t = (int)(q - b * kk);
    int ix, iy;
    if (keys) {
        morton_decode(keys[b], &ix, &iy);
    } else {
        const int side = 1 << level;
        ix = (int)(b % side);
        iy = (int)(b / side);
    }
    const double h = ldexp(g.width, -level);
    x[q] = node_coord(g.lox, ix, g.xhat[t % g.k], h);
    y[q] = node_coord(g.loy, iy, g.xhat[t / g.k], h);
}

// F = max |f| over the caller's values on the f-scale grid.
__global__ void fmax_values_kernel(const double* __restrict__ f, int64_t n, double* __restrict__ out) {
    double m = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, fabs(f[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(out, m);
}

}  // namespace vfmm

// Refinement state of a tree whose f the caller evaluates (same test, order and balance as
// vfmm_tree_build).
struct vfmm_tree_builder {
    vfmm_tree_params prm{};
    cudaStream_t st = nullptr;
    vfmm::BuildCtx B;
    int phase = 0;  // 0: f wanted on the f-scale grid; 1: on the candidates of `level`; 2: refined; 3: finished
    int level = 0, m0 = 0, depth = 0;
    double F = 0.0, thresh = 0.0;
    std::vector<vfmm::DBuf<uint32_t>> keys;
    std::vector<int64_t> cnt;
    vfmm::DBuf<double> scal;  // [0] F, [1] smallest |tail / threshold - 1|
};

namespace vfmm {

// Splits the candidates of the builder's current level: every box (fv null) or those whose tail
// on the caller's values fv exceeds the threshold; phase 2 when none splits.
static int builder_split(vfmm_tree_builder* b, const double* fv) {
    const int l = b->level, k = b->prm.k;
    const int64_t n = b->cnt[l];
    cudaStream_t st = b->st;
    DBuf<int32_t> flags, offs;
    VFMM_CHECK(flags.alloc(n, st));
    VFMM_CHECK(offs.alloc(n, st));
    if (!fv)
        fill_kernel<<<nblk(n), 256, 0, st>>>(flags.p, n, 1);
    else
        refine_kernel<<<(unsigned)n, ((k * k + 31) / 32) * 32, 0, st>>>(b->B.g, SourceDev(), l, b->keys[l].p, (int)n,
                                                                         b->B.C.p, b->thresh, flags.p, b->scal.p + 1,
                                                                         fv);
    VFMM_CUDA(cudaGetLastError());
    int64_t m = 0;
    VFMM_CHECK(exclusive_scan(flags.p, offs.p, n, &m, st));
    if (m == 0) {
        b->phase = 2;
        return VFMM_OK;
    }
    VFMM_CHECK(b->keys[l + 1].alloc_keep(4 * m));
    emit_children_kernel<<<nblk(n), 256, 0, st>>>(b->keys[l].p, flags.p, offs.p, (int)n, b->keys[l + 1].p);
    VFMM_CUDA(cudaGetLastError());
    b->cnt[l + 1] = 4 * m;
    b->depth = l + 1;
    b->level = l + 1;
    return VFMM_OK;
}

// Levels below min_depth split without a test; then either the candidates of the current level
// want f (phase 1) or the refinement is over (phase 2: max_depth reached).
static int builder_advance(vfmm_tree_builder* b) {
    while (b->phase != 2 && b->level < b->prm.max_depth && b->level < b->prm.min_depth)
        VFMM_CHECK(builder_split(b, nullptr));
    if (b->phase != 2) b->phase = b->level < b->prm.max_depth ? 1 : 2;
    return VFMM_OK;
}

static int64_t builder_pending(const vfmm_tree_builder* b) {
    const int64_t kk = (int64_t)b->prm.k * b->prm.k;
    if (b->phase == 0) return (1ll << (2 * b->m0)) * kk;
    if (b->phase == 1) return b->cnt[b->level] * kk;
    return 0;
}

}  // namespace vfmm

using namespace vfmm;

extern "C" int vfmm_tree_begin(const vfmm_tree_params* prm, void* stream, vfmm_tree_builder** out) {
    if (!out) return fail(VFMM_ERR_INVALID_ARG, "null out");
    *out = nullptr;
    VFMM_CHECK(check_params(prm));
    if (prm->max_depth < 0 || prm->max_depth > kMaxDepth || prm->min_depth < 0 || prm->min_depth > prm->max_depth)
        return fail(VFMM_ERR_INVALID_ARG, "need 0 <= min_depth <= max_depth <= 16");
    if (!(prm->tol >= 0.0)) return fail(VFMM_ERR_INVALID_ARG, "tol must be >= 0");
    vfmm_tree_builder* b = new vfmm_tree_builder();
    b->prm = *prm;
    b->st = (cudaStream_t)stream;
    b->B.st = b->st;
    b->m0 = std::min(5, prm->max_depth);
    b->keys.resize(prm->max_depth + 1);
    b->cnt.assign(prm->max_depth + 1, 0);
    b->B.keep = true;
    int rc = upload_node_tables(prm->k, b->B);
    b->B.g = NodeGeom{prm->cx - prm->width / 2.0, prm->cy - prm->width / 2.0, prm->width, prm->k, b->B.xhat.p};
    if (rc == VFMM_OK) rc = b->keys[0].alloc_keep(1);
    if (rc == VFMM_OK) rc = b->scal.alloc_keep(2);
    if (rc == VFMM_OK) {
        const uint32_t zero = 0;
        const double init[2] = {0.0, INFINITY};
        cudaError_t e = cudaMemcpyAsync(b->keys[0].p, &zero, sizeof(zero), cudaMemcpyHostToDevice, b->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->scal.p, init, sizeof(init), cudaMemcpyHostToDevice, b->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
        if (e != cudaSuccess) rc = cuda_fail(e, "tree begin");
    }
    if (rc != VFMM_OK) {
        delete b;
        return rc;
    }
    b->cnt[0] = 1;
    *out = b;
    return VFMM_OK;
}

extern "C" int vfmm_tree_pending(const vfmm_tree_builder* b, int64_t* n_nodes) {
    if (!b || !n_nodes) return fail(VFMM_ERR_INVALID_ARG, "null argument");
    *n_nodes = builder_pending(b);
    return VFMM_OK;
}

extern "C" int vfmm_tree_pending_nodes(const vfmm_tree_builder* b, double* x_dev, double* y_dev) {
    if (!b || !x_dev || !y_dev) return fail(VFMM_ERR_INVALID_ARG, "null argument");
    const int64_t n = builder_pending(b);
    if (n == 0) return fail(VFMM_ERR_INVALID_ARG, "no nodes pending");
    const int64_t nbox = n / ((int64_t)b->prm.k * b->prm.k);
    if (b->phase == 0)
        pending_nodes_kernel<<<nblk(n), 256, 0, b->st>>>(b->B.g, b->m0, nullptr, nbox, x_dev, y_dev);
    else
        pending_nodes_kernel<<<nblk(n), 256, 0, b->st>>>(b->B.g, b->level, b->keys[b->level].p, nbox, x_dev, y_dev);
    VFMM_CUDA(cudaGetLastError());
    return VFMM_OK;
}

extern "C" int vfmm_tree_submit(vfmm_tree_builder* b, const double* f_dev) {
    if (!b || !f_dev) return fail(VFMM_ERR_INVALID_ARG, "null argument");
    if (b->phase >= 2) return fail(VFMM_ERR_INVALID_ARG, "refinement is complete: no f wanted");
    if (b->phase == 0) {
        const int64_t n = builder_pending(b);
        fmax_values_kernel<<<(unsigned)std::min<int64_t>(1024, nblk(n)), 256, 0, b->st>>>(f_dev, n, b->scal.p);
        VFMM_CUDA(cudaGetLastError());
        VFMM_CUDA(cudaMemcpyAsync(&b->F, b->scal.p, sizeof(double), cudaMemcpyDeviceToHost, b->st));
        VFMM_CUDA(cudaStreamSynchronize(b->st));
        b->thresh = b->prm.tol * b->F;
        b->phase = 1;
        return builder_advance(b);
    }
    VFMM_CHECK(builder_split(b, f_dev));
    VFMM_CHECK(builder_advance(b));
    VFMM_CUDA(cudaStreamSynchronize(b->st));  // f_dev may be reused or freed once this returns
    return VFMM_OK;
}

extern "C" int vfmm_tree_finish(vfmm_tree_builder* b, vfmm_tree** out) {
    if (!b || !out) return fail(VFMM_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (b->phase != 2) return fail(VFMM_ERR_INVALID_ARG, b->phase == 3 ? "tree already finished" : "f still pending");
    vfmm_tree* t = new vfmm_tree();
    DeviceTree* T = &t->t;
    T->k = b->prm.k;
    T->cx = b->prm.cx;
    T->cy = b->prm.cy;
    T->width = b->prm.width;
    T->f_scale = b->F;
    T->n_capped = -1;  // the last level's boxes were not offered for a test
    double mm = INFINITY;
    cudaError_t e = cudaMemcpyAsync(&mm, b->scal.p + 1, sizeof(double), cudaMemcpyDeviceToHost, b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    int rc = e == cudaSuccess ? VFMM_OK : cuda_fail(e, "tree finish");
    T->min_margin = mm;
    if (rc == VFMM_OK) rc = finalize(b->keys, b->cnt, b->depth, b->st, T);
    b->phase = 3;
    // balancing replaced keys by stream-ordered temporaries: release them on b->st while it is
    // known to be valid (the builder may outlive the caller's stream)
    for (auto& kb : b->keys) kb.reset();
    if (rc != VFMM_OK) {
        free_tree(T);
        delete t;
        return rc;
    }
    *out = t;
    return VFMM_OK;
}

extern "C" int vfmm_tree_builder_destroy(vfmm_tree_builder* b) {
    delete b;
    return VFMM_OK;
}

extern "C" int vfmm_tree_build_rule(const vfmm_tree_params* prm, const vfmm_source* src, int32_t rule, void* stream,
                                    vfmm_tree** out) {
    if (!out) return fail(VFMM_ERR_INVALID_ARG, "null out");
    *out = nullptr;
    if (rule < VFMM_REFINE_TAIL || rule > VFMM_REFINE_INTERP_MIXED) return fail(VFMM_ERR_INVALID_ARG, "unknown rule");
    VFMM_CHECK(check_params(prm));
    if (prm->max_depth < 0 || prm->max_depth > kMaxDepth || prm->min_depth < 0 || prm->min_depth > prm->max_depth)
        return fail(VFMM_ERR_INVALID_ARG, "need 0 <= min_depth <= max_depth <= 16");
    if (!(prm->tol >= 0.0)) return fail(VFMM_ERR_INVALID_ARG, "tol must be >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    DBuf<double> pbuf;
    SourceDev sd;
    VFMM_CHECK(make_source(src, pbuf, &sd, st));
    vfmm_tree* t = new vfmm_tree();
    int r = build(prm, &sd, 0, 0, st, &t->t, rule);
    if (r != VFMM_OK) {
        free_tree(&t->t);
        delete t;
        return r;
    }
    *out = t;
    return VFMM_OK;
}

extern "C" int vfmm_tree_build(const vfmm_tree_params* prm, const vfmm_source* src, void* stream, vfmm_tree** out) {
    if (!out) return fail(VFMM_ERR_INVALID_ARG, "null out");
    *out = nullptr;
    VFMM_CHECK(check_params(prm));
    if (prm->max_depth < 0 || prm->max_depth > kMaxDepth || prm->min_depth < 0 || prm->min_depth > prm->max_depth)
        return fail(VFMM_ERR_INVALID_ARG, "need 0 <= min_depth <= max_depth <= 16");
    if (!(prm->tol >= 0.0)) return fail(VFMM_ERR_INVALID_ARG, "tol must be >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    DBuf<double> pbuf;
    SourceDev sd;
    VFMM_CHECK(make_source(src, pbuf, &sd, st));
    vfmm_tree* t = new vfmm_tree();
    int r = build(prm, &sd, 0, 0, st, &t->t);
    if (r != VFMM_OK) {
        free_tree(&t->t);
        delete t;
        return r;
    }
    *out = t;
    return VFMM_OK;
}

extern "C" int vfmm_tree_build_leaves(const vfmm_tree_params* prm, const vfmm_source* src, int64_t n_leaves,
                                      void* stream, vfmm_tree** out) {
    if (!out) return fail(VFMM_ERR_INVALID_ARG, "null out");
    *out = nullptr;
    VFMM_CHECK(check_params(prm));
    if (prm->max_depth < 0 || prm->max_depth > kMaxDepth) return fail(VFMM_ERR_INVALID_ARG, "need 0 <= max_depth <= 16");
    if (n_leaves < 1 || n_leaves > (1ll << 26)) return fail(VFMM_ERR_INVALID_ARG, "n_leaves must be in [1, 2^26]");
    cudaStream_t st = (cudaStream_t)stream;
    DBuf<double> pbuf;
    SourceDev sd;
    VFMM_CHECK(make_source(src, pbuf, &sd, st));
    vfmm_tree* t = new vfmm_tree();
    int r = build(prm, &sd, 0, n_leaves, st, &t->t);
    if (r != VFMM_OK) {
        free_tree(&t->t);
        delete t;
        return r;
    }
    *out = t;
    return VFMM_OK;
}

extern "C" int vfmm_tree_build_many(const vfmm_tree_params* prm, const vfmm_source* src, const int64_t* n_leaves,
                                    int32_t n, int32_t n_threads, vfmm_tree** out) {
    if (!prm || !src || !n_leaves || !out || n < 0) return fail(VFMM_ERR_INVALID_ARG, "null argument or n < 0");
    for (int32_t i = 0; i < n; ++i) out[i] = nullptr;
    if (n == 0) return VFMM_OK;
    int dev = 0;
    VFMM_CUDA(cudaGetDevice(&dev));
    int nt = n_threads > 0 ? n_threads : (int)std::min(16u, std::max(1u, std::thread::hardware_concurrency()));
    nt = std::max(1, std::min(nt, (int)n));
    std::atomic<int32_t> next(0);
    std::atomic<int> first_err(VFMM_OK);
    std::mutex msg_mu;
    std::string msg;
    auto worker = [&]() {
        cudaStream_t st = nullptr;
        int rc = VFMM_OK;
        if (cudaSetDevice(dev) != cudaSuccess) rc = fail(VFMM_ERR_CUDA, "cudaSetDevice failed");
        if (rc == VFMM_OK && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
            rc = fail(VFMM_ERR_CUDA, "cudaStreamCreateWithFlags failed");
        for (int32_t i = next++; rc == VFMM_OK && i < n && first_err.load() == VFMM_OK; i = next++)
            rc = n_leaves[i] > 0 ? vfmm_tree_build_leaves(&prm[i], &src[i], n_leaves[i], st, &out[i])
                                 : vfmm_tree_build(&prm[i], &src[i], st, &out[i]);
        if (rc != VFMM_OK) {
            int expected = VFMM_OK;
            if (first_err.compare_exchange_strong(expected, rc)) {
                std::lock_guard<std::mutex> lock(msg_mu);
                msg = vfmm_last_error_detail();
            }
        }
        if (st) cudaStreamDestroy(st);
    };
    std::vector<std::thread> pool;
    for (int w = 1; w < nt; ++w) pool.emplace_back(worker);
    worker();
    for (auto& t : pool) t.join();
    if (first_err.load() != VFMM_OK) {
        for (int32_t i = 0; i < n; ++i) {
            if (out[i]) vfmm_tree_destroy(out[i]);
            out[i] = nullptr;
        }
        return fail(first_err.load(), "tree build of the batch failed: " + msg);
    }
    return VFMM_OK;
}

extern "C" int vfmm_tree_build_uniform(const vfmm_tree_params* prm, int32_t depth, void* stream, vfmm_tree** out) {
    if (!out) return fail(VFMM_ERR_INVALID_ARG, "null out");
    *out = nullptr;
    VFMM_CHECK(check_params(prm));
    if (depth < 0 || depth > 10) return fail(VFMM_ERR_INVALID_ARG, "uniform depth must be in [0, 10]");
    vfmm_tree* t = new vfmm_tree();
    int r = build(prm, nullptr, depth, 0, (cudaStream_t)stream, &t->t);
    if (r != VFMM_OK) {
        free_tree(&t->t);
        delete t;
        return r;
    }
    *out = t;
    return VFMM_OK;
}

extern "C" int vfmm_tree_info(const vfmm_tree* tree, vfmm_tree_info_t* info) {
    if (!tree || !info) return fail(VFMM_ERR_INVALID_ARG, "null argument");
    const DeviceTree& T = tree->t;
    info->n_boxes = T.n_boxes;
    info->n_leaves = T.n_leaves;
    info->depth = T.depth;
    info->k = T.k;
    for (int q = 0; q < 4; ++q) info->list_len[q] = T.llen[q];
    info->f_scale = T.f_scale;
    info->min_margin = T.min_margin;
    info->n_depth_capped = T.n_capped;
    return VFMM_OK;
}

extern "C" int vfmm_tree_export_boxes(const vfmm_tree* tree, int32_t* level, int32_t* ix, int32_t* iy) {
    if (!tree) return fail(VFMM_ERR_INVALID_ARG, "null tree");
    const DeviceTree& T = tree->t;
    size_t bytes = (size_t)T.n_boxes * sizeof(int32_t);
    if (level) VFMM_CUDA(cudaMemcpy(level, T.level, bytes, cudaMemcpyDeviceToHost));
    if (ix) VFMM_CUDA(cudaMemcpy(ix, T.ix, bytes, cudaMemcpyDeviceToHost));
    if (iy) VFMM_CUDA(cudaMemcpy(iy, T.iy, bytes, cudaMemcpyDeviceToHost));
    return VFMM_OK;
}

extern "C" int vfmm_tree_export_list(const vfmm_tree* tree, int32_t which, int32_t* ptr, int32_t* idx, int32_t* cfg) {
    if (!tree || which < 0 || which > 3) return fail(VFMM_ERR_INVALID_ARG, "bad tree or list id");
    const DeviceTree& T = tree->t;
    if (ptr) VFMM_CUDA(cudaMemcpy(ptr, T.lptr[which], (T.n_boxes + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
    size_t bytes = (size_t)T.llen[which] * sizeof(int32_t);
    if (idx && bytes) VFMM_CUDA(cudaMemcpy(idx, T.lidx[which], bytes, cudaMemcpyDeviceToHost));
    if (cfg && bytes) VFMM_CUDA(cudaMemcpy(cfg, T.lcfg[which], bytes, cudaMemcpyDeviceToHost));
    return VFMM_OK;
}

extern "C" int vfmm_tree_leaf_nodes(const vfmm_tree* tree, double* x_dev, double* y_dev, void* stream) {
    if (!tree || !x_dev || !y_dev) return fail(VFMM_ERR_INVALID_ARG, "null argument");
    return leaf_nodes_impl(&tree->t, nullptr, x_dev, y_dev, (cudaStream_t)stream);
}

extern "C" int vfmm_source_sample(const vfmm_tree* tree, const vfmm_source* src, double* f_dev, void* stream) {
    if (!tree || !src || !f_dev) return fail(VFMM_ERR_INVALID_ARG, "null argument");
    return leaf_nodes_impl(&tree->t, src, f_dev, nullptr, (cudaStream_t)stream);
}

extern "C" int vfmm_tree_destroy(vfmm_tree* tree) {
    if (!tree) return VFMM_OK;
    free_tree(&tree->t);
    delete tree;
    return VFMM_OK;
}
