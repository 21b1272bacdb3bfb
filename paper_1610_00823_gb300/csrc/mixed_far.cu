// Split-BF16 far field (VFMM_MIXED): S2M, M2L, S2L and the leaf evaluation of local and W-list
// multipole expansions (L2T + M2T), all as split contractions on the tensor cores (see mixed.cu
// for the arithmetic), with FP64 kept for the log(h) terms, the coefficient-0 terms, M2M, L2L and
// the final per-target sums. S2L takes the f slices of the near field (global exponent) and
// 20 tables of coefficients 1..p; its row 0 and log(h) term are FP64 (m2l_c0_kernel).
//
// Normalisation (each product must be exact per diagonal, so every A row and every table row
// carries a power-of-two scale):
//  * S2M: A = f slices (global exponent, shared with the near field); table rows = S2M rows of
//    coefficients 1..p (row exponents). Coefficient 0 (the mass) is an FP64 dot product.
//  * M2L: A = multipole coefficient k (k runs over real and imaginary parts of a_0..a_p) times
//    2^(floor(k/4) - G(l)): 2^-floor(n/2), n = k/2, bounds the decay of scaled coefficient n, and
//    G(l) is the level's exponent, so every level shares one table set (columns times
//    2^-floor(k/4), rows normalised once) and all levels go in one launch. Output row r is
//    scaled back by 2^(G(l) + E_r). Output coefficient 0 and the log(h) term are added in FP64
//    by the downward kernel.
//  * Leaf: A = the leaf's own local coefficients 1..p and the multipoles of its W boxes, all
//    divided by 2^E_t, E_t the exponent of the leaf's largest such value; tables: L2T and the
//    20 M2T configurations (factor h / h_w = 2 folded into the gradient rows), row exponents.
//    The local coefficient 0 and a_0 log(h_w) are added in FP64 by the leaf kernel.
#include <cuda_bf16.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <complex>
#include <string>
#include <vector>

#include "mixed.cuh"
#include "ops.cuh"
#include "vfmm_internal.cuh"

namespace vfmm {

using bf16 = __nv_bfloat16;

__device__ inline int exp_of(double m) {
    int e = 0;
    if (m > 0.0) frexp(m, &e);
    return e;
}

// ---------------------------------------------------------------- operator tables
// E[r] = exponent of max_{c,k} |M[c][r][k]|
__global__ void rows_exp_kernel(const double* __restrict__ M, int nc, int R, int K, int* __restrict__ E) {
    __shared__ double red[256];
    const int r = blockIdx.x;
    double m = 0.0;
    for (int q = threadIdx.x; q < nc * K; q += blockDim.x) m = fmax(m, fabs(M[((size_t)(q / K) * R + r) * K + q % K]));
    red[threadIdx.x] = m;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) E[r] = exp_of(red[0]);
}

// out[c][r][i][k] = slice i of M[c][r][k] / 2^E[r]; rows >= R and columns >= K are zero.
__global__ void rows_slice_kernel(const double* __restrict__ M, int R, int K, int Rp, int Kp,
                                  const int* __restrict__ E, bf16* __restrict__ out) {
    const int r = blockIdx.x, c = blockIdx.y;
    for (int k = threadIdx.x; k < Kp; k += blockDim.x) {
        double v = (r < R && k < K) ? M[((size_t)c * R + r) * K + k] : 0.0;
        slice_fixed(v, r < R ? E[r] : 0, out + slice_at((size_t)c * Rp + r, Kp, k), kKBlock);
    }
}

static int slice_table(const std::vector<double>& M, int nc, int R, int K, int Rp, int Kp, void** out, int** E,
                       cudaStream_t st) {
    double* dM = nullptr;
    VFMM_CUDA(cudaMalloc(&dM, M.size() * sizeof(double)));
    VFMM_CUDA(cudaMemcpyAsync(dM, M.data(), M.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    VFMM_CUDA(cudaMalloc(E, Rp * sizeof(int)));
    VFMM_CUDA(cudaMemsetAsync(*E, 0, Rp * sizeof(int), st));
    VFMM_CUDA(cudaMalloc(out, (size_t)nc * Rp * kSlices * Kp * sizeof(bf16)));
    rows_exp_kernel<<<R, 256, 0, st>>>(dM, nc, R, K, *E);
    rows_slice_kernel<<<dim3(Rp, nc), 128, 0, st>>>(dM, R, K, Rp, Kp, *E, (bf16*)*out);
    VFMM_CUDA(cudaGetLastError());
    VFMM_CUDA(cudaStreamSynchronize(st));
    cudaFree(dM);
    return VFMM_OK;
}

int far_prepare(vfmm_ops* o, cudaStream_t st) {
    MixedOps* mo = (MixedOps*)o->mixed;
    const int k = o->k, kk = k * k, p = o->p, P = p + 1;
    const int R = 3 * kk;
    mo->Kx = (2 * P + kKBlock - 1) / kKBlock * kKBlock;
    mo->Rx = 2 * p <= kTileNSmall ? kTileNSmall : (2 * p + kTileN - 1) / kTileN * kTileN;
    const int rx_tile = table_rows_per_tile(false, mo->Rx);
    const double inv2pi = 1.0 / (2.0 * 3.14159265358979323846);
    // S2M rows 2..2p+1 (coefficients 1..p)
    std::vector<double> s2m((size_t)2 * P * kk);
    VFMM_CUDA(cudaMemcpy(s2m.data(), o->s2m, s2m.size() * sizeof(double), cudaMemcpyDeviceToHost));
    std::vector<double> S((size_t)2 * p * kk);
    std::copy(s2m.begin() + 2 * kk, s2m.end(), S.begin());
    VFMM_CHECK(slice_table(S, 1, 2 * p, kk, mo->Rx, mo->Kp, &mo->s2m_sl, &mo->s2m_E, st));
    VFMM_CHECK(make_table_map(mo->s2m_sl, mo->Rx, mo->Kp, rx_tile, &mo->tm_s2m));
    // M2L as real matrices: rows 2..2p+1, columns 0..2p+1
    std::vector<double> mt((size_t)kVCfg * P * P * 2);
    VFMM_CUDA(cudaMemcpy(mt.data(), o->m2l_t, mt.size() * sizeof(double), cudaMemcpyDeviceToHost));
    std::vector<double> MR((size_t)kVCfg * mo->Rx * mo->Kx, 0.0);
    for (int c = 0; c < kVCfg; ++c)
        for (int l = 1; l <= p; ++l)
            for (int n = 0; n <= p; ++n) {
                double re = mt[(((size_t)c * P + n) * P + l) * 2], im = mt[(((size_t)c * P + n) * P + l) * 2 + 1];
                size_t rr = (size_t)c * mo->Rx + 2 * (l - 1);
                MR[rr * mo->Kx + 2 * n] = re;
                MR[rr * mo->Kx + 2 * n + 1] = -im;
                MR[(rr + 1) * mo->Kx + 2 * n] = im;
                MR[(rr + 1) * mo->Kx + 2 * n + 1] = re;
            }
    // |a~_n| <= mass (1/sqrt 2)^n for a box's scaled multipole coefficients, so column k (coefficient
    // n = k / 2) carries the bound 2^-floor(n/2); the operand is divided by it and the table times it
    for (size_t r = 0; r < (size_t)kVCfg * mo->Rx; ++r)
        for (int q = 0; q < mo->Kx; ++q) MR[r * mo->Kx + q] = std::ldexp(MR[r * mo->Kx + q], -(q >> 2));
    VFMM_CHECK(slice_table(MR, kVCfg, mo->Rx, mo->Kx, mo->Rx, mo->Kx, &mo->m2l_sl, &mo->m2l_E, st));
    {
        // output coefficient 0 stays FP64: its row of every M2L matrix, [offset][n] complex
        std::vector<double> r0((size_t)kVCfg * P * 2);
        for (int c = 0; c < kVCfg; ++c)
            for (int n = 0; n <= p; ++n) {
                r0[((size_t)c * P + n) * 2] = mt[(((size_t)c * P + n) * P + 0) * 2];
                r0[((size_t)c * P + n) * 2 + 1] = mt[(((size_t)c * P + n) * P + 0) * 2 + 1];
            }
        VFMM_CUDA(cudaMalloc(&mo->m2l_r0, r0.size() * sizeof(double)));
        VFMM_CUDA(cudaMemcpy(mo->m2l_r0, r0.data(), r0.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    VFMM_CHECK(make_table_map(mo->m2l_sl, (int64_t)kVCfg * mo->Rx, mo->Kx, rx_tile, &mo->tm_m2l));
    // leaf tables: 0 = L2T without coefficient 0, 1 + c = M2T of W configuration c
    std::vector<double> l2t((size_t)R * 2 * P), xh(k);
    VFMM_CUDA(cudaMemcpy(l2t.data(), o->l2t, l2t.size() * sizeof(double), cudaMemcpyDeviceToHost));
    VFMM_CUDA(cudaMemcpy(xh.data(), o->xhat, k * sizeof(double), cudaMemcpyDeviceToHost));
    const int KX = 2 * P;
    std::vector<double> F((size_t)(1 + kFarCfg) * R * KX, 0.0);
    for (int r = 0; r < R; ++r)
        for (int q = 2; q < KX; ++q) F[(size_t)r * KX + q] = l2t[(size_t)r * KX + q];
    typedef std::complex<double> cd;
    for (int c = 0; c < kFarCfg; ++c) {
        int px, py;
        far_pattern(c, &px, &py);
        double* Fc = F.data() + (size_t)(1 + c) * R * KX;
        for (int t = 0; t < kk; ++t) {
            cd zeta(2.0 * (xh[t % k] - px / 4.0), 2.0 * (xh[t / k] - py / 4.0));
            cd zi = 1.0 / zeta;
            // potential row: -(1/2pi) Re(a_0 log zeta + sum_n a_n zeta^-n)
            Fc[(size_t)t * KX + 0] = -inv2pi * std::log(std::abs(zeta));
            Fc[(size_t)t * KX + 1] = inv2pi * std::arg(zeta);
            cd zp = 1.0;
            for (int n = 1; n <= p; ++n) {
                zp *= zi;
                Fc[(size_t)t * KX + 2 * n] = -inv2pi * zp.real();
                Fc[(size_t)t * KX + 2 * n + 1] = inv2pi * zp.imag();
            }
            // gradient rows (times h): 2 sum_n c_n a_n, c_0 = 1/zeta, c_n = -n zeta^(-n-1)
            cd zq = zi;  // zeta^(-n-1) at step n
            for (int n = 0; n <= p; ++n) {
                cd cn = n == 0 ? zi : -(double)n * zq;
                Fc[(size_t)(kk + t) * KX + 2 * n] = -2.0 * inv2pi * cn.real();
                Fc[(size_t)(kk + t) * KX + 2 * n + 1] = 2.0 * inv2pi * cn.imag();
                Fc[(size_t)(2 * kk + t) * KX + 2 * n] = 2.0 * inv2pi * cn.imag();
                Fc[(size_t)(2 * kk + t) * KX + 2 * n + 1] = 2.0 * inv2pi * cn.real();
                zq *= zi;
            }
        }
    }
    VFMM_CHECK(slice_table(F, 1 + kFarCfg, R, KX, mo->Rp, mo->Kx, &mo->far_sl, &mo->far_E, st));
    VFMM_CHECK(make_table_map(mo->far_sl, (int64_t)(1 + kFarCfg) * mo->Rp, mo->Kx,
                              table_rows_per_tile(near_transposed(o->k)), &mo->tm_far));
    // S2L: rows 2..2p+1 (Re, Im of coefficients 1..p) over the k*k source values; row 0 kept in FP64
    std::vector<double> st_((size_t)kFarCfg * kk * P * 2);
    VFMM_CUDA(cudaMemcpy(st_.data(), o->s2l_t, st_.size() * sizeof(double), cudaMemcpyDeviceToHost));
    std::vector<double> XL((size_t)kFarCfg * 2 * p * kk), X0((size_t)kFarCfg * kk);
    for (int c = 0; c < kFarCfg; ++c)
        for (int s = 0; s < kk; ++s) {
            X0[(size_t)c * kk + s] = st_[(((size_t)c * kk + s) * P + 0) * 2];
            for (int l = 1; l <= p; ++l) {
                XL[((size_t)c * 2 * p + 2 * (l - 1)) * kk + s] = st_[(((size_t)c * kk + s) * P + l) * 2];
                XL[((size_t)c * 2 * p + 2 * (l - 1) + 1) * kk + s] = st_[(((size_t)c * kk + s) * P + l) * 2 + 1];
            }
        }
    VFMM_CHECK(slice_table(XL, kFarCfg, 2 * p, kk, mo->Rx, mo->Kp, &mo->s2l_sl, &mo->s2l_E, st));
    VFMM_CHECK(make_table_map(mo->s2l_sl, (int64_t)kFarCfg * mo->Rx, mo->Kp, rx_tile, &mo->tm_s2l));
    VFMM_CUDA(cudaMalloc(&mo->s2l_r0, X0.size() * sizeof(double)));
    VFMM_CUDA(cudaMemcpy(mo->s2l_r0, X0.data(), X0.size() * sizeof(double), cudaMemcpyHostToDevice));
    return VFMM_OK;
}

void far_free(MixedOps* mo) {
    void* ps[] = {mo->s2m_sl, mo->s2m_E, mo->m2l_sl, mo->m2l_E, mo->far_sl, mo->far_E,
                  mo->s2l_sl, mo->s2l_E, mo->s2l_r0, mo->m2l_r0};
    for (void* p : ps)
        if (p) cudaFree(p);
}

// ---------------------------------------------------------------- schedules
// Rows of the leaf far-field operand: per leaf, slot 0 = its own local (L2T), slot 1 + j = its
// j-th W entry; far_slot[leaf] = first slot (right-hand side r of slot s is row s * R + r).
// Pinned staging for the plan builders' reads of device arrays: one buffer per host thread, grown on
// demand, so that all reads go out as asynchronous copies followed by one synchronisation.
static int pinned_stage(size_t bytes, void** out) {
    struct Stage {
        void* p = nullptr;
        size_t n = 0;
        ~Stage() {
            if (p) cudaFreeHost(p);
        }
    };
    thread_local Stage s;
    if (s.n < bytes) {
        if (s.p) cudaFreeHost(s.p);
        s.p = nullptr;
        s.n = 0;
        VFMM_CUDA(cudaMallocHost(&s.p, bytes));
        s.n = bytes;
    }
    *out = s.p;
    return VFMM_OK;
}

int fetch_host_lists(const DeviceTree& T, HostLists* H) {
    const int nb = T.n_boxes, nl = T.n_leaves;
    struct Piece {
        const int32_t* src;
        std::vector<int32_t>* dst;
        size_t n;
    };
    std::vector<Piece> pieces = {{T.box_of_leaf, &H->bol, (size_t)nl}, {T.leaf_of_box, &H->lob, (size_t)nb}};
    for (int q = 0; q < 4; ++q) {
        pieces.push_back({T.lptr[q], &H->ptr[q], (size_t)nb + 1});
        pieces.push_back({T.lidx[q], &H->idx[q], (size_t)T.llen[q]});
        pieces.push_back({T.lcfg[q], &H->cfg[q], (size_t)T.llen[q]});
    }
    size_t total = 0;
    for (const Piece& pc : pieces) total += pc.n;
    void* stage = nullptr;
    VFMM_CHECK(pinned_stage(std::max<size_t>(1, total) * sizeof(int32_t), &stage));
    int32_t* h = static_cast<int32_t*>(stage);
    size_t o = 0;
    for (const Piece& pc : pieces) {
        if (pc.n)
            VFMM_CUDA(cudaMemcpyAsync(h + o, pc.src, pc.n * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                      cudaStreamPerThread));
        o += pc.n;
    }
    VFMM_CUDA(cudaStreamSynchronize(cudaStreamPerThread));
    o = 0;
    for (const Piece& pc : pieces) {
        pc.dst->assign(h + o, h + o + pc.n);
        o += pc.n;
    }
    return VFMM_OK;
}

int build_far_slots(DeviceTree* T, const HostLists& H, cudaStream_t st) {
    const int nl = T->n_leaves;
    const std::vector<int32_t>& bol = H.bol;
    const std::vector<int32_t>& ptr = H.ptr[VFMM_LIST_W];
    std::vector<int32_t> slot(nl + 1, 0);
    for (int t = 0; t < nl; ++t) slot[t + 1] = slot[t] + 1 + (ptr[bol[t] + 1] - ptr[bol[t]]);
    T->n_far_slots = slot[nl];
    VFMM_CHECK(tree_malloc(reinterpret_cast<void**>(&T->far_slot), (nl + 1) * sizeof(int32_t), st));
    VFMM_CUDA(cudaMemcpyAsync(T->far_slot, slot.data(), (nl + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    return VFMM_OK;
}

int build_far_plan(int which, const DeviceTree& T, int R, const HostLists& H, PlanArena& A, PlanSet* PS) {
    const int nb = T.n_boxes, nl = T.n_leaves;
    // K blocks per table: k^2 for S2M and S2L; 2(p+1) for M2L and the leaf far field, where p is not
    // known to the tree (3 blocks = p up to 47; only the default split-K choice depends on it)
    const int Kp = (T.k * T.k + kKBlock - 1) / kKBlock * kKBlock;
    constexpr int kFarKb = 3;
    const std::vector<int32_t>& bol = H.bol;
    const std::vector<int32_t>& lob = H.lob;
    // boxes with a non-empty list q as targets, one item per entry (table = its configuration)
    auto list_items = [&](int q, bool src_leaf, PlanItems* I) {
        const std::vector<int32_t>& ptr = H.ptr[q];
        const std::vector<int32_t>& idx = H.idx[q];
        const std::vector<int32_t>& cfg = H.cfg[q];
        I->tab.reserve(idx.size());
        I->src.reserve(idx.size());
        for (int b = 0; b < nb; ++b) {
            if (ptr[b + 1] == ptr[b]) continue;
            uint64_t sig = 0;
            for (int e = ptr[b]; e < ptr[b + 1]; ++e) {
                I->add(cfg[e], src_leaf ? lob[idx[e]] : idx[e]);
                sig |= 1ull << cfg[e];
            }
            I->close(b, sig, (uint64_t)b);
        }
    };
    PlanItems I;
    switch (which) {
        case kCtrS2M: {  // every leaf, one table, gathered row = the leaf
            for (int t = 0; t < nl; ++t) {
                I.add(0, t);
                I.close(t, 0, (uint64_t)t);
            }
            std::vector<int32_t> order(nl);
            for (int t = 0; t < nl; ++t) order[t] = t;
            return build_split_plan(I, order, 1, 1, R, false, Kp / kKBlock, A, &PS->s2m);
        }
        case kCtrM2L:  // boxes with a V list, tables = the 40 offsets, gathered row = source box
            list_items(VFMM_LIST_V, false, &I);
            // slab costs relative to the tensor work per column: K = 2(p+1) padded (about 96), rows <= 128
            return build_contraction_plan(I, kVCfg, 1, R, false, kFarKb, 0.5, 128 * sizeof(float2), A, &PS->m2l);
        case kCtrS2L:  // boxes with an X list, tables 20 configurations, gathered row = source leaf
            list_items(VFMM_LIST_X, true, &I);
            return build_contraction_plan(I, kFarCfg, 1, R, false, Kp / kKBlock, 48.0 / Kp, 128 * sizeof(float2), A,
                                          &PS->s2l);
        case kCtrFar: {  // leaf far field: slot 0 = own local (L2T), slot 1 + j = j-th W entry (table 1 + its configuration)
            const std::vector<int32_t>& ptr = H.ptr[VFMM_LIST_W];
            const std::vector<int32_t>& cfg = H.cfg[VFMM_LIST_W];
            int32_t slot = 0;
            for (int t = 0; t < nl; ++t) {
                const int b = bol[t];
                I.add(0, slot);
                uint64_t sig = 0;
                for (int e = ptr[b]; e < ptr[b + 1]; ++e) {
                    I.add(1 + cfg[e], slot + 1 + (e - ptr[b]));
                    sig |= 1ull << cfg[e];
                }
                slot += 1 + (ptr[b + 1] - ptr[b]);
                I.close(t, sig, (uint64_t)t);
            }
            const int rows = 3 * T.k * T.k;
            const bool tr = near_transposed(T.k);
            const int tile_rows = table_rows_per_tile(tr);
            return build_contraction_plan(I, 1 + kFarCfg, (rows + tile_rows - 1) / tile_rows, R, tr, kFarKb, 0.5,
                                          (size_t)rows * sizeof(float2), A, &PS->far);
        }
        default:
            return fail(VFMM_ERR_INTERNAL, "unknown far-field contraction");
    }
}

// Partial-sum buffers of the split contractions (float2 elements): room for kMaxSplit partial sets
// wherever a contraction may split (so that vfmm_tune can pick any factor without a new
// workspace), the current factor elsewhere, and the slab of an entry-major contraction. The near
// field and S2L each have their own, since they may run beside each other and beside the rest.
void split_part_elems(const DeviceTree& T, const PlanSet& PS, const vfmm_ops& o, size_t elems[3]) {
    const MixedOps* mo = (const MixedOps*)o.mixed;
    const size_t R = (size_t)PS.R;
    auto need1 = [](const SplitPlan& P, size_t rows, int Rp) -> size_t {
        if (P.entry) return (size_t)P.slab_rows * Rp;  // one slab row per entry
        const int f = P.may_split ? kMaxSplit : P.split;
        return f > 1 ? (size_t)f * rows * Rp : 0;
    };
    // room for the alternative form too, so that vfmm_tune can switch without a new workspace
    auto need = [&](const SplitPlan& P, size_t rows, int Rp) -> size_t {
        return std::max(need1(P, rows, Rp), P.alt ? need1(*P.alt, rows, Rp) : size_t(0));
    };
    size_t a = need(PS.near, T.n_leaves * R, mo->Rp);
    size_t b = need(PS.m2l, T.n_boxes * R, mo->Rx);
    size_t c = need(PS.far, T.n_leaves * R, mo->Rp);
    size_t d = need(PS.s2l, T.n_boxes * R, mo->Rx);
    size_t e = need(PS.s2m, T.n_leaves * R, mo->Rx);
    elems[0] = std::max(std::max(b, c), e);
    elems[1] = a;
    elems[2] = d;
}

// ---------------------------------------------------------------- S2M
// One CTA per virtual leaf (leaf, r): coefficient 0 (the mass) in FP64, the rest from the split
// contraction scaled back by 2^(E_f[r] + E_row).
// With split > 1 the contraction's split-K partial sums part[s][row][Rx] are summed here (the
// reduction kernel's order and arithmetic) instead of read from out.
__global__ void s2m_finish_kernel(int nleaf, int R, int kk, int p, int Rx, const int32_t* __restrict__ box_of_leaf,
                                  const int32_t* __restrict__ level, double width, const double* __restrict__ f,
                                  const double* __restrict__ s2m, const float2* __restrict__ out,
                                  const float2* __restrict__ part, int split, size_t part_stride,
                                  const int* __restrict__ E, const int* __restrict__ Ef, double* __restrict__ Mexp,
                                  unsigned* __restrict__ glev) {
    const int vl = blockIdx.x;
    const int leaf = vl / R, r = vl - leaf * R;
    const int b = box_of_leaf[leaf];
    const double h = ldexp(width, -level[b]);
    const int P2 = 2 * (p + 1);
    double* M = Mexp + ((size_t)b * R + r) * P2;
    const double* fl = f + ((size_t)r * nleaf + leaf) * kk;
    int e = INT_MIN;  // exponent bound of this thread's parts (level exponents of the M2L operand)
    if (threadIdx.x < 32) {
        double m = 0.0;
        for (int s = threadIdx.x; s < kk; s += 32) m += s2m[s] * fl[s];
        for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
        if (threadIdx.x == 0) {
            M[0] = h * h * m;
            M[1] = 0.0;
            e = part_exp(M[0], 0);
        }
    }
    // h^2 = wm^2 2^(2 (lw - level)): the power of two goes into the exponent bits
    int lw = 0;
    const double wm = 2.0 * frexp(width, &lw);
    const int ef = Ef[r] + 2 * (lw - 1 - level[b]);
    for (int q = threadIdx.x; q < 2 * p; q += blockDim.x) {
        float2 v;
        if (split > 1) {
            float hi = 0.0f, lo = 0.0f;
            for (int sp = 0; sp < split; ++sp) df_add(hi, lo, part[(size_t)sp * part_stride + (size_t)vl * Rx + q]);
            v = df_final(hi, lo);
        } else {
            v = out[(size_t)vl * Rx + q];
        }
        const double m = f2d_scaled(v.x, ef + E[q]) + f2d_scaled(v.y, ef + E[q]);
        M[2 + q] = wm == 1.0 ? m : wm * wm * m;
        e = max(e, part_exp(M[2 + q], 2 + q));
    }
    // one atomic per CTA (the level slots are few and shared by every leaf of a level)
    if (level[b] >= 2) level_exp_max_block(e, glev + (size_t)level[b] * R + r);
}

int s2m_mixed(const DeviceTree& T, const PlanSet& PS, const vfmm_ops& o, const double* f, double* Mexp,
              const MixedWork& w, cudaStream_t st) {
    const MixedOps* mo = (const MixedOps*)o.mixed;
    VFMM_CHECK(split_gemm(PS.s2m, w.fsl, mo->tm_s2m, mo->Kp, mo->Rx, w.s2m_out, w.err, w.part,
                          (size_t)T.n_leaves * PS.R, mo->slices[kCtrS2M], st, w.cev ? w.cev + 2 : nullptr,
                          kDeferSplits));
    // the split-K partials (when the plan splits) are summed by the finishing kernel
    const int sp = (!PS.s2m.entry && w.part) ? PS.s2m.split : 1;
    const size_t stride = (size_t)T.n_leaves * PS.R * mo->Rx;
    s2m_finish_kernel<<<T.n_leaves * PS.R, 128, 0, st>>>(T.n_leaves, PS.R, o.k * o.k, o.p, mo->Rx, T.box_of_leaf,
                                                         T.level, T.width, f, o.s2m, w.s2m_out, w.part, sp, stride,
                                                         mo->s2m_E, w.Ef, Mexp, w.glev);
    VFMM_CUDA(cudaGetLastError());
    return VFMM_OK;
}

// ---------------------------------------------------------------- M2L
// Level exponents of the non-leaf multipoles of levels >= 2 when no persistent pass computed them as
// it wrote them (per-level translation launches): a warp per virtual box.
__global__ void box_exp_kernel(const int32_t* __restrict__ boxes, int nbox, int R, int P2, const int32_t* __restrict__ level,
                               const double* __restrict__ Mexp, unsigned* __restrict__ glev) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= (int64_t)nbox * R) return;
    const int b = boxes[w / R], r = (int)(w % R);
    int e = INT_MIN;
    for (int k = lane; k < P2; k += 32) e = max(e, part_exp(Mexp[((size_t)b * R + r) * P2 + k], k));
    level_exp_max(e, glev + (size_t)level[b] * R + r);
}

// One thread per 8 consecutive coefficients of a virtual box (one 16-byte store per slice).
__global__ void multipole_slice_kernel(const int32_t* __restrict__ level, int64_t vb0, int64_t vb1, int R, int P2,
                                       int Kx, const double* __restrict__ Mexp, const unsigned* __restrict__ G,
                                       bf16* __restrict__ msl) {
    const int cpr = Kx / 8;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (vb1 - vb0) * cpr) return;
    const int64_t vb = vb0 + q / cpr;
    const int c = (int)(q % cpr);
    const int64_t b = vb / R;
    const int r = (int)(vb - b * R);
    // coefficient k is scaled by 2^(floor(k/4) - G): within a chunk of 8, k/4 takes two values
    const int g = level_exp_value(G[(size_t)level[b] * R + r]);
    double v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int k = 8 * c + j;
        v[j] = k < P2 ? Mexp[(size_t)vb * P2 + k] : 0.0;
    }
    __align__(16) bf16 tmp[kSlices][8];
#pragma unroll
    for (int j = 0; j < 8; ++j) slice_fixed(v[j], g - ((8 * c + j) >> 2), &tmp[0][j], 8);
    bf16* out = msl + slice_at(vb, Kx, 8 * c);
#pragma unroll
    for (int i = 0; i < kSlices; ++i)
        *reinterpret_cast<uint4*>(out + (size_t)i * kKBlock) = *reinterpret_cast<uint4*>(tmp[i]);
}

int m2l_mixed(const DeviceTree& T, const PlanSet& PS, const vfmm_ops& o, const double* Mexp, const MixedWork& w,
              bool exps_done, cudaStream_t st) {
    const MixedOps* mo = (const MixedOps*)o.mixed;
    if (T.depth < 2 || PS.m2l.n_groups == 0) return VFMM_OK;
    const int P2 = 2 * (o.p + 1), R = PS.R;
    const int64_t vb0 = (int64_t)T.level_start[2] * R, vb1 = (int64_t)T.level_start[T.depth + 1] * R;
    // leaf multipoles took their level maxima in s2m_finish_kernel, non-leaf ones in the persistent
    // upward pass (exps_done) or here
    const int nb0 = T.nonleaf_start[2], nnl = T.nonleaf_start[T.depth + 1] - nb0;
    if (!exps_done && nnl > 0)
        box_exp_kernel<<<(unsigned)(((int64_t)nnl * R + 7) / 8), 256, 0, st>>>(T.nonleaf + nb0, nnl, R, P2, T.level,
                                                                             Mexp, w.glev);
    const int64_t n2 = (vb1 - vb0) * (mo->Kx / 8);
    multipole_slice_kernel<<<(unsigned)((n2 + 255) / 256), 256, 0, st>>>(T.level, vb0, vb1, R, P2, mo->Kx, Mexp,
                                                                          w.glev, (bf16*)w.msl);
    VFMM_CUDA(cudaGetLastError());
    // split-K partials (grouped form) are summed by the downward kernels that read the locals
    return split_gemm(PS.m2l, w.msl, mo->tm_m2l, mo->Kx, mo->Rx, w.m2l_out, w.err, w.part, (size_t)T.n_boxes * R,
                      mo->slices[kCtrM2L], st, w.cev ? w.cev + 4 : nullptr, kDeferSplits);
}

// ---------------------------------------------------------------- S2L
int s2l_mixed(const DeviceTree& T, const PlanSet& PS, const vfmm_ops& o, const MixedWork& w, cudaStream_t st) {
    const MixedOps* mo = (const MixedOps*)o.mixed;
    return split_gemm(PS.s2l, w.fsl, mo->tm_s2l, mo->Kp, mo->Rx, w.s2l_out, w.err, w.part_s2l,
                      (size_t)T.n_boxes * PS.R, mo->slices[kCtrS2L], st, w.cev ? w.cev + 6 : nullptr);
}

// ---------------------------------------------------------------- leaf far field
// One CTA per virtual leaf (leaf, r): operand rows (own local without coefficient 0, W multipoles)
// scaled by 2^-E_t, E_t the exponent of the largest of them.
__global__ void far_operand_kernel(int nleaf, int R, int P2, int Kx, const int32_t* __restrict__ box_of_leaf,
                                   const int32_t* __restrict__ far_slot, const int32_t* __restrict__ wptr,
                                   const int32_t* __restrict__ widx, const double* __restrict__ Mexp,
                                   const double* __restrict__ Lexp, int* __restrict__ Et, bf16* __restrict__ aprep) {
    __shared__ int red[4];
    const int vl = blockIdx.x;
    const int leaf = vl / R, r = vl - leaf * R;
    const int b = box_of_leaf[leaf];
    const int s0 = far_slot[leaf], ns = far_slot[leaf + 1] - s0;
    auto value = [&](int j, int k) -> double {
        if (k >= P2) return 0.0;
        if (j == 0) return k >= 2 ? Lexp[((size_t)b * R + r) * P2 + k] : 0.0;
        return Mexp[((size_t)widx[wptr[b] + j - 1] * R + r) * P2 + k];
    };
    // E_t = exponent bound of the largest value, as the largest exponent bound (integer work). Both
    // passes walk the same (slot, k < Kx) positions, so the first keeps up to kCache values per thread
    // in registers for the second (values of k >= P2 are zero).
    constexpr int kCache = 16;
    double cache[kCache];
    int em = INT_MIN;
    const int nq = ns * Kx;
#pragma unroll
    for (int c = 0; c < kCache; ++c) {
        const int q = threadIdx.x + c * (int)blockDim.x;
        cache[c] = q < nq ? value(q / Kx, q % Kx) : 0.0;
        if (cache[c] != 0.0) em = max(em, exp_bound(cache[c]));
    }
    for (int q = threadIdx.x + kCache * (int)blockDim.x; q < nq; q += blockDim.x) {
        const double v = value(q / Kx, q % Kx);
        if (v != 0.0) em = max(em, exp_bound(v));
    }
    for (int o = 16; o > 0; o >>= 1) em = max(em, __shfl_xor_sync(0xffffffffu, em, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = em;
    __syncthreads();
    int e = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) e = max(e, red[w]);
    if (e == INT_MIN) e = 0;  // all zero
    if (threadIdx.x == 0) Et[vl] = e;
#pragma unroll
    for (int c = 0; c < kCache; ++c) {
        const int q = threadIdx.x + c * (int)blockDim.x;
        if (q < nq) slice_fixed(cache[c], e, aprep + slice_at((size_t)(s0 + q / Kx) * R + r, Kx, q % Kx), kKBlock);
    }
    for (int q = threadIdx.x + kCache * (int)blockDim.x; q < nq; q += blockDim.x) {
        const int j = q / Kx, k = q % Kx;
        slice_fixed(value(j, k), e, aprep + slice_at((size_t)(s0 + j) * R + r, Kx, k), kKBlock);
    }
}

int far_leaf_mixed(const DeviceTree& T, const PlanSet& PS, const vfmm_ops& o, const double* Mexp, const double* Lexp,
                   const MixedWork& w, cudaStream_t st) {
    const MixedOps* mo = (const MixedOps*)o.mixed;
    far_operand_kernel<<<T.n_leaves * PS.R, 128, 0, st>>>(T.n_leaves, PS.R, 2 * (o.p + 1), mo->Kx, T.box_of_leaf,
                                                          T.far_slot, T.lptr[VFMM_LIST_W], T.lidx[VFMM_LIST_W], Mexp,
                                                          Lexp, w.Et, (bf16*)w.aprep);
    VFMM_CUDA(cudaGetLastError());
    return split_gemm(PS.far, w.aprep, mo->tm_far, mo->Kx, mo->Rp, w.far_out, w.err, w.part,
                      (size_t)T.n_leaves * PS.R, mo->slices[kCtrFar], st, w.cev ? w.cev + 8 : nullptr,
                      kDeferSegments);
}

}  // namespace vfmm

using namespace vfmm;

extern "C" int vfmm_solve_work(const vfmm_tree* tree, const vfmm_ops* ops, int32_t nrhs, double* out) {
    if (!tree || !ops || !out) return fail(VFMM_ERR_INVALID_ARG, "null argument");
    if (nrhs < 1) return fail(VFMM_ERR_INVALID_ARG, "nrhs must be >= 1");
    const DeviceTree& T = tree->t;
    for (int i = 0; i < VFMM_N_WORK; ++i) out[i] = 0.0;
    const double kk = (double)ops->k * ops->k;
    out[5] = 2.0 * 3.0 * kk * kk * (double)T.llen[VFMM_LIST_U] * nrhs;
    out[6] = (double)T.llen[VFMM_LIST_U];
    const MixedOps* mo = (const MixedOps*)ops->mixed;
    if (ops->precision != VFMM_MIXED || !mo) return VFMM_OK;
    const PlanSet* PS = nullptr;
    VFMM_CHECK(plans_for(T, nrhs, &PS));
    // per table of a tile and per K value: S (S + 1) / 2 products of 128 x 80 MACs
    auto tc = [&](const SplitPlan& P, int Kp, int Rp, int ctr) {
        const int S = mo->slices[ctr];
        return 2.0 * (double)P.entries * (Rp / table_rows_per_tile(P.transposed, Rp)) * (double)Kp * (S * (S + 1) / 2) *
               kTileM * mma_n(P.transposed, Rp);
    };
    out[0] = tc(PS->near, mo->Kp, mo->Rp, kCtrNear);
    out[1] = tc(PS->m2l, mo->Kx, mo->Rx, kCtrM2L);
    out[2] = tc(PS->far, mo->Kx, mo->Rp, kCtrFar);
    out[3] = tc(PS->s2l, mo->Kp, mo->Rx, kCtrS2L);
    out[4] = tc(PS->s2m, mo->Kp, mo->Rx, kCtrS2M);
    out[7] = (PS->near.entry ? 1 : 0) + (PS->m2l.entry ? 2 : 0) + (PS->far.entry ? 4 : 0) + (PS->s2l.entry ? 8 : 0);
    out[8] = PS->near.ctas;
    out[9] = PS->pass_ctas;
    return VFMM_OK;
}

extern "C" int vfmm_ops_set_slices(vfmm_ops* ops, const int32_t* slices) {
    if (!ops || !slices) return fail(VFMM_ERR_INVALID_ARG, "null argument");
    if (ops->precision != VFMM_MIXED || !ops->mixed) return fail(VFMM_ERR_INVALID_ARG, "not a VFMM_MIXED operator set");
    for (int c = 0; c < kNumCtr; ++c)
        if (slices[c] < kMinSlices || slices[c] > kSlices)
            return fail(VFMM_ERR_INVALID_ARG, "slice counts must lie in [" + std::to_string(kMinSlices) + ", " +
                                                  std::to_string(kSlices) + "]");
    MixedOps* mo = (MixedOps*)ops->mixed;
    for (int c = 0; c < kNumCtr; ++c) mo->slices[c] = slices[c];
    return VFMM_OK;
}

extern "C" int vfmm_ops_get_slices(const vfmm_ops* ops, int32_t* slices) {
    if (!ops || !slices) return fail(VFMM_ERR_INVALID_ARG, "null argument");
    if (ops->precision != VFMM_MIXED || !ops->mixed) return fail(VFMM_ERR_INVALID_ARG, "not a VFMM_MIXED operator set");
    const MixedOps* mo = (const MixedOps*)ops->mixed;
    for (int c = 0; c < kNumCtr; ++c) slices[c] = mo->slices[c];
    return VFMM_OK;
}
