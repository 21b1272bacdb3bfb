// The FMM passes of the box code (Section 3.1), with the gradient from differentiated tables and
// expansions (Section 3.2), and the solve driver of both forms (FP64 below; the split-BF16
// contractions of the mixed form are in mixed.cu and mixed_far.cu).
//
//   S2M      leaf multipoles  a = h^2 Q f                 (gather GEMM, all leaves)
//   M2M      finest parents first: one cooperative persistent pass for small trees (position-DFT
//            form, readiness counters), else one launch per level
//   M2L      dense per V entry (gather GEMM per offset) or plane-wave (planewave.cu)
//   DOWN     per level from 2 down the tree, one CTA per box:
//            b = L2L(parent) + sum_V M2L a_c (+ a_0(c) log h) + sum_X (2h)^2 R f_c (+ a_0(c) log h)
//   NEAR     per near configuration, T_cfg f_src for every U-list entry (gather GEMM into
//            a per-entry slab of the workspace; one launch for all 33 configurations)
//   L2T      far-field values from the leaf's local expansion (gather GEMM)
//   LEAF     one CTA per leaf: u = h^2 sum_U T f - (1/2pi) log(h) sum_U a_0(src) + L2T + sum_W M2T,
//            gradient = h sum_U T' f + L2T'/h + sum_W M2T'
//
// Workspace (caller-owned, from vfmm_workspace_size): status word, multipoles and locals
// [n_boxes][2(p+1)], near slabs [n_U][3kk], far values [n_leaves][3kk], M2L/S2L slabs or
// plane-waves, the mixed form's operands and outputs (+ I/O copies); see layout().
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "mixed.cuh"
#include "ops.cuh"
#include "tc_ptx.cuh"
#include "vfmm_internal.cuh"

namespace vfmm {

constexpr double kInv2Pi = 0.15915494309189533577;

// 2^e as a double, built from its exponent bits (exact, no libm call).

// Re of local coefficient 0 from the V and X lists of each virtual box (box, r): sum over V of
// Re(row 0 of M2L_c . a_c) + a_0(c) log h, and over X of (2h)^2 Re(S2L row 0) . f_c + a_0(c) log h.
// FP64; the other coefficients come from the split-precision M2L and S2L. Persistent CTAs hold the
// row-0 tables in shared memory; one warp per virtual box, the (entry, coefficient) pairs of eight
// V entries at a time spread over the lanes.
__global__ void __launch_bounds__(256) m2l_c0_kernel(int begin, int end, int R, int P, double width,
                                                     const int32_t* __restrict__ level,
                                                     const int32_t* __restrict__ vptr, const int32_t* __restrict__ vidx,
                                                     const int32_t* __restrict__ vcfg, const double2* __restrict__ m2l_r0,
                                                     const double* __restrict__ Mexp, double* __restrict__ c0,
                                                     const int32_t* __restrict__ xptr, const int32_t* __restrict__ xidx,
                                                     const int32_t* __restrict__ xcfg,
                                                     const int32_t* __restrict__ leaf_of_box,
                                                     const double* __restrict__ s2l_r0, const double* __restrict__ f,
                                                     int nleaf, int kk) {
    extern __shared__ __align__(16) unsigned char c0_raw[];
    double2* sM = reinterpret_cast<double2*>(c0_raw);           // [40][P]
    double* sX = reinterpret_cast<double*>(sM + kVCfg * P);      // [20][kk]
    for (int q = threadIdx.x; q < kVCfg * P; q += blockDim.x) sM[q] = m2l_r0[q];
    for (int q = threadIdx.x; q < kFarCfg * kk; q += blockDim.x) sX[q] = s2l_r0[q];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t total = (int64_t)(end - begin) * R;
    for (int64_t vw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; vw < total;
         vw += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int b = begin + (int)(vw / R), r = (int)(vw % R);
        const double h = ldexp(width, -level[b]);
        const double logh = log(h);
        // V list: the warp walks the entries; lane n takes coefficients n, n + 32 of the source
        // multipole (coalesced), partial sums stay per lane until one final reduction
        double acc = 0.0;
        const int e_end = vptr[b + 1];
        // V list in batches of 8 entries: the batch's (entry, coefficient) pairs spread over the lanes,
        // so all 32 lanes work whatever p is (coalesced within an entry's multipole)
        for (int e0 = vptr[b]; e0 < e_end; e0 += 8) {
            const int nb = min(8, e_end - e0);
            int j = 0, n = lane;
            while (n >= P) {
                n -= P;
                ++j;
            }
#pragma unroll 4
            for (int item = lane; item < nb * P; item += 32) {
                const int e = e0 + j;
                const double2 x = reinterpret_cast<const double2*>(Mexp + ((size_t)vidx[e] * R + r) * 2 * P)[n];
                const double2 m = sM[vcfg[e] * P + n];
                acc += m.x * x.x - m.y * x.y;
                n += 32;
                while (n >= P) {
                    n -= P;
                    ++j;
                }
            }
        }
        // log(h) a_0(c) of every V entry: one lane per entry
        double a0 = 0.0;
        for (int e = vptr[b] + lane; e < e_end; e += 32) a0 += Mexp[((size_t)vidx[e] * R + r) * 2 * P];
        acc += a0 * logh;
        // X list: (2h)^2 [Re(S2L row 0) . f_c + log(h) W . f_c], with W . f_c = a_0(c) / (2h)^2
        for (int e = xptr[b]; e < xptr[b + 1]; ++e) {
            const double* fc = f + ((size_t)r * nleaf + leaf_of_box[xidx[e]]) * kk;
            const double* r0 = sX + xcfg[e] * kk;
            double part = 0.0;
            for (int s = lane; s < kk; s += 32) part += r0[s] * fc[s];
            acc += 4.0 * h * h * part;
            if (lane == 0) acc += logh * Mexp[((size_t)xidx[e] * R + r) * 2 * P];
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) c0[(size_t)b * R + r] = acc;
    }
}

// ---------------------------------------------------------------- FP64 gather GEMM tile
// C_j[r] = scale_j * sum_s A[r][s] B_j[s] for rows r in [row0, row0 + 64), columns j < ncols.
constexpr int GBM = 64, GBN = 64, GBK = 16;

struct ColPtrs {
    const double* b[GBN];
    double* c[GBN];
    double scale[GBN];
};

__device__ inline void gemm_tile_fp64(const double* __restrict__ A, int M, int K, int row0, int ncols,
                                      const ColPtrs& cp) {
    __shared__ double As[GBK][GBM + 1];
    __shared__ double Bs[GBK][GBN + 1];
    const int t = threadIdx.x;
    const int tx = t % 16, ty = t / 16;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    const int lr = t / 4, lk = (t % 4) * 4;  // loader: row/column lr, k offset lk
    for (int k0 = 0; k0 < K; k0 += GBK) {
        {
            int r = row0 + lr;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int kk = k0 + lk + q;
                As[lk + q][lr] = (r < M && kk < K) ? A[(size_t)r * K + kk] : 0.0;
            }
            const double* bp = lr < ncols ? cp.b[lr] : nullptr;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int kk = k0 + lk + q;
                Bs[lk + q][lr] = (bp && kk < K) ? bp[kk] : 0.0;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GBK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        int c = tx * 4 + j;
        if (c >= ncols) continue;
        double* cptr = cp.c[c];
        double sc = cp.scale[c];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int r = row0 + ty * 4 + i;
            if (r < M) cptr[r] = sc * acc[i][j];
        }
    }
}

// Near field: one tile = (configuration, range of its U entries). Every gather GEMM here takes
// its column tile from blockIdx.x (no 65,535 limit) and its row tile from blockIdx.y.
__global__ void __launch_bounds__(256) near_gemm_kernel(const int4* __restrict__ tiles, const double* __restrict__ T,
                                                        int kk, const int32_t* __restrict__ u_by_cfg,
                                                        const int32_t* __restrict__ lidxU,
                                                        const int32_t* __restrict__ leaf_of_box,
                                                        const double* __restrict__ f, double* __restrict__ slab) {
    __shared__ ColPtrs cp;
    const int4 tl = tiles[blockIdx.x];  // cfg, begin, end
    const int ncols = min(GBN, tl.z - tl.y);
    if (threadIdx.x < GBN) {
        int j = threadIdx.x;
        if (j < ncols) {
            int e = u_by_cfg[tl.y + j];
            cp.b[j] = f + (size_t)leaf_of_box[lidxU[e]] * kk;
            cp.c[j] = slab + (size_t)e * 3 * kk;
        } else {
            cp.b[j] = nullptr;
            cp.c[j] = nullptr;
        }
        cp.scale[j] = 1.0;
    }
    __syncthreads();
    gemm_tile_fp64(T + (size_t)tl.x * 3 * kk * kk, 3 * kk, kk, blockIdx.y * GBM, ncols, cp);
}

// FP64 M2L over the V list: one tile = (offset, run of its V entries in offset order); column j =
// entry e, slab row e = M2L_real[offset] . multipole of the entry's source box (all 2(p+1) rows).
__global__ void __launch_bounds__(256) v_gemm_kernel(const int4* __restrict__ tiles, const double* __restrict__ A,
                                                     int P2, const int32_t* __restrict__ by_cfg,
                                                     const int32_t* __restrict__ lidxV, const double* __restrict__ Mexp,
                                                     double* __restrict__ vslab) {
    __shared__ ColPtrs cp;
    const int4 tl = tiles[blockIdx.x];  // offset, begin, end
    const int ncols = min(GBN, tl.z - tl.y);
    if (threadIdx.x < GBN) {
        const int j = threadIdx.x;
        if (j < ncols) {
            const int e = by_cfg[tl.y + j];
            cp.b[j] = Mexp + (size_t)lidxV[e] * P2;
            cp.c[j] = vslab + (size_t)e * P2;
        } else {
            cp.b[j] = nullptr;
            cp.c[j] = nullptr;
        }
        cp.scale[j] = 1.0;
    }
    __syncthreads();
    gemm_tile_fp64(A + (size_t)tl.x * P2 * P2, P2, P2, blockIdx.y * GBM, ncols, cp);
}

// FP64 S2L over the X list: column j = entry e (target box b, source leaf c), slab row e =
// (2 h_b)^2 S2L_real[configuration] . f_c.
__global__ void __launch_bounds__(256) x_gemm_kernel(const int4* __restrict__ tiles, const double* __restrict__ A,
                                                     int P2, int kk, const int32_t* __restrict__ by_cfg,
                                                     const int32_t* __restrict__ lidxX, const int32_t* __restrict__ x_tgt,
                                                     const int32_t* __restrict__ level, double width,
                                                     const int32_t* __restrict__ leaf_of_box,
                                                     const double* __restrict__ f, double* __restrict__ xslab) {
    __shared__ ColPtrs cp;
    const int4 tl = tiles[blockIdx.x];
    const int ncols = min(GBN, tl.z - tl.y);
    if (threadIdx.x < GBN) {
        const int j = threadIdx.x;
        if (j < ncols) {
            const int e = by_cfg[tl.y + j];
            const double h = ldexp(width, -level[x_tgt[e]]);
            cp.b[j] = f + (size_t)leaf_of_box[lidxX[e]] * kk;
            cp.c[j] = xslab + (size_t)e * P2;
            cp.scale[j] = 4.0 * h * h;
        } else {
            cp.b[j] = nullptr;
            cp.c[j] = nullptr;
            cp.scale[j] = 0.0;
        }
    }
    __syncthreads();
    gemm_tile_fp64(A + (size_t)tl.x * P2 * kk, P2, kk, blockIdx.y * GBM, ncols, cp);
}

// S2M: columns are leaves; output row = multipole of the leaf's box, scaled by h^2.
__global__ void __launch_bounds__(256) s2m_gemm_kernel(const double* __restrict__ S2M, int P2, int kk, int nleaf,
                                                       const int32_t* __restrict__ box_of_leaf,
                                                       const int32_t* __restrict__ level, double width,
                                                       const double* __restrict__ f, double* __restrict__ Mexp) {
    __shared__ ColPtrs cp;
    const int col0 = blockIdx.x * GBN;
    const int ncols = min(GBN, nleaf - col0);
    if (threadIdx.x < GBN) {
        int j = threadIdx.x;
        if (j < ncols) {
            int leaf = col0 + j;
            int b = box_of_leaf[leaf];
            double h = ldexp(width, -level[b]);
            cp.b[j] = f + (size_t)leaf * kk;
            cp.c[j] = Mexp + (size_t)b * P2;
            cp.scale[j] = h * h;
        } else {
            cp.b[j] = nullptr;
            cp.c[j] = nullptr;
            cp.scale[j] = 0.0;
        }
    }
    __syncthreads();
    gemm_tile_fp64(S2M, P2, kk, blockIdx.y * GBM, ncols, cp);
}

// L2T: columns are leaves; input = local expansion of the leaf's box.
__global__ void __launch_bounds__(256) l2t_gemm_kernel(const double* __restrict__ L2T, int P2, int kk, int nleaf,
                                                       const int32_t* __restrict__ box_of_leaf,
                                                       const double* __restrict__ Lexp, double* __restrict__ far) {
    __shared__ ColPtrs cp;
    const int col0 = blockIdx.x * GBN;
    const int ncols = min(GBN, nleaf - col0);
    if (threadIdx.x < GBN) {
        int j = threadIdx.x;
        if (j < ncols) {
            int leaf = col0 + j;
            cp.b[j] = Lexp + (size_t)box_of_leaf[leaf] * P2;
            cp.c[j] = far + (size_t)leaf * 3 * kk;
        } else {
            cp.b[j] = nullptr;
            cp.c[j] = nullptr;
        }
        cp.scale[j] = 1.0;
    }
    __syncthreads();
    gemm_tile_fp64(L2T, 3 * kk, P2, blockIdx.y * GBM, ncols, cp);
}

// Outputs j and P-1-j of one position of a triangular translation (mode 0, M2M: output o takes
// inputs n <= o; mode 1, L2L: n >= o), n ascending for each, fused into one loop of P + 1 steps so
// that every thread of a warp runs the same number of steps. M: [n][o] complex, x: inputs.
__device__ __forceinline__ void translate_pair(int mode, const double2* __restrict__ M, const double2* x, int P, int j,
                                               double2* out) {
    const int oa = j, ob = P - 1 - j;
    const int la = mode == 0 ? oa + 1 : P - oa;
    const int lb = ob != oa ? (mode == 0 ? ob + 1 : P - ob) : 0;
    const int na = mode == 0 ? 0 : oa, nb = mode == 0 ? 0 : ob;
    double re = 0.0, im = 0.0;
    for (int i = 0; i < la + lb; ++i) {
        if (i == la) {
            out[oa] = make_double2(re, im);
            re = im = 0.0;
        }
        const bool first = i < la;
        const int o = first ? oa : ob;
        const int n = first ? na + i : nb + (i - la);
        const double2 m = M[(size_t)n * P + o], v = x[n];
        re = fma(m.x, v.x, fma(-m.y, v.y, re));
        im = fma(m.x, v.y, fma(m.y, v.x, im));
    }
    out[lb ? ob : oa] = make_double2(re, im);
}

// ---------------------------------------------------------------- M2M and L2L (one CTA per non-leaf box)
// The translations are triangular: M2M output l of the parent takes child coefficients n <= l,
// L2L output m of a child takes parent coefficients l >= m. A thread owns one child position and
// the output pair (j, P-1-j), so every thread does P + 1 complex multiply-adds and no zero
// entry is read. mode 0 (M2M): in = the 4 consecutive child multipoles, out = parent multipole.
// mode 1 (L2L): in = parent local, out = the 4 child locals (written, later added to by the
// downward pass). Tables [pos][in][out] complex.
// ---- rotated real form of M2M and L2L (the factorisation is written out in tables.cu): for child
// position pos (sx = +1 when pos & 1, sy = +1 when pos & 2, s = sx sy), M2M is
// A_l = sigma_l sum_n Rm[n][l] (rho_n a_n) and L2L is c_m = rho_m sum_l Rl[l][m] (sigma_l b_l), with
// the Gaussian integers sigma_l = (i s)^floor(l/2) (sx + i sy)^(l mod 2) and rho_n = conj(sigma_n):
// one real triangular matrix for the four positions, 2 FP64 FMAs per entry instead of 4.

// x with its sign bit flipped when neg = 0x80000000 (integer work, no FP64 operation)
__device__ __forceinline__ double flip_sign(double x, unsigned neg) {
    return __hiloint2double(__double2hiint(x) ^ (int)neg, __double2loint(x));
}

// v sigma_n (sig) or v rho_n (!sig) for child position pos: sign changes and swaps, then one
// addition per component, exact for even n (the added term is zero).
__device__ __forceinline__ double2 rotate(double2 v, int pos, int n, bool sig) {
    constexpr unsigned kNeg = 0x80000000u;
    const unsigned nx = (pos & 1) ? 0u : kNeg, ny = (pos & 2) ? 0u : kNeg;
    const unsigned nc = sig ? (nx ^ ny) : (nx ^ ny ^ kNeg);  // unit u = i c: c = s (sigma), -s (rho)
    const unsigned ne = sig ? ny : (ny ^ kNeg);              // odd factor sx + i e: e = sy (sigma), -sy (rho)
    double wx, wy;  // v u^floor(n/2)
    switch ((n >> 1) & 3) {
        case 0: wx = v.x; wy = v.y; break;
        case 1: wx = flip_sign(v.y, nc ^ kNeg); wy = flip_sign(v.x, nc); break;
        case 2: wx = flip_sign(v.x, kNeg); wy = flip_sign(v.y, kNeg); break;
        default: wx = flip_sign(v.y, nc); wy = flip_sign(v.x, nc ^ kNeg); break;
    }
    // times (sx + i e) for odd n: (wx sx - wy e) + i (wy sx + wx e)
    const bool odd = n & 1;
    const double ax = odd ? flip_sign(wx, nx) : wx, bx = odd ? flip_sign(wy, ne ^ kNeg) : 0.0;
    const double ay = odd ? flip_sign(wy, nx) : wy, by = odd ? flip_sign(wx, ne) : 0.0;
    return make_double2(ax + bx, ay + by);
}

// One CTA per virtual box of a level, in the rotated real form (for levels with many boxes, where
// the FP64 pipes bound the translations): the four rotated input vectors are staged in shared
// memory, each thread takes one child position and one output row pair (j, P-1-j) of the real
// triangular matrix Mr [in][out] (P + 1 real-times-complex multiply-adds), rotates its two rows
// back, and M2M sums the four positions. mode 0 (M2M): in = the 4 consecutive child multipoles,
// out = parent multipole; mode 1 (L2L): in = parent local, out = the 4 child locals.
__global__ void __launch_bounds__(128) translate_kernel(int mode, const int32_t* __restrict__ boxes, int nbox, int R,
                                                        const int32_t* __restrict__ child0, int P,
                                                        const double* __restrict__ Mr, double2* __restrict__ ex) {
    extern __shared__ double2 sx[];  // [4P] rotated inputs, [4P] per-position results
    const int bi = blockIdx.x / R, r = blockIdx.x - bi * R;  // virtual box (box, right-hand side)
    if (bi >= nbox) return;
    const int b = boxes[bi], c0 = child0[b];
    double2* s_in = sx;
    double2* s_out = sx + 4 * P;
    for (int q = threadIdx.x; q < 4 * P; q += blockDim.x) {
        const int pos = q / P, n = q - pos * P;
        const double2 v = mode == 0 ? ex[((size_t)(c0 + pos) * R + r) * P + n] : ex[((size_t)b * R + r) * P + n];
        s_in[q] = rotate(v, pos, n, mode == 1);  // rho for M2M inputs, sigma for L2L inputs
    }
    __syncthreads();
    const int npair = (P + 1) / 2;
    for (int task = threadIdx.x; task < 4 * npair; task += blockDim.x) {
        const int pos = task / npair, j = task - pos * npair;
        const int oa = j, ob = P - 1 - j;
        const double2* x = s_in + pos * P;
        double ar = 0.0, ai = 0.0, br = 0.0, bi2 = 0.0;
        if (mode == 0) {
            for (int n = 0; n <= ob; ++n) {  // row oa takes n <= oa, row ob n <= ob
                const double2 v = x[n];
                if (n <= oa) {
                    const double m = __ldg(Mr + (size_t)n * P + oa);
                    ar = fma(m, v.x, ar);
                    ai = fma(m, v.y, ai);
                }
                const double m = __ldg(Mr + (size_t)n * P + ob);
                br = fma(m, v.x, br);
                bi2 = fma(m, v.y, bi2);
            }
        } else {
            for (int n = oa; n < P; ++n) {  // row oa takes n >= oa, row ob n >= ob
                const double2 v = x[n];
                const double m = __ldg(Mr + (size_t)n * P + oa);
                ar = fma(m, v.x, ar);
                ai = fma(m, v.y, ai);
                if (n >= ob) {
                    const double mb = __ldg(Mr + (size_t)n * P + ob);
                    br = fma(mb, v.x, br);
                    bi2 = fma(mb, v.y, bi2);
                }
            }
        }
        // rotate back: sigma for M2M outputs, rho for L2L outputs
        s_out[pos * P + oa] = rotate(make_double2(ar, ai), pos, oa, mode == 0);
        if (ob != oa) s_out[pos * P + ob] = rotate(make_double2(br, bi2), pos, ob, mode == 0);
    }
    __syncthreads();
    if (mode == 0) {
        for (int o = threadIdx.x; o < P; o += blockDim.x) {
            const double2 a0 = s_out[o], a1 = s_out[P + o], a2 = s_out[2 * P + o], a3 = s_out[3 * P + o];
            ex[((size_t)b * R + r) * P + o] =
                make_double2((a0.x + a1.x) + (a2.x + a3.x), (a0.y + a1.y) + (a2.y + a3.y));
        }
    } else {
        for (int q = threadIdx.x; q < 4 * P; q += blockDim.x) ex[((size_t)(c0 + q / P) * R + r) * P + q % P] = s_out[q];
    }
}

// After a CTA has given up waiting for a bulk copy into its shared memory, thread 0 waits once
// more, with a longer bound, for the copy to land (the other threads may leave): the CTA's shared
// memory stays allocated, and no copy is left writing into it, until the copy has completed or
// this second wait also runs out.
__device__ __forceinline__ void settle_bulk_copy(uint32_t bar_a, const volatile int* never) {
    if (threadIdx.x == 0) tc::mbar_wait(bar_a, 0, never, 1ll << 27);
}

// Same translations with the 4 position tables held in shared memory (one bulk copy per CTA),
// persistent CTAs looping over the virtual boxes of the level: the table is read from L2 once
// per CTA instead of once per multiply-add. Used when 4 P^2 complex values fit (P <= 58).
constexpr int kTranslateThreads = 128;
__global__ void __launch_bounds__(kTranslateThreads) translate_smem_kernel(int mode, const int32_t* __restrict__ boxes,
                                                                           int nbox, int R,
                                                                           const int32_t* __restrict__ child0, int P,
                                                                           const double2* __restrict__ tab,
                                                                           double2* __restrict__ ex, int* err) {
    extern __shared__ __align__(128) unsigned char sm_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ volatile int no_abort;
    double2* sT = reinterpret_cast<double2*>(sm_raw);  // [4][P][P]
    double2* s_in = sT + 4 * P * P;                    // [4P]
    double2* s_out = s_in + 4 * P;                     // [4P]
    const uint32_t bar_a = tc::smem_u32(&bar);
    const uint32_t bytes = (uint32_t)(4 * P * P) * sizeof(double2);
    if (threadIdx.x == 0) {
        no_abort = 0;
        tc::mbar_init(bar_a, 1);
        tc::mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        tc::mbar_arrive_expect_tx(bar_a, bytes);
        constexpr uint32_t kChunk = 32768;
        for (uint32_t off = 0; off < bytes; off += kChunk)
            tc::bulk_copy_g2s(tc::smem_u32(sm_raw) + off, reinterpret_cast<const char*>(tab) + off,
                              min(kChunk, bytes - off), bar_a);
    }
    const bool landed = tc::mbar_wait(bar_a, 0, &no_abort);
    if (!__syncthreads_and(landed)) {  // one decision for the whole CTA
        if (threadIdx.x == 0 && err) atomicExch(err, 5);
        settle_bulk_copy(bar_a, &no_abort);
        return;
    }
    const int npair = (P + 1) / 2;
    for (int item = blockIdx.x; item < nbox * R; item += gridDim.x) {
        const int bi = item / R, r = item - bi * R;  // virtual box (box, right-hand side)
        const int b = boxes[bi], c0 = child0[b];
        if (mode == 0) {
            for (int q = threadIdx.x; q < 4 * P; q += blockDim.x)
                s_in[q] = ex[((size_t)(c0 + q / P) * R + r) * P + q % P];
        } else {
            for (int q = threadIdx.x; q < P; q += blockDim.x) s_in[q] = ex[((size_t)b * R + r) * P + q];
        }
        __syncthreads();
        for (int task = threadIdx.x; task < 4 * npair; task += blockDim.x) {
            const int pos = task / npair, j = task - pos * npair;
            const double2* M = sT + pos * P * P;
            const double2* x = mode == 0 ? s_in + pos * P : s_in;
            translate_pair(mode, M, x, P, j, s_out + pos * P);
        }
        __syncthreads();
        if (mode == 0) {
            for (int o = threadIdx.x; o < P; o += blockDim.x) {
                const double2 a0 = s_out[o], a1 = s_out[P + o], a2 = s_out[2 * P + o], a3 = s_out[3 * P + o];
                ex[((size_t)b * R + r) * P + o] =
                    make_double2((a0.x + a1.x) + (a2.x + a3.x), (a0.y + a1.y) + (a2.y + a3.y));
            }
        } else {
            for (int q = threadIdx.x; q < 4 * P; q += blockDim.x)
                ex[((size_t)(c0 + q / P) * R + r) * P + q % P] = s_out[q];
        }
        __syncthreads();
    }
}

static int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

static void launch_translate(int mode, const DeviceTree& T, int level, int R, int P, const double* tab,
                             const double* tab_r, double* ex, int* err, cudaStream_t st) {
    const int nbox = T.nonleaf_start[level + 1] - T.nonleaf_start[level];
    if (nbox <= 0) return;
    const size_t smem = (size_t)(4 * P * P + 8 * P) * sizeof(double2);
    // small levels: the table is fetched once per CTA; large levels (at least ~8 boxes per SM): one CTA
    // per box keeps many warps per SM feeding the FP64 pipes, the table staying in L1/L2
    if (smem <= 113 * 1024 && (long long)nbox * R <= 8ll * sm_count()) {  // two CTAs per SM
        static thread_local int attr_dev = -1;
        int dev = 0;
        cudaGetDevice(&dev);
        if (attr_dev != dev) {
            cudaFuncSetAttribute(translate_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 113 * 1024);
            attr_dev = dev;
        }
        const int grid = std::min<long long>((long long)nbox * R, 2ll * sm_count());
        translate_smem_kernel<<<grid, kTranslateThreads, smem, st>>>(
            mode, T.nonleaf + T.nonleaf_start[level], nbox, R, T.child0, P, reinterpret_cast<const double2*>(tab),
            reinterpret_cast<double2*>(ex), err);
        return;
    }
    const int threads = std::min(128, ((4 * ((P + 1) / 2) + 31) / 32) * 32);
    translate_kernel<<<(unsigned)nbox * R, threads, (size_t)8 * P * sizeof(double2), st>>>(
        mode, T.nonleaf + T.nonleaf_start[level], nbox, R, T.child0, P, tab_r, reinterpret_cast<double2*>(ex));
}

// ---------------------------------------------------------------- downward pass (one CTA per box)
struct DownArgs {
    int begin, end, P, kk, level;
    int R, nleaf;  // right-hand sides folded into the box rows (virtual box = box * R + r); leaves
    double width;
    const int32_t* parent;
    const int32_t* ix;
    const int32_t* iy;
    const int32_t *vptr, *vidx, *vcfg;
    const int32_t *xptr, *xidx, *xcfg;
    const int32_t* leaf_of_box;
    const double* l2l_t;
    const double* m2l_t;
    const double* s2l_t;
    const double* Mexp;
    const double* f;
    double* Lexp;
    // split-precision M2L rows 2..2p+1 (null in the FP64 form): (hi, lo) scaled by 2^-E[level][r]
    const float2* m2l_out;
    // split-K M2L: its partial sums [split][n_boxes * R][Rx], summed here when m2l_split > 1 (the
    // reduction kernel's order and arithmetic; that kernel is then not launched)
    const float2* m2l_part;
    int m2l_split;
    size_t m2l_stride;
    const int* m2l_E;   // [Rx] row exponents of the M2L tables
    const unsigned* m2l_G;  // [(depth + 1) R] biased level exponents of the multipole operand
    const double* m2l_c0;  // Re of local coefficient 0 from the V and X lists, with the log(h) terms
    const double* vslab;   // FP64 form: [n_V][2(p+1)] M2L of every V entry
    const double* xslab;   // FP64 form: [n_X][2(p+1)] S2L of every X entry
    const double* pwloc;   // FP64 form, plane-wave M2L: [n_boxes][2(p+1)] V-list locals (null: vslab)
    int lw;                 // root width = wm 2^lw, wm in [1, 2)
    double wm;
    const float2* s2l_out; // split-precision S2L rows 2..2p+1, scaled by 2^-(E_f + E_r)
    const int* s2l_E;
    const int* Ef;
    int Rx;
};

// M2L output (hi, lo) of virtual box vb, row q: from the split-K partials or the reduced output.
__device__ __forceinline__ float2 m2l_value(const DownArgs& d, size_t vb, int q) {
    if (d.m2l_split > 1) {
        float hi = 0.0f, lo = 0.0f;
        for (int s = 0; s < d.m2l_split; ++s) df_add(hi, lo, d.m2l_part[(size_t)s * d.m2l_stride + vb * d.Rx + q]);
        return df_final(hi, lo);
    }
    return d.m2l_out[vb * d.Rx + q];
}

__global__ void __launch_bounds__(64) down_kernel(DownArgs d) {
    const int R = d.R;
    const int b = d.begin + blockIdx.x / R, r = blockIdx.x % R;
    if (b >= d.end) return;
    const size_t vb = (size_t)b * R + r;
    const int P = d.P, t = threadIdx.x;
    const double h = ldexp(d.width, -d.level);
    const double logh = log(h);
    double re = 0.0, im = 0.0;
    if (d.level >= 3 && t < P) {
        // L2L from the parent, written by translate_kernel just before this launch
        re = d.Lexp[vb * 2 * P + 2 * t];
        im = d.Lexp[vb * 2 * P + 2 * t + 1];
    }
    if (!d.m2l_out && t < P) {
        // FP64 form: M2L and S2L rows from the per-entry slabs of the V and X GEMMs, in list order,
        // with the log(h) a_0 terms of the scaling
        if (d.pwloc) {
            re += d.pwloc[(size_t)b * 2 * P + 2 * t];
            im += d.pwloc[(size_t)b * 2 * P + 2 * t + 1];
        }
        for (int e = d.vptr[b]; e < d.vptr[b + 1]; ++e) {
            if (!d.pwloc) {
                re += d.vslab[(size_t)e * 2 * P + 2 * t];
                im += d.vslab[(size_t)e * 2 * P + 2 * t + 1];
            }
            if (t == 0) re += d.Mexp[((size_t)d.vidx[e] * R + r) * 2 * P] * logh;
        }
        for (int e = d.xptr[b]; e < d.xptr[b + 1]; ++e) {
            re += d.xslab[(size_t)e * 2 * P + 2 * t];
            im += d.xslab[(size_t)e * 2 * P + 2 * t + 1];
            if (t == 0) re += logh * d.Mexp[((size_t)d.xidx[e] * R + r) * 2 * P];
        }
    }
    if (d.m2l_out && t >= 1 && t < P && d.xptr[b + 1] > d.xptr[b]) {
        const float2 vr = d.s2l_out[vb * d.Rx + 2 * (t - 1)];
        const float2 vi = d.s2l_out[vb * d.Rx + 2 * (t - 1) + 1];
        const double sc = 4.0 * h * h * pow2(d.Ef[r]);
        re += sc * ((double)vr.x + (double)vr.y) * pow2(d.s2l_E[2 * (t - 1)]);
        im += sc * ((double)vi.x + (double)vi.y) * pow2(d.s2l_E[2 * (t - 1) + 1]);
    }
    if (d.m2l_out && t < P && (d.vptr[b + 1] > d.vptr[b] || d.xptr[b + 1] > d.xptr[b])) {
        if (t == 0) {
            re += d.m2l_c0[vb];
        } else if (d.vptr[b + 1] > d.vptr[b]) {
            const float2 vr = m2l_value(d, vb, 2 * (t - 1));
            const float2 vi = m2l_value(d, vb, 2 * (t - 1) + 1);
            const int g = level_exp_value(d.m2l_G[(size_t)d.level * R + r]);
            re += ((double)vr.x + (double)vr.y) * pow2(g + d.m2l_E[2 * (t - 1)]);
            im += ((double)vi.x + (double)vi.y) * pow2(g + d.m2l_E[2 * (t - 1) + 1]);
        }
    }
    if (t < P) {
        d.Lexp[vb * 2 * P + 2 * t] = re;
        d.Lexp[vb * 2 * P + 2 * t + 1] = im;
    }
}

// Mixed form: coefficient t of the local expansion of virtual box (b, r) at `level` = the L2L
// value (re, im) plus the split-precision M2L and S2L outputs scaled back by their exponents and
// the FP64 coefficient 0 (V and X rows 0 with the log(h) terms).
__device__ __forceinline__ double2 combine_local(const DownArgs& d, int level, int b, int r, int t, double re,
                                                 double im) {
    // (hi, lo) outputs to FP64 with their power-of-two scales folded into the exponent bits; the
    // S2L factor (2h)^2 = wm^2 2^(2 + 2 (lw - level)) for a root width wm 2^lw
    const size_t vb = (size_t)b * d.R + r;
    const bool has_v = d.vptr[b + 1] > d.vptr[b], has_x = d.xptr[b + 1] > d.xptr[b];
    if (has_x && t >= 1) {
        const float2 vr = d.s2l_out[vb * d.Rx + 2 * (t - 1)];
        const float2 vi = d.s2l_out[vb * d.Rx + 2 * (t - 1) + 1];
        const int e = d.Ef[r] + 2 + 2 * (d.lw - level);
        const int er = e + d.s2l_E[2 * (t - 1)], ei = e + d.s2l_E[2 * (t - 1) + 1];
        double sr = f2d_scaled(vr.x, er) + f2d_scaled(vr.y, er);
        double si = f2d_scaled(vi.x, ei) + f2d_scaled(vi.y, ei);
        if (d.wm != 1.0) {
            sr *= d.wm * d.wm;
            si *= d.wm * d.wm;
        }
        re += sr;
        im += si;
    }
    if (has_v || has_x) {
        if (t == 0) {
            re += d.m2l_c0[vb];
        } else if (has_v) {
            const float2 vr = m2l_value(d, vb, 2 * (t - 1));
            const float2 vi = m2l_value(d, vb, 2 * (t - 1) + 1);
            const int g = level_exp_value(d.m2l_G[(size_t)level * d.R + r]);
            const int er = g + d.m2l_E[2 * (t - 1)], ei = g + d.m2l_E[2 * (t - 1) + 1];
            re += f2d_scaled(vr.x, er) + f2d_scaled(vr.y, er);
            im += f2d_scaled(vi.x, ei) + f2d_scaled(vi.y, ei);
        }
    }
    return make_double2(re, im);
}

// Mixed form, one level: one thread per (virtual box, coefficient).
__global__ void down_mixed_kernel(DownArgs d) {
    const int P = d.P, R = d.R;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)(d.end - d.begin) * R * P) return;
    const size_t vb = (size_t)d.begin * R + (size_t)(q / P);
    const int t = (int)(q % P);
    const int b = (int)(vb / R), r = (int)(vb % R);
    double re = 0.0, im = 0.0;
    if (d.level >= 3) {  // L2L from the parent, written by the translation kernel just before
        re = d.Lexp[vb * 2 * P + 2 * t];
        im = d.Lexp[vb * 2 * P + 2 * t + 1];
    }
    const double2 v = combine_local(d, d.level, b, r, t, re, im);
    d.Lexp[vb * 2 * P + 2 * t] = v.x;
    d.Lexp[vb * 2 * P + 2 * t + 1] = v.y;
}

// ---------------------------------------------------------------- persistent tree passes
// One cooperative launch walks all levels. A unit is one virtual box, taken by a group of
// kGroupThreads threads (one warp on each of the SM's four schedulers, synchronised by a named
// barrier), and the real triangular matrix of the translation sits in shared memory for the whole
// pass. There is no barrier between levels: a unit waits (bounded) only for the expansions it reads,
// through per-box readiness counters, so a box starts as soon as its children (M2M) or its parent
// (L2L) are done. Every unit's inputs are produced by work that comes earlier in the global order,
// and each group takes its units in that order, so the earliest unfinished unit can always proceed
// (all CTAs are resident: cooperative launch). Data written by other CTAs are read through L2
// (ld.global.cg).
//
// Position-DFT form of the translations (this part retires about 2 FP64 FMAs per clock per SM, so
// the FP64 operation count per box sets the time of a level). With the rotated real form (tables.cu)
// M2M is A_l = sum_pos sigma^pos_l sum_n Rm[n][l] rho^pos_n a^pos_n, and the four child shifts
// are the Gaussian integers g_pos = i^e g_0, g_0 = 1 + i, with e = 0, 1, 2, 3 for the children
// at (+,+), (-,+), (-,-), (+,-) (child slots 3, 2, 0, 1). Then sigma^pos_l = i^(e l) sigma0_l and
// rho^pos_n = i^(-e n) rho0_n with sigma0_l = i^floor(l/2) (1 + i)^(l mod 2), rho0_n = conj(sigma0_n), so
//   M2M:  A_l = sigma0_l sum_{n<=l} Rm[n][l] E^(l mod 4)_n,   E^(c)_n = rho0_n F^((c - n) mod 4)_n,
//         F^(k)_n = sum_e i^(e k) a^(e)_n (a 4-point DFT over the children);
//   L2L:  c^(e)_m = rho0_m sum_c i^(e c) S^(c)_m,   S^(c)_m = sum_{l>=m, l-m = c mod 4} Rl[l][m] sigma0_l b_l.
// One real matrix-vector product per box instead of four complex ones: about P^2 FMAs plus 16 adds
// per coefficient for the DFT, against 8 P^2 FMAs with the four complex position tables.
constexpr int kPassThreads = 512;
constexpr int kGroupThreads = 128;
constexpr int kPassGroups = kPassThreads / kGroupThreads;
constexpr int kPassWarps = kPassThreads / 32;
constexpr int kPassMaxCtas = 152;  // largest pass grid

// Readiness counters of the dataflow tree passes: a producer publishes with a release add after its
// writes, a consumer polls with acquire loads before reading the expansion through L2.
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add_u32(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Waits (bounded) until *flag >= need. Gives up, recording code 6 in the status word, when the
// bound runs out; gives up at once when another wait already did (the status word is set).
__device__ bool wait_ready(const unsigned* flag, unsigned need, int* err) {
    for (long long it = 0; it < (1ll << 22); ++it) {
        if (ld_acquire_u32(flag) >= need) return true;
        if ((it & 63) == 63 && *(volatile int*)err) return false;
        __nanosleep(32);
    }
    atomicExch(err, 6);
    return false;
}

// Barrier of the kGroupThreads threads of group `grp` (named barrier 1 + grp; 0 is __syncthreads).
__device__ __forceinline__ void group_sync(int grp) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + grp), "n"(kGroupThreads) : "memory");
}

// v i^m (sign changes and swaps; exact).
__device__ __forceinline__ double2 mul_ipow(double2 v, int m) {
    switch (m & 3) {
        case 0: return v;
        case 1: return make_double2(-v.y, v.x);
        case 2: return make_double2(-v.x, -v.y);
        default: return make_double2(v.y, -v.x);
    }
}
// v sigma0_l = v i^floor(l/2) (1 + i)^(l mod 2): one addition per component for odd l.
__device__ __forceinline__ double2 mul_sigma0(double2 v, int l) {
    if (l & 1) v = make_double2(v.x - v.y, v.x + v.y);
    return mul_ipow(v, l >> 1);
}
// v rho0_n = v (-i)^floor(n/2) (1 - i)^(n mod 2).
__device__ __forceinline__ double2 mul_rho0(double2 v, int n) {
    if (n & 1) v = make_double2(v.x + v.y, v.y - v.x);
    return mul_ipow(v, -(n >> 1));
}
// sum_e i^(e k) x_e (one output of a 4-point DFT): (x0 +- x2) + i^k (x1 +- x3).
__device__ __forceinline__ double2 dft4(double2 x0, double2 x1, double2 x2, double2 x3, int k) {
    const bool odd = k & 1;
    const double2 u = odd ? make_double2(x0.x - x2.x, x0.y - x2.y) : make_double2(x0.x + x2.x, x0.y + x2.y);
    const double2 w = mul_ipow(odd ? make_double2(x1.x - x3.x, x1.y - x3.y) : make_double2(x1.x + x3.x, x1.y + x3.y), k);
    return make_double2(u.x + w.x, u.y + w.y);
}
// Child slot of DFT index e (g_pos = i^e (1 + i)).
__device__ __forceinline__ int child_of_e(int e) { return (0x1023 >> (4 * e)) & 0xF; }

struct PassArgs {
    int depth, R, P;
    const int32_t* nonleaf;
    const int32_t* nonleaf_start;  // device, depth + 2
    const int32_t* level_start;    // device, depth + 2
    const int32_t* child0;
    const double* tab;     // the real triangular matrix of the rotated form, [in][out]
    double2* ex;           // Mexp (upward) or Lexp (downward), [n_boxes * R][P] complex
    const int32_t* parent;
    unsigned int* ready;   // [n_boxes * R] readiness counters, zero at launch
    unsigned* glev;        // upward pass, mixed form: biased level exponents of the M2L operand (or null)
    const int32_t* level;
    int* err;
};

// Shared memory of a pass: the real matrix [P][P] (rounded up to 16 bytes), then per group the
// scratch of one unit: M2M E [4][P] and the partial sums [kGroupThreads][2]; L2L sigma0 b [P] and
// S [4][P] (complex).
__host__ __device__ inline size_t pass_table_bytes(int P) { return ((size_t)P * P * sizeof(double) + 15) & ~(size_t)15; }
__host__ __device__ inline size_t pass_group_bytes(int P) { return (size_t)(4 * P + 2 * kGroupThreads) * sizeof(double2); }
__host__ __device__ inline size_t pass_smem_bytes(int P) { return pass_table_bytes(P) + kPassGroups * pass_group_bytes(P); }

// The real matrix into shared memory (plain loads; P^2 doubles need not be a multiple of 16 bytes).
__device__ __forceinline__ void load_real_table(double* sR, const double* tab, int P) {
    for (int q = threadIdx.x; q < P * P; q += blockDim.x) sR[q] = __ldg(tab + q);
    __syncthreads();
}

// All M2M levels, finest parents first (the global unit order): unit = one virtual parent box.
__global__ void __launch_bounds__(kPassThreads, 1) upward_pass_kernel(PassArgs a) {
    extern __shared__ __align__(128) unsigned char pass_raw[];
    __shared__ int abort_grp[kPassGroups];
    const int P = a.P, R = a.R;
    double* sR = reinterpret_cast<double*>(pass_raw);
    const int grp = threadIdx.x / kGroupThreads, g = threadIdx.x % kGroupThreads;
    double2* sE = reinterpret_cast<double2*>(pass_raw + pass_table_bytes(P) + grp * pass_group_bytes(P));
    double2* sPart = sE + 4 * P;
    if (g == 0) abort_grp[grp] = 0;
    load_real_table(sR, a.tab, P);
    const int npair = (P + 1) / 2, ns = max(1, kGroupThreads / npair);  // row pairs x slices
    const int slot = grp * gridDim.x + blockIdx.x, nslots = gridDim.x * kPassGroups;
    int l = a.depth - 1, lbase = 0;
    int lunits = l >= 2 ? (a.nonleaf_start[l + 1] - a.nonleaf_start[l]) * R : 0;
    for (int u = slot;; u += nslots) {
        while (l >= 2 && u >= lbase + lunits) {
            lbase += lunits;
            if (--l >= 2) lunits = (a.nonleaf_start[l + 1] - a.nonleaf_start[l]) * R;
        }
        if (l < 2) break;
        const int vi = u - lbase, bi = vi / R, r = vi - bi * R;
        const int b = a.nonleaf[a.nonleaf_start[l] + bi], c0 = a.child0[b];
        // the non-leaf children's multipoles must be complete (leaf multipoles come from S2M)
        if (g < 4 && a.child0[c0 + g] >= 0 && !wait_ready(a.ready + (size_t)(c0 + g) * R + r, 1u, a.err))
            abort_grp[grp] = 1;
        group_sync(grp);
        if (abort_grp[grp]) return;
        // E^(c)_n over the (k, n) pairs, the four children read once per pair
        const double2* x = a.ex + ((size_t)c0 * R + r) * P;
        const size_t xs = (size_t)R * P;
        for (int q = g; q < 4 * P; q += kGroupThreads) {
            const int k = q / P, n = q - k * P;
            const double2 f = dft4(__ldcg(x + 3 * xs + n), __ldcg(x + 2 * xs + n), __ldcg(x + n),
                                   __ldcg(x + xs + n), k);
            sE[((k + n) & 3) * P + n] = mul_rho0(f, n);
        }
        group_sync(grp);
        // row pair (j, P-1-j), slice s of the fused loop over both rows' inputs (row oa takes n <= oa)
        if (g < npair * ns) {
            const int j = g / ns, s = g - j * ns;
            const int oa = j, ob = P - 1 - j;
            const int la = oa + 1, lb = ob != oa ? ob + 1 : 0;
            const double2* ea = sE + (oa & 3) * P;
            const double2* eb = sE + (ob & 3) * P;
            double ar = 0.0, ai = 0.0, br = 0.0, bi2 = 0.0;
            for (int i = s; i < la + lb; i += ns) {
                if (i < la) {
                    const double m = sR[i * P + oa];
                    const double2 e = ea[i];
                    ar = fma(m, e.x, ar);
                    ai = fma(m, e.y, ai);
                } else {
                    const int n = i - la;
                    const double m = sR[n * P + ob];
                    const double2 e = eb[n];
                    br = fma(m, e.x, br);
                    bi2 = fma(m, e.y, bi2);
                }
            }
            sPart[2 * g] = make_double2(ar, ai);
            sPart[2 * g + 1] = make_double2(br, bi2);
        }
        group_sync(grp);
        // row l: its slices summed in order, rotated by sigma0_l
        int e = INT_MIN;
        if (g < P) {
            const int j = min(g, P - 1 - g), w = g == j ? 0 : 1;
            double2 acc = sPart[2 * j * ns + w];
            for (int s = 1; s < ns; ++s) {
                const double2 t = sPart[2 * (j * ns + s) + w];
                acc = make_double2(acc.x + t.x, acc.y + t.y);
            }
            acc = mul_sigma0(acc, g);
            a.ex[((size_t)b * R + r) * P + g] = acc;
            e = max(part_exp(acc.x, 2 * g), part_exp(acc.y, 2 * g + 1));
            __threadfence();
        }
        // the M2L operand's level exponent (mixed form), taken as the coefficients are written
        if (a.glev && g < ((P + 31) & ~31)) level_exp_max(e, a.glev + (size_t)l * R + r);
        group_sync(grp);
        if (g == 0) red_release_add_u32(a.ready + (size_t)b * R + r, 1u);
    }
}

// Mixed form, all downward levels. First every box of level >= 2 gets its own terms (the M2L and
// S2L outputs and coefficient 0) in one warp unit per virtual box, counted 1 on its readiness word
// (level 2 boxes are then complete). Then, level by level, each non-leaf parent's local is shifted
// to its 4 children (L2L) and added to their own terms, counted 1 more (complete at 2).
__global__ void __launch_bounds__(kPassThreads, 1) downward_pass_kernel(PassArgs a, DownArgs d) {
    extern __shared__ __align__(128) unsigned char pass_raw[];
    __shared__ int abort_grp[kPassGroups];
    const int P = a.P, R = a.R;
    double* sR = reinterpret_cast<double*>(pass_raw);
    const int grp = threadIdx.x / kGroupThreads, g = threadIdx.x % kGroupThreads;
    double2* sG = reinterpret_cast<double2*>(pass_raw + pass_table_bytes(P) + grp * pass_group_bytes(P));
    double2* sS = sG + P;
    if (g == 0) abort_grp[grp] = 0;
    load_real_table(sR, a.tab, P);
    // own terms: one warp per virtual box
    {
        const int lane = threadIdx.x & 31;
        const int wslot = (threadIdx.x >> 5) * gridDim.x + blockIdx.x, nw = gridDim.x * kPassWarps;
        const int64_t vb0 = (int64_t)a.level_start[2] * R, vb1 = (int64_t)a.level_start[a.depth + 1] * R;
        for (int64_t vb = vb0 + wslot; vb < vb1; vb += nw) {
            const int b = (int)(vb / R), r = (int)(vb % R), lv = a.level[b];
            for (int t = lane; t < P; t += 32) a.ex[(size_t)vb * P + t] = combine_local(d, lv, b, r, t, 0.0, 0.0);
            __threadfence();
            __syncwarp();
            if (lane == 0) red_release_add_u32(a.ready + vb, 1u);
        }
    }
    const int npair = (P + 1) / 2;
    const int slot = grp * gridDim.x + blockIdx.x, nslots = gridDim.x * kPassGroups;
    int l = 3, lbase = 0;  // l: the children's level
    int lunits = l <= a.depth ? (a.nonleaf_start[l] - a.nonleaf_start[l - 1]) * R : 0;
    for (int u = slot;; u += nslots) {
        while (l <= a.depth && u >= lbase + lunits) {
            lbase += lunits;
            if (++l <= a.depth) lunits = (a.nonleaf_start[l] - a.nonleaf_start[l - 1]) * R;
        }
        if (l > a.depth) break;
        const int vi = u - lbase, bi = vi / R, r = vi - bi * R;
        const int b = a.nonleaf[a.nonleaf_start[l - 1] + bi], c0 = a.child0[b];
        // the parent's local must be complete, the children's own terms written
        bool ok = true;
        if (g == 4) ok = wait_ready(a.ready + (size_t)b * R + r, l - 1 == 2 ? 1u : 2u, a.err);
        else if (g < 4) ok = wait_ready(a.ready + (size_t)(c0 + g) * R + r, 1u, a.err);
        if (!ok) abort_grp[grp] = 1;
        group_sync(grp);
        if (abort_grp[grp]) return;
        const double2* bl = a.ex + ((size_t)b * R + r) * P;
        for (int t = g; t < P; t += kGroupThreads) sG[t] = mul_sigma0(__ldcg(bl + t), t);
        group_sync(grp);
        // S^(c) of the row pair (oa, ob): thread (j, c)
        for (int q = g; q < 4 * npair; q += kGroupThreads) {
            const int j = q >> 2, c = q & 3;
            const int oa = j, ob = P - 1 - j;
            double ar = 0.0, ai = 0.0;
            for (int li = oa + c; li < P; li += 4) {
                const double m = sR[li * P + oa];
                ar = fma(m, sG[li].x, ar);
                ai = fma(m, sG[li].y, ai);
            }
            sS[c * P + oa] = make_double2(ar, ai);
            if (ob != oa) {
                double br = 0.0, bi2 = 0.0;
                for (int li = ob + c; li < P; li += 4) {
                    const double m = sR[li * P + ob];
                    br = fma(m, sG[li].x, br);
                    bi2 = fma(m, sG[li].y, bi2);
                }
                sS[c * P + ob] = make_double2(br, bi2);
            }
        }
        group_sync(grp);
        // child e, coefficient m: own terms + rho0_m sum_c i^(e c) S^(c)_m
        for (int q = g; q < 4 * P; q += kGroupThreads) {
            const int e = q / P, m = q - e * P;
            const double2 h = mul_rho0(dft4(sS[m], sS[P + m], sS[2 * P + m], sS[3 * P + m], e), m);
            double2* out = a.ex + ((size_t)(c0 + child_of_e(e)) * R + r) * P + m;
            const double2 own = __ldcg(out);
            *out = make_double2(own.x + h.x, own.y + h.y);
        }
        __threadfence();
        group_sync(grp);
        if (g < 4) red_release_add_u32(a.ready + (size_t)(c0 + g) * R + r, 1u);
    }
}

// Mixed form, one CTA per virtual leaf (leaf, r), one thread per node: u, u_x, u_y = near + far +
// scalar, the split contraction outputs (hi, lo) scaled back by their power-of-two exponents. The
// scalar part, the same at every node of the leaf, is FP64:
// -(1/2pi) [log(h) sum_U a_0 + Re b_0 + sum_W a_0 (log h_w)], h_w = h / 2 (first warp, fixed-order sums).
struct LeafMixedArgs {
    int nleaf, R, kk, Rp, P, lw;
    double wm, width;
    const int32_t* box_of_leaf;
    const int32_t* level;
    const int32_t *uptr, *uidx, *wptr, *widx;
    const double* Mexp;
    const double* Lexp;
    const float2* nearmix;
    const int* Er;
    const int* Ef;
    const float2* farmix;
    const int* farE;
    const int* Et;
    // entry-major near field / leaf far field: the slab rows of every leaf's entries, summed here in
    // entry order (the arithmetic of the separate segmented sum, which these contractions then skip);
    // null: nearmix / farmix hold the sums
    const float2* near_slab;
    const int32_t* near_seg;  // [n_leaves + 1] first entry of each leaf
    const float2* far_slab;
    const int32_t* far_seg;
    double *u, *ux, *uy;
};

// Sum of the slab rows of entries [e0, e1), right-hand side r, row `row` (double-float, entry order).
__device__ __forceinline__ float2 slab_sum(const float2* __restrict__ slab, int e0, int e1, int R, int r, int Rp,
                                           int row) {
    float hi = 0.0f, lo = 0.0f;
#pragma unroll 4
    for (int e = e0; e < e1; ++e) df_add(hi, lo, slab[((size_t)e * R + r) * Rp + row]);
    return df_final(hi, lo);
}

__global__ void leaf_mixed_kernel(LeafMixedArgs a) {
    // width = wm 2^lw with wm in [1, 2): h = wm 2^(lw - lv), so every power-of-two scale is folded
    // into the exponents (f2d_scaled), times wm^(2, 1, -1) when wm is not one
    __shared__ double s_scal;
    const int nleaf = a.nleaf, R = a.R, kk = a.kk, Rp = a.Rp, lw = a.lw;
    const double wm = a.wm;
    const unsigned vl = blockIdx.x;
    const int t = threadIdx.x;
    const unsigned leaf = vl / (unsigned)R, r = vl - leaf * (unsigned)R;
    const int b = a.box_of_leaf[leaf];
    const int lv = a.level[b];
    // the node values first (their loads overlap the first warp's scalar sums), then the barrier
    double n0 = 0.0, n1 = 0.0, n2 = 0.0, f0 = 0.0, f1 = 0.0, f2 = 0.0;
    if (t < kk) {
        const float2* __restrict__ nearmix = a.nearmix;
        const float2* __restrict__ farmix = a.farmix;
        const int* __restrict__ Er = a.Er;
        const int* __restrict__ farE = a.farE;
        const int* __restrict__ Et = a.Et;
        const int* __restrict__ Ef = a.Ef;
        const float2* nm = nearmix + (size_t)vl * Rp;
        const float2* fm = farmix + (size_t)vl * Rp;
        const int en = Ef[r] + lw - lv, ef = Et[vl] + lv - lw;  // near scale h 2^E_f, far scale 2^E_t / h
        float2 v0, v1, v2, w0, w1, w2;
        if (a.near_slab) {
            const int s0 = a.near_seg[leaf], s1 = a.near_seg[leaf + 1];
            v0 = slab_sum(a.near_slab, s0, s1, R, r, Rp, t);
            v1 = slab_sum(a.near_slab, s0, s1, R, r, Rp, kk + t);
            v2 = slab_sum(a.near_slab, s0, s1, R, r, Rp, 2 * kk + t);
        } else {
            v0 = nm[t];
            v1 = nm[kk + t];
            v2 = nm[2 * kk + t];
        }
        if (a.far_slab) {
            const int s0 = a.far_seg[leaf], s1 = a.far_seg[leaf + 1];
            w0 = slab_sum(a.far_slab, s0, s1, R, r, Rp, t);
            w1 = slab_sum(a.far_slab, s0, s1, R, r, Rp, kk + t);
            w2 = slab_sum(a.far_slab, s0, s1, R, r, Rp, 2 * kk + t);
        } else {
            w0 = fm[t];
            w1 = fm[kk + t];
            w2 = fm[2 * kk + t];
        }
        const int e0 = en + lw - lv + Er[t], e1 = en + Er[kk + t], e2 = en + Er[2 * kk + t];
        n0 = f2d_scaled(v0.x, e0) + f2d_scaled(v0.y, e0);  // h^2 x near u
        n1 = f2d_scaled(v1.x, e1) + f2d_scaled(v1.y, e1);  // h x near u_x
        n2 = f2d_scaled(v2.x, e2) + f2d_scaled(v2.y, e2);
        const int g0 = Et[vl] + farE[t], g1 = ef + farE[kk + t], g2 = ef + farE[2 * kk + t];
        f0 = f2d_scaled(w0.x, g0) + f2d_scaled(w0.y, g0);
        f1 = f2d_scaled(w1.x, g1) + f2d_scaled(w1.y, g1);  // far u_x / h
        f2 = f2d_scaled(w2.x, g2) + f2d_scaled(w2.y, g2);
        if (wm != 1.0) {
            n0 *= wm * wm;
            n1 *= wm;
            n2 *= wm;
            f1 /= wm;
            f2 /= wm;
        }
    }
    if (t < 32) {
        const size_t P2 = 2 * (size_t)a.P;
        const double logh = log(ldexp(a.width, -lv));
        double m = 0.0, w0 = 0.0;
        for (int e = a.uptr[b] + t; e < a.uptr[b + 1]; e += 32) m += a.Mexp[((size_t)a.uidx[e] * R + r) * P2];
        for (int e = a.wptr[b] + t; e < a.wptr[b + 1]; e += 32) w0 += a.Mexp[((size_t)a.widx[e] * R + r) * P2];
        for (int o = 16; o > 0; o >>= 1) {
            m += __shfl_xor_sync(0xffffffffu, m, o);
            w0 += __shfl_xor_sync(0xffffffffu, w0, o);
        }
        if (t == 0)
            s_scal = -kInv2Pi * logh * m -
                     kInv2Pi * (a.Lexp[((size_t)b * R + r) * P2] + w0 * (logh - 0.6931471805599453));
    }
    __syncthreads();
    if (t >= kk) return;
    const size_t o = ((size_t)r * nleaf + leaf) * kk + t;
    a.u[o] = n0 + s_scal + f0;
    a.ux[o] = n1 + f1;
    a.uy[o] = n2 + f2;
}

// ---------------------------------------------------------------- leaf pass (one CTA per leaf)
struct LeafArgs {
    int nleaf, kk, k, P;
    double width;
    const int32_t* box_of_leaf;
    const int32_t* level;
    const int32_t *uptr, *uidx;
    const int32_t *wptr, *widx, *wcfg;
    const double* xhat;
    const double* slab;
    const double* far;
    const double* Mexp;
    double* u;
    double* ux;
    double* uy;
};

// FP64 form: one CTA per leaf sums the near-field slab rows, the log(h) term, the far values
// and the W-list multipoles (direct series) at its nodes.
__global__ void __launch_bounds__(256) leaf_kernel(LeafArgs a) {
    __shared__ double sa[2 * 64];
    const int leaf = blockIdx.x;
    const int t = threadIdx.x;
    const int kk = a.kk, P = a.P;
    const bool act = t < kk;
    const int b = a.box_of_leaf[leaf];
    const double h = ldexp(a.width, -a.level[b]);
    double u = 0.0, gx = 0.0, gy = 0.0, mass = 0.0;
    for (int e = a.uptr[b]; e < a.uptr[b + 1]; ++e) {
        if (act) {
            const double* s = a.slab + (size_t)e * 3 * kk;
            u += s[t];
            gx += s[kk + t];
            gy += s[2 * kk + t];
        }
        mass += a.Mexp[(size_t)a.uidx[e] * 2 * P];
    }
    u = h * h * u - kInv2Pi * log(h) * mass;
    gx *= h;
    gy *= h;
    const double hw = 0.5 * h;
    if (act) {
        const double* fr = a.far + (size_t)leaf * 3 * kk;
        u += fr[t];
        gx += fr[kk + t] / h;
        gy += fr[2 * kk + t] / h;
    }
    const double xt = act ? a.xhat[t % a.k] : 0.0, yt = act ? a.xhat[t / a.k] : 0.0;
    for (int e = a.wptr[b]; e < a.wptr[b + 1]; ++e) {
        const int w = a.widx[e];
        for (int q = t; q < 2 * P; q += blockDim.x) sa[q] = a.Mexp[(size_t)w * 2 * P + q];
        __syncthreads();
        if (act) {
            int px, py;
            far_pattern(a.wcfg[e], &px, &py);
            // zeta = (z - z_w)/h_w = 2 (xhat - D), D = (px, py)/4
            double zr = 2.0 * (xt - px / 4.0), zi = 2.0 * (yt - py / 4.0);
            double r2 = zr * zr + zi * zi;
            double vr = zr / r2, vi = -zi / r2;  // z^-1
            // S = sum_{n>=1} a_n v^n and S' = sum n a_n v^n by Horner
            double Sr = 0.0, Si = 0.0, Tr = 0.0, Ti = 0.0;
            for (int n = P - 1; n >= 1; --n) {
                double ar = sa[2 * n], ai = sa[2 * n + 1];
                double nr = Sr + ar, ni = Si + ai;
                Sr = nr * vr - ni * vi;
                Si = nr * vi + ni * vr;
                double mr = Tr + n * ar, mi = Ti + n * ai;
                Tr = mr * vr - mi * vi;
                Ti = mr * vi + mi * vr;
            }
            const double a0r = sa[0], a0i = sa[1];
            const double lz = 0.5 * log(r2), th = atan2(zi, zr);
            // Re Phi = Re(a0 (log h_w + log zeta)) + Re S
            double phir = a0r * (log(hw) + lz) - a0i * th + Sr;
            // dPhi/dzeta = v (a0 - S'), Phi' = dPhi/dzeta / h_w
            double dr = a0r - Tr, di = a0i - Ti;
            double pr = (vr * dr - vi * di) / hw, pi = (vr * di + vi * dr) / hw;
            u += -kInv2Pi * phir;
            gx += -kInv2Pi * pr;
            gy += kInv2Pi * pi;
        }
        __syncthreads();
    }
    if (act) {
        const size_t o = (size_t)leaf * kk + t;
        a.u[o] = u;
        a.ux[o] = gx;
        a.uy[o] = gy;
    }
}

// ---------------------------------------------------------------- host side
struct Workspace {
    bool fork = false;  // mixed form: run the near field and S2L on the thread's second stream
    double* vslab;      // FP64 form: per V entry M2L rows
    double* xslab;      // FP64 form: per X entry S2L rows
    double* pwX;        // FP64 form, plane-wave M2L: [n_boxes][4][s] outgoing coefficients (null: dense)
    double* pwL;        // FP64 form, plane-wave M2L: [n_boxes][2(p+1)] V-list local coefficients
    const PlanSet* ps;  // split-contraction plans for the folded right-hand sides (mixed form)
    unsigned int* ready; // [2][n_boxes * R] readiness counters of the persistent tree passes, then
                         // [(depth + 1) R] biased level exponents (mixed form)
    size_t ready_words;
    double* Mexp;
    double* Lexp;
    double* slab;
    double* far;
    double* io;  // f, u, ux, uy copies for the host entry point
    MixedWork mix;
    size_t bytes;
};

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Workspace carving. The mixed form folds all nrhs right-hand sides into one solve (every
// per-box and per-leaf buffer has nrhs rows per box); the FP64 form solves them one at a time.
static int layout(const DeviceTree& T, const vfmm_ops& o, int nrhs, bool io, Workspace* w, char* base,
                  size_t* bytes) {
    const size_t P2 = 2 * (size_t)(o.p + 1), kk = (size_t)o.k * o.k;
    size_t off = 0;
    auto take = [&](double** p, size_t n) {
        if (w) *p = (double*)(base + off);
        off += align256(std::max<size_t>(1, n) * sizeof(double));
    };
    double* dummy;
    const bool mixed = o.precision == VFMM_MIXED;
    const size_t R = mixed ? (size_t)nrhs : 1;
    // the status word comes first in both forms, so that it can be read back knowing only the
    // workspace address (vfmm_workspace_status)
    int* err = nullptr;
    {
        double* e = nullptr;
        take(&e, 1);
        err = reinterpret_cast<int*>(e);
    }
    take(w ? &w->Mexp : &dummy, (size_t)T.n_boxes * R * P2);
    take(w ? &w->Lexp : &dummy, (size_t)T.n_boxes * R * P2);
    {
        // readiness counters of the persistent passes, then the mixed form's biased level exponents:
        // one zeroing at the start of a solve covers both
        double* g = nullptr;
        const size_t words = 2 * (size_t)T.n_boxes * R + (size_t)(T.depth + 1) * R;
        take(&g, (words + 1) / 2);
        if (w) {
            w->ready = reinterpret_cast<unsigned int*>(g);
            w->ready_words = words;
        }
    }
    take(w ? &w->slab : &dummy, mixed ? 1 : (size_t)T.llen[VFMM_LIST_U] * 3 * kk);
    take(w ? &w->far : &dummy, mixed ? 1 : (size_t)T.n_leaves * 3 * kk);
    const bool pw = !mixed && o.m2l_form == VFMM_M2L_PLANEWAVE;
    take(w ? &w->vslab : &dummy, mixed || pw ? 1 : (size_t)T.llen[VFMM_LIST_V] * P2);
    if (pw) {
        take(w ? &w->pwX : &dummy, planewave_work_doubles(T.n_boxes, o));
        take(w ? &w->pwL : &dummy, (size_t)T.n_boxes * P2);
    } else if (w) {
        w->pwX = w->pwL = nullptr;
    }
    take(w ? &w->xslab : &dummy, mixed ? 1 : (size_t)T.llen[VFMM_LIST_X] * P2);
    if (mixed) {
        const MixedOps* mo = (const MixedOps*)o.mixed;
        const PlanSet* PS = nullptr;
        VFMM_CHECK(plans_for(T, (int)R, &PS));
        if (w) w->ps = PS;
        const size_t nl = (size_t)T.n_leaves * R, nb = (size_t)T.n_boxes * R;
        double* p = nullptr;
        take(&p, (nl * kSlices * mo->Kp * 2 + 7) / 8);
        if (w) w->mix.fsl = (void*)p;
        take(&p, nl * mo->Rp);
        if (w) w->mix.out = (float2*)p;
        take(&p, R);
        if (w) w->mix.fmax = (unsigned long long*)p;
        take(&p, (R + 1) / 2);
        if (w) w->mix.Ef = (int*)p;
        take(&p, nl * mo->Rx);
        if (w) w->mix.s2m_out = (float2*)p;
        if (w) w->mix.glev = w->ready + 2 * (size_t)T.n_boxes * R;
        take(&p, (nb * kSlices * mo->Kx * 2 + 7) / 8);
        if (w) w->mix.msl = (void*)p;
        take(&p, nb * mo->Rx);
        if (w) w->mix.m2l_out = (float2*)p;
        take(&p, nb);
        if (w) w->mix.m2l_c0 = p;
        take(&p, nb * mo->Rx);
        if (w) w->mix.s2l_out = (float2*)p;
        take(&p, ((size_t)T.n_far_slots * R * kSlices * mo->Kx * 2 + 7) / 8);
        if (w) w->mix.aprep = (void*)p;
        take(&p, (nl + 1) / 2);
        if (w) w->mix.Et = (int*)p;
        take(&p, nl * mo->Rp);
        if (w) w->mix.far_out = (float2*)p;
        size_t np[3] = {0, 0, 0};
        split_part_elems(T, *PS, o, np);
        float2** bufs[3] = {w ? &w->mix.part : nullptr, w ? &w->mix.part_side : nullptr,
                            w ? &w->mix.part_s2l : nullptr};
        for (int i = 0; i < 3; ++i) {
            take(&p, std::max<size_t>(np[i], 1));  // one float2 per double
            if (w) *bufs[i] = np[i] ? (float2*)p : nullptr;
        }
    } else if (w) {
        w->mix = MixedWork();
        w->ps = &T.plans;
    }
    if (w) w->mix.err = err;
    if (io) take(w ? &w->io : &dummy, (size_t)4 * nrhs * T.n_leaves * kk);
    else if (w) w->io = nullptr;
    if (w) w->bytes = off;
    *bytes = off;
    return VFMM_OK;
}

// V or X list grouped by configuration (host counting sort of the entries) and cut into GEMM
// tiles of at most GBN entries of one configuration; all device arrays in one allocation.
static int build_list_groups(DeviceTree* T, const std::vector<int32_t>& cfg, const std::vector<int32_t>& ptr, int ncfg,
                             int32_t** by_cfg, int32_t** tiles_out, int32_t* n_tiles, int32_t** tgt_out,
                             cudaStream_t st) {
    const int64_t n = (int64_t)cfg.size();
    std::vector<int64_t> start(ncfg + 1, 0);
    for (int64_t e = 0; e < n; ++e) ++start[cfg[e] + 1];
    for (int c = 0; c < ncfg; ++c) start[c + 1] += start[c];
    std::vector<int32_t> order(std::max<int64_t>(n, 1));
    std::vector<int64_t> fill(start.begin(), start.end() - 1);
    for (int64_t e = 0; e < n; ++e) order[fill[cfg[e]]++] = (int32_t)e;
    std::vector<int4> tiles;
    for (int c = 0; c < ncfg; ++c)
        for (int64_t b = start[c]; b < start[c + 1]; b += GBN)
            tiles.push_back(make_int4(c, (int)b, (int)std::min<int64_t>(b + GBN, start[c + 1]), 0));
    *n_tiles = (int32_t)tiles.size();
    std::vector<int32_t> tgt;
    if (tgt_out) {
        tgt.assign(std::max<int64_t>(n, 1), 0);
        for (int b = 0; b < T->n_boxes; ++b)
            for (int e = ptr[b]; e < ptr[b + 1]; ++e) tgt[e] = b;
    }
    // [tiles (int4)][order][tgt], each piece 16-byte aligned
    const size_t n_tile_ints = 4 * std::max<size_t>(1, tiles.size());
    const size_t n_order = (order.size() + 3) / 4 * 4;
    std::vector<int32_t> host(n_tile_ints + n_order + tgt.size(), 0);
    if (!tiles.empty()) std::memcpy(host.data(), tiles.data(), tiles.size() * sizeof(int4));
    std::copy(order.begin(), order.end(), host.begin() + n_tile_ints);
    std::copy(tgt.begin(), tgt.end(), host.begin() + n_tile_ints + n_order);
    int32_t* dev = nullptr;
    VFMM_CHECK(tree_malloc(reinterpret_cast<void**>(&dev), host.size() * sizeof(int32_t), st));
    VFMM_CUDA(cudaMemcpyAsync(dev, host.data(), host.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    *tiles_out = dev;  // owns the allocation
    *by_cfg = dev + n_tile_ints;
    if (tgt_out) *tgt_out = dev + n_tile_ints + n_order;
    return VFMM_OK;
}

int build_near_tiles(DeviceTree* T, const HostLists& H, cudaStream_t st) {
    VFMM_CHECK(build_list_groups(T, H.cfg[VFMM_LIST_V], H.ptr[VFMM_LIST_V], kVCfg, &T->v_by_cfg, &T->v_tiles,
                                 &T->n_v_tiles, nullptr, st));
    VFMM_CHECK(build_list_groups(T, H.cfg[VFMM_LIST_X], H.ptr[VFMM_LIST_X], kFarCfg, &T->x_by_cfg, &T->x_tiles,
                                 &T->n_x_tiles, &T->x_tgt, st));
    std::vector<int4> tiles;
    for (int c = 0; c < kNearCfg; ++c)
        for (int64_t b = T->u_cfg_start[c]; b < T->u_cfg_start[c + 1]; b += GBN)
            tiles.push_back(make_int4(c, (int)b, (int)std::min<int64_t>(b + GBN, T->u_cfg_start[c + 1]), 0));
    T->n_near_tiles = (int)tiles.size();
    tree_free(T->near_tiles);
    T->near_tiles = nullptr;
    VFMM_CHECK(tree_malloc(reinterpret_cast<void**>(&T->near_tiles), std::max<size_t>(1, tiles.size()) * sizeof(int4), st));
    if (!tiles.empty())
        VFMM_CUDA(cudaMemcpyAsync(T->near_tiles, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
    return VFMM_OK;
}

// Optional stage timing: a start and a stop event around every stage.
struct StageEvents {
    cudaEvent_t ev[2 * VFMM_N_STAGES];
    int launches = 0;
};

enum { ST_S2M = 0, ST_M2M = 1, ST_DOWN = 2, ST_NEAR = 3, ST_L2T = 4, ST_LEAF = 5, ST_CONTRACTIONS = 6 };

static inline void mark(StageEvents* se, int stage, bool stop, cudaStream_t st) {
    if (se) cudaEventRecord(se->ev[2 * stage + (stop ? 1 : 0)], st);
}

static void fill_down_args(DownArgs& d, const DeviceTree& T, const vfmm_ops& o, const double* f, const Workspace& w,
                           int l, int R) {
    const MixedOps* mo = (const MixedOps*)o.mixed;
    d.R = R;
    d.nleaf = T.n_leaves;
    d.wm = 2.0 * std::frexp(T.width, &d.lw);
    d.lw -= 1;
    d.begin = T.level_start[l];
    d.end = T.level_start[l + 1];
    d.P = o.p + 1;
    d.kk = o.k * o.k;
    d.level = l;
    d.width = T.width;
    d.parent = T.parent;
    d.ix = T.ix;
    d.iy = T.iy;
    d.vptr = T.lptr[VFMM_LIST_V];
    d.vidx = T.lidx[VFMM_LIST_V];
    d.vcfg = T.lcfg[VFMM_LIST_V];
    d.xptr = T.lptr[VFMM_LIST_X];
    d.xidx = T.lidx[VFMM_LIST_X];
    d.xcfg = T.lcfg[VFMM_LIST_X];
    d.leaf_of_box = T.leaf_of_box;
    d.l2l_t = o.l2l_t;
    d.m2l_t = o.m2l_t;
    d.s2l_t = o.s2l_t;
    d.Mexp = w.Mexp;
    d.f = f;
    d.Lexp = w.Lexp;
    d.vslab = w.vslab;
    d.xslab = w.xslab;
    d.pwloc = w.pwL;
    d.m2l_out = mo ? w.mix.m2l_out : nullptr;
    // a grouped split-K M2L leaves its partial sums to the downward kernels (m2l_mixed defers them)
    const bool m2l_parts = mo && !w.ps->m2l.entry && w.ps->m2l.split > 1 && w.mix.part;
    d.m2l_part = m2l_parts ? w.mix.part : nullptr;
    d.m2l_split = m2l_parts ? w.ps->m2l.split : 1;
    d.m2l_stride = (size_t)T.n_boxes * R * (mo ? mo->Rx : 0);
    d.m2l_E = mo ? mo->m2l_E : nullptr;
    d.m2l_G = mo ? w.mix.glev : nullptr;
    d.m2l_c0 = mo ? w.mix.m2l_c0 : nullptr;
    d.s2l_out = mo ? w.mix.s2l_out : nullptr;
    d.s2l_E = mo ? mo->s2l_E : nullptr;
    d.Ef = mo ? w.mix.Ef : nullptr;
    d.Rx = mo ? mo->Rx : 0;
}

// Persistent passes (one cooperative launch for all levels) when every level is small enough that
// per-level launches would mostly wait on launch latency; larger levels keep one launch per level.
static bool use_passes(const DeviceTree& T, int R, int P) {
    const size_t smem = pass_smem_bytes(P);
    if (smem > 200 * 1024 || T.depth < 3) return false;
    int widest = 0;
    for (int l = 1; l <= T.depth; ++l) widest = std::max(widest, T.nonleaf_start[l + 1] - T.nonleaf_start[l]);
    return (long long)widest * R <= 16ll * sm_count();
}

template <typename... Args>
static int launch_pass(void (*kernel)(Args...), int R, int P, int widest_items, int cap, cudaStream_t st,
                       Args... args) {
    const size_t smem = pass_smem_bytes(P);
    static thread_local int attr_dev[2] = {-1, -1};
    const int slot = (void*)kernel == (void*)upward_pass_kernel ? 0 : 1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_dev[slot] != dev) {
        VFMM_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr_dev[slot] = dev;
    }
    int per_sm = 0;
    VFMM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kPassThreads, smem));
    if (per_sm < 1) return fail(VFMM_ERR_INTERNAL, "tree pass kernel does not fit on an SM");
    // A cooperative launch: a unit may wait for units held by any other CTA, so all CTAs must be
    // resident. One CTA per box of the widest level (the first group of each CTA takes a level's
    // first boxes, so that they run on different SMs), at most one per SM and at most kPassMaxCtas:
    // a smaller grid starts sooner when another stream's kernels still hold SMs (the launch waits
    // until the whole grid fits).
    int grid = std::max(1, std::min(std::min(per_sm * sm_count(), kPassMaxCtas), widest_items));
    if (cap > 0) grid = std::min(grid, cap);  // any grid works: units wait only on lower-numbered units
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeCooperative;
    attr.val.cooperative = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kPassThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    VFMM_CUDA(cudaLaunchKernelEx(&cfg, kernel, args...));
    return VFMM_OK;
}

// Second stream of the calling host thread on the current device, with its fork and join events:
// a split-precision solve runs its S2L and near-field contractions there, beside S2M, M2M and M2L.
// Created by the first call outside stream capture (a call under capture before that runs on one
// stream) and kept for the life of the process. One per thread, so that the event sequence of a
// solve cannot interleave with another thread's.
struct SideStream {
    cudaStream_t s = nullptr;    // S2L and the near field, lowest priority
    cudaStream_t hp = nullptr;   // everything else, highest priority: first to get SMs that free up
    cudaStream_t aux = nullptr;  // coefficient 0 beside M2L, highest priority
    // f sliced; S2L done; near field done; solve start; solve end; M2M done; coefficient 0 done
    cudaEvent_t ev[7] = {};
};

static SideStream* side_stream(cudaStream_t st) {
    constexpr int kMaxDevices = 16;
    thread_local SideStream slots[kMaxDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    SideStream& ss = slots[dev];
    if (ss.s) return &ss;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return nullptr;
    SideStream n;
    int least = 0, greatest = 0;
    bool ok = cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess;
    ok = ok && cudaStreamCreateWithPriority(&n.s, cudaStreamNonBlocking, least) == cudaSuccess;
    ok = ok && cudaStreamCreateWithPriority(&n.hp, cudaStreamNonBlocking, greatest) == cudaSuccess;
    ok = ok && cudaStreamCreateWithPriority(&n.aux, cudaStreamNonBlocking, greatest) == cudaSuccess;
    for (int i = 0; i < 7 && ok; ++i) ok = cudaEventCreateWithFlags(&n.ev[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        for (cudaEvent_t e : n.ev)
            if (e) cudaEventDestroy(e);
        if (n.s) cudaStreamDestroy(n.s);
        if (n.hp) cudaStreamDestroy(n.hp);
        if (n.aux) cudaStreamDestroy(n.aux);
        cudaGetLastError();
        return nullptr;
    }
    ss = n;
    return &ss;
}

// Kernels one split contraction launches: the contraction, and its split-K or segmented reduction
// unless the consumer takes that sum over (split_gemm's defer bits).
static int gemm_launches(const SplitPlan& P, int defer = 0) {
    const bool reduce = P.entry ? !(defer & kDeferSegments) : (P.split > 1 && !(defer & kDeferSplits));
    return P.n_groups > 0 ? 1 + (reduce ? 1 : 0) : 0;
}

// One solve of R right-hand sides (f: [R][n_leaves][k^2]). The mixed form folds them into the
// rows of every contraction (PS holds plans for R); the FP64 form takes R = 1.
static int solve_steps(const DeviceTree& T, const PlanSet& PS, const vfmm_ops& o, const double* f, double* u,
                       double* ux, double* uy, const Workspace& w, cudaStream_t st, StageEvents* se,
                       SideStream* side);

static int solve_one(const DeviceTree& T, const PlanSet& PS, const vfmm_ops& o, const double* f, double* u,
                     double* ux, double* uy, const Workspace& w, cudaStream_t st, StageEvents* se = nullptr) {
    // Mixed form with side streams: once f is sliced, S2L and then the near field run on a
    // low-priority stream while a high-priority stream takes every other step; the latter waits
    // for S2L before the downward combine and for the near field before the leaf kernels, and the
    // caller's stream waits for it at the end. Timed calls keep to the caller's stream.
    SideStream* side = (o.precision == VFMM_MIXED && w.fork && !se && !w.mix.cev) ? side_stream(st) : nullptr;
    if (!side) return solve_steps(T, PS, o, f, u, ux, uy, w, st, se, nullptr);
    VFMM_CUDA(cudaEventRecord(side->ev[3], st));
    VFMM_CUDA(cudaStreamWaitEvent(side->hp, side->ev[3], 0));
    VFMM_CHECK(solve_steps(T, PS, o, f, u, ux, uy, w, side->hp, se, side));
    VFMM_CUDA(cudaEventRecord(side->ev[4], side->hp));
    VFMM_CUDA(cudaStreamWaitEvent(st, side->ev[4], 0));
    return VFMM_OK;
}

static int solve_steps(const DeviceTree& T, const PlanSet& PS, const vfmm_ops& o, const double* f, double* u,
                       double* ux, double* uy, const Workspace& w, cudaStream_t st, StageEvents* se,
                       SideStream* side) {
    const int P = o.p + 1, P2 = 2 * P, kk = o.k * o.k;
    const int nleaf = T.n_leaves;
    const bool mixed = o.precision == VFMM_MIXED;
    const int R = PS.R;
    if (!mixed && R != 1) return fail(VFMM_ERR_INTERNAL, "the FP64 form solves one right-hand side at a time");
    const MixedOps* mo = (const MixedOps*)o.mixed;
    int launches = 0;
    const bool passes = use_passes(T, R, P);
    // readiness counters (persistent passes) and level exponents (mixed form) start at zero
    if (passes || mixed) VFMM_CUDA(cudaMemsetAsync(w.ready, 0, w.ready_words * sizeof(unsigned int), st));
    if (mixed) {
        // near field first: its f slices also feed S2M and S2L
        mark(se, ST_NEAR, false, st);
        VFMM_CHECK(near_slices(T, PS, o, f, w.mix, st));
        launches += 2;
        if (side) {
            VFMM_CUDA(cudaEventRecord(side->ev[0], st));
            VFMM_CUDA(cudaStreamWaitEvent(side->s, side->ev[0], 0));
            if (T.depth >= 2) {
                VFMM_CHECK(s2l_mixed(T, PS, o, w.mix, side->s));
                launches += gemm_launches(PS.s2l);
            }
            VFMM_CUDA(cudaEventRecord(side->ev[1], side->s));
            VFMM_CHECK(near_contract(T, PS, o, w.mix, side->s));
            VFMM_CUDA(cudaEventRecord(side->ev[2], side->s));
        } else {
            VFMM_CHECK(near_contract(T, PS, o, w.mix, st));
        }
        launches += gemm_launches(PS.near);
        mark(se, ST_NEAR, true, st);
    }
    // S2M
    mark(se, ST_S2M, false, st);
    if (mixed) {
        VFMM_CHECK(s2m_mixed(T, PS, o, f, w.Mexp, w.mix, st));
        launches += 1 + gemm_launches(PS.s2m, kDeferSplits);
    } else {
        ++launches;
        dim3 g((nleaf + GBN - 1) / GBN, (P2 + GBM - 1) / GBM);
        s2m_gemm_kernel<<<g, 256, 0, st>>>(o.s2m, P2, kk, nleaf, T.box_of_leaf, T.level, T.width, f, w.Mexp);
    }
    mark(se, ST_S2M, true, st);
    // M2M, finest parents first (levels >= 2 are the ones the lists read)
    mark(se, ST_M2M, false, st);
    int widest = 0;
    for (int l = 1; l <= T.depth; ++l) widest = std::max(widest, T.nonleaf_start[l + 1] - T.nonleaf_start[l]);
    if (passes) {
        PassArgs pa;
        pa.depth = T.depth;
        pa.R = R;
        pa.P = P;
        pa.nonleaf = T.nonleaf;
        pa.nonleaf_start = T.nonleaf_start_dev;
        pa.level_start = T.level_start_dev;
        pa.child0 = T.child0;
        pa.tab = o.m2m_r;
        pa.ex = reinterpret_cast<double2*>(w.Mexp);
        pa.parent = T.parent;
        pa.ready = w.ready;
        pa.glev = mixed ? w.mix.glev : nullptr;
        pa.level = T.level;
        pa.err = w.mix.err;
        VFMM_CHECK(launch_pass(upward_pass_kernel, R, P, widest * R, mixed ? PS.pass_ctas : 0, st, pa));
        ++launches;
    } else {
        for (int l = T.depth - 1; l >= 2; --l) {
            if (T.nonleaf_start[l + 1] > T.nonleaf_start[l]) ++launches;
            launch_translate(0, T, l, R, P, o.m2m_t, o.m2m_r, w.Mexp, w.mix.err, st);
        }
    }
    mark(se, ST_M2M, true, st);
    // downward pass
    mark(se, ST_DOWN, false, st);
    if (mixed && T.depth >= 2) {
        // coefficient 0 (FP64) needs only the multipoles: beside M2L when forked
        cudaStream_t c0s = st;
        if (side) {
            VFMM_CUDA(cudaEventRecord(side->ev[5], st));
            VFMM_CUDA(cudaStreamWaitEvent(side->aux, side->ev[5], 0));
            c0s = side->aux;
        }
        VFMM_CHECK(m2l_mixed(T, PS, o, w.Mexp, w.mix, passes, st));
        if (PS.m2l.n_groups > 0) launches += 3 + gemm_launches(PS.m2l, kDeferSplits);
        const int begin = T.level_start[2], end = T.level_start[T.depth + 1];
        const int64_t warps = (int64_t)(end - begin) * R;
        const size_t c0_smem = (size_t)kVCfg * P * sizeof(double2) + (size_t)kFarCfg * kk * sizeof(double);
        static thread_local int c0_attr_dev = -1;
        int dev = 0;
        cudaGetDevice(&dev);
        if (c0_attr_dev != dev) {
            cudaFuncSetAttribute(m2l_c0_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
            c0_attr_dev = dev;
        }
        const unsigned c0_grid = (unsigned)std::min<int64_t>((warps + 7) / 8, 3ll * sm_count());
        m2l_c0_kernel<<<c0_grid, 256, c0_smem, c0s>>>(
            begin, end, R, P, T.width, T.level, T.lptr[VFMM_LIST_V], T.lidx[VFMM_LIST_V], T.lcfg[VFMM_LIST_V],
            reinterpret_cast<const double2*>(mo->m2l_r0), w.Mexp, w.mix.m2l_c0, T.lptr[VFMM_LIST_X],
            T.lidx[VFMM_LIST_X], T.lcfg[VFMM_LIST_X], T.leaf_of_box, mo->s2l_r0, f, nleaf, kk);
        ++launches;
        if (side) {
            VFMM_CUDA(cudaEventRecord(side->ev[6], side->aux));
            VFMM_CUDA(cudaStreamWaitEvent(st, side->ev[6], 0));
        }
        if (!side) {
            VFMM_CHECK(s2l_mixed(T, PS, o, w.mix, st));
            launches += gemm_launches(PS.s2l);
        }
    }
    if (side) VFMM_CUDA(cudaStreamWaitEvent(st, side->ev[1], 0));
    if (!mixed) {
        // FP64 form: every M2L (V list) and S2L (X list) product as gather GEMMs grouped by
        // configuration, one slab row per list entry; the per-level kernels below sum them
        if (w.pwX) {
            // plane-wave form: outgoing waves of every box, then diagonal translations and the
            // incoming conversion per target box
            if (T.depth >= 2) {
                launches += 2;
                VFMM_CHECK(planewave_m2l(o, T.level_start[2], T.n_boxes, T.lptr[VFMM_LIST_V],
                                         T.lidx[VFMM_LIST_V], T.lcfg[VFMM_LIST_V], w.Mexp, w.pwX, w.pwL, st));
            }
        } else if (T.n_v_tiles > 0) {
            ++launches;
            dim3 g(T.n_v_tiles, (P2 + GBM - 1) / GBM);
            v_gemm_kernel<<<g, 256, 0, st>>>((const int4*)T.v_tiles, o.m2l_real, P2, T.v_by_cfg,
                                             T.lidx[VFMM_LIST_V], w.Mexp, w.vslab);
        }
        if (T.n_x_tiles > 0) {
            ++launches;
            dim3 g(T.n_x_tiles, (P2 + GBM - 1) / GBM);
            x_gemm_kernel<<<g, 256, 0, st>>>((const int4*)T.x_tiles, o.s2l_real, P2, kk, T.x_by_cfg,
                                             T.lidx[VFMM_LIST_X], T.x_tgt, T.level, T.width, T.leaf_of_box, f,
                                             w.xslab);
        }
    }
    if (mixed && passes) {
        DownArgs d;
        fill_down_args(d, T, o, f, w, 2, R);
        PassArgs pa;
        pa.depth = T.depth;
        pa.R = R;
        pa.P = P;
        pa.nonleaf = T.nonleaf;
        pa.nonleaf_start = T.nonleaf_start_dev;
        pa.level_start = T.level_start_dev;
        pa.child0 = T.child0;
        pa.tab = o.l2l_r;
        pa.ex = reinterpret_cast<double2*>(w.Lexp);
        pa.parent = T.parent;
        pa.ready = w.ready + (size_t)T.n_boxes * R;
        pa.glev = nullptr;
        pa.level = T.level;
        pa.err = w.mix.err;
        VFMM_CHECK(launch_pass(downward_pass_kernel, R, P, std::max(widest * R, 16 * R), PS.pass_ctas, st, pa, d));
        ++launches;
    }
    for (int l = 2; l <= T.depth && !(mixed && passes); ++l) {
        DownArgs d;
        fill_down_args(d, T, o, f, w, l, R);
        int n = d.end - d.begin;
        if (n <= 0) continue;
        if (l >= 3) {
            // L2L for every box of level l (children of the non-leaf boxes of level l - 1)
            launch_translate(1, T, l - 1, R, P, o.l2l_t, o.l2l_r, w.Lexp, w.mix.err, st);
            ++launches;
        }
        ++launches;
        if (mixed) {
            const int64_t nt = (int64_t)n * R * P;
            down_mixed_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(d);
        } else {
            down_kernel<<<(unsigned)n * R, 64, 0, st>>>(d);
        }
    }
    if (T.depth < 2) VFMM_CUDA(cudaMemsetAsync(w.Lexp, 0, (size_t)T.n_boxes * R * P2 * sizeof(double), st));
    else VFMM_CUDA(cudaMemsetAsync(w.Lexp, 0, (size_t)T.level_start[2] * R * P2 * sizeof(double), st));
    mark(se, ST_DOWN, true, st);
    if (!mixed) {
        mark(se, ST_NEAR, false, st);
        if (T.n_near_tiles > 0) {
            ++launches;
            dim3 g(T.n_near_tiles, (3 * kk + GBM - 1) / GBM);
            near_gemm_kernel<<<g, 256, 0, st>>>((const int4*)T.near_tiles, o.near, kk, T.u_by_cfg,
                                                T.lidx[VFMM_LIST_U], T.leaf_of_box, f, w.slab);
        }
        mark(se, ST_NEAR, true, st);
    }
    // far field at the leaves
    mark(se, ST_L2T, false, st);
    if (mixed) {
        VFMM_CHECK(far_leaf_mixed(T, PS, o, w.Mexp, w.Lexp, w.mix, st));
        launches += 1 + gemm_launches(PS.far, kDeferSegments);
    } else {
        ++launches;
        dim3 g((nleaf + GBN - 1) / GBN, (3 * kk + GBM - 1) / GBM);
        l2t_gemm_kernel<<<g, 256, 0, st>>>(o.l2t, P2, kk, nleaf, T.box_of_leaf, w.Lexp, w.far);
    }
    mark(se, ST_L2T, true, st);
    mark(se, ST_LEAF, false, st);
    LeafArgs a;
    a.nleaf = nleaf;
    a.kk = kk;
    a.k = o.k;
    a.P = P;
    a.width = T.width;
    a.box_of_leaf = T.box_of_leaf;
    a.level = T.level;
    a.uptr = T.lptr[VFMM_LIST_U];
    a.uidx = T.lidx[VFMM_LIST_U];
    a.wptr = T.lptr[VFMM_LIST_W];
    a.widx = T.lidx[VFMM_LIST_W];
    a.wcfg = T.lcfg[VFMM_LIST_W];
    a.xhat = o.xhat;
    a.slab = w.slab;
    a.far = w.far;
    a.Mexp = w.Mexp;
    a.u = u;
    a.ux = ux;
    a.uy = uy;
    if (mixed) {
        const int64_t nv = (int64_t)nleaf * R;
        int lw = 0;
        const double wm = 2.0 * std::frexp(T.width, &lw);  // width = wm 2^lw, wm in [1, 2)
        lw -= 1;
        if (side) VFMM_CUDA(cudaStreamWaitEvent(st, side->ev[2], 0));  // the near-field output
        LeafMixedArgs la;
        la.nleaf = nleaf;
        la.R = R;
        la.kk = kk;
        la.Rp = mo->Rp;
        la.P = P;
        la.lw = lw;
        la.wm = wm;
        la.width = T.width;
        la.box_of_leaf = T.box_of_leaf;
        la.level = T.level;
        la.uptr = T.lptr[VFMM_LIST_U];
        la.uidx = T.lidx[VFMM_LIST_U];
        la.wptr = T.lptr[VFMM_LIST_W];
        la.widx = T.lidx[VFMM_LIST_W];
        la.Mexp = w.Mexp;
        la.Lexp = w.Lexp;
        la.nearmix = w.mix.out;
        la.Er = mo->Er;
        la.Ef = w.mix.Ef;
        la.farmix = w.mix.far_out;
        la.farE = mo->far_E;
        la.Et = w.mix.Et;
        // an entry-major leaf far field leaves its per-leaf sums (a few entries per leaf) to this kernel;
        // the near field (about nine entries per leaf, on the side stream) keeps its segmented-sum kernel
        la.near_slab = nullptr;
        la.near_seg = nullptr;
        la.far_slab = PS.far.entry ? w.mix.part : nullptr;
        la.far_seg = PS.far.entry ? PS.far.seg : nullptr;
        la.u = u;
        la.ux = ux;
        la.uy = uy;
        leaf_mixed_kernel<<<(unsigned)nv, std::max(32, ((kk + 31) / 32) * 32), 0, st>>>(la);
        ++launches;
    } else {
        leaf_kernel<<<(unsigned)nleaf, ((kk + 31) / 32) * 32, 0, st>>>(a);
        ++launches;
    }
    mark(se, ST_LEAF, true, st);
    VFMM_CUDA(cudaGetLastError());
    if (se) se->launches += launches;
    return VFMM_OK;
}

}  // namespace vfmm

using namespace vfmm;

static int check_solve_args(const vfmm_tree* tree, const vfmm_ops* ops, int32_t nrhs) {
    if (!tree || !ops) return fail(VFMM_ERR_INVALID_ARG, "null tree or ops");
    if (tree->t.k != ops->k) return fail(VFMM_ERR_INVALID_ARG, "tree and ops differ in k");
    if (nrhs < 1) return fail(VFMM_ERR_INVALID_ARG, "nrhs must be >= 1");
    if (ops->p + 1 > 64) return fail(VFMM_ERR_INVALID_ARG, "p too large for the solve kernels");
    return VFMM_OK;
}

extern "C" int vfmm_workspace_size(const vfmm_tree* tree, const vfmm_ops* ops, int32_t nrhs, int32_t with_io,
                                   size_t* bytes) {
    VFMM_CHECK(check_solve_args(tree, ops, nrhs));
    if (!bytes) return fail(VFMM_ERR_INVALID_ARG, "null bytes");
    return layout(tree->t, *ops, nrhs, with_io != 0, nullptr, nullptr, bytes);
}

// All right-hand sides: one folded solve in the mixed form, one solve per right-hand side in FP64.
static int solve_all(const DeviceTree& T, const vfmm_ops& o, const double* f, int nrhs, double* u, double* ux,
                     double* uy, const Workspace& w, cudaStream_t st, StageEvents* se = nullptr) {
    if (o.precision == VFMM_MIXED) return solve_one(T, *w.ps, o, f, u, ux, uy, w, st, se);
    const size_t n = (size_t)T.n_leaves * o.k * o.k;
    for (int r = 0; r < nrhs; ++r) VFMM_CHECK(solve_one(T, T.plans, o, f + r * n, u + r * n, ux + r * n, uy + r * n, w, st, se));
    return VFMM_OK;
}

static int reset_status(const Workspace& w, cudaStream_t st) {
    if (w.mix.err) VFMM_CUDA(cudaMemsetAsync(w.mix.err, 0, sizeof(int), st));
    return VFMM_OK;
}

// What a non-zero status word means: where the first bounded device wait that ran out was.
static const char* status_site(int code) {
    switch (code) {
        case 1: return "a tensor-core producer waiting for a free stage";
        case 2: return "the tensor-core MMA issuer waiting for operands";
        case 3: return "a tensor-core epilogue waiting for its accumulators";
        case 4: return "the tensor-core MMA issuer waiting for drained accumulators";
        case 5: return "a translation-table copy into shared memory";
        case 6: return "a persistent tree pass waiting for an expansion another unit writes";
        case 7: return "the failure-path self-test's wait on an mbarrier nothing arrives on (expected)";
        default: return "an unknown site";
    }
}

// Reads the status word at `word` (device) after the solve that wrote it has finished.
int vfmm::read_status_word(const int* word) {
    if (!word) return VFMM_OK;
    int h = 0;
    VFMM_CUDA(cudaMemcpy(&h, word, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) return fail(VFMM_ERR_TIMEOUT, std::string("a bounded wait ran out: ") + status_site(h) +
                                             " (code " + std::to_string(h) + ")");
    return VFMM_OK;
}

// After a synchronised solve: a bounded device wait that expired shows up here.
static int read_status(const Workspace& w) { return read_status_word(w.mix.err); }

int vfmm::volume_potential(const vfmm_tree* tree, const vfmm_ops* ops, const double* f_dev, int32_t nrhs,
                           double* u_dev, double* ux_dev, double* uy_dev, void* workspace_dev, size_t workspace_bytes,
                           cudaStream_t st, bool fork, bool reset) {
    VFMM_CHECK(check_solve_args(tree, ops, nrhs));
    if (!f_dev || !u_dev || !ux_dev || !uy_dev || !workspace_dev) return fail(VFMM_ERR_INVALID_ARG, "null buffer");
    Workspace w;
    size_t need = 0;
    VFMM_CHECK(layout(tree->t, *ops, nrhs, false, &w, (char*)workspace_dev, &need));
    if (workspace_bytes < need) return fail(VFMM_ERR_WORKSPACE, "workspace too small");
    w.fork = fork;
    if (reset) VFMM_CHECK(reset_status(w, st));
    return solve_all(tree->t, *ops, f_dev, nrhs, u_dev, ux_dev, uy_dev, w, st);
}

int vfmm::solve_expansions(const vfmm_tree* tree, const vfmm_ops* ops, const void* workspace_dev,
                           size_t workspace_bytes, const double** Mexp, const double** Lexp, int* R) {
    Workspace w;
    size_t need = 0;
    VFMM_CHECK(layout(tree->t, *ops, 1, false, &w, (char*)const_cast<void*>(workspace_dev), &need));
    if (workspace_bytes < need) return fail(VFMM_ERR_WORKSPACE, "workspace smaller than a one-right-hand-side solve's");
    *Mexp = w.Mexp;
    *Lexp = w.Lexp;
    *R = 1;
    return VFMM_OK;
}

extern "C" int vfmm_workspace_status(const void* workspace_dev) {
    if (!workspace_dev) {
        // the allocation-free entry point's scratch on the current device
        const int* word = nullptr;
        VFMM_CHECK(noalloc_status_word(&word));
        return read_status_word(word);
    }
    return read_status_word(static_cast<const int*>(workspace_dev));
}

extern "C" int vfmm_volume_potential(const vfmm_tree* tree, const vfmm_ops* ops, const double* f_dev, int32_t nrhs,
                                     double* u_dev, double* ux_dev, double* uy_dev, void* workspace_dev,
                                     size_t workspace_bytes, void* stream) {
    return volume_potential(tree, ops, f_dev, nrhs, u_dev, ux_dev, uy_dev, workspace_dev, workspace_bytes,
                            (cudaStream_t)stream, true);
}

extern "C" int vfmm_volume_potential_host(const vfmm_tree* tree, const vfmm_ops* ops, const double* f_host,
                                          int32_t nrhs, double* u_host, double* ux_host, double* uy_host,
                                          void* workspace_dev, size_t workspace_bytes, void* stream) {
    VFMM_CHECK(check_solve_args(tree, ops, nrhs));
    if (!f_host || !u_host || !ux_host || !uy_host || !workspace_dev) return fail(VFMM_ERR_INVALID_ARG, "null buffer");
    Workspace w;
    size_t need = 0;
    VFMM_CHECK(layout(tree->t, *ops, nrhs, true, &w, (char*)workspace_dev, &need));
    if (workspace_bytes < need) return fail(VFMM_ERR_WORKSPACE, "workspace too small (with_io = 1 required)");
    w.fork = true;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = (size_t)tree->t.n_leaves * ops->k * ops->k * nrhs;
    double* f = w.io;
    double* u = w.io + n;
    double* ux = w.io + 2 * n;
    double* uy = w.io + 3 * n;
    VFMM_CHECK(reset_status(w, st));
    VFMM_CUDA(cudaMemcpyAsync(f, f_host, n * sizeof(double), cudaMemcpyHostToDevice, st));
    VFMM_CHECK(solve_all(tree->t, *ops, f, nrhs, u, ux, uy, w, st));
    VFMM_CUDA(cudaMemcpyAsync(u_host, u, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    VFMM_CUDA(cudaMemcpyAsync(ux_host, ux, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    VFMM_CUDA(cudaMemcpyAsync(uy_host, uy, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    VFMM_CUDA(cudaStreamSynchronize(st));
    return read_status(w);
}

extern "C" int vfmm_volume_potential_profiled(const vfmm_tree* tree, const vfmm_ops* ops, const double* f_dev,
                                              int32_t nrhs, double* u_dev, double* ux_dev, double* uy_dev,
                                              void* workspace_dev, size_t workspace_bytes, void* stream,
                                              float* stage_ms, int32_t* launches) {
    VFMM_CHECK(check_solve_args(tree, ops, nrhs));
    if (!f_dev || !u_dev || !ux_dev || !uy_dev || !workspace_dev || !stage_ms || !launches)
        return fail(VFMM_ERR_INVALID_ARG, "null buffer");
    Workspace w;
    size_t need = 0;
    VFMM_CHECK(layout(tree->t, *ops, nrhs, false, &w, (char*)workspace_dev, &need));
    if (workspace_bytes < need) return fail(VFMM_ERR_WORKSPACE, "workspace too small");
    cudaStream_t st = (cudaStream_t)stream;
    VFMM_CHECK(reset_status(w, st));
    StageEvents se;
    for (int i = 0; i < 2 * VFMM_N_STAGES; ++i) VFMM_CUDA(cudaEventCreate(&se.ev[i]));
    for (int i = 0; i < VFMM_N_STAGES; ++i) stage_ms[i] = 0.0f;
    if (ops->precision == VFMM_MIXED) {
        // contraction timers: recorded once here so that a contraction the tree lacks reads 0
        w.mix.cev = se.ev + 2 * ST_CONTRACTIONS;
        for (int i = 2 * ST_CONTRACTIONS; i < 2 * VFMM_N_STAGES; ++i) VFMM_CUDA(cudaEventRecord(se.ev[i], st));
    }
    const size_t n = (size_t)tree->t.n_leaves * ops->k * ops->k;
    const bool folded = ops->precision == VFMM_MIXED;
    int rc = VFMM_OK;
    for (int r = 0; r < (folded ? 1 : nrhs) && rc == VFMM_OK; ++r) {
        rc = folded ? solve_one(tree->t, *w.ps, *ops, f_dev, u_dev, ux_dev, uy_dev, w, st, &se)
                    : solve_one(tree->t, tree->t.plans, *ops, f_dev + r * n, u_dev + r * n, ux_dev + r * n,
                                uy_dev + r * n, w, st, &se);
        if (rc != VFMM_OK) break;
        cudaError_t e = cudaEventSynchronize(se.ev[2 * ST_LEAF + 1]);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "cudaEventSynchronize");
            break;
        }
        const int n_timed = ops->precision == VFMM_MIXED ? VFMM_N_STAGES : ST_CONTRACTIONS;
        for (int i = 0; i < n_timed; ++i) {
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, se.ev[2 * i], se.ev[2 * i + 1]);
            stage_ms[i] += ms;
        }
    }
    for (int i = 0; i < 2 * VFMM_N_STAGES; ++i) cudaEventDestroy(se.ev[i]);
    *launches = se.launches;
    if (rc == VFMM_OK) rc = read_status(w);
    return rc;
}

extern "C" int vfmm_graph_create(const vfmm_tree* tree, const vfmm_ops* ops, const double* f_dev, int32_t nrhs,
                                 double* u_dev, double* ux_dev, double* uy_dev, void* workspace_dev,
                                 size_t workspace_bytes, void* stream, vfmm_graph** out) {
    if (!out) return fail(VFMM_ERR_INVALID_ARG, "null out");
    *out = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    if (st == nullptr) return fail(VFMM_ERR_INVALID_ARG, "graph capture needs a non-default stream");
    VFMM_CHECK(vfmm_volume_potential(tree, ops, f_dev, nrhs, u_dev, ux_dev, uy_dev, workspace_dev, workspace_bytes,
                                     stream));
    VFMM_CUDA(cudaStreamSynchronize(st));
    vfmm_graph* g = new vfmm_graph();
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        delete g;
        return cuda_fail(e, "cudaStreamBeginCapture");
    }
    int rc = vfmm_volume_potential(tree, ops, f_dev, nrhs, u_dev, ux_dev, uy_dev, workspace_dev, workspace_bytes,
                                   stream);
    e = cudaStreamEndCapture(st, &g->graph);
    if (rc != VFMM_OK || e != cudaSuccess) {
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        return rc != VFMM_OK ? rc : cuda_fail(e, "cudaStreamEndCapture");
    }
    // kernels keep the priority of the stream they were captured on
    e = cudaGraphInstantiate(&g->exec, g->graph, cudaGraphInstantiateFlagUseNodePriority);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g->graph);
        delete g;
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    *out = g;
    return VFMM_OK;
}

extern "C" int vfmm_graph_launch(const vfmm_graph* g, void* stream) {
    if (!g) return fail(VFMM_ERR_INVALID_ARG, "null graph");
    VFMM_CUDA(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
    return VFMM_OK;
}

extern "C" int vfmm_graph_destroy(vfmm_graph* g) {
    if (!g) return VFMM_OK;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return VFMM_OK;
}

// ---------------------------------------------------------------- schedule autotuner
extern "C" int vfmm_tune(const vfmm_tree* tree, const vfmm_ops* ops, const double* f_dev, int32_t nrhs, double* u_dev,
                         double* ux_dev, double* uy_dev, void* workspace_dev, size_t workspace_bytes, void* stream,
                         int32_t* splits) {
    VFMM_CHECK(check_solve_args(tree, ops, nrhs));
    if (!f_dev || !u_dev || !ux_dev || !uy_dev || !workspace_dev) return fail(VFMM_ERR_INVALID_ARG, "null buffer");
    cudaStream_t st = (cudaStream_t)stream;
    Workspace w;
    size_t need = 0;
    VFMM_CHECK(layout(tree->t, *ops, nrhs, false, &w, (char*)workspace_dev, &need));
    if (workspace_bytes < need) return fail(VFMM_ERR_WORKSPACE, "workspace too small");
    if (splits)
        for (int i = 0; i < 4; ++i) splits[i] = 1;
    if (ops->precision != VFMM_MIXED) return VFMM_OK;
    const DeviceTree& T = tree->t;
    const MixedOps* mo = (const MixedOps*)ops->mixed;
    // one solve leaves every contraction's operands in the workspace
    VFMM_CHECK(reset_status(w, st));
    VFMM_CHECK(solve_all(T, *ops, f_dev, nrhs, u_dev, ux_dev, uy_dev, w, st));
    VFMM_CUDA(cudaStreamSynchronize(st));
    PlanSet* PS = const_cast<PlanSet*>(w.ps);
    const size_t R = (size_t)PS->R;
    struct Job {
        SplitPlan* P;
        const void* a;
        const CUtensorMap* map;
        int Kp, Rp;
        float2* out;
        size_t rows;
        int slices;
    } jobs[4] = {{&PS->near, w.mix.fsl, &mo->tm_near, mo->Kp, mo->Rp, w.mix.out, T.n_leaves * R, mo->slices[kCtrNear]},
                 {&PS->m2l, w.mix.msl, &mo->tm_m2l, mo->Kx, mo->Rx, w.mix.m2l_out, T.n_boxes * R, mo->slices[kCtrM2L]},
                 {&PS->s2l, w.mix.fsl, &mo->tm_s2l, mo->Kp, mo->Rx, w.mix.s2l_out, T.n_boxes * R, mo->slices[kCtrS2L]},
                 {&PS->far, w.mix.aprep, &mo->tm_far, mo->Kx, mo->Rp, w.mix.far_out, T.n_leaves * R,
                  mo->slices[kCtrFar]}};
    cudaEvent_t e0, e1;
    VFMM_CUDA(cudaEventCreate(&e0));
    VFMM_CUDA(cudaEventCreate(&e1));
    int rc = VFMM_OK;
    // fastest split-K factor of one form of a contraction (its current factor when it cannot split)
    auto time_form = [&](const Job& jb, SplitPlan* P, float2* part, int* best_sp, float* best_ms) {
        const double avg_units = (double)P->entries * (jb.Kp / kKBlock) / std::max(1, P->n_groups);
        const int max_sp = P->may_split ? kMaxSplit : 1;
        const int keep = P->split;
        *best_sp = keep;
        *best_ms = -1.0f;
        for (int sp = P->may_split ? 1 : keep; sp <= std::max(max_sp, keep) && rc == VFMM_OK; sp *= 2) {
            if (P->may_split && sp > std::max(1.0, avg_units)) break;
            P->split = sp;
            float total = 0.0f;
            for (int rep = 0; rep < 4 && rc == VFMM_OK; ++rep) {
                cudaEventRecord(e0, st);
                rc = split_gemm(*P, jb.a, *jb.map, jb.Kp, jb.Rp, jb.out, w.mix.err, part, jb.rows, jb.slices, st);
                cudaEventRecord(e1, st);
                if (rc != VFMM_OK) break;
                cudaError_t e = cudaEventSynchronize(e1);
                float ms = 0.0f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) rc = cuda_fail(e, "timing a split contraction");
                if (rep > 0) total += ms;  // the first run warms up
            }
            if (rc == VFMM_OK && (*best_ms < 0.0f || total < *best_ms)) {
                *best_ms = total;
                *best_sp = sp;
            }
            if (!P->may_split) break;
        }
        P->split = *best_sp;
    };
    // persistent CTAs (one per SM, each walking several work items) against one CTA per item, for a
    // contraction with more items than SMs; the faster is kept
    auto time_ctas = [&](const Job& jb, SplitPlan* P, float2* part) {
        const int nchunks = jb.Rp / table_rows_per_tile(P->transposed, jb.Rp);
        const long long items = (long long)P->n_groups * (P->entry ? 1 : P->split) * nchunks;
        const int sms = sm_count();
        if (items <= sms) return;
        float best = -1.0f;
        int best_c = P->ctas;
        for (int c : {0, sms}) {
            P->ctas = c;
            float total = 0.0f;
            for (int rep = 0; rep < 4 && rc == VFMM_OK; ++rep) {
                cudaEventRecord(e0, st);
                rc = split_gemm(*P, jb.a, *jb.map, jb.Kp, jb.Rp, jb.out, w.mix.err, part, jb.rows, jb.slices, st);
                cudaEventRecord(e1, st);
                if (rc != VFMM_OK) break;
                cudaError_t e = cudaEventSynchronize(e1);
                float ms = 0.0f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) rc = cuda_fail(e, "timing a split contraction");
                if (rep > 0) total += ms;
            }
            if (rc == VFMM_OK && (best < 0.0f || total < best)) {
                best = total;
                best_c = c;
            }
        }
        P->ctas = best_c;
    };
    for (int j = 0; j < 4 && rc == VFMM_OK; ++j) {
        Job& jb = jobs[j];
        if (jb.P->n_groups == 0 || (!jb.P->may_split && !jb.P->alt)) continue;
        float2* part = j == 0 ? w.mix.part_side : j == 2 ? w.mix.part_s2l : w.mix.part;
        int sp = 1;
        float ms = -1.0f;
        time_form(jb, jb.P, part, &sp, &ms);
        if (rc == VFMM_OK && jb.P->alt && jb.P->alt->n_groups > 0) {
            // the other form (grouped or entry-major): kept if faster
            int sp_alt = 1;
            float ms_alt = -1.0f;
            time_form(jb, jb.P->alt, part, &sp_alt, &ms_alt);
            if (rc == VFMM_OK && ms_alt >= 0.0f && ms_alt < ms) {
                SplitPlan* alt = jb.P->alt;
                jb.P->alt = nullptr;
                std::swap(*jb.P, *alt);
                jb.P->alt = alt;
            }
        }
        if (rc == VFMM_OK) time_ctas(jb, jb.P, part);
        if (splits) splits[j] = jb.P->split;
    }
    // Co-scheduling of the whole step: in a forked solve the near field (low-priority stream) and the
    // main chain share the SMs, and a near-field CTA leaves no registers for anything else on its SM.
    // Timed on the forked solve itself: the near field on every SM, or capped at 7/8 ... 4/8 of them,
    // the cooperative tree passes capped to the SMs it leaves free (they can start only when their
    // whole grid fits); the fastest is kept (the uncapped schedule unless a cap is faster).
    if (rc == VFMM_OK && PS->near.n_groups > 0 && PS->near.ctas > 0 && use_passes(T, PS->R, ops->p + 1)) {
        const int sms = sm_count();
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, upward_pass_kernel, kPassThreads, pass_smem_bytes(ops->p + 1));
        Workspace wf = w;
        wf.fork = true;
        const int near0 = PS->near.ctas, pass0 = PS->pass_ctas;
        float best = -1.0f;
        int best_near = near0, best_pass = pass0;
        const int fracs[5] = {8, 7, 6, 5, 4};  // eighths of the SMs
        for (int c = 0; c < 5 && rc == VFMM_OK; ++c) {
            const int ncta = fracs[c] == 8 ? near0 : std::max(1, sms * fracs[c] / 8);
            PS->near.ctas = ncta;
            PS->pass_ctas = fracs[c] == 8 ? pass0 : std::max(1, per_sm * (sms - ncta));
            float total = 0.0f;
            for (int rep = 0; rep < 6 && rc == VFMM_OK; ++rep) {
                cudaEventRecord(e0, st);
                rc = solve_all(T, *ops, f_dev, nrhs, u_dev, ux_dev, uy_dev, wf, st);
                cudaEventRecord(e1, st);
                if (rc != VFMM_OK) break;
                cudaError_t e = cudaEventSynchronize(e1);
                float ms = 0.0f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) rc = cuda_fail(e, "timing a forked solve");
                if (rep > 0) total += ms;  // the first run warms up
            }
            if (rc == VFMM_OK && (best < 0.0f || total < best)) {
                best = total;
                best_near = PS->near.ctas;
                best_pass = PS->pass_ctas;
            }
        }
        PS->near.ctas = best_near;
        PS->pass_ctas = best_pass;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    VFMM_CHECK(rc);
    // leave the outputs of an ordinary solve with the chosen schedule
    VFMM_CHECK(solve_all(T, *ops, f_dev, nrhs, u_dev, ux_dev, uy_dev, w, st));
    VFMM_CUDA(cudaStreamSynchronize(st));
    return read_status(w);
}

extern "C" int vfmm_schedule_get(const vfmm_tree* tree, int32_t nrhs, int32_t* near_ctas, int32_t* pass_ctas) {
    if (!tree || !near_ctas || !pass_ctas || nrhs < 1) return fail(VFMM_ERR_INVALID_ARG, "bad schedule query");
    const PlanSet* PS = nullptr;
    VFMM_CHECK(plans_for(tree->t, nrhs, &PS));
    *near_ctas = PS->near.ctas;
    *pass_ctas = PS->pass_ctas;
    return VFMM_OK;
}

extern "C" int vfmm_schedule_set(vfmm_tree* tree, int32_t nrhs, int32_t near_ctas, int32_t pass_ctas) {
    if (!tree || nrhs < 1 || near_ctas < 0 || pass_ctas < 0) return fail(VFMM_ERR_INVALID_ARG, "bad schedule");
    const PlanSet* PS = nullptr;
    VFMM_CHECK(plans_for(tree->t, nrhs, &PS));
    PlanSet* ps = const_cast<PlanSet*>(PS);
    ps->near.ctas = near_ctas;
    ps->pass_ctas = pass_ctas;
    return VFMM_OK;
}
