// The leaf interpolant v~ at arbitrary points (Section 3.1: values away from the collocation
// nodes come from the polynomial that interpolates the computed values on the leaf holding the
// point; Section 3.3 on their error).
//
// One thread per point: the leaf is found by descending from the root with the point's integer
// coordinates at the finest level, floor(2^D (x - lo) / W) clamped to 2^D - 1 (a point on an edge
// shared by two leaves belongs to the one above or to the right), then every field is evaluated
// by the tensor Lagrange interpolant on the leaf's first-kind Chebyshev nodes:
// r_j = sum_i l_i(x^) V[j][i], value = sum_j l_j(y^) r_j, with the product form
// l_i(t) = prod_{m<i} (t - t_m) prod_{m>i} (t - t_m) w_i, w_i = 1 / prod_{m != i} (t_i - t_m),
// from prefix and suffix products (no division; exact 0 and 1 at the nodes).
#include <cmath>

#include "vfmm_internal.cuh"

namespace vfmm {

constexpr int kMaxFields = 8;

struct InterpArgs {
    const double* f[kMaxFields];  // [n_leaves][k*k] each
    double* o[kMaxFields];        // [n] each
    int nf, k, depth;
    double lox, loy, width;
    double t[16];  // nodes on [-1, 1], ascending
    double w[16];  // 1 / prod_{m != i} (t_i - t_m)
};

// Lagrange basis at t (k <= 16), product form: l[i] = (prefix product before i) (suffix product
// after i) w_i. K > 0: k = K, unrolled.
template <int K>
__device__ inline void lagrange_basis(const InterpArgs& a, double t, double* l) {
    const int k = K > 0 ? K : a.k;
    double pre = 1.0;
#pragma unroll
    for (int i = 0; i < k; ++i) {
        l[i] = pre;
        pre *= t - a.t[i];
    }
    double suf = 1.0;
#pragma unroll
    for (int i = k - 1; i >= 0; --i) {
        l[i] *= suf * a.w[i];
        suf *= t - a.t[i];
    }
}

template <int K>
__global__ void __launch_bounds__(128) leaf_interp_kernel(InterpArgs a, const int32_t* __restrict__ child0,
                                                          const int32_t* __restrict__ level,
                                                          const int32_t* __restrict__ ix,
                                                          const int32_t* __restrict__ iy,
                                                          const int32_t* __restrict__ leaf_of_box, int64_t n,
                                                          const double* __restrict__ x,
                                                          const double* __restrict__ y, int32_t* __restrict__ leaf_out) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double px = x[p], py = y[p];
    const double X = (px - a.lox) / a.width, Y = (py - a.loy) / a.width;
    if (!(X >= 0.0 && X <= 1.0 && Y >= 0.0 && Y <= 1.0)) {
        for (int q = 0; q < a.nf; ++q) a.o[q][p] = __longlong_as_double(0x7ff8000000000000ll);  // NaN
        if (leaf_out) leaf_out[p] = -1;
        return;
    }
    const int D = a.depth;
    const double side = ldexp(1.0, D);
    const int ixd = (int)fmin(floor(X * side), side - 1.0), iyd = (int)fmin(floor(Y * side), side - 1.0);
    int b = 0, l = 0;
    while (child0[b] >= 0) {
        ++l;
        const int cx = (ixd >> (D - l)) & 1, cy = (iyd >> (D - l)) & 1;
        b = child0[b] + ((cy << 1) | cx);
    }
    const int leaf = leaf_of_box[b];
    if (leaf_out) leaf_out[p] = leaf;
    const double h = ldexp(a.width, -level[b]);
    const double cxb = a.lox + ((double)ix[b] + 0.5) * h, cyb = a.loy + ((double)iy[b] + 0.5) * h;
    double lx[16], ly[16];
    lagrange_basis<K>(a, (px - cxb) * (2.0 / h), lx);
    lagrange_basis<K>(a, (py - cyb) * (2.0 / h), ly);
    const int k = K > 0 ? K : a.k, kk = k * k;
    for (int q = 0; q < a.nf; ++q) {
        const double* V = a.f[q] + (size_t)leaf * kk;
        double acc = 0.0;
        if (K > 0) {
            // even k: rows of 16-byte pairs (a leaf's k*k doubles start on a 16-byte boundary)
            const double2* V2 = reinterpret_cast<const double2*>(V);
#pragma unroll
            for (int j = 0; j < k; ++j) {
                double r = 0.0;
#pragma unroll
                for (int i = 0; i < k; i += 2) {
                    const double2 v = __ldg(V2 + (j * k + i) / 2);
                    r = fma(lx[i], v.x, r);
                    r = fma(lx[i + 1], v.y, r);
                }
                acc = fma(ly[j], r, acc);
            }
        } else {
            for (int j = 0; j < k; ++j) {
                double r = 0.0;
                for (int i = 0; i < k; ++i) r = fma(lx[i], __ldg(V + j * k + i), r);
                acc = fma(ly[j], r, acc);
            }
        }
        a.o[q][p] = acc;
    }
}

}  // namespace vfmm

using namespace vfmm;

extern "C" int vfmm_leaf_interpolate(const vfmm_tree* tree, int32_t n_fields, const double* const* fields_dev,
                                     int64_t n_points, const double* x_dev, const double* y_dev,
                                     double* const* out_dev, int32_t* leaf_dev, void* stream) {
    if (!tree || !fields_dev || !out_dev) return fail(VFMM_ERR_INVALID_ARG, "null argument");
    if (n_fields < 1 || n_fields > kMaxFields) return fail(VFMM_ERR_INVALID_ARG, "n_fields must be in [1, 8]");
    if (n_points < 0) return fail(VFMM_ERR_INVALID_ARG, "n_points must be >= 0");
    if (n_points == 0) return VFMM_OK;
    if (!x_dev || !y_dev) return fail(VFMM_ERR_INVALID_ARG, "null point coordinates");
    const DeviceTree& T = tree->t;
    InterpArgs a = {};
    for (int q = 0; q < n_fields; ++q) {
        if (!fields_dev[q] || !out_dev[q]) return fail(VFMM_ERR_INVALID_ARG, "null field or output");
        a.f[q] = fields_dev[q];
        a.o[q] = out_dev[q];
    }
    a.nf = n_fields;
    a.k = T.k;
    a.depth = T.depth;
    a.lox = T.cx - T.width / 2.0;
    a.loy = T.cy - T.width / 2.0;
    a.width = T.width;
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < T.k; ++i) a.t[i] = -std::cos(pi * (2.0 * i + 1.0) / (2.0 * T.k));
    for (int i = 0; i < T.k; ++i) {
        double prod = 1.0;
        for (int m = 0; m < T.k; ++m)
            if (m != i) prod *= a.t[i] - a.t[m];
        a.w[i] = 1.0 / prod;
    }
    const unsigned grid = (unsigned)((n_points + 127) / 128);
    cudaStream_t st = (cudaStream_t)stream;
    if (T.k == 16)
        leaf_interp_kernel<16><<<grid, 128, 0, st>>>(a, T.child0, T.level, T.ix, T.iy, T.leaf_of_box, n_points, x_dev,
                                                     y_dev, leaf_dev);
    else if (T.k == 8)
        leaf_interp_kernel<8><<<grid, 128, 0, st>>>(a, T.child0, T.level, T.ix, T.iy, T.leaf_of_box, n_points, x_dev,
                                                    y_dev, leaf_dev);
    else
        leaf_interp_kernel<0><<<grid, 128, 0, st>>>(a, T.child0, T.level, T.ix, T.iy, T.leaf_of_box, n_points, x_dev,
                                                    y_dev, leaf_dev);
    VFMM_CUDA(cudaGetLastError());
    return VFMM_OK;
}
