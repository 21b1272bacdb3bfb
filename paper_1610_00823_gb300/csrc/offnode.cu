// The computed potential at arbitrary points from the stored expansions (Section 5.3: the FMM's
// multipole and local expansions are kept so that a new target costs O(p) for its far field
// instead of a new FMM; Section 3.1 for the split into near and far field).
//
// For a point t of leaf b (located as the leaf interpolant locates it):
//   V f~(t) = -(1/2 pi) Re [ sum_l b~_l ((t - z_b)/h)^l + sum over W(b) of the multipole at t ]
//           + sum over U(b) of -(1/2 pi) int_{B_s} log|t - y| f~_s(y) dy,
// with the gradient from the differentiated expansions and kernels (Section 3.2). The far part
// reads the expansions a solve left in its workspace; the near part is an on-the-fly quadrature
// per (point, neighbour leaf): the source box is cut into triangles with apex at its point nearest
// to t (near_quad.cuh, the construction of the near-field tables) and integrated with tanh-sinh
// rules in both directions, f~_s evaluated from its Chebyshev coefficients at every node.
//
// One CTA per point: warp 0 sums the far part, then all threads share the quadrature nodes of each
// neighbour leaf in turn (fixed order, so results are deterministic).
#include <cmath>

#include "near_quad.cuh"
#include "ops.cuh"
#include "vfmm_internal.cuh"

namespace vfmm {

constexpr int kOffThreads = 256;
// tanh-sinh rules of the on-the-fly near-field quadrature, by the distance d from the point to the
// boundary of the source leaf (width hs): step 0.1 (65 nodes per direction) when the point lies on
// that boundary or d >= hs / 4; 0.05 (141 nodes, the near-field tables' rule) for hs / 1000 <= d <
// hs / 4; 0.035 (201 nodes) closer. Measured on the unit box against a step of 0.015: the gradient
// of a point 1e-4 inside an edge is off by 1e-8 with step 0.1, 6e-13 with 0.05; 1e-6 inside, 4e-12
// with 0.05 and 2e-13 with 0.035.
constexpr int kOffRules = 3;
__host__ __device__ constexpr double off_step(int r) { return r == 0 ? 0.1 : (r == 1 ? 0.05 : 0.035); }
// nodes j in [-half, half]: |u| <= 3.2, 3.5, 3.5
__host__ __device__ constexpr int off_half(int r) { return r == 0 ? 32 : (r == 1 ? 70 : 100); }
// first node of rule r in the shared node table
__host__ __device__ constexpr int off_first(int r) { return r == 0 ? 0 : (r == 1 ? 65 : 65 + 141); }
constexpr int kOffDENodes = 65 + 141 + 201;

struct OffArgs {
    int k, P, depth, R;
    int64_t n;
    double lox, loy, width;
    const int32_t *child0, *level, *ix, *iy, *leaf_of_box;
    const int32_t *uptr, *uidx, *wptr, *widx, *wcfg;
    const double* f;     // [n_leaves][k*k] leaf values of right-hand side 0
    const double* Mexp;  // [n_boxes][R][2P] scaled multipoles of the solve
    const double* Lexp;  // [n_boxes][R][2P] scaled locals of the solve
    const double *x, *y;
    double *u, *ux, *uy;
    double A[16 * 16];   // values -> Chebyshev coefficients, A[m][i] = (2 - d_m0)/k T_m(x_i)
};

__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < kOffThreads / 32; ++w) s += red[w];  // every thread, same order
    return s;
}

__global__ void __launch_bounds__(kOffThreads) offnode_kernel(OffArgs a) {
    __shared__ double sDE[3][kOffDENodes];  // the three rules' nodes one after another
    __shared__ double sC[16 * 16];    // Chebyshev coefficients of the current source leaf, [n][m]
    __shared__ double sTmp[16 * 16];
    __shared__ QuadPiece pcs[8];
    __shared__ int s_npc;
    __shared__ double red[kOffThreads / 32];
    __shared__ double s_far[3];
    __shared__ int s_b;
    const int tid = threadIdx.x, k = a.k, kk = k * k;
    const int64_t p = blockIdx.x;
    const double px = a.x[p], py = a.y[p];
    for (int r = 0; r < kOffRules; ++r)
        for (int j = tid; j < 2 * off_half(r) + 1; j += blockDim.x) {
            const DENode d = de_node(j - off_half(r), off_step(r));
            sDE[0][off_first(r) + j] = d.x;
            sDE[1][off_first(r) + j] = d.xc;
            sDE[2][off_first(r) + j] = d.w;
        }
    if (tid == 0) {
        // the leaf holding the point: integer coordinates at the finest level, a descent from the root
        const double X = (px - a.lox) / a.width, Y = (py - a.loy) / a.width;
        int b = -1;
        if (X >= 0.0 && X <= 1.0 && Y >= 0.0 && Y <= 1.0) {
            const int D = a.depth;
            const double side = ldexp(1.0, D);
            const int ixd = (int)fmin(floor(X * side), side - 1.0), iyd = (int)fmin(floor(Y * side), side - 1.0);
            b = 0;
            int l = 0;
            while (a.child0[b] >= 0) {
                ++l;
                const int cx = (ixd >> (D - l)) & 1, cy = (iyd >> (D - l)) & 1;
                b = a.child0[b] + ((cy << 1) | cx);
            }
        }
        s_b = b;
    }
    __syncthreads();
    const int b = s_b;
    if (b < 0) {  // outside the closed root box, or a NaN coordinate
        if (tid == 0) a.u[p] = a.ux[p] = a.uy[p] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    const double h = ldexp(a.width, -a.level[b]);
    const double cxb = a.lox + ((double)a.ix[b] + 0.5) * h, cyb = a.loy + ((double)a.iy[b] + 0.5) * h;
    const double inv2pi = 0.15915494309189533577;
    const int P = a.P;
    if (tid < 32) {
        // far part: b's local expansion at zeta = (t - z_b)/h (lanes split the coefficients), then the
        // W multipoles (lanes split the boxes); fixed-order shuffle sums
        const double zr = (px - cxb) / h, zi = (py - cyb) / h;
        double phr = 0.0, dr = 0.0, di = 0.0;
        const double* L = a.Lexp + (size_t)b * a.R * 2 * P;
        for (int l = tid; l < P; l += 32) {
            // zeta^l and l zeta^(l-1) by repeated multiplication (l <= 63)
            double pr = 1.0, pi = 0.0, qr = 0.0, qi = 0.0;  // zeta^l, zeta^(l-1)
            for (int e = 0; e < l; ++e) {
                qr = pr;
                qi = pi;
                const double t = pr * zr - pi * zi;
                pi = pr * zi + pi * zr;
                pr = t;
            }
            const double br = L[2 * l], bi = L[2 * l + 1];
            phr += br * pr - bi * pi;
            dr += l * (br * qr - bi * qi) / h;  // Phi' = (1/h) sum_l l b~_l zeta^(l-1)
            di += l * (br * qi + bi * qr) / h;
        }
        // W list: box c of width h/2 at offset (dx, dy) (units of h/4 in the pattern): zeta_w = 2 (zeta - D)
        for (int e = a.wptr[b] + tid; e < a.wptr[b + 1]; e += 32) {
            const int c = a.widx[e];
            const int cfg = a.wcfg[e];
            int qx, qy;
            far_pattern(cfg, &qx, &qy);
            const double wr = 2.0 * (zr - qx / 4.0), wi = 2.0 * (zi - qy / 4.0);
            const double hw = 0.5 * h;
            const double* M = a.Mexp + (size_t)c * a.R * 2 * P;
            const double a0 = M[0];
            // a_0 (log h_w + log zeta_w) + sum_n a_n zeta_w^-n, derivative a_0/zeta_w - sum n a_n zeta_w^(-n-1)
            const double m2 = wr * wr + wi * wi;
            const double ir = wr / m2, ii = -wi / m2;  // 1/zeta_w
            double sr = a0 * (log(hw) + 0.5 * log(m2));  // Re of a_0 (log h_w + log zeta_w)
            double gr = a0 * ir, gi = a0 * ii;
            double zr_n = 1.0, zi_n = 0.0;  // zeta_w^-n
            for (int n = 1; n < P; ++n) {
                // derivative term -n a_n zeta^(-n-1) = -n a_n zeta^-n / zeta
                const double ar = M[2 * n], ai = M[2 * n + 1];
                const double t1 = zr_n * ir - zi_n * ii, t2 = zr_n * ii + zi_n * ir;  // zeta^-(n) * 1/zeta
                zr_n = t1;
                zi_n = t2;  // now zeta^-n
                sr += ar * zr_n - ai * zi_n;
                const double u1 = zr_n * ir - zi_n * ii, u2 = zr_n * ii + zi_n * ir;  // zeta^-(n+1)
                gr -= n * (ar * u1 - ai * u2);
                gi -= n * (ar * u2 + ai * u1);
            }
            phr += sr;
            dr += gr / hw;  // d zeta_w / dz = 1 / h_w
            di += gi / hw;
        }
        for (int o = 16; o > 0; o >>= 1) {
            phr += __shfl_xor_sync(0xffffffffu, phr, o);
            dr += __shfl_xor_sync(0xffffffffu, dr, o);
            di += __shfl_xor_sync(0xffffffffu, di, o);
        }
        if (tid == 0) {
            s_far[0] = -inv2pi * phr;
            s_far[1] = -inv2pi * dr;
            s_far[2] = inv2pi * di;
        }
    }
    // near part, one neighbour leaf after another
    double n0 = 0.0, n1 = 0.0, n2 = 0.0;
    for (int e = a.uptr[b]; e < a.uptr[b + 1]; ++e) {
        const int s = a.uidx[e];
        const int ls = a.leaf_of_box[s];
        const double hs = ldexp(a.width, -a.level[s]);
        const double cxs = a.lox + ((double)a.ix[s] + 0.5) * hs, cys = a.loy + ((double)a.iy[s] + 0.5) * hs;
        __syncthreads();  // sC, pcs free
        // Chebyshev coefficients of f~_s: tmp[j][m] = sum_i A[m][i] V[j][i], C[n][m] = sum_j A[n][j] tmp[j][m]
        const double* V = a.f + (size_t)ls * kk;
        for (int q = tid; q < kk; q += blockDim.x) {
            const int j = q / k, m = q - j * k;
            double acc = 0.0;
            for (int i = 0; i < k; ++i) acc += a.A[m * 16 + i] * V[j * k + i];
            sTmp[q] = acc;
        }
        if (tid == 0) s_npc = make_pieces(px, py, cxs, cys, hs, pcs);
        __syncthreads();
        for (int q = tid; q < kk; q += blockDim.x) {
            const int nn = q / k, m = q - nn * k;
            double acc = 0.0;
            for (int j = 0; j < k; ++j) acc += a.A[nn * 16 + j] * sTmp[j * k + m];
            sC[q] = acc;
        }
        __syncthreads();
        const int npc = s_npc;
        // the rule: distance from the point to the boundary of the closed source box
        const double lox = cxs - hs / 2, hix = cxs + hs / 2, loy = cys - hs / 2, hiy = cys + hs / 2;
        const double ox = fmax(fmax(lox - px, px - hix), 0.0), oy = fmax(fmax(loy - py, py - hiy), 0.0);
        const double din = fmin(fmin(px - lox, hix - px), fmin(py - loy, hiy - py));
        const double d = (ox > 0.0 || oy > 0.0) ? sqrt(ox * ox + oy * oy) : din;  // 0 on the boundary
        const int rule = (d <= 0.0 || d >= 0.25 * hs) ? 0 : (d >= 1e-3 * hs ? 1 : 2);
        const int N = 2 * off_half(rule) + 1;
        const int o0 = off_first(rule);
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        const int total = npc * N * N;
        for (int g = tid; g < total; g += blockDim.x) {
            const int ip = g / (N * N), rem = g - ip * N * N;
            const int js = o0 + rem / N, jt = o0 + rem % N;
            const DENode ds{sDE[0][js], sDE[1][js], sDE[2][js]};
            const DENode dt{sDE[0][jt], sDE[1][jt], sDE[2][jt]};
            double w3[3], yx, yy;
            node_weights(pcs[ip], px, py, ds, dt, w3, &yx, &yy);
            // f~_s at y: sum_n T_n(y^) sum_m C[n][m] T_m(x^), x^, y^ in [-1, 1]
            const double xh = 2.0 * (yx - cxs) / hs, yh = 2.0 * (yy - cys) / hs;
            double tx[16];
            tx[0] = 1.0;
            if (k > 1) tx[1] = xh;
            for (int m = 2; m < k; ++m) tx[m] = 2.0 * xh * tx[m - 1] - tx[m - 2];
            double fv = 0.0, tm2 = 0.0, tm1 = 0.0;
            for (int nn = 0; nn < k; ++nn) {
                const double tn = nn == 0 ? 1.0 : (nn == 1 ? yh : 2.0 * yh * tm1 - tm2);
                tm2 = tm1;
                tm1 = tn;
                double row = 0.0;
                for (int m = 0; m < k; ++m) row += sC[nn * k + m] * tx[m];
                fv += tn * row;
            }
            a0 += w3[0] * fv;
            a1 += w3[1] * fv;
            a2 += w3[2] * fv;
        }
        n0 += block_sum(a0, red);
        n1 += block_sum(a1, red);
        n2 += block_sum(a2, red);
    }
    __syncthreads();
    if (tid == 0) {
        a.u[p] = s_far[0] + n0;
        a.ux[p] = s_far[1] + n1;
        a.uy[p] = s_far[2] + n2;
    }
}

}  // namespace vfmm

using namespace vfmm;

extern "C" int vfmm_evaluate_points(const vfmm_tree* tree, const vfmm_ops* ops, const double* f_dev,
                                    const void* workspace_dev, size_t workspace_bytes, int64_t n_points,
                                    const double* x_dev, const double* y_dev, double* u_dev, double* ux_dev,
                                    double* uy_dev, void* stream) {
    if (!tree || !ops) return fail(VFMM_ERR_INVALID_ARG, "null tree or ops");
    if (tree->t.k != ops->k) return fail(VFMM_ERR_INVALID_ARG, "tree and ops differ in k");
    if (n_points < 0) return fail(VFMM_ERR_INVALID_ARG, "n_points < 0");
    if (n_points == 0) return VFMM_OK;
    if (!f_dev || !workspace_dev || !x_dev || !y_dev || !u_dev || !ux_dev || !uy_dev)
        return fail(VFMM_ERR_INVALID_ARG, "null buffer");
    if (n_points > (int64_t)INT32_MAX) return fail(VFMM_ERR_INVALID_ARG, "too many points for one call");
    const DeviceTree& T = tree->t;
    const double* Mexp = nullptr;
    const double* Lexp = nullptr;
    int R = 1;
    VFMM_CHECK(solve_expansions(tree, ops, workspace_dev, workspace_bytes, &Mexp, &Lexp, &R));
    OffArgs a;
    a.k = ops->k;
    a.P = ops->p + 1;
    a.depth = T.depth;
    a.R = R;
    a.n = n_points;
    a.lox = T.cx - T.width / 2.0;
    a.loy = T.cy - T.width / 2.0;
    a.width = T.width;
    a.child0 = T.child0;
    a.level = T.level;
    a.ix = T.ix;
    a.iy = T.iy;
    a.leaf_of_box = T.leaf_of_box;
    a.uptr = T.lptr[VFMM_LIST_U];
    a.uidx = T.lidx[VFMM_LIST_U];
    a.wptr = T.lptr[VFMM_LIST_W];
    a.widx = T.lidx[VFMM_LIST_W];
    a.wcfg = T.lcfg[VFMM_LIST_W];
    a.f = f_dev;
    a.Mexp = Mexp;
    a.Lexp = Lexp;
    a.x = x_dev;
    a.y = y_dev;
    a.u = u_dev;
    a.ux = ux_dev;
    a.uy = uy_dev;
    const int k = ops->k;
    const double pi = 3.14159265358979323846;
    for (int m = 0; m < 16; ++m)
        for (int i = 0; i < 16; ++i) {
            double v = 0.0;
            if (m < k && i < k) {
                const double th = pi * (2 * i + 1) / (2.0 * k);  // x_i = -cos(th), T_m(x_i) = cos(m (pi - th))
                v = (m == 0 ? 1.0 : 2.0) / k * std::cos(m * (pi - th));
            }
            a.A[m * 16 + i] = v;
        }
    offnode_kernel<<<(unsigned)n_points, kOffThreads, 0, (cudaStream_t)stream>>>(a);
    VFMM_CUDA(cudaGetLastError());
    return VFMM_OK;
}
