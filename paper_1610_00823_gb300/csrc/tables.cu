// Unit-scale operators of the box code, generated on the device (Section 3.1: the near-field
// tables are computed once for a unit box and reused at every level up to scale; Section 3.2 for
// the gradient tables).
//
// Scaling: a box of width h stores its multipole coefficients as a_n / h^n and its
// local coefficients as b_l h^l; the expansions represent
// Phi(z) = int log(z - w) f(w) dA(w), u = -(1/2pi) Re Phi, u_x - i u_y = -(1/2pi) Phi'.
// With this scaling each operator is level independent; the solve applies the
// area factors h^2 and the additive log(h) terms.
//
// Translations (series of log(z - w) and (z - w)^-n):
//   M2M (child -> parent, tau = (z_c - z_P)/h_P):
//       A_0 = a_0, A_l = -a_0 tau^l / l + sum_{n=1..l} a_n 2^-n C(l-1, n-1) tau^(l-n)
//   M2L (D = (z_c - z_b)/h, same level):
//       b_0 = a_0 log|D| + sum_n a_n (-D)^-n,  b_l = -a_0/(l D^l) + D^-l sum_n a_n (-D)^-n C(n+l-1, l)
//   L2L (parent -> child, sigma = (z_c - z_P)/h_P):
//       c_m = 2^-m sum_{l>=m} b_l C(l, m) sigma^(l-m)
//
// Rotated real form of M2M and L2L. For child position pos the shift is tau = g / 4 with the
// Gaussian integer g = sx + i sy (sx, sy = +-1, |g|^2 = 2), so tau^(l-n) = g^l g^-n / 4^(l-n)
// factors into a rotation of the input, a real matrix and a rotation of the output. With
//   g^l  = sigma_l 2^floor(l/2),  sigma_l = (i s)^floor(l/2) (sx + i sy)^(l mod 2),
//   g^-n = rho_n 2^-ceil(n/2),    rho_n = conj(sigma_n),  s = sx sy,
// M2M is A_l = sigma_l sum_n Rm[n][l] (rho_n a_n) and L2L is c_m = rho_m sum_l Rl[l][m] (sigma_l b_l):
//   Rm[n][l] = 2^-n C(l-1, n-1) 4^(n-l) 2^(floor(l/2) - ceil(n/2))  (n >= 1),
//   Rm[0][l] = -4^-l / l 2^floor(l/2) (l >= 1), Rm[0][0] = 1,
//   Rl[l][m] = 2^-m C(l, m) 4^(m-l) 2^(floor(l/2) - ceil(m/2))  (l >= m).
// The real matrix is the same for the four positions, and rho_n, sigma_l are Gaussian integers
// whose products with an expansion coefficient take sign changes, swaps and at most one addition
// per component: half the FP64 work of the complex form.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "near_quad.cuh"
#include "ops.cuh"
#include "vfmm_internal.cuh"

namespace vfmm {

// ---------------------------------------------------------------- near tables
constexpr double kDEStep = 0.05;  // tanh-sinh step
constexpr int kDEHalf = 70;       // nodes j in [-70, 70]: |u| <= 3.5
constexpr int kChunk = 128;

// grid (kk targets, 33 configurations); 256 threads. Thread t accumulates basis
// function s = t % kk over the slice t / kk of every chunk of quadrature nodes.
__global__ void __launch_bounds__(256) near_table_kernel(int k, const double* __restrict__ xs,
                                                         const double* __restrict__ bw, double* __restrict__ out) {
    __shared__ double sW[3][kChunk];
    __shared__ double sBX[kChunk][16];
    __shared__ double sBY[kChunk][16];
    __shared__ double sDE[3][2 * kDEHalf + 1];
    __shared__ double sxs[16], sbw[16];
    __shared__ QuadPiece pcs[8];
    __shared__ int npc;
    __shared__ double red[3][256];
    const int kk = k * k;
    const int t = threadIdx.x;
    const int tgt = blockIdx.x, cfg = blockIdx.y;
    double rho, dx, dy;
    near_config_geometry(cfg, &rho, &dx, &dy);
    if (t < k) {
        sxs[t] = xs[t];
        sbw[t] = bw[t];
    }
    const int N = 2 * kDEHalf + 1;
    for (int j = t; j < N; j += blockDim.x) {
        DENode d = de_node(j - kDEHalf, kDEStep);
        sDE[0][j] = d.x;
        sDE[1][j] = d.xc;
        sDE[2][j] = d.w;
    }
    const double x = xs[tgt % k], y = xs[tgt / k];
    if (t == 0) npc = make_pieces(x, y, dx, dy, rho, pcs);
    __syncthreads();
    const int parts = blockDim.x / kk;  // >= 1 for k <= 16
    const int s = t % kk, part = t / kk;
    const int si = s % k, sj = s / k;
    double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
    const long long total = (long long)npc * N * N;
    for (long long base = 0; base < total; base += kChunk) {
        if (t < kChunk) {
            long long g = base + t;
            double w3[3] = {0.0, 0.0, 0.0};
            double yx = dx, yy = dy;
            if (g < total) {
                int ip = (int)(g / ((long long)N * N));
                int rem = (int)(g % ((long long)N * N));
                int js = rem / N, jt = rem % N;
                DENode ds{sDE[0][js], sDE[1][js], sDE[2][js]};
                DENode dt{sDE[0][jt], sDE[1][jt], sDE[2][jt]};
                node_weights(pcs[ip], x, y, ds, dt, w3, &yx, &yy);
            }
            sW[0][t] = w3[0];
            sW[1][t] = w3[1];
            sW[2][t] = w3[2];
            double bx[16], by[16];
            bary_basis(k, sxs, sbw, (yx - dx) / rho, bx);
            bary_basis(k, sxs, sbw, (yy - dy) / rho, by);
            for (int i = 0; i < k; ++i) {
                sBX[t][i] = bx[i];
                sBY[t][i] = by[i];
            }
        }
        __syncthreads();
        if (part < parts) {
            for (int c = part; c < kChunk; c += parts) {
                double b = sBX[c][si] * sBY[c][sj];
                acc0 += sW[0][c] * b;
                acc1 += sW[1][c] * b;
                acc2 += sW[2][c] * b;
            }
        }
        __syncthreads();
    }
    red[0][t] = acc0;
    red[1][t] = acc1;
    red[2][t] = acc2;
    __syncthreads();
    if (part == 0) {
        for (int q = 0; q < 3; ++q) {
            double v = 0.0;
            for (int pp = 0; pp < parts; ++pp) v += red[q][pp * kk + s];
            out[(((size_t)cfg * 3 + q) * kk + tgt) * kk + s] = v;
        }
    }
}

// ---------------------------------------------------------------- S2M (1-D moments)
// mu[i][m] = int_{-1/2}^{1/2} l_i(x) x^m dx by Gauss-Legendre (exact).
__global__ void moments_kernel(int k, int p, const double* __restrict__ xs, const double* __restrict__ bw,
                               const double* __restrict__ gx, const double* __restrict__ gw, int ng,
                               double* __restrict__ mu) {
    int i = blockIdx.x, m = threadIdx.x;
    if (m > p) return;
    double acc = 0.0;
    double bx[16];
    for (int a = 0; a < ng; ++a) {
        bary_basis(k, xs, bw, gx[a], bx);
        acc += gw[a] * bx[i] * pow(gx[a], (double)m);
    }
    mu[i * (p + 1) + m] = acc;
}

__device__ inline double binom_d(int n, int r) {
    if (r < 0 || r > n) return 0.0;
    double v = 1.0;
    if (r > n - r) r = n - r;
    for (int q = 1; q <= r; ++q) v = v * (n - r + q) / q;
    return v;
}

// Q_n,s = -(1/n) int l_i(x) l_j(y) (x + i y)^n = -(1/n) sum_m C(n,m) i^(n-m) mu_i,m mu_j,n-m.
// Output rows 2n (real part) and 2n+1 (imaginary part) of the [2(p+1)][kk] S2M matrix.
__global__ void s2m_kernel(int k, int p, const double* __restrict__ mu, double* __restrict__ s2m) {
    int n = blockIdx.x, s = threadIdx.x;
    int kk = k * k;
    if (s >= kk) return;
    int i = s % k, j = s / k;
    double re = 0.0, im = 0.0;
    if (n == 0) {
        re = mu[i * (p + 1)] * mu[j * (p + 1)];
    } else {
        for (int m = 0; m <= n; ++m) {
            double v = binom_d(n, m) * mu[i * (p + 1) + m] * mu[j * (p + 1) + (n - m)];
            switch ((n - m) & 3) {  // i^(n-m)
                case 0: re += v; break;
                case 1: im += v; break;
                case 2: re -= v; break;
                default: im -= v; break;
            }
        }
        re *= -1.0 / n;
        im *= -1.0 / n;
    }
    s2m[(size_t)(2 * n) * kk + s] = re;
    s2m[(size_t)(2 * n + 1) * kk + s] = im;
}

// ---------------------------------------------------------------- S2L (X list)
// R[cfg][l][s] = -(1/l) int l_s(w) (D + 2w)^-l dw (l >= 1), R[cfg][0][s] = int l_s log|D + 2w|,
// composite Gauss-Legendre on the unit box. Stored transposed: s2l_t[cfg][s][l] complex.
__global__ void s2l_kernel(int k, int p, const double* __restrict__ xs, const double* __restrict__ bw,
                           const double* __restrict__ gx, const double* __restrict__ gw, int ng,
                           double* __restrict__ s2l_t) {
    __shared__ double LX[128][16];
    __shared__ double zr[256], zi[256];
    const int cfg = blockIdx.x, l = blockIdx.y;
    const int kk = k * k;
    const int t = threadIdx.x;
    int px, py;
    far_pattern(cfg, &px, &py);
    const double Dx = px / 2.0, Dy = py / 2.0;
    for (int a = t; a < ng; a += blockDim.x) {
        double bx[16];
        bary_basis(k, xs, bw, gx[a], bx);
        for (int i = 0; i < k; ++i) LX[a][i] = bx[i];
    }
    __syncthreads();
    const int i = t % k, j = t / k;
    double ar = 0.0, ai = 0.0;
    const int total = ng * ng;
    for (int base = 0; base < total; base += 256) {
        int g = base + t;
        double vr = 0.0, vi = 0.0;
        if (g < total) {
            int a = g % ng, b = g / ng;
            double zx = Dx + 2.0 * gx[a], zy = Dy + 2.0 * gx[b];
            double w = gw[a] * gw[b];
            if (l == 0) {
                vr = w * 0.5 * log(zx * zx + zy * zy);
            } else {
                // (zx + i zy)^-l = r^-l e^{-i l theta}
                double lr = 0.5 * log(zx * zx + zy * zy);
                double th = atan2(zy, zx);
                double mag = exp(-l * lr) * (-1.0 / l) * w;
                double sn, cs;
                sincos(-l * th, &sn, &cs);
                vr = mag * cs;
                vi = mag * sn;
            }
        }
        zr[t] = vr;
        zi[t] = vi;
        __syncthreads();
        if (t < kk) {
            int lim = min(256, total - base);
            for (int c = 0; c < lim; ++c) {
                int gg = base + c;
                int a = gg % ng, b = gg / ng;
                double bas = LX[a][i] * LX[b][j];
                ar += zr[c] * bas;
                ai += zi[c] * bas;
            }
        }
        __syncthreads();
    }
    if (t < kk) {
        size_t o = (((size_t)cfg * kk + t) * (p + 1) + l) * 2;
        s2l_t[o] = ar;
        s2l_t[o + 1] = ai;
    }
}

// ---------------------------------------------------------------- host helpers
static void gauss_legendre(int n, double a, double b, std::vector<double>& x, std::vector<double>& w) {
    // Newton iteration on P_n from the Chebyshev initial guess
    const double pi = 3.14159265358979323846;
    x.resize(n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = 0.0;
            for (int j = 1; j <= n; ++j) {
                double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
            }
            dp = n * (z * p0 - p1) / (z * z - 1.0);
            double dz = p0 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = 0.0;
        for (int j = 1; j <= n; ++j) {
            double p2 = p1;
            p1 = p0;
            p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
        }
        dp = n * (z * p0 - p1) / (z * z - 1.0);
        x[n - 1 - i] = 0.5 * (a + b) + 0.5 * (b - a) * z;
        w[n - 1 - i] = (b - a) / ((1.0 - z * z) * dp * dp);
    }
}

static double binom(int n, int r) {
    if (r < 0 || r > n) return 0.0;
    double v = 1.0;
    if (r > n - r) r = n - r;
    for (int q = 1; q <= r; ++q) v = v * (n - r + q) / q;
    return v;
}

typedef std::complex<double> cd;

// The real matrices of the rotated M2M and L2L ([in][out]).
static void rotated_ops(int p, std::vector<double>& m2m_r, std::vector<double>& l2l_r) {
    const int P = p + 1;
    m2m_r.assign((size_t)P * P, 0.0);
    l2l_r.assign((size_t)P * P, 0.0);
    // 2^(floor(a / 2) - ceil(b / 2)): a is the index rotated by sigma, b the one rotated by rho
    auto scale = [](int a, int b) { return std::ldexp(1.0, a / 2 - (b + 1) / 2); };
    m2m_r[0] = 1.0;
    for (int l = 1; l <= p; ++l) {
        m2m_r[l] = -std::ldexp(1.0, -2 * l) / (double)l * scale(l, 0);
        for (int n = 1; n <= l; ++n)
            m2m_r[(size_t)n * P + l] = std::ldexp(binom(l - 1, n - 1), -n + 2 * (n - l)) * scale(l, n);
    }
    for (int m = 0; m <= p; ++m)
        for (int l = m; l <= p; ++l)
            l2l_r[(size_t)l * P + m] = std::ldexp(binom(l, m), -m + 2 * (m - l)) * scale(l, m);
}

static void closed_form_ops(int p, std::vector<double>& m2m_t, std::vector<double>& l2l_t, std::vector<double>& m2l_t) {
    const int P = p + 1;
    m2m_t.assign((size_t)4 * P * P * 2, 0.0);
    l2l_t.assign((size_t)4 * P * P * 2, 0.0);
    m2l_t.assign((size_t)kVCfg * P * P * 2, 0.0);
    auto put = [&](std::vector<double>& v, int blk, int in, int out, cd z) {
        size_t o = (((size_t)blk * P + in) * P + out) * 2;
        v[o] = z.real();
        v[o + 1] = z.imag();
    };
    for (int pos = 0; pos < 4; ++pos) {
        cd tau(((pos & 1) ? 1.0 : -1.0) / 4.0, ((pos >> 1) ? 1.0 : -1.0) / 4.0);
        put(m2m_t, pos, 0, 0, 1.0);
        for (int l = 1; l <= p; ++l) {
            put(m2m_t, pos, 0, l, -std::pow(tau, l) / (double)l);
            for (int n = 1; n <= l; ++n)
                put(m2m_t, pos, n, l, std::ldexp(1.0, -n) * binom(l - 1, n - 1) * std::pow(tau, l - n));
        }
        for (int m = 0; m <= p; ++m)
            for (int l = m; l <= p; ++l)
                put(l2l_t, pos, l, m, std::ldexp(1.0, -m) * binom(l, m) * std::pow(tau, l - m));
    }
    for (int c = 0; c < kVCfg; ++c) {
        int dx, dy;
        v_offset(c, &dx, &dy);
        cd D(dx, dy);
        cd mD = -D;
        put(m2l_t, c, 0, 0, std::log(std::abs(D)));
        for (int n = 1; n <= p; ++n) put(m2l_t, c, n, 0, std::pow(mD, -n));
        for (int l = 1; l <= p; ++l) {
            put(m2l_t, c, 0, l, -1.0 / ((double)l * std::pow(D, l)));
            for (int n = 1; n <= p; ++n) put(m2l_t, c, n, l, std::pow(D, -l) * std::pow(mD, -n) * binom(n + l - 1, l));
        }
    }
}

// L2T as a real [3kk][2(p+1)] matrix acting on (Re b_0, Im b_0, Re b_1, ...):
// rows t: u = -(1/2pi) Re(sum_l zeta_t^l b_l); rows kk+t, 2kk+t: h u_x, h u_y from
// Phi' = (1/h) sum_l l zeta^(l-1) b_l with u_x = -(1/2pi) Re Phi', u_y = (1/2pi) Im Phi'.
static void l2t_matrix(int k, int p, const std::vector<double>& xh, std::vector<double>& A) {
    const int kk = k * k, P = p + 1;
    const double c = 1.0 / (2.0 * 3.14159265358979323846);
    A.assign((size_t)3 * kk * 2 * P, 0.0);
    for (int t = 0; t < kk; ++t) {
        cd z(xh[t % k], xh[t / k]);
        for (int l = 0; l <= p; ++l) {
            cd E = std::pow(z, l);
            cd dE = l ? (double)l * std::pow(z, l - 1) : cd(0.0);
            A[(size_t)t * 2 * P + 2 * l] = -c * E.real();
            A[(size_t)t * 2 * P + 2 * l + 1] = c * E.imag();
            A[(size_t)(kk + t) * 2 * P + 2 * l] = -c * dE.real();
            A[(size_t)(kk + t) * 2 * P + 2 * l + 1] = c * dE.imag();
            A[(size_t)(2 * kk + t) * 2 * P + 2 * l] = c * dE.imag();
            A[(size_t)(2 * kk + t) * 2 * P + 2 * l + 1] = c * dE.real();
        }
    }
}

template <class T>
static int dalloc_copy(T** dst, const std::vector<T>& v, cudaStream_t st) {
    VFMM_CUDA(cudaMalloc(dst, std::max<size_t>(1, v.size()) * sizeof(T)));
    if (!v.empty()) VFMM_CUDA(cudaMemcpyAsync(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    return VFMM_OK;
}

static int create(int k, int p, int precision, cudaStream_t st, vfmm_ops* o) {
    o->k = k;
    o->p = p;
    o->precision = precision;
    const int kk = k * k, P = p + 1;
    const double pi = 3.14159265358979323846;
    std::vector<double> xh(k), bw(k), W(kk), w1(k);
    for (int i = 0; i < k; ++i) {
        xh[i] = -std::cos(pi * (2.0 * i + 1.0) / (2.0 * k)) / 2.0;
        bw[i] = ((i & 1) ? -1.0 : 1.0) * std::sin((2.0 * i + 1.0) * pi / (2.0 * k));
    }
    VFMM_CHECK(dalloc_copy(&o->xhat, xh, st));
    double* d_bw = nullptr;
    VFMM_CHECK(dalloc_copy(&d_bw, bw, st));
    // near tables
    VFMM_CUDA(cudaMalloc(&o->near, (size_t)kNearCfg * 3 * kk * kk * sizeof(double)));
    near_table_kernel<<<dim3(kk, kNearCfg), 256, 0, st>>>(k, o->xhat, d_bw, o->near);
    VFMM_CUDA(cudaGetLastError());
    // S2M from 1-D moments
    std::vector<double> gx, gw;
    int ng = (k + p) / 2 + 4;
    gauss_legendre(ng, -0.5, 0.5, gx, gw);
    double *d_gx = nullptr, *d_gw = nullptr, *d_mu = nullptr;
    VFMM_CHECK(dalloc_copy(&d_gx, gx, st));
    VFMM_CHECK(dalloc_copy(&d_gw, gw, st));
    VFMM_CUDA(cudaMalloc(&d_mu, (size_t)k * P * sizeof(double)));
    moments_kernel<<<k, 64, 0, st>>>(k, p, o->xhat, d_bw, d_gx, d_gw, ng, d_mu);
    VFMM_CUDA(cudaMalloc(&o->s2m, (size_t)2 * P * kk * sizeof(double)));
    s2m_kernel<<<P, 256, 0, st>>>(k, p, d_mu, o->s2m);
    VFMM_CUDA(cudaGetLastError());
    // S2L: 4 x 4 panels of 32-point Gauss-Legendre on the unit interval
    std::vector<double> cx, cw;
    for (int piece = 0; piece < 4; ++piece) {
        std::vector<double> x, w;
        gauss_legendre(32, -0.5 + 0.25 * piece, -0.25 + 0.25 * piece, x, w);
        cx.insert(cx.end(), x.begin(), x.end());
        cw.insert(cw.end(), w.begin(), w.end());
    }
    double *d_cx = nullptr, *d_cw = nullptr;
    VFMM_CHECK(dalloc_copy(&d_cx, cx, st));
    VFMM_CHECK(dalloc_copy(&d_cw, cw, st));
    VFMM_CUDA(cudaMalloc(&o->s2l_t, (size_t)kFarCfg * kk * P * 2 * sizeof(double)));
    s2l_kernel<<<dim3(kFarCfg, P), 256, 0, st>>>(k, p, o->xhat, d_bw, d_cx, d_cw, (int)cx.size(), o->s2l_t);
    VFMM_CUDA(cudaGetLastError());
    // closed forms
    std::vector<double> m2m_t, l2l_t, m2l_t, l2t;
    closed_form_ops(p, m2m_t, l2l_t, m2l_t);
    l2t_matrix(k, p, xh, l2t);
    VFMM_CHECK(dalloc_copy(&o->m2m_t, m2m_t, st));
    VFMM_CHECK(dalloc_copy(&o->l2l_t, l2l_t, st));
    {
        std::vector<double> m2m_r, l2l_r;
        rotated_ops(p, m2m_r, l2l_r);
        VFMM_CHECK(dalloc_copy(&o->m2m_r, m2m_r, st));
        VFMM_CHECK(dalloc_copy(&o->l2l_r, l2l_r, st));
    }
    VFMM_CHECK(dalloc_copy(&o->m2l_t, m2l_t, st));
    VFMM_CHECK(dalloc_copy(&o->l2t, l2t, st));
    if (precision == VFMM_FP64) {
        // real M2L and S2L matrices: complex c_l = sum M[n][l] x_n -> rows (Re c_l, Im c_l)
        const size_t P2 = 2 * (size_t)P;
        std::vector<double> mr((size_t)kVCfg * P2 * P2), sr((size_t)kFarCfg * P2 * kk), st_((size_t)kFarCfg * kk * P * 2);
        for (int c = 0; c < kVCfg; ++c)
            for (int n = 0; n < P; ++n)
                for (int l = 0; l < P; ++l) {
                    const double re = m2l_t[(((size_t)c * P + n) * P + l) * 2],
                                 im = m2l_t[(((size_t)c * P + n) * P + l) * 2 + 1];
                    double* A = mr.data() + (size_t)c * P2 * P2;
                    A[(2 * l) * P2 + 2 * n] = re;
                    A[(2 * l) * P2 + 2 * n + 1] = -im;
                    A[(2 * l + 1) * P2 + 2 * n] = im;
                    A[(2 * l + 1) * P2 + 2 * n + 1] = re;
                }
        VFMM_CUDA(cudaMemcpyAsync(st_.data(), o->s2l_t, st_.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        VFMM_CUDA(cudaStreamSynchronize(st));
        for (int c = 0; c < kFarCfg; ++c)
            for (int s = 0; s < kk; ++s)
                for (int l = 0; l < P; ++l) {
                    sr[((size_t)c * P2 + 2 * l) * kk + s] = st_[(((size_t)c * kk + s) * P + l) * 2];
                    sr[((size_t)c * P2 + 2 * l + 1) * kk + s] = st_[(((size_t)c * kk + s) * P + l) * 2 + 1];
                }
        VFMM_CHECK(dalloc_copy(&o->m2l_real, mr, st));
        VFMM_CHECK(dalloc_copy(&o->s2l_real, sr, st));
        VFMM_CHECK(planewave_prepare(o, st));
    }
    VFMM_CUDA(cudaStreamSynchronize(st));
    cudaFree(d_bw);
    cudaFree(d_gx);
    cudaFree(d_gw);
    cudaFree(d_mu);
    cudaFree(d_cx);
    cudaFree(d_cw);
    if (precision == VFMM_MIXED) VFMM_CHECK(mixed_prepare(o, st));
    return VFMM_OK;
}

void free_ops(vfmm_ops* o) {
    double* ps[] = {o->xhat,  o->near,  o->s2m, o->s2l_t,    o->m2m_t,   o->l2l_t,
                    o->m2m_r, o->l2l_r, o->m2l_t, o->l2t, o->m2l_real, o->s2l_real};
    for (double* p : ps)
        if (p) cudaFree(p);
    mixed_free(o);
    planewave_free(o);
}

}  // namespace vfmm

using namespace vfmm;

extern "C" int vfmm_ops_create(int32_t k, int32_t p, int32_t precision, void* stream, vfmm_ops** out) {
    if (!out) return fail(VFMM_ERR_INVALID_ARG, "null out");
    *out = nullptr;
    if (k < 4 || k > 16) return fail(VFMM_ERR_INVALID_ARG, "k must be in [4, 16]");
    if (p < 1 || p > 60) return fail(VFMM_ERR_INVALID_ARG, "p must be in [1, 60]");
    if (precision != VFMM_FP64 && precision != VFMM_MIXED) return fail(VFMM_ERR_INVALID_ARG, "unknown precision");
    vfmm_ops* o = new vfmm_ops();
    int r = create(k, p, precision, (cudaStream_t)stream, o);
    if (r != VFMM_OK) {
        free_ops(o);
        delete o;
        return r;
    }
    *out = o;
    return VFMM_OK;
}

extern "C" int vfmm_ops_destroy(vfmm_ops* ops) {
    if (!ops) return VFMM_OK;
    free_ops(ops);
    delete ops;
    return VFMM_OK;
}

extern "C" int vfmm_ops_export(const vfmm_ops* o, int32_t which, double* host, int64_t n_doubles) {
    if (!o || !host) return fail(VFMM_ERR_INVALID_ARG, "null argument");
    const int kk = o->k * o->k, P = o->p + 1;
    std::vector<double> buf;
    auto fetch = [&](const double* src, size_t n) -> int {
        buf.resize(n);
        VFMM_CUDA(cudaMemcpy(buf.data(), src, n * sizeof(double), cudaMemcpyDeviceToHost));
        return VFMM_OK;
    };
    std::vector<double> res;
    switch (which) {
        case VFMM_OP_NEAR:
            VFMM_CHECK(fetch(o->near, (size_t)kNearCfg * 3 * kk * kk));
            res = buf;
            break;
        case VFMM_OP_S2M: {  // [p+1][kk] complex
            VFMM_CHECK(fetch(o->s2m, (size_t)2 * P * kk));
            res.resize((size_t)P * kk * 2);
            for (int n = 0; n < P; ++n)
                for (int s = 0; s < kk; ++s) {
                    res[((size_t)n * kk + s) * 2] = buf[(size_t)(2 * n) * kk + s];
                    res[((size_t)n * kk + s) * 2 + 1] = buf[(size_t)(2 * n + 1) * kk + s];
                }
            break;
        }
        case VFMM_OP_S2L: {  // [20][p+1][kk] complex from [20][kk][p+1]
            VFMM_CHECK(fetch(o->s2l_t, (size_t)kFarCfg * kk * P * 2));
            res.resize(buf.size());
            for (int c = 0; c < kFarCfg; ++c)
                for (int s = 0; s < kk; ++s)
                    for (int l = 0; l < P; ++l)
                        for (int r = 0; r < 2; ++r)
                            res[(((size_t)c * P + l) * kk + s) * 2 + r] = buf[(((size_t)c * kk + s) * P + l) * 2 + r];
            break;
        }
        case VFMM_OP_M2M:
        case VFMM_OP_L2L:
        case VFMM_OP_M2L: {  // [blk][out][in] complex from [blk][in][out]
            const double* src = which == VFMM_OP_M2M ? o->m2m_t : (which == VFMM_OP_L2L ? o->l2l_t : o->m2l_t);
            int nb = which == VFMM_OP_M2L ? kVCfg : 4;
            VFMM_CHECK(fetch(src, (size_t)nb * P * P * 2));
            res.resize(buf.size());
            for (int b = 0; b < nb; ++b)
                for (int i = 0; i < P; ++i)
                    for (int j = 0; j < P; ++j)
                        for (int r = 0; r < 2; ++r)
                            res[(((size_t)b * P + j) * P + i) * 2 + r] = buf[(((size_t)b * P + i) * P + j) * 2 + r];
            break;
        }
        default:
            return fail(VFMM_ERR_INVALID_ARG, "unknown operator id");
    }
    if ((int64_t)res.size() != n_doubles) return fail(VFMM_ERR_INVALID_ARG, "size mismatch for operator export");
    std::copy(res.begin(), res.end(), host);
    return VFMM_OK;
}
