// Plane-wave (diagonalised) M2L for the FP64 form: the far-field speed-up Section 3.1 attributes
// to the box code it builds on, written for the scaled Laurent/Taylor expansions of this library.
//
// For a V-list pair (source box c, target box b, same width h, source centre offset D = (z_c -
// z_b) / h) the multipole terms of c at a target zeta (offset from z_b in units of h) are
// (zeta - D)^-n. A rotation d = i^q (q = 0..3) chosen by the offset's side puts the source on the
// negative real side: zeta - D = d (U0 + zeta / d), U0 = -D / d, Re U0 in {2, 3}, |Im U0| <= 3.
// With the Laplace transform 1/u^n = 1/(n-1)! int_0^inf lambda^(n-1) e^(-lambda u) d lambda and a
// quadrature rule (lambda_j, omega_j) exact for the moments this needs (planewave_rule.h):
//
//   outgoing  X_q(c)[j] = sum_{n=1..p} a~_n d_q^-n lambda_j^(n-1) / (n-1)!        (per box, per q)
//   translate Y_q(b)[j] = sum_{c in V(b), side q} e^(-lambda_j U0(c, b)) X_q(c)[j]  (diagonal)
//   incoming  b~_l(b)  = sum_j omega_j (-lambda_j)^l / l! sum_q d_q^-l Y_q(b)[j]
//
// The log term of the multipole (a~_0 log(z - z_c)) is added exactly per entry: a~_0 log|D| to
// b~_0 and -a~_0 / (l D^l) to b~_l; the additive a~_0 log h stays with the downward kernel, as for
// the dense M2L. The result equals the dense translation up to the rule's error (about 2e-15 of
// the expansions' scale for the rules in use).
#include <cmath>
#include <complex>
#include <vector>

#include "ops.cuh"
#include "planewave_rule.h"
#include "vfmm_internal.cuh"

namespace vfmm {

namespace {

constexpr int kPwWarps = 4;  // boxes per CTA (one warp each)

// Side of a V offset: q with d = i^q and Re(-D / d) >= 2.
int pw_side(int dx, int dy) {
    if (dy >= 2) return 3;
    if (dy <= -2) return 1;
    return dx >= 2 ? 2 : 0;
}

// a * (-i)^k
__device__ __forceinline__ double2 rot_mi(double2 a, int k) {
    double x = a.x, y = a.y;
    if (k & 1) {
        const double t = x;
        x = y;
        y = -t;
    }
    if (k & 2) {
        x = -x;
        y = -y;
    }
    return make_double2(x, y);
}

// Outgoing plane waves of every box in [begin, end): one warp per box, lane j + 32 t for node j.
__global__ void __launch_bounds__(32 * kPwWarps) pw_out_kernel(int begin, int end, int P, int S,
                                                              const double* __restrict__ C,
                                                              const double2* __restrict__ Mexp,
                                                              double2* __restrict__ X) {
    const int lane = threadIdx.x & 31;
    const int b = begin + blockIdx.x * kPwWarps + (threadIdx.x >> 5);
    if (b >= end) return;
    const double2* a = Mexp + (size_t)b * P;
    double xr[4][3], xi[4][3];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int t = 0; t < 3; ++t) xr[q][t] = xi[q][t] = 0.0;
    // n in steps of 4 from 1, so that every rotation (q n) mod 4 is known at compile time
    for (int n0 = 1; n0 < P; n0 += 4) {
#pragma unroll
        for (int dn = 0; dn < 4; ++dn) {
            const int n = n0 + dn;
            if (n >= P) break;
            const double2 an = a[n];
            double c[3];
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                const int j = lane + 32 * t;
                c[t] = j < S ? C[(size_t)(n - 1) * S + j] : 0.0;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const double2 r = rot_mi(an, (q * (1 + dn)) & 3);  // d_q^-n = (-i)^(q n), n = 1 + dn mod 4
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    xr[q][t] = fma(c[t], r.x, xr[q][t]);
                    xi[q][t] = fma(c[t], r.y, xi[q][t]);
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const int j = lane + 32 * t;
            if (j < S) X[((size_t)b * 4 + q) * S + j] = make_double2(xr[q][t], xi[q][t]);
        }
}

// Incoming: local coefficients b~_0..b~_p of every box in [begin, end) from its V list (zero for
// boxes without one). One warp per box: the diagonal translations with nodes over the lanes, the
// four sides folded into the four phases d_q^-l (l mod 4) in shared memory, then one lane per l.
__global__ void __launch_bounds__(32 * kPwWarps) pw_in_kernel(int begin, int end, int P, int S, int Sp,
                                                             const int32_t* __restrict__ vptr,
                                                             const int32_t* __restrict__ vidx,
                                                             const int32_t* __restrict__ vcfg,
                                                             const int32_t* __restrict__ side,
                                                             const double2* __restrict__ E,
                                                             const double* __restrict__ G,
                                                             const double2* __restrict__ A0,
                                                             const double2* __restrict__ X,
                                                             const double2* __restrict__ Mexp,
                                                             double* __restrict__ L) {
    extern __shared__ __align__(16) unsigned char pw_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = begin + blockIdx.x * kPwWarps + warp;
    if (b >= end) return;
    double2* Z = reinterpret_cast<double2*>(pw_raw) + (size_t)warp * 4 * Sp;
    const int e0 = vptr[b], e1 = vptr[b + 1];
    // one pass over the V list per side q: Y_q[j] = sum e^(-lambda_j U0) X_q(c)[j] in registers, then
    // folded into the four phases Z_r[j] = sum_q d_q^-r Y_q[j] (r = l mod 4)
    double zr[4][3], zi[4][3];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int t = 0; t < 3; ++t) zr[r][t] = zi[r][t] = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        double yr[3] = {0.0, 0.0, 0.0}, yi[3] = {0.0, 0.0, 0.0};
        for (int e = e0; e < e1; ++e) {
            const int cf = vcfg[e];
            if (side[cf] != q) continue;
            const size_t xo = ((size_t)vidx[e] * 4 + q) * S;
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                const int j = lane + 32 * t;
                if (j < S) {
                    const double2 ex = E[(size_t)cf * S + j];
                    const double2 x = X[xo + j];
                    yr[t] = fma(ex.x, x.x, fma(-ex.y, x.y, yr[t]));
                    yi[t] = fma(ex.x, x.y, fma(ex.y, x.x, yi[t]));
                }
            }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                const double2 v = rot_mi(make_double2(yr[t], yi[t]), (q * r) & 3);
                zr[r][t] += v.x;
                zi[r][t] += v.y;
            }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const int j = lane + 32 * t;
            if (j < S) Z[r * Sp + j] = make_double2(zr[r][t], zi[r][t]);
        }
    __syncwarp();
    for (int l = lane; l < P; l += 32) {
        const double2* Zr = Z + (l & 3) * Sp;
        double re = 0.0, im = 0.0;
        for (int j = 0; j < S; ++j) {
            const double g = G[(size_t)j * P + l];
            const double2 z = Zr[j];
            re = fma(g, z.x, re);
            im = fma(g, z.y, im);
        }
        // the multipoles' log terms, exactly
        for (int e = e0; e < e1; ++e) {
            const double2 a0 = Mexp[(size_t)vidx[e] * P];
            const double2 t = A0[(size_t)vcfg[e] * P + l];
            re += a0.x * t.x - a0.y * t.y;
            im += a0.x * t.y + a0.y * t.x;
        }
        L[((size_t)b * P + l) * 2] = re;
        L[((size_t)b * P + l) * 2 + 1] = im;
    }
}

template <typename T>
int upload(T** dst, const std::vector<T>& v, cudaStream_t st) {
    VFMM_CUDA(cudaMalloc(dst, v.size() * sizeof(T)));
    VFMM_CUDA(cudaMemcpyAsync(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    return VFMM_OK;
}

}  // namespace

// Shared-memory row stride of the four phase rows: congruent to 2 mod 8 double2 values, so that
// the four rows a warp reads at once sit in different banks.
int pw_stride(int S) { return S + ((2 - S % 8) + 8) % 8; }

int planewave_prepare(vfmm_ops* o, cudaStream_t st) {
    const PlaneWaveRule* rule = nullptr;
    for (const PlaneWaveRule& r : kPlaneWaveRules)
        if (o->p <= r.pmax) {
            rule = &r;
            break;
        }
    if (!rule) return fail(VFMM_ERR_INVALID_ARG, "no plane-wave rule for this p");
    const int S = rule->s, p = o->p, P = p + 1;
    if (S > 96) return fail(VFMM_ERR_INTERNAL, "plane-wave rule longer than 96 nodes");
    std::vector<double> C((size_t)std::max(p, 1) * S), G((size_t)S * P);
    for (int j = 0; j < S; ++j) {
        const double lam = rule->lambda[j];
        double v = 1.0;  // lambda^(n-1) / (n-1)!
        for (int n = 1; n <= p; ++n) {
            C[(size_t)(n - 1) * S + j] = v;
            v *= lam / n;
        }
        double g = rule->omega[j];  // omega (-lambda)^l / l!
        for (int l = 0; l <= p; ++l) {
            G[(size_t)j * P + l] = g;
            g *= -lam / (l + 1);
        }
    }
    std::vector<double2> E((size_t)kVCfg * S), A0((size_t)kVCfg * P);
    std::vector<int32_t> side(kVCfg);
    for (int cf = 0; cf < kVCfg; ++cf) {
        int dx = 0, dy = 0;
        v_offset(cf, &dx, &dy);
        const int q = pw_side(dx, dy);
        side[cf] = q;
        const std::complex<double> D(dx, dy);
        const std::complex<double> iq[4] = {{1, 0}, {0, 1}, {-1, 0}, {0, -1}};
        const std::complex<double> U0 = -D / iq[q];
        for (int j = 0; j < S; ++j) {
            const std::complex<double> v = std::exp(-rule->lambda[j] * U0);
            E[(size_t)cf * S + j] = make_double2(v.real(), v.imag());
        }
        A0[(size_t)cf * P] = make_double2(std::log(std::abs(D)), 0.0);
        std::complex<double> Dl = 1.0;
        for (int l = 1; l <= p; ++l) {
            Dl *= D;
            const std::complex<double> v = -1.0 / ((double)l * Dl);
            A0[(size_t)cf * P + l] = make_double2(v.real(), v.imag());
        }
    }
    o->pw_s = S;
    VFMM_CHECK(upload(&o->pw_C, C, st));
    VFMM_CHECK(upload(&o->pw_G, G, st));
    VFMM_CHECK(upload(&o->pw_E, E, st));
    VFMM_CHECK(upload(&o->pw_A0, A0, st));
    VFMM_CHECK(upload(&o->pw_side, side, st));
    VFMM_CUDA(cudaStreamSynchronize(st));
    return VFMM_OK;
}

void planewave_free(vfmm_ops* o) {
    void* ps[] = {o->pw_C, o->pw_G, o->pw_E, o->pw_A0, o->pw_side};
    for (void* q : ps)
        if (q) cudaFree(q);
    o->pw_C = o->pw_G = nullptr;
    o->pw_E = o->pw_A0 = nullptr;
    o->pw_side = nullptr;
}

size_t planewave_work_doubles(int64_t n_boxes, const vfmm_ops& o) { return (size_t)n_boxes * 4 * o.pw_s * 2; }

// V-list local coefficients of boxes [begin, n_boxes) into L [n_boxes][2(p+1)] (rows below begin
// untouched); X: [n_boxes][4][s] complex scratch.
int planewave_m2l(const vfmm_ops& o, int begin, int n_boxes, const int32_t* vptr, const int32_t* vidx,
                  const int32_t* vcfg, const double* Mexp, double* X, double* L, cudaStream_t st) {
    const int n = n_boxes - begin;
    if (n <= 0) return VFMM_OK;
    const int P = o.p + 1, S = o.pw_s, Sp = pw_stride(S);
    const unsigned grid = (unsigned)((n + kPwWarps - 1) / kPwWarps);
    pw_out_kernel<<<grid, 32 * kPwWarps, 0, st>>>(begin, n_boxes, P, S, o.pw_C,
                                                   reinterpret_cast<const double2*>(Mexp),
                                                   reinterpret_cast<double2*>(X));
    const size_t smem = (size_t)kPwWarps * 4 * Sp * sizeof(double2);
    pw_in_kernel<<<grid, 32 * kPwWarps, smem, st>>>(begin, n_boxes, P, S, Sp, vptr, vidx, vcfg, o.pw_side,
                                                     o.pw_E, o.pw_G, o.pw_A0,
                                                     reinterpret_cast<const double2*>(X),
                                                     reinterpret_cast<const double2*>(Mexp), L);
    VFMM_CUDA(cudaGetLastError());
    return VFMM_OK;
}

}  // namespace vfmm

using namespace vfmm;

extern "C" int vfmm_ops_set_m2l(vfmm_ops* ops, int32_t form) {
    if (!ops) return fail(VFMM_ERR_INVALID_ARG, "null ops");
    if (form != VFMM_M2L_DENSE && form != VFMM_M2L_PLANEWAVE) return fail(VFMM_ERR_INVALID_ARG, "unknown M2L form");
    if (form == VFMM_M2L_PLANEWAVE && ops->precision != VFMM_FP64)
        return fail(VFMM_ERR_INVALID_ARG, "the plane-wave M2L is a kernel of the FP64 form");
    ops->m2l_form = form;
    return VFMM_OK;
}

extern "C" int vfmm_ops_get_m2l(const vfmm_ops* ops, int32_t* form, int32_t* n_waves) {
    if (!ops || !form) return fail(VFMM_ERR_INVALID_ARG, "null argument");
    *form = ops->m2l_form;
    if (n_waves) *n_waves = ops->pw_s;
    return VFMM_OK;
}
