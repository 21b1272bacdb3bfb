// Device evaluation of the built-in right-hand sides (layouts in vfmm.h).
#pragma once

#include <cuda_runtime.h>

#include "vfmm.h"

namespace vfmm {

struct SourceDev {
    int kind = 0;
    int n = 0;
    const double* params = nullptr;  // device copy of the parameter array
};

__device__ inline double gauss_sum_eval(const double* rows, int n, double x, double y) {
    double acc = 0.0;
    for (int g = 0; g < n; ++g) {
        double cx = rows[4 * g], cy = rows[4 * g + 1], sig = rows[4 * g + 2], amp = rows[4 * g + 3];
        double dx = x - cx, dy = y - cy;
        acc += amp * exp(-(dx * dx + dy * dy) / (2.0 * sig * sig));
    }
    return acc;
}

// psi(t) = e^{-1/t} / (e^{-1/t} + e^{-1/(1-t)}) on (0, 1), 0 below, 1 above.
__device__ inline double smooth_step_eval(double t) {
    if (t <= 0.0) return 0.0;
    if (t >= 1.0) return 1.0;
    double a = exp(-1.0 / t), b = exp(-1.0 / (1.0 - t));
    return a / (a + b);
}

__device__ inline double source_eval(const SourceDev& s, double x, double y) {
    if (s.kind == VFMM_SRC_CONSTANT) return s.params[0];
    if (s.kind == VFMM_SRC_GAUSS_SUM) return gauss_sum_eval(s.params, s.n, x, y);
    // kinked: f = g max(0, phi) + h, phi = r_chi^2 - |x|^2
    const double* a = s.params;
    const double* c = s.params + 7;
    double rho = hypot(x, y);
    double th = atan2(y, x);
    double sum = 0.0;
    for (int i = 0; i < 7; ++i) sum += a[i] * cos((i + 2) * th + c[i]);
    double chi = smooth_step_eval((rho - 0.1) / 0.2);
    double r = 0.6 + chi * sum;
    double phi = r * r - rho * rho;
    double g = gauss_sum_eval(s.params + 14, 5, x, y);
    double h = gauss_sum_eval(s.params + 34, 5, x, y);
    return g * (phi > 0.0 ? phi : 0.0) + h;
}

// Level set of the kinked source, phi = r_chi^2 - |x|^2 (its zero set is the curve where f is only
// continuous); the same arithmetic as in source_eval. Other sources: 1 (no boundary).
__device__ inline double source_phi(const SourceDev& s, double x, double y) {
    if (s.kind != VFMM_SRC_KINKED) return 1.0;
    const double* a = s.params;
    const double* c = s.params + 7;
    double rho = hypot(x, y);
    double th = atan2(y, x);
    double sum = 0.0;
    for (int i = 0; i < 7; ++i) sum += a[i] * cos((i + 2) * th + c[i]);
    double chi = smooth_step_eval((rho - 0.1) / 0.2);
    double r = 0.6 + chi * sum;
    return r * r - rho * rho;
}

}  // namespace vfmm
