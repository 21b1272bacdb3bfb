// Operator-set handle (device-resident unit-scale tables).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "vfmm.h"

struct vfmm_ops {
    int k = 0, p = 0, precision = VFMM_FP64;
    double* xhat = nullptr;   // [k] node positions on [-1/2, 1/2]
    double* near = nullptr;   // [33][3kk][kk]: rows q*kk + t (q = u, u_x, u_y), columns s
    double* s2m = nullptr;    // [2(p+1)][kk]: rows 2n (Re), 2n+1 (Im)
    double* s2l_t = nullptr;  // [20][kk][p+1] complex
    double* m2m_t = nullptr;  // [4][in][out] complex
    double* l2l_t = nullptr;  // [4][in][out] complex
    // the same translations in rotated form (one real [in][out] matrix for all four child
    // positions; the rotations are applied by the kernels, see tables.cu)
    double* m2m_r = nullptr;  // [in][out] real
    double* l2l_r = nullptr;  // [in][out] real
    double* m2l_t = nullptr;  // [40][in][out] complex
    double* l2t = nullptr;    // [3kk][2(p+1)] real
    // real forms for the FP64 form's gather GEMMs: rows 2l (Re), 2l + 1 (Im) of output coefficient l
    double* m2l_real = nullptr;  // [40][2(p+1)][2(p+1)]: columns 2n, 2n + 1 of input coefficient n
    double* s2l_real = nullptr;  // [20][2(p+1)][kk]
    // split-precision near-field operands (VFMM_MIXED)
    void* mixed = nullptr;
};

namespace vfmm {
int mixed_prepare(vfmm_ops* o, cudaStream_t st);
void mixed_free(vfmm_ops* o);
void free_ops(vfmm_ops* o);
}  // namespace vfmm
