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
    // plane-wave M2L (FP64 form, planewave.cu): rule length s, outgoing [p][s] lambda^(n-1)/(n-1)!,
    // incoming [s][p+1] omega (-lambda)^l / l!, diagonal [40][s] e^(-lambda U0), log terms [40][p+1],
    // side q of each V offset [40]
    int m2l_form = VFMM_M2L_DENSE;
    int pw_s = 0;
    double* pw_C = nullptr;
    double* pw_G = nullptr;
    double2* pw_E = nullptr;
    double2* pw_A0 = nullptr;
    int32_t* pw_side = nullptr;
};

namespace vfmm {
int mixed_prepare(vfmm_ops* o, cudaStream_t st);
void mixed_free(vfmm_ops* o);
void free_ops(vfmm_ops* o);
int planewave_prepare(vfmm_ops* o, cudaStream_t st);
void planewave_free(vfmm_ops* o);
int pw_stride(int S);
size_t planewave_work_doubles(int64_t n_boxes, const vfmm_ops& o);
int planewave_m2l(const vfmm_ops& o, int begin, int n_boxes, const int32_t* vptr, const int32_t* vidx,
                  const int32_t* vcfg, const double* Mexp, double* X, double* L, cudaStream_t st);
}  // namespace vfmm
