// Error reporting shared by every C-ABI entry point.
#include <string>

#include "ops.cuh"
#include "vfmm_internal.cuh"

namespace vfmm {

static thread_local std::string g_detail;

void set_error(const std::string& msg) { g_detail = msg; }

int fail(int code, const std::string& msg) {
    g_detail = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    g_detail = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return e == cudaErrorMemoryAllocation ? VFMM_ERR_OOM : VFMM_ERR_CUDA;
}

}  // namespace vfmm

extern "C" const char* vfmm_strerror(int code) {
    switch (code) {
        case VFMM_OK: return "ok";
        case VFMM_ERR_INVALID_ARG: return "invalid argument";
        case VFMM_ERR_OOM: return "out of device memory";
        case VFMM_ERR_CUDA: return "CUDA error";
        case VFMM_ERR_NOT_BUILT: return "not built";
        case VFMM_ERR_TIMEOUT: return "bounded device wait expired";
        case VFMM_ERR_WORKSPACE: return "workspace too small";
        case VFMM_ERR_INTERNAL: return "internal error";
        default: return "unknown error code";
    }
}

extern "C" const char* vfmm_last_error_detail(void) { return vfmm::g_detail.c_str(); }
