// Allocation-free solve: vfmm_volume_potential with its workspace in a static device array.
//
// Who needs this: a host whose device memory is handed out entirely by its own
// pool allocator (a framework's caching allocator, or a service that reserves a
// fixed memory budget at start-up) can neither give this library a workspace
// buffer nor let it call cudaMalloc, which would fail or fragment the pool.
// This entry point needs neither: the scratch it works in is a file-scope
// __device__ array of fixed size that exists on every GPU that loads the library,
// for as long as the process lives.
#include <mutex>

#include "ops.cuh"
#include "vfmm_internal.cuh"

namespace vfmm {

// 32 MiB of scratch: room for trees of a few hundred leaves at k = 8 or about a
// hundred at k = 16 (multipole and local expansions, near-field partial
// products, far-field values of one right-hand side at a time).
constexpr size_t kStaticScratchBytes = 32u << 20;

static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

// Device address of g_scratch, resolved once per device. In host code the name
// g_scratch is only a host-side stand-in, so kernels must be given this address.
constexpr int kMaxDevices = 64;
static void* g_scratch_addr[kMaxDevices] = {nullptr};
static std::mutex g_scratch_mu;

static int scratch_address(void** out) {
    int dev = 0;
    VFMM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(VFMM_ERR_INVALID_ARG, "device index out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_scratch)");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return VFMM_OK;
}

// The solve keeps its status word at the start of its workspace, here the start of the scratch.
int noalloc_status_word(const int** word) {
    void* scratch = nullptr;
    VFMM_CHECK(scratch_address(&scratch));
    *word = static_cast<const int*>(scratch);
    return VFMM_OK;
}

}  // namespace vfmm

using namespace vfmm;

extern "C" int vfmm_volume_potential_noalloc(const vfmm_tree* tree, const vfmm_ops* ops, const double* f_dev,
                                             int32_t nrhs, double* u_dev, double* ux_dev, double* uy_dev,
                                             void* stream) {
    if (!tree || !ops) return fail(VFMM_ERR_INVALID_ARG, "null tree or ops");
    if (nrhs < 1) return fail(VFMM_ERR_INVALID_ARG, "nrhs must be >= 1");
    if (!f_dev || !u_dev || !ux_dev || !uy_dev) return fail(VFMM_ERR_INVALID_ARG, "null buffer");
    // One right-hand side per solve: the schedules for a single right-hand side are built with the
    // tree, whereas folding several into one solve (the mixed form's usual path) would build new
    // schedules in device memory on first use.
    size_t need = 0;
    VFMM_CHECK(vfmm_workspace_size(tree, ops, 1, 0, &need));
    if (need > kStaticScratchBytes)
        return fail(VFMM_ERR_WORKSPACE, "tree needs " + std::to_string(need) +
                                            " bytes of scratch; the static scratch holds " +
                                            std::to_string(kStaticScratchBytes) + " bytes");
    void* scratch = nullptr;
    VFMM_CHECK(scratch_address(&scratch));
    // Everything runs on `stream` alone (no second stream is created). Nothing in the scratch has
    // to start at zero but the status word at its start, cleared here once for the whole call (a
    // bounded wait that ran out for any right-hand side stays reported): the solve writes every
    // expansion, partial product and far value before reading it, and clears the
    // local expansions of levels 0 and 1 (and its barrier counters) itself on every call.
    VFMM_CUDA(cudaMemsetAsync(scratch, 0, sizeof(int), (cudaStream_t)stream));
    const size_t n = (size_t)tree->t.n_leaves * ops->k * ops->k;
    for (int r = 0; r < nrhs; ++r)
        VFMM_CHECK(volume_potential(tree, ops, f_dev + r * n, 1, u_dev + r * n, ux_dev + r * n, uy_dev + r * n,
                                    scratch, kStaticScratchBytes, (cudaStream_t)stream, false, false));
    return VFMM_OK;
}
