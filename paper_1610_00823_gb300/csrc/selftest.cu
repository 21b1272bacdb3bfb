// Self-test of the failure path of the tensor-core kernels (no counterpart in the paper).
//
// Every wait in those kernels (on a stage's mbarrier, the accumulator barriers, a grid barrier)
// is bounded: when it runs out, the kernel records an error word and returns, and the host turns
// the word into VFMM_ERR_TIMEOUT instead of hanging. This entry point makes such a wait run out
// on purpose, without any fault: one thread waits, through the same bounded-wait routine, on an
// mbarrier that nothing will ever arrive on, gives up after `polls` polls and records the error
// word, which the host reads back exactly as a solve does.
#include "tc_ptx.cuh"
#include "vfmm_internal.cuh"

namespace vfmm {

__global__ void wait_timeout_kernel(long long polls, int* err) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ volatile int no_abort;
    const uint32_t b = tc::smem_u32(&bar);
    if (threadIdx.x == 0) {
        no_abort = 0;
        tc::mbar_init(b, 1);  // expects one arrival that never comes
        tc::mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !tc::mbar_wait(b, 0, &no_abort, polls)) atomicExch(err, 7);
}

}  // namespace vfmm

using namespace vfmm;

extern "C" int vfmm_selftest_wait_timeout(int64_t polls, void* stream) {
    if (polls < 1 || polls > (1ll << 20)) return fail(VFMM_ERR_INVALID_ARG, "polls must be in [1, 2^20]");
    cudaStream_t st = (cudaStream_t)stream;
    int* err = nullptr;
    VFMM_CUDA(cudaMalloc(&err, sizeof(int)));
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        wait_timeout_kernel<<<1, 32, 0, st>>>(polls, err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    // read back by the routine that reads a solve's status word
    const int rc = e == cudaSuccess ? read_status_word(err) : VFMM_OK;
    cudaFree(err);
    if (e != cudaSuccess) return cuda_fail(e, "wait self-test");
    if (rc != VFMM_OK) return rc;
    return fail(VFMM_ERR_INTERNAL, "the self-test wait completed although nothing arrived");
}
