// Diagnostic: exercise the bounded device-side wait that every pipelined
// kernel of the library uses, on an mbarrier that nothing ever arrives at.
// The wait gives up after the requested time, raises the abort flag, records
// the timeout bit in a status word and the kernel returns normally, so the
// context stays usable; the host reads the word and reports BF_ERR_TIMEOUT.
// This is how a stalled pipeline (a lost TMA completion, a peer that never
// signals) surfaces, tested without faulting or hanging the GPU.
#include "bf_internal.h"
#include "ptx.cuh"

namespace bfi {

__global__ void k_wait_selftest(unsigned *err, unsigned long long limit_cycles)
{
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // phase 0 never completes: no thread arrives
        if (mbar_wait(smem_u32(&bar), 0, &abort_flag, err, limit_cycles)) atomicOr(err, 0x80000000u);
    }
    __syncthreads();
}

}  // namespace bfi

using namespace bfi;

extern "C" bf_status bf_selftest_timeout(double limit_ms, void *stream)
{
    clear_error();
    if (!(limit_ms > 0.0) || limit_ms > 10000.0) return set_error(BF_ERR_ARG, "limit_ms must be in (0, 10000]");
    int dev = 0, khz = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
    if (e != cudaSuccess) return cuda_error(e, "device query");
    unsigned *d_err = nullptr;
    if ((e = cudaMalloc((void **)&d_err, sizeof(unsigned))) != cudaSuccess) return cuda_error(e, "status word");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned h = 0;
    const unsigned long long cycles = (unsigned long long)(limit_ms * (double)khz);
    if ((e = cudaMemsetAsync(d_err, 0, sizeof(unsigned), s)) == cudaSuccess) {
        k_wait_selftest<<<1, 32, 0, s>>>(d_err, cycles);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_err);
    if (e != cudaSuccess) return cuda_error(e, "self-test kernel");
    if (h & 0x80000000u) return set_error(BF_ERR_CUDA, "the unsignalled barrier completed (unexpected)");
    if (h & kErrTimeout) return set_error(BF_ERR_TIMEOUT, "bounded wait gave up as expected");
    return set_error(BF_ERR_CUDA, "bounded wait returned without recording a timeout");
}
