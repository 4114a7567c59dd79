// Diagnostics.  bf_selftest_timeout exercises the bounded device-side wait that every pipelined
// kernel of the library uses, on an mbarrier that nothing ever arrives at.
// The wait gives up after the requested time, raises the abort flag, records
// the timeout bit in a status word and the kernel returns normally, so the
// context stays usable; the host reads the word and reports BF_ERR_TIMEOUT.
// This is how a stalled pipeline (a lost TMA completion, a peer that never
// signals) surfaces, tested without faulting or hanging the GPU.
#include <algorithm>

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

// FP32 FFMA throughput probe: every thread runs 8 independent chains of
// a = a * b + c (2 FLOP each), 128 per chain per loop trip; the sums are
// stored so the arithmetic is not removed.  b < 1 keeps the values bounded.
__global__ void __launch_bounds__(256) k_ffma_probe(float *out, int trips, float b, float c)
{
    float a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = 1e-3f * (float)threadIdx.x + (float)i;
    for (int k = 0; k < trips; ++k) {
#pragma unroll
        for (int u = 0; u < 128; ++u)
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = fmaf(a[i], b, c);
    }
    float sum = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) sum += a[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = sum;
}

}  // namespace bfi

using namespace bfi;

extern "C" bf_status bf_measure_ffma(double seconds, double *tflops, void *stream)
{
    clear_error();
    if (!tflops) return set_error(BF_ERR_ARG, "tflops is NULL");
    if (!(seconds > 0.0) || seconds > 60.0) return set_error(BF_ERR_ARG, "seconds must be in (0, 60]");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_error(e, "device query");
    const int grid = sms * 8, threads = 256;   // 64 warps per SM: every sub-partition saturated
    float *d_out = nullptr;
    if ((e = cudaMalloc((void **)&d_out, sizeof(float) * grid * threads)) != cudaSuccess)
        return cuda_error(e, "probe output");
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto run = [&](int trips, float *ms) -> cudaError_t {
        cudaEventRecord(e0, s);
        k_ffma_probe<<<grid, threads, 0, s>>>(d_out, trips, 0.999999f, 1e-6f);
        cudaEventRecord(e1, s);
        cudaError_t r = cudaEventSynchronize(e1);
        if (r == cudaSuccess) r = cudaGetLastError();
        if (r == cudaSuccess) r = cudaEventElapsedTime(ms, e0, e1);
        return r;
    };
    float ms = 0.f;
    int trips = 64;
    e = run(trips, &ms);   // warm-up and calibration
    if (e == cudaSuccess) {
        trips = (int)std::min(2.0e9, std::max(64.0, trips * seconds * 1e3 / std::max(ms, 1e-3f)));
        e = run(trips, &ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d_out);
    if (e != cudaSuccess) return cuda_error(e, "FFMA probe");
    const double flop = 2.0 * 8 * 128 * (double)trips * grid * threads;
    *tflops = flop / (ms * 1e-3) / 1e12;
    return BF_OK;
}

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
