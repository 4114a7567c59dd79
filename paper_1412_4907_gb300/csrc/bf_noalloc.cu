// bf_execute_nct_static: the antenna-major execute path (corner turn, then
// the tensor-core beamformer) with its scratch in a fixed device array
// instead of memory the plan allocates.
//
// Some callers cannot allocate device memory at the time they execute: code
// running under an allocator that forbids cudaMalloc outside set-up, real-time
// loops where an allocation (and the device-wide synchronisation that freeing
// the old buffer needs) would break the latency budget, or processes whose
// memory is budgeted up front.  This entry point serves them: it calls no
// cudaMalloc, cudaFree or other allocating routine.  The scratch is a
// file-scope __device__ array of kStaticScratchBytes bytes; every GPU that
// loads the library holds it until the process exits.
#include <cudaTypedefs.h>

#include <mutex>

#include "batch.h"
#include "bf_internal.h"

namespace bfi {

constexpr size_t kStaticScratchBytes = 64ull << 20;   // 64 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch per device, with the ID of the context
// it was looked up in: after cudaDeviceReset the device gets a new primary
// context (a new ID) and the address is looked up again.
struct ScratchSlot {
    unsigned long long ctx_id;
    void *addr;
};
static ScratchSlot g_scratch[kMaxDevices];
static std::mutex g_scratch_mutex;

// ID of the calling thread's current context (driver entry points fetched once).
static cudaError_t current_context_id(unsigned long long *id)
{
    static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(f);
    });
    if (!get_current || !get_id) return cudaErrorNotSupported;
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorDeviceUninitialized;
    return get_id(ctx, id) == CUDA_SUCCESS ? cudaSuccess : cudaErrorDeviceUninitialized;
}

// The array's device address on the current device (looked up on the first
// call per device and context, with that device current).
static cudaError_t static_scratch(int device, void **out)
{
    unsigned long long id = 0;
    cudaError_t e = cudaSetDevice(device);   // makes the device's primary context current on this thread
    if (e != cudaSuccess) return e;
    if ((e = current_context_id(&id)) != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    ScratchSlot &slot = g_scratch[device];
    if (!slot.addr || slot.ctx_id != id) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess) return e;
        slot.addr = ptr;
        slot.ctx_id = id;
    }
    *out = slot.addr;
    return cudaSuccess;
}

}  // namespace bfi

using namespace bfi;

extern "C" bf_status bf_execute_nct_static(bf_plan *p, const void *x, int T, float *out, void *stream)
{
    clear_error();
    if (!p) return set_error(BF_ERR_ARG, "plan is NULL");
    if (p->layout != BF_LAYOUT_NCT || p->wf.simt)
        return set_error(BF_ERR_UNSUPPORTED, "bf_execute_nct_static runs antenna-major tensor-core plans");
    if (T < 0) return set_error(BF_ERR_ARG, "n_samp must be >= 0");
    if (T / p->t_int == 0) return BF_OK;
    if (!x || !out) return set_error(BF_ERR_ARG, "NULL voltage or output pointer");
    if (((uintptr_t)x & 15) || ((uintptr_t)out & 3))
        return set_error(BF_ERR_ARG, "voltages must be 16-byte aligned and outputs 4-byte aligned");
    const size_t n_samp = (size_t)p->C * T * p->N;
    const size_t turned = (n_samp * dtype_sample_bytes(p->dtype) + 255) / 256 * 256;
    // 8/4-bit inputs: the resident-weight kernel widens them itself; the
    // streamed pipeline reads an FP16 widening from the scratch
    const bool expand = (p->dtype == BF_CI8 || p->dtype == BF_CI4) && p->tc.raw_kb == 0;
    const size_t need = turned + (expand ? n_samp * 4 : 0);
    if (need > kStaticScratchBytes)
        return set_error(BF_ERR_ARG, "input needs " + std::to_string(need) + " bytes of scratch; the static scratch holds " +
                                         std::to_string(kStaticScratchBytes) + " (use bf_execute, or fewer samples)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return set_error(BF_ERR_UNSUPPORTED, "device index out of range");
    void *scr = nullptr;
    if ((e = static_scratch(dev, &scr)) != cudaSuccess) return cuda_error(e, "static scratch address");
    cudaStream_t s = stream ? (cudaStream_t)stream : p->stream;
    if (p->wbufs == 2) {   // stream-ordered after the latest weight refresh
        e = cudaStreamWaitEvent(s, p->ev_wready, 0);
        if (e != cudaSuccess) return cuda_error(e, "weight ordering");
    }
    uint8_t *base = (uint8_t *)scr;
    e = launch_corner_turn(x, p->dtype, base, p->dtype, p->N, p->C, T, nullptr, s);
    if (e != cudaSuccess) return cuda_error(e, "corner turn");
    const void *xin = base;
    if (expand) {
        e = launch_expand_to_f16(base, p->dtype, base + turned, (long long)n_samp, p->N, s);
        if (e != cudaSuccess) return cuda_error(e, "integer expansion");
        xin = base + turned;
    }
    if (p->tc.stream) {
        // weights too large to stay resident: the batched kernel's streamed
        // pipeline with one job, as bf_execute runs it (the launch set-up is
        // host arithmetic on a core kept on the stack)
        BatchCore core;
        bf_plan *const one[1] = {p};
        bf_status st = batch_core_init(&core, one, 1, p->tc.nt);
        if (st != BF_OK) return st;
        BatchJob J;
        st = batch_fill_job(core, &J, p, xin, T, out, 0, nullptr, nullptr);
        if (st != BF_OK) return st;
        e = batch_core_launch_one(core, J, p->d_err, s);
        if (e != cudaSuccess) return cuda_error(e, "tensor-core kernel (streamed)");
    } else {
        TcArgs ta;
        ta.x = xin;
        ta.c_base = 0;
        ta.c_launch = p->C;
        ta.c_total = p->C;
        ta.T = T;
        ta.T_o = T / p->t_int;
        ta.t_int = p->t_int;
        ta.complex_out = 0;
        ta.out = out;
        std::string why;
        e = launch_tc(p, ta, s, &why);
        if (e != cudaSuccess) {
            if (!why.empty()) return set_error(BF_ERR_CUDA, "tensor-core kernel: " + why);
            return cuda_error(e, "tensor-core kernel");
        }
    }
    if (p->wbufs == 2 && (e = cudaEventRecord(p->ev_wused[p->wcur], s)) != cudaSuccess)
        return cuda_error(e, "weight event");
    return BF_OK;
}
