// Host side of the C ABI in include/bf.h: plan validation and ownership,
// weight-format choice, kernel dispatch, the pipelined host-memory execute
// (copies overlapped with kernels on separate streams, Section 2.2), and
// status reporting.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "batch.h"
#include "bf_internal.h"

namespace bfi {

static thread_local std::string g_last_error;

bf_status set_error(bf_status s, const std::string &msg)
{
    g_last_error = msg;
    return s;
}

void clear_error() { g_last_error.clear(); }

bf_status cuda_error(cudaError_t e, const char *what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? BF_ERR_NOMEM : BF_ERR_CUDA;
}

}  // namespace bfi

using namespace bfi;

#define BF_CUDA(call, what)                                \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_error(e_, what); \
    } while (0)

static bool valid_dtype(int d) { return d >= BF_C32 && d <= BF_CI4; }

static bf_status check_dirs(const double *dirs, int B)
{
    for (int b = 0; b < B; ++b) {
        const double *s = dirs + 3 * b;
        if (!std::isfinite(s[0]) || !std::isfinite(s[1]) || !std::isfinite(s[2]))
            return set_error(BF_ERR_ARG, "direction " + std::to_string(b) + " is not finite");
        double n2 = s[0] * s[0] + s[1] * s[1] + s[2] * s[2];
        if (std::fabs(n2 - 1.0) > 2e-6)
            return set_error(BF_ERR_ARG, "direction " + std::to_string(b) + " is not a unit vector");
    }
    return BF_OK;
}

static void plan_free(bf_plan *p)
{
    if (!p) return;
    if (p->stream) cudaStreamSynchronize(p->stream);
    if (p->stream2) cudaStreamSynchronize(p->stream2);
    if (p->stream3) cudaStreamSynchronize(p->stream3);
    if (p->wstream) cudaStreamSynchronize(p->wstream);
    if (p->wbufs == 2) {   // the buffers that are not the current ones
        const int o = 1 - p->wcur;
        if (p->wbuf[o]) cudaFree(p->wbuf[o]);
        if (p->wscale_buf[o]) cudaFree(p->wscale_buf[o]);
        if (p->wsig_buf[o]) cudaFree(p->wsig_buf[o]);
    }
    for (cudaEvent_t ev : {p->ev_wready, p->ev_wused[0], p->ev_wused[1]})
        if (ev) cudaEventDestroy(ev);
    if (p->wstream) cudaStreamDestroy(p->wstream);
    void *ptrs[] = {p->d_pos, p->d_freqs, p->d_dirs, p->d_mask, p->d_tau, p->d_ab, p->d_w, p->d_wscale,
                    p->d_wsig, p->d_scratch, p->d_hx, p->d_hp, p->d_err};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    for (int i = 0; i < bf_plan::kEvents; ++i)
        if (p->ev[i]) cudaEventDestroy(p->ev[i]);
    if (p->stream2) cudaStreamDestroy(p->stream2);
    if (p->stream3) cudaStreamDestroy(p->stream3);
    delete p->bcore;
    delete p;
}

static bf_status upload_geometry(bf_plan *p)
{
    // antenna n of the array sits in input slot perm[n]; the weight of slot m
    // is the weight of the antenna it holds (the reorder lookup of Section 3,
    // applied to the weights so the voltages need no gather)
    std::vector<double> pos(3 * (size_t)p->N);
    std::vector<uint8_t> mask((size_t)p->N, 1);
    for (int n = 0; n < p->N; ++n) {
        int m = p->perm.empty() ? n : p->perm[n];
        for (int k = 0; k < 3; ++k) pos[3 * (size_t)m + k] = p->pos[3 * (size_t)n + k];
        mask[m] = p->mask.empty() ? 1 : p->mask[n];
    }
    BF_CUDA(cudaMemcpy(p->d_pos, pos.data(), pos.size() * sizeof(double), cudaMemcpyHostToDevice), "copy positions");
    BF_CUDA(cudaMemcpy(p->d_mask, mask.data(), mask.size(), cudaMemcpyHostToDevice), "copy mask");
    return BF_OK;
}

static bf_status regenerate(bf_plan *p)
{
    if (p->wbufs == 2) {
        // fill the other buffer on the weight stream once the last execute that
        // read it is done, then make it current; executes wait for ev_wready
        const int back = 1 - p->wcur;
        BF_CUDA(cudaStreamWaitEvent(p->wstream, p->ev_wused[back], 0), "weight stream ordering");
        p->wcur = back;
        p->d_w = p->wbuf[back];
        p->d_wscale = p->wscale_buf[back];
        p->d_wsig = p->wsig_buf[back];
        BF_CUDA(launch_delays(p, p->wstream), "delay kernel");
        BF_CUDA(launch_weights(p, p->wstream), "weight kernel");
        BF_CUDA(cudaEventRecord(p->ev_wready, p->wstream), "weight event");
        return BF_OK;
    }
    BF_CUDA(launch_delays(p, p->stream), "delay kernel");
    BF_CUDA(launch_weights(p, p->stream), "weight kernel");
    return BF_OK;
}

// Stream-order an execute on s after the latest weight refresh, and (after
// its launches) mark the current buffer as read by s.
static bf_status weights_acquire(bf_plan *p, cudaStream_t s)
{
    if (p->wbufs == 2) BF_CUDA(cudaStreamWaitEvent(s, p->ev_wready, 0), "weight ordering");
    return BF_OK;
}
static bf_status weights_release(bf_plan *p, cudaStream_t s)
{
    if (p->wbufs == 2) BF_CUDA(cudaEventRecord(p->ev_wused[p->wcur], s), "weight event");
    return BF_OK;
}

static bool choose_format(bf_plan *p, std::string *why)
{
    WeightFormat &f = p->wf;
    f = WeightFormat();
    f.b_pad = (p->B + kBeamsPerMTile - 1) / kBeamsPerMTile * kBeamsPerMTile;
    if (p->dtype == BF_C32) {
        f.simt = true;
        f.es = 8;
        return true;
    }
    switch (p->dtype) {
    case BF_C16F: f.op = kOpF16; break;
    case BF_C16BF: f.op = kOpBF16; break;
    case BF_C8E4M3: f.op = kOpE4M3; f.qmax = 448.f; break;
    case BF_CI8: f.op = kOpF16; f.qmax = 127.f; break;
    default: f.op = kOpF16; break;   // BF_CI4: FP16 weights, unscaled
    }
    f.es = f.op == kOpE4M3 ? 1 : 2;
    f.ke = kKBlockBytes / f.es;
    f.kb = (2 * p->N + f.ke - 1) / f.ke;
    f.k_pad = f.kb * f.ke;
    f.m_pad = f.b_pad / kBeamsPerMTile * kRowsPerMTile;
    if ((2 * p->N * f.es) % 16 != 0) {
        *why = "tensor-core modes need 2*N*bytes_per_element to be a multiple of 16 (N % 4 == 0 for "
               "16-bit and integer modes, N % 8 == 0 for FP8)";
        return false;
    }
    return tc_choose(p, p->tc_req, &p->tc, why);
}

extern "C" {

const char *bf_last_error(void) { return g_last_error.c_str(); }

bf_status bf_plan_create(bf_plan **out, int n_ant, const double *pos_m, const uint8_t *mask, int n_chan,
                         const double *freqs_hz, int n_beam, const double *dirs, int dtype, int t_int,
                         int layout, void *stream)
{
    g_last_error.clear();
    if (!out) return set_error(BF_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!pos_m || !freqs_hz || !dirs) return set_error(BF_ERR_ARG, "NULL geometry, frequency or direction array");
    if (n_ant < 1 || n_chan < 1 || n_beam < 1 || t_int < 1)
        return set_error(BF_ERR_ARG, "n_ant, n_chan, n_beam and t_int must be >= 1");
    if (!valid_dtype(dtype)) return set_error(BF_ERR_ARG, "unknown dtype");
    if (layout != BF_LAYOUT_CTN && layout != BF_LAYOUT_NCT) return set_error(BF_ERR_ARG, "unknown layout");
    for (int i = 0; i < 3 * n_ant; ++i)
        if (!std::isfinite(pos_m[i])) return set_error(BF_ERR_ARG, "non-finite antenna position");
    for (int c = 0; c < n_chan; ++c)
        if (!std::isfinite(freqs_hz[c]) || freqs_hz[c] <= 0.0)
            return set_error(BF_ERR_ARG, "channel frequencies must be finite and > 0");
    bf_status st = check_dirs(dirs, n_beam);
    if (st != BF_OK) return st;

    bf_plan *p = new bf_plan();
    p->N = n_ant;
    p->C = n_chan;
    p->B = n_beam;
    p->dtype = dtype;
    p->t_int = t_int;
    p->layout = layout;
    p->stream = (cudaStream_t)stream;
    p->pos.assign(pos_m, pos_m + 3 * (size_t)n_ant);
    p->freqs.assign(freqs_hz, freqs_hz + n_chan);
    p->dirs.assign(dirs, dirs + 3 * (size_t)n_beam);
    if (mask) p->mask.assign(mask, mask + n_ant);
    p->kernel = dtype == BF_C32 ? BF_KERNEL_SIMT : BF_KERNEL_TC;
    // uniformly spaced channels use the exact fixed-point phase recurrence
    p->f0 = freqs_hz[0];
    p->df = n_chan > 1 ? (freqs_hz[n_chan - 1] - freqs_hz[0]) / (n_chan - 1) : 0.0;
    p->uniform_freqs = true;
    for (int c = 0; c < n_chan; ++c)
        if (std::fabs(freqs_hz[c] - (p->f0 + c * p->df)) > 1e-6) p->uniform_freqs = false;

    std::string why;
    if (!choose_format(p, &why)) {
        plan_free(p);
        return set_error(BF_ERR_UNSUPPORTED, why);
    }
    cudaError_t e;
    if ((e = cudaGetDevice(&p->device)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device)) != cudaSuccess) {
        plan_free(p);
        return cuda_error(e, "device query");
    }
    const WeightFormat &f = p->wf;
    if (f.simt) p->w_bytes = (size_t)p->C * f.b_pad * p->N * 8;
    else p->w_bytes = (size_t)p->C * f.m_pad * f.k_pad * f.es;
    struct Alloc {
        void **ptr;
        size_t bytes;
    } allocs[] = {
        {(void **)&p->d_pos, 3 * (size_t)p->N * sizeof(double)},
        {(void **)&p->d_freqs, (size_t)p->C * sizeof(double)},
        {(void **)&p->d_dirs, 3 * (size_t)p->B * sizeof(double)},
        {(void **)&p->d_mask, (size_t)p->N},
        {(void **)&p->d_tau, (size_t)p->N * p->B * sizeof(double)},
        {(void **)&p->d_ab, (size_t)p->N * p->B * 2 * sizeof(unsigned long long)},
        {(void **)&p->d_w, p->w_bytes},
        {(void **)&p->d_wscale, (size_t)p->C * f.b_pad * sizeof(float)},
        {(void **)&p->d_wsig, (size_t)p->C * f.b_pad * sizeof(float)},
        {(void **)&p->d_err, sizeof(unsigned)},
    };
    for (auto &a : allocs) {
        if ((e = cudaMalloc(a.ptr, a.bytes)) != cudaSuccess) {
            plan_free(p);
            return cuda_error(e, "plan allocation");
        }
        p->dev_bytes += a.bytes;
    }
    if ((e = cudaMemset(p->d_err, 0, sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMemcpy(p->d_freqs, freqs_hz, p->C * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(p->d_dirs, dirs, 3 * (size_t)p->B * sizeof(double), cudaMemcpyHostToDevice)) !=
            cudaSuccess) {
        plan_free(p);
        return cuda_error(e, "plan upload");
    }
    for (int i = 0; i < bf_plan::kEvents; ++i)
        if ((e = cudaEventCreateWithFlags(&p->ev[i], cudaEventDisableTiming)) != cudaSuccess) {
            plan_free(p);
            return cuda_error(e, "event creation");
        }
    if ((e = cudaStreamCreateWithFlags(&p->stream2, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&p->stream3, cudaStreamNonBlocking)) != cudaSuccess) {
        plan_free(p);
        return cuda_error(e, "stream creation");
    }
    if ((st = upload_geometry(p)) != BF_OK || (st = regenerate(p)) != BF_OK) {
        std::string msg = g_last_error;
        plan_free(p);
        return set_error(st, msg);
    }
    *out = p;
    return BF_OK;
}

bf_status bf_weights(bf_plan *p, const double *dirs)
{
    g_last_error.clear();
    if (!p) return set_error(BF_ERR_ARG, "plan is NULL");
    if (dirs) {
        bf_status st = check_dirs(dirs, p->B);
        if (st != BF_OK) return st;
        p->dirs.assign(dirs, dirs + 3 * (size_t)p->B);
        BF_CUDA(cudaMemcpyAsync(p->d_dirs, p->dirs.data(), 3 * (size_t)p->B * sizeof(double),
                                cudaMemcpyHostToDevice, p->wbufs == 2 ? p->wstream : p->stream),
                "copy directions");
    }
    return regenerate(p);
}

bf_status bf_plan_set_input_order(bf_plan *p, const int *perm)
{
    g_last_error.clear();
    if (!p) return set_error(BF_ERR_ARG, "plan is NULL");
    if (!perm) {
        p->perm.clear();
    } else {
        std::vector<char> seen((size_t)p->N, 0);
        for (int n = 0; n < p->N; ++n) {
            if (perm[n] < 0 || perm[n] >= p->N || seen[perm[n]])
                return set_error(BF_ERR_ARG, "perm is not a permutation of 0..N-1");
            seen[perm[n]] = 1;
        }
        p->perm.assign(perm, perm + p->N);
    }
    BF_CUDA(cudaStreamSynchronize(p->stream), "sync before geometry upload");
    bf_status st = upload_geometry(p);
    if (st != BF_OK) return st;
    return regenerate(p);
}

static bf_status ensure(void **ptr, size_t *have, size_t need, bf_plan *p, const char *what)
{
    if (*have >= need) return BF_OK;
    cudaDeviceSynchronize();   // nothing of this plan may still use the old buffer
    if (*ptr) {
        cudaFree(*ptr);
        p->dev_bytes -= *have;
        *ptr = nullptr;
        *have = 0;
    }
    cudaError_t e = cudaMalloc(ptr, need);
    if (e != cudaSuccess) return cuda_error(e, what);
    *have = need;
    p->dev_bytes += need;
    return BF_OK;
}

// Run the beamformer on channels [c_base, c_base + c_launch) whose voltages
// start at x (CTN) or on all channels (NCT, c_base = 0).
static bf_status run_range_body(bf_plan *p, const void *x, int c_base, int c_launch, int T, float *out, int mode,
                                cudaStream_t s)
{
    const int T_o = T / p->t_int;
    if (mode == 2) {   // incoherent
        // an all-ones mask is passed as none (the kernel's unmasked paths are faster)
        const bool masked = std::find(p->mask.begin(), p->mask.end(), (uint8_t)0) != p->mask.end();
        BF_CUDA(launch_incoherent(x, p->dtype, p->layout, masked ? p->d_mask : nullptr, p->N, c_launch, T, p->t_int,
                                  out + (size_t)c_base * T_o, s),
                "incoherent kernel");
        return BF_OK;
    }
    if (p->wf.simt) {
        BF_CUDA(launch_simt_range(p, x, c_base, c_launch, T, out, mode, s), "FP32 beamformer kernel");
        return BF_OK;
    }
    const size_t sb = dtype_sample_bytes(p->dtype);
    const size_t n_samp = (size_t)c_launch * T * p->N;
    const void *xin = x;
    size_t need = 0;
    const bool ct = p->layout == BF_LAYOUT_NCT;
    // 8/4-bit inputs: the resident-weight kernel widens them itself (each
    // voltage tile serves a group of M tiles) when TMA can read their rows;
    // the streamed pipeline uses a voltage block for one M tile, so it (and
    // rows TMA cannot read) take an FP16 widening from scratch
    const bool expand = (p->dtype == BF_CI8 || p->dtype == BF_CI4) && p->tc.raw_kb == 0;
    if (ct) need += (n_samp * sb + 255) / 256 * 256;
    if (expand) need += n_samp * 4;
    if (need) {
        bf_status st = ensure(&p->d_scratch, &p->scratch_bytes, need, p, "scratch allocation");
        if (st != BF_OK) return st;
    }
    uint8_t *scr = (uint8_t *)p->d_scratch;
    if (ct) {
        BF_CUDA(launch_corner_turn(x, p->dtype, scr, p->dtype, p->N, c_launch, T, nullptr, s), "corner turn");
        xin = scr;
        scr += (n_samp * sb + 255) / 256 * 256;
    }
    if (expand) {
        BF_CUDA(launch_expand_to_f16(xin, p->dtype, scr, (long long)n_samp, p->N, s), "integer expansion");
        xin = scr;
    }
    if (p->tc.stream) {
        // large antenna counts: the batched kernel's streamed pipeline with one
        // job (its CTAs walk neighbouring tiles of one channel together, so the
        // weight and voltage tiles are shared in L2), for powers and for
        // complex beams
        if (!p->bcore) {
            BatchCore core;
            bf_plan *const one[1] = {p};
            bf_status st = batch_core_init(&core, one, 1, p->tc.nt);
            if (st != BF_OK) return st;
            p->bcore = new BatchCore(core);
        }
        BatchCore core = *p->bcore;
        core.cpx = mode == 1;
        BatchJob J;
        bf_status st = batch_fill_job(core, &J, p, xin, T, out, 0, nullptr, nullptr, c_base, c_launch);
        if (st != BF_OK) return st;
        BF_CUDA(batch_core_launch_one(core, J, p->d_err, s), "tensor-core kernel (streamed)");
        return BF_OK;
    }
    TcArgs ta;
    ta.x = xin;
    ta.c_base = c_base;
    ta.c_launch = c_launch;
    ta.c_total = p->C;
    ta.T = T;
    ta.T_o = T_o;
    ta.t_int = p->t_int;
    ta.complex_out = mode;
    ta.out = out;
    std::string why;
    cudaError_t e = launch_tc(p, ta, s, &why);
    if (e != cudaSuccess) {
        if (!why.empty()) return set_error(BF_ERR_CUDA, "tensor-core kernel: " + why);
        return cuda_error(e, "tensor-core kernel");
    }
    return BF_OK;
}

// One launch range with the weight ordering of double-buffered plans.
static bf_status run_range(bf_plan *p, const void *x, int c_base, int c_launch, int T, float *out, int mode,
                           cudaStream_t s)
{
    if (mode == 2) return run_range_body(p, x, c_base, c_launch, T, out, mode, s);   // no weights
    bf_status st = weights_acquire(p, s);
    if (st == BF_OK) st = run_range_body(p, x, c_base, c_launch, T, out, mode, s);
    if (st == BF_OK) st = weights_release(p, s);
    return st;
}

// Returns BF_OK with *noop set when the call has nothing to compute.
static bf_status exec_checks(bf_plan *p, const void *x, int T, const void *out, int mode, bool *noop)
{
    *noop = false;
    if (!p) return set_error(BF_ERR_ARG, "plan is NULL");
    if (T < 0) return set_error(BF_ERR_ARG, "n_samp must be >= 0");
    if (T == 0 || (mode != 1 && T / p->t_int == 0)) {
        *noop = true;   // no sample or no complete window: pointers are not used
        return BF_OK;
    }
    if (!x || !out) return set_error(BF_ERR_ARG, "NULL voltage or output pointer");
    if (T < 0) return set_error(BF_ERR_ARG, "n_samp must be >= 0");
    if (((uintptr_t)x & 15) || ((uintptr_t)out & 3))
        return set_error(BF_ERR_ARG, "voltages must be 16-byte aligned and outputs 4-byte aligned");
    return BF_OK;
}

bf_status bf_execute(bf_plan *p, const void *x, int T, float *out, void *stream)
{
    g_last_error.clear();
    bool noop;
    bf_status st = exec_checks(p, x, T, out, 0, &noop);
    if (st != BF_OK || noop) return st;
    return run_range(p, x, 0, p->C, T, out, 0, stream ? (cudaStream_t)stream : p->stream);
}

bf_status bf_execute_complex(bf_plan *p, const void *x, int T, float *out, void *stream)
{
    g_last_error.clear();
    bool noop;
    bf_status st = exec_checks(p, x, T, out, 1, &noop);
    if (st != BF_OK || noop) return st;
    if ((uintptr_t)out & 7) return set_error(BF_ERR_ARG, "complex beams must be 8-byte aligned (float pairs)");
    return run_range(p, x, 0, p->C, T, out, 1, stream ? (cudaStream_t)stream : p->stream);
}

bf_status bf_execute_incoherent(bf_plan *p, const void *x, int T, float *out, void *stream)
{
    g_last_error.clear();
    bool noop;
    bf_status st = exec_checks(p, x, T, out, 2, &noop);
    if (st != BF_OK || noop) return st;
    return run_range(p, x, 0, p->C, T, out, 2, stream ? (cudaStream_t)stream : p->stream);
}

bf_status bf_execute_host(bf_plan *p, const void *hx, int T, float *hp)
{
    g_last_error.clear();
    if (!p) return set_error(BF_ERR_ARG, "plan is NULL");
    if (T < 0) return set_error(BF_ERR_ARG, "n_samp must be >= 0");
    if (T / p->t_int == 0) return BF_OK;
    if (!hx || !hp) return set_error(BF_ERR_ARG, "NULL host pointer");
    if (p->layout != BF_LAYOUT_CTN) return set_error(BF_ERR_UNSUPPORTED, "host execute needs the CTN layout");
    const int T_o = T / p->t_int;
    const size_t row = (size_t)T * p->N * dtype_sample_bytes(p->dtype);   // bytes per channel
    const size_t in_bytes = row * p->C;
    const size_t out_bytes = (size_t)p->B * p->C * T_o * sizeof(float);
    bf_status st = ensure(&p->d_hx, &p->hx_bytes, std::max<size_t>(in_bytes, 16), p, "host staging");
    if (st != BF_OK) return st;
    st = ensure((void **)&p->d_hp, &p->hp_bytes, std::max<size_t>(out_bytes, 16), p, "host staging");
    if (st != BF_OK) return st;
    // channel blocks: copy-in of block k+1 and copy-out of block k-1 overlap the kernel of block k
    const int n_blk = std::min(p->C, bf_plan::kEvents / 2);
    const int cb = (p->C + n_blk - 1) / n_blk;
    cudaStream_t s = p->stream;
    for (int k = 0, c0 = 0; c0 < p->C; ++k, c0 += cb) {
        const int cn = std::min(cb, p->C - c0);
        cudaEvent_t ev_in = p->ev[2 * k], ev_run = p->ev[2 * k + 1];
        BF_CUDA(cudaMemcpyAsync((uint8_t *)p->d_hx + c0 * row, (const uint8_t *)hx + c0 * row, cn * row,
                                cudaMemcpyHostToDevice, p->stream2),
                "copy voltages in");
        BF_CUDA(cudaEventRecord(ev_in, p->stream2), "event");
        BF_CUDA(cudaStreamWaitEvent(s, ev_in, 0), "event wait");
        st = run_range(p, (const uint8_t *)p->d_hx + c0 * row, c0, cn, T, p->d_hp, 0, s);
        if (st != BF_OK) return st;
        BF_CUDA(cudaEventRecord(ev_run, s), "event");
        BF_CUDA(cudaStreamWaitEvent(p->stream3, ev_run, 0), "event wait");
        if (T_o > 0)
            BF_CUDA(cudaMemcpy2DAsync(hp + (size_t)c0 * T_o, (size_t)p->C * T_o * sizeof(float),
                                      p->d_hp + (size_t)c0 * T_o, (size_t)p->C * T_o * sizeof(float),
                                      (size_t)cn * T_o * sizeof(float), p->B, cudaMemcpyDeviceToHost, p->stream3),
                    "copy powers out");
    }
    BF_CUDA(cudaStreamSynchronize(p->stream3), "host execute");
    BF_CUDA(cudaStreamSynchronize(s), "host execute");
    return BF_OK;
}

bf_status bf_sync(bf_plan *p)
{
    g_last_error.clear();
    if (!p) return set_error(BF_ERR_ARG, "plan is NULL");
    BF_CUDA(cudaStreamSynchronize(p->stream), "stream synchronize");
    BF_CUDA(cudaStreamSynchronize(p->stream2), "stream synchronize");
    BF_CUDA(cudaStreamSynchronize(p->stream3), "stream synchronize");
    if (p->wstream) BF_CUDA(cudaStreamSynchronize(p->wstream), "stream synchronize");
    unsigned err = 0;
    BF_CUDA(cudaMemcpy(&err, p->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost), "read status word");
    if (err) {
        BF_CUDA(cudaMemset(p->d_err, 0, sizeof(unsigned)), "clear status word");
        return set_error(BF_ERR_TIMEOUT, "a device-side wait timed out; results of the affected calls are invalid");
    }
    return BF_OK;
}

bf_status bf_destroy(bf_plan *p)
{
    g_last_error.clear();
    plan_free(p);
    return BF_OK;
}

bf_status bf_plan_set_kernel(bf_plan *p, int kernel, int tile_t)
{
    g_last_error.clear();
    if (!p) return set_error(BF_ERR_ARG, "plan is NULL");
    if (kernel < BF_KERNEL_AUTO || kernel > BF_KERNEL_TC) return set_error(BF_ERR_ARG, "unknown kernel");
    if (kernel == BF_KERNEL_SIMT && p->dtype != BF_C32)
        return set_error(BF_ERR_UNSUPPORTED, "the SIMT kernel runs only BF_C32");
    if (kernel == BF_KERNEL_TC && p->dtype == BF_C32)
        return set_error(BF_ERR_UNSUPPORTED, "the tensor-core kernel does not run BF_C32");
    return bf_plan_set_tiles(p, tile_t, p->tc_req.group_tiles, p->tc_req.x_stages);
}

bf_status bf_plan_set_tiles(bf_plan *p, int tile_t, int group_tiles, int x_stages)
{
    g_last_error.clear();
    if (!p) return set_error(BF_ERR_ARG, "plan is NULL");
    if (tile_t < 0 || group_tiles < 0 || group_tiles > 16 || x_stages < 0 || x_stages == 1 || x_stages > 4)
        return set_error(BF_ERR_ARG, "tile_t >= 0, 0 <= group_tiles <= 16, x_stages in {0, 2, 3, 4}");
    if (p->wf.simt) return BF_OK;   // the SIMT kernel has a fixed tiling
    TcRequest req;
    req.tile_t = tile_t;
    req.group_tiles = group_tiles;
    req.x_stages = x_stages;
    TcConfig cfg;
    std::string why;
    if (!tc_choose(p, req, &cfg, &why)) return set_error(BF_ERR_UNSUPPORTED, why);
    p->tc = cfg;
    p->tc_req = req;
    delete p->bcore;   // re-derived from the new tiling on the next streamed launch
    p->bcore = nullptr;
    return BF_OK;
}

bf_status bf_plan_set_weight_buffers(bf_plan *p, int n)
{
    g_last_error.clear();
    if (!p) return set_error(BF_ERR_ARG, "plan is NULL");
    if (n != 1 && n != 2) return set_error(BF_ERR_ARG, "weight buffers must be 1 or 2");
    if (n == p->wbufs) return BF_OK;
    BF_CUDA(cudaStreamSynchronize(p->stream), "stream synchronize");
    if (p->wstream) BF_CUDA(cudaStreamSynchronize(p->wstream), "stream synchronize");
    const size_t sb = (size_t)p->C * p->wf.b_pad * sizeof(float);
    if (n == 2) {
        void *w = nullptr;
        float *sc = nullptr, *sg = nullptr;
        cudaError_t e = cudaMalloc(&w, p->w_bytes);
        if (e == cudaSuccess) e = cudaMalloc((void **)&sc, sb);
        if (e == cudaSuccess) e = cudaMalloc((void **)&sg, sb);
        if (e == cudaSuccess && !p->wstream) e = cudaStreamCreateWithFlags(&p->wstream, cudaStreamNonBlocking);
        for (cudaEvent_t *ev : {&p->ev_wready, &p->ev_wused[0], &p->ev_wused[1]})
            if (e == cudaSuccess && !*ev) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            if (w) cudaFree(w);
            if (sc) cudaFree(sc);
            if (sg) cudaFree(sg);
            return cuda_error(e, "second weight buffer");
        }
        p->wbuf[0] = p->d_w;
        p->wscale_buf[0] = p->d_wscale;
        p->wsig_buf[0] = p->d_wsig;
        p->wbuf[1] = w;
        p->wscale_buf[1] = sc;
        p->wsig_buf[1] = sg;
        p->wcur = 0;
        p->wbufs = 2;
        p->dev_bytes += p->w_bytes + 2 * sb;
        return BF_OK;
    }
    const int o = 1 - p->wcur;   // keep the current buffer
    cudaFree(p->wbuf[o]);
    cudaFree(p->wscale_buf[o]);
    cudaFree(p->wsig_buf[o]);
    p->wbuf[0] = p->wbuf[1] = nullptr;
    p->wscale_buf[0] = p->wscale_buf[1] = p->wsig_buf[0] = p->wsig_buf[1] = nullptr;
    p->wcur = 0;
    p->wbufs = 1;
    p->dev_bytes -= p->w_bytes + 2 * sb;
    return BF_OK;
}

bf_status bf_plan_query(const bf_plan *p, int *kernel, int *tile_t, int *group_tiles, size_t *device_bytes)
{
    g_last_error.clear();
    if (!p) return set_error(BF_ERR_ARG, "plan is NULL");
    if (kernel) *kernel = p->kernel;
    if (tile_t) *tile_t = p->wf.simt ? 64 : p->tc.nt;
    if (group_tiles) *group_tiles = p->wf.simt ? 0 : p->tc.group;
    if (device_bytes) *device_bytes = p->dev_bytes;
    return BF_OK;
}

bf_status bf_plan_query_tiles(const bf_plan *p, int *tile_t, int *group_tiles, int *x_stages, int *n_groups)
{
    g_last_error.clear();
    if (!p) return set_error(BF_ERR_ARG, "plan is NULL");
    const bool s = p->wf.simt;
    if (tile_t) *tile_t = s ? 64 : p->tc.nt;
    if (group_tiles) *group_tiles = s ? 0 : p->tc.group;
    if (x_stages) *x_stages = s ? 0 : p->tc.xst;
    if (n_groups) *n_groups = s ? 0 : p->tc.n_groups;
    return BF_OK;
}

bf_status bf_export_weights(bf_plan *p, float *d_w, float *d_scale)
{
    g_last_error.clear();
    if (!p || !d_w) return set_error(BF_ERR_ARG, "NULL plan or output");
    bf_status st = weights_acquire(p, p->stream);
    if (st != BF_OK) return st;
    BF_CUDA(launch_export_weights(p, d_w, d_scale, p->stream), "weight export");
    return weights_release(p, p->stream);
}

bf_status bf_corner_turn(const void *d_in, int in_dtype, void *d_out, int out_dtype, int n_ant, int n_chan,
                         int n_samp, const int *perm, void *stream)
{
    g_last_error.clear();
    if (!d_in || !d_out) return set_error(BF_ERR_ARG, "NULL pointer");
    if (n_ant < 1 || n_chan < 1 || n_samp < 0) return set_error(BF_ERR_ARG, "bad shape");
    if (!valid_dtype(in_dtype) || !valid_dtype(out_dtype)) return set_error(BF_ERR_ARG, "unknown dtype");
    if (in_dtype != out_dtype && in_dtype != BF_C32)
        return set_error(BF_ERR_UNSUPPORTED, "only BF_C32 input converts to another dtype");
    cudaStream_t s = (cudaStream_t)stream;
    int *d_perm = nullptr;
    if (perm) {
        std::vector<char> seen((size_t)n_ant, 0);
        for (int n = 0; n < n_ant; ++n) {
            if (perm[n] < 0 || perm[n] >= n_ant || seen[perm[n]])
                return set_error(BF_ERR_ARG, "perm is not a permutation of 0..N-1");
            seen[perm[n]] = 1;
        }
        BF_CUDA(cudaMallocAsync((void **)&d_perm, n_ant * sizeof(int), s), "perm allocation");
        BF_CUDA(cudaMemcpyAsync(d_perm, perm, n_ant * sizeof(int), cudaMemcpyHostToDevice, s), "perm copy");
    }
    cudaError_t e = launch_corner_turn(d_in, in_dtype, d_out, out_dtype, n_ant, n_chan, n_samp, d_perm, s);
    if (d_perm) cudaFreeAsync(d_perm, s);
    if (e != cudaSuccess) return cuda_error(e, "corner turn");
    return BF_OK;
}

}  // extern "C"
