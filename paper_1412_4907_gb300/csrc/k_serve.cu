// Real-time serving loop: voltage chunks of several streams (sub-arrays or
// observing configurations, one plan each) arrive on the host at any time;
// a scheduler thread admits each one into device memory as soon as its block
// fits (its host-to-device copy is enqueued at once, so the link stays busy
// while earlier chunks compute), groups the admitted chunks into steps (at
// most one chunk per stream per step) and runs each step as one batched
// tensor-core launch, and copies the powers back as soon as their step ends.  Weights (in the plans) and
// the open integration window of every stream stay resident on the device
// between chunks, so a stream cut into chunks of any length integrates
// exactly as the same samples in one piece (Section 2.1 power detection and
// integration; Section 3 real-time operation of the beamformer on a stream
// of voltage buffers).
//
// Host-side pieces: a first-fit allocator over one device arena (admission
// by memory), a FIFO of pending chunks, a ring of step slots (pinned job
// table, device job table, status word, events), and completion records
// with host timestamps taken when a chunk was submitted, when its step was
// enqueued and when its powers had landed in host memory.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "batch.h"

namespace bfi {

static double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) with 256-byte granularity.
class Arena {
public:
    void reset(size_t size)
    {
        free_.clear();
        if (size) free_[0] = size;
        used_ = peak_ = 0;
    }
    // Offset of a free block of `bytes`, or SIZE_MAX.
    size_t alloc(size_t bytes)
    {
        bytes = (bytes + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const size_t off = it->first, len = it->second;
            free_.erase(it);
            if (len > bytes) free_[off + bytes] = len - bytes;
            used_ += bytes;
            peak_ = std::max(peak_, used_);
            return off;
        }
        return SIZE_MAX;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = (bytes + 255) / 256 * 256;
        used_ -= bytes;
        auto next = free_.lower_bound(off);
        size_t start = off, len = bytes;
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                start = prev->first;
                len += prev->second;
                free_.erase(prev);
            }
        }
        if (next != free_.end() && off + bytes == next->first) {
            len += next->second;
            free_.erase(next);
        }
        free_[start] = len;
    }
    size_t peak() const { return peak_; }

private:
    std::map<size_t, size_t> free_;   // offset -> length
    size_t used_ = 0, peak_ = 0;
};

struct Request {
    long long id = 0;
    int cfg = 0;
    const void *hx = nullptr;
    int T = 0;
    float *hout = nullptr;
    double t_submit = 0, t_start = 0, t_done = 0;
    size_t off = 0, bytes = 0;      // arena block
    size_t in_bytes = 0, x_off = 0, out_off = 0;
    cudaEvent_t ev_c0 = nullptr, ev_c1 = nullptr;   // its host-to-device copy
    int n_windows = 0;
    int status = BF_OK;
    int step = -1;
};

struct Stream {   // one configuration: its plan and its open window
    bf_plan *plan = nullptr;
    size_t sample_bytes = 0;
    bool expand = false;
    float *acc[2] = {nullptr, nullptr};   // [B][C] partial window sums (ping-pong)
    int cur = 0;                          // acc[cur] holds the open window
    int carry = 0;                        // samples in the open window
};

struct Slot {
    BatchJob *h_jobs = nullptr;   // the step's job table (passed in the launch parameters)
    unsigned *d_err = nullptr;
    unsigned long long *d_next = nullptr;   // the step launch's work counter
    unsigned *h_err = nullptr;    // pinned
    cudaEvent_t ev_k0 = nullptr, ev_k1 = nullptr;
    std::vector<Request *> reqs;
    std::vector<cudaEvent_t> copy_ev;   // the step's chunks' copy events (start, end, ...)
    std::vector<size_t> copy_bytes;
    bool busy = false, done = false;
    bf_server *owner = nullptr;
};

}  // namespace bfi

using namespace bfi;

struct bf_server {
    std::vector<Stream> streams;
    BatchCore core;
    int device = 0;
    uint8_t *arena_base = nullptr;
    size_t arena_bytes = 0;
    Arena arena;
    std::vector<Slot> slots;
    cudaStream_t s_in = nullptr, s_k = nullptr, s_out = nullptr;

    std::mutex mu;
    std::condition_variable cv;        // wakes the scheduler
    std::condition_variable cv_done;   // wakes pollers
    std::deque<Request *> pending;                 // submitted, not yet in device memory
    std::vector<std::deque<Request *>> admitted;   // per stream: copy enqueued, not yet in a step
    std::vector<cudaEvent_t> ev_pool;              // spare copy events
    std::deque<Request *> completed;
    long long next_id = 1, submitted = 0, n_completed = 0, steps = 0;
    int inflight = 0, max_jobs = 0;
    double flops_done = 0.0, kernel_ms = 0.0, copy_in_ms = 0.0;
    double copy_in_bytes = 0.0;
    bool stop = false;
    bool paused = false;                // admit nothing (chunks queue)
    std::string fault;                  // first CUDA error the scheduler met
    std::thread thread;
};

namespace bfi {

static size_t round256(size_t b) { return (b + 255) / 256 * 256; }

// Host function at the end of a step's stream work: powers are in host
// memory.  No CUDA calls here.
static void CUDART_CB step_done(void *arg)
{
    Slot *sl = (Slot *)arg;
    bf_server *s = sl->owner;
    const double t = now_s();
    std::lock_guard<std::mutex> lock(s->mu);
    const int st = *sl->h_err ? BF_ERR_TIMEOUT : BF_OK;
    for (Request *r : sl->reqs) {
        r->t_done = t;
        if (r->status == BF_OK) r->status = st;
        s->arena.release(r->off, r->bytes);
        s->completed.push_back(r);
        s->flops_done += 8.0 * s->streams[r->cfg].plan->N * s->streams[r->cfg].plan->B *
                         s->streams[r->cfg].plan->C * (double)r->T;
        ++s->n_completed;
    }
    sl->done = true;
    s->cv.notify_all();
    s->cv_done.notify_all();
}

// Arena bytes of a chunk: its voltages, their FP16 widening (8/4-bit
// inputs) and room for every window it can complete (at most ceil(T / T_int),
// whatever window the stream left open).
static void chunk_layout(const Stream &st, Request *r)
{
    const bf_plan *p = st.plan;
    const size_t n_samp = (size_t)p->C * r->T * p->N;
    const size_t in_b = round256(n_samp * st.sample_bytes);
    const size_t ex_b = st.expand ? round256(n_samp * 4) : 0;
    const size_t out_b = round256((size_t)p->B * p->C * ((r->T + p->t_int - 1) / p->t_int) * sizeof(float));
    r->bytes = in_b + ex_b + out_b;
    r->in_bytes = n_samp * st.sample_bytes;
    r->x_off = st.expand ? in_b : 0;      // relative until admitted
    r->out_off = in_b + ex_b;
}

// Chunks of one stream admitted ahead of its steps.  Steps take one chunk
// per stream, so admitting more would only lengthen the copy queue (and the
// wait of every later chunk behind it) without raising throughput.
constexpr size_t kAdmitAhead = 2;

// Admits pending chunks (lock held): FIFO order, a stream's chunks in order
// (a chunk that does not fit holds back the rest of its stream, other
// streams may pass), each as soon as its arena block fits and its stream has
// fewer than kAdmitAhead chunks waiting for a step.
static std::vector<Request *> admit(bf_server *s)
{
    std::vector<Request *> got;
    std::vector<char> blocked(s->streams.size(), 0);
    std::vector<size_t> ahead(s->streams.size());
    for (size_t i = 0; i < ahead.size(); ++i) ahead[i] = s->admitted[i].size();
    for (auto it = s->pending.begin(); it != s->pending.end();) {
        Request *r = *it;
        if (blocked[r->cfg] || ahead[r->cfg] >= kAdmitAhead) {
            blocked[r->cfg] = 1;
            ++it;
            continue;
        }
        Stream &st = s->streams[r->cfg];
        chunk_layout(st, r);
        const size_t off = s->arena.alloc(r->bytes);
        if (off == SIZE_MAX) {
            blocked[r->cfg] = 1;
            ++it;
            continue;
        }
        r->off = off;
        r->x_off += off;
        r->out_off += off;
        ++ahead[r->cfg];
        got.push_back(r);
        it = s->pending.erase(it);
    }
    return got;
}

// Picks the chunks of the next step (lock held): the oldest admitted chunk of
// every stream, so a stream's chunks run in order in successive steps.
static std::vector<Request *> select_step(bf_server *s)
{
    std::vector<Request *> pick;
    for (auto &q : s->admitted)
        if (!q.empty()) {
            pick.push_back(q.front());
            q.pop_front();
        }
    return pick;
}

// Enqueues the host-to-device copies of newly admitted chunks (lock not held).
static std::string launch_copies(bf_server *s, std::vector<Request *> &got)
{
    cudaError_t e;
    for (Request *r : got) {
        r->t_start = now_s();
        if ((e = cudaEventRecord(r->ev_c0, s->s_in)) != cudaSuccess ||
            (r->in_bytes && (e = cudaMemcpyAsync(s->arena_base + r->off, r->hx, r->in_bytes, cudaMemcpyHostToDevice,
                                                 s->s_in)) != cudaSuccess) ||
            (e = cudaEventRecord(r->ev_c1, s->s_in)) != cudaSuccess)
            return std::string("chunk copy: ") + cudaGetErrorString(e);
    }
    return "";
}

// Enqueues one step (lock not held).  Returns an error message or "".
static std::string launch_step(bf_server *s, Slot &sl)
{
    cudaError_t e;
    for (Request *r : sl.reqs)
        if ((e = cudaStreamWaitEvent(s->s_k, r->ev_c1, 0)) != cudaSuccess)
            return std::string("step ordering: ") + cudaGetErrorString(e);
    if ((e = cudaMemsetAsync(sl.d_err, 0, sizeof(unsigned), s->s_k)) != cudaSuccess)
        return std::string("step ordering: ") + cudaGetErrorString(e);
    int n = 0;
    for (Request *r : sl.reqs) {
        Stream &st = s->streams[r->cfg];
        bf_plan *p = st.plan;
        if (st.expand && r->T > 0) {
            e = launch_expand_to_f16(s->arena_base + r->off, p->dtype, s->arena_base + r->x_off,
                                     (long long)p->C * r->T * p->N, p->N, s->s_k);
            if (e != cudaSuccess) return std::string("integer expansion: ") + cudaGetErrorString(e);
        }
        // carried window: read acc[cur], leave the new open window in acc[1 - cur]
        const int frame = st.carry + r->T;
        const int rem = frame % p->t_int;
        r->n_windows = frame / p->t_int;
        bf_status bs = batch_fill_job(s->core, &sl.h_jobs[n], p, s->arena_base + r->x_off, r->T,
                                      (float *)(s->arena_base + r->out_off), st.carry, st.acc[st.cur],
                                      st.acc[1 - st.cur]);
        if (bs != BF_OK) return std::string("job setup: ") + bf_last_error();
        if (rem) st.cur = 1 - st.cur;
        st.carry = rem;
        ++n;
    }
    const long long units = batch_index(sl.h_jobs, n);
    // the job table travels in the launch parameters: a table copy here would
    // sit in the host-to-device queue behind the chunks admitted for later
    // steps and hold this launch back
    if ((e = cudaEventRecord(sl.ev_k0, s->s_k)) != cudaSuccess ||
        (e = n <= kParamJobs ? batch_core_launch_params(s->core, sl.h_jobs, n, units, sl.d_err, sl.d_next, s->s_k)
                             : cudaErrorInvalidValue) != cudaSuccess ||
        (e = cudaEventRecord(sl.ev_k1, s->s_k)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(s->s_out, sl.ev_k1, 0)) != cudaSuccess)
        return std::string("step launch: ") + cudaGetErrorString(e);
    for (Request *r : sl.reqs) {
        const bf_plan *p = s->streams[r->cfg].plan;
        const size_t ob = (size_t)p->B * p->C * r->n_windows * sizeof(float);
        if (ob && (e = cudaMemcpyAsync(r->hout, s->arena_base + r->out_off, ob, cudaMemcpyDeviceToHost,
                                       s->s_out)) != cudaSuccess)
            return std::string("power copy: ") + cudaGetErrorString(e);
    }
    if ((e = cudaMemcpyAsync(sl.h_err, sl.d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, s->s_out)) !=
            cudaSuccess ||
        (e = cudaLaunchHostFunc(s->s_out, step_done, &sl)) != cudaSuccess)
        return std::string("step completion: ") + cudaGetErrorString(e);
    return "";
}

static void fail_requests(bf_server *s, std::vector<Request *> &reqs, int status)
{
    const double t = now_s();
    for (Request *r : reqs) {
        r->status = status;
        r->t_done = t;
        s->completed.push_back(r);
        ++s->n_completed;
    }
    reqs.clear();
}

static cudaEvent_t take_event(bf_server *s)
{
    if (!s->ev_pool.empty()) {
        cudaEvent_t e = s->ev_pool.back();
        s->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

static bool all_admitted_empty(const bf_server *s)
{
    for (const auto &q : s->admitted)
        if (!q.empty()) return false;
    return true;
}

// Fails every chunk not yet in a step (lock held): after a CUDA error the
// server serves nothing more.
static void fail_queued(bf_server *s)
{
    std::vector<Request *> rest(s->pending.begin(), s->pending.end());
    s->pending.clear();
    for (auto &q : s->admitted) {
        for (Request *r : q) {
            s->arena.release(r->off, r->bytes);
            rest.push_back(r);
        }
        q.clear();
    }
    fail_requests(s, rest, BF_ERR_CUDA);
    s->cv_done.notify_all();
}

static void scheduler(bf_server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lock(s->mu);
    for (;;) {
        // retire finished steps: kernel and copy times from the events
        for (Slot &sl : s->slots) {
            if (!sl.busy || !sl.done) continue;
            float ms = 0.f;
            double copy_ms = 0.0;
            lock.unlock();
            const bool ok_k = cudaEventElapsedTime(&ms, sl.ev_k0, sl.ev_k1) == cudaSuccess;
            for (size_t i = 0; i + 1 < sl.copy_ev.size(); i += 2) {
                float c = 0.f;
                if (cudaEventElapsedTime(&c, sl.copy_ev[i], sl.copy_ev[i + 1]) == cudaSuccess) copy_ms += c;
            }
            lock.lock();
            if (ok_k) s->kernel_ms += ms;
            s->copy_in_ms += copy_ms;
            for (size_t b : sl.copy_bytes) s->copy_in_bytes += (double)b;
            s->ev_pool.insert(s->ev_pool.end(), sl.copy_ev.begin(), sl.copy_ev.end());
            sl.copy_ev.clear();
            sl.copy_bytes.clear();
            sl.busy = sl.done = false;
            sl.reqs.clear();
            --s->inflight;
        }
        if (s->stop && s->pending.empty() && all_admitted_empty(s) && s->inflight == 0) break;
        const bool go = s->fault.empty() && (!s->paused || s->stop);
        // admission: copies start as soon as a chunk's block fits
        std::vector<Request *> got;
        if (go && !s->pending.empty()) got = admit(s);
        if (!got.empty()) {
            for (Request *r : got) {
                r->ev_c0 = take_event(s);
                r->ev_c1 = take_event(s);
            }
            lock.unlock();
            const std::string err = launch_copies(s, got);
            lock.lock();
            if (!err.empty()) {
                if (s->fault.empty()) s->fault = err;
                for (Request *r : got) s->arena.release(r->off, r->bytes);
                fail_requests(s, got, BF_ERR_CUDA);
                fail_queued(s);
                continue;
            }
            for (Request *r : got) s->admitted[r->cfg].push_back(r);
        }
        // a step: the oldest admitted chunk of every stream
        Slot *free_slot = nullptr;
        for (Slot &sl : s->slots)
            if (!sl.busy) {
                free_slot = &sl;
                break;
            }
        std::vector<Request *> pick;
        if (free_slot && go) pick = select_step(s);
        if (pick.empty()) {
            if (!s->fault.empty() && (!s->pending.empty() || !all_admitted_empty(s))) {
                fail_queued(s);
                continue;
            }
            if (got.empty()) s->cv.wait_for(lock, std::chrono::milliseconds(50));
            continue;
        }
        free_slot->busy = true;
        free_slot->done = false;
        free_slot->reqs = pick;
        for (Request *r : pick) {
            r->step = (int)s->steps;
            free_slot->copy_ev.push_back(r->ev_c0);
            free_slot->copy_ev.push_back(r->ev_c1);
            free_slot->copy_bytes.push_back(r->in_bytes);
        }
        ++s->steps;
        ++s->inflight;
        s->max_jobs = std::max(s->max_jobs, (int)pick.size());
        lock.unlock();
        const std::string err = launch_step(s, *free_slot);
        lock.lock();
        if (!err.empty()) {
            // nothing of this step may complete through the callback now;
            // wait for the streams, then fail its chunks
            lock.unlock();
            cudaStreamSynchronize(s->s_in);
            cudaStreamSynchronize(s->s_k);
            cudaStreamSynchronize(s->s_out);
            lock.lock();
            if (s->fault.empty()) s->fault = err;
            if (!free_slot->done) {
                for (Request *r : free_slot->reqs) s->arena.release(r->off, r->bytes);
                fail_requests(s, free_slot->reqs, BF_ERR_CUDA);
                free_slot->busy = false;
                --s->inflight;
            }
            s->cv_done.notify_all();
        }
    }
}

static void server_free(bf_server *s)
{
    if (!s) return;
    if (s->thread.joinable()) {
        {
            std::lock_guard<std::mutex> lock(s->mu);
            s->stop = true;
        }
        s->cv.notify_all();
        s->thread.join();
    }
    if (s->s_in) cudaStreamSynchronize(s->s_in);
    if (s->s_k) cudaStreamSynchronize(s->s_k);
    if (s->s_out) cudaStreamSynchronize(s->s_out);
    for (Slot &sl : s->slots) {
        if (sl.h_jobs) cudaFreeHost(sl.h_jobs);
        if (sl.d_err) cudaFree(sl.d_err);
        if (sl.d_next) cudaFree(sl.d_next);
        if (sl.h_err) cudaFreeHost(sl.h_err);
        if (sl.ev_k0) cudaEventDestroy(sl.ev_k0);
        if (sl.ev_k1) cudaEventDestroy(sl.ev_k1);
    }
    for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
    for (Stream &st : s->streams)
        for (float *a : st.acc)
            if (a) cudaFree(a);
    if (s->arena_base) cudaFree(s->arena_base);
    for (cudaStream_t q : {s->s_in, s->s_k, s->s_out})
        if (q) cudaStreamDestroy(q);
    for (Request *r : s->pending) delete r;
    for (Request *r : s->completed) delete r;
    delete s;
}

}  // namespace bfi

extern "C" {

double bf_server_now(void) { return now_s(); }

bf_status bf_server_create(bf_server **out, bf_plan *const *plans, int n_configs, size_t mem_bytes, int max_steps,
                           int tile_t)
{
    clear_error();
    if (!out) return set_error(BF_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (max_steps < 1 || max_steps > 8) return set_error(BF_ERR_ARG, "max_steps must be in 1..8");
    if (mem_bytes < 4096) return set_error(BF_ERR_ARG, "memory budget too small");
    if (n_configs > kParamJobs)
        return set_error(BF_ERR_UNSUPPORTED, "a server takes at most " + std::to_string(kParamJobs) + " streams");
    for (int i = 0; plans && i < n_configs; ++i) {
        if (plans[i] && plans[i]->layout != BF_LAYOUT_CTN)   // chunks arrive in the [C][T][N] packet order
            return set_error(BF_ERR_UNSUPPORTED, "servers take the CTN layout");
        if (plans[i] && plans[i]->wbufs != 1)
            return set_error(BF_ERR_UNSUPPORTED, "plans with double-buffered weights cannot join a server");
    }
    BatchCore core;
    bf_status st = batch_core_init(&core, plans, n_configs, tile_t);
    if (st != BF_OK) return st;
    for (int i = 0; i < n_configs; ++i) {
        const bf_plan *p = plans[i];
        const int row = 2 * p->N * p->wf.es;   // bytes per sample row as the MMA reads it
        if (row % 16) return set_error(BF_ERR_UNSUPPORTED, "antenna count gives a row stride that TMA cannot read");
    }
    bf_server *s = new bf_server();
    s->core = core;
    s->device = plans[0]->device;
    s->streams.resize(n_configs);
    s->admitted.resize(n_configs);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < n_configs && e == cudaSuccess; ++i) {
        Stream &q = s->streams[i];
        q.plan = plans[i];
        q.sample_bytes = dtype_sample_bytes(plans[i]->dtype);
        q.expand = plans[i]->dtype == BF_CI8 || plans[i]->dtype == BF_CI4;
        const size_t ab = (size_t)plans[i]->B * plans[i]->C * sizeof(float);
        for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaMalloc((void **)&q.acc[k], ab);
        if (e == cudaSuccess) e = cudaStreamSynchronize(plans[i]->stream);   // weights are ready
    }
    if (e == cudaSuccess) e = cudaMalloc((void **)&s->arena_base, mem_bytes);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_in, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_k, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_out, cudaStreamNonBlocking);
    s->slots.resize(max_steps);
    for (int i = 0; i < max_steps && e == cudaSuccess; ++i) {
        Slot &sl = s->slots[i];
        sl.owner = s;
        if ((e = cudaHostAlloc((void **)&sl.h_jobs, sizeof(BatchJob) * n_configs, cudaHostAllocDefault)) ==
                cudaSuccess &&
            (e = cudaMalloc((void **)&sl.d_err, sizeof(unsigned))) == cudaSuccess &&
            (e = cudaMalloc((void **)&sl.d_next, sizeof(unsigned long long))) == cudaSuccess &&
            (e = cudaHostAlloc((void **)&sl.h_err, sizeof(unsigned), cudaHostAllocDefault)) == cudaSuccess &&
            (e = cudaEventCreate(&sl.ev_k0)) == cudaSuccess)
            e = cudaEventCreate(&sl.ev_k1);
        if (e == cudaSuccess) *sl.h_err = 0;
    }
    if (e != cudaSuccess) {
        server_free(s);
        return cuda_error(e, "server allocation");
    }
    s->arena_bytes = mem_bytes;
    s->arena.reset(mem_bytes);
    s->thread = std::thread(scheduler, s);
    *out = s;
    return BF_OK;
}

bf_status bf_server_submit(bf_server *s, int config, const void *h_voltages, int n_samp, float *h_power,
                           long long *id)
{
    clear_error();
    if (!s) return set_error(BF_ERR_ARG, "server is NULL");
    if (config < 0 || config >= (int)s->streams.size()) return set_error(BF_ERR_ARG, "config out of range");
    if (n_samp < 1) return set_error(BF_ERR_ARG, "a chunk needs at least one sample");
    if (!h_voltages || !h_power) return set_error(BF_ERR_ARG, "NULL voltage or power pointer");
    const Stream &st = s->streams[config];
    const bf_plan *p = st.plan;
    const size_t n = (size_t)p->C * n_samp * p->N;
    const size_t worst = round256(n * st.sample_bytes) + (st.expand ? round256(n * 4) : 0) +
                         round256((size_t)p->B * p->C * ((n_samp + p->t_int - 1) / p->t_int) * sizeof(float));
    if (worst > s->arena_bytes) return set_error(BF_ERR_ARG, "chunk larger than the server's memory budget");
    Request *r = new Request();
    r->cfg = config;
    r->hx = h_voltages;
    r->T = n_samp;
    r->hout = h_power;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stop) {
            delete r;
            return set_error(BF_ERR_STATE, "server is shutting down");
        }
        r->id = s->next_id++;
        r->t_submit = now_s();
        s->pending.push_back(r);
        ++s->submitted;
    }
    s->cv.notify_all();
    if (id) *id = r->id;
    return BF_OK;
}

bf_status bf_server_poll(bf_server *s, bf_completion *out, int max, int *n_out, int timeout_ms)
{
    clear_error();
    if (!s || !n_out || (max > 0 && !out)) return set_error(BF_ERR_ARG, "NULL argument");
    *n_out = 0;
    std::unique_lock<std::mutex> lock(s->mu);
    if (s->completed.empty() && timeout_ms > 0)
        s->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), [&] { return !s->completed.empty(); });
    int n = 0;
    while (n < max && !s->completed.empty()) {
        Request *r = s->completed.front();
        s->completed.pop_front();
        bf_completion &c = out[n++];
        c.id = r->id;
        c.config = r->cfg;
        c.status = r->status;
        c.n_windows = r->n_windows;
        c.step = r->step;
        c.n_samp = r->T;
        c.t_submit = r->t_submit;
        c.t_start = r->t_start;
        c.t_done = r->t_done;
        delete r;
    }
    *n_out = n;
    return BF_OK;
}

bf_status bf_server_drain(bf_server *s, int timeout_ms)
{
    clear_error();
    if (!s) return set_error(BF_ERR_ARG, "server is NULL");
    std::unique_lock<std::mutex> lock(s->mu);
    const bool ok = s->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms), [&] {
        return s->n_completed == s->submitted;
    });
    if (!ok) return set_error(BF_ERR_TIMEOUT, "chunks still in flight after the timeout");
    if (!s->fault.empty()) return set_error(BF_ERR_CUDA, s->fault);
    return BF_OK;
}

bf_status bf_server_pause(bf_server *s, int paused)
{
    clear_error();
    if (!s) return set_error(BF_ERR_ARG, "server is NULL");
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->paused = paused != 0;
    }
    s->cv.notify_all();
    return BF_OK;
}

bf_status bf_server_stats(bf_server *s, bf_server_counters *out)
{
    clear_error();
    if (!s || !out) return set_error(BF_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    out->submitted = s->submitted;
    out->completed = s->n_completed;
    out->steps = s->steps;
    out->max_jobs_per_step = s->max_jobs;
    out->flops = s->flops_done;
    out->kernel_ms = s->kernel_ms;
    out->copy_in_ms = s->copy_in_ms;
    out->copy_in_bytes = s->copy_in_bytes;
    out->arena_bytes = s->arena_bytes;
    out->arena_peak = s->arena.peak();
    out->tile_t = s->core.nt;
    return BF_OK;
}

bf_status bf_server_destroy(bf_server *s)
{
    clear_error();
    if (!s) return BF_OK;
    server_free(s);
    return BF_OK;
}

}  // extern "C"
