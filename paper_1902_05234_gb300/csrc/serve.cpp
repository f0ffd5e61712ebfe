// serve.cpp -- continuous-batching ECB request server (aes_srv_*).
//
// Requests name a resident key (expanded once with aes_expand_key and kept in
// device memory), a direction and caller-owned device buffers.  A dispatcher
// thread owned by the server:
//   * admits requests in arrival order while the bytes in flight (input +
//     output of every admitted, unfinished request) stay within the budget;
//     a request that does not fit waits, and so do the ones behind it (FIFO);
//   * packs the admitted requests (at most budget / slots bytes) into one
//     batch as soon as one of the in-flight slots is free, plans it on the
//     host (order and chunk prefix; the requests were validated at
//     submission) and launches it (descriptor and plan upload, the persistent
//     batch kernel, completion event) on that slot's stream -- so requests
//     that arrive while earlier batches run are
//     admitted as slots and budget free up, and consecutive batches overlap
//     on the device;
//   * retires a slot when its event has completed: the requests' statuses and
//     completion times are recorded and their bytes leave the budget.
// The dispatcher holds the server's mutex only while it picks a slot and packs
// requests, and while it retires slots; the plan, the upload and the launch run
// outside it, so submissions and polls never wait behind CUDA calls.  Keys are
// uploaded on a server-owned stream; a batch's stream waits for the newest
// upload (an event) before its kernel.  A key that a queued or in-flight request
// names cannot be replaced.  With device timing on (aes_srv_set_device_timing),
// two timing events bound each batch's device interval: from the moment its
// stream reaches the kernel (descriptors uploaded) to the kernel's completion;
// the intervals show how many batches were on the device at once.  It is off
// by default: timing events on a batch's stream added about 10 us to a
// light-load request's latency, so the event the dispatcher polls never times.
// Host waits are bounded (condition variables with timeouts); nothing on the
// device waits.  Latency is host arrival -> host-observed completion.
// Queued requests can be cancelled; an optional registry of device ranges
// confines every request's buffers to the caller's allocations, checked on
// the host at submission.  The dispatcher marks each batch's planning and
// launch, and each retirement, as NVTX ranges (domain "aesgb") for nsys/ncu
// timelines; with no tool attached they cost a few nanoseconds.
#if defined(__linux__)
#include <sys/prctl.h>
#endif
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <iterator>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "batch_internal.h"
#include "capi_internal.h"

namespace aesgb {
namespace {

using Clock = std::chrono::steady_clock;

double now_s() {
    return std::chrono::duration<double>(Clock::now().time_since_epoch()).count();
}

struct Req {
    int key_id = 0, dir = 0;
    const uint8_t *in = nullptr;
    uint8_t *out = nullptr;
    size_t nbytes = 0;
    double arrival = 0, admitted = 0, done_t = 0;
    int status = 0;
    bool done = false;
    bool released = false;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;        // after the batch kernel (no timing: the dispatcher polls it)
    cudaEvent_t t_start = nullptr;   // device timing: the stream has reached the batch (unless it opened a period)
    cudaEvent_t t_end = nullptr;     // device timing: the batch kernel has completed
    uint64_t key_gen_seen = 0;       // key uploads this slot's stream has waited for
    bool timed = false;              // the batch carries the two timing events
    bool opened_period = false;      // the batch opened a busy period (it starts at Server::ref)
    // One page-locked buffer and its device copy per slot, uploaded with one
    // copy per batch: n descriptors at the start, the host-built plan (the
    // batch kernel's workspace) at the next 256-byte boundary.
    aes_desc *h_desc = nullptr;
    aes_desc *d_desc = nullptr;
    size_t buf_bytes = 0;
    bool busy = false;
    size_t bytes = 0;
    std::vector<uint64_t> tickets;
};

struct Server {
    int dev = 0;
    size_t budget = 0, inflight = 0, peak_inflight = 0;
    int max_keys = 0, max_batch = 0;
    uint32_t *d_rk_enc = nullptr, *d_rk_dec = nullptr;  // max_keys x 64 words
    std::vector<int> key_nr;
    std::vector<uint32_t> key_users;  // queued or in-flight requests naming each key
    std::vector<char> key_updating;   // an upload of this key is in progress
    cudaStream_t key_stream = nullptr;
    cudaEvent_t key_ev = nullptr;     // recorded after the newest key upload
    uint64_t key_gen = 0;             // key uploads so far
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> pending;
    // requests by ticket: tickets are consecutive, reqs[t - base] is ticket t;
    // released requests are dropped from the front
    std::deque<Req> reqs;
    uint64_t base = 1;
    Req *find(uint64_t t) { return t >= base && t - base < reqs.size() ? &reqs[t - base] : nullptr; }
    // registered device ranges, base -> bytes (disjoint); empty: no check
    std::map<uintptr_t, size_t> regs;
    // [p, p + n) inside one registered range
    bool covered(const void *p, size_t n) const {
        const uintptr_t a = reinterpret_cast<uintptr_t>(p);
        auto it = regs.upper_bound(a);
        if (it == regs.begin()) return false;
        --it;
        return a - it->first <= it->second && n <= it->second - (a - it->first);
    }
    std::thread worker;
    bool stop = false;
    int worker_error = AES_OK;
    // statistics
    uint64_t n_submitted = 0, n_completed = 0, n_batches = 0, bytes_completed = 0, n_cancelled = 0;
    double first_arrival = 0, last_done = 0;
    size_t peak_busy = 0;  // most slots busy at once
    // Device intervals of the batches of the current busy period (from the
    // launch that found every slot idle until all are retired again), in
    // seconds after `ref`, an event recorded at the period's first launch.
    cudaEvent_t ref = nullptr;
    bool device_timing = false;  // aes_srv_set_device_timing
    bool period_timed = false;   // the current busy period was opened by a timed batch
    std::vector<std::pair<double, double>> period_iv;
    uint64_t timed_batches = 0, peak_dev = 0;
    double overlap_s = 0;
};

// Largest number of intervals that contain one instant, and the time covered
// by two or more of them (a sweep over the sorted ends; an end before a start
// at the same instant).
std::pair<uint64_t, double> sweep(const std::vector<std::pair<double, double>> &iv) {
    std::vector<std::pair<double, int>> ev;
    ev.reserve(2 * iv.size());
    for (const auto &x : iv) {
        ev.emplace_back(x.first, +1);
        ev.emplace_back(x.second, -1);
    }
    std::sort(ev.begin(), ev.end());
    uint64_t peak = 0;
    int cur = 0;
    double two = 0, last = 0;
    for (const auto &e : ev) {
        if (cur >= 2) two += e.first - last;
        last = e.first;
        cur += e.second;
        if (cur > 0 && static_cast<uint64_t>(cur) > peak) peak = static_cast<uint64_t>(cur);
    }
    return {peak, two};
}

// Fold the finished busy period's intervals into the totals (mu held).
void fold_period_locked(Server *s) {
    const auto r = sweep(s->period_iv);
    s->peak_dev = std::max(s->peak_dev, r.first);
    s->overlap_s += r.second;
    s->period_iv.clear();
}

constexpr uint32_t kRkStrideWords = 64;

void free_server(Server *s) {
    if (s->key_stream) cudaStreamSynchronize(s->key_stream);
    for (Slot &sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.t_start) cudaEventDestroy(sl.t_start);
        if (sl.t_end) cudaEventDestroy(sl.t_end);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.h_desc) cudaFreeHost(sl.h_desc);
        if (sl.d_desc) cudaFree(sl.d_desc);
    }
    if (s->key_ev) cudaEventDestroy(s->key_ev);
    if (s->key_stream) cudaStreamDestroy(s->key_stream);
    if (s->ref) cudaEventDestroy(s->ref);
    if (s->d_rk_enc) cudaFree(s->d_rk_enc);
    if (s->d_rk_dec) cudaFree(s->d_rk_dec);
    delete s;
}

// Offset of the plan in a slot's buffer, after n descriptors (the workspace
// wants 256-byte alignment).
size_t plan_offset(int n) { return (sizeof(aes_desc) * static_cast<size_t>(n) + 255) & ~static_cast<size_t>(255); }

// Batch configuration for a batch of `total_blocks`: chunks small enough that
// every warp of the grid gets several (latency at light load), at most the
// throughput-tuned chunk size.
aes_batch_cfg serve_cfg(int sms, unsigned long long total_blocks) {
    aes_batch_cfg c = batch_cfg_for(0);
    const unsigned long long warps = static_cast<unsigned long long>(sms) * (c.threads / 32);
    const unsigned long long per_pass = 32ull * c.blocks_per_thread;
    unsigned long long passes = total_blocks / (warps * 4 * per_pass);
    if (passes < 1) passes = 1;
    if (passes > static_cast<unsigned long long>(c.chunk_passes)) passes = c.chunk_passes;
    c.chunk_passes = static_cast<int32_t>(passes);
    return c;
}

nvtxDomainHandle_t nvtx_domain() {
    static const nvtxDomainHandle_t d = nvtxDomainCreateA("aesgb");
    return d;
}

// One NVTX range on the dispatcher thread for the lifetime of this object.
struct NvtxRange {
    explicit NvtxRange(const char *name) {
        nvtxEventAttributes_t a{};
        a.version = NVTX_VERSION;
        a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
        a.messageType = NVTX_MESSAGE_TYPE_ASCII;
        a.message.ascii = name;
        nvtxDomainRangePushEx(nvtx_domain(), &a);
    }
    ~NvtxRange() { nvtxDomainRangePop(nvtx_domain()); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Retire finished slots (mu held).
void retire_locked(Server *s) {
    for (Slot &sl : s->slots) {
        if (!sl.busy) continue;
        const cudaError_t q = cudaEventQuery(sl.ev);
        if (q == cudaErrorNotReady) continue;
        const NvtxRange range("aes_srv retire");
        const double t = now_s();
        const bool ok = q == cudaSuccess;
        if (!ok) (void)cudaGetLastError();
        float a = 0.f, b = 0.f;
        if (ok && sl.timed &&
            (sl.opened_period || cudaEventElapsedTime(&a, s->ref, sl.t_start) == cudaSuccess) &&
            cudaEventElapsedTime(&b, s->ref, sl.t_end) == cudaSuccess) {
            s->period_iv.emplace_back(1e-3 * a, 1e-3 * b);
            s->timed_batches++;
        }
        (void)cudaGetLastError();
        for (size_t i = 0; i < sl.tickets.size(); ++i) {
            Req *rp = s->find(sl.tickets[i]);
            if (!rp) continue;
            Req &r = *rp;
            s->key_users[r.key_id]--;
            r.done = true;
            r.done_t = t;
            r.status = ok ? AES_OK : AES_E_CUDA;  // requests were validated at submission
            s->n_completed++;
            s->bytes_completed += r.nbytes;
            s->last_done = t;
        }
        s->inflight -= sl.bytes;
        sl.bytes = 0;
        sl.tickets.clear();
        sl.busy = false;
    }
}

// A batch packed under the mutex, to be planned and launched without it.
struct Launch {
    Slot *sl = nullptr;
    int n = 0;
    unsigned long long blocks = 0;
    bool new_period = false;  // every other slot was idle: the batch opens a busy period
    bool timed = false;       // record the batch's device interval
    bool wait_keys = false;   // keys were uploaded since this slot's stream last waited
};

// Admit requests into a free slot's descriptors (mu held).  The slot is marked
// busy and its bytes counted in flight before the mutex is released, so that
// nothing else takes the slot or the budget; only the dispatcher thread
// touches slots.  Returns false if there is no free slot or nothing to admit.
bool pack_locked(Server *s, Launch *L) {
    Slot *sl = nullptr;
    size_t busy = 0;
    for (Slot &x : s->slots) {
        if (x.busy) ++busy;
        else if (!sl) sl = &x;
    }
    if (!sl || s->pending.empty()) return false;
    const double t = now_s();
    int n = 0;
    size_t bytes = 0;
    unsigned long long blocks = 0;
    // one batch takes at most its share of the budget, so that under load
    // several batches are queued on the device and the next one is already
    // there when one finishes (a single request larger than the share still
    // goes alone)
    const size_t share = s->budget / s->slots.size();
    while (!s->pending.empty() && n < s->max_batch) {
        Req &r = *s->find(s->pending.front());
        if (r.arrival > t) break;                          // not arrived yet
        const size_t need = 2 * r.nbytes;
        if (s->inflight + bytes + need > s->budget) break;  // FIFO: wait for budget
        if (n > 0 && bytes + need > share) break;
        const int nr = s->key_nr[r.key_id];
        aes_desc &d = sl->h_desc[n];
        d.rk = (r.dir == 0 ? s->d_rk_enc : s->d_rk_dec) + static_cast<size_t>(r.key_id) * kRkStrideWords;
        d.in = r.in;
        d.out = r.out;
        d.nblocks = r.nbytes / 16;
        d.nrounds = nr;
        d.dir = r.dir;
        r.admitted = t;
        sl->tickets.push_back(s->pending.front());
        s->pending.pop_front();
        bytes += need;
        blocks += d.nblocks;
        ++n;
    }
    if (n == 0) return false;
    if (busy == 0) fold_period_locked(s);  // the previous busy period has ended
    sl->busy = true;
    sl->bytes = bytes;
    s->inflight += bytes;
    s->peak_inflight = std::max(s->peak_inflight, s->inflight);
    s->peak_busy = std::max(s->peak_busy, busy + 1);
    L->sl = sl;
    L->n = n;
    L->blocks = blocks;
    L->new_period = busy == 0;
    // a period is timed as a whole: only if timing was on when it opened
    if (L->new_period) s->period_timed = s->device_timing;
    L->timed = s->period_timed;
    sl->opened_period = L->new_period;
    sl->timed = L->timed;
    L->wait_keys = sl->key_gen_seen < s->key_gen;
    sl->key_gen_seen = s->key_gen;
    return true;
}

// Plan the packed batch on the host and launch it on the slot's stream (mu
// NOT held): the plan (message order, chunk prefix, zeroed counters) is built
// here -- every request was validated at submission -- and uploaded with the
// descriptors, so only the persistent kernel runs on the device.
bool launch_unlocked(Server *s, const Launch &L, int sms) {
    const NvtxRange range("aes_srv plan+launch");
    Slot *sl = L.sl;
    const aes_batch_cfg cfg = serve_cfg(sms, L.blocks);
    const size_t ws_off = plan_offset(L.n);
    plan_on_host(sl->h_desc, L.n, batch_chunk_blocks(cfg), reinterpret_cast<uint8_t *>(sl->h_desc) + ws_off);
    bool ok = cudaMemcpyAsync(sl->d_desc, sl->h_desc, ws_off + batch_ws_bytes(L.n), cudaMemcpyHostToDevice,
                              sl->stream) == cudaSuccess;
    ok = ok && (!L.wait_keys || cudaStreamWaitEvent(sl->stream, s->key_ev, 0) == cudaSuccess);
    // the batch that opens a busy period starts at the period's reference
    // event itself (interval start 0): one event record per launch fewer
    ok = ok && (!L.timed || cudaEventRecord(L.new_period ? s->ref : sl->t_start, sl->stream) == cudaSuccess);
    ok = ok && enqueue_batch_kernel(sl->d_desc, L.n, reinterpret_cast<uint8_t *>(sl->d_desc) + ws_off, cfg,
                                    sl->stream) == AES_OK;
    ok = ok && (!L.timed || cudaEventRecord(sl->t_end, sl->stream) == cudaSuccess);
    ok = ok && cudaEventRecord(sl->ev, sl->stream) == cudaSuccess;
    if (!ok) (void)cudaGetLastError();
    return ok;
}

// Count a launched batch, or complete its requests with AES_E_CUDA if the
// launch failed (mu held).
void finish_launch_locked(Server *s, const Launch &L, bool ok) {
    Slot *sl = L.sl;
    if (ok) {
        s->n_batches++;
        return;
    }
    s->worker_error = AES_E_CUDA;
    // the event may not have been recorded: mark the batch done now
    for (size_t i = 0; i < sl->tickets.size(); ++i) {
        Req &r = *s->find(sl->tickets[i]);
        s->key_users[r.key_id]--;
        r.done = true;
        r.done_t = now_s();
        r.status = AES_E_CUDA;
        s->n_completed++;
    }
    sl->tickets.clear();
    s->inflight -= sl->bytes;
    sl->bytes = 0;
    sl->busy = false;
}

void worker_main(Server *s) {
    cudaSetDevice(s->dev);
#if defined(__linux__)
    // The dispatcher's timed waits are microseconds (event polls, arrival
    // times); a normal thread's default 50 us timer slack would stretch each
    // one to tens of microseconds, which is most of a light-load request's
    // latency.  This thread's slack only, for its lifetime.
    (void)prctl(PR_SET_TIMERSLACK, 1UL, 0UL, 0UL, 0UL);
#endif
    const int sms = sm_count(s->dev) > 0 ? sm_count(s->dev) : 1;
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        const uint64_t before = s->n_completed;
        retire_locked(s);
        bool launched = false;
        Launch L;
        while (!s->stop && pack_locked(s, &L)) {
            lk.unlock();
            const bool ok = launch_unlocked(s, L, sms);
            lk.lock();
            finish_launch_locked(s, L, ok);
            launched = true;
        }
        if (s->n_completed != before) s->cv_done.notify_all();
        bool any_busy = false;
        for (const Slot &sl : s->slots) any_busy |= sl.busy;
        if (launched) continue;
        if (any_busy) {
            // poll the slots' events again shortly (host side, bounded); a
            // completion is seen within a few microseconds
            s->cv_work.wait_for(lk, std::chrono::microseconds(3));
        } else if (!s->pending.empty()) {
            const double wait = s->find(s->pending.front())->arrival - now_s();
            if (wait > 0)
                s->cv_work.wait_for(lk, std::chrono::duration<double>(std::min(wait, 0.01)));
        } else {
            s->cv_work.wait_for(lk, std::chrono::milliseconds(10));
        }
    }
}

}  // namespace
}  // namespace aesgb

using namespace aesgb;

struct aes_server {};  // opaque handle type of the C ABI (aesgb::Server behind it)

static Server *as_server(aes_server *h) { return reinterpret_cast<Server *>(h); }

extern "C" {

int aes_srv_create(size_t mem_budget_bytes, int max_keys, int max_batch, int slots, aes_server **out) {
    if (!out || mem_budget_bytes < 32 || max_keys <= 0 || max_batch <= 0 || slots <= 0 || slots > 16)
        return AES_E_ARG;
    if (max_batch > AES_BATCH_MAX_DESCS) return AES_E_RANGE;
    *out = nullptr;
    Server *s = new Server();
    s->budget = mem_budget_bytes;
    s->max_keys = max_keys;
    s->max_batch = max_batch;
    s->key_nr.assign(static_cast<size_t>(max_keys), -1);
    s->key_users.assign(static_cast<size_t>(max_keys), 0u);
    s->key_updating.assign(static_cast<size_t>(max_keys), 0);
    int st = current_device(&s->dev);
    const size_t rk_bytes = static_cast<size_t>(max_keys) * kRkStrideWords * 4;
    void *rk_enc = nullptr, *rk_dec = nullptr;
    bool ok = st == AES_OK && (st = lib_malloc_device(&rk_enc, rk_bytes)) == AES_OK &&
              (st = lib_malloc_device(&rk_dec, rk_bytes)) == AES_OK;
    s->d_rk_enc = static_cast<uint32_t *>(rk_enc);
    s->d_rk_dec = static_cast<uint32_t *>(rk_dec);
    if (ok && (cudaStreamCreateWithFlags(&s->key_stream, cudaStreamNonBlocking) != cudaSuccess ||
               cudaEventCreateWithFlags(&s->key_ev, cudaEventDisableTiming) != cudaSuccess ||
               cudaEventCreate(&s->ref) != cudaSuccess)) {
        ok = false;
        st = AES_E_CUDA;
    }
    s->slots.resize(static_cast<size_t>(slots));
    for (Slot &sl : s->slots) {
        if (!ok) break;
        sl.buf_bytes = plan_offset(max_batch) + aes_batch_workspace_bytes(max_batch);
        void *hb = nullptr, *db = nullptr;
        ok = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreate(&sl.t_start) == cudaSuccess && cudaEventCreate(&sl.t_end) == cudaSuccess;
        if (!ok) st = AES_E_CUDA;
        ok = ok && (st = lib_malloc_host(&hb, sl.buf_bytes)) == AES_OK &&
             (st = lib_malloc_device(&db, sl.buf_bytes)) == AES_OK;
        sl.h_desc = static_cast<aes_desc *>(hb);
        sl.d_desc = static_cast<aes_desc *>(db);
        sl.tickets.reserve(static_cast<size_t>(max_batch));
    }
    if (!ok) {
        (void)cudaGetLastError();
        free_server(s);
        return st == AES_OK ? AES_E_CUDA : st;
    }
    s->worker = std::thread(worker_main, s);
    *out = reinterpret_cast<aes_server *>(s);
    return AES_OK;
}

// Keep both schedules (HOST, kRkStrideWords words each) resident under key_id.
static int put_schedules(Server *s, int key_id, const uint32_t *enc, const uint32_t *dec, int nr) {
    {
        std::lock_guard<std::mutex> lk(s->mu);
        // a queued or launched request would otherwise run with the new key
        if (s->key_users[key_id] > 0 || s->key_updating[key_id]) return AES_E_BUSY;
        s->key_updating[key_id] = 1;  // submissions naming it answer AES_E_BUSY meanwhile
    }
    // Upload on the server's key stream, outside the mutex.  The sources are
    // pageable, so each copy returns once its bytes are staged; the event
    // orders the upload before the next batch of every slot.
    const size_t off = static_cast<size_t>(key_id) * kRkStrideWords;
    const size_t bytes = kRkStrideWords * sizeof(uint32_t);
    int prev = 0;
    const bool have_prev = cudaGetDevice(&prev) == cudaSuccess;
    bool ok = cudaSetDevice(s->dev) == cudaSuccess &&
              cudaMemcpyAsync(s->d_rk_enc + off, enc, bytes, cudaMemcpyHostToDevice, s->key_stream) == cudaSuccess &&
              cudaMemcpyAsync(s->d_rk_dec + off, dec, bytes, cudaMemcpyHostToDevice, s->key_stream) == cudaSuccess &&
              cudaEventRecord(s->key_ev, s->key_stream) == cudaSuccess;
    if (!ok) (void)cudaGetLastError();
    if (have_prev) (void)cudaSetDevice(prev);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->key_updating[key_id] = 0;
        if (ok) {
            s->key_nr[key_id] = nr;
            s->key_gen++;
        }
    }
    return ok ? AES_OK : AES_E_CUDA;
}

int aes_srv_put_key(aes_server *h, int key_id, int keybits, const uint8_t *key) {
    Server *s = as_server(h);
    if (!s || key_id < 0 || key_id >= s->max_keys) return AES_E_ARG;
    uint32_t enc[kRkStrideWords] = {0}, dec[kRkStrideWords] = {0};
    const int nr = expand_key_host(keybits, key, enc, dec);
    if (nr < 0) return nr;
    return put_schedules(s, key_id, enc, dec, nr);
}

int aes_srv_put_schedule(aes_server *h, int key_id, const uint32_t *rk_enc, const uint32_t *rk_dec, int nrounds) {
    Server *s = as_server(h);
    if (!s || key_id < 0 || key_id >= s->max_keys || !rk_enc || !rk_dec) return AES_E_ARG;
    const int st = check_nrounds(nrounds);
    if (st != AES_OK) return st;
    uint32_t enc[kRkStrideWords] = {0}, dec[kRkStrideWords] = {0};
    std::memcpy(enc, rk_enc, 16u * static_cast<unsigned>(nrounds + 1));
    std::memcpy(dec, rk_dec, 16u * static_cast<unsigned>(nrounds + 1));
    return put_schedules(s, key_id, enc, dec, nrounds);
}

static int submit_locked(Server *s, int key_id, int dir, const uint8_t *in, uint8_t *out, size_t nbytes,
                         double arrival, uint64_t *ticket) {
    if (key_id < 0 || key_id >= s->max_keys) return AES_E_NOTFOUND;
    if (s->key_updating[key_id]) return AES_E_BUSY;
    if (s->key_nr[key_id] < 0) return AES_E_NOTFOUND;
    if (dir != 0 && dir != 1) return AES_E_ARG;
    if (nbytes % 16) return AES_E_ARG;
    if (nbytes > s->budget / 2) return AES_E_RANGE;  // input + output within the budget (no overflow)
    if (nbytes && (!in || !out)) return AES_E_ARG;
    const int st = check_buffers(in ? in : reinterpret_cast<const uint8_t *>(16),
                                 out ? out : reinterpret_cast<uint8_t *>(16), nbytes / 16);
    if (nbytes && st != AES_OK) return st;
    if (nbytes && !s->regs.empty() && !(s->covered(in, nbytes) && s->covered(out, nbytes)))
        return AES_E_UNREGISTERED;
    const uint64_t t = s->base + s->reqs.size();
    Req r;
    r.key_id = key_id;
    r.dir = dir;
    r.in = in;
    r.out = out;
    r.nbytes = nbytes;
    r.arrival = arrival;
    s->reqs.push_back(r);
    s->pending.push_back(t);
    s->key_users[key_id]++;
    if (s->n_submitted == 0 || arrival < s->first_arrival) s->first_arrival = arrival;
    s->n_submitted++;
    *ticket = t;
    return AES_OK;
}

int aes_srv_submit(aes_server *h, int key_id, int dir, const uint8_t *in_dev, uint8_t *out_dev, size_t nbytes,
                   uint64_t *ticket) {
    Server *s = as_server(h);
    if (!s || !ticket) return AES_E_ARG;
    int st;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        st = submit_locked(s, key_id, dir, in_dev, out_dev, nbytes, now_s(), ticket);
    }
    if (st == AES_OK) s->cv_work.notify_one();
    return st;
}

int aes_srv_submit_many(aes_server *h, int n, const int32_t *key_ids, const int32_t *dirs,
                        const uint64_t *in_devs, const uint64_t *out_devs, const uint64_t *nbytes,
                        const double *arrival_offsets_s, uint64_t *tickets) {
    Server *s = as_server(h);
    if (!s || n < 0 || (n > 0 && (!key_ids || !dirs || !in_devs || !out_devs || !nbytes || !tickets)))
        return AES_E_ARG;
    const double t0 = now_s();
    int first_err = AES_OK;
    // in slices, releasing the lock in between, so that the dispatcher starts
    // on the first requests while the rest are still being queued
    constexpr int kSlice = 1024;
    for (int lo = 0; lo < n; lo += kSlice) {
        const int hi = n - lo < kSlice ? n : lo + kSlice;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (int i = lo; i < hi; ++i) {
                const double arr = t0 + (arrival_offsets_s ? arrival_offsets_s[i] : 0.0);
                const int st = submit_locked(s, key_ids[i], dirs[i], reinterpret_cast<const uint8_t *>(in_devs[i]),
                                             reinterpret_cast<uint8_t *>(out_devs[i]), nbytes[i], arr, &tickets[i]);
                if (st != AES_OK) {
                    tickets[i] = 0;
                    if (first_err == AES_OK) first_err = st;
                }
            }
        }
        s->cv_work.notify_one();
    }
    return first_err;
}

int aes_srv_poll(aes_server *h, uint64_t ticket, int *done, int *status, double *latency_s) {
    Server *s = as_server(h);
    if (!s || !done) return AES_E_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    const Req *r = s->find(ticket);
    if (!r || r->released) return AES_E_NOTFOUND;
    *done = r->done ? 1 : 0;
    if (status) *status = r->done ? r->status : AES_OK;
    if (latency_s) *latency_s = r->done ? r->done_t - r->arrival : -1.0;
    return AES_OK;
}

int aes_srv_wait(aes_server *h, uint64_t ticket, int timeout_ms, int *status, double *latency_s) {
    Server *s = as_server(h);
    if (!s || timeout_ms < 0) return AES_E_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    if (!s->find(ticket) || s->find(ticket)->released) return AES_E_NOTFOUND;
    const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] {
        const Req *r = s->find(ticket);
        return !r || r->done;
    });
    const Req *r = s->find(ticket);
    if (!r) return AES_E_NOTFOUND;
    if (!ok) return AES_E_TIMEOUT;
    if (status) *status = r->status;
    if (latency_s) *latency_s = r->done_t - r->arrival;
    return AES_OK;
}

int aes_srv_drain(aes_server *h, int timeout_ms) {
    Server *s = as_server(h);
    if (!s || timeout_ms < 0) return AES_E_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                        [&] { return s->n_completed >= s->n_submitted; });
    return ok ? AES_OK : AES_E_TIMEOUT;
}

int aes_srv_results(aes_server *h, int n, const uint64_t *tickets, int32_t *status, double *latency_s,
                    double *queue_s, int release) {
    Server *s = as_server(h);
    if (!s || n < 0 || (n > 0 && !tickets)) return AES_E_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    int missing = 0;
    for (int i = 0; i < n; ++i) {
        Req *r = s->find(tickets[i]);
        if (!r || r->released || !r->done) {
            ++missing;
            if (status) status[i] = (!r || r->released) ? AES_E_NOTFOUND : AES_E_BUSY;
            if (latency_s) latency_s[i] = -1.0;
            if (queue_s) queue_s[i] = -1.0;
            continue;
        }
        if (status) status[i] = r->status;
        if (latency_s) latency_s[i] = r->done_t - r->arrival;
        if (queue_s) queue_s[i] = r->admitted - r->arrival;
        if (release) r->released = true;
    }
    while (!s->reqs.empty() && s->reqs.front().released) {
        s->reqs.pop_front();
        s->base++;
    }
    return missing == 0 ? AES_OK : AES_E_BUSY;
}

int aes_srv_cancel(aes_server *h, uint64_t ticket) {
    Server *s = as_server(h);
    if (!s) return AES_E_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        Req *r = s->find(ticket);
        if (!r || r->released) return AES_E_NOTFOUND;
        // queued requests are exactly those still in `pending`: the
        // dispatcher removes a request from it when it packs it into a batch
        const auto it = std::find(s->pending.begin(), s->pending.end(), ticket);
        if (r->done || it == s->pending.end()) return AES_E_BUSY;
        s->pending.erase(it);
        s->key_users[r->key_id]--;
        r->done = true;
        r->done_t = now_s();
        r->admitted = r->done_t;
        r->status = AES_E_CANCELLED;
        s->n_completed++;
        s->n_cancelled++;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_one();  // the requests behind it may fit now
    return AES_OK;
}

int aes_srv_register(aes_server *h, const void *base_dev, size_t bytes) {
    Server *s = as_server(h);
    if (!s || !base_dev || bytes == 0) return AES_E_ARG;
    const uintptr_t a = reinterpret_cast<uintptr_t>(base_dev);
    if (bytes > UINTPTR_MAX - a) return AES_E_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    // disjoint from its neighbours on both sides
    auto next = s->regs.lower_bound(a);
    if (next != s->regs.end() && next->first - a < bytes) return AES_E_OVERLAP;
    if (next != s->regs.begin()) {
        auto prev = std::prev(next);
        if (a - prev->first < prev->second) return AES_E_OVERLAP;
    }
    s->regs.emplace(a, bytes);
    return AES_OK;
}

int aes_srv_unregister(aes_server *h, const void *base_dev) {
    Server *s = as_server(h);
    if (!s || !base_dev) return AES_E_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    return s->regs.erase(reinterpret_cast<uintptr_t>(base_dev)) ? AES_OK : AES_E_NOTFOUND;
}

int aes_srv_set_device_timing(aes_server *h, int on) {
    Server *s = as_server(h);
    if (!s) return AES_E_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    s->device_timing = on != 0;
    return AES_OK;
}

int aes_srv_stats(aes_server *h, aes_srv_stats_t *out) {
    Server *s = as_server(h);
    if (!s || !out) return AES_E_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    out->submitted = s->n_submitted;
    out->completed = s->n_completed;
    out->batches = s->n_batches;
    out->bytes_completed = s->bytes_completed;
    out->inflight_bytes = s->inflight;
    out->peak_inflight_bytes = s->peak_inflight;
    out->pending = s->pending.size();
    out->busy_s = s->last_done > s->first_arrival ? s->last_done - s->first_arrival : 0.0;
    out->worker_status = s->worker_error;
    out->reserved = 0;
    out->cancelled = s->n_cancelled;
    out->peak_busy_slots = s->peak_busy;
    out->timed_batches = s->timed_batches;
    const auto cur = sweep(s->period_iv);  // the busy period still open
    out->peak_device_batches = std::max(s->peak_dev, cur.first);
    out->device_overlap_s = s->overlap_s + cur.second;
    return AES_OK;
}

int aes_srv_destroy(aes_server *h) {
    Server *s = as_server(h);
    if (!s) return AES_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->dev);
    free_server(s);
    return AES_OK;
}

}  // extern "C"
