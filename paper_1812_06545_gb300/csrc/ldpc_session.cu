// ldpc_session: a serving loop over the decoders (Sec. III-C: several workers each feeding
// its own stream so that the GPU decodes several sets of frames at once; here one dispatcher
// thread keeps up to max_inflight launches going on their own streams).
//
// Continuous batching: submitted requests wait in a FIFO queue.  Whenever a stream slot is
// free, the dispatcher admits the head of the queue together with the queued requests that
// share its parameter set (up to max_batch requests over at most MULTI_MAX_GROUPS codes, as
// memory allows), and issues them as one launch on that stream: copies in, one persistent multi-request decode
// (every codeword an item of the work queue), copies out, and a host callback that stamps
// the requests' latencies and returns their memory.  Requests that arrive while others are
// on the GPU are therefore admitted as soon as memory and a slot free up, and their work
// overlaps the running launches on the device.  Request buffers come from one device arena
// of the configured budget (first fit, coalescing frees).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string.h>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ldpc_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

constexpr size_t kAlign = 256;
constexpr size_t kLookahead = 1024;  // queued requests the dispatcher scans for a batch
inline size_t al(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

struct Block {
    size_t off = 0, size = 0;
};

// First-fit allocator over one device region; free blocks are kept sorted and coalesced.
class Arena {
  public:
    void init(char *base, size_t bytes)
    {
        base_ = base;
        free_.clear();
        free_[0] = bytes;
        used_ = peak_ = 0;
    }
    bool alloc(size_t bytes, Block *b)
    {
        bytes = al(bytes ? bytes : 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            b->off = it->first;
            b->size = bytes;
            const size_t rest = it->second - bytes, off = it->first + bytes;
            free_.erase(it);
            if (rest) free_[off] = rest;
            used_ += bytes;
            peak_ = std::max(peak_, used_);
            return true;
        }
        return false;
    }
    void release(const Block &b)
    {
        if (!b.size) return;
        used_ -= b.size;
        auto it = free_.emplace(b.off, b.size).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    char *at(size_t off) const { return base_ + off; }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }

  private:
    char *base_ = nullptr;
    std::map<size_t, size_t> free_;
    size_t used_ = 0, peak_ = 0;
};

enum ReqState { RS_QUEUED = 0, RS_RUNNING = 1, RS_DONE = 2, RS_FAILED = 3, RS_CANCELLED = 4 };

struct SessReq {
    const ldpc_code *code;
    ldpc_decode_params p;
    const float *llr_host;
    int64_t n_cw;
    uint8_t *bits_host;
    int32_t *iters_host;
    size_t bytes, ws_bytes;
    bool batchable;
    Block blk;
    Clock::time_point t_submit, t_done;
    int state = RS_QUEUED;
    ldpc_status status = LDPC_OK;
};

struct Slot {
    cudaStream_t stream = nullptr;
    bool busy = false;
    Block ws;  // the slot decoders' work counters
    std::vector<uint64_t> ids;
    ldpc_status launch_status = LDPC_OK;
    struct ldpc_session *sess = nullptr;
};

}  // namespace

struct ldpc_session {
    ldpc_session_config cfg{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_done, cv_work;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, SessReq> reqs;
    uint64_t next_id = 1;
    std::thread worker;
    bool stop = false, paused = false;
    char *arena_dev = nullptr;
    Arena arena;
    std::vector<Slot> slots;
    int64_t allocs = 0;
    ldpc_session_stats st{};
};

namespace {

ldpc_status sfail(ldpc_status s, const char *msg)
{
    ldpc::set_error(msg);
    return s;
}

bool same_params(const ldpc_decode_params &a, const ldpc_decode_params &b) { return memcmp(&a, &b, sizeof a) == 0; }

// Host callback at the end of a launch's stream work: no CUDA calls here.
void CUDART_CB launch_done(void *arg)
{
    Slot *sl = static_cast<Slot *>(arg);
    ldpc_session *s = sl->sess;
    std::lock_guard<std::mutex> lk(s->mu);
    const auto now = Clock::now();
    for (uint64_t id : sl->ids) {
        auto it = s->reqs.find(id);
        if (it == s->reqs.end()) continue;
        SessReq &r = it->second;
        s->arena.release(r.blk);
        r.blk = Block();
        r.t_done = now;
        r.state = sl->launch_status == LDPC_OK ? RS_DONE : RS_FAILED;
        r.status = sl->launch_status;
        if (r.state == RS_DONE)
            s->st.completed++;
        else
            s->st.failed++;
    }
    sl->ids.clear();
    sl->busy = false;
    s->cv_done.notify_all();
    s->cv_work.notify_one();
}

// Issue one admitted batch on its slot's stream (called without the session lock; the
// requests are RUNNING, so nothing else touches them).
void issue(ldpc_session *s, Slot &sl, std::vector<SessReq *> &batch)
{
    ldpc_status st = LDPC_OK;
    cudaStream_t strm = sl.stream;
    for (SessReq *r : batch) {
        char *base = s->arena.at(r->blk.off);
        const size_t N = (size_t)r->code->host.N;
        if (cudaMemcpyAsync(base, r->llr_host, (size_t)r->n_cw * N * sizeof(float), cudaMemcpyHostToDevice, strm) !=
            cudaSuccess)
            st = LDPC_ECUDA;
    }
    if (st == LDPC_OK) {
        if (batch[0]->batchable) {
            ldpc_request q[ldpc::MULTI_MAX_REQS];
            for (size_t i = 0; i < batch.size(); i++) {
                SessReq *r = batch[i];
                char *base = s->arena.at(r->blk.off);
                const size_t N = (size_t)r->code->host.N;
                q[i].code = r->code;
                q[i].llr_dev = base;
                q[i].n_cw = r->n_cw;
                q[i].bits_dev = reinterpret_cast<uint8_t *>(base + al((size_t)r->n_cw * N * 4));
                q[i].iters_dev =
                    reinterpret_cast<int32_t *>(base + al((size_t)r->n_cw * N * 4) + al((size_t)r->n_cw * N));
                q[i].app_dev = nullptr;
            }
            st = ldpc_decode_multi(q, (int32_t)batch.size(), &batch[0]->p, LDPC_LLR_F32, s->arena.at(sl.ws.off),
                                   sl.ws.size, strm);
        } else {
            SessReq *r = batch[0];
            char *base = s->arena.at(r->blk.off);
            const size_t N = (size_t)r->code->host.N;
            const size_t o1 = al((size_t)r->n_cw * N * 4), o2 = o1 + al((size_t)r->n_cw * N),
                         o3 = o2 + al((size_t)r->n_cw * 4);
            st = ldpc_decode_batch(r->code, &r->p, base, LDPC_LLR_F32, r->n_cw, reinterpret_cast<uint8_t *>(base + o1),
                                   reinterpret_cast<int32_t *>(base + o2), nullptr, r->ws_bytes ? base + o3 : nullptr,
                                   r->ws_bytes, strm);
        }
    }
    for (SessReq *r : batch) {
        if (st != LDPC_OK) break;
        char *base = s->arena.at(r->blk.off);
        const size_t N = (size_t)r->code->host.N;
        const size_t o1 = al((size_t)r->n_cw * N * 4), o2 = o1 + al((size_t)r->n_cw * N);
        if (cudaMemcpyAsync(r->bits_host, base + o1, (size_t)r->n_cw * N, cudaMemcpyDeviceToHost, strm) != cudaSuccess)
            st = LDPC_ECUDA;
        if (st == LDPC_OK && r->iters_host &&
            cudaMemcpyAsync(r->iters_host, base + o2, (size_t)r->n_cw * 4, cudaMemcpyDeviceToHost, strm) != cudaSuccess)
            st = LDPC_ECUDA;
    }
    sl.launch_status = st;
    if (cudaLaunchHostFunc(strm, launch_done, &sl) != cudaSuccess) {
        cudaStreamSynchronize(strm);
        sl.launch_status = LDPC_ECUDA;
        launch_done(&sl);
    }
}

void worker_loop(ldpc_session *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        if (s->stop) break;
        Slot *free_slot = nullptr;
        for (auto &sl : s->slots)
            if (!sl.busy) {
                free_slot = &sl;
                break;
            }
        std::vector<SessReq *> batch;
        std::vector<uint64_t> ids;
        if (free_slot && !s->paused) {
            // The head of the queue always goes first; batchable requests further back with
            // the head's parameters join it (within a look-ahead window), so a mix of forms
            // still fills launches.  The first request that does not fit in memory stops the
            // scan: nothing overtakes a request waiting for memory.
            const ldpc_code *codes[ldpc::MULTI_MAX_GROUPS];
            int ncodes = 0;
            size_t scanned = 0;
            for (auto qi = s->queue.begin(); qi != s->queue.end() && (int)batch.size() < s->cfg.max_batch &&
                                             scanned < kLookahead;
                 scanned++) {
                const uint64_t id = *qi;
                SessReq &r = s->reqs[id];
                if (!batch.empty() && (!batch[0]->batchable || !r.batchable || !same_params(r.p, batch[0]->p))) {
                    ++qi;
                    continue;
                }
                int g = 0;
                while (g < ncodes && codes[g] != r.code) g++;
                if (g == ncodes && ncodes == ldpc::MULTI_MAX_GROUPS) {
                    ++qi;
                    continue;
                }
                bool ok = true;
                if (s->cfg.fail_alloc_after > 0 && ++s->allocs == s->cfg.fail_alloc_after) {
                    ok = false;  // injected allocation failure: this request fails, the rest go on
                } else if (!s->arena.alloc(r.bytes, &r.blk)) {
                    break;  // wait for memory to come back
                }
                qi = s->queue.erase(qi);
                if (!ok) {
                    r.state = RS_FAILED;
                    r.status = LDPC_ENOMEM;
                    r.t_done = Clock::now();
                    s->st.failed++;
                    s->cv_done.notify_all();
                    continue;
                }
                if (g == ncodes) codes[ncodes++] = r.code;
                r.state = RS_RUNNING;
                batch.push_back(&r);
                ids.push_back(id);
                if (!r.batchable) break;
            }
        }
        if (!batch.empty()) {
            free_slot->busy = true;
            free_slot->ids = ids;
            s->st.launches++;
            lk.unlock();
            issue(s, *free_slot, batch);
            lk.lock();
            continue;
        }
        s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
    }
}

}  // namespace

extern "C" {

ldpc_status ldpc_session_default_config(ldpc_session_config *c)
{
    if (!c) return sfail(LDPC_EINVAL, "config is NULL");
    memset(c, 0, sizeof *c);
    c->hbm_budget_bytes = (size_t)1 << 30;
    c->max_inflight = 4;
    c->max_batch = ldpc::MULTI_MAX_REQS;
    return LDPC_OK;
}

ldpc_status ldpc_session_create(const ldpc_session_config *cfg, ldpc_session **out)
{
    if (!cfg || !out) return sfail(LDPC_EINVAL, "config or out is NULL");
    if (cfg->hbm_budget_bytes < ((size_t)1 << 20)) return sfail(LDPC_EINVAL, "hbm_budget_bytes must be >= 1 MiB");
    if (cfg->max_inflight < 1 || cfg->max_inflight > 16) return sfail(LDPC_EINVAL, "max_inflight must be in [1, 16]");
    if (cfg->max_batch < 1 || cfg->max_batch > ldpc::MULTI_MAX_REQS)
        return sfail(LDPC_EINVAL, "max_batch must be in [1, 128]");
    ldpc_session *s = new (std::nothrow) ldpc_session;
    if (!s) return sfail(LDPC_ENOMEM, "host allocation failed");
    s->cfg = *cfg;
    s->paused = cfg->start_paused != 0;
    s->st.budget_bytes = cfg->hbm_budget_bytes;
    cudaGetDevice(&s->device);
    const size_t reserve = (size_t)cfg->max_inflight * al(ldpc::SLOTS_WS_BYTES);
    if (cudaMalloc(&s->arena_dev, cfg->hbm_budget_bytes + reserve) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return sfail(LDPC_ENOMEM, "could not reserve the session's device memory");
    }
    s->arena.init(s->arena_dev, cfg->hbm_budget_bytes + reserve);
    s->slots.resize(cfg->max_inflight);
    for (auto &sl : s->slots) {
        sl.sess = s;
        s->arena.alloc(ldpc::SLOTS_WS_BYTES, &sl.ws);  // each slot's work counters, carved first
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) {
            for (auto &x : s->slots)
                if (x.stream) cudaStreamDestroy(x.stream);
            cudaFree(s->arena_dev);
            delete s;
            return sfail(LDPC_ECUDA, "stream creation failed");
        }
    }
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return LDPC_OK;
}

ldpc_status ldpc_session_submit(ldpc_session *s, const ldpc_code *code, const ldpc_decode_params *p,
                                const float *llr_host, int64_t n_cw, uint8_t *bits_host, int32_t *iters_host,
                                uint64_t *req_id)
{
    if (!s || !code || !p || !req_id) return sfail(LDPC_EINVAL, "session, code, params and req_id must be non-NULL");
    if (n_cw < 1 || !llr_host || !bits_host) return sfail(LDPC_EINVAL, "need n_cw >= 1 and host llr / bits buffers");
    size_t wsb = 0;
    ldpc_status st = ldpc_workspace_size(code, p, n_cw, &wsb);
    if (st != LDPC_OK) return st;
    SessReq r;
    r.code = code;
    r.p = *p;
    r.llr_host = llr_host;
    r.n_cw = n_cw;
    r.bits_host = bits_host;
    r.iters_host = iters_host;
    r.batchable = p->impl == LDPC_IMPL_AUTO && wsb == ldpc::SLOTS_WS_BYTES;
    r.ws_bytes = r.batchable ? 0 : wsb;
    const size_t N = (size_t)code->host.N;
    r.bytes = al((size_t)n_cw * N * 4) + al((size_t)n_cw * N) + al((size_t)n_cw * 4) + al(r.ws_bytes);
    if (r.bytes > s->cfg.hbm_budget_bytes) return sfail(LDPC_ENOMEM, "request larger than the session's memory budget");
    r.t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        const uint64_t id = s->next_id++;
        s->reqs.emplace(id, r);
        s->queue.push_back(id);
        s->st.submitted++;
        *req_id = id;
    }
    s->cv_work.notify_one();
    return LDPC_OK;
}

static bool terminal(int state) { return state >= RS_DONE; }

ldpc_status ldpc_session_poll(ldpc_session *s, uint64_t id, int32_t *state, double *latency_s)
{
    if (!s) return sfail(LDPC_EINVAL, "session is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(LDPC_EINVAL, "unknown or already collected request id");
    SessReq &r = it->second;
    if (state) *state = r.state;
    if (!terminal(r.state)) return LDPC_OK;
    if (latency_s) *latency_s = std::chrono::duration<double>(r.t_done - r.t_submit).count();
    const ldpc_status st = r.status;
    s->reqs.erase(it);
    return st;
}

ldpc_status ldpc_session_wait(ldpc_session *s, uint64_t id, double timeout_s, double *latency_s)
{
    if (!s) return sfail(LDPC_EINVAL, "session is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(LDPC_EINVAL, "unknown or already collected request id");
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                             std::chrono::duration<double>(timeout_s < 0 ? 0 : timeout_s));
    // the record is looked up again after every wait: another thread may have collected it
    // (poll or wait) meanwhile, and operator[] would then insert a fresh queued record
    while (!terminal(it->second.state)) {
        const bool timed_out = s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout;
        it = s->reqs.find(id);
        if (it == s->reqs.end()) return sfail(LDPC_EINVAL, "request collected by another caller while waiting");
        if (timed_out && !terminal(it->second.state))
            return sfail(LDPC_ETIMEDOUT, "request not finished within the timeout");
    }
    SessReq &r = it->second;
    if (latency_s) *latency_s = std::chrono::duration<double>(r.t_done - r.t_submit).count();
    const ldpc_status st = r.status;
    s->reqs.erase(it);
    return st;
}

ldpc_status ldpc_session_cancel(ldpc_session *s, uint64_t id)
{
    if (!s) return sfail(LDPC_EINVAL, "session is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(LDPC_EINVAL, "unknown or already collected request id");
    SessReq &r = it->second;
    if (r.state == RS_RUNNING) return sfail(LDPC_EBUSY, "request already on the GPU");
    if (r.state != RS_QUEUED) return LDPC_OK;
    s->queue.erase(std::find(s->queue.begin(), s->queue.end(), id));
    r.state = RS_CANCELLED;
    r.status = LDPC_OK;
    r.t_done = Clock::now();
    s->st.cancelled++;
    s->cv_done.notify_all();
    return LDPC_OK;
}

ldpc_status ldpc_session_pause(ldpc_session *s, int32_t paused)
{
    if (!s) return sfail(LDPC_EINVAL, "session is NULL");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->paused = paused != 0;
    }
    s->cv_work.notify_one();
    return LDPC_OK;
}

ldpc_status ldpc_session_stats_get(ldpc_session *s, ldpc_session_stats *out)
{
    if (!s || !out) return sfail(LDPC_EINVAL, "session or out is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    out->queued = (int64_t)s->queue.size();
    out->bytes_in_use = s->arena.used() - (size_t)s->cfg.max_inflight * al(ldpc::SLOTS_WS_BYTES);
    out->peak_bytes = s->arena.peak() - (size_t)s->cfg.max_inflight * al(ldpc::SLOTS_WS_BYTES);
    return LDPC_OK;
}

void ldpc_session_destroy(ldpc_session *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_one();
    if (s->worker.joinable()) s->worker.join();
    for (auto &sl : s->slots)
        if (sl.stream) cudaStreamSynchronize(sl.stream);
    for (auto &sl : s->slots)
        if (sl.stream) cudaStreamDestroy(sl.stream);
    cudaFree(s->arena_dev);
    delete s;
}

}  // extern "C"
