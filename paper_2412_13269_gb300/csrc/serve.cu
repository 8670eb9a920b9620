// Serving: a request loop inside the library.
//
// Clients submit encrypted queries from any thread; each submission copies
// its input ciphertexts into pinned host memory and returns a ticket.  One
// server thread owns the GPU work of the context: it admits queued requests
// while an in-flight slot is free and the device memory of the program
// instance the request needs fits the budget (idle instances of other query
// shapes are released first), replays that instance's captured graph on the
// instance's own stream, and moves on without waiting.  Requests admitted
// while others run therefore overlap on the device (continuous admission at
// request granularity; within a request every launch already covers all of
// its database's blocks).  A host callback enqueued after each request's
// device-to-host copy marks its ticket done.  Results are bit-identical to
// the same query evaluated alone: every kernel is deterministic and requests
// share no buffers.
//
// No CUDA call is made while the server's mutex is held: host callbacks of
// running requests take that mutex, and a CUDA call that synchronises the
// device (freeing memory does) would otherwise wait for them forever.
// Pinned input buffers are pooled for that reason, and instances released
// to make room are destroyed after the mutex is dropped.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>

#include "program.h"

namespace tetris {

namespace {

using Clock = std::chrono::steady_clock;
constexpr size_t kSubmitCopyThreads = 8;           // host threads copying a submission into pinned memory
constexpr size_t kWordsPerCopyThread = 1u << 22;   // at least 32 MB each

struct Request {
    uint64_t ticket = 0;
    uint32_t db = 0;
    QuerySpec spec;
    std::string key;
    u64 *pinned_in = nullptr;      // all input ciphertexts, slot order
    std::vector<size_t> in_words;  // words per slot
    size_t total_in = 0;
    Clock::time_point t_submit, t_done;
    // result
    bool done = false;
    int status = TETRIS_OK;
    std::string error;
    std::vector<u64> out;
    int level = 0, ncomp = 0;
    double scale = 0;
};

struct Instance {
    std::unique_ptr<Program> prog;
    std::string key;
    size_t bytes = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_start = nullptr, ev_end = nullptr;  // the running request's first and last device work
    float t_start = 0, t_end = 0;                        // their times after the server's reference event (ms)
    u64 *pinned_out = nullptr;
    std::shared_ptr<Request> req;
    bool busy = false;
    uint64_t last_use = 0;
    ~Instance() {
        if (stream) {
            cudaStreamSynchronize(stream);
            cudaStreamDestroy(stream);
        }
        if (ev_start) cudaEventDestroy(ev_start);
        if (ev_end) cudaEventDestroy(ev_end);
        if (pinned_out) cudaFreeHost(pinned_out);
    }
};

}  // namespace

struct Server {
    Ctx *C = nullptr;
    size_t budget = 0;
    uint32_t max_inflight = 0;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> queue;
    std::map<uint64_t, std::shared_ptr<Request>> tickets;
    std::vector<std::unique_ptr<Instance>> instances;
    std::map<std::string, size_t> bytes_of;  // measured device bytes per instance of a query shape
    std::vector<Instance *> finished;        // set by host callbacks, drained by the server thread
    std::vector<std::unique_ptr<Instance>> graveyard;  // released instances, destroyed outside the mutex
    std::multimap<size_t, u64 *> pinned_free;          // reusable pinned input buffers, by words
    uint64_t next_ticket = 1, use_clock = 0;
    bool stopping = false;
    size_t used = 0, peak = 0;
    std::vector<double> latencies_ms;
    uint64_t submitted = 0, completed = 0, rejected = 0, cancelled = 0;
    // overlap evidence: admitted requests in flight at once, and the device
    // intervals [first work, last work] of completed requests (ms after ref)
    cudaEvent_t ref = nullptr;
    uint32_t max_admitted = 0;
    std::vector<std::pair<double, double>> intervals;

    void loop();
    bool admit_one(std::unique_lock<std::mutex> &lk);
    void retire(Instance *in);
};

namespace {

void CUDART_CB on_done(void *arg) {
    auto *pr = static_cast<std::pair<Server *, Instance *> *>(arg);
    Server *S = pr->first;
    Instance *in = pr->second;
    delete pr;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->finished.push_back(in);
    }
    S->cv_work.notify_one();
}

}  // namespace

void Server::retire(Instance *in) {
    auto r = in->req;
    if (in->t_end > 0) intervals.push_back({in->t_start, in->t_end});
    r->out.assign(in->pinned_out, in->pinned_out + in->prog->out_words);
    r->level = in->prog->out_level;
    r->ncomp = in->prog->out_comps;
    r->scale = in->prog->out_scale;
    r->t_done = Clock::now();
    r->done = true;
    pinned_free.insert({r->total_in, r->pinned_in});
    r->pinned_in = nullptr;
    latencies_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
    completed++;
    in->req.reset();
    in->busy = false;
    in->last_use = ++use_clock;
}

// Called with the lock held; may release it around GPU calls.
bool Server::admit_one(std::unique_lock<std::mutex> &lk) {
    if (queue.empty()) return false;
    uint32_t inflight = 0;
    for (auto &i : instances) inflight += i->busy;
    if (inflight >= max_inflight) return false;
    auto req = queue.front();
    Instance *in = nullptr;
    for (auto &i : instances)
        if (!i->busy && i->key == req->key) {
            in = i.get();
            break;
        }
    if (!in) {
        auto evict_one = [&]() -> bool {  // release the least recently used idle instance
            Instance *victim = nullptr;
            for (auto &i : instances)
                if (!i->busy && (!victim || i->last_use < victim->last_use)) victim = i.get();
            if (!victim) return false;
            used -= victim->bytes;
            for (auto it = instances.begin(); it != instances.end(); ++it)
                if (it->get() == victim) {
                    graveyard.push_back(std::move(*it));
                    instances.erase(it);
                    break;
                }
            return true;
        };
        auto reject = [&](int code, const std::string &msg) {
            // the request may have been withdrawn while the lock was released
            if (!queue.empty() && queue.front() == req) queue.pop_front();
            req->status = code;
            req->error = msg;
            req->done = true;
            rejected++;
            cv_done.notify_all();
        };
        auto est = bytes_of.find(req->key);
        if (est != bytes_of.end()) {
            while (used + est->second > budget && evict_one()) {
            }
            if (used + est->second > budget) {
                if (inflight > 0) return false;  // wait for running queries to free memory
                reject(TETRIS_EBUSY, "query needs more device memory than the serving budget");
                return true;
            }
        } else {
            // first query of this shape: size it by recording it while nothing else runs
            if (inflight > 0) return false;
            while (evict_one()) {
            }
        }
        auto db_it = C->dbs.find(req->db);
        std::unique_ptr<Instance> ni(new Instance);
        ni->key = req->key;
        std::vector<std::unique_ptr<Instance>> dead;
        dead.swap(graveyard);
        lk.unlock();
        dead.clear();  // evicted instances give their memory back before the new one allocates
        int code = TETRIS_OK;
        std::string msg;
        try {
            TREQUIRE(db_it != C->dbs.end(), TETRIS_ENOTFOUND, "unknown database handle");
            ni->prog = record_query(*C, db_it->second, req->spec);
            ni->bytes = ni->prog->pool.bytes_held();
            TCHECK_CUDA(cudaStreamCreateWithFlags(&ni->stream, cudaStreamNonBlocking));
            TCHECK_CUDA(cudaEventCreate(&ni->ev_start));
            TCHECK_CUDA(cudaEventCreate(&ni->ev_end));
            TCHECK_CUDA(cudaMallocHost(&ni->pinned_out, ni->prog->out_words * 8));
        } catch (const Error &e) {
            code = e.code;
            msg = e.what();
        }
        lk.lock();
        if (code != TETRIS_OK) {
            graveyard.push_back(std::move(ni));
            reject(code, msg);
            return true;
        }
        bytes_of[req->key] = ni->bytes;
        if (used + ni->bytes > budget) {
            graveyard.push_back(std::move(ni));
            reject(TETRIS_EBUSY, "query needs more device memory than the serving budget");
            return true;
        }
        used += ni->bytes;
        in = ni.get();
        instances.push_back(std::move(ni));
        // the device bytes the server's programs hold right after an allocation
        // (the high-water points): every instance and anything not yet freed
        size_t held = 0;
        for (auto &i : instances) held += i->prog ? i->prog->pool.bytes_held() : 0;
        for (auto &i : graveyard) held += i->prog ? i->prog->pool.bytes_held() : 0;
        peak = std::max(peak, held);
        // withdrawn (tetris_cancel) while it was recorded: keep the instance idle
        if (queue.empty() || queue.front() != req) {
            in->last_use = ++use_clock;
            return true;
        }
    }
    queue.pop_front();
    in->busy = true;
    in->req = req;
    {
        uint32_t n = 0;
        for (auto &i : instances) n += i->busy;
        max_admitted = std::max(max_admitted, n);
    }
    Program &P = *in->prog;
    lk.unlock();
    try {
        TCHECK_CUDA(cudaEventRecord(in->ev_start, in->stream));
        size_t off = 0;
        for (size_t s = 0; s < P.in_slots.size(); s++) {  // the pinned copy holds each slot's rows back to back
            TCHECK_CUDA(cudaMemcpyAsync(P.in_slots[s].dst, req->pinned_in + off, P.in_slots[s].words() * 8,
                                        cudaMemcpyHostToDevice, in->stream));
            off += P.in_slots[s].words();
        }
        P.run_graph(in->stream);
        TCHECK_CUDA(cudaMemcpyAsync(in->pinned_out, P.out_base, P.out_words * 8, cudaMemcpyDeviceToHost, in->stream));
        TCHECK_CUDA(cudaEventRecord(in->ev_end, in->stream));
        TCHECK_CUDA(cudaLaunchHostFunc(in->stream, on_done, new std::pair<Server *, Instance *>(this, in)));
    } catch (const Error &e) {
        lk.lock();
        req->status = e.code;
        req->error = e.what();
        req->done = true;
        in->busy = false;
        in->req.reset();
        cv_done.notify_all();
        return true;
    }
    lk.lock();
    return true;
}

void Server::loop() {
    // the device was made current and checked by serve_start on the same ordinal
    cudaSetDevice(C->device);
    std::unique_lock<std::mutex> lk(mu);
    bool blocked = false;  // the head of the queue waits for running queries (memory or sizing)
    for (;;) {
        if (!finished.empty()) {
            std::vector<Instance *> fin;
            fin.swap(finished);
            lk.unlock();
            for (Instance *in : fin) {  // both events have completed: the callback follows the stream's last work
                if (cudaEventElapsedTime(&in->t_start, ref, in->ev_start) != cudaSuccess ||
                    cudaEventElapsedTime(&in->t_end, ref, in->ev_end) != cudaSuccess) {
                    cudaGetLastError();
                    in->t_start = in->t_end = 0;
                }
            }
            lk.lock();
            for (Instance *in : fin) retire(in);
            blocked = false;
            cv_done.notify_all();
        }
        while (admit_one(lk)) {
        }
        if (!graveyard.empty()) {
            std::vector<std::unique_ptr<Instance>> dead;
            dead.swap(graveyard);
            lk.unlock();
            dead.clear();  // stream sync + cudaFree/cudaFreeHost, without the mutex
            lk.lock();
            continue;  // memory came back: try admitting again
        }
        {
            uint32_t n = 0;
            for (auto &i : instances) n += i->busy;
            blocked = !queue.empty() && n < max_inflight;
        }
        bool busy = false;
        for (auto &i : instances) busy |= i->busy;
        if (stopping && queue.empty() && !busy) break;
        cv_work.wait(lk, [&] {
            if (!finished.empty() || stopping) return true;
            if (queue.empty() || blocked) return false;
            uint32_t n = 0;
            for (auto &i : instances) n += i->busy;
            return n < max_inflight;
        });
    }
}

static Server *server_of(Ctx &C) { return reinterpret_cast<Server *>(C.server); }

void serve_start(Ctx &C, size_t budget, uint32_t max_inflight) {
    TREQUIRE(!C.server, TETRIS_EINVAL, "serving already started");
    TREQUIRE(budget > 0 && max_inflight > 0, TETRIS_EINVAL, "serving needs a memory budget and at least one slot");
    auto *S = new Server;
    S->C = &C;
    S->budget = budget;
    S->max_inflight = max_inflight;
    cudaError_t e = cudaEventCreate(&S->ref);
    if (e == cudaSuccess) e = cudaEventRecord(S->ref, C.stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(S->ref);
    if (e != cudaSuccess) {
        if (S->ref) cudaEventDestroy(S->ref);
        delete S;
        cudaGetLastError();
        throw Error(TETRIS_ECUDA, std::string("serve_start: ") + cudaGetErrorString(e));
    }
    C.server = S;
    S->th = std::thread([S] { S->loop(); });
}

uint64_t serve_submit(Ctx &C, uint32_t db, const tetris_query *q) {
    Server *S = server_of(C);
    TREQUIRE(S, TETRIS_EINVAL, "serving not started");
    auto it = C.dbs.find(db);
    TREQUIRE(it != C.dbs.end(), TETRIS_ENOTFOUND, "unknown database handle");
    auto req = std::make_shared<Request>();
    req->db = db;
    req->spec = spec_of(C, it->second, q);
    req->spec.bpl = 0;
    req->key = req->spec.key(db);
    const std::vector<const tetris_ct_in *> ins = query_inputs(q);
    const std::vector<InSlot> shapes = query_slot_shapes(C, it->second, req->spec);  // only the limbs the circuit reads
    TREQUIRE(shapes.size() == ins.size(), TETRIS_EINVAL, "query: inputs do not match the plan");
    for (auto &sh : shapes) {
        req->in_words.push_back(sh.words());
        req->total_in += sh.words();
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->pinned_free.find(req->total_in);
        if (it != S->pinned_free.end()) {
            req->pinned_in = it->second;
            S->pinned_free.erase(it);
        }
    }
    if (!req->pinned_in) TCHECK_CUDA(cudaMallocHost(&req->pinned_in, req->total_in * 8));
    // the rows to copy (one per ciphertext component), then split over a few
    // host threads: a query's inputs reach a gigabyte
    struct Row {
        u64 *dst;
        const u64 *src;
        size_t words;
    };
    std::vector<Row> rows;
    size_t off = 0;
    for (size_t i = 0; i < ins.size(); i++) {
        const InSlot &sh = shapes[i];
        const u64 *src = static_cast<const u64 *>(ins[i]->data);
        for (size_t r = 0; r < sh.rows; r++) rows.push_back({req->pinned_in + off + r * sh.row_words, src + r * sh.src_pitch, sh.row_words});
        off += sh.words();
    }
    const size_t nthreads = std::min<size_t>(kSubmitCopyThreads, std::max<size_t>(1, req->total_in / kWordsPerCopyThread));
    auto copy_part = [&](size_t t) {  // thread t copies the t-th share of every row
        for (const Row &rw : rows) {
            const size_t a = rw.words * t / nthreads, b = rw.words * (t + 1) / nthreads;
            if (b > a) std::memcpy(rw.dst + a, rw.src + a, (b - a) * 8);
        }
    };
    std::vector<std::thread> helpers;
    for (size_t t = 1; t < nthreads; t++) helpers.emplace_back(copy_part, t);
    copy_part(0);
    for (auto &h : helpers) h.join();
    req->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        req->ticket = S->next_ticket++;
        S->tickets[req->ticket] = req;
        S->queue.push_back(req);
        S->submitted++;
    }
    S->cv_work.notify_one();
    return req->ticket;
}

int serve_poll(Ctx &C, uint64_t ticket, tetris_ct_out *out, uint32_t timeout_ms) {
    Server *S = server_of(C);
    TREQUIRE(S, TETRIS_EINVAL, "serving not started");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    TREQUIRE(it != S->tickets.end(), TETRIS_ENOTFOUND, "unknown ticket");
    auto req = it->second;
    if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return req->done; }))
        return TETRIS_ETIMEOUT;
    if (req->status != TETRIS_OK) {
        S->tickets.erase(it);
        throw Error(req->status, req->error);
    }
    // a buffer too small keeps the ticket: the caller may poll again with a larger one
    TREQUIRE(out && out->data && out->cap_words >= req->out.size(), TETRIS_EINVAL, "output buffer too small");
    S->tickets.erase(it);
    std::memcpy(out->data, req->out.data(), req->out.size() * 8);
    out->level = req->level;
    out->ncomp = req->ncomp;
    out->scale = req->scale;
    return TETRIS_OK;
}

void serve_cancel(Ctx &C, uint64_t ticket) {
    Server *S = server_of(C);
    TREQUIRE(S, TETRIS_EINVAL, "serving not started");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    TREQUIRE(it != S->tickets.end(), TETRIS_ENOTFOUND, "unknown ticket");
    auto req = it->second;
    if (!req->done) {
        auto q = std::find(S->queue.begin(), S->queue.end(), req);
        TREQUIRE(q != S->queue.end(), TETRIS_EBUSY, "the query is running on the device; poll it");
        S->queue.erase(q);
        if (req->pinned_in) S->pinned_free.insert({req->total_in, req->pinned_in});
        req->pinned_in = nullptr;
        S->cancelled++;
    }
    S->tickets.erase(it);
}

void serve_stats(Ctx &C, tetris_serve_stats *st, bool reset) {
    Server *S = server_of(C);
    TREQUIRE(S && st, TETRIS_EINVAL, "serving not started");
    std::lock_guard<std::mutex> lk(S->mu);
    std::vector<double> l = S->latencies_ms;
    std::sort(l.begin(), l.end());
    auto pct = [&](double p) { return l.empty() ? 0.0 : l[std::min(l.size() - 1, (size_t)(p * (l.size() - 1) + 0.5))]; };
    st->submitted = S->submitted;
    st->completed = S->completed;
    st->rejected = S->rejected;
    st->cancelled = S->cancelled;
    st->p50_ms = pct(0.50);
    st->p99_ms = pct(0.99);
    st->device_bytes = S->used;
    st->peak_device_bytes = S->peak;
    st->max_admitted = S->max_admitted;
    // the most completed requests whose device intervals share one instant
    std::vector<std::pair<double, int>> ev;
    for (auto &iv : S->intervals) {
        ev.push_back({iv.first, 1});
        ev.push_back({iv.second, -1});
    }
    std::sort(ev.begin(), ev.end(), [](auto &a, auto &b) { return a.first < b.first || (a.first == b.first && a.second < b.second); });
    int cur = 0, best = 0;
    for (auto &e : ev) best = std::max(best, cur += e.second);
    st->max_overlap = (uint32_t)best;
    if (reset) {
        S->latencies_ms.clear();
        S->intervals.clear();
        S->submitted = S->completed = S->rejected = S->cancelled = 0;
        S->peak = S->used;
        S->max_admitted = 0;
    }
}

void serve_stop(Ctx &C) {
    Server *S = server_of(C);
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
    }
    S->cv_work.notify_all();
    S->th.join();
    S->instances.clear();
    S->graveyard.clear();
    if (S->ref) cudaEventDestroy(S->ref);
    for (auto &kv : S->pinned_free) cudaFreeHost(kv.second);
    for (auto &kv : S->tickets)
        if (kv.second->pinned_in) cudaFreeHost(kv.second->pinned_in);
    delete S;
    C.server = nullptr;
}

}  // namespace tetris
