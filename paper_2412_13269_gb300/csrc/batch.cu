// Batches of independent ciphertext jobs at uneven ring degrees and levels.
//
// Each item runs the chain  y = rescale(ct * pt);  y = Rot(y) r times;
// out = relinearise(y * y)  on its own context (its ring degree).  Two
// schedules compute identical ciphertexts:
//   per-item: items one after another, every operation its own launches;
//   merged:   the chain of every item is recorded separately, then the k-th
//             launch of all items of one ring degree that use the same kernel
//             and mode becomes a single launch (job tables concatenated; the
//             jobs of one launch may sit at different levels, since every job
//             carries its own prime).  Items of one degree form one program;
//             the programs of different degrees run on their own streams.
// A third schedule, fused, merges the k-th launches of all items whatever
// their ring degree into one launch (see emit_fused).  The automatic schedule
// times them and keeps the fastest one's result.
#include <algorithm>
#include <chrono>
#include <cstring>

#include "program.h"

namespace tetris {

namespace {

struct ItemState {
    const tetris_batch_item *it;
    std::unique_ptr<Pool> pool;  // the item's own buffers: reused only by its own later operations
    std::vector<Deferred> launches;
    CtH out;
};

struct Group {
    Ctx *C;
    std::vector<ItemState *> items;
    std::unique_ptr<Program> P;
    cudaStream_t stream = nullptr;
};

void record_item(Rec &R, ItemState &st) {
    Ctx &C = R.C;
    const tetris_batch_item &it = *st.it;
    const int l = (int)it.level;
    TREQUIRE(l >= 1 && l <= C.L() && it.ct && it.pt && it.out, TETRIS_EINVAL, "batch item: bad level or buffer");
    R.pool_override = st.pool.get();
    R.defer = &st.launches;
    CtH x = R.new_ct(1, 2, l);
    R.P.hold.push_back(x.buf);
    TCHECK_CUDA(cudaMemcpyAsync(x.base, it.ct, x.bstride * 8, cudaMemcpyHostToDevice, C.stream));
    CtH pt = R.new_ct(1, 1, l);
    R.P.hold.push_back(pt.buf);
    TCHECK_CUDA(cudaMemcpyAsync(pt.base, it.pt, pt.bstride * 8, cudaMemcpyHostToDevice, C.stream));
    R.to_ntt(x);
    R.to_ntt(pt);
    CtH y = R.rescale(R.mul_plain(x, pt.base, 0));
    for (uint32_t i = 0; i < it.rotations; i++) {
        const uint32_t k = i % (uint32_t)(C.log_n - 1);
        y = R.rotate(y, (uint32_t)h_powmod(5, 1ull << k, 2 * C.N));
    }
    st.out = R.from_ntt(R.relin(R.tensor(y, y)));
    R.P.hold.push_back(st.out.buf);
    R.defer = nullptr;
    R.pool_override = nullptr;
}

// the k-th launches of all items that share kernel and mode become one launch
void emit_merged(Rec &R, std::vector<ItemState *> &items) {
    size_t waves = 0;
    for (auto *st : items) waves = std::max(waves, st->launches.size());
    for (size_t k = 0; k < waves; k++) {
        std::map<std::string, Deferred> groups;
        std::vector<std::string> order;
        for (auto *st : items) {
            if (k >= st->launches.size()) continue;
            const Deferred &d = st->launches[k];
            const std::string key = d.merge_key();
            auto g = groups.find(key);
            if (g == groups.end()) {
                groups.emplace(key, d);
                order.push_back(key);
            } else {
                g->second.jobs.insert(g->second.jobs.end(), d.jobs.begin(), d.jobs.end());
            }
        }
        for (auto &key : order) R.emit(groups[key]);
    }
}

// ---------------------------------------------------------------------------
// Fused schedule: the k-th launches of all items, whatever their ring degree,
// that share kernel and mode become one launch; every job names its
// context's table set (tab), automorphism jobs carry their own Galois
// element; NTT passes and the fused ModUp row pass run as persistent kernels
// over the jobs' tiles.
// ---------------------------------------------------------------------------
template <class JOB, class F>
void for_jobs(Deferred &d, F &&f) {
    const size_t n = d.jobs.size() / sizeof(JOB);
    for (size_t i = 0; i < n; i++) {
        JOB j;
        std::memcpy(&j, d.jobs.data() + i * sizeof(JOB), sizeof(JOB));
        f(j);
        std::memcpy(d.jobs.data() + i * sizeof(JOB), &j, sizeof(JOB));
    }
}

// name the table set of every job (and the Galois element of automorphism jobs)
void tag_jobs(Deferred &d, uint32_t tab) {
    switch (d.type) {
        case 0: for_jobs<NttJob>(d, [&](NttJob &j) { j.tab = tab; }); break;
        case 1: for_jobs<EwJob>(d, [&](EwJob &j) { j.tab = tab; }); break;
        case 2: for_jobs<AutJob>(d, [&](AutJob &j) { j.tab = tab; j.g = d.galois; }); break;
        case 3: for_jobs<KsJob>(d, [&](KsJob &j) { j.tab = tab; }); break;
        default: throw Error(TETRIS_EINVAL, "fused batch: launch kind not supported across ring degrees");
    }
}

std::string fused_key(const Deferred &d) {
    Deferred k = d;
    k.galois = 0;  // automorphism jobs carry their own element
    k.jobs.clear();
    return k.merge_key();
}

// tile_start table of a list of jobs (njobs + 1 entries) from each job's tiles
template <class JOB>
std::vector<uint32_t> tile_table(const Deferred &d, const std::vector<int> &logn_of_tab, int (*tiles)(int, bool),
                                 bool col) {
    std::vector<uint32_t> ts(1, 0);
    const size_t n = d.jobs.size() / sizeof(JOB);
    for (size_t i = 0; i < n; i++) {
        JOB j;
        std::memcpy(&j, d.jobs.data() + i * sizeof(JOB), sizeof(JOB));
        ts.push_back(ts.back() + (uint32_t)tiles(logn_of_tab[j.tab], col));
    }
    return ts;
}

int ks_tiles(int log_n, bool) { return keyswitch_up_tiles(log_n); }

void emit_fused(Program &P, const Deferred &d, size_t tabs_off, const std::vector<int> &logn_of_tab) {
    const int max_logn = *std::max_element(logn_of_tab.begin(), logn_of_tab.end());
    const size_t off = P.add_jobs(d.jobs.data(), d.jobs.size());
    const std::string kind = "fused." + d.kind;
    switch (d.type) {
        case 0: {
            const int n = (int)(d.jobs.size() / sizeof(NttJob));
            const bool inv = d.inverse;
            const int lm = d.load_mode, sm = d.store_mode;
            for (int pass = 0; pass < 2; pass++) {
                if (!(d.passes & (1 << pass))) continue;
                // forward: column pass first; inverse: row pass first
                const bool col = inv ? pass == 1 : pass == 0;
                const auto ts = tile_table<NttJob>(d, logn_of_tab, ntt_pass_tiles, col);
                const size_t toff = P.add_jobs(ts.data(), ts.size() * sizeof(uint32_t));
                const int total = (int)ts.back();
                P.add_launch([=](cudaStream_t s, const uint8_t *a) {
                    launch_ntt_pass_multi(inv, pass, reinterpret_cast<const TabEntry *>(a + tabs_off),
                                          reinterpret_cast<const NttJob *>(a + off),
                                          reinterpret_cast<const uint32_t *>(a + toff), n, total, lm, sm, s);
                }, kind + (inv ? "ntt_inv_p" : "ntt_fwd_p") + std::to_string(pass + 1), 0);
            }
            break;
        }
        case 1: {
            const int n = (int)(d.jobs.size() / sizeof(EwJob));
            bool tensor = true;
            for_jobs<EwJob>(const_cast<Deferred &>(d), [&](EwJob &j) {
                tensor = tensor && (j.op == EW_TENSOR || j.op == EW_TENSOR_ACC);
            });
            P.add_launch([=](cudaStream_t s, const uint8_t *a) {
                const TabEntry *tb = reinterpret_cast<const TabEntry *>(a + tabs_off);
                const EwJob *jobs = reinterpret_cast<const EwJob *>(a + off);
                if (tensor) launch_tensor(jobs, n, max_logn, nullptr, s, tb);
                else launch_ew(jobs, n, max_logn, nullptr, s, tb);
            }, kind + "ew", 0);
            break;
        }
        case 2: {
            const int n = (int)(d.jobs.size() / sizeof(AutJob));
            P.add_launch([=](cudaStream_t s, const uint8_t *a) {
                launch_automorphism_multi(reinterpret_cast<const AutJob *>(a + off), n,
                                          reinterpret_cast<const TabEntry *>(a + tabs_off), max_logn, s);
            }, kind + "automorphism", 0);
            break;
        }
        case 3: {
            const int n = (int)(d.jobs.size() / sizeof(KsJob));
            const auto ts = tile_table<KsJob>(d, logn_of_tab, ks_tiles, false);
            const size_t toff = P.add_jobs(ts.data(), ts.size() * sizeof(uint32_t));
            const int total = (int)ts.back();
            P.add_launch([=](cudaStream_t s, const uint8_t *a) {
                launch_keyswitch_up_multi(reinterpret_cast<const TabEntry *>(a + tabs_off),
                                          reinterpret_cast<const KsJob *>(a + off),
                                          reinterpret_cast<const uint32_t *>(a + toff), n, total, s);
            }, kind + "modup_keyip", 0);
            break;
        }
        default: throw Error(TETRIS_EINVAL, "fused batch: launch kind not supported across ring degrees");
    }
}

void emit_sequential(Rec &R, std::vector<ItemState *> &items) {
    for (auto *st : items)
        for (auto &d : st->launches) R.emit(d);
}

double run_groups(std::vector<Group> &groups, bool concurrent) {
    cudaStream_t s0 = groups[0].C->stream;
    for (auto &g : groups) TCHECK_CUDA(cudaStreamSynchronize(g.C->stream));
    cudaEvent_t t0, t1;
    TCHECK_CUDA(cudaEventCreate(&t0));
    TCHECK_CUDA(cudaEventCreate(&t1));
    TCHECK_CUDA(cudaEventRecord(t0, s0));
    std::vector<cudaEvent_t> ends;
    for (auto &g : groups) {
        cudaStream_t st = concurrent ? g.stream : s0;
        if (concurrent) TCHECK_CUDA(cudaStreamWaitEvent(st, t0, 0));
        g.P->run(st);
        if (concurrent) {
            cudaEvent_t e;
            TCHECK_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            TCHECK_CUDA(cudaEventRecord(e, st));
            TCHECK_CUDA(cudaStreamWaitEvent(s0, e, 0));
            ends.push_back(e);
        }
    }
    TCHECK_CUDA(cudaEventRecord(t1, s0));
    TCHECK_CUDA(cudaEventSynchronize(t1));
    float ms = 0;
    TCHECK_CUDA(cudaEventElapsedTime(&ms, t0, t1));
    for (auto e : ends) cudaEventDestroy(e);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    return ms;
}

double run_schedule(const tetris_batch_item *items, uint32_t n, bool merged, bool download) {
    std::vector<ItemState> states(n);
    std::vector<Group> groups;
    for (uint32_t i = 0; i < n; i++) {
        TREQUIRE(items[i].ctx, TETRIS_EINVAL, "batch item without a context");
        states[i].it = &items[i];
        states[i].pool.reset(new Pool);
        Ctx *C = &items[i].ctx->c;
        auto g = std::find_if(groups.begin(), groups.end(), [&](const Group &x) { return x.C == C; });
        if (g == groups.end()) {
            TREQUIRE(groups.empty() || groups[0].C->device == C->device, TETRIS_EINVAL, "batch items on different devices");
            groups.push_back(Group{C, {}, std::unique_ptr<Program>(new Program), nullptr});
            g = groups.end() - 1;
        }
        g->items.push_back(&states[i]);
    }
    for (auto &g : groups) {
        Rec R(*g.C, *g.P);
        for (auto *st : g.items) record_item(R, *st);
        if (merged) emit_merged(R, g.items);
        else emit_sequential(R, g.items);
        g.P->finalize();
        TCHECK_CUDA(cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking));
    }
    double ms = 0;
    try {
        ms = run_groups(groups, merged);
        if (download)
            for (auto &st : states) {
                const CtH &o = st.out;
                TCHECK_CUDA(cudaMemcpy(st.it->out, o.base, o.bstride * 8, cudaMemcpyDeviceToHost));
            }
    } catch (...) {
        for (auto &g : groups) cudaStreamDestroy(g.stream);
        throw;
    }
    for (auto &g : groups) cudaStreamDestroy(g.stream);
    return ms;
}

// One program for all items across ring degrees (TETRIS_SCHED_FUSED).
double run_fused(const tetris_batch_item *items, uint32_t n, bool download) {
    std::vector<ItemState> states(n);
    std::vector<Ctx *> ctxs;  // one table set per distinct context
    std::vector<uint32_t> tab_of(n);
    for (uint32_t i = 0; i < n; i++) {
        TREQUIRE(items[i].ctx, TETRIS_EINVAL, "batch item without a context");
        Ctx *C = &items[i].ctx->c;
        auto it = std::find(ctxs.begin(), ctxs.end(), C);
        if (it == ctxs.end()) {
            TREQUIRE(ctxs.size() < (size_t)kMaxTabs, TETRIS_EINVAL, "fused batch: at most 4 contexts");
            TREQUIRE(ctxs.empty() || ctxs[0]->device == C->device, TETRIS_EINVAL, "batch items on different devices");
            ntt_pass_tiles(C->log_n, true);  // refuses ring degrees the persistent kernels do not take
            ctxs.push_back(C);
            it = ctxs.end() - 1;
        }
        tab_of[i] = (uint32_t)(it - ctxs.begin());
        states[i].it = &items[i];
        states[i].pool.reset(new Pool);
    }
    Program P;
    P.ctx = ctxs[0];
    for (uint32_t i = 0; i < n; i++) {
        Rec R(*ctxs[tab_of[i]], P);
        record_item(R, states[i]);
        for (auto &d : states[i].launches) tag_jobs(d, tab_of[i]);
    }
    std::vector<TabEntry> tabs;
    std::vector<int> logn_of_tab;
    for (Ctx *C : ctxs) {
        TabEntry te;
        te.t = C->nt;
        te.log_n = C->log_n;
        tabs.push_back(te);
        logn_of_tab.push_back(C->log_n);
    }
    const size_t tabs_off = P.add_jobs(tabs.data(), tabs.size() * sizeof(TabEntry));
    size_t waves = 0;
    for (auto &st : states) waves = std::max(waves, st.launches.size());
    for (size_t k = 0; k < waves; k++) {
        std::map<std::string, Deferred> groups;
        std::vector<std::string> order;
        for (auto &st : states) {
            if (k >= st.launches.size()) continue;
            const Deferred &d = st.launches[k];
            const std::string key = fused_key(d);
            auto g = groups.find(key);
            if (g == groups.end()) {
                groups.emplace(key, d);
                order.push_back(key);
            } else {
                g->second.jobs.insert(g->second.jobs.end(), d.jobs.begin(), d.jobs.end());
            }
        }
        for (auto &key : order) emit_fused(P, groups[key], tabs_off, logn_of_tab);
    }
    P.finalize();
    for (Ctx *C : ctxs) TCHECK_CUDA(cudaStreamSynchronize(C->stream));  // the inputs' copies
    cudaStream_t st = ctxs[0]->stream;
    cudaEvent_t t0, t1;
    TCHECK_CUDA(cudaEventCreate(&t0));
    TCHECK_CUDA(cudaEventCreate(&t1));
    TCHECK_CUDA(cudaEventRecord(t0, st));
    P.run(st);
    TCHECK_CUDA(cudaEventRecord(t1, st));
    cudaError_t e = cudaEventSynchronize(t1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    TCHECK_CUDA(e);
    if (download)
        for (auto &stt : states)
            TCHECK_CUDA(cudaMemcpy(stt.it->out, stt.out.base, stt.out.bstride * 8, cudaMemcpyDeviceToHost));
    return ms;
}

}  // namespace

void batch_run(const tetris_batch_item *items, uint32_t n, int schedule, int *used, double *device_ms) {
    TREQUIRE(items && n > 0, TETRIS_EINVAL, "empty batch");
    for (uint32_t i = 0; i < n; i++) {
        TREQUIRE(items[i].ctx, TETRIS_EINVAL, "batch item without a context");
        TCHECK_CUDA(cudaSetDevice(items[i].ctx->c.device));
    }
    TREQUIRE(schedule >= TETRIS_SCHED_PER_ITEM && schedule <= TETRIS_SCHED_FUSED, TETRIS_EINVAL, "unknown schedule");
    double ms;
    int chosen = schedule;
    if (schedule == TETRIS_SCHED_AUTO) {
        double best = run_schedule(items, n, false, false);
        chosen = TETRIS_SCHED_PER_ITEM;
        const double b = run_schedule(items, n, true, false);
        if (b <= best) {
            best = b;
            chosen = TETRIS_SCHED_MERGED;
        }
        bool fusable = true;  // every ring degree one the persistent kernels take
        for (uint32_t i = 0; i < n; i++) fusable = fusable && items[i].ctx->c.log_n >= 14 && items[i].ctx->c.log_n <= 16;
        if (fusable) {
            const double c = run_fused(items, n, false);
            if (c <= best) chosen = TETRIS_SCHED_FUSED;
        }
    }
    ms = chosen == TETRIS_SCHED_FUSED ? run_fused(items, n, true)
                                     : run_schedule(items, n, chosen == TETRIS_SCHED_MERGED, true);
    if (used) *used = chosen;
    if (device_ms) *device_ms = ms;
}

}  // namespace tetris
