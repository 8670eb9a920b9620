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
// The automatic schedule times both and keeps the faster one's result.
#include <chrono>

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

}  // namespace

void batch_run(const tetris_batch_item *items, uint32_t n, int schedule, int *used, double *device_ms) {
    TREQUIRE(items && n > 0, TETRIS_EINVAL, "empty batch");
    for (uint32_t i = 0; i < n; i++) {
        TREQUIRE(items[i].ctx, TETRIS_EINVAL, "batch item without a context");
        TCHECK_CUDA(cudaSetDevice(items[i].ctx->c.device));
    }
    double ms;
    int chosen = schedule;
    if (schedule == TETRIS_SCHED_AUTO) {
        const double a = run_schedule(items, n, false, false);
        const double b = run_schedule(items, n, true, false);
        chosen = b <= a ? TETRIS_SCHED_MERGED : TETRIS_SCHED_PER_ITEM;
    }
    ms = run_schedule(items, n, chosen == TETRIS_SCHED_MERGED, true);
    if (used) *used = chosen;
    if (device_ms) *device_ms = ms;
}

}  // namespace tetris
