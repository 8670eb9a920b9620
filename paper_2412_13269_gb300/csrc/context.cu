// Context creation, memory pool, recorded programs and the ciphertext-level
// recorder.  Paper references: Section 2.2 (ring), 2.4.1 (SwitchKey), 2.5
// (rescale), Appendix A.2 (relinearisation, automorphism + key switch).
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <type_traits>

#include "program.h"

namespace tetris {

// ---------------------------------------------------------------------------
// Pool
// ---------------------------------------------------------------------------
Pool::Pool() : guard_(std::getenv("TETRIS_GUARD_WORDS") != nullptr) {}

Pool::~Pool() {
    *alive_ = 0;
    for (auto &a : all_) cudaFree(a.first - (guard_ ? kGuardWords : 0));
}

BufPtr Pool::alloc(size_t words, bool fresh) {
    words = std::max<size_t>(words, 2);
    u64 *ptr = nullptr;
    // best fit among the free buffers up to 4x the request (a buffer keeps its
    // own size when it comes back), so requests of several sizes share buffers
    auto it = fresh ? free_.end() : free_.lower_bound(words);
    if (it != free_.end() && it->first <= 4 * words) {
        ptr = it->second;
        words = it->first;
        free_.erase(it);
    } else {
        const size_t g = guard_ ? kGuardWords : 0, total = words + 2 * g;
        cudaError_t e = cudaMalloc(&ptr, total * 8);
        if (e != cudaSuccess) {
            cudaGetLastError();
            trim();
            e = cudaMalloc(&ptr, total * 8);
            if (e != cudaSuccess) {
                cudaGetLastError();
                throw Error(TETRIS_ENOMEM, "device allocation of " + std::to_string(total * 8) + " bytes failed");
            }
        }
        if (g) {
            TCHECK_CUDA(cudaMemset(ptr, kGuardByte, g * 8));
            TCHECK_CUDA(cudaMemset(ptr + g + words, kGuardByte, g * 8));
            ptr += g;
        }
        all_.push_back({ptr, words});
        held_ += total * 8;
    }
    std::weak_ptr<int> alive = alive_;
    auto *fl = &free_;
    return BufPtr(new DevBuf{ptr, words}, [alive, fl](DevBuf *b) {
        if (auto a = alive.lock())
            if (*a) fl->insert({b->words, b->ptr});
        delete b;
    });
}

void Pool::trim() {
    const size_t g = guard_ ? kGuardWords : 0;
    for (auto &f : free_) {
        cudaFree(f.second - g);
        auto it = std::find_if(all_.begin(), all_.end(), [&](auto &a) { return a.first == f.second; });
        if (it != all_.end()) {
            held_ -= (it->second + 2 * g) * 8;
            all_.erase(it);
        }
    }
    free_.clear();
}

bool Pool::contains(const void *p, size_t words) const {
    const u64 *q = static_cast<const u64 *>(p);
    for (auto &a : all_)
        if (q >= a.first && q + words <= a.first + a.second) return true;
    return false;
}

std::vector<std::string> Pool::check_guards() const {
    std::vector<std::string> bad;
    if (!guard_) return bad;
    std::vector<u64> h(kGuardWords);
    u64 pat;
    std::memset(&pat, kGuardByte, 8);
    for (auto &a : all_)
        for (int side = 0; side < 2; side++) {
            const u64 *g = side == 0 ? a.first - kGuardWords : a.first + a.second;
            TCHECK_CUDA(cudaMemcpy(h.data(), g, kGuardWords * 8, cudaMemcpyDeviceToHost));
            for (u64 w : h)
                if (w != pat) {
                    std::ostringstream o;
                    o << a.first << (side == 0 ? ":before" : ":after");
                    bad.push_back(o.str());
                    break;
                }
        }
    return bad;
}

void Pool::plant_guard_fault() {
    TREQUIRE(guard_ && !all_.empty(), TETRIS_EINVAL, "no guarded buffer to plant a fault in");
    TCHECK_CUDA(cudaMemset(all_.front().first + all_.front().second, 0, 8));  // the first word after the buffer
}

size_t Ctx::bytes_held() const {
    size_t b = pool.bytes_held();
    for (auto &kv : programs) b += kv.second->pool.bytes_held();
    return b;
}

int64_t round_half_up(double x) {
    TREQUIRE(std::fabs(x) < 0x1p62, TETRIS_EINVAL, "a scaled constant does not fit 62 bits");
    return (int64_t)std::floor(x + 0.5);
}

const Key &find_key(const Ctx &c, uint32_t galois) {
    if (galois == 0) {
        TREQUIRE(c.relin.buf, TETRIS_ENOTFOUND, "relinearisation key not loaded");
        return c.relin;
    }
    auto it = c.rot.find(galois);
    TREQUIRE(it != c.rot.end(), TETRIS_ENOTFOUND, "rotation key for galois element " + std::to_string(galois) + " not loaded");
    return it->second;
}

// ---------------------------------------------------------------------------
// Program
// ---------------------------------------------------------------------------
Program::~Program() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (side) {
        cudaStreamSynchronize(side);
        cudaStreamDestroy(side);
    }
    for (auto &g : groups) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
        if (g.ev) cudaEventDestroy(g.ev);
    }
    if (early_ev) cudaEventDestroy(early_ev);
}

void Program::add_input_wait(size_t first) {
    TREQUIRE(first <= in_slots.size() && (groups.empty() || first > groups.back().first), TETRIS_EINVAL,
             "input groups: slots out of order");
    if (!side) {
        TCHECK_CUDA(cudaEventCreateWithFlags(&early_ev, cudaEventDisableTiming));
        TCHECK_CUDA(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
    }
    InGroup g;
    g.first = first;
    TCHECK_CUDA(cudaEventCreateWithFlags(&g.ev, cudaEventDisableTiming));
    cudaEvent_t ev = g.ev;
    Launch l;
    l.fn = [ev](cudaStream_t s, const uint8_t *) { TCHECK_CUDA(cudaStreamWaitEvent(s, ev, 0)); };
    l.kind = "wait_inputs";
    l.kernel = false;
    g.wait_at = launches.size();
    launches.push_back(std::move(l));
    groups.push_back(g);
}

void InSlot::copy_from(const void *src, cudaMemcpyKind kind, cudaStream_t s) const {
    if (rows == 1 || src_pitch == row_words)
        TCHECK_CUDA(cudaMemcpyAsync(dst, src, words() * 8, kind, s));
    else
        TCHECK_CUDA(cudaMemcpy2DAsync(dst, row_words * 8, src, src_pitch * 8, row_words * 8, rows, kind, s));
}

void Program::copy_inputs(const std::vector<const void *> &srcs, cudaMemcpyKind kind, cudaStream_t s) {
    TREQUIRE(srcs.size() == in_slots.size(), TETRIS_EINVAL, "inputs do not match the program");
    const size_t split = groups.empty() ? srcs.size() : std::min(groups[0].first, srcs.size());
    for (size_t i = 0; i < split; i++) in_slots[i].copy_from(srcs[i], kind, s);
    if (groups.empty()) return;
    // the side stream starts after the first group's copies, which follow the previous run on s
    TCHECK_CUDA(cudaEventRecord(early_ev, s));
    TCHECK_CUDA(cudaStreamWaitEvent(side, early_ev, 0));
    for (size_t k = 0; k < groups.size(); k++) {
        const size_t end = k + 1 < groups.size() ? groups[k + 1].first : srcs.size();
        for (size_t i = groups[k].first; i < end; i++) in_slots[i].copy_from(srcs[i], kind, side);
        TCHECK_CUDA(cudaEventRecord(groups[k].ev, side));
    }
}

size_t Program::add_jobs(const void *p, size_t bytes) {
    size_t off = (arena.size() + 255) & ~(size_t)255;
    arena.resize(off + bytes);
    std::memcpy(arena.data() + off, p, bytes);
    return off;
}

void Program::finalize() {
    if (arena.empty()) arena.resize(256);
    // a fresh buffer: one freed during recording may still be written by the
    // program's own launches (reuse is safe in launch order, not after it)
    arena_dev = pool.alloc((arena.size() + 7) / 8, true);
    TCHECK_CUDA(cudaMemcpy(arena_dev->ptr, arena.data(), arena.size(), cudaMemcpyHostToDevice));
}

void Program::add_launch(std::function<void(cudaStream_t, const uint8_t *)> fn, const std::string &kind, double bytes,
                         double modmuls, double units) {
    launches.push_back({std::move(fn), kind, bytes, modmuls, true, units});
    kernel_launches += 1;
}

void Program::run(cudaStream_t s) {
    const uint8_t *a = reinterpret_cast<const uint8_t *>(arena_dev->ptr);
    for (auto &l : launches) l.fn(s, a);
    TCHECK_CUDA(cudaGetLastError());
}

// Eager replay with a CUDA event pair around every launch on the same stream.
void Program::run_profiled(cudaStream_t s, std::map<std::string, KernelStat> &stats) {
    const uint8_t *a = reinterpret_cast<const uint8_t *>(arena_dev->ptr);
    std::vector<cudaEvent_t> ev(2 * launches.size());
    for (auto &e : ev) TCHECK_CUDA(cudaEventCreate(&e));
    for (size_t i = 0; i < launches.size(); i++) {
        TCHECK_CUDA(cudaEventRecord(ev[2 * i], s));
        launches[i].fn(s, a);
        TCHECK_CUDA(cudaEventRecord(ev[2 * i + 1], s));
    }
    TCHECK_CUDA(cudaStreamSynchronize(s));
    TCHECK_CUDA(cudaGetLastError());
    double ks_ms = 0;
    for (size_t i = 0; i < launches.size(); i++) {
        if (!launches[i].kernel) continue;
        float ms = 0;
        TCHECK_CUDA(cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]));
        KernelStat &k = stats[launches[i].kind];
        k.launches += 1;
        k.ms += ms;
        k.bytes += launches[i].bytes;
        k.modmuls += launches[i].modmuls;
        k.units += launches[i].units;
        if (launches[i].kind.compare(0, 3, "ks.") == 0) ks_ms += ms;
    }
    if (ks_count) {
        KernelStat &k = stats["keyswitch(total)"];
        k.launches += ks_count;
        k.ms += ks_ms;
        k.bytes += ks_bytes;
    }
    for (auto &e : ev) cudaEventDestroy(e);
}

// The launches captured as one CUDA graph, or as one per segment between the
// waits for input groups (a plain stream wait between two graph launches).
void Program::run_graph(cudaStream_t s) {
    const size_t cut = groups.empty() ? launches.size() : groups[0].wait_at;
    auto capture = [&](size_t i0, size_t i1, cudaGraph_t &g, cudaGraphExec_t &x) {
        cudaStream_t cs;
        TCHECK_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        TCHECK_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
        const uint8_t *a = reinterpret_cast<const uint8_t *>(arena_dev->ptr);
        for (size_t i = i0; i < i1; i++) launches[i].fn(cs, a);
        cudaError_t e = cudaStreamEndCapture(cs, &g);
        cudaStreamDestroy(cs);
        TCHECK_CUDA(e);
        TCHECK_CUDA(cudaGraphInstantiate(&x, g, 0));
    };
    if (!exec) {
        capture(0, cut, graph, exec);
        for (size_t k = 0; k < groups.size(); k++) {
            const size_t end = k + 1 < groups.size() ? groups[k + 1].wait_at : launches.size();
            capture(groups[k].wait_at + 1, end, groups[k].graph, groups[k].exec);
        }
    }
    TCHECK_CUDA(cudaGraphLaunch(exec, s));
    for (auto &g : groups) {
        TCHECK_CUDA(cudaStreamWaitEvent(s, g.ev, 0));
        TCHECK_CUDA(cudaGraphLaunch(g.exec, s));
    }
}

// ---------------------------------------------------------------------------
// Recorder primitives
// ---------------------------------------------------------------------------
CtH Rec::new_ct(int B, int comps, int level) {
    CtH c;
    c.N = C.N;
    c.B = B;
    c.comps = comps;
    c.level = level;
    c.cstride = (size_t)(level + 1) * C.N;
    c.bstride = c.cstride * comps;
    c.buf = pool().alloc(c.bstride * B);
    c.base = c.buf->ptr;
    return c;
}

CtH Rec::view(const BufPtr &buf, u64 *base, int B, int comps, int level, size_t bstride, size_t cstride, double scale) {
    CtH c;
    c.N = C.N;
    c.buf = buf;
    c.base = base;
    c.B = B;
    c.comps = comps;
    c.level = level;
    c.bstride = bstride;
    c.cstride = cstride;
    c.scale = scale;
    return c;
}

namespace {
// distinct limbs among a set of pointers, in bytes of N words each
double distinct_bytes(const std::vector<const void *> &ptrs, size_t N) {
    std::vector<const void *> v;
    for (auto p : ptrs)
        if (p) v.push_back(p);
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    return (double)v.size() * N * 8;
}
const char *load_name(int m) {
    switch (m) {
        case LOAD_CONV_PRE: return "convpre";
        case LOAD_REDUCE: return "reduce";
        case LOAD_INT64: return "int64";
        case LOAD_PIECE: return "piece";
    }
    return "plain";
}
const char *ew_name(int op) {
    switch (op) {
        case EW_ADD: return "add";
        case EW_SUB: return "sub";
        case EW_MUL: return "mul";
        case EW_MUL_CONST: return "mulc";
        case EW_ADD_CONST: return "addc";
        case EW_NEG: return "neg";
        case EW_COPY: return "copy";
        case EW_FMA: return "fma";
        case EW_TENSOR: return "tensor";
        case EW_TENSOR_ACC: return "tensor_acc";
        case EW_RESCALE_COEF: return "rescale_coef";
        case EW_ADD_MUL_CONST: return "addmulc";
        case EW_REDUCE: return "reduce";
    }
    return "?";
}
}  // namespace

template <class J>
static Deferred make_deferred(int type, const std::vector<J> &jobs, const std::string &kind, double bytes) {
    Deferred d;
    d.type = type;
    d.job_size = sizeof(J);
    d.jobs.resize(jobs.size() * sizeof(J));
    std::memcpy(d.jobs.data(), jobs.data(), d.jobs.size());
    d.kind = kind;
    d.bytes = bytes;
    return d;
}

// ---------------------------------------------------------------------------
// Debug checks: the device ranges of every job, checked on the host before the
// job is recorded (nothing is launched with a range outside the allocations)
// ---------------------------------------------------------------------------
size_t Rec::tab_offset() {
    if (P.tab_off == SIZE_MAX) {
        TabEntry te;
        te.t = C.nt;
        te.log_n = C.log_n;
        P.tab_off = P.add_jobs(&te, sizeof te);
    }
    return P.tab_off;
}

void Rec::check_range(const void *p, size_t words, const std::string &what) {
    if (!p) return;
    C.checked_ranges++;
    if (C.pool.contains(p, words) || P.pool.contains(p, words) || (pool_override && pool_override->contains(p, words)))
        return;
    std::ostringstream o;
    o << "debug check: " << what << " [" << p << ", +" << words << " words) lies outside every live allocation";
    throw Error(TETRIS_EINVAL, o.str());
}

void Rec::check_prime(uint32_t prime, const std::string &what) {
    TREQUIRE(prime < (uint32_t)C.nqp(), TETRIS_EINVAL, "debug check: " + what + " names prime " + std::to_string(prime));
}

void Rec::check(const std::vector<NttJob> &jobs, int load_mode, int store_mode) {
    const size_t N = C.N;
    for (size_t i = 0; i < jobs.size(); i++) {
        const NttJob &j = jobs[i];
        const std::string w = "NTT job " + std::to_string(i);
        check_prime(j.prime, w);
        const size_t ns = load_mode == LOAD_CONV_PRE ? j.nsrc : 1;
        TREQUIRE(ns >= 1 && ns <= (size_t)kMaxConvSrc, TETRIS_EINVAL, "debug check: " + w + " has a bad source count");
        check_range(j.src, (ns - 1) * j.src_stride + N, w + " source");
        check_range(j.dst, N, w + " destination");
        const size_t nb = (store_mode == STORE_SCALED_CONV && j.nsrc) ? j.nsrc : 1;
        check_range(j.base, (nb - 1) * j.src_stride + N, w + " base");
        check_range(j.extra, N, w + " extra");
    }
}

void Rec::check(const std::vector<EwJob> &jobs) {
    const size_t N = C.N;
    for (size_t i = 0; i < jobs.size(); i++) {
        const EwJob &j = jobs[i];
        const std::string w = "elementwise job " + std::to_string(i);
        check_prime(j.prime, w);
        if (j.op == EW_RESCALE_COEF) check_prime(j.prime2, w);
        for (const void *p : {(const void *)j.a, (const void *)j.b, (const void *)j.c, (const void *)j.dst,
                              (const void *)j.a1, (const void *)j.b1, (const void *)j.d1, (const void *)j.d2,
                              (const void *)j.c1, (const void *)j.c2})
            check_range(p, N, w);
    }
}

void Rec::check(const std::vector<AutJob> &jobs) {
    for (size_t i = 0; i < jobs.size(); i++) {
        check_range(jobs[i].src, C.N, "automorphism job " + std::to_string(i) + " source");
        check_range(jobs[i].dst, C.N, "automorphism job " + std::to_string(i) + " destination");
    }
}

void Rec::check(const std::vector<KsJob> &jobs) {
    const size_t N = C.N;
    for (size_t i = 0; i < jobs.size(); i++) {
        const KsJob &j = jobs[i];
        const std::string w = "key-switch job " + std::to_string(i);
        check_prime(j.prime, w);
        TREQUIRE(j.ndig >= 1 && j.ndig <= (uint32_t)kMaxKeyDigits, TETRIS_EINVAL, "debug check: " + w + " digits");
        for (uint32_t d = 0; d < j.ndig; d++) {
            check_range(j.src[d], N, w + " digit source");
            check_range(j.key[d], 2 * N, w + " key");
        }
        for (const void *p : {(const void *)j.acc0, (const void *)j.acc1, (const void *)j.ex0, (const void *)j.ex1})
            check_range(p, N, w);
    }
}

void Rec::check(const std::vector<LinJob> &jobs) {
    const size_t N = C.N;
    for (size_t i = 0; i < jobs.size(); i++) {
        const LinJob &j = jobs[i];
        const std::string w = "linear-combination job " + std::to_string(i);
        check_prime(j.prime, w);
        for (uint32_t a = 0; a < j.nattr; a++) {
            check_range(j.pt + a * j.pt_stride, N, w + " plaintext");
            check_range(j.w0 + a * j.w_stride, N, w + " coefficient");
            check_range(j.w1 + a * j.w_stride, N, w + " coefficient");
        }
        check_range(j.d0, N, w);
        check_range(j.d1, N, w);
    }
}

void Rec::check(const std::vector<RedJob> &jobs) {
    for (size_t i = 0; i < jobs.size(); i++) {
        check_prime(jobs[i].prime, "reduction job " + std::to_string(i));
        check_range(jobs[i].src, C.N, "reduction job " + std::to_string(i));
        check_range(jobs[i].dst, C.N, "reduction job " + std::to_string(i));
    }
}

void Rec::emit(const Deferred &d) {
    auto *saved = defer;
    defer = nullptr;
    emitting_ = true;  // checked when deferred (the item pools are not reachable from here)
    const size_t n = d.jobs.size() / d.job_size;
    auto as = [&](auto *tag) {
        using J = std::remove_pointer_t<decltype(tag)>;
        std::vector<J> v(n);
        std::memcpy(v.data(), d.jobs.data(), d.jobs.size());
        return v;
    };
    const std::string saved_prefix = prefix;
    prefix.clear();
    switch (d.type) {
        case 0: ntt(d.inverse, as((NttJob *)nullptr), d.load_mode, d.store_mode, -1, STORE_PLAIN, d.passes); break;
        case 1: ew(as((EwJob *)nullptr)); break;
        case 2: aut(as((AutJob *)nullptr), d.galois); break;
        case 3: ksup(as((KsJob *)nullptr)); break;
        case 4: lin(as((LinJob *)nullptr)); break;
        case 5: red(as((RedJob *)nullptr)); break;
    }
    prefix = saved_prefix;
    defer = saved;
    emitting_ = false;
}

static const char *store_name(int m) {
    switch (m) {
        case STORE_COMBINE: return "combine";
        case STORE_SCALED: return "scaled";
        case STORE_SCALED_CONV: return "scaledconv";
    }
    return "plain";
}

void Rec::ntt(bool inverse, const std::vector<NttJob> &jobs_in, int load_mode, int store_mode, int split,
              int store_mode_b, int passes) {
    if (jobs_in.empty()) return;
    // The column pass's outer stage has one twiddle, psi^(N/2) forward (its
    // first stage) and psi^-(N/2) = -psi^(N/2) inverse (its last): a forward
    // conversion load also forms the conversion times it for the upper half of
    // every column, an inverse scaled store the scale times its inverse.
    std::vector<NttJob> folded;
    if ((load_mode == LOAD_CONV_PRE && !inverse) || inverse) {
        folded = jobs_in;
        for (auto &j : folded) {
            const u64 q = C.all[j.prime], w1 = h_powmod(C.psi[j.prime], C.N / 2, q);
            if (inverse) {
                j.mul_w = h_mulmod(j.mul, q - w1, q);
                j.mul_w_sh = h_shoup(j.mul_w, q);
                continue;
            }
            for (uint32_t s = 0; s < j.nsrc; s++) {
                j.c2w[s] = h_mulmod(j.c2[s], w1, q);
                j.c2w_sh[s] = h_shoup(j.c2w[s], q);
            }
            j.conv_sub_w = h_mulmod(j.conv_sub, w1, q);
        }
    }
    const std::vector<NttJob> &jobs = folded.empty() ? jobs_in : folded;
    TREQUIRE(split < 0 || !defer, TETRIS_EINVAL, "split transforms are not deferred");
    TREQUIRE(passes >= 1 && passes <= 3, TETRIS_EINVAL, "no transform pass selected");
    if (checking()) check(jobs_in, load_mode, split >= 0 ? std::max(store_mode, store_mode_b) : store_mode);
    if (defer) {
        Deferred d = make_deferred(0, jobs, prefix, 0);
        d.inverse = inverse;
        d.load_mode = load_mode;
        d.store_mode = store_mode;
        d.passes = passes;
        defer->push_back(std::move(d));
        return;
    }
    size_t off = P.add_jobs(jobs.data(), jobs.size() * sizeof(NttJob));
    int n = (int)jobs.size(), logn = C.log_n;
    NttTables t = C.nt;
    const size_t N = C.N;
    std::vector<const void *> srcs;
    for (auto &j : jobs) {
        if (load_mode == LOAD_CONV_PRE)
            for (uint32_t s = 0; s < j.nsrc; s++) srcs.push_back(j.src + s * j.src_stride);
        else
            srcs.push_back(j.src);
    }
    const double limb = (double)N * 8, w = n * limb;
    const std::string dir = inverse ? "ntt_inv" : "ntt_fwd";
    const int log1 = (logn + 1) / 2, log2 = logn / 2;
    double conv = 0;
    if (load_mode == LOAD_CONV_PRE)
        for (auto &j : jobs) conv += j.nsrc;
    if (load_mode == LOAD_PIECE) conv = n;  // one Shoup product per element
    const double first_log = inverse ? log2 : log1, second_log = inverse ? log1 : log2;
    const double mm1 = (double)n * N * first_log / 2 + conv * N;
    // one launch of pass `pass` over jobs [j0, j0 + m): a CTA per tile, or
    // (persistent) resident CTAs walking the tiles
    auto pass_fn = [&](int pass, size_t o, int m, int mode) -> std::function<void(cudaStream_t, const uint8_t *)> {
        if (!persistent) {
            return [=](cudaStream_t s, const uint8_t *a) {
                launch_ntt(inverse, logn, t, reinterpret_cast<const NttJob *>(a + o), m, load_mode, mode, s, pass);
            };
        }
        const uint32_t tiles = (uint32_t)ntt_pass_tiles(logn, inverse ? pass == 1 : pass == 0);
        std::vector<uint32_t> ts(m + 1);
        for (int k = 0; k <= m; k++) ts[k] = (uint32_t)k * tiles;
        const size_t toff = P.add_jobs(ts.data(), ts.size() * sizeof(uint32_t)), tb = tab_offset();
        const int total = (int)(m * tiles);
        return [=](cudaStream_t s, const uint8_t *a) {
            launch_ntt_pass_multi(inverse, pass, reinterpret_cast<const TabEntry *>(a + tb),
                                  reinterpret_cast<const NttJob *>(a + o), reinterpret_cast<const uint32_t *>(a + toff), m,
                                  total, load_mode, mode, s);
        };
    };
    if (passes & 1)
        P.add_launch(pass_fn(0, off, n, store_mode), prefix + dir + "_p1_" + load_name(load_mode),
                     distinct_bytes(srcs, N) + w, mm1, n);
    if (!(passes & 2)) return;
    // second pass: one launch per store segment
    auto second = [&](int j0, int j1, int mode) {
        const int m = j1 - j0;
        if (m <= 0) return;
        double b2 = 2.0 * m * limb, extra_mm = 0;
        std::vector<const void *> rd;
        for (int j = j0; j < j1; j++) {
            if (mode == STORE_COMBINE) {
                rd.push_back(jobs[j].base);
                rd.push_back(jobs[j].extra);
            } else if (mode == STORE_SCALED_CONV) {
                for (uint32_t k = 0; k < jobs[j].nsrc; k++) rd.push_back(jobs[j].base + k * jobs[j].src_stride);
                extra_mm += jobs[j].nsrc;
            }
        }
        b2 += distinct_bytes(rd, N);
        const double mm2 = (double)m * N * (second_log / 2 + ((mode != STORE_PLAIN || inverse) ? 1 : 0)) + extra_mm * N;
        const size_t o2 = off + (size_t)j0 * sizeof(NttJob);
        P.add_launch(pass_fn(1, o2, m, mode), prefix + dir + "_p2_" + store_name(mode), b2, mm2, m);
    };
    if (split < 0 || split >= n) {
        second(0, n, store_mode);
    } else {
        second(0, split, store_mode);
        second(split, n, store_mode_b);
    }
}

void Rec::ew(const std::vector<EwJob> &jobs) {
    if (jobs.empty()) return;
    if (checking()) check(jobs);
    if (defer) {
        defer->push_back(make_deferred(1, jobs, prefix + std::to_string(jobs[0].op), 0));
        return;
    }
    size_t off = P.add_jobs(jobs.data(), jobs.size() * sizeof(EwJob));
    int n = (int)jobs.size(), logn = C.log_n;
    const ModInfo *m = C.nt.mods;
    std::vector<const void *> rd;
    double writes = 0;
    for (auto &j : jobs) {
        rd.push_back(j.a);
        rd.push_back(j.b);
        rd.push_back(j.c);
        rd.push_back(j.a1);
        rd.push_back(j.b1);
        rd.push_back(j.c1);
        rd.push_back(j.c2);
        writes += (j.op == EW_TENSOR || j.op == EW_TENSOR_ACC) ? 3 : 1;
    }
    bool tensor = true;
    for (auto &j : jobs) tensor = tensor && (j.op == EW_TENSOR || j.op == EW_TENSOR_ACC);
    P.add_launch([=](cudaStream_t s, const uint8_t *a) {
        if (tensor) launch_tensor(reinterpret_cast<const EwJob *>(a + off), n, logn, m, s);
        else launch_ew(reinterpret_cast<const EwJob *>(a + off), n, logn, m, s);
    }, prefix + "ew_" + ew_name(jobs[0].op), distinct_bytes(rd, C.N) + writes * C.N * 8);
}

void Rec::aut(const std::vector<AutJob> &jobs, uint32_t g) {
    if (jobs.empty()) return;
    if (checking()) check(jobs);
    if (defer) {
        Deferred d = make_deferred(2, jobs, prefix, 0);
        d.galois = g;
        defer->push_back(std::move(d));
        return;
    }
    size_t off = P.add_jobs(jobs.data(), jobs.size() * sizeof(AutJob));
    int n = (int)jobs.size(), logn = C.log_n;
    P.add_launch([=](cudaStream_t s, const uint8_t *a) {
        launch_automorphism(reinterpret_cast<const AutJob *>(a + off), n, logn, g, s);
    }, prefix + "automorphism", 2.0 * n * C.N * 8);
}

void Rec::ksup(const std::vector<KsJob> &jobs) {
    if (jobs.empty()) return;
    if (checking()) check(jobs);
    if (defer) {
        defer->push_back(make_deferred(3, jobs, prefix, 0));
        return;
    }
    size_t off = P.add_jobs(jobs.data(), jobs.size() * sizeof(KsJob));
    int n = (int)jobs.size(), logn = C.log_n;
    NttTables t = C.nt;
    std::vector<const void *> rd;
    double prods = 0, transforms = 0;
    for (auto &j : jobs) {
        for (uint32_t d = 0; d < j.ndig; d++) {
            rd.push_back(j.src[d]);
            rd.push_back(j.key[d]);  // both components: 2N words
            rd.push_back(j.key[d] + C.N);
            if ((int)d != j.own) transforms += 1;
        }
        rd.push_back(j.ex0);
        rd.push_back(j.ex1);
        prods += 2.0 * j.ndig + (j.own >= 0 ? 1 : 0) + (j.ex0 ? 1 : 0) + (j.ex1 ? 1 : 0);
    }
    // the row pass of each transformed digit (log2(N2)/2 butterfly products per word) and the products above
    const double mm = (transforms * (logn / 2) / 2.0 + prods) * C.N;
    std::function<void(cudaStream_t, const uint8_t *)> fn;
    if (!persistent) {
        fn = [=](cudaStream_t s, const uint8_t *a) {
            launch_keyswitch_up(logn, t, reinterpret_cast<const KsJob *>(a + off), n, s);
        };
    } else {
        const uint32_t tiles = (uint32_t)keyswitch_up_tiles(logn);
        std::vector<uint32_t> ts(n + 1);
        for (int k = 0; k <= n; k++) ts[k] = (uint32_t)k * tiles;
        const size_t toff = P.add_jobs(ts.data(), ts.size() * sizeof(uint32_t)), tb = tab_offset();
        const int total = (int)(n * tiles);
        fn = [=](cudaStream_t s, const uint8_t *a) {
            launch_keyswitch_up_multi(reinterpret_cast<const TabEntry *>(a + tb), reinterpret_cast<const KsJob *>(a + off),
                                      reinterpret_cast<const uint32_t *>(a + toff), n, total, s);
        };
    }
    P.add_launch(fn, prefix + "modup_keyip", distinct_bytes(rd, C.N) + 2.0 * n * C.N * 8, mm, n);
}

void Rec::lin(const std::vector<LinJob> &jobs) {
    if (jobs.empty()) return;
    if (checking()) check(jobs);
    if (defer) {
        defer->push_back(make_deferred(4, jobs, prefix, 0));
        return;
    }
    size_t off = P.add_jobs(jobs.data(), jobs.size() * sizeof(LinJob));
    int n = (int)jobs.size(), logn = C.log_n;
    const ModInfo *m = C.nt.mods;
    std::vector<const void *> rd;
    for (auto &j : jobs)
        for (uint32_t a = 0; a < j.nattr; a++) {
            rd.push_back(j.pt + a * j.pt_stride);
            rd.push_back(j.w0 + a * j.w_stride);
            rd.push_back(j.w1 + a * j.w_stride);
        }
    P.add_launch([=](cudaStream_t s, const uint8_t *a) {
        launch_lincomb(reinterpret_cast<const LinJob *>(a + off), n, logn, m, s);
    }, prefix + "lincomb", distinct_bytes(rd, C.N) + 2.0 * n * C.N * 8);
}

void Rec::red(const std::vector<RedJob> &jobs) {
    if (jobs.empty()) return;
    if (checking()) check(jobs);
    if (defer) {
        defer->push_back(make_deferred(5, jobs, prefix, 0));
        return;
    }
    size_t off = P.add_jobs(jobs.data(), jobs.size() * sizeof(RedJob));
    int n = (int)jobs.size(), logn = C.log_n;
    const ModInfo *m = C.nt.mods;
    P.add_launch([=](cudaStream_t s, const uint8_t *a) {
        launch_reduce_i64(reinterpret_cast<const RedJob *>(a + off), n, logn, m, s);
    }, prefix + "reduce_i64", 2.0 * n * C.N * 8);
}

static EwJob ewj(EwOp op, uint32_t prime, u64 *dst, const u64 *a, const u64 *b = nullptr) {
    EwJob j{};
    j.op = op;
    j.prime = prime;
    j.dst = dst;
    j.a = a;
    j.b = b;
    return j;
}

// ---------------------------------------------------------------------------
// Ciphertext operations
// ---------------------------------------------------------------------------
void Rec::to_ntt(const CtH &a) {
    std::vector<NttJob> jobs;
    for (int b = 0; b < a.B; b++)
        for (int c = 0; c < a.comps; c++)
            for (int i = 0; i <= a.level; i++) {
                NttJob j{};
                j.src = j.dst = a.limb(b, c, i);
                j.prime = i;
                jobs.push_back(j);
            }
    ntt(false, jobs, LOAD_PLAIN, STORE_PLAIN);
}

CtH Rec::from_ntt(const CtH &a) {
    CtH o = new_ct(a.B, a.comps, a.level);
    o.scale = a.scale;
    std::vector<NttJob> jobs;
    for (int b = 0; b < a.B; b++)
        for (int c = 0; c < a.comps; c++)
            for (int i = 0; i <= a.level; i++) {
                NttJob j{};
                j.src = a.limb(b, c, i);
                j.dst = o.limb(b, c, i);
                j.prime = i;
                jobs.push_back(j);
            }
    ntt(true, jobs, LOAD_PLAIN, STORE_PLAIN);
    return o;
}

CtH Rec::add(const CtH &a, const CtH &b) {
    TREQUIRE(a.level == b.level && a.comps == b.comps, TETRIS_EINVAL, "add: level/components differ");
    TREQUIRE(a.B == b.B || a.B == 1 || b.B == 1, TETRIS_EINVAL, "add: batch sizes differ");
    int B = std::max(a.B, b.B);
    CtH o = new_ct(B, a.comps, a.level);
    o.scale = a.scale;
    std::vector<EwJob> jobs;
    for (int k = 0; k < B; k++)
        for (int c = 0; c < a.comps; c++)
            for (int i = 0; i <= a.level; i++) jobs.push_back(ewj(EW_ADD, i, o.limb(k, c, i), a.limb(k, c, i), b.limb(k, c, i)));
    ew(jobs);
    return o;
}

CtH Rec::sub(const CtH &a, const CtH &b) {
    TREQUIRE(a.level == b.level && a.comps == b.comps, TETRIS_EINVAL, "sub: level/components differ");
    TREQUIRE(a.B == b.B || a.B == 1 || b.B == 1, TETRIS_EINVAL, "sub: batch sizes differ");
    int B = std::max(a.B, b.B);
    CtH o = new_ct(B, a.comps, a.level);
    o.scale = a.scale;
    std::vector<EwJob> jobs;
    for (int k = 0; k < B; k++)
        for (int c = 0; c < a.comps; c++)
            for (int i = 0; i <= a.level; i++) jobs.push_back(ewj(EW_SUB, i, o.limb(k, c, i), a.limb(k, c, i), b.limb(k, c, i)));
    ew(jobs);
    return o;
}


CtH Rec::mul_int(const CtH &a, int64_t cst) {
    CtH o = new_ct(a.B, a.comps, a.level);
    o.scale = a.scale;
    std::vector<EwJob> jobs;
    for (int k = 0; k < a.B; k++)
        for (int c = 0; c < a.comps; c++)
            for (int i = 0; i <= a.level; i++) {
                EwJob j = ewj(EW_MUL_CONST, i, o.limb(k, c, i), a.limb(k, c, i));
                j.k = signed_mod(cst, C.q[i]);
                j.k_sh = h_shoup(j.k, C.q[i]);
                jobs.push_back(j);
            }
    ew(jobs);
    return o;
}

CtH Rec::add_int(const CtH &a, int64_t cst) {
    CtH o = new_ct(a.B, a.comps, a.level);
    o.scale = a.scale;
    std::vector<EwJob> jobs;
    for (int k = 0; k < a.B; k++)
        for (int c = 0; c < a.comps; c++)
            for (int i = 0; i <= a.level; i++) {
                if (c == 0) {
                    // the constant polynomial is the same constant at every evaluation point
                    EwJob j = ewj(EW_ADD_CONST, i, o.limb(k, c, i), a.limb(k, c, i));
                    j.k = signed_mod(cst, C.q[i]);
                    jobs.push_back(j);
                } else {
                    jobs.push_back(ewj(EW_COPY, i, o.limb(k, c, i), a.limb(k, c, i)));
                }
            }
    ew(jobs);
    return o;
}

CtH Rec::mul_plain(const CtH &a, const u64 *pt, size_t pt_bstride) {
    CtH o = new_ct(a.B, a.comps, a.level);
    std::vector<EwJob> jobs;
    for (int k = 0; k < a.B; k++)
        for (int c = 0; c < a.comps; c++)
            for (int i = 0; i <= a.level; i++)
                jobs.push_back(ewj(EW_MUL, i, o.limb(k, c, i), a.limb(k, c, i), pt + k * pt_bstride + (size_t)i * C.N));
    ew(jobs);
    return o;
}

CtH Rec::tensor(const CtH &a, const CtH &b) { return tensor_add(CtH(), a, b); }

// acc + a (x) b in one pass (acc empty: the tensor alone)
CtH Rec::tensor_add(const CtH &acc, const CtH &a, const CtH &b) {
    TREQUIRE(a.level == b.level && a.comps == 2 && b.comps == 2, TETRIS_EINVAL, "tensor: operands differ");
    TREQUIRE(a.B == b.B || a.B == 1 || b.B == 1, TETRIS_EINVAL, "tensor: batch sizes differ");
    int B = std::max(a.B, b.B);
    const bool add = acc.buf != nullptr;
    if (add) {
        TREQUIRE(acc.comps == 3 && acc.level == a.level && (acc.B == B || acc.B == 1), TETRIS_EINVAL,
                 "tensor_add: accumulator differs");
        B = std::max(B, acc.B);
    }
    CtH o = new_ct(B, 3, a.level);
    o.scale = a.scale * b.scale;
    std::vector<EwJob> jobs;
    for (int k = 0; k < B; k++)
        for (int i = 0; i <= a.level; i++) {
            EwJob j = ewj(add ? EW_TENSOR_ACC : EW_TENSOR, i, o.limb(k, 0, i), a.limb(k, 0, i), b.limb(k, 0, i));
            j.a1 = a.limb(k, 1, i);
            j.b1 = b.limb(k, 1, i);
            j.d1 = o.limb(k, 1, i);
            j.d2 = o.limb(k, 2, i);
            if (add) {
                j.c = acc.limb(k, 0, i);
                j.c1 = acc.limb(k, 1, i);
                j.c2 = acc.limb(k, 2, i);
            }
            jobs.push_back(j);
        }
    ew(jobs);
    return o;
}

// Fast base conversion from the consecutive primes first..first+nsrc-1 to
// dst_prime: x -> sum_s [x_s * (Qs/q_s)^-1]_{q_s} * (Qs/q_s mod q_dst).
// The recorded transforms fold the first factor into the inverse NTT that
// produces the sources (STORE_SCALED) and load with LOAD_CONV_PRE, which only
// uses c2 = Qs/q_s mod q_dst.
NttJob Rec::conv_job(uint32_t dst_prime, const u64 *src, uint32_t first, int nsrc) {
    NttJob j{};
    j.src = src;
    j.src_stride = C.N;
    j.nsrc = nsrc;
    j.prime = dst_prime;
    const u64 qd = C.all[dst_prime];
    for (int s = 0; s < nsrc; s++) {
        u64 hat_d = 1 % qd;
        for (int r = 0; r < nsrc; r++)
            if (r != s) hat_d = h_mulmod(hat_d, C.all[first + r] % qd, qd);
        j.c2[s] = hat_d;
        j.c2_sh[s] = h_shoup(hat_d, qd);
    }
    return j;
}

// Hybrid SwitchKey (Section 2.4.1) on B polynomials d(b, i), i <= l, NTT domain:
// ModUp each CRT digit to Q_l P, inner product with the key, ModDown by P.
// extra(b, c, i) (may return null) is added to component c of the result.
//
// rescale_after (l >= 1, K < 4): the result is rescaled by q_l as well, with
// the same arithmetic as rescale(keyswitch(...)) but one forward transform per
// remaining target instead of two.  By linearity of the NTT modulo q_i, for
// i < l
//   out_i = ((acc_i + P e_i) - NTT(P u_i)) (P q_l)^-1,
//   u_i   = sum_k y_k [p_k^-1]_{q_i} + [a_l]_{q_i} - [floor(P/2) P^-1 + floor(q_l/2)]_{q_i},
// where y_k are the scaled special limbs (step 4), e the extra term and a_l the
// coefficient-domain top limb of the unrescaled result plus floor(q_l/2), which
// the inverse transform of acc_l + P e_l yields with the conversion to q_l
// subtracted in its store.  P e is folded into the key inner product.
CtH Rec::keyswitch(int B, int l, const std::function<const u64 *(int, int)> &d, const Key &key,
                   const std::function<const u64 *(int, int, int)> &extra, bool rescale_after) {
    const int nl = l + 1, K = C.K(), ntg = nl + K, alpha = C.alpha;
    const bool fused = rescale_after && l >= 1 && K + 1 <= kMaxConvSrc;
    const int dnum = (nl + alpha - 1) / alpha;
    const size_t N = C.N;
    TREQUIRE(K >= 1 && K <= kMaxConvSrc && alpha <= kMaxConvSrc, TETRIS_EINVAL, "keyswitch: K or alpha too large");
    const int pieces = key.pieces;  // base-2^w pieces per one-prime digit (1: plain hybrid)
    TREQUIRE(pieces == 1 || alpha == 1, TETRIS_EINVAL, "keyswitch: base-2^w pieces need one-prime digits");
    const int nd = pieces == 1 ? dnum : nl * pieces;  // key digits this level uses
    TREQUIRE(nd <= key.dnum && nd <= kMaxKeyDigits, TETRIS_EINVAL, "keyswitch: key has too few digits");
    const int nQP = C.nqp();
    const std::string saved_prefix = prefix;
    prefix = "ks." + prefix;
    P.ks_count += 1;
    // algorithmic bytes of one batched keyswitch: B inputs, the key limbs it uses once, 2B outputs
    P.ks_bytes += ((double)B * nl + 2.0 * nd * ntg + 2.0 * B * nl) * N * 8;
    // 1. d -> coefficient domain, each limb already multiplied by its digit's
    //    [(Q_j/q_i)^-1]_{q_i} (folded with N^-1 into the transform's last store)
    BufPtr dcoef = pool().alloc((size_t)B * nl * N);
    {
        std::vector<NttJob> jobs;
        for (int i = 0; i < nl; i++) {
            const int lo = (i / alpha) * alpha, hi = std::min(nl, lo + alpha);
            const u64 qi = C.q[i];
            u64 hat = 1 % qi;
            for (int r = lo; r < hi; r++)
                if (r != i) hat = h_mulmod(hat, C.q[r] % qi, qi);
            NttJob proto{};
            proto.prime = i;
            proto.mul = h_mulmod(C.mods_host[i].ninv, h_invmod(hat, qi), qi);
            proto.mul_sh = h_shoup(proto.mul, qi);
            proto.conv_sub = 0;
            for (int b = 0; b < B; b++) {
                NttJob j = proto;
                j.src = d(b, i);
                j.dst = dcoef->ptr + ((size_t)b * nl + i) * N;
                jobs.push_back(j);
            }
        }
        ntt(true, jobs, LOAD_PLAIN, STORE_SCALED);
    }
    // 2. ModUp, first (column) pass: digit j -> every prime outside it, the
    //    conversion fused into the load; its constants carry R = 2^64 mod q_t
    //    for the Montgomery products of step 3.  With base-2^w pieces: piece
    //    (i, b) = (d_i >> w b) mod 2^w is the same small integer modulo every
    //    prime, so every target is its R-scaled transform (no conversion).
    BufPtr mu = pool().alloc((size_t)B * nd * ntg * N);
    auto mul = [&](int b, int j, int t) { return mu->ptr + (((size_t)b * nd + j) * ntg + t) * N; };
    if (pieces > 1) {
        std::vector<NttJob> jobs;
        for (int j = 0; j < nd; j++) {
            const int i = j / pieces, pc = j % pieces;
            for (int t = 0; t < ntg; t++) {
                const uint32_t gp = C.qp_prime(l, t);
                NttJob proto{};
                proto.prime = gp;
                proto.c2[0] = C.mods_host[gp].r64;
                proto.c2_sh[0] = C.mods_host[gp].r64_sh;
                proto.piece_shift = (uint32_t)(C.base2 * pc);
                proto.piece_mask = (C.base2 >= 64) ? ~0ull : ((1ull << C.base2) - 1);
                for (int b = 0; b < B; b++) {
                    NttJob jb = proto;
                    jb.src = dcoef->ptr + ((size_t)b * nl + i) * N;
                    jb.dst = mul(b, j, t);
                    jobs.push_back(jb);
                }
            }
        }
        ntt(false, jobs, LOAD_PIECE, STORE_PLAIN, -1, STORE_PLAIN, 1);
    } else {
        std::vector<NttJob> jobs;
        for (int j = 0; j < dnum; j++) {
            const int lo = j * alpha, hi = std::min(nl, (j + 1) * alpha);
            for (int t = 0; t < ntg; t++) {
                if (t >= lo && t < hi) continue;
                const uint32_t gp = C.qp_prime(l, t);
                const u64 qt = C.all[gp];
                NttJob proto = conv_job(gp, nullptr, lo, hi - lo);
                for (int s2 = 0; s2 < hi - lo; s2++) {
                    proto.c2[s2] = h_mulmod(proto.c2[s2], C.mods_host[gp].r64, qt);
                    proto.c2_sh[s2] = h_shoup(proto.c2[s2], qt);
                }
                for (int b = 0; b < B; b++) {
                    NttJob jb = proto;
                    jb.src = dcoef->ptr + ((size_t)b * nl + lo) * N;
                    jb.dst = mul(b, j, t);
                    jobs.push_back(jb);
                }
            }
        }
        ntt(false, jobs, LOAD_CONV_PRE, STORE_PLAIN, -1, STORE_PLAIN, 1);
    }
    // P mod q_i, floor(P/2) mod q_i
    auto pmod = [&](int i) {
        const u64 qi = C.q[i];
        u64 pm = 1 % qi;
        for (int k = 0; k < K; k++) pm = h_mulmod(pm, C.p[k] % qi, qi);
        return pm;
    };
    auto halfp = [&](int i) {
        const u64 qi = C.q[i];
        return h_mulmod((pmod(i) + qi - 1) % qi, h_invmod(2, qi), qi);
    };
    // 3. ModUp second (row) pass of every digit fused with the key inner
    //    product over Q_l P; blocks innermost, so the B jobs of one target read
    //    the same key limbs back to back and the key comes from DRAM once
    BufPtr acc = pool().alloc((size_t)B * 2 * ntg * N);
    auto accl = [&](int b, int c, int t) { return acc->ptr + (((size_t)b * 2 + c) * ntg + t) * N; };
    {
        std::vector<KsJob> jobs;
        for (int t = 0; t < ntg; t++)
            for (int b = 0; b < B; b++) {
                KsJob k{};
                const uint32_t gp = C.qp_prime(l, t);
                const u64 qt = C.all[gp];
                k.own = -1;
                for (int j = 0; j < nd; j++) {
                    const int lo = j * alpha, hi = std::min(nl, (j + 1) * alpha);
                    const bool own = pieces == 1 && t >= lo && t < hi;
                    if (own) k.own = j;
                    k.src[j] = own ? d(b, t) : mul(b, j, t);
                    k.key[j] = key.buf->ptr + ((size_t)j * nQP + gp) * 2 * N;
                }
                k.acc0 = accl(b, 0, t);
                k.acc1 = accl(b, 1, t);
                k.prime = gp;
                k.ndig = nd;
                k.qinv = h_inv64(qt);
                if (fused && t < nl && extra) {
                    k.ex0 = extra(b, 0, t);
                    k.ex1 = extra(b, 1, t);
                    k.pm = pmod(t);
                    k.pm_sh = h_shoup(k.pm, qt);
                }
                jobs.push_back(k);
            }
        ksup(jobs);
    }
    mu.reset();
    dcoef.reset();
    if (fused) {
        // 4'. the special limbs as in step 4 into slots 0..K-1 of each (b, c), and
        //     acc_l + P e_l into slot K as a_l = [x N^-1 P^-1 - sum_k y_k p_k^-1
        //     + floor(P/2) P^-1 + floor(q_l/2)]_{q_l} (its store reads slots 0..K-1)
        const int K1 = K + 1;
        BufPtr pc = pool().alloc((size_t)B * 2 * K1 * N);
        auto slot = [&](int b, int c, int k) { return pc->ptr + (((size_t)b * 2 + c) * K1 + k) * N; };
        std::vector<NttJob> jobs;
        for (int k = 0; k < K; k++) {
            const uint32_t gp = C.L() + 1 + k;
            const u64 pk = C.p[k];
            u64 hat = 1 % pk;
            for (int r = 0; r < K; r++)
                if (r != k) hat = h_mulmod(hat, C.p[r] % pk, pk);
            const u64 c1 = h_invmod(hat, pk);
            NttJob proto{};
            proto.prime = gp;
            proto.mul = h_mulmod(C.mods_host[gp].ninv, c1, pk);
            proto.mul_sh = h_shoup(proto.mul, pk);
            proto.conv_sub = h_mulmod((pk - 1) / 2, c1, pk);
            for (int b = 0; b < B; b++)
                for (int c = 0; c < 2; c++) {
                    NttJob j = proto;
                    j.src = accl(b, c, nl + k);
                    j.dst = slot(b, c, k);
                    jobs.push_back(j);
                }
        }
        const int split = (int)jobs.size();
        {
            const u64 ql = C.q[l];
            const u64 pinv = h_invmod(pmod(l), ql);
            NttJob proto{};
            proto.prime = l;
            proto.mul = h_mulmod(C.mods_host[l].ninv, pinv, ql);
            proto.mul_sh = h_shoup(proto.mul, ql);
            proto.conv_sub = (h_mulmod(halfp(l), pinv, ql) + (ql - 1) / 2) % ql;
            proto.nsrc = K;
            proto.src_stride = N;
            for (int k = 0; k < K; k++) {
                proto.c2[k] = h_invmod(C.p[k] % ql, ql);
                proto.c2_sh[k] = h_shoup(proto.c2[k], ql);
            }
            for (int b = 0; b < B; b++)
                for (int c = 0; c < 2; c++) {
                    NttJob j = proto;
                    j.src = accl(b, c, l);
                    j.dst = slot(b, c, K);
                    j.base = slot(b, c, 0);
                    jobs.push_back(j);
                }
        }
        ntt(true, jobs, LOAD_PLAIN, STORE_SCALED, split, STORE_SCALED_CONV);
        // 5'. targets i < l: load P u_i (K + 1 sources), out_i = (acc_i - x) (P q_l)^-1
        CtH out = new_ct(B, 2, l - 1);
        jobs.clear();
        const u64 ql = C.q[l];
        for (int i = 0; i < l; i++) {
            const u64 qi = C.q[i];
            const u64 pm = pmod(i);
            NttJob proto = conv_job(i, nullptr, C.L() + 1, K);
            proto.nsrc = K1;
            proto.c2[K] = pm;
            proto.c2_sh[K] = h_shoup(pm, qi);
            proto.conv_sub = (halfp(i) + h_mulmod(pm, ((ql - 1) / 2) % qi, qi)) % qi;
            proto.mul = h_invmod(h_mulmod(pm, ql % qi, qi), qi);
            proto.mul_sh = h_shoup(proto.mul, qi);
            for (int b = 0; b < B; b++)
                for (int c = 0; c < 2; c++) {
                    NttJob jb = proto;
                    jb.src = slot(b, c, 0);
                    jb.base = accl(b, c, i);
                    jb.dst = out.limb(b, c, i);
                    jobs.push_back(jb);
                }
        }
        ntt(false, jobs, LOAD_CONV_PRE, STORE_COMBINE);
        P.rescales++;
        prefix = saved_prefix;
        return out;
    }
    // 4. ModDown: special limbs to the coefficient domain, stored as
    //    [(c_k + floor(P/2)) * (P/p_k)^-1]_{p_k} (floor(P/2) = (p_k - 1)/2 mod p_k)
    BufPtr pc = pool().alloc((size_t)B * 2 * K * N);
    {
        std::vector<NttJob> jobs;
        for (int k = 0; k < K; k++) {
            const uint32_t gp = C.L() + 1 + k;
            const u64 pk = C.p[k];
            u64 hat = 1 % pk;
            for (int r = 0; r < K; r++)
                if (r != k) hat = h_mulmod(hat, C.p[r] % pk, pk);
            const u64 c1 = h_invmod(hat, pk);
            NttJob proto{};
            proto.prime = gp;
            proto.mul = h_mulmod(C.mods_host[gp].ninv, c1, pk);
            proto.mul_sh = h_shoup(proto.mul, pk);
            proto.conv_sub = h_mulmod((pk - 1) / 2, c1, pk);
            for (int b = 0; b < B; b++)
                for (int c = 0; c < 2; c++) {
                    NttJob j = proto;
                    j.src = accl(b, c, nl + k);
                    j.dst = pc->ptr + (((size_t)b * 2 + c) * K + k) * N;
                    jobs.push_back(j);
                }
        }
        ntt(true, jobs, LOAD_PLAIN, STORE_SCALED);
    }
    // 5. convert (c_P + floor(P/2)) to each q_i, subtract [floor(P/2)]_{q_i} from
    //    every coefficient, NTT, and combine: out_i = extra + (acc_i - x) * P^-1
    CtH out = new_ct(B, 2, l);
    {
        std::vector<NttJob> jobs;
        for (int i = 0; i < nl; i++) {
            const u64 qi = C.q[i];
            u64 pm = 1 % qi;
            for (int k = 0; k < K; k++) pm = h_mulmod(pm, C.p[k] % qi, qi);
            const u64 half = h_mulmod((pm + qi - 1) % qi, h_invmod(2, qi), qi);
            const u64 pinv = h_invmod(pm, qi);
            NttJob proto = conv_job(i, nullptr, C.L() + 1, K);
            proto.conv_sub = half;
            proto.mul = pinv;
            proto.mul_sh = h_shoup(pinv, qi);
            for (int b = 0; b < B; b++)
                for (int c = 0; c < 2; c++) {
                    NttJob jb = proto;
                    jb.src = pc->ptr + (((size_t)b * 2 + c) * K) * N;
                    jb.base = accl(b, c, i);
                    jb.extra = extra ? extra(b, c, i) : nullptr;
                    jb.dst = out.limb(b, c, i);
                    jobs.push_back(jb);
                }
        }
        ntt(false, jobs, LOAD_CONV_PRE, STORE_COMBINE);
    }
    prefix = saved_prefix;
    return out;
}

CtH Rec::relin(const CtH &t) {
    TREQUIRE(t.comps == 3, TETRIS_EINVAL, "relin: needs a degree-2 ciphertext");
    const Key &k = find_key(C, 0);
    CtH o = keyswitch(t.B, t.level, [&](int b, int i) { return (const u64 *)t.limb(b, 2, i); }, k,
                      [&](int b, int c, int i) { return (const u64 *)t.limb(b, c, i); });
    o.scale = t.scale;
    P.relins++;
    return o;
}

CtH Rec::relin_rescale(const CtH &t) {
    TREQUIRE(t.comps == 3, TETRIS_EINVAL, "relin: needs a degree-2 ciphertext");
    TREQUIRE(t.level >= 1, TETRIS_ELEVEL, "rescale at level 0");
    if (defer || C.K() + 1 > kMaxConvSrc) return rescale(relin(t));
    const Key &k = find_key(C, 0);
    CtH o = keyswitch(t.B, t.level, [&](int b, int i) { return (const u64 *)t.limb(b, 2, i); }, k,
                      [&](int b, int c, int i) { return (const u64 *)t.limb(b, c, i); }, true);
    o.scale = t.scale / (double)C.q[t.level];
    P.relins++;
    return o;
}

// A batched key switch's work buffers grow with its blocks (the ModUp output
// alone is blocks x dnum x (l + 1 + K) limbs), and launches of this many
// blocks already fill the GPU: batches stop there.
constexpr int kRelinBatchBlocks = 12;

std::vector<CtH> Rec::relin_rescale_many(const std::vector<CtH> &ts) {
    std::vector<CtH> outs;
    if (ts.empty()) return outs;
    bool same = true;
    for (const CtH &t : ts) same = same && t.level == ts[0].level && t.comps == 3;
    if (ts.size() == 1 || !same || defer || C.K() + 1 > kMaxConvSrc) {
        for (const CtH &t : ts) outs.push_back(relin_rescale(t));
        return outs;
    }
    int total = 0;
    for (const CtH &t : ts) total += t.B;
    if (total > kRelinBatchBlocks) {  // consecutive groups of at most kRelinBatchBlocks blocks
        std::vector<CtH> group;
        int gb = 0;
        auto flush = [&]() {
            for (CtH &o : relin_rescale_many(group)) outs.push_back(o);
            group.clear();
            gb = 0;
        };
        for (const CtH &t : ts) {
            if (!group.empty() && gb + t.B > kRelinBatchBlocks) flush();
            group.push_back(t);
            gb += t.B;
        }
        flush();
        return outs;
    }
    TREQUIRE(ts[0].level >= 1, TETRIS_ELEVEL, "rescale at level 0");
    // block b of the batch is block loc[b].second of ts[loc[b].first]
    std::vector<std::pair<int, int>> loc;
    for (size_t n = 0; n < ts.size(); n++)
        for (int b = 0; b < ts[n].B; b++) loc.push_back({(int)n, b});
    const Key &k = find_key(C, 0);
    CtH o = keyswitch((int)loc.size(), ts[0].level,
                      [&](int b, int i) { return (const u64 *)ts[loc[b].first].limb(loc[b].second, 2, i); }, k,
                      [&](int b, int c, int i) { return (const u64 *)ts[loc[b].first].limb(loc[b].second, c, i); },
                      true);
    int b0 = 0;
    for (const CtH &t : ts) {
        CtH v = view(o.buf, o.base + (size_t)b0 * o.bstride, t.B, o.comps, o.level, o.bstride, o.cstride,
                     t.scale / (double)C.q[t.level]);
        outs.push_back(v);
        b0 += t.B;
        P.relins++;
    }
    P.rescales += (int)ts.size() - 1;  // the key switch counted one; one per ciphertext
    return outs;
}

// Rescale (Section 2.5), per coefficient:
//   out_i = (a_i + [floor(q_l/2)]_{q_i} - [[a_l + floor(q_l/2)]_{q_l}]_{q_i}) * q_l^-1;
// the two constants are folded into the converted top limb before its NTT.
// With an integer factor f the input is f*a (rescale(mul_int(a, f))): f goes
// into the top limb's inverse-transform store, and for i < l
//   out_i = (a_i - NTT(f^-1 ([t]_{q_i} - [floor(q_l/2)]_{q_i}))) * f q_l^-1,
// t the converted top limb, which needs f invertible modulo every q_i.
CtH Rec::rescale(const CtH &a, int64_t factor) { return rescale_many({{a, factor}})[0]; }

// Independent rescales, each at its own level and factor, in one inverse and
// one forward transform (every job carries its own prime).
std::vector<CtH> Rec::rescale_many(const std::vector<std::pair<CtH, int64_t>> &items) {
    std::vector<CtH> outs(items.size());
    const size_t N = C.N;
    std::vector<size_t> idx;
    size_t words = 0;
    for (size_t n = 0; n < items.size(); n++) {
        const CtH &a = items[n].first;
        const int64_t factor = items[n].second;
        TREQUIRE(a.level >= 1, TETRIS_ELEVEL, "rescale at level 0");
        bool invertible = true;
        if (factor != 1)
            for (int i = 0; i <= a.level; i++) invertible = invertible && signed_mod(factor, C.q[i]) != 0;
        if (!invertible) {
            outs[n] = rescale(mul_int(a, factor));
            continue;
        }
        idx.push_back(n);
        words += (size_t)a.B * a.comps * N;
    }
    if (idx.empty()) return outs;
    // top limbs to the coefficient domain, stored as [f a_l + floor(q_l/2)]_{q_l}
    BufPtr tmp = pool().alloc(words);
    std::vector<NttJob> ji, jf;
    size_t off = 0;
    for (size_t n : idx) {
        const CtH &a = items[n].first;
        const int64_t factor = items[n].second;
        const int l = a.level;
        const u64 ql = C.q[l], half = (ql - 1) / 2;
        u64 *top = tmp->ptr + off;
        off += (size_t)a.B * a.comps * N;
        for (int b = 0; b < a.B; b++)
            for (int c = 0; c < a.comps; c++) {
                NttJob j{};
                j.src = a.limb(b, c, l);
                j.dst = top + ((size_t)b * a.comps + c) * N;
                j.prime = l;
                j.mul = h_mulmod(C.mods_host[l].ninv, signed_mod(factor, ql), ql);
                j.mul_sh = h_shoup(j.mul, ql);
                j.conv_sub = half;
                ji.push_back(j);
            }
        CtH o = new_ct(a.B, a.comps, l - 1);
        o.scale = a.scale / (double)C.q[l];
        for (int i = 0; i < l; i++) {
            const u64 qi = C.q[i];
            NttJob proto{};
            proto.prime = i;
            proto.conv_sub = half % qi;
            proto.mul = h_invmod(ql % qi, qi);
            if (factor != 1) {
                const u64 f = signed_mod(factor, qi), finv = h_invmod(f, qi);
                proto.c2[0] = finv;
                proto.c2_sh[0] = h_shoup(finv, qi);
                proto.conv_sub = h_mulmod(proto.conv_sub, finv, qi);
                proto.mul = h_mulmod(proto.mul, f, qi);
            }
            proto.mul_sh = h_shoup(proto.mul, qi);
            for (int b = 0; b < a.B; b++)
                for (int c = 0; c < a.comps; c++) {
                    NttJob jb = proto;
                    jb.src = top + ((size_t)b * a.comps + c) * N;
                    jb.base = a.limb(b, c, i);
                    jb.dst = o.limb(b, c, i);
                    jf.push_back(jb);
                }
        }
        outs[n] = o;
        P.rescales++;
    }
    ntt(true, ji, LOAD_PLAIN, STORE_SCALED);
    ntt(false, jf, LOAD_REDUCE, STORE_COMBINE);
    return outs;
}

CtH Rec::drop(const CtH &a, int level) {
    TREQUIRE(level <= a.level && level >= 0, TETRIS_ELEVEL, "drop: bad level");
    CtH o = a;
    o.level = level;
    return o;
}

CtH Rec::automorphism(const CtH &a, uint32_t g) {
    TREQUIRE(g & 1, TETRIS_EINVAL, "galois element must be odd");
    g &= (uint32_t)(2 * C.N - 1);
    CtH o = new_ct(a.B, a.comps, a.level);
    o.scale = a.scale;
    std::vector<AutJob> jobs;
    for (int b = 0; b < a.B; b++)
        for (int c = 0; c < a.comps; c++)
            for (int i = 0; i <= a.level; i++) jobs.push_back({a.limb(b, c, i), o.limb(b, c, i)});
    aut(jobs, g);
    return o;
}

// Automorphism then SwitchKey(phi(c1), swk_{phi(s)->s}) + (phi(c0), 0) (Appendix A.2).
CtH Rec::rotate(const CtH &a, uint32_t g) {
    TREQUIRE(a.comps == 2, TETRIS_EINVAL, "rotate: needs a degree-1 ciphertext");
    const Key &k = find_key(C, g & (uint32_t)(2 * C.N - 1));
    CtH t = automorphism(a, g);
    CtH o = keyswitch(t.B, t.level, [&](int b, int i) { return (const u64 *)t.limb(b, 1, i); }, k,
                      [&](int b, int c, int i) { return c == 0 ? (const u64 *)t.limb(b, 0, i) : (const u64 *)nullptr; });
    o.scale = a.scale;
    P.rotations++;
    return o;
}

CtH Rec::sum_batch(const CtH &a) {
    if (a.B == 1) return a;
    // pairwise tree of additions over the batch entries
    CtH cur = a;
    int n = a.B;
    while (n > 1) {
        int h = n / 2;
        CtH nx = new_ct((n + 1) / 2, a.comps, a.level);
        std::vector<EwJob> jobs;
        for (int k = 0; k < (n + 1) / 2; k++)
            for (int c = 0; c < a.comps; c++)
                for (int i = 0; i <= a.level; i++) {
                    if (k < h)
                        jobs.push_back(ewj(EW_ADD, i, nx.limb(k, c, i), cur.limb(k, c, i), cur.limb(k + h, c, i)));
                    else
                        jobs.push_back(ewj(EW_COPY, i, nx.limb(k, c, i), cur.limb(n - 1, c, i)));
                }
        ew(jobs);
        cur = nx;
        n = (n + 1) / 2;
    }
    cur.scale = a.scale;
    return cur;
}

// Move to level lt with the standard scale S[lt], applying a public factor:
// keep q_0..q_{lt+1}, multiply by floor(factor * S[lt] * q_{lt+1} / scale + 1/2), rescale.
CtH Rec::adjust(const CtH &a, int lt, double factor) { return adjust_many({{a, lt, factor}})[0]; }

// adjust_many on coefficient-domain ciphertexts, where the rescale is a per
// coefficient operation (the formula of rescale() with no transform); results
// stay in the coefficient domain.  Items already at their level are returned as they are.
std::vector<CtH> Rec::adjust_many_coef(const std::vector<AdjustItem> &items) {
    std::vector<CtH> outs(items.size());
    std::vector<EwJob> jobs;
    for (size_t n = 0; n < items.size(); n++) {
        const CtH &a = items[n].ct;
        const int lt = items[n].level;
        const double factor = items[n].factor;
        if (a.level == lt) {
            TREQUIRE(factor == 1.0 && a.scale == C.S[lt], TETRIS_EINVAL, "adjust at the same level");
            outs[n] = a;
            continue;
        }
        TREQUIRE(a.level > lt, TETRIS_ELEVEL, "input ciphertext level too low");
        const int64_t f = round_half_up(((factor * C.S[lt]) * (double)C.q[lt + 1]) / a.scale);
        const int l = lt + 1;
        const u64 ql = C.q[l], half = (ql - 1) / 2;
        CtH o = new_ct(a.B, a.comps, lt);
        o.scale = C.S[lt];
        for (int i = 0; i < l; i++) {
            const u64 qi = C.q[i];
            EwJob proto{};
            proto.op = EW_RESCALE_COEF;
            proto.prime = i;
            proto.prime2 = l;
            proto.k = signed_mod(f, qi);
            proto.k_sh = h_shoup(proto.k, qi);
            proto.k2 = signed_mod(f, ql);
            proto.k2_sh = h_shoup(proto.k2, ql);
            proto.k3 = h_invmod(ql % qi, qi);
            proto.k3_sh = h_shoup(proto.k3, qi);
            proto.k4 = half;
            proto.k5 = half % qi;
            for (int b = 0; b < a.B; b++)
                for (int c = 0; c < a.comps; c++) {
                    EwJob j = proto;
                    j.a = a.limb(b, c, i);
                    j.b = a.limb(b, c, l);
                    j.dst = o.limb(b, c, i);
                    jobs.push_back(j);
                }
        }
        outs[n] = o;
        P.rescales++;
    }
    ew(jobs);
    return outs;
}

// Independent adjusts recorded as one rescale_many.
std::vector<CtH> Rec::adjust_many(const std::vector<AdjustItem> &items) {
    std::vector<CtH> outs(items.size());
    std::vector<std::pair<CtH, int64_t>> rs;
    std::vector<size_t> where;
    for (size_t n = 0; n < items.size(); n++) {
        const CtH &a = items[n].ct;
        const int lt = items[n].level;
        const double factor = items[n].factor;
        if (a.level == lt) {
            TREQUIRE(factor == 1.0 && a.scale == C.S[lt], TETRIS_EINVAL, "adjust at the same level");
            outs[n] = a;
            continue;
        }
        TREQUIRE(a.level > lt, TETRIS_ELEVEL, "input ciphertext level too low");
        const int64_t cst = round_half_up(((factor * C.S[lt]) * (double)C.q[lt + 1]) / a.scale);
        rs.push_back({drop(a, lt + 1), cst});
        where.push_back(n);
    }
    std::vector<CtH> r = rescale_many(rs);
    for (size_t k = 0; k < where.size(); k++) {
        outs[where[k]] = r[k];
        outs[where[k]].scale = C.S[items[where[k]].level];
    }
    return outs;
}

CtH Rec::mul(const CtH &a, const CtH &b) {
    TREQUIRE(a.level == b.level, TETRIS_EINVAL, "mul: levels differ");
    CtH o = relin_rescale(tensor(a, b));
    o.scale = C.S[a.level - 1];
    return o;
}

}  // namespace tetris
