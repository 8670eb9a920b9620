// Context, recorded programs and the ciphertext-level recorder.
//
// Work is recorded once as a list of kernel launches whose per-limb job
// tables live in one device arena; the list is then replayed on a stream (or
// captured once into a CUDA graph and replayed).  Buffers are shared_ptrs
// into a pool: when the recorder drops the last handle, the memory returns to
// the pool's free list and later operations of the same program reuse it
// (launches run in program order on one stream, so reuse after the last use
// is safe).
#pragma once
#include <array>
#include <cmath>
#include <cstring>
#include <mutex>
#include <sstream>

#include "internal.h"
#include "../../include/tetris.h"

namespace tetris {

struct Key {
    BufPtr buf;      // NTT domain [dnum][nQP][N][2]: both components of a word side by side
    int dnum = 0;    // key digits: CRT digits times base-2^w pieces
    int pieces = 1;  // base-2^w pieces per one-prime digit (1: no decomposition)
};

struct Database {
    uint64_t records = 0;
    int attrs = 0;
    int blocks = 0;
    BufPtr pts;        // NTT domain [blocks][attrs][n_q][N]
    BufPtr mask_real;  // double[N] on device (bytes in words), or null
};

struct Program;

struct KernelStat {
    uint32_t launches = 0;
    double ms = 0, bytes = 0, modmuls = 0, units = 0;
};

struct Ctx {
    int device = 0;
    int log_n = 0;
    size_t N = 0;
    std::vector<u64> q, p, all, psi;
    double scale = 0;
    std::vector<double> S;  // standard scales
    double pt_scale = 0;
    std::vector<ModInfo> mods_host;
    BufPtr tables;          // tw, itw (twiddle + companion pairs), mods, encoder tables
    NttTables nt{};
    const double *enc_tw = nullptr;
    Pool pool;
    int alpha = 0;
    int base2 = 0;  // bits w of the base-2^w decomposition of one-prime key-switch digits (0: none)
    Key relin;
    std::map<uint32_t, Key> rot;
    std::map<uint32_t, Database> dbs;
    uint32_t next_db = 1;
    cudaStream_t stream = nullptr;
    int blocks_per_launch = 0;
    int use_graph = 1;
    int profile = 0;
    int query_stage = 0;    // TETRIS_OPT_QUERY_STAGE: 0 the whole query, else the stage whose values are returned
    int debug_checks = 0;   // TETRIS_OPT_DEBUG_CHECKS: bounds-check every recorded job on the host
    int persistent = 0;     // TETRIS_OPT_PERSISTENT: NTT passes and fused row passes as persistent launches
    uint64_t checked_ranges = 0;  // device ranges checked so far (debug)
    std::map<std::string, KernelStat> stats;
    void *server = nullptr;  // serve.cu
    std::map<std::string, std::unique_ptr<Program>> programs;

    int L() const { return (int)q.size() - 1; }
    int K() const { return (int)p.size(); }
    int nqp() const { return (int)all.size(); }
    // prime index of limb t of a buffer over q_0..q_l, p_0..p_{K-1}
    uint32_t qp_prime(int l, int t) const { return t <= l ? (uint32_t)t : (uint32_t)(L() + 1 + (t - l - 1)); }
    size_t bytes_held() const;
};

struct CtH {
    BufPtr buf;
    u64 *base = nullptr;
    int level = -1, comps = 0, B = 0;
    size_t bstride = 0, cstride = 0;
    double scale = 0;
    size_t N = 0;
    u64 *limb(int b, int c, int i) const {
        return base + (size_t)(B == 1 ? 0 : b) * bstride + (size_t)c * cstride + (size_t)i * N;
    }
};

// One recorded kernel launch: the launcher, a kind tag for profiling and the
// algorithmic bytes it must move (distinct inputs read once + outputs written).
struct Launch {
    std::function<void(cudaStream_t, const uint8_t *)> fn;
    std::string kind;
    double bytes = 0;
    double modmuls = 0;  // algorithmic modular multiplications (butterflies, conversion and key products)
    bool kernel = true;  // false: a stream wait, neither timed nor counted
    double units = 0;    // limb jobs (N-word limbs) the launch processes
};

// A device staging slot for one input: rows (ciphertext components) of
// row_words words (the limbs the program uses), copied from a source whose
// rows lie src_pitch words apart (the caller's [comps][level+1][N] layout,
// of which only the first limbs of each component are read).
struct InSlot {
    u64 *dst = nullptr;
    size_t rows = 1, row_words = 0, src_pitch = 0;
    size_t words() const { return rows * row_words; }
    // enqueue the copy of src into dst (host-to-device or device-to-device)
    void copy_from(const void *src, cudaMemcpyKind kind, cudaStream_t s) const;
};

struct Program {
    Ctx *ctx = nullptr;
    Pool pool;
    std::vector<uint8_t> arena;
    BufPtr arena_dev;
    std::vector<Launch> launches;
    int kernel_launches = 0;
    std::vector<BufPtr> hold;
    // query programs: input staging slots (device pointer, words) and output
    std::vector<InSlot> in_slots;
    BufPtr out_buf;
    u64 *out_base = nullptr;
    size_t out_words = 0;
    int out_level = 0, out_comps = 0;
    double out_scale = 0;
    // Inputs arrive in groups: in_slots[0, groups[0].first) are copied before the
    // program runs; each later group may arrive while it runs (copy_inputs sends
    // the groups in order on a side stream, recording each group's event), and
    // the program waits for a group's event just before its first use.  A CUDA
    // graph is captured per segment between two waits.
    struct InGroup {
        size_t first = 0;           // its first slot (it ends at the next group's)
        size_t wait_at = 0;         // index of its wait in launches
        cudaEvent_t ev = nullptr;
        cudaGraph_t graph = nullptr;        // the launches after its wait
        cudaGraphExec_t exec = nullptr;
    };
    std::vector<InGroup> groups;
    cudaEvent_t early_ev = nullptr;
    cudaStream_t side = nullptr;
    cudaGraph_t graph = nullptr;  // the launches before the first wait
    cudaGraphExec_t exec = nullptr;
    // counters
    int relins = 0, rescales = 0, rotations = 0;
    int ks_count = 0;
    size_t tab_off = SIZE_MAX;  // the context's table set in the arena (persistent launches)
    double ks_bytes = 0;  // per keyswitch: input d + key limbs used + output, summed

    ~Program();
    size_t add_jobs(const void *p, size_t bytes);
    void finalize();
    void run(cudaStream_t s);
    void run_graph(cudaStream_t s);
    void run_profiled(cudaStream_t s, std::map<std::string, KernelStat> &stats);
    void add_launch(std::function<void(cudaStream_t, const uint8_t *)> fn, const std::string &kind, double bytes,
                    double modmuls = 0, double units = 0);
    // from here on the program may use in_slots[first..] (groups in slot order)
    void add_input_wait(size_t first);
    // copies srcs[i] into in_slots[i] (kind H2D or D2D), the later groups on the side stream
    void copy_inputs(const std::vector<const void *> &srcs, cudaMemcpyKind kind, cudaStream_t s);
};

// A launch recorded but not yet emitted (batch schedules merge these): the
// kernel, its parameters and its job table.
struct Deferred {
    int type = 0;  // 0 NTT, 1 elementwise, 2 automorphism, 3 ModUp row pass + key inner product, 4 lincomb, 5 reduce
    bool inverse = false;
    int load_mode = 0, store_mode = 0, passes = 3;
    uint32_t galois = 0;
    size_t job_size = 0;
    std::vector<uint8_t> jobs;
    std::string kind;
    double bytes = 0;
    std::string merge_key() const {
        return std::to_string(type) + ":" + std::to_string(inverse) + ":" + std::to_string(load_mode) + ":" +
               std::to_string(store_mode) + ":" + std::to_string(passes) + ":" + std::to_string(galois) + ":" + kind;
    }
};

class Rec {
  public:
    Rec(Ctx &c, Program &p) : C(c), P(p) {}
    Ctx &C;
    Program &P;
    std::string prefix;                     // prepended to the kind of every launch recorded (profiling scopes)
    std::vector<Deferred> *defer = nullptr; // when set, launches are collected here instead of emitted
    Pool *pool_override = nullptr;          // when set, buffers come from (and return to) this pool
    bool persistent = false;                // NTT passes and fused row passes as persistent launches
    Pool &pool() { return pool_override ? *pool_override : P.pool; }
    void emit(const Deferred &d);           // turn a collected launch into a real one

    CtH new_ct(int B, int comps, int level);
    CtH view(const BufPtr &buf, u64 *base, int B, int comps, int level, size_t bstride, size_t cstride, double scale);

    // split >= 0: the second pass stores jobs[0, split) with store_mode, then
    // jobs[split, n) with store_mode_b (a later launch, so it may read the former)
    // passes: 1 = first pass only, 2 = second only, 3 = both
    void ntt(bool inverse, const std::vector<NttJob> &jobs, int load_mode, int store_mode, int split = -1,
             int store_mode_b = STORE_PLAIN, int passes = 3);
    void ew(const std::vector<EwJob> &jobs);
    void aut(const std::vector<AutJob> &jobs, uint32_t g);
    void ksup(const std::vector<KsJob> &jobs);
    void lin(const std::vector<LinJob> &jobs);
    void red(const std::vector<RedJob> &jobs);

    // ciphertext operations (NTT domain)
    void to_ntt(const CtH &a);           // in place, coefficient -> NTT
    CtH from_ntt(const CtH &a);          // new buffer, NTT -> coefficient
    CtH add(const CtH &a, const CtH &b);
    CtH sub(const CtH &a, const CtH &b);
    CtH mul_int(const CtH &a, int64_t c);
    CtH add_int(const CtH &a, int64_t c);
    CtH mul_plain(const CtH &a, const u64 *pt_limb0, size_t pt_bstride);
    CtH tensor(const CtH &a, const CtH &b);
    CtH tensor_add(const CtH &acc, const CtH &a, const CtH &b);  // acc + a (x) b
    // rescale_after: return the result rescaled by q_l (relin_rescale), exactly
    // as rescale(keyswitch(...)) computes it
    CtH keyswitch(int B, int l, const std::function<const u64 *(int, int)> &d, const Key &key,
                  const std::function<const u64 *(int, int, int)> &extra, bool rescale_after = false);
    CtH relin(const CtH &t3);
    CtH relin_rescale(const CtH &t3);    // rescale(relin(t3)) in one pass over the targets
    // independent degree-2 ciphertexts at one level, relinearised and rescaled by one
    // batched key switch (their blocks side by side); each result as relin_rescale's
    std::vector<CtH> relin_rescale_many(const std::vector<CtH> &ts);
    CtH rescale(const CtH &a, int64_t factor = 1);  // rescale(mul_int(a, factor))
    std::vector<CtH> rescale_many(const std::vector<std::pair<CtH, int64_t>> &items);
    CtH drop(const CtH &a, int level);
    CtH automorphism(const CtH &a, uint32_t g);
    CtH rotate(const CtH &a, uint32_t g);
    CtH sum_batch(const CtH &a);
    CtH adjust(const CtH &a, int lt, double factor);
    struct AdjustItem {
        CtH ct;
        int level;
        double factor;
    };
    std::vector<CtH> adjust_many(const std::vector<AdjustItem> &items);
    std::vector<CtH> adjust_many_coef(const std::vector<AdjustItem> &items);  // coefficient domain in and out
    CtH mul(const CtH &a, const CtH &b);

  private:
    NttJob conv_job(uint32_t dst_prime, const u64 *src, uint32_t first_src_prime, int nsrc);
    size_t tab_offset();  // the context's table set in the program arena (persistent launches)
    // debug checks (TETRIS_OPT_DEBUG_CHECKS): every range a job reads or writes
    // lies inside a live allocation of the context, the program or the item
    bool emitting_ = false;  // jobs already checked when they were deferred
    bool checking() const { return C.debug_checks && !emitting_; }
    void check_range(const void *p, size_t words, const std::string &what);
    void check_prime(uint32_t prime, const std::string &what);
    void check(const std::vector<NttJob> &jobs, int load_mode, int store_mode);
    void check(const std::vector<EwJob> &jobs);
    void check(const std::vector<AutJob> &jobs);
    void check(const std::vector<KsJob> &jobs);
    void check(const std::vector<LinJob> &jobs);
    void check(const std::vector<RedJob> &jobs);
};

int64_t round_half_up(double x);
// c mod q in [0, q) for a signed c
inline u64 signed_mod(int64_t c, u64 q) { return c >= 0 ? (u64)c % q : q - 1 - (u64)(-(c + 1)) % q; }
const Key &find_key(const Ctx &c, uint32_t galois);

// Shape of a query: what a recorded program depends on.
struct QuerySpec {
    int attrs = 0, degree = 0;
    std::vector<int> c_level;
    std::vector<double> c_scale;
    int t_level = 0;
    double t_scale = 0;
    std::vector<std::vector<double>> stages;   // per stage: coefficients of x, x^3, ... (4 or 8)
    int bpl = 0;
    int loge = 3;                // NTT register-group width (log2 elements per thread)
    uint64_t total_records = 0;  // 0: the database's own record count
    int stage = 0;               // 0: the whole query; 1..4: stop after x, y, y - t or the step values
    int persistent = 0;          // persistent NTT / fused row-pass launches
    // global threshold (none when gstages is empty): t1's level and scale
    int g_level = 0;
    double g_scale = 0;
    std::vector<std::vector<double>> gstages;
    std::string key(uint32_t db) const {
        std::ostringstream o;
        o << "q" << db << ":" << attrs << ":" << degree << ":" << bpl << ":" << loge << ":" << t_level << ":"
          << total_records << ":" << stage << ":" << persistent << ":";
        auto bits = [&](double v) {
            uint64_t b;
            std::memcpy(&b, &v, 8);
            o << std::hex << b << std::dec << ",";
        };
        bits(t_scale);
        for (size_t i = 0; i < c_level.size(); i++) {
            o << c_level[i] << "/";
            bits(c_scale[i]);
        }
        for (auto &s : stages)
            for (double v : s) bits(v);
        if (!gstages.empty()) {
            o << "g" << g_level << ":";
            bits(g_scale);
            for (auto &s : gstages)
                for (double v : s) bits(v);
        }
        return o.str();
    }
};

// query.cu
std::unique_ptr<Program> record_query(Ctx &C, const Database &db, const QuerySpec &q);
QuerySpec spec_of(const Ctx &C, const Database &db, const tetris_query *q);
std::vector<const tetris_ct_in *> query_inputs(const tetris_query *q);  // in input-slot order
// the input slots a query program copies, in input-slot order (dst unset):
// only the limbs the circuit reads of each input
std::vector<InSlot> query_slot_shapes(const Ctx &C, const Database &db, const QuerySpec &q);
void evaluate_query(Ctx &C, uint32_t db, const tetris_query *q, tetris_ct_out *out, cudaStream_t s, bool device);
void plan_info(Ctx &C, uint32_t db, uint32_t degree, uint32_t stages, tetris_plan_info *out);
void drop_programs_of_db(Ctx &C, uint32_t db);
void reduce_sum(Ctx &C, u64 *data, int level, int ncomp, cudaStream_t s);
void autotune(Ctx &C, uint32_t db, const tetris_query *q, int reps, std::vector<tetris_tune_entry> &out);

// serve.cu
void serve_start(Ctx &C, size_t budget, uint32_t max_inflight);
uint64_t serve_submit(Ctx &C, uint32_t db, const tetris_query *q);
int serve_poll(Ctx &C, uint64_t ticket, tetris_ct_out *out, uint32_t timeout_ms);
void serve_stats(Ctx &C, tetris_serve_stats *st, bool reset);
void serve_cancel(Ctx &C, uint64_t ticket);
void serve_stop(Ctx &C);

// batch.cu
void batch_run(const tetris_batch_item *items, uint32_t n, int schedule, int *used, double *device_ms);

// noalloc.cu
void rescale_ntt_noalloc(Ctx &C, const u64 *in, u64 *out, int level, int ncomp, cudaStream_t s);
size_t noalloc_scratch_bytes();

// repack.cu
void repack(Ctx &C, const u64 *cts, uint32_t count, int level, double scale, u64 *out, cudaStream_t s, bool device);

// pfe.cu
void pfe_scores(Ctx &C, const u64 *u, uint32_t m, const uint32_t *exps, uint64_t p, u64 *out, cudaStream_t s);

}  // namespace tetris

// the opaque handle of the C ABI
struct tetris_ctx {
    tetris::Ctx c;
};
