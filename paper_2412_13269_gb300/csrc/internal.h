// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <atomic>

#include <cstdint>
#include <functional>
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "modarith.cuh"

namespace tetris {

constexpr int kMaxPrimes = 64;
constexpr int kMaxConvSrc = 4;   // primes per digit (alpha) and special primes (K) at most

// ---------------------------------------------------------------------------
// Errors: thrown inside the library, converted to a status at the C ABI.
// ---------------------------------------------------------------------------
struct Error : std::runtime_error {
    int code;
    Error(int c, const std::string &m) : std::runtime_error(m), code(c) {}
};
void set_last_error(const std::string &msg);
#define TCHECK_CUDA(x)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (x);                                                                 \
        if (e_ != cudaSuccess)                                                                \
            throw ::tetris::Error(-3, std::string(#x) + ": " + cudaGetErrorString(e_));        \
    } while (0)
#define TREQUIRE(cond, code, msg)                              \
    do {                                                       \
        if (!(cond)) throw ::tetris::Error((code), (msg));     \
    } while (0)

// ---------------------------------------------------------------------------
// Host modular arithmetic (hostmath.cu)
// ---------------------------------------------------------------------------
u64 h_mulmod(u64 a, u64 b, u64 q);
u64 h_powmod(u64 a, u64 e, u64 q);
u64 h_invmod(u64 a, u64 q);
u64 h_shoup(u64 w, u64 q);  // floor(w * 2^64 / q)
u64 h_inv64(u64 q);          // q^-1 mod 2^64 (q odd)
bool h_is_prime(u64 n);
u64 h_primitive_2n_root(u64 q, u64 n);
std::vector<u64> h_gen_primes(int bits, int count, int cong_log2, const std::vector<u64> &exclude);
uint32_t bitrev(uint32_t x, int bits);

// ---------------------------------------------------------------------------
// Device memory: buffers owned through shared_ptr; a size-keyed free list
// lets a recorded program reuse memory after a buffer's last use.
// ---------------------------------------------------------------------------
struct DevBuf {
    u64 *ptr = nullptr;
    size_t words = 0;
};
using BufPtr = std::shared_ptr<DevBuf>;

// With the environment variable TETRIS_GUARD_WORDS set when a pool is made,
// every buffer it allocates is framed by kGuardWords words of a known pattern
// on each side; check_guards() reads them back.
constexpr size_t kGuardWords = 32;
constexpr unsigned char kGuardByte = 0xA5;

class Pool {
  public:
    Pool();
    ~Pool();
    // fresh: a new device buffer, never one freed earlier (the job arena of a
    // recorded program: buffers freed during recording are still used by its launches)
    BufPtr alloc(size_t words, bool fresh = false);
    size_t bytes_held() const { return held_; }
    void trim();
    // true iff [p, p + words) lies inside one buffer of this pool
    bool contains(const void *p, size_t words) const;
    // buffers whose guard words were overwritten (each as "ptr:side"); empty without guards
    std::vector<std::string> check_guards() const;
    // overwrite one guard word of the first buffer (a self-test of check_guards)
    void plant_guard_fault();
    bool guarded() const { return guard_; }

  private:
    std::multimap<size_t, u64 *> free_;
    std::vector<std::pair<u64 *, size_t>> all_;  // user pointer and words
    size_t held_ = 0;
    bool guard_ = false;
    std::shared_ptr<int> alive_ = std::make_shared<int>(1);
};

// ---------------------------------------------------------------------------
// Kernel job descriptors
// ---------------------------------------------------------------------------
// LOAD_CONV_PRE: sum_s src_s * c2_s - conv_sub (sources already scaled by their
//                factor [(Q/q_s)^-1]_{q_s}, see STORE_SCALED; each product a lazy
//                Shoup product, so nsrc * 2q < 2^64)
// LOAD_REDUCE:   [src * c]_{q_dst} - conv_sub (a single source of another prime;
//                c = c2[0] when nonzero, else 1)
// LOAD_INT64:    signed 64-bit integers reduced modulo q_dst
// LOAD_PIECE:    ((src >> shift) & mask) * c2[0] mod q_dst (a base-2^w piece of a
//                coefficient-domain residue, times the constant c2[0])
// Forward transforms take every load mode; inverse transforms load plain limbs.
enum LoadMode { LOAD_PLAIN = 0, LOAD_INT64 = 2, LOAD_CONV_PRE = 3, LOAD_REDUCE = 4, LOAD_PIECE = 5 };
// STORE_COMBINE (forward only): (extra ? extra : 0) + (base - x) * mul.
// STORE_SCALED (inverse only): x * mul + conv_sub, where mul already carries
// N^-1; it precomputes the per-source factor of a following conversion.
// STORE_SCALED_CONV (inverse only): x * mul + conv_sub - sum_s base_s * c2_s, the
// nsrc sources base + s*src_stride in the coefficient domain.
enum StoreMode { STORE_PLAIN = 0, STORE_COMBINE = 1, STORE_SCALED = 2, STORE_SCALED_CONV = 3 };

// One limb transform: src -> dst (in place when equal), prime index `prime`.
struct NttJob {
    const u64 *src;
    u64 *dst;
    const u64 *base;
    const u64 *extra;
    uint32_t prime;
    uint32_t nsrc;
    uint64_t src_stride;
    u64 c2[kMaxConvSrc], c2_sh[kMaxConvSrc];  // c2_sh: Shoup companions of c2 modulo q_dst
    // forward conversion loads: c2 and conv_sub times the first butterfly
    // stage's twiddle psi^(N/2) (filled in by the recorder)
    u64 c2w[kMaxConvSrc], c2w_sh[kMaxConvSrc], conv_sub_w;
    u64 conv_sub, mul, mul_sh;
    u64 mul_w, mul_w_sh;                      // inverse scaled stores: mul times the last stage's twiddle psi^-(N/2)
    u64 piece_mask;                           // LOAD_PIECE
    uint32_t piece_shift;
    uint32_t tab;                             // launches over several ring degrees: the job's table set
};

struct NttTables {
    const u64 *tw;      // [nprimes][N][2]: psi^brv(k) and its Shoup companion
    const u64 *itw;     // [nprimes][N][2]: psi^-brv(k) and its Shoup companion
    const ModInfo *mods;
    int loge = 3;       // log2 of the elements a thread holds (3 or 4)
};

// Launches whose jobs come from contexts of different ring degrees (batches
// of uneven jobs): each job names its context's table set, an entry of a
// device array of these.
constexpr int kMaxTabs = 4;
struct TabEntry {
    NttTables t;
    int log_n = 0;
    int pad = 0;
};

// launchers (ntt.cu)
// pass: 0 = first pass only, 1 = second pass only, -1 = both
void launch_ntt(bool inverse, int log_n, const NttTables &t, const NttJob *jobs_dev, int njobs, int load_mode,
                int store_mode, cudaStream_t s, int pass = -1);

// ---------------------------------------------------------------------------
// Elementwise kernels (elementwise.cu).  A "limb list" kernel walks njobs
// limbs of N words; per-limb pointers and constants come from a job table.
// ---------------------------------------------------------------------------
enum EwOp {
    EW_ADD = 0,       // dst = a + b
    EW_SUB = 1,       // dst = a - b
    EW_MUL = 2,       // dst = a * b (variable)
    EW_MUL_CONST = 3, // dst = a * k (k, k_sh per limb)
    EW_ADD_CONST = 4, // dst = a + k
    EW_NEG = 5,       // dst = -a
    EW_COPY = 6,      // dst = a
    EW_FMA = 7,       // dst = a * b + c
    EW_TENSOR = 8,    // a0,a1,b0,b1 -> d0,d1,d2 (pointers a,b,c,d with strides)
    EW_ADD_MUL_CONST = 9, // dst = b + k * a  (used by key generation)
    EW_REDUCE = 10,       // dst = a mod q for any 64-bit a
    EW_TENSOR_ACC = 11,   // tensor of (a, a1) and (b, b1) plus the degree-2 ciphertext (c, c1, c2)
    EW_RESCALE_COEF = 12  // coefficient domain: dst = (k a - [[k2 b + k4]_{q2}]_q + k5) * k3, b the top
                          // limb modulo q2 = prime2 (rescale of k * ciphertext by q2)
};
struct EwJob {
    const u64 *a, *b, *c;
    u64 *dst;
    uint32_t prime;
    uint32_t op;
    u64 k, k_sh;
    // tensor: second components
    const u64 *a1, *b1;
    u64 *d1, *d2;
    // tensor with accumulation: components 1 and 2 of the added ciphertext (c is component 0)
    const u64 *c1, *c2;
    // coefficient-domain rescale: second prime and constants
    u64 k2, k2_sh, k3, k3_sh, k4, k5;
    uint32_t prime2;
    uint32_t tab;  // launches over several ring degrees: the job's table set
};
// tabs (device, may be null): jobs of several ring degrees, each reading its own
// log N and primes from tabs[job.tab]; log_n is then the largest of them
void launch_ew(const EwJob *jobs_dev, int njobs, int log_n, const ModInfo *mods, cudaStream_t s,
               const TabEntry *tabs = nullptr);
// every job EW_TENSOR or EW_TENSOR_ACC
void launch_tensor(const EwJob *jobs_dev, int njobs, int log_n, const ModInfo *mods, cudaStream_t s,
                   const TabEntry *tabs = nullptr);

// automorphism in the NTT domain: dst[k] = src[perm_g(k)]
struct AutJob {
    const u64 *src;
    u64 *dst;
    uint32_t g;    // Galois element (launches over several ring degrees; else the launch's)
    uint32_t tab;  // launches over several ring degrees: the job's table set
};
void launch_automorphism(const AutJob *jobs_dev, int njobs, int log_n, uint32_t galois, cudaStream_t s);
// key layout conversion: [rows][2][nl][n] limbs <-> [rows][nl][n] pairs (component 0, component 1)
void launch_interleave_pairs(u64 *limbs, u64 *pairs, size_t rows, size_t nl, size_t n, bool to_pairs,
                             cudaStream_t s);
// per-job Galois element and ring degree (tabs[job.tab].log_n); max_log_n the largest
void launch_automorphism_multi(const AutJob *jobs_dev, int njobs, const TabEntry *tabs, int max_log_n, cudaStream_t s);

// ModUp second pass fused with the key inner product (ntt.cu), one job per
// (target limb t, block): for every digit j, x_j is the row pass of src[j] (the
// ModUp column-pass output, whose conversion constants carry R = 2^64 mod q_t)
// or, for the digit own that holds t, R * src[own] (the input limb, NTT domain);
// then acc_c[t] = sum_j x_j key_j[c][t] R^-1 (Montgomery products) + pm ex_c[t].
constexpr int kMaxKeyDigits = 64;
struct KsJob {
    const u64 *src[kMaxKeyDigits];
    const u64 *key[kMaxKeyDigits];  // digit j's key limb for prime t: N (component 0, component 1) pairs
    u64 *acc0, *acc1;
    const u64 *ex0, *ex1;  // optional: P e folded in (pm = [P]_{q_t}, Shoup companion pm_sh)
    u64 pm, pm_sh;
    u64 qinv;              // q_t^-1 mod 2^64
    uint32_t prime, ndig;
    int32_t own;           // digit whose source is the NTT-domain input, -1 if none
    uint32_t tab;          // launches over several ring degrees: the job's table set
};
void launch_keyswitch_up(int log_n, const NttTables &t, const KsJob *jobs_dev, int njobs, cudaStream_t s);

// Persistent launches over jobs of several ring degrees (log N in [14, 16]):
// job j takes tiles [tile_start[j], tile_start[j+1]) of the pass (device array
// of njobs + 1 entries); a grid of resident CTAs walks the tiles and each tile
// reads its job's table set tabs[job.tab] (device).  One launch per pass.
int ntt_pass_tiles(int log_n, bool col);  // tiles of one limb in a column or row pass
void launch_ntt_pass_multi(bool inverse, int pass, const TabEntry *tabs, const NttJob *jobs_dev,
                           const uint32_t *tile_start, int njobs, int total_tiles, int load_mode, int store_mode,
                           cudaStream_t s);
int keyswitch_up_tiles(int log_n);
void launch_keyswitch_up_multi(const TabEntry *tabs, const KsJob *jobs_dev, const uint32_t *tile_start, int njobs,
                               int total_tiles, cudaStream_t s);

// linear combination: dst_c[limb] = sum_j pt_j[limb] * w_j[c][limb], c = 0,1
struct LinJob {
    const u64 *pt;      // first attribute's plaintext limb
    uint64_t pt_stride; // words between attributes
    const u64 *w0, *w1; // first attribute's ciphertext limbs
    uint64_t w_stride;  // words between attributes
    u64 *d0, *d1;
    uint32_t prime;
    uint32_t nattr;
};
void launch_lincomb(const LinJob *jobs_dev, int njobs, int log_n, const ModInfo *mods, cudaStream_t s);

// int64 coefficients -> residues modulo a prime
struct RedJob {
    const int64_t *src;
    u64 *dst;
    uint32_t prime;
};
void launch_reduce_i64(const RedJob *jobs_dev, int njobs, int log_n, const ModInfo *mods, cudaStream_t s);

// measured lazy-Shoup modular multiplications per second (G/s) on the current device
double modmul_peak_probe();

// Dynamic shared memory above 48 KB needs an opt-in per kernel and device:
// done once for the current device (a bit per device in done), safe to race
// from several threads (they all set the same value).
void opt_in_smem(const void *func, int bytes, std::atomic<uint64_t> &done);
// the current device's SM count (queried once per device)
int sm_count();

// ---------------------------------------------------------------------------
// FP64 encoder (encode.cu)
// ---------------------------------------------------------------------------
// slots [batch][n_slots] (real) -> m [batch][N] real coefficients
void encode_real_batch(const double *slots, double *m, int batch, int log_n, const double *twid_dev,
                       double *work, cudaStream_t s);
// database columns: vals u8 [records][attrs] -> slots [blocks][attrs][n_slots]
void db_slots(const uint8_t *vals, uint64_t records, int attrs, int blocks, int log_n, double *slots,
              cudaStream_t s);
// m [batch][N] -> int64 floor(scale * m + 1/2)
void round_scale(const double *m, int64_t *out, size_t count, double scale, cudaStream_t s);

}  // namespace tetris
