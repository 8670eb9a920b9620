/*
 * tetris.h -- C ABI of the GB300 library for the server side of the TETRIS
 * private functional exploration (arXiv 2412.13269): RNS-CKKS evaluation of
 * an encrypted query over a plaintext database.
 *
 * Paper references are to that paper's sections, equations, algorithms and
 * tables.
 *
 * Conventions (every entry point):
 *   - Returns a tetris_status (0 on success, negative on error); nothing is
 *     thrown across the ABI.  tetris_last_error() gives a message for the
 *     calling thread's last failure.  An error leaves the context usable.
 *   - Host buffers passed in are owned by the caller, read during the call
 *     and not retained.  Output host buffers are owned by the caller.
 *   - Polynomials at the boundary are in the coefficient domain: residues in
 *     [0, q) of the coefficients of X^0 .. X^{N-1}, one limb of N uint64 per
 *     prime, limbs in prime order.  A ciphertext at level l is
 *     [ncomp][l+1][N] uint64 (components c0, c1[, c2]), modulo q_0 .. q_l.
 *   - Device state (keys, databases, work buffers) is owned by the context.
 *   - Not thread-safe per context: one thread drives a context at a time.
 */
#ifndef TETRIS_H
#define TETRIS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tetris_ctx tetris_ctx;

typedef enum {
    TETRIS_OK = 0,
    TETRIS_EINVAL = -1,     /* bad argument: size, layout, level, scale */
    TETRIS_ENOMEM = -2,     /* device allocation failed */
    TETRIS_ECUDA = -3,      /* CUDA runtime error */
    TETRIS_ELEVEL = -4,     /* circuit needs more levels than the ciphertexts have */
    TETRIS_ENOTFOUND = -5,  /* unknown handle or missing key */
    TETRIS_ETIMEOUT = -6,   /* poll deadline passed */
    TETRIS_EBUSY = -7       /* admission refused: not enough device memory now */
} tetris_status;

/* ---------------------------------------------------------------------------
 * Context.  The ring R_Q = Z_Q[X]/(X^N + 1) of Section 2.2 with
 * Q = q_0 ... q_{n_q-1} (RNS, q_0 first and dropped last by rescale) and the
 * special modulus P = p_0 ... p_{n_p-1} of SwitchKey (Section 2.4.1).
 * Every prime must be below 2^61 and = 1 mod 2N; all distinct.  log_n in
 * [10, 16].  scale is Delta of fresh ciphertexts (Section 2.5).  device is
 * the CUDA ordinal.  The context owns its device memory until destroyed.
 * ------------------------------------------------------------------------- */
int tetris_ctx_create(tetris_ctx **out, uint32_t log_n,
                      const uint64_t *q, uint32_t n_q,
                      const uint64_t *p, uint32_t n_p,
                      double scale, int device);
void tetris_ctx_destroy(tetris_ctx *ctx);
const char *tetris_last_error(void);

typedef struct {
    uint32_t log_n, n_q, n_p;
    double scale;         /* Delta */
    double pt_scale;      /* scale of database plaintexts: S[L-1] * q_L / S[L] */
    size_t device_bytes;  /* device memory the context holds now */
} tetris_ctx_info;
int tetris_get_info(const tetris_ctx *ctx, tetris_ctx_info *out);

/* Standard scale S[level]: S[L] = Delta, S[l-1] = S[l] * S[l] / q_l (double
 * arithmetic in that order).  Every ciphertext inside a query at level l
 * carries S[l]; Section 2.5 gives the multiply-then-rescale rule it follows. */
int tetris_standard_scale(const tetris_ctx *ctx, uint32_t level, double *out);

/* The count largest primes q < 2^bits with q = 1 mod 2^congruence_log2, in
 * descending order, skipping the n_exclude values of exclude (may be NULL). */
int tetris_gen_primes(uint32_t bits, uint32_t count, uint32_t congruence_log2,
                      const uint64_t *exclude, uint32_t n_exclude, uint64_t *out);

/* ---------------------------------------------------------------------------
 * Keys (Section 2.4.1, SwitchKeyGen; Appendix A.2 for their use).
 * A switching key is [dnum][2][n_q + n_p][N] uint64, coefficient domain,
 * limbs q_0..q_{n_q-1}, p_0..p_{n_p-1}; digit j covers the primes
 * q_{j*alpha} .. q_{j*alpha+alpha-1} (CRT gadget), dnum = ceil(n_q / alpha).
 * n_words must equal dnum * 2 * (n_q + n_p) * N.  The context copies the key
 * to device memory (converted to its internal NTT domain); loading a key for
 * an element that already has one replaces it.  All keys of a context share
 * one alpha: loading a key with a different alpha drops every loaded key.
 * alpha is 1..4 (EINVAL otherwise).  A digit wider than P is accepted: its
 * key-switch noise ~ (Q_j / P) sigma sqrt(N dnum) is harmless where the
 * switched ciphertext's scale is far above it (relinearisation, at scale
 * Delta^2; rotations at level 1), and the caller's choice elsewhere.
 * ------------------------------------------------------------------------- */
int tetris_load_relin_key(tetris_ctx *ctx, const uint64_t *evk, size_t n_words, uint32_t alpha);
int tetris_load_rotation_key(tetris_ctx *ctx, uint32_t galois_elt, const uint64_t *evk,
                             size_t n_words, uint32_t alpha);
/* Copy a loaded key back (coefficient domain, same layout); galois_elt 0
 * selects the relinearisation key. */
int tetris_get_key(tetris_ctx *ctx, uint32_t galois_elt, uint64_t *out, size_t cap_words);

/* Client-side key generation on the GPU from caller-drawn randomness
 * (Section 2.3 distributions): s int64[N] ternary secret; a uint64
 * [dnum][n_q+n_p][N] uniform residues; e int64[dnum][N] errors.  Builds
 * swk_j = (-a_j s + e_j + w_j P s', a_j) with s' = s^2 (relinearisation) or
 * s(X^g) (rotation by galois element g) and loads it as above. */
int tetris_keygen_relin(tetris_ctx *ctx, const int64_t *s, const uint64_t *a, const int64_t *e,
                        uint32_t alpha);
int tetris_keygen_rotation(tetris_ctx *ctx, uint32_t galois_elt, const int64_t *s,
                           const uint64_t *a, const int64_t *e, uint32_t alpha);

/* ---------------------------------------------------------------------------
 * Ciphertexts at the boundary.
 * ------------------------------------------------------------------------- */
typedef struct {
    uint32_t level;        /* l: data holds l+1 limbs per component */
    uint32_t ncomp;        /* 2 (or 3 for a degree-2 ciphertext, 1 for a plaintext) */
    double scale;
    const uint64_t *data;  /* [ncomp][level+1][N] */
} tetris_ct_in;

typedef struct {
    uint32_t level;        /* set by the library */
    uint32_t ncomp;        /* set by the library */
    double scale;          /* set by the library */
    uint64_t *data;        /* caller buffer */
    size_t cap_words;      /* its capacity in uint64 words */
} tetris_ct_out;

/* Secret-key encryption (Section 2.3): (c0, c1) = (-a s + e + m, a) mod Q_level.
 * m int64[N] message coefficients; a uint64[level+1][N]; e int64[N]. */
int tetris_encrypt(tetris_ctx *ctx, const int64_t *m, const int64_t *s, const uint64_t *a,
                   const int64_t *e, uint32_t level, double scale, tetris_ct_out *out);

/* ---------------------------------------------------------------------------
 * Database (the plaintext matrix P, p x h, of Section 3.3): row-major u8
 * [records][attrs].  Records fill the N/2 slots of consecutive blocks; slot
 * value = ((v - 127.5) / 127.5) / attrs.  The library encodes each
 * (block, attribute) column with its FP64 canonical-embedding encoder
 * (Appendix A.1.2) at the context's pt_scale and keeps the plaintexts resident
 * on the device (NTT domain, all n_q primes).  *db_out receives a handle.
 * ------------------------------------------------------------------------- */
int tetris_upload_database(tetris_ctx *ctx, const uint8_t *vals, uint64_t records, uint32_t attrs,
                           uint32_t *db_out);
/* Same, with the encoding done by the caller: coeffs int64 [blocks][attrs][N]
 * (the integer plaintext polynomials at pt_scale), blocks = ceil(records / (N/2));
 * mask_real float64[N]: the real coefficients (scale 1) of the encoding of the
 * live-slot indicator of the last block, required iff records is not a
 * multiple of N/2 (else NULL). */
int tetris_upload_database_encoded(tetris_ctx *ctx, const int64_t *coeffs, const double *mask_real,
                                   uint64_t records, uint32_t attrs, uint32_t *db_out);
int tetris_free_database(tetris_ctx *ctx, uint32_t db);

/* FP64 encoder alone: slots float64[n_values] (n_values <= N/2, rest zero) ->
 * coeffs int64[N] = floor(scale * m_i + 1/2), m = canonical-embedding preimage. */
int tetris_encode(tetris_ctx *ctx, const double *slots, uint32_t n_values, double scale,
                  int64_t *coeffs);
/* The real coefficients m (before scaling) of the same map. */
int tetris_encode_real(tetris_ctx *ctx, const double *slots, uint32_t n_values, double *m_out);

/* ---------------------------------------------------------------------------
 * Query (server side of Algorithm 2's local threshold and InnerSum):
 *   x = sum_j P[.,j] * Enc(w_j)                (attribute selection, Sec. 3.3)
 *   y = sum_{k=0}^{d} Enc(c_k) x^k             (private polynomial)
 *   z = (y - Enc(t)) / 2                       (private threshold, Sec. 4.3.2)
 *   u = (p_S(...p_1(z)) + 1) / (2 * records)   (composite sign -> step)
 *   out = InnerSum(sum over blocks of u)       (Algorithm 2, InnerSum)
 * Each p_s is odd of degree sign_degree, 7 or 15: sign_coeffs holds, per
 * stage, the (sign_degree + 1)/2 coefficients of x, x^3, ...; a degree-7 stage
 * takes 3 levels, a degree-15 stage 4 (Table 2's [15, 15, 15] composites).  w: n_attrs fresh ciphertexts at the
 * top level with scale Delta; f_coeffs: f_degree+1 ciphertexts, threshold:
 * one, each at any level at or above where it is used (the library moves it
 * down).  Keys needed: relinearisation and rotations by 5^(2^k) mod 2N,
 * k < log_n - 1.  The result, at the level reported in out, decrypts to
 * count / records in every slot (or, with a global threshold, to the bit
 * [count >= t1]).
 * ------------------------------------------------------------------------- */
typedef struct {
    uint32_t n_attrs;
    const tetris_ct_in *w;
    uint32_t f_degree;
    const tetris_ct_in *f_coeffs;
    const tetris_ct_in *threshold;
    uint32_t sign_stages;
    uint32_t sign_degree;
    const double *sign_coeffs;
    uint64_t total_records;   /* the count is normalised by this many records (0: the
                                 database's own); set it to the total over the partitions
                                 when a database is split across GPUs or owners (the
                                 horizontally partitioned database of Section 5.6): the
                                 partitions' results then add up residue-wise */
    /* Optional global threshold (Algorithm 2, last line), NULL for none: the
     * result becomes step((count - t1 + 1/2) / records) in every slot, i.e. 1 iff
     * at least t1 records pass (the 1/2 is Section 5.4.2's epsilon/2 shift for
     * integer counts).  global_threshold encrypts t1 as a count (not normalised),
     * at a level above the step values'; global_stages odd stages of degree
     * sign_degree, global_coeffs their coefficients (laid out as sign_coeffs).
     * Needs 3 (4) levels per degree-7 (15) stage below the step values' level. */
    const tetris_ct_in *global_threshold;
    uint32_t global_stages;
    const double *global_coeffs;
} tetris_query;

/* Host buffers in and out; blocks until the result is in out. */
int tetris_evaluate_query(tetris_ctx *ctx, uint32_t db, const tetris_query *query, tetris_ct_out *out);
/* Device buffers in and out (every data pointer of query and out is device
 * memory); enqueued on the CUDA stream `stream` (cudaStream_t, NULL for the
 * legacy default stream); returns before the work completes. */
int tetris_evaluate_query_device(tetris_ctx *ctx, uint32_t db, const tetris_query *query,
                                 tetris_ct_out *out, void *stream);

/* Residue-wise sum of partition results: data (device, [ncomp][level+1][N])
 * holds, per residue, the plain integer sum of at most 8 residues of the same
 * prime (< 2^63, e.g. after an all-reduce over ranks); reduces it mod q_i in
 * place, on the given CUDA stream. */
int tetris_reduce_sum_device(tetris_ctx *ctx, uint64_t *data, uint32_t level, uint32_t ncomp, void *stream);

typedef struct {
    int32_t l_lin, l_d, l_y, l_u, l_out; /* l_out: level of the summed step values (scale S[l_out]) */
    uint32_t ragged;
    uint32_t relins, rescales, rotations, kernel_launches;
    double pt_scale, mask_scale;
    int32_t l_ret; /* level of the returned ciphertext: InnerSum runs after dropping to it */
    uint32_t pad;
    uint64_t input_words; /* input words copied to the device per query (fresh inputs at the top
                             level): only the limbs the circuit reads of each ciphertext */
} tetris_plan_info;
/* Levels and operation counts of the plan for a query shape on a database. */
int tetris_plan(tetris_ctx *ctx, uint32_t db, uint32_t f_degree, uint32_t sign_stages,
                tetris_plan_info *out);

/* Autotuner: times the query's recorded program (device time, CUDA events,
 * reps replays after one warm-up) under each candidate schedule -- blocks per
 * launch in {all, 8, 4, 2, 1} (those below the database's block count) times
 * NTT register groups of 8 or 16 elements per thread or, for log N in
 * [14, 16], persistent launches -- keeps the fastest as the context's options
 * (TETRIS_OPT_BLOCKS_PER_LAUNCH, TETRIS_OPT_NTT_GROUP, TETRIS_OPT_PERSISTENT)
 * and writes up to cap timings.  The keyswitch digit size is fixed by the
 * loaded keys (chosen by the client at key generation). */
typedef struct {
    int32_t blocks_per_launch;  /* 0 = all */
    int32_t ntt_group_log2;     /* 3 or 4 */
    double ms;                  /* device time per query */
    int32_t persistent;         /* 1: persistent launches (TETRIS_OPT_PERSISTENT) */
    int32_t pad;
} tetris_tune_entry;
int tetris_autotune(tetris_ctx *ctx, uint32_t db, const tetris_query *query, uint32_t reps,
                    tetris_tune_entry *out, uint32_t cap, uint32_t *n_out);

/* Options. */
enum {
    TETRIS_OPT_BLOCKS_PER_LAUNCH = 1,  /* 0: all blocks of a database in each launch (batched);
                                          k: k blocks per launch (1 = plain per-ciphertext form) */
    TETRIS_OPT_USE_GRAPH = 2,          /* 1: replay the query as a captured CUDA graph */
    TETRIS_OPT_KS_ALPHA = 3,           /* read-only: alpha of the loaded keys */
    TETRIS_OPT_PROFILE = 4,            /* 1: run queries eagerly with a CUDA event pair around
                                          every launch, accumulating per-kernel statistics */
    TETRIS_OPT_NTT_GROUP = 5,          /* log2 of the NTT elements a thread holds: 3 or 4 */
    TETRIS_OPT_KS_BASE2 = 6,           /* w of the base-2^w decomposition of key-switch digits
                                          (Table 1's base2), 0 for none, else 8..62; needs
                                          alpha 1; keys then carry (L+1) ceil(bits/w) digits,
                                          digit i B + b with P 2^(w b) on limb i.  Set before
                                          loading or generating keys: changing it drops them */
    TETRIS_OPT_PERSISTENT = 9,         /* 1: queries record every NTT pass and every ModUp row pass +
                                          key inner product as one persistent launch (resident CTAs
                                          walking the tiles of all its limbs; log N in [14, 16]); 0
                                          (default): one CTA per tile.  Same results; the autotuner
                                          times both */
    TETRIS_OPT_DEBUG_CHECKS = 8,       /* 1: before a program is recorded, every device range each of
                                          its kernel jobs will read or write is checked on the host
                                          to lie inside a live allocation of the context, the program
                                          or the batch item (TETRIS_EINVAL naming the job otherwise,
                                          nothing launched); see tetris_debug_check */
    TETRIS_OPT_QUERY_STAGE = 7         /* 0 (default): queries return the InnerSum result.
                                          1..4: queries stop after a stage of every block and
                                          return its ciphertexts, block after block
                                          ([blocks][2][level+1][N], out->ncomp = 2, out->level
                                          and out->scale that stage's): 1 x (linear
                                          combination), 2 y = f(x), 3 y - t, 4 the step values
                                          u / records (before the block sum).  For checking the
                                          stages slot by slot; a ragged last block's dead slots
                                          carry whatever the circuit leaves there */
};
enum {
    TETRIS_STAGE_FULL = 0,
    TETRIS_STAGE_X = 1,
    TETRIS_STAGE_Y = 2,
    TETRIS_STAGE_D = 3,
    TETRIS_STAGE_U = 4
};
int tetris_set_option(tetris_ctx *ctx, int option, int64_t value);
/* Debug: with the environment variable TETRIS_GUARD_WORDS set when a context
 * (and its programs) allocate, every device buffer is framed by 32 words of a
 * fixed pattern on each side.  This reads all of them back (context and
 * recorded programs) and returns TETRIS_EINVAL naming the buffers whose guard
 * words changed (a write past a buffer's end or before its start), else
 * TETRIS_OK.  plant != 0 first overwrites one guard word (a test of the check
 * itself).  *checked_ranges (may be NULL) receives the device ranges the
 * TETRIS_OPT_DEBUG_CHECKS bounds check has verified so far. */
int tetris_debug_check(tetris_ctx *ctx, int plant, uint64_t *checked_ranges);
int tetris_get_option(tetris_ctx *ctx, int option, int64_t *value);

/* Per-kernel statistics gathered while TETRIS_OPT_PROFILE is on: for each
 * kernel kind, its launches, their summed event-timed duration and the
 * algorithmic bytes they move (distinct inputs read once plus outputs
 * written once).  Writes up to cap entries and *n_out; clears the tally. */
typedef struct {
    char kind[48];
    uint32_t launches;
    double total_ms;
    double alg_bytes;
    double alg_modmuls;   /* modular multiplications: butterflies, conversion and key products */
    double units;         /* limb jobs (N-word limbs) processed, summed over the launches */
} tetris_kernel_stat;

/* Measured throughput of lazy Shoup modular multiplications (the operation
 * every butterfly, conversion and constant product is built on) on a device:
 * independent products in registers, no memory traffic, timed with CUDA
 * events.  The integer-ALU roofline of the transforms is quoted against it. */
int tetris_modmul_peak(int device, double *gmodmul_per_s);
int tetris_get_kernel_stats(tetris_ctx *ctx, tetris_kernel_stat *out, uint32_t cap, uint32_t *n_out);

/* ---------------------------------------------------------------------------
 * Single primitives on caller ciphertexts (host buffers), for parity checks.
 * ------------------------------------------------------------------------- */
enum {
    TETRIS_OP_ADD = 1,          /* a + b */
    TETRIS_OP_SUB = 2,          /* a - b */
    TETRIS_OP_TENSOR = 3,       /* (a0 b0, a0 b1 + a1 b0, a1 b1), Appendix A.2 */
    TETRIS_OP_RELIN = 4,        /* a is degree 2: SwitchKey(a2, swk_{s^2->s}) + (a0, a1) */
    TETRIS_OP_RESCALE = 5,      /* divide by q_l with rounding, drop q_l (Section 2.5) */
    TETRIS_OP_MUL_INT = 6,      /* a * arg (signed integer constant) */
    TETRIS_OP_ADD_INT = 7,      /* a + arg as a constant polynomial */
    TETRIS_OP_AUTOMORPHISM = 8, /* a(X^arg), no key switch (Section 2.2) */
    TETRIS_OP_ROTATE = 9,       /* automorphism X -> X^arg then SwitchKey back to s */
    TETRIS_OP_KEYSWITCH = 10,   /* a has one component d: SwitchKey(d, key arg) (0 = relin key) */
    TETRIS_OP_MUL_PLAIN = 11,   /* b is a plaintext (ncomp = 1, residues): a * b */
    TETRIS_OP_NTT = 12,         /* a -> internal evaluation order NTT (bit-reversed order) */
    TETRIS_OP_INNERSUM = 13,    /* sum of rotations by 2^k, k < log_n - 1 */
    TETRIS_OP_DROP = 14,        /* keep primes q_0..q_arg */
    TETRIS_OP_RELIN_RESCALE = 15, /* rescale(relin(a)) in one pass over the targets (same result) */
    TETRIS_OP_RESCALE_MUL_INT = 16 /* rescale(a * arg) with the factor folded into the rescale (same result) */
};
int tetris_op(tetris_ctx *ctx, int opcode, const tetris_ct_in *a, const tetris_ct_in *b,
              int64_t arg, tetris_ct_out *out);

/* ---------------------------------------------------------------------------
 * Batches of independent ciphertext jobs at uneven ring degrees and levels.
 * Item i, on its own context (ring degree), computes
 *     y = rescale(ct * pt)                   (Section 2.5, App. A.1.2 slot product)
 *     y = Rot(y), rotations times            (Rot by 5^(2^(k mod (log_n - 1))), k = 0, 1, ...)
 *     out = relinearise(y * y)               (Appendix A.2)
 * ct: [2][level+1][N] and pt: [level+1][N] host, coefficient domain,
 * 1 <= level < n_q; out: [2][level][N] host.  Every item's context needs the
 * relinearisation key and the rotation keys it uses; all contexts must be on
 * one device.  Schedules give identical results:
 *   TETRIS_SCHED_PER_ITEM  items one after another, each operation its own launches;
 *   TETRIS_SCHED_MERGED    the k-th launch of all items of one ring degree that
 *                          share kernel and mode is one launch (mixing levels);
 *                          ring degrees run as concurrent programs;
 *   TETRIS_SCHED_FUSED     the k-th launch of all items that share kernel and mode is
 *                          one launch whatever their ring degree (log N in [14, 16], at
 *                          most 4 contexts): each job reads its own context's tables,
 *                          NTT passes and the ModUp row pass + key inner product run as
 *                          persistent kernels (resident CTAs walking the jobs' tiles);
 *   TETRIS_SCHED_AUTO      times them (fused only when every degree allows it), keeps
 *                          the fastest (*schedule_used).
 * *device_ms receives the device time of the run (CUDA events). */
typedef struct {
    tetris_ctx *ctx;
    uint32_t level;
    const uint64_t *ct;
    const uint64_t *pt;
    uint32_t rotations;
    uint64_t *out;
} tetris_batch_item;
enum { TETRIS_SCHED_PER_ITEM = 0, TETRIS_SCHED_MERGED = 1, TETRIS_SCHED_AUTO = 2, TETRIS_SCHED_FUSED = 3 };
int tetris_batch_run(const tetris_batch_item *items, uint32_t n_items, int schedule, int *schedule_used,
                     double *device_ms);

/* ---------------------------------------------------------------------------
 * Serving.  tetris_serve_start starts a server thread that owns the GPU work
 * of the context until tetris_serve_stop; in between, only tetris_submit,
 * tetris_poll, tetris_serve_stats and tetris_serve_stop may be called on the
 * context (from any thread).  tetris_submit copies the limbs the circuit
 * reads of the query's inputs (host buffers, as for tetris_evaluate_query)
 * into pinned memory, split over up to 8 host threads, and returns a ticket.  The server admits queued queries in arrival order while
 * fewer than max_inflight are running and the device memory of the program
 * instance a query needs fits memory_budget_bytes (idle instances of other
 * query shapes are released first; the first instance of a shape is sized by
 * recording it).  Each running query has its own buffers and stream, so
 * queries admitted while others run overlap on the device.  tetris_poll
 * waits up to timeout_ms for the ticket (TETRIS_ETIMEOUT if still running)
 * and copies the result into out, exactly as tetris_evaluate_query would
 * have returned it; a query that cannot fit the budget even alone fails
 * with TETRIS_EBUSY.  Latency is measured from submit to completion.
 * ------------------------------------------------------------------------- */
typedef struct {
    uint64_t submitted, completed, rejected;
    double p50_ms, p99_ms;
    size_t device_bytes;       /* device bytes of the program instances kept now */
    size_t peak_device_bytes;  /* most device bytes the server's programs held at once, measured
                                  from their allocations right after each new instance
                                  (released instances that are not freed yet included) */
    uint64_t cancelled;        /* queries withdrawn by tetris_cancel before admission */
    uint32_t max_admitted;  /* most requests admitted and not yet completed at one time */
    uint32_t max_overlap;   /* most completed requests whose device work (CUDA events at the
                               first copy in and after the copy out, on each request's
                               stream) spans one instant: overlap on the device itself */
} tetris_serve_stats;
int tetris_serve_start(tetris_ctx *ctx, size_t memory_budget_bytes, uint32_t max_inflight);
int tetris_submit(tetris_ctx *ctx, uint32_t db, const tetris_query *query, uint64_t *ticket);
int tetris_poll(tetris_ctx *ctx, uint64_t ticket, tetris_ct_out *out, uint32_t timeout_ms);
/* Counters and submit-to-completion latency percentiles since the start (or
 * the last reset); reset != 0 clears them after reading. */
int tetris_serve_stats_get(tetris_ctx *ctx, tetris_serve_stats *out, int reset);
/* Withdraw a ticket.  A query still waiting for admission is removed before
 * any of its work reaches the device; a finished query's result is dropped.
 * Either way the ticket becomes unknown (TETRIS_ENOTFOUND afterwards).  A
 * query already admitted cannot be stopped: TETRIS_EBUSY, poll it instead. */
int tetris_cancel(tetris_ctx *ctx, uint64_t ticket);
int tetris_serve_stop(tetris_ctx *ctx);

/* ---------------------------------------------------------------------------
 * Allocation-free rescale (the paper has no counterpart; this is an
 * interface for callers that cannot let the library allocate).
 *
 * cudaFree synchronises the whole device and cudaMalloc fails or fragments
 * once a serving process or another framework's caching allocator has
 * reserved the GPU, so a caller that drives the GPU that way may not let a
 * library allocate behind its back.  This call allocates nothing: in and out
 * are caller-owned device buffers and its scratch is one fixed device array
 * inside the library (tetris_noalloc_scratch_bytes() bytes: the top limb of
 * up to 3 components at N <= 2^16 plus the job tables of two transforms),
 * which every GPU that loads the library holds until the process exits.
 *
 * in:  device pointer, [ncomp][level+1][N] uint64 in the library's NTT order
 *      (the order TETRIS_OP_NTT returns), 1 <= level <= n_q - 1, ncomp <= 3.
 * out: device pointer, [ncomp][level][N], same order; must not overlap in.
 * stream: cudaStream_t (NULL = legacy default stream); the call enqueues the
 *      work and returns without waiting for it.  Its job tables are written
 *      on the device by a small kernel from that kernel's launch parameters,
 *      so nothing in host memory is read after the call returns.
 * The first call on each device resolves the scratch array's address there
 * (with that device current).  All calls share the array and it keeps the
 * last call's contents (nothing in it needs to start at zero); calls whose
 * work overlaps on the GPU race on it, so callers serialise them.
 * Errors: TETRIS_EINVAL for sizes beyond the maximum, overlap, null buffers
 * or buffers that are not device (or managed) memory of the context's device
 * (checked before anything is launched), TETRIS_ELEVEL for a level outside
 * [1, n_q - 1].
 * ------------------------------------------------------------------------- */
int tetris_rescale_ntt_noalloc(tetris_ctx *ctx, const uint64_t *in, uint64_t *out, uint32_t level,
                               uint32_t ncomp, void *stream);
size_t tetris_noalloc_scratch_bytes(void);

/* ---------------------------------------------------------------------------
 * PFE scoring step (Section 5.4.1; Algorithm 2, the loop building ct_i): for
 * every record i,
 *   out[i] = sum_{j<m} X^{exps[i*m + j]} u[j]   in (Z_{q_0}[X] / (X^N + 1))^2,
 * where u[j] encrypts the scientist's scoring polynomial u_{f_j} (its value
 * table placed so that X^k u_{f_j} has f_j at point k in coefficient 0) and
 * exps holds the records' attribute values in the exponent (taken mod 2N).
 * Uses the context's N and first prime q_0 (the paper's Set I: N = 2^12, one
 * 55-bit modulus).
 * u:    [m][2][N] uint64 residues mod q_0, coefficient domain;
 * exps: [p][m] uint32; out: [p][2][N] uint64.
 * _device: all three are device pointers (caller-owned), enqueued on stream
 * (cudaStream_t, NULL = legacy default), nothing allocated.  Without the
 * suffix: host pointers; the call copies in, runs and copies out (blocking).
 * Errors: TETRIS_EINVAL for null buffers, m outside [1, 4096] or p outside
 * [1, 2^30 - 1].
 * ------------------------------------------------------------------------- */
int tetris_pfe_scores(tetris_ctx *ctx, const uint64_t *u, uint32_t m, const uint32_t *exps, uint64_t p,
                      uint64_t *out);
int tetris_pfe_scores_device(tetris_ctx *ctx, const uint64_t *u, uint32_t m, const uint32_t *exps, uint64_t p,
                             uint64_t *out, void *stream);

/* ---------------------------------------------------------------------------
 * Ring repacking (Algorithm 1): n <= N ciphertexts whose messages carry x_i in
 * their constant coefficient become one ciphertext of sum_i x_i X^i (every
 * input premultiplied by N^-1 mod Q, then log N rounds of
 * c_j <- (c_j + X^t c_{j+t}) + phi_g(c_j - X^t c_{j+t}), g = 2N - 1 first,
 * then 5^(2^(r-1)) mod 2N).  Needs rotation keys for those Galois elements.
 * cts: [n][2][level+1][N] uint64, coefficient domain, all at `level` with the
 * same scale; out->data: [2][level+1][N] (cap_words >= 2 (level+1) N).
 * _device: device pointers, enqueued on stream; otherwise host pointers,
 * blocking.  The recorded program is kept per (n, level, scale).
 * Errors: TETRIS_EINVAL (n outside [1, N], null buffers, small output),
 * TETRIS_ELEVEL (level), TETRIS_ENOTFOUND (a rotation key missing).
 * ------------------------------------------------------------------------- */
int tetris_repack(tetris_ctx *ctx, const uint64_t *cts, uint32_t n, uint32_t level, double scale,
                  tetris_ct_out *out);
int tetris_repack_device(tetris_ctx *ctx, const uint64_t *cts, uint32_t n, uint32_t level, double scale,
                         tetris_ct_out *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* TETRIS_H */
