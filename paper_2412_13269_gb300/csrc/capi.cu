// The C ABI (include/tetris.h): argument checks, host<->device copies and
// dispatch into the recorder.  Every entry point catches library errors and
// returns a status; the message is kept per thread.
#include <cmath>
#include <cstring>

#include "program.h"

namespace tetris {

static thread_local std::string g_last_error;
void set_last_error(const std::string &m) { g_last_error = m; }

template <class F>
static int guarded(F &&f) {
    try {
        f();
        return TETRIS_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        cudaGetLastError();
        return e.code;
    } catch (const std::bad_alloc &) {
        set_last_error("host allocation failed");
        return TETRIS_ENOMEM;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return TETRIS_EINVAL;
    }
}

static void run_now(Ctx &C, Program &P) {
    P.finalize();
    P.run(C.stream);
    TCHECK_CUDA(cudaStreamSynchronize(C.stream));
}

static BufPtr upload(Pool &pool, const void *src, size_t bytes, cudaStream_t s) {
    BufPtr b = pool.alloc((bytes + 7) / 8);
    TCHECK_CUDA(cudaMemcpyAsync(b->ptr, src, bytes, cudaMemcpyHostToDevice, s));
    return b;
}

static void build_tables(Ctx &C) {
    const size_t N = C.N, np = C.all.size();
    // [prime][N] pairs (psi^brv(k), its Shoup companion): one 16-byte load per twiddle
    std::vector<u64> tw(2 * np * N), itw(2 * np * N);
    C.mods_host.resize(np);
    for (size_t t = 0; t < np; t++) {
        const u64 q = C.all[t], psi = C.psi[t], ipsi = h_invmod(psi, q);
        std::vector<u64> pw(N), ipw(N);
        pw[0] = ipw[0] = 1;
        for (size_t e = 1; e < N; e++) {
            pw[e] = h_mulmod(pw[e - 1], psi, q);
            ipw[e] = h_mulmod(ipw[e - 1], ipsi, q);
        }
        for (size_t k = 0; k < N; k++) {
            const uint32_t r = bitrev((uint32_t)k, C.log_n);
            tw[2 * (t * N + k)] = pw[r];
            tw[2 * (t * N + k) + 1] = h_shoup(pw[r], q);
            itw[2 * (t * N + k)] = ipw[r];
            itw[2 * (t * N + k) + 1] = h_shoup(ipw[r], q);
        }
        ModInfo &m = C.mods_host[t];
        m.q = q;
        m.r64 = (u64)((((u128)1) << 64) % q);
        m.r64_sh = h_shoup(m.r64, q);
        m.one_sh = (u64)((((u128)1) << 64) / q);
        m.ninv = h_invmod(N % q, q);
        m.ninv_sh = h_shoup(m.ninv, q);
    }
    // encoder: [N/2] exp(-2 pi i k/N), [N] exp(-pi i k/N), [N/2] int u_j
    std::vector<double> enc(2 * (N / 2) + 2 * N + N / 4 + 2, 0.0);
    for (size_t k = 0; k < N / 2; k++) {
        const double a = 2.0 * M_PI * (double)k / (double)N;
        enc[2 * k] = std::cos(a);
        enc[2 * k + 1] = -std::sin(a);
    }
    double *twist = enc.data() + N;
    for (size_t k = 0; k < N; k++) {
        const double a = M_PI * (double)k / (double)N;
        twist[2 * k] = std::cos(a);
        twist[2 * k + 1] = -std::sin(a);
    }
    int *uj = reinterpret_cast<int *>(twist + 2 * N);
    u64 e = 1;
    for (size_t j = 0; j < N / 2; j++) {
        uj[j] = (int)((e - 1) / 2);
        e = e * 5 % (2 * N);
    }
    const size_t w = np * N;
    // regions start on 256-byte boundaries: the encoder reads its table as double2
    const size_t mods_words = (np * sizeof(ModInfo) + 255) / 256 * 32;
    const size_t enc_words = enc.size();
    C.tables = C.pool.alloc(4 * w + mods_words + enc_words);
    u64 *base = C.tables->ptr;
    TCHECK_CUDA(cudaMemcpy(base, tw.data(), 2 * w * 8, cudaMemcpyHostToDevice));
    TCHECK_CUDA(cudaMemcpy(base + 2 * w, itw.data(), 2 * w * 8, cudaMemcpyHostToDevice));
    TCHECK_CUDA(cudaMemcpy(base + 4 * w, C.mods_host.data(), np * sizeof(ModInfo), cudaMemcpyHostToDevice));
    TCHECK_CUDA(cudaMemcpy(base + 4 * w + mods_words, enc.data(), enc_words * 8, cudaMemcpyHostToDevice));
    C.nt.tw = base;
    C.nt.itw = base + 2 * w;
    C.nt.mods = reinterpret_cast<const ModInfo *>(base + 4 * w);
    C.enc_tw = reinterpret_cast<const double *>(base + 4 * w + mods_words);
}

// ---------------------------------------------------------------------------
// Keys
// ---------------------------------------------------------------------------
// base-2^w pieces of a one-prime digit (1 without the decomposition)
static int key_pieces(const Ctx &C) {
    if (C.base2 == 0) return 1;
    int bits = 0;
    for (u64 q : C.q) bits = std::max(bits, 64 - __builtin_clzll(q));
    return (bits + C.base2 - 1) / C.base2;
}

static void drop_keys(Ctx &C) {
    cudaStreamSynchronize(C.stream);
    C.programs.clear();
    C.relin = Key();
    C.rot.clear();
}

static void set_alpha(Ctx &C, uint32_t alpha) {
    TREQUIRE(alpha >= 1 && (int)alpha <= kMaxConvSrc, TETRIS_EINVAL, "alpha must be in [1, 4]");
    TREQUIRE(C.base2 == 0 || alpha == 1, TETRIS_EINVAL, "the base-2^w decomposition takes one-prime digits (alpha 1)");
    const int dnum = (C.L() + 1 + alpha - 1) / alpha * key_pieces(C);
    TREQUIRE(dnum <= kMaxKeyDigits, TETRIS_EINVAL, "too many key digits (at most 64)");
    if (C.alpha != 0 && C.alpha != (int)alpha) drop_keys(C);  // a new digit size: the old keys are unusable with it
    C.alpha = alpha;
}

// A key's device form: for each digit and prime, N (component 0, component 1)
// pairs, so the key inner product reads both with one 16-byte load.
static Key key_from_limbs(Ctx &C, u64 *limbs, int dnum) {
    Key k;
    k.dnum = dnum;
    k.pieces = key_pieces(C);
    k.buf = C.pool.alloc((size_t)dnum * 2 * C.nqp() * C.N);
    launch_interleave_pairs(limbs, k.buf->ptr, dnum, C.nqp(), C.N, true, C.stream);
    TCHECK_CUDA(cudaGetLastError());
    TCHECK_CUDA(cudaStreamSynchronize(C.stream));
    return k;
}

static Key load_key(Ctx &C, const uint64_t *evk, size_t n_words, uint32_t alpha) {
    // every check before set_alpha, which drops the loaded keys on a new digit size:
    // a malformed key leaves the context as it was
    TREQUIRE(alpha >= 1 && (int)alpha <= kMaxConvSrc, TETRIS_EINVAL, "alpha must be in [1, 4]");
    const int dnum = (C.L() + 1 + alpha - 1) / alpha * key_pieces(C), nqp = C.nqp();
    const size_t N = C.N;
    TREQUIRE(evk, TETRIS_EINVAL, "key: null buffer");
    TREQUIRE(n_words == (size_t)dnum * 2 * nqp * N, TETRIS_EINVAL,
             "key: wrong size (" + std::to_string(n_words) + " words for " + std::to_string(dnum) + " digits, " +
                 std::to_string((size_t)dnum * 2 * nqp * N) + " expected)");
    for (size_t row = 0; row < (size_t)dnum * 2 * nqp; row++) {  // residues of limb t below its prime
        const u64 qt = C.all[row % nqp];
        const uint64_t *r = evk + row * N;
        u64 bad = 0;
        for (size_t i = 0; i < N; i++) bad |= (u64)(r[i] >= qt);
        TREQUIRE(!bad, TETRIS_EINVAL, "key: residue out of range in limb " + std::to_string(row % nqp) + " of row " +
                                          std::to_string(row));
    }
    set_alpha(C, alpha);
    Program P;
    Rec R(C, P);
    BufPtr limbs = upload(P.pool, evk, n_words * 8, C.stream);  // [dnum][2][nqp][N], transformed in place
    P.hold.push_back(limbs);
    std::vector<NttJob> jobs;
    for (int j = 0; j < dnum; j++)
        for (int c = 0; c < 2; c++)
            for (int t = 0; t < nqp; t++) {
                NttJob jb{};
                jb.src = jb.dst = limbs->ptr + (((size_t)j * 2 + c) * nqp + t) * N;
                jb.prime = t;
                jobs.push_back(jb);
            }
    R.ntt(false, jobs, LOAD_PLAIN, STORE_PLAIN);
    run_now(C, P);
    return key_from_limbs(C, limbs->ptr, dnum);
}

// s (int64, N) -> NTT-domain residues over every prime [nqp][N]
static BufPtr secret_ntt(Ctx &C, Program &P, Rec &R, const int64_t *s, int nlimbs) {
    BufPtr sd = upload(P.pool, s, C.N * 8, C.stream);
    P.hold.push_back(sd);
    BufPtr out = P.pool.alloc((size_t)nlimbs * C.N);
    std::vector<NttJob> jobs;
    for (int t = 0; t < nlimbs; t++) {
        NttJob j{};
        j.src = sd->ptr;
        j.dst = out->ptr + (size_t)t * C.N;
        j.prime = t;
        jobs.push_back(j);
    }
    R.ntt(false, jobs, LOAD_INT64, STORE_PLAIN);
    return out;
}

// swk_j = (-a_j s + e_j + w_j P s_from, a_j) over Q P, NTT domain (Section 2.4.1);
// with the base-2^w decomposition (Table 1 base2) digit j = i B + b carries
// P 2^(w b) s_from on limb i.
static Key gen_key(Ctx &C, const int64_t *s, const uint64_t *a, const int64_t *e, uint32_t alpha, uint32_t galois) {
    TREQUIRE(alpha >= 1 && (int)alpha <= kMaxConvSrc, TETRIS_EINVAL, "alpha must be in [1, 4]");
    TREQUIRE(s && a && e, TETRIS_EINVAL, "keygen: null input");
    const int B = key_pieces(C);
    const int dnum = (C.L() + 1 + alpha - 1) / alpha * B, nqp = C.nqp();
    const size_t N = C.N;
    for (size_t row = 0; row < (size_t)dnum * nqp; row++) {  // the uniform a: residues below their primes
        const u64 qt = C.all[row % nqp];
        u64 bad = 0;
        for (size_t i = 0; i < N; i++) bad |= (u64)(a[row * N + i] >= qt);
        TREQUIRE(!bad, TETRIS_EINVAL, "keygen: residue of a out of range in limb " + std::to_string(row % nqp));
    }
    set_alpha(C, alpha);
    Program P;
    Rec R(C, P);
    BufPtr sn = secret_ntt(C, P, R, s, nqp);
    BufPtr sf = P.pool.alloc((size_t)nqp * N);
    if (galois == 0) {
        std::vector<EwJob> jobs;
        for (int t = 0; t < nqp; t++) {
            EwJob j{};
            j.op = EW_MUL;
            j.prime = t;
            j.a = j.b = sn->ptr + (size_t)t * N;
            j.dst = sf->ptr + (size_t)t * N;
            jobs.push_back(j);
        }
        R.ew(jobs);
    } else {
        std::vector<AutJob> jobs;
        for (int t = 0; t < nqp; t++) jobs.push_back({sn->ptr + (size_t)t * N, sf->ptr + (size_t)t * N});
        R.aut(jobs, galois & (uint32_t)(2 * N - 1));
    }
    BufPtr kb = P.pool.alloc((size_t)dnum * 2 * nqp * N);  // [dnum][2][nqp][N]
    P.hold.push_back(kb);
    BufPtr ad = upload(P.pool, a, (size_t)dnum * nqp * N * 8, C.stream);
    BufPtr ed = upload(P.pool, e, (size_t)dnum * N * 8, C.stream);
    P.hold.push_back(ad);
    P.hold.push_back(ed);
    auto kl = [&](int j, int c, int t) { return kb->ptr + (((size_t)j * 2 + c) * nqp + t) * N; };
    std::vector<NttJob> ja, je;
    for (int j = 0; j < dnum; j++)
        for (int t = 0; t < nqp; t++) {
            NttJob x{};
            x.src = ad->ptr + ((size_t)j * nqp + t) * N;
            x.dst = kl(j, 1, t);
            x.prime = t;
            ja.push_back(x);
            NttJob y{};
            y.src = ed->ptr + (size_t)j * N;
            y.dst = kl(j, 0, t);
            y.prime = t;
            je.push_back(y);
        }
    R.ntt(false, ja, LOAD_PLAIN, STORE_PLAIN);
    R.ntt(false, je, LOAD_INT64, STORE_PLAIN);
    BufPtr tmp = P.pool.alloc((size_t)dnum * nqp * N);
    std::vector<EwJob> m1, m2, m3;
    for (int j = 0; j < dnum; j++)
        for (int t = 0; t < nqp; t++) {
            EwJob x{};
            x.op = EW_MUL;
            x.prime = t;
            x.a = kl(j, 1, t);
            x.b = sn->ptr + (size_t)t * N;
            x.dst = tmp->ptr + ((size_t)j * nqp + t) * N;
            m1.push_back(x);
            EwJob y{};
            y.op = EW_SUB;
            y.prime = t;
            y.a = kl(j, 0, t);
            y.b = x.dst;
            y.dst = kl(j, 0, t);
            m2.push_back(y);
            const int jd = j / B, piece = j % B;  // CRT digit and base-2^w piece
            const int lo = jd * (int)alpha, hi = std::min(C.L() + 1, (jd + 1) * (int)alpha);
            if (t >= lo && t < hi) {
                const u64 qt = C.all[t];
                u64 pm = 1 % qt;
                for (u64 pk : C.p) pm = h_mulmod(pm, pk % qt, qt);
                for (int r = 0; r < piece * C.base2; r++) pm = h_mulmod(pm, 2, qt);
                EwJob z{};
                z.op = EW_ADD_MUL_CONST;
                z.prime = t;
                z.a = sf->ptr + (size_t)t * N;
                z.b = kl(j, 0, t);
                z.dst = kl(j, 0, t);
                z.k = pm;
                z.k_sh = h_shoup(pm, qt);
                m3.push_back(z);
            }
        }
    R.ew(m1);
    R.ew(m2);
    R.ew(m3);
    run_now(C, P);
    return key_from_limbs(C, kb->ptr, dnum);
}

// ---------------------------------------------------------------------------
// Ciphertext upload / download helpers for single operations
// ---------------------------------------------------------------------------
static CtH upload_ct(Ctx &C, Program &P, Rec &R, const tetris_ct_in &c, bool to_ntt) {
    TREQUIRE(c.data && c.ncomp >= 1 && c.ncomp <= 3 && (int)c.level <= C.L(), TETRIS_EINVAL, "ciphertext: bad shape");
    CtH h = R.new_ct(1, c.ncomp, c.level);
    h.scale = c.scale;
    P.hold.push_back(h.buf);
    TCHECK_CUDA(cudaMemcpyAsync(h.base, c.data, h.bstride * 8, cudaMemcpyHostToDevice, C.stream));
    if (to_ntt) R.to_ntt(h);
    return h;
}

static void download_ct(Ctx &C, Program &P, const CtH &h, tetris_ct_out *out) {
    TREQUIRE(out && out->data, TETRIS_EINVAL, "null output");
    const size_t words = (size_t)h.comps * (h.level + 1) * C.N;
    TREQUIRE(out->cap_words >= words, TETRIS_EINVAL, "output buffer too small");
    P.finalize();
    P.run(C.stream);
    // h may be a view with component stride > (level+1)*N
    for (int c = 0; c < h.comps; c++)
        TCHECK_CUDA(cudaMemcpyAsync(out->data + (size_t)c * (h.level + 1) * C.N, h.limb(0, c, 0),
                                    (size_t)(h.level + 1) * C.N * 8, cudaMemcpyDeviceToHost, C.stream));
    TCHECK_CUDA(cudaStreamSynchronize(C.stream));
    out->level = h.level;
    out->ncomp = h.comps;
    out->scale = h.scale;
}

}  // namespace tetris

using namespace tetris;

extern "C" {

const char *tetris_last_error(void) { return g_last_error.c_str(); }

int tetris_gen_primes(uint32_t bits, uint32_t count, uint32_t cong, const uint64_t *exclude, uint32_t n_ex, uint64_t *out) {
    return guarded([&] {
        TREQUIRE(out, TETRIS_EINVAL, "null output");
        std::vector<u64> ex(exclude, exclude + (exclude ? n_ex : 0));
        auto v = h_gen_primes((int)bits, (int)count, (int)cong, ex);
        std::memcpy(out, v.data(), v.size() * 8);
    });
}

int tetris_ctx_create(tetris_ctx **out, uint32_t log_n, const uint64_t *q, uint32_t n_q, const uint64_t *p, uint32_t n_p,
                      double scale, int device) {
    return guarded([&] {
        TREQUIRE(out && q && p, TETRIS_EINVAL, "ctx_create: null pointer");
        TREQUIRE(log_n >= 10 && log_n <= 16, TETRIS_EINVAL, "log_n must be in [10, 16]");
        TREQUIRE(n_q >= 1 && n_p >= 1 && n_p <= (uint32_t)kMaxConvSrc && n_q + n_p <= (uint32_t)kMaxPrimes, TETRIS_EINVAL,
                 "prime counts out of range");
        TREQUIRE(scale > 0 && std::isfinite(scale), TETRIS_EINVAL, "scale must be positive");
        const u64 N = 1ull << log_n;
        std::vector<u64> all(q, q + n_q);
        all.insert(all.end(), p, p + n_p);
        for (size_t i = 0; i < all.size(); i++) {
            TREQUIRE(all[i] < (1ull << 61) && all[i] > 2 * N && (all[i] - 1) % (2 * N) == 0 && h_is_prime(all[i]),
                     TETRIS_EINVAL, "every modulus must be a prime below 2^61 with q = 1 mod 2N");
            for (size_t j = 0; j < i; j++) TREQUIRE(all[i] != all[j], TETRIS_EINVAL, "moduli must be distinct");
        }
        int ndev = 0;
        TCHECK_CUDA(cudaGetDeviceCount(&ndev));
        TREQUIRE(device >= 0 && device < ndev, TETRIS_EINVAL, "no such CUDA device");
        TCHECK_CUDA(cudaSetDevice(device));
        auto *h = new tetris_ctx();
        Ctx &C = h->c;
        try {
            C.device = device;
            C.log_n = log_n;
            C.N = N;
            C.q.assign(q, q + n_q);
            C.p.assign(p, p + n_p);
            C.all = all;
            for (u64 m : all) C.psi.push_back(h_primitive_2n_root(m, N));
            C.scale = scale;
            C.S.assign(n_q, 0.0);
            C.S[n_q - 1] = scale;
            for (int l = (int)n_q - 1; l > 0; l--) C.S[l - 1] = (C.S[l] * C.S[l]) / (double)C.q[l];
            const int L = (int)n_q - 1;
            C.pt_scale = L >= 1 ? (C.S[L - 1] * (double)C.q[L]) / C.S[L] : 0.0;
            TCHECK_CUDA(cudaStreamCreateWithFlags(&C.stream, cudaStreamNonBlocking));
            build_tables(C);
        } catch (...) {
            if (C.stream) cudaStreamDestroy(C.stream);
            delete h;
            throw;
        }
        *out = h;
    });
}

void tetris_ctx_destroy(tetris_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->c.device);
    try {
        serve_stop(ctx->c);
    } catch (...) {
    }
    cudaStreamSynchronize(ctx->c.stream);
    cudaStream_t s = ctx->c.stream;
    delete ctx;
    cudaStreamDestroy(s);
}

int tetris_get_info(const tetris_ctx *ctx, tetris_ctx_info *out) {
    return guarded([&] {
        TREQUIRE(ctx && out, TETRIS_EINVAL, "null pointer");
        const Ctx &C = ctx->c;
        out->log_n = C.log_n;
        out->n_q = (uint32_t)C.q.size();
        out->n_p = (uint32_t)C.p.size();
        out->scale = C.scale;
        out->pt_scale = C.pt_scale;
        out->device_bytes = C.bytes_held();
    });
}

int tetris_standard_scale(const tetris_ctx *ctx, uint32_t level, double *out) {
    return guarded([&] {
        TREQUIRE(ctx && out && level < ctx->c.S.size(), TETRIS_EINVAL, "bad level");
        *out = ctx->c.S[level];
    });
}

int tetris_load_relin_key(tetris_ctx *ctx, const uint64_t *evk, size_t n_words, uint32_t alpha) {
    return guarded([&] {
        TREQUIRE(ctx, TETRIS_EINVAL, "null context");
        TCHECK_CUDA(cudaSetDevice(ctx->c.device));
        ctx->c.relin = load_key(ctx->c, evk, n_words, alpha);
        ctx->c.programs.clear();
    });
}

int tetris_load_rotation_key(tetris_ctx *ctx, uint32_t g, const uint64_t *evk, size_t n_words, uint32_t alpha) {
    return guarded([&] {
        TREQUIRE(ctx && (g & 1), TETRIS_EINVAL, "galois element must be odd");
        TCHECK_CUDA(cudaSetDevice(ctx->c.device));
        ctx->c.rot[g & (uint32_t)(2 * ctx->c.N - 1)] = load_key(ctx->c, evk, n_words, alpha);
        ctx->c.programs.clear();
    });
}

int tetris_keygen_relin(tetris_ctx *ctx, const int64_t *s, const uint64_t *a, const int64_t *e, uint32_t alpha) {
    return guarded([&] {
        TREQUIRE(ctx, TETRIS_EINVAL, "null context");
        TCHECK_CUDA(cudaSetDevice(ctx->c.device));
        ctx->c.relin = gen_key(ctx->c, s, a, e, alpha, 0);
        ctx->c.programs.clear();
    });
}

int tetris_keygen_rotation(tetris_ctx *ctx, uint32_t g, const int64_t *s, const uint64_t *a, const int64_t *e, uint32_t alpha) {
    return guarded([&] {
        TREQUIRE(ctx && (g & 1), TETRIS_EINVAL, "galois element must be odd");
        TCHECK_CUDA(cudaSetDevice(ctx->c.device));
        ctx->c.rot[g & (uint32_t)(2 * ctx->c.N - 1)] = gen_key(ctx->c, s, a, e, alpha, g);
        ctx->c.programs.clear();
    });
}

int tetris_get_key(tetris_ctx *ctx, uint32_t g, uint64_t *out, size_t cap) {
    return guarded([&] {
        TREQUIRE(ctx && out, TETRIS_EINVAL, "null pointer");
        Ctx &C = ctx->c;
        TCHECK_CUDA(cudaSetDevice(C.device));
        const Key &k = find_key(C, g & (uint32_t)(2 * C.N - 1));
        const int nqp = C.nqp();
        const size_t words = (size_t)k.dnum * 2 * nqp * C.N;
        TREQUIRE(cap >= words, TETRIS_EINVAL, "output buffer too small");
        Program P;
        Rec R(C, P);
        BufPtr limbs = P.pool.alloc(words), o = P.pool.alloc(words);
        launch_interleave_pairs(limbs->ptr, k.buf->ptr, k.dnum, nqp, C.N, false, C.stream);  // pairs -> limbs
        TCHECK_CUDA(cudaGetLastError());
        std::vector<NttJob> jobs;
        for (size_t l = 0; l < (size_t)k.dnum * 2 * nqp; l++) {
            NttJob j{};
            j.src = limbs->ptr + l * C.N;
            j.dst = o->ptr + l * C.N;
            j.prime = (uint32_t)(l % nqp);
            jobs.push_back(j);
        }
        R.ntt(true, jobs, LOAD_PLAIN, STORE_PLAIN);
        run_now(C, P);
        TCHECK_CUDA(cudaMemcpy(out, o->ptr, words * 8, cudaMemcpyDeviceToHost));
    });
}

int tetris_encrypt(tetris_ctx *ctx, const int64_t *m, const int64_t *s, const uint64_t *a, const int64_t *e,
                   uint32_t level, double scale, tetris_ct_out *out) {
    return guarded([&] {
        TREQUIRE(ctx && m && s && a && e, TETRIS_EINVAL, "null pointer");
        Ctx &C = ctx->c;
        TCHECK_CUDA(cudaSetDevice(C.device));
        TREQUIRE((int)level <= C.L(), TETRIS_EINVAL, "level out of range");
        const int nl = level + 1;
        const size_t N = C.N;
        Program P;
        Rec R(C, P);
        BufPtr sn = secret_ntt(C, P, R, s, nl);
        CtH ct = R.new_ct(1, 2, level);
        ct.scale = scale;
        BufPtr md = upload(P.pool, m, N * 8, C.stream), ed = upload(P.pool, e, N * 8, C.stream);
        P.hold.push_back(md);
        P.hold.push_back(ed);
        TCHECK_CUDA(cudaMemcpyAsync(ct.limb(0, 1, 0), a, (size_t)nl * N * 8, cudaMemcpyHostToDevice, C.stream));
        BufPtr mn = P.pool.alloc((size_t)nl * N), en = P.pool.alloc((size_t)nl * N), as = P.pool.alloc((size_t)nl * N);
        std::vector<NttJob> jm, je, ja;
        for (int i = 0; i < nl; i++) {
            NttJob x{};
            x.prime = i;
            x.src = md->ptr;
            x.dst = mn->ptr + (size_t)i * N;
            jm.push_back(x);
            x.src = ed->ptr;
            x.dst = en->ptr + (size_t)i * N;
            je.push_back(x);
            x.src = x.dst = ct.limb(0, 1, i);
            ja.push_back(x);
        }
        R.ntt(false, jm, LOAD_INT64, STORE_PLAIN);
        R.ntt(false, je, LOAD_INT64, STORE_PLAIN);
        R.ntt(false, ja, LOAD_PLAIN, STORE_PLAIN);
        std::vector<EwJob> j1, j2;
        for (int i = 0; i < nl; i++) {
            EwJob x{};
            x.op = EW_ADD;
            x.prime = i;
            x.a = mn->ptr + (size_t)i * N;
            x.b = en->ptr + (size_t)i * N;
            x.dst = mn->ptr + (size_t)i * N;
            j1.push_back(x);
            EwJob y{};
            y.op = EW_MUL;
            y.prime = i;
            y.a = ct.limb(0, 1, i);
            y.b = sn->ptr + (size_t)i * N;
            y.dst = as->ptr + (size_t)i * N;
            j1.push_back(y);
            EwJob z{};
            z.op = EW_SUB;
            z.prime = i;
            z.a = mn->ptr + (size_t)i * N;
            z.b = as->ptr + (size_t)i * N;
            z.dst = ct.limb(0, 0, i);
            j2.push_back(z);
        }
        // m+e and a*s are independent; the subtraction runs after both
        R.ew(j1);
        R.ew(j2);
        CtH o = R.from_ntt(ct);
        download_ct(C, P, o, out);
    });
}

int tetris_upload_database(tetris_ctx *ctx, const uint8_t *vals, uint64_t records, uint32_t attrs, uint32_t *db_out) {
    return guarded([&] {
        TREQUIRE(ctx && vals && db_out && records > 0 && attrs > 0, TETRIS_EINVAL, "upload_database: bad arguments");
        Ctx &C = ctx->c;
        TCHECK_CUDA(cudaSetDevice(C.device));
        TREQUIRE(C.L() >= 1, TETRIS_ELEVEL, "context has a single prime");
        const size_t N = C.N, n = N / 2, nq = C.q.size();
        Database db;
        db.records = records;
        db.attrs = attrs;
        db.blocks = (int)((records + n - 1) / n);
        db.pts = C.pool.alloc((size_t)db.blocks * attrs * nq * N);
        Program P;
        Rec R(C, P);
        BufPtr vd = upload(P.pool, vals, records * attrs, C.stream);
        const size_t npt = (size_t)db.blocks * attrs;
        BufPtr slots = P.pool.alloc(npt * n);
        db_slots(reinterpret_cast<const uint8_t *>(vd->ptr), records, attrs, db.blocks, C.log_n,
                 reinterpret_cast<double *>(slots->ptr), C.stream);
        const size_t chunk = 32;
        BufPtr m = P.pool.alloc(chunk * N), work = P.pool.alloc(chunk * N * 4), ints = P.pool.alloc(chunk * N);
        for (size_t c0 = 0; c0 < npt; c0 += chunk) {
            const size_t cnt = std::min(chunk, npt - c0);
            encode_real_batch(reinterpret_cast<const double *>(slots->ptr) + c0 * n, reinterpret_cast<double *>(m->ptr),
                              (int)cnt, C.log_n, C.enc_tw, reinterpret_cast<double *>(work->ptr), C.stream);
            round_scale(reinterpret_cast<const double *>(m->ptr), reinterpret_cast<int64_t *>(ints->ptr), cnt * N, C.pt_scale,
                        C.stream);
            Program Q;
            Rec RQ(C, Q);
            std::vector<NttJob> jobs;
            for (size_t k = 0; k < cnt; k++)
                for (size_t i = 0; i < nq; i++) {
                    NttJob j{};
                    j.src = ints->ptr + k * N;
                    j.dst = db.pts->ptr + ((c0 + k) * nq + i) * N;
                    j.prime = (uint32_t)i;
                    jobs.push_back(j);
                }
            RQ.ntt(false, jobs, LOAD_INT64, STORE_PLAIN);
            run_now(C, Q);
        }
        if (records % n) {
            const uint64_t live = records - (uint64_t)(db.blocks - 1) * n;
            std::vector<double> z(n, 0.0);
            for (uint64_t i = 0; i < live; i++) z[i] = 1.0;
            BufPtr zs = upload(P.pool, z.data(), n * 8, C.stream);
            db.mask_real = C.pool.alloc(N);
            encode_real_batch(reinterpret_cast<const double *>(zs->ptr), reinterpret_cast<double *>(db.mask_real->ptr), 1,
                              C.log_n, C.enc_tw, reinterpret_cast<double *>(work->ptr), C.stream);
            TCHECK_CUDA(cudaStreamSynchronize(C.stream));
        }
        TCHECK_CUDA(cudaStreamSynchronize(C.stream));
        TCHECK_CUDA(cudaGetLastError());
        const uint32_t h = C.next_db++;
        C.dbs[h] = db;
        *db_out = h;
    });
}

int tetris_upload_database_encoded(tetris_ctx *ctx, const int64_t *coeffs, const double *mask_real, uint64_t records,
                                   uint32_t attrs, uint32_t *db_out) {
    return guarded([&] {
        TREQUIRE(ctx && coeffs && db_out && records > 0 && attrs > 0, TETRIS_EINVAL, "upload_database_encoded: bad arguments");
        Ctx &C = ctx->c;
        TCHECK_CUDA(cudaSetDevice(C.device));
        const size_t N = C.N, n = N / 2, nq = C.q.size();
        TREQUIRE((records % n == 0) == (mask_real == nullptr), TETRIS_EINVAL,
                 "mask_real is required exactly when the last block is partly filled");
        Database db;
        db.records = records;
        db.attrs = attrs;
        db.blocks = (int)((records + n - 1) / n);
        db.pts = C.pool.alloc((size_t)db.blocks * attrs * nq * N);
        const size_t npt = (size_t)db.blocks * attrs;
        const size_t chunk = 64;
        for (size_t c0 = 0; c0 < npt; c0 += chunk) {
            const size_t cnt = std::min(chunk, npt - c0);
            Program P;
            Rec R(C, P);
            BufPtr cd = upload(P.pool, coeffs + c0 * N, cnt * N * 8, C.stream);
            std::vector<NttJob> jobs;
            for (size_t k = 0; k < cnt; k++)
                for (size_t i = 0; i < nq; i++) {
                    NttJob j{};
                    j.src = cd->ptr + k * N;
                    j.dst = db.pts->ptr + ((c0 + k) * nq + i) * N;
                    j.prime = (uint32_t)i;
                    jobs.push_back(j);
                }
            R.ntt(false, jobs, LOAD_INT64, STORE_PLAIN);
            run_now(C, P);
        }
        if (mask_real) db.mask_real = upload(C.pool, mask_real, N * 8, C.stream);
        TCHECK_CUDA(cudaStreamSynchronize(C.stream));
        const uint32_t h = C.next_db++;
        C.dbs[h] = db;
        *db_out = h;
    });
}

int tetris_free_database(tetris_ctx *ctx, uint32_t db) {
    return guarded([&] {
        TREQUIRE(ctx, TETRIS_EINVAL, "null context");
        auto it = ctx->c.dbs.find(db);
        TREQUIRE(it != ctx->c.dbs.end(), TETRIS_ENOTFOUND, "unknown database handle");
        TCHECK_CUDA(cudaSetDevice(ctx->c.device));
        cudaStreamSynchronize(ctx->c.stream);
        drop_programs_of_db(ctx->c, db);
        ctx->c.dbs.erase(it);
    });
}

static void encode_common(Ctx &C, const double *slots, uint32_t nv, double *m_host, int64_t *ints_host, double scale) {
    const size_t N = C.N, n = N / 2;
    TREQUIRE(slots && nv <= n, TETRIS_EINVAL, "encode: too many slot values");
    Pool pool;
    std::vector<double> z(n, 0.0);
    std::memcpy(z.data(), slots, nv * 8);
    BufPtr zs = upload(pool, z.data(), n * 8, C.stream);
    BufPtr m = pool.alloc(N), work = pool.alloc(4 * N), ints = pool.alloc(N);
    encode_real_batch(reinterpret_cast<const double *>(zs->ptr), reinterpret_cast<double *>(m->ptr), 1, C.log_n, C.enc_tw,
                      reinterpret_cast<double *>(work->ptr), C.stream);
    if (ints_host) round_scale(reinterpret_cast<const double *>(m->ptr), reinterpret_cast<int64_t *>(ints->ptr), N, scale, C.stream);
    TCHECK_CUDA(cudaStreamSynchronize(C.stream));
    TCHECK_CUDA(cudaGetLastError());
    if (m_host) TCHECK_CUDA(cudaMemcpy(m_host, m->ptr, N * 8, cudaMemcpyDeviceToHost));
    if (ints_host) TCHECK_CUDA(cudaMemcpy(ints_host, ints->ptr, N * 8, cudaMemcpyDeviceToHost));
}

int tetris_encode(tetris_ctx *ctx, const double *slots, uint32_t nv, double scale, int64_t *coeffs) {
    return guarded([&] {
        TREQUIRE(ctx && coeffs, TETRIS_EINVAL, "null pointer");
        TCHECK_CUDA(cudaSetDevice(ctx->c.device));
        encode_common(ctx->c, slots, nv, nullptr, coeffs, scale);
    });
}

int tetris_encode_real(tetris_ctx *ctx, const double *slots, uint32_t nv, double *m_out) {
    return guarded([&] {
        TREQUIRE(ctx && m_out, TETRIS_EINVAL, "null pointer");
        TCHECK_CUDA(cudaSetDevice(ctx->c.device));
        encode_common(ctx->c, slots, nv, m_out, nullptr, 1.0);
    });
}

int tetris_evaluate_query(tetris_ctx *ctx, uint32_t db, const tetris_query *q, tetris_ct_out *out) {
    return guarded([&] {
        TREQUIRE(ctx, TETRIS_EINVAL, "null context");
        TCHECK_CUDA(cudaSetDevice(ctx->c.device));
        evaluate_query(ctx->c, db, q, out, ctx->c.stream, false);
    });
}

int tetris_evaluate_query_device(tetris_ctx *ctx, uint32_t db, const tetris_query *q, tetris_ct_out *out, void *stream) {
    return guarded([&] {
        TREQUIRE(ctx, TETRIS_EINVAL, "null context");
        TCHECK_CUDA(cudaSetDevice(ctx->c.device));
        evaluate_query(ctx->c, db, q, out, reinterpret_cast<cudaStream_t>(stream), true);
    });
}

int tetris_autotune(tetris_ctx *ctx, uint32_t db, const tetris_query *q, uint32_t reps, tetris_tune_entry *out,
                    uint32_t cap, uint32_t *n_out) {
    return guarded([&] {
        TREQUIRE(ctx && n_out && (out || cap == 0), TETRIS_EINVAL, "null pointer");
        TCHECK_CUDA(cudaSetDevice(ctx->c.device));
        std::vector<tetris_tune_entry> v;
        autotune(ctx->c, db, q, (int)std::max(1u, reps), v);
        *n_out = (uint32_t)std::min<size_t>(v.size(), cap);
        for (uint32_t i = 0; i < *n_out; i++) out[i] = v[i];
    });
}

int tetris_reduce_sum_device(tetris_ctx *ctx, uint64_t *data, uint32_t level, uint32_t ncomp, void *stream) {
    return guarded([&] {
        TREQUIRE(ctx, TETRIS_EINVAL, "null context");
        TCHECK_CUDA(cudaSetDevice(ctx->c.device));
        reduce_sum(ctx->c, data, (int)level, (int)ncomp, reinterpret_cast<cudaStream_t>(stream));
    });
}

int tetris_plan(tetris_ctx *ctx, uint32_t db, uint32_t f_degree, uint32_t sign_stages, tetris_plan_info *out) {
    return guarded([&] {
        TREQUIRE(ctx && out, TETRIS_EINVAL, "null pointer");
        TCHECK_CUDA(cudaSetDevice(ctx->c.device));
        plan_info(ctx->c, db, f_degree, sign_stages, out);
    });
}

int tetris_set_option(tetris_ctx *ctx, int option, int64_t value) {
    return guarded([&] {
        TREQUIRE(ctx, TETRIS_EINVAL, "null context");
        Ctx &C = ctx->c;
        switch (option) {
            case TETRIS_OPT_BLOCKS_PER_LAUNCH:
                TREQUIRE(value >= 0 && value < (1 << 20), TETRIS_EINVAL, "bad value");
                if (C.blocks_per_launch != (int)value) C.blocks_per_launch = (int)value;
                break;
            case TETRIS_OPT_USE_GRAPH:
                C.use_graph = value ? 1 : 0;
                break;
            case TETRIS_OPT_PROFILE:
                C.profile = value ? 1 : 0;
                break;
            case TETRIS_OPT_NTT_GROUP:
                TREQUIRE(value == 3 || value == 4, TETRIS_EINVAL, "NTT group must be 3 or 4");
                C.nt.loge = (int)value;
                break;
            case TETRIS_OPT_KS_BASE2:
                TREQUIRE(value == 0 || (value >= 8 && value <= 62), TETRIS_EINVAL, "base2 bits must be 0 or 8..62");
                if (C.base2 != (int)value) {
                    drop_keys(C);
                    C.base2 = (int)value;
                    C.alpha = 0;
                }
                break;
            case TETRIS_OPT_QUERY_STAGE:
                TREQUIRE(value >= TETRIS_STAGE_FULL && value <= TETRIS_STAGE_U, TETRIS_EINVAL, "query stage must be 0..4");
                C.query_stage = (int)value;
                break;
            case TETRIS_OPT_DEBUG_CHECKS:
                C.debug_checks = value ? 1 : 0;
                break;
            case TETRIS_OPT_PERSISTENT:
                if (value) ntt_pass_tiles(C.log_n, true);  // refuses ring degrees the persistent kernels do not take
                C.persistent = value ? 1 : 0;
                break;
            default:
                throw Error(TETRIS_EINVAL, "unknown or read-only option");
        }
    });
}

int tetris_get_option(tetris_ctx *ctx, int option, int64_t *value) {
    return guarded([&] {
        TREQUIRE(ctx && value, TETRIS_EINVAL, "null pointer");
        Ctx &C = ctx->c;
        switch (option) {
            case TETRIS_OPT_BLOCKS_PER_LAUNCH: *value = C.blocks_per_launch; break;
            case TETRIS_OPT_USE_GRAPH: *value = C.use_graph; break;
            case TETRIS_OPT_KS_ALPHA: *value = C.alpha; break;
            case TETRIS_OPT_KS_BASE2: *value = C.base2; break;
            case TETRIS_OPT_PROFILE: *value = C.profile; break;
            case TETRIS_OPT_NTT_GROUP: *value = C.nt.loge; break;
            case TETRIS_OPT_QUERY_STAGE: *value = C.query_stage; break;
            case TETRIS_OPT_DEBUG_CHECKS: *value = C.debug_checks; break;
            case TETRIS_OPT_PERSISTENT: *value = C.persistent; break;
            default: throw Error(TETRIS_EINVAL, "unknown option");
        }
    });
}

int tetris_batch_run(const tetris_batch_item *items, uint32_t n, int schedule, int *used, double *device_ms) {
    return guarded([&] {
        TREQUIRE(schedule >= TETRIS_SCHED_PER_ITEM && schedule <= TETRIS_SCHED_FUSED, TETRIS_EINVAL, "unknown schedule");
        batch_run(items, n, schedule, used, device_ms);
    });
}

int tetris_serve_start(tetris_ctx *ctx, size_t budget, uint32_t max_inflight) {
    return guarded([&] {
        TREQUIRE(ctx, TETRIS_EINVAL, "null context");
        TCHECK_CUDA(cudaSetDevice(ctx->c.device));
        cudaStreamSynchronize(ctx->c.stream);
        serve_start(ctx->c, budget, max_inflight);
    });
}

int tetris_cancel(tetris_ctx *ctx, uint64_t ticket) {
    return guarded([&] {
        TREQUIRE(ctx, TETRIS_EINVAL, "null context");
        serve_cancel(ctx->c, ticket);
    });
}

int tetris_submit(tetris_ctx *ctx, uint32_t db, const tetris_query *q, uint64_t *ticket) {
    return guarded([&] {
        TREQUIRE(ctx && ticket, TETRIS_EINVAL, "null pointer");
        TCHECK_CUDA(cudaSetDevice(ctx->c.device));
        *ticket = serve_submit(ctx->c, db, q);
    });
}

int tetris_poll(tetris_ctx *ctx, uint64_t ticket, tetris_ct_out *out, uint32_t timeout_ms) {
    int rc = TETRIS_OK;
    int g = guarded([&] {
        TREQUIRE(ctx, TETRIS_EINVAL, "null context");
        rc = serve_poll(ctx->c, ticket, out, timeout_ms);
        if (rc == TETRIS_ETIMEOUT) set_last_error("poll: ticket still running");
    });
    return g != TETRIS_OK ? g : rc;
}

int tetris_serve_stats_get(tetris_ctx *ctx, tetris_serve_stats *out, int reset) {
    return guarded([&] {
        TREQUIRE(ctx && out, TETRIS_EINVAL, "null pointer");
        serve_stats(ctx->c, out, reset != 0);
    });
}

int tetris_serve_stop(tetris_ctx *ctx) {
    return guarded([&] {
        TREQUIRE(ctx, TETRIS_EINVAL, "null context");
        TCHECK_CUDA(cudaSetDevice(ctx->c.device));
        serve_stop(ctx->c);
    });
}

int tetris_rescale_ntt_noalloc(tetris_ctx *ctx, const uint64_t *in, uint64_t *out, uint32_t level, uint32_t ncomp,
                               void *stream) {
    return guarded([&] {
        TREQUIRE(ctx, TETRIS_EINVAL, "null context");
        TCHECK_CUDA(cudaSetDevice(ctx->c.device));
        rescale_ntt_noalloc(ctx->c, in, out, (int)level, (int)ncomp, reinterpret_cast<cudaStream_t>(stream));
    });
}

size_t tetris_noalloc_scratch_bytes(void) { return noalloc_scratch_bytes(); }

static int repack_call(tetris_ctx *ctx, const uint64_t *cts, uint32_t n, uint32_t level, double scale,
                       tetris_ct_out *out, void *stream, bool device) {
    return guarded([&] {
        TREQUIRE(ctx && out && out->data, TETRIS_EINVAL, "repack: null pointer");
        Ctx &C = ctx->c;
        TCHECK_CUDA(cudaSetDevice(C.device));
        TREQUIRE((int)level <= C.L(), TETRIS_ELEVEL, "repack: bad level");
        TREQUIRE(out->cap_words >= (size_t)2 * (level + 1) * C.N, TETRIS_EINVAL, "repack: output buffer too small");
        cudaStream_t s = device ? reinterpret_cast<cudaStream_t>(stream) : C.stream;
        repack(C, cts, n, (int)level, scale, out->data, s, device);
        out->level = level;
        out->ncomp = 2;
        out->scale = scale;
    });
}

int tetris_repack(tetris_ctx *ctx, const uint64_t *cts, uint32_t n, uint32_t level, double scale,
                  tetris_ct_out *out) {
    return repack_call(ctx, cts, n, level, scale, out, nullptr, false);
}

int tetris_repack_device(tetris_ctx *ctx, const uint64_t *cts, uint32_t n, uint32_t level, double scale,
                         tetris_ct_out *out, void *stream) {
    return repack_call(ctx, cts, n, level, scale, out, stream, true);
}

int tetris_pfe_scores_device(tetris_ctx *ctx, const uint64_t *u, uint32_t m, const uint32_t *exps, uint64_t p,
                             uint64_t *out, void *stream) {
    return guarded([&] {
        TREQUIRE(ctx, TETRIS_EINVAL, "null context");
        TCHECK_CUDA(cudaSetDevice(ctx->c.device));
        pfe_scores(ctx->c, u, m, exps, p, out, reinterpret_cast<cudaStream_t>(stream));
    });
}

int tetris_pfe_scores(tetris_ctx *ctx, const uint64_t *u, uint32_t m, const uint32_t *exps, uint64_t p,
                      uint64_t *out) {
    return guarded([&] {
        TREQUIRE(ctx && u && exps && out, TETRIS_EINVAL, "pfe: null pointer");
        TREQUIRE(m >= 1 && m <= 4096 && p >= 1 && p < (1ull << 30), TETRIS_EINVAL, "pfe: bad sizes");
        Ctx &C = ctx->c;
        TCHECK_CUDA(cudaSetDevice(C.device));
        const size_t uw = (size_t)m * 2 * C.N, ow = (size_t)p * 2 * C.N, ew = (size_t)p * m;
        u64 *du = nullptr, *dout = nullptr;
        uint32_t *de = nullptr;
        auto release = [&] {
            cudaFree(du);
            cudaFree(dout);
            cudaFree(de);
        };
        try {
            TCHECK_CUDA(cudaMalloc(&du, uw * 8));
            TCHECK_CUDA(cudaMalloc(&dout, ow * 8));
            TCHECK_CUDA(cudaMalloc(&de, ew * 4));
            TCHECK_CUDA(cudaMemcpyAsync(du, u, uw * 8, cudaMemcpyHostToDevice, C.stream));
            TCHECK_CUDA(cudaMemcpyAsync(de, exps, ew * 4, cudaMemcpyHostToDevice, C.stream));
            pfe_scores(C, du, m, de, p, dout, C.stream);
            TCHECK_CUDA(cudaMemcpyAsync(out, dout, ow * 8, cudaMemcpyDeviceToHost, C.stream));
            TCHECK_CUDA(cudaStreamSynchronize(C.stream));
        } catch (...) {
            cudaStreamSynchronize(C.stream);
            release();
            throw;
        }
        release();
    });
}

int tetris_modmul_peak(int device, double *rate) {
    return guarded([&] {
        TREQUIRE(rate, TETRIS_EINVAL, "null pointer");
        TCHECK_CUDA(cudaSetDevice(device));
        *rate = modmul_peak_probe();
    });
}

int tetris_debug_check(tetris_ctx *ctx, int plant, uint64_t *checked_ranges) {
    return guarded([&] {
        TREQUIRE(ctx, TETRIS_EINVAL, "null context");
        Ctx &C = ctx->c;
        TCHECK_CUDA(cudaSetDevice(C.device));
        TCHECK_CUDA(cudaDeviceSynchronize());
        if (checked_ranges) *checked_ranges = C.checked_ranges;
        if (plant) C.pool.plant_guard_fault();
        std::vector<std::string> bad = C.pool.check_guards();
        for (auto &kv : C.programs)
            for (auto &b : kv.second->pool.check_guards()) bad.push_back(b);
        if (!bad.empty()) {
            std::string m = "guard words overwritten: ";
            for (size_t i = 0; i < bad.size() && i < 8; i++) m += (i ? ", " : "") + bad[i];
            throw Error(TETRIS_EINVAL, m);
        }
    });
}

int tetris_get_kernel_stats(tetris_ctx *ctx, tetris_kernel_stat *out, uint32_t cap, uint32_t *n_out) {
    return guarded([&] {
        TREQUIRE(ctx && n_out && (out || cap == 0), TETRIS_EINVAL, "null pointer");
        uint32_t n = 0;
        for (auto &kv : ctx->c.stats) {
            if (n < cap) {
                tetris_kernel_stat &o = out[n];
                std::memset(o.kind, 0, sizeof(o.kind));
                std::strncpy(o.kind, kv.first.c_str(), sizeof(o.kind) - 1);
                o.launches = kv.second.launches;
                o.total_ms = kv.second.ms;
                o.alg_bytes = kv.second.bytes;
                o.alg_modmuls = kv.second.modmuls;
                o.units = kv.second.units;
            }
            n++;
        }
        *n_out = std::min(n, cap);
        ctx->c.stats.clear();
    });
}

int tetris_op(tetris_ctx *ctx, int op, const tetris_ct_in *a, const tetris_ct_in *b, int64_t arg, tetris_ct_out *out) {
    return guarded([&] {
        TREQUIRE(ctx && a, TETRIS_EINVAL, "null pointer");
        Ctx &C = ctx->c;
        TCHECK_CUDA(cudaSetDevice(C.device));
        Program P;
        Rec R(C, P);
        CtH x = upload_ct(C, P, R, *a, true);
        CtH r;
        switch (op) {
            case TETRIS_OP_ADD:
            case TETRIS_OP_SUB: {
                TREQUIRE(b, TETRIS_EINVAL, "needs b");
                CtH y = upload_ct(C, P, R, *b, true);
                r = op == TETRIS_OP_ADD ? R.add(x, y) : R.sub(x, y);
                break;
            }
            case TETRIS_OP_TENSOR: {
                TREQUIRE(b, TETRIS_EINVAL, "needs b");
                r = R.tensor(x, upload_ct(C, P, R, *b, true));
                break;
            }
            case TETRIS_OP_RELIN: r = R.relin(x); break;
            case TETRIS_OP_RESCALE: r = R.rescale(x); break;
            case TETRIS_OP_MUL_INT: r = R.mul_int(x, arg); break;
            case TETRIS_OP_ADD_INT: r = R.add_int(x, arg); break;
            case TETRIS_OP_AUTOMORPHISM: r = R.automorphism(x, (uint32_t)arg); break;
            case TETRIS_OP_ROTATE: r = R.rotate(x, (uint32_t)arg); break;
            case TETRIS_OP_KEYSWITCH: {
                TREQUIRE(x.comps == 1, TETRIS_EINVAL, "keyswitch takes one polynomial");
                const Key &k = find_key(C, (uint32_t)arg & (uint32_t)(2 * C.N - 1));
                r = R.keyswitch(1, x.level, [&](int, int i) { return (const u64 *)x.limb(0, 0, i); }, k,
                                [](int, int, int) { return (const u64 *)nullptr; });
                break;
            }
            case TETRIS_OP_MUL_PLAIN: {
                TREQUIRE(b && b->ncomp == 1 && b->level >= a->level, TETRIS_EINVAL, "plaintext must have one component");
                CtH y = upload_ct(C, P, R, *b, true);
                r = R.mul_plain(x, y.base, 0);
                break;
            }
            case TETRIS_OP_NTT: {
                TREQUIRE(out && out->data && out->cap_words >= x.bstride, TETRIS_EINVAL, "output buffer too small");
                P.finalize();
                P.run(C.stream);
                for (int c = 0; c < x.comps; c++)
                    TCHECK_CUDA(cudaMemcpyAsync(out->data + (size_t)c * (x.level + 1) * C.N, x.limb(0, c, 0),
                                                (size_t)(x.level + 1) * C.N * 8, cudaMemcpyDeviceToHost, C.stream));
                TCHECK_CUDA(cudaStreamSynchronize(C.stream));
                out->level = x.level;
                out->ncomp = x.comps;
                out->scale = x.scale;
                return;
            }
            case TETRIS_OP_INNERSUM: {
                r = x;
                for (int k = 0; k + 1 < C.log_n; k++) {
                    const uint32_t g = (uint32_t)h_powmod(5, 1ull << k, 2 * C.N);
                    r = R.add(r, R.rotate(r, g));
                }
                break;
            }
            case TETRIS_OP_DROP: r = R.drop(x, (int)arg); break;
            case TETRIS_OP_RELIN_RESCALE: r = R.relin_rescale(x); break;
            case TETRIS_OP_RESCALE_MUL_INT: r = R.rescale(x, arg); break;
            default: throw Error(TETRIS_EINVAL, "unknown opcode");
        }
        CtH o = R.from_ntt(r);
        download_ct(C, P, o, out);
    });
}

}  // extern "C"
