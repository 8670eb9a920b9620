// Negacyclic NTT over 64-bit RNS primes, batched over a job list of limbs.
//
// Forward transform: Cooley-Tukey butterflies with the bit-reversed powers
// tw[k] = psi^brv(k) (psi a primitive 2N-th root), natural-order input,
// output A(psi^(2*brv(k)+1)) at index k.  Inverse: Gentleman-Sande with
// psi^-brv(k), then N^-1.  The ring is the negacyclic Z_q[X]/(X^N+1) of the
// paper's Section 2.2; this transform evaluates at its N roots.
//
// An N = N1*N2 transform runs as two passes over HBM: a column pass (the
// first log N1 stages; each column of the N1 x N2 row-major view is an
// N1-point sub-problem) and a row pass (the remaining log N2 stages within
// each contiguous row).  Inside a pass a CTA stages its tile in shared
// memory; each thread holds E = 8 (or 16) elements in registers and runs
// three (four) butterfly stages per visit: radix-8 groups use 64 registers
// and four CTAs per SM, radix-16 groups 80 registers and three.  A thread loads its first
// group straight from global memory and stores its last group straight back
// (both coalesced across the warp), so a 256-point sub-problem needs two
// shared-memory exchanges.  Stage bit b of a sub-problem of size
// M uses twiddle index (M >> (b+1)) * o + (r >> (b+1)), with o = 1 in the
// column pass and o = N1 + row in the row pass; the tables hold each twiddle
// beside its Shoup companion, one 16-byte load per twiddle.
//
// Load modes fuse the producer: plain, int64 -> residue, or a fast base
// conversion from up to four source limbs (ModUp / ModDown / rescale), less a
// per-coefficient constant.  The combine store fuses the consumer:
// (extra) + (base - x) * mul; the inverse stores can scale, add a constant and
// subtract a base conversion.  Butterflies are lazy: forward transforms modulo
// primes below 2^57 run with no correction at all (their products use a
// Shoup quotient estimated from three partial products, < 4q; values grow by
// at most 4q per stage and stay below 94q), the others as Harvey's, in [0, 4q) (forward)
// or [0, 2q) (inverse) between stages and passes; the second pass reduces.
#include "internal.h"

namespace tetris {

namespace {

constexpr int kThreads = 256;
// Register-group width: a thread holds 2^LOGEV elements.  Both widths are
// compiled; NttTables::loge picks one per context (the autotuner's knob).

struct PassParams {
    NttTables t;
    const NttJob *jobs;
    int log1, log2;
    int load_mode, store_mode;
    int scale_out;
    int first;
};

// Harvey's lazy butterflies.  Forward (Cooley-Tukey): inputs in [0, 4q),
// outputs in [0, 4q).  Inverse (Gentleman-Sande): inputs and outputs in [0, 2q).
__device__ __forceinline__ void ct_bfly(u64 &x, u64 &y, u64 w, u64 wsh, u64 q, u64 q2) {
    u64 X = x >= q2 ? x - q2 : x;
    u64 T = shoup_lazy(y, w, wsh, q);
    x = X + T;
    y = X - T + q2;
}
// a * w mod q in [0, 4q) for any 64-bit a and w < q: the Shoup quotient
// floor(a w' / 2^64) estimated from three of its four 32 x 32 partial
// products, a1 w'1 + hi(a1 w'0) + hi(a0 w'1), which is at most 2 below it
// (the dropped a0 w'0 and the two truncated high halves add less than 3)
__device__ __forceinline__ u64 shoup_lazy4(u64 a, u64 w, u64 wsh, u64 q) {
    const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32), s0 = (uint32_t)wsh, s1 = (uint32_t)(wsh >> 32);
    const u64 qt = (u64)a1 * s1 + __umulhi(a1, s0) + __umulhi(a0, s1);
    return a * w - qt * q;
}
// Forward butterfly without correction: the estimated-quotient product is
// < 4q for any 64-bit y, so each stage adds at most 4q to the bound of its
// inputs (q4 = 4q keeps X - T + q4 non-negative).
__device__ __forceinline__ void ct_bfly_open(u64 &x, u64 &y, u64 w, u64 wsh, u64 q, u64 q2) {
    u64 T = shoup_lazy4(y, w, wsh, q);
    u64 X = x;
    x = X + T;
    y = X - T + q2;
}
__device__ __forceinline__ void gs_bfly(u64 &x, u64 &y, u64 w, u64 wsh, u64 q, u64 q2) {
    u64 S = x + y;
    S = S >= q2 ? S - q2 : S;
    u64 D = x - y + q2;
    x = S;
    y = shoup_lazy(D, w, wsh, q);
}

// Forward transforms modulo q < 2^57 run "open" (no correction inside the two
// passes): loads give values below q + 4 * 4q = 17q (a conversion from four
// sources); the first stage of a conversion pass, whose upper inputs already
// carry the twiddle, adds and subtracts them (< 34q); each later stage adds at
// most 4q, so after seven more stages of the first pass and eight of the
// second every intermediate stays below 34q + 60q = 94q < 2^64; the second
// pass's store reduces once.  Larger primes (the 60-bit special primes) take
// Harvey's corrected butterflies with exact Shoup products.
constexpr u64 kOpenBound = 1ull << 57;

// Register window of butterfly group g: the thread holds the E elements whose
// row index differs only in bits [lo, lo + LOGE); stages run on bits [blo, bhi].
template <int LOGM, int LOGE, bool INV>
struct Group {
    __host__ __device__ static constexpr int bhi(int g) {
        return INV ? ((g * LOGE + LOGE - 1) > LOGM - 1 ? LOGM - 1 : g * LOGE + LOGE - 1) : LOGM - 1 - g * LOGE;
    }
    __host__ __device__ static constexpr int blo(int g) {
        return INV ? g * LOGE : ((LOGM - 1 - g * LOGE - LOGE + 1) < 0 ? 0 : LOGM - 1 - g * LOGE - LOGE + 1);
    }
    __host__ __device__ static constexpr int lo(int g) {
        return INV ? (g * LOGE < LOGM - LOGE ? g * LOGE : LOGM - LOGE) : blo(g);
    }
};

// MODE: first pass (forward) loading plain / int64 / pre-scaled conversion
//       sources / a reduction; second pass storing plain / combined;
//       inverse: first pass plain, second pass storing plain / x * mul + add /
//       as the latter less a base conversion of coefficient-domain sources.
enum { M_PLAIN = 0, M_INT64 = 1, M_STORE = 3, M_COMBINE = 4, M_CONVPRE = 5, M_REDUCE = 6, M_SCALED = 7,
       M_SCALED_CONV = 8, M_PIECE = 9 };
constexpr bool is_second(int m) { return m == M_STORE || m == M_COMBINE || m == M_SCALED || m == M_SCALED_CONV; }

// Geometry of one pass: which sub-problem s and lane t a thread takes, where
// its elements sit in global and shared memory, and the register windows.
template <int LOGM, bool INV, bool COL, int LOGEV>
struct Geo {
    static constexpr int M = 1 << LOGM;
    static constexpr int LOGE = LOGM >= LOGEV ? LOGEV : LOGM;
    static constexpr int E = 1 << LOGE;
    static constexpr int T = M / E;
    static constexpr int NG = (LOGM + LOGE - 1) / LOGE;
    using G = Group<LOGM, LOGE, INV>;
    // In the row pass a group whose register window is the low bits holds
    // contiguous words per thread; those ends go through shared memory so the
    // global accesses stay coalesced (lane t takes words t, t + T, t + 2T, ...).
    static constexpr bool IN_STAGE = !COL && G::lo(0) != LOGM - LOGE;
    static constexpr bool OUT_STAGE = !COL && G::lo(NG - 1) != LOGM - LOGE;
    // A row-pass sub-problem lives in one warp (T <= 32 consecutive threads),
    // so its exchanges only synchronise the warp; column sub-problems span warps.
    static_assert(COL || T <= 32, "row sub-problem wider than a warp");

    int N1, N2, sub_cta, sub0, s, t;
    u64 o;
    // log1, log2: the N1 x N2 split of the transform; tile: which group of
    // sub_cta sub-problems this CTA takes
    __device__ Geo(int log1, int log2, int tile) {
        N1 = 1 << log1;
        N2 = 1 << log2;
        const int nsub = COL ? N2 : N1;
        sub_cta = min(kThreads / T, nsub);
        sub0 = tile * sub_cta;
        // consecutive threads take consecutive columns in the column pass and
        // consecutive lanes of a row in the row pass
        s = COL ? (int)threadIdx.x % sub_cta : (int)threadIdx.x / T;
        t = COL ? (int)threadIdx.x / sub_cta : (int)threadIdx.x % T;
        o = COL ? 1 : (u64)(N1 + sub0 + s);
    }
    __device__ int smidx(int r) const { return COL ? r * sub_cta + s : s * (M + M / 16) + r + (r >> 4); }
    __device__ size_t gidx(int r) const { return COL ? (size_t)r * N2 + sub0 + s : (size_t)(sub0 + s) * N2 + r; }
    __device__ int row(int g, int k) const {
        const int l = G::lo(g);
        return (t & ((1 << l) - 1)) | (k << l) | ((t >> l) << (l + LOGE));
    }
    __device__ int lrow(int k) const { return IN_STAGE ? t + T * k : row(0, k); }
    __device__ int srow(int k) const { return OUT_STAGE ? t + T * k : row(NG - 1, k); }
    __device__ void sync() const {
        if (COL) __syncthreads();
        else __syncwarp();
    }
};

// The butterfly stages of one pass on the thread's registers x (loaded at
// lrow), leaving them at srow: shared-memory exchanges between groups and the
// staging of non-coalesced ends.
//
// FOLD (column pass): the outer stage's one twiddle is folded into a job
// constant.  Forward (open): the first stage's upper elements were loaded
// already multiplied by it (a conversion load whose constants carry it), each
// below 17q, so the stage only adds and subtracts.  Inverse: the last stage
// leaves its differences x - y + 2q (< 4q) for the scaled store, whose
// constant for the upper half carries the twiddle.
template <int LOGM, bool INV, bool COL, int LOGEV, bool OPEN, bool FOLD = false>
__device__ __forceinline__ void run_stages(const Geo<LOGM, INV, COL, LOGEV> &g, u64 (&x)[Geo<LOGM, INV, COL, LOGEV>::E],
                                           u64 *sm, const u64 *tw, u64 q) {
    using GG = Geo<LOGM, INV, COL, LOGEV>;
    using G = typename GG::G;
    constexpr int M = GG::M, E = GG::E, LOGE = GG::LOGE, NG = GG::NG;
    const u64 q2 = 2 * q;
    // the open butterfly adds 4q, the bound of its estimated-quotient product
    const u64 qb = OPEN ? 4 * q : q2;
    if (GG::IN_STAGE) {
#pragma unroll
        for (int k = 0; k < E; k++) sm[g.smidx(g.lrow(k))] = x[k];
        g.sync();
#pragma unroll
        for (int k = 0; k < E; k++) x[k] = sm[g.smidx(g.row(0, k))];
    }
#pragma unroll
    for (int gi = 0; gi < NG; gi++) {
        if (gi > 0) {
            g.sync();  // (gi > 1) every thread has read the previous exchange
#pragma unroll
            for (int k = 0; k < E; k++) sm[g.smidx(g.row(gi - 1, k))] = x[k];
            g.sync();
#pragma unroll
            for (int k = 0; k < E; k++) x[k] = sm[g.smidx(g.row(gi, k))];
        }
        const int blo = G::blo(gi), bhi = G::bhi(gi), lo = G::lo(gi);
        const int tlow = g.t & ((1 << lo) - 1);
        const int thigh = (g.t >> lo) << (lo + LOGE);
#pragma unroll
        for (int st = 0; st < LOGE; st++) {
            const int b = INV ? blo + st : bhi - st;
            if (b >= blo && b <= bhi) {
                const int bb = b - lo;
                if (INV && FOLD && b == LOGM - 1) {
#pragma unroll
                    for (int j = 0; j < E; j++) {
                        if (j >= (1 << bb)) continue;
                        const u64 X = x[j], Y = x[j + (1 << bb)];
                        const u64 S = X + Y;
                        x[j] = S >= q2 ? S - q2 : S;
                        x[j + (1 << bb)] = X - Y + q2;
                    }
                    continue;
                }
                if (!INV && FOLD && gi == 0 && st == 0) {
                    const u64 q17 = 17 * q;
#pragma unroll
                    for (int j = 0; j < E; j++) {
                        if (j >= (1 << bb)) continue;
                        const u64 X = x[j], T = x[j + (1 << bb)];
                        x[j] = X + T;
                        x[j + (1 << bb)] = X - T + q17;
                    }
                    continue;
                }
#pragma unroll
                for (int k = 0; k < E; k++) {
                    if (k & (1 << bb)) continue;
                    // pairs that agree above bit bb share a twiddle; load it once
                    if (k & ((1 << bb) - 1)) continue;
                    const int r0 = tlow | (k << lo) | thigh;
                    const u64 widx = (u64)(M >> (b + 1)) * g.o + (u64)(r0 >> (b + 1));
                    const ulonglong2 wp = __ldg(reinterpret_cast<const ulonglong2 *>(tw) + widx);
                    const u64 w = wp.x, wsh = wp.y;
#pragma unroll
                    for (int j = 0; j < E; j++) {
                        if (j >= (1 << bb)) continue;
                        if (INV) gs_bfly(x[k + j], x[k + j + (1 << bb)], w, wsh, q, q2);
                        else if (OPEN) ct_bfly_open(x[k + j], x[k + j + (1 << bb)], w, wsh, q, qb);
                        else ct_bfly(x[k + j], x[k + j + (1 << bb)], w, wsh, q, q2);
                    }
                }
            }
        }
    }
    if (GG::OUT_STAGE) {
        g.sync();
#pragma unroll
        for (int k = 0; k < E; k++) sm[g.smidx(g.row(NG - 1, k))] = x[k];
        g.sync();
#pragma unroll
        for (int k = 0; k < E; k++) x[k] = sm[g.smidx(g.srow(k))];
    }
}

template <int LOGM, bool INV, bool COL, int MODE, int LOGEV, bool OPEN>
__device__ __forceinline__ void pass_body(NttTables tb, int log1, int log2, int tile, const NttJob &J, u64 *sm,
                                          const ModInfo &mi) {
    using GG = Geo<LOGM, INV, COL, LOGEV>;
    constexpr int E = GG::E;
    const GG g(log1, log2, tile);
    const u64 q = mi.q, q2 = 2 * q;
    const size_t N = (size_t)g.N1 * g.N2;
    const u64 *tw = (INV ? tb.itw : tb.tw) + (size_t)J.prime * 2 * N;  // (twiddle, companion) pairs

    u64 x[E];
    // 1. load straight into the first group's registers, through the producer's load mode.
    //    Conversion sources and the stores' operands take the read-only data path
    //    (__ldg): a position is read and written only by the thread that owns it, so
    //    an operand that is also the output (in place) is read before it is written.
    //    (Measured: the combine pass 16% faster; the plain first-pass load is no faster.)
    if (is_second(MODE)) {
#pragma unroll
        for (int k = 0; k < E; k++) x[k] = J.dst[g.gidx(g.lrow(k))];
    } else if (MODE == M_REDUCE) {
        const u64 *src = J.src;
        const u64 sub = J.conv_sub;
        const u64 c = J.c2[0] ? J.c2[0] : 1, csh = J.c2[0] ? J.c2_sh[0] : mi.one_sh;
#pragma unroll
        for (int k = 0; k < E; k++) {
            u64 v = shoup_lazy(__ldg(src + g.gidx(g.lrow(k))), c, csh, q);  // [0, 2q) for any 64-bit source
            if (OPEN) {
                x[k] = v + (q - sub);  // < 3q
            } else {
                v = v >= q ? v - q : v;
                x[k] = sub_mod(v, sub, q);
            }
        }
    } else if (MODE == M_CONVPRE) {
        // sum_s y_s * c2_s with lazy Shoup products: each term < 4q (open: estimated
        // quotient) or < 2q, the sum < 16q.  Open (a forward column pass): the
        // upper half of the first stage's pairs, k >= E/2, takes the constants
        // times that stage's twiddle (c2w, conv_sub_w) and the stage no product.
        const u64 *src = J.src;
        const u64 stride = J.src_stride;
        const int ns = (int)J.nsrc;
        const u64 sub = J.conv_sub, q4 = 4 * q;
#pragma unroll
        for (int k = 0; k < E; k++) x[k] = OPEN ? q - (k >= E / 2 ? J.conv_sub_w : sub) : 0;
#pragma unroll
        for (int sidx = 0; sidx < kMaxConvSrc; sidx++) {
            if (sidx < ns) {
                const u64 c2 = J.c2[sidx], c2sh = J.c2_sh[sidx];
                const u64 *sp = src + sidx * stride;
                if (OPEN) {
#pragma unroll
                    for (int k = 0; k < E / 2; k++) x[k] += shoup_lazy4(__ldg(sp + g.gidx(g.lrow(k))), c2, c2sh, q);
                    const u64 c2w = J.c2w[sidx], c2wsh = J.c2w_sh[sidx];
#pragma unroll
                    for (int k = E / 2; k < E; k++) x[k] += shoup_lazy4(__ldg(sp + g.gidx(g.lrow(k))), c2w, c2wsh, q);
                } else {
#pragma unroll
                    for (int k = 0; k < E; k++) x[k] += shoup_lazy(__ldg(sp + g.gidx(g.lrow(k))), c2, c2sh, q);
                }
            }
        }
        if (!OPEN) {
#pragma unroll
            for (int k = 0; k < E; k++) {
                u64 v = x[k];
                v = v >= q4 ? v - q4 : v;
                v = v >= q2 ? v - q2 : v;
                v = v >= q ? v - q : v;
                x[k] = sub_mod(v, sub, q);
            }
        }
    } else if (MODE == M_PLAIN) {
        const u64 *src = J.src;
#pragma unroll
        for (int k = 0; k < E; k++) x[k] = src[g.gidx(g.lrow(k))];
    } else if (MODE == M_PIECE) {
        // a base-2^w piece (< 2^w) of the source residue times c2[0]: a lazy Shoup product, [0, 2q)
        const u64 *src = J.src;
        const uint32_t sh = J.piece_shift;
        const u64 mk = J.piece_mask, c = J.c2[0], csh = J.c2_sh[0];
#pragma unroll
        for (int k = 0; k < E; k++) x[k] = shoup_lazy((src[g.gidx(g.lrow(k))] >> sh) & mk, c, csh, q);
    } else {  // M_INT64
        const int64_t *src = reinterpret_cast<const int64_t *>(J.src);
#pragma unroll
        for (int k = 0; k < E; k++) {
            const int64_t v = src[g.gidx(g.lrow(k))];
            x[k] = v >= 0 ? (u64)v % q : q - 1 - ((u64)(-(v + 1)) % q);
        }
    }

    // 2. butterfly groups
    constexpr bool FOLD_INV = INV && COL && (MODE == M_SCALED || MODE == M_SCALED_CONV);
    run_stages<LOGM, INV, COL, LOGEV, OPEN, (MODE == M_CONVPRE && OPEN && !INV && COL) || FOLD_INV>(g, x, sm, tw, q);

    // 3. store straight from the last group's registers; the first pass keeps
    //    lazy values, the second reduces them and fuses the consumer
    u64 *dst = J.dst;
    if (!is_second(MODE)) {
#pragma unroll
        for (int k = 0; k < E; k++) dst[g.gidx(g.srow(k))] = x[k];
    } else {
        const u64 *base = J.base, *extra = J.extra;
        const u64 mul = J.mul, mulsh = J.mul_sh, addk = J.conv_sub;
#pragma unroll
        for (int k = 0; k < E; k++) {
            const size_t gi = g.gidx(g.srow(k));
            u64 v = x[k];
            if (MODE == M_SCALED || MODE == M_SCALED_CONV) {
                // the upper half's constant carries the last stage's twiddle
                const bool up = FOLD_INV && k >= E / 2;
                v = add_mod(shoup(v, up ? J.mul_w : mul, up ? J.mul_w_sh : mulsh, q), addk, q);
            }
            else if (INV) v = shoup(v, mi.ninv, mi.ninv_sh, q);
            else if (OPEN) {
                v = v - __umul64hi(v, mi.one_sh) * q;  // Shoup product with w = 1: [0, 2q)
                v = v >= q ? v - q : v;
            } else {
                v = v >= q2 ? v - q2 : v;
                v = v >= q ? v - q : v;
            }
            if (MODE == M_COMBINE) {
                v = shoup(sub_mod(__ldg(base + gi), v, q), mul, mulsh, q);
                if (extra) v = add_mod(v, __ldg(extra + gi), q);
            }
            if (MODE == M_SCALED_CONV) {
                // sum_s base_s * c2_s as lazy Shoup products (< 8q), reduced, subtracted
                u64 c = 0;
#pragma unroll
                for (int sidx = 0; sidx < kMaxConvSrc; sidx++)
                    if (sidx < (int)J.nsrc) c += shoup_lazy(__ldg(base + sidx * J.src_stride + gi), J.c2[sidx], J.c2_sh[sidx], q);
                c = c >= 4 * q ? c - 4 * q : c;
                c = c >= q2 ? c - q2 : c;
                c = c >= q ? c - q : c;
                v = sub_mod(v, c, q);
            }
            dst[gi] = v;
        }
    }
}

// open butterflies for forward transforms modulo primes below 2^57, Harvey's otherwise
template <int LOGM, bool INV, bool COL, int MODE, int LOGEV>
__device__ __forceinline__ void pass_dispatch(NttTables tb, int log1, int log2, int tile, const NttJob &J,
                                              u64 *sm, const ModInfo &mi) {
    if constexpr (!INV) {
        if (mi.q < kOpenBound) pass_body<LOGM, INV, COL, MODE, LOGEV, true>(tb, log1, log2, tile, J, sm, mi);
        else pass_body<LOGM, INV, COL, MODE, LOGEV, false>(tb, log1, log2, tile, J, sm, mi);
    } else {
        pass_body<LOGM, INV, COL, MODE, LOGEV, false>(tb, log1, log2, tile, J, sm, mi);
    }
}

template <int LOGM, bool INV, bool COL, int MODE, int LOGEV>
__global__ void __launch_bounds__(kThreads, LOGEV >= 4 ? 3 : 4) ntt_pass_kernel(PassParams P) {
    extern __shared__ u64 sm[];
    __shared__ NttJob J;
    {   // the job descriptor, once per CTA
        const u64 *gj = reinterpret_cast<const u64 *>(P.jobs + blockIdx.y);
        u64 *dj = reinterpret_cast<u64 *>(&J);
        for (int i = threadIdx.x; i < (int)(sizeof(NttJob) / 8); i += blockDim.x) dj[i] = gj[i];
    }
    __syncthreads();
    const ModInfo mi = P.t.mods[J.prime];
    pass_dispatch<LOGM, INV, COL, MODE, LOGEV>(P.t, P.log1, P.log2, blockIdx.x, J, sm, mi);
}

template <int LOGM, bool INV, bool COL, int MODE, int LOGEV>
void run_pass(const PassParams &P, int njobs, cudaStream_t st) {
    constexpr int M = 1 << LOGM;
    constexpr int LOGE = LOGM >= LOGEV ? LOGEV : LOGM;
    constexpr int T = M >> LOGE;
    const int nsub = COL ? (1 << P.log2) : (1 << P.log1);
    const int sub_cta = std::min(kThreads / T, nsub);
    const int threads = sub_cta * T;
    constexpr int NG = (LOGM + LOGE - 1) / LOGE;
    const size_t smem = COL ? (NG < 2 ? 0 : (size_t)M * sub_cta * 8) : (size_t)sub_cta * (M + M / 16) * 8;
    for (int j0 = 0; j0 < njobs; j0 += 65535) {
        PassParams Q = P;
        Q.jobs = P.jobs + j0;
        dim3 grid(nsub / sub_cta, std::min(65535, njobs - j0));
        ntt_pass_kernel<LOGM, INV, COL, MODE, LOGEV><<<grid, threads, smem, st>>>(Q);
    }
}

template <bool INV, bool COL, int MODE, int LOGEV>
void by_size_v(int logm, const PassParams &P, int njobs, cudaStream_t st) {
    switch (logm) {
        case 5: run_pass<5, INV, COL, MODE, LOGEV>(P, njobs, st); break;
        case 6: run_pass<6, INV, COL, MODE, LOGEV>(P, njobs, st); break;
        case 7: run_pass<7, INV, COL, MODE, LOGEV>(P, njobs, st); break;
        case 8: run_pass<8, INV, COL, MODE, LOGEV>(P, njobs, st); break;
        default: throw Error(-1, "unsupported NTT pass size");
    }
}

template <bool INV, bool COL, int MODE>
void by_size(int logm, const PassParams &P, int njobs, cudaStream_t st) {
    if (P.t.loge == 4) by_size_v<INV, COL, MODE, 4>(logm, P, njobs, st);
    else by_size_v<INV, COL, MODE, 3>(logm, P, njobs, st);
}

// first pass: forward = column pass, inverse = row pass (inverse loads are plain)
template <bool INV>
void first_pass(int load_mode, int logm, const PassParams &P, int njobs, cudaStream_t st) {
    if constexpr (INV) {
        if (load_mode != LOAD_PLAIN) throw Error(-1, "inverse transforms load plain limbs");
        by_size<INV, !INV, M_PLAIN>(logm, P, njobs, st);
    } else {
        if (load_mode == LOAD_CONV_PRE) by_size<INV, !INV, M_CONVPRE>(logm, P, njobs, st);
        else if (load_mode == LOAD_REDUCE) by_size<INV, !INV, M_REDUCE>(logm, P, njobs, st);
        else if (load_mode == LOAD_INT64) by_size<INV, !INV, M_INT64>(logm, P, njobs, st);
        else if (load_mode == LOAD_PIECE) by_size<INV, !INV, M_PIECE>(logm, P, njobs, st);
        else if (load_mode == LOAD_PLAIN) by_size<INV, !INV, M_PLAIN>(logm, P, njobs, st);
        else throw Error(-1, "unsupported load mode");
    }
}

template <bool INV>
void second_pass(int store_mode, int logm, const PassParams &P, int njobs, cudaStream_t st) {
    if constexpr (INV) {
        if (store_mode == STORE_SCALED) by_size<INV, INV, M_SCALED>(logm, P, njobs, st);
        else if (store_mode == STORE_SCALED_CONV) by_size<INV, INV, M_SCALED_CONV>(logm, P, njobs, st);
        else if (store_mode == STORE_PLAIN) by_size<INV, INV, M_STORE>(logm, P, njobs, st);
        else throw Error(-1, "unsupported inverse store mode");
    } else {
        if (store_mode == STORE_COMBINE) by_size<INV, INV, M_COMBINE>(logm, P, njobs, st);
        else if (store_mode == STORE_PLAIN) by_size<INV, INV, M_STORE>(logm, P, njobs, st);
        else throw Error(-1, "unsupported forward store mode");
    }
}

// x * k * 2^-64 mod q in (0, 2q) for any 64-bit x and k < q (Montgomery
// reduction with R = 2^64: m = (x k mod R) q^-1 mod R cancels the low word,
// (x k - m q) / R = hi(x k) - hi(m q) lies in (-q, q)).
__device__ __forceinline__ u64 mont_lazy(u64 x, u64 k, u64 q, u64 qinv) {
    const u64 lo = x * k, hi = __umul64hi(x, k);
    const u64 m = lo * qinv;
    return (hi + q) - __umul64hi(m, q);
}

// Shared memory of the fused kernel: the row-pass exchange buffer, then the
// two accumulators of every thread's E elements, thread-private slots laid out
// [component][element][thread] (consecutive threads, consecutive words).
template <int LOGM, int LOGEV>
struct KsSmem {
    using GG = Geo<LOGM, false, false, LOGEV>;
    __host__ __device__ static size_t exch_words(int sub_cta) { return (size_t)sub_cta * (GG::M + GG::M / 16); }
    __host__ __device__ static size_t bytes(int sub_cta) {
        return (exch_words(sub_cta) + 2 * (size_t)GG::E * kThreads) * 8;
    }
};

// Bulk-copy (TMA) prefetch of a contiguous range into L2: no shared memory, no
// completion to wait for.  The address must be 16-byte aligned and the size a
// multiple of 16 bytes.
__device__ __forceinline__ void prefetch_l2_bulk(const void *p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

template <int LOGM, int LOGEV, bool OPEN>
__device__ __forceinline__ void keyswitch_up_body(NttTables tb, int log1, int log2, int tile, const KsJob &J,
                                                  u64 *sm, const ModInfo &mi) {
    using GG = Geo<LOGM, false, false, LOGEV>;
    constexpr int E = GG::E;
    const GG g(log1, log2, tile);
    const u64 q = mi.q, q2 = 2 * q;
    const size_t N = (size_t)g.N1 * g.N2;
    const u64 *tw = tb.tw + (size_t)J.prime * 2 * N;
    const int nthr = blockDim.x, tid = threadIdx.x;
    u64 *acc = sm + KsSmem<LOGM, LOGEV>::exch_words(g.sub_cta);
    auto slot = [&](int c, int k) -> u64 & { return acc[(c * E + k) * nthr + tid]; };
    const int nd = (int)J.ndig;
    // the CTA's rows are one contiguous tile of every limb it reads: while digit
    // d is transformed, the tiles of digit d + 1 (two key limbs and its source)
    // are prefetched into L2 by the bulk-copy engine
    const uint32_t tile_off = (uint32_t)g.sub0 * (uint32_t)g.N2;
    const uint32_t tile_bytes = (uint32_t)g.sub_cta * (uint32_t)g.N2 * 8;
    auto prefetch_digit = [&](int d) {
        if (tid == 0 && d < nd && tile_bytes % 16 == 0) {
            prefetch_l2_bulk(J.key[d] + 2 * (size_t)tile_off, 2 * tile_bytes);
            prefetch_l2_bulk(J.src[d] + tile_off, tile_bytes);
        }
    };
    prefetch_digit(0);
    for (int d = 0; d < nd; d++) {
        prefetch_digit(d + 1);
        u64 x[E];
        const u64 *src = J.src[d];
        if (d == J.own) {
#pragma unroll
            for (int k = 0; k < E; k++) x[k] = shoup_lazy(__ldg(src + g.gidx(g.srow(k))), mi.r64, mi.r64_sh, q);
        } else {
#pragma unroll
            for (int k = 0; k < E; k++) x[k] = __ldg(src + g.gidx(g.lrow(k)));
            run_stages<LOGM, false, false, LOGEV, OPEN>(g, x, sm, tw, q);
        }
        const ulonglong2 *kp = reinterpret_cast<const ulonglong2 *>(J.key[d]);  // (component 0, 1) pairs
#pragma unroll
        for (int k = 0; k < E; k++) {
            const size_t gi = g.gidx(g.srow(k));
            const ulonglong2 kk = __ldg(kp + gi);
            u64 v0 = mont_lazy(x[k], kk.x, q, J.qinv);
            u64 v1 = mont_lazy(x[k], kk.y, q, J.qinv);
            if (d > 0) {
                v0 += slot(0, k);
                v1 += slot(1, k);
                v0 = v0 >= q2 ? v0 - q2 : v0;
                v1 = v1 >= q2 ? v1 - q2 : v1;
            }
            slot(0, k) = v0;
            slot(1, k) = v1;
        }
    }
#pragma unroll
    for (int k = 0; k < E; k++) {
        const size_t gi = g.gidx(g.srow(k));
        u64 v0 = slot(0, k), v1 = slot(1, k);
        if (J.ex0) {
            v0 += shoup_lazy(J.ex0[gi], J.pm, J.pm_sh, q);
            v0 = v0 >= q2 ? v0 - q2 : v0;
        }
        if (J.ex1) {
            v1 += shoup_lazy(J.ex1[gi], J.pm, J.pm_sh, q);
            v1 = v1 >= q2 ? v1 - q2 : v1;
        }
        J.acc0[gi] = v0 >= q ? v0 - q : v0;
        J.acc1[gi] = v1 >= q ? v1 - q : v1;
    }
}

template <int LOGM, int LOGEV>
__global__ void __launch_bounds__(kThreads, LOGEV >= 4 ? 2 : 4) keyswitch_up_kernel(PassParams P, const KsJob *jobs) {
    extern __shared__ u64 sm[];
    __shared__ KsJob J;
    {
        const u64 *gj = reinterpret_cast<const u64 *>(jobs + blockIdx.y);
        u64 *dj = reinterpret_cast<u64 *>(&J);
        for (int i = threadIdx.x; i < (int)(sizeof(KsJob) / 8); i += blockDim.x) dj[i] = gj[i];
    }
    __syncthreads();
    const ModInfo mi = P.t.mods[J.prime];
    if (mi.q < kOpenBound) keyswitch_up_body<LOGM, LOGEV, true>(P.t, P.log1, P.log2, blockIdx.x, J, sm, mi);
    else keyswitch_up_body<LOGM, LOGEV, false>(P.t, P.log1, P.log2, blockIdx.x, J, sm, mi);
}

template <int LOGM, int LOGEV>
void run_keyswitch_up(const PassParams &P, const KsJob *jobs, int njobs, cudaStream_t st) {
    using GG = Geo<LOGM, false, false, LOGEV>;
    const int nsub = 1 << P.log1;
    const int sub_cta = std::min(kThreads / GG::T, nsub);
    TREQUIRE(sub_cta * GG::T == kThreads, -1, "fused ModUp pass needs full CTAs");
    const size_t smem = KsSmem<LOGM, LOGEV>::bytes(sub_cta);
    static std::atomic<uint64_t> opted{0};
    opt_in_smem((const void *)keyswitch_up_kernel<LOGM, LOGEV>, (int)KsSmem<LOGM, LOGEV>::bytes(kThreads / GG::T), opted);
    for (int j0 = 0; j0 < njobs; j0 += 65535) {
        dim3 grid(nsub / sub_cta, std::min(65535, njobs - j0));
        keyswitch_up_kernel<LOGM, LOGEV><<<grid, sub_cta * GG::T, smem, st>>>(P, jobs + j0);
    }
}

template <int LOGEV>
void keyswitch_up_by_size(int logm, const PassParams &P, const KsJob *jobs, int njobs, cudaStream_t st) {
    switch (logm) {
        case 5: run_keyswitch_up<5, LOGEV>(P, jobs, njobs, st); break;
        case 6: run_keyswitch_up<6, LOGEV>(P, jobs, njobs, st); break;
        case 7: run_keyswitch_up<7, LOGEV>(P, jobs, njobs, st); break;
        case 8: run_keyswitch_up<8, LOGEV>(P, jobs, njobs, st); break;
        default: throw Error(-1, "unsupported NTT pass size");
    }
}

// ---------------------------------------------------------------------------
// Persistent launches over jobs of several ring degrees.  Every pass of a
// transform of log N in [14, 16] has sub-problems of 128 or 256 points, a
// full CTA of 256 threads holds 256 / T of them and a tile is one such CTA's
// share of a limb.  The grid is a few resident CTAs per SM; each walks the
// tiles blockIdx.x, blockIdx.x + gridDim.x, ..., finds a tile's job in the
// tile_start prefix table, stages the job and its table set in shared memory
// when the job changes, and runs the job's pass body at the job's own size.
// (Contiguous runs of tiles per CTA, one search each, measured slower: 70.9
// against 63.3 ms for the 64-item batch.)
// ---------------------------------------------------------------------------
// Resident CTAs per SM of the persistent launches: a tile's geometry and
// table pointers live in registers (the single-degree kernels read them as
// kernel parameters), so these take up to 80 registers a thread.
constexpr int kMultiCtas = 3;  // 4 measured the same (62.96 vs 63.14 ms for the 64-item batch)
constexpr int kMultiKsCtas = 2;  // the fused ModUp row pass + key inner product: up to 128 registers

struct MultiParams {
    const TabEntry *tabs;
    const void *jobs;
    const uint32_t *tile_start;
    int njobs, total;
};

// the job a tile belongs to: the last j with tile_start[j] <= u
__device__ __forceinline__ int find_job(const uint32_t *ts, int njobs, uint32_t u) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(ts + mid) <= u) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// stage job j of a job array into shared memory (8-byte words)
template <class JOB>
__device__ __forceinline__ void stage_job(JOB &dst, const JOB *jobs, int j) {
    const u64 *gj = reinterpret_cast<const u64 *>(jobs + j);
    u64 *dj = reinterpret_cast<u64 *>(&dst);
    for (int i = threadIdx.x; i < (int)(sizeof(JOB) / 8); i += blockDim.x) dj[i] = gj[i];
}

template <bool INV, bool COL, int MODE>
__global__ void __launch_bounds__(kThreads, kMultiCtas) ntt_pass_multi_kernel(MultiParams P) {
    extern __shared__ u64 sm[];
    __shared__ NttJob J;
    // the job's table set, read from shared memory where used (raw storage: TabEntry's
    // default member initialisers cannot run for a __shared__ variable)
    __shared__ __align__(16) unsigned char te_raw[sizeof(TabEntry)];
    TabEntry &TE = *reinterpret_cast<TabEntry *>(te_raw);
    __shared__ int sj;
    const NttJob *jobs = static_cast<const NttJob *>(P.jobs);
    int jcur = -1;  // the staged job
    uint32_t jbeg = 0;
    for (uint32_t u = blockIdx.x; u < (uint32_t)P.total; u += gridDim.x) {
        __syncthreads();  // the previous tile is done with the exchange buffer (and J)
        if (threadIdx.x == 0) sj = find_job(P.tile_start, P.njobs, u);
        __syncthreads();
        if (sj != jcur) {  // uniform: stage the job and its table set when the job changes
            jcur = sj;
            stage_job(J, jobs, jcur);
            __syncthreads();
            stage_job(TE, P.tabs, (int)J.tab);
            jbeg = __ldg(P.tile_start + jcur);
            __syncthreads();
        }
        const NttTables &tb = TE.t;
        const int log1 = (TE.log_n + 1) / 2, log2 = TE.log_n / 2;
        const int tile = (int)(u - jbeg);
        const ModInfo mi = tb.mods[J.prime];
        switch (COL ? log1 : log2) {
            case 7: pass_dispatch<7, INV, COL, MODE, 3>(tb, log1, log2, tile, J, sm, mi); break;
            case 8: pass_dispatch<8, INV, COL, MODE, 3>(tb, log1, log2, tile, J, sm, mi); break;
            default: break;  // refused on the host
        }
    }
}

__global__ void __launch_bounds__(kThreads, kMultiKsCtas) keyswitch_up_multi_kernel(MultiParams P) {
    extern __shared__ u64 sm[];
    __shared__ KsJob J;
    // the job's table set, read from shared memory where used (raw storage: TabEntry's
    // default member initialisers cannot run for a __shared__ variable)
    __shared__ __align__(16) unsigned char te_raw[sizeof(TabEntry)];
    TabEntry &TE = *reinterpret_cast<TabEntry *>(te_raw);
    __shared__ int sj;
    const KsJob *jobs = static_cast<const KsJob *>(P.jobs);
    int jcur = -1;  // the staged job
    uint32_t jbeg = 0;
    for (uint32_t u = blockIdx.x; u < (uint32_t)P.total; u += gridDim.x) {
        __syncthreads();  // the previous tile is done with the exchange buffer (and J)
        if (threadIdx.x == 0) sj = find_job(P.tile_start, P.njobs, u);
        __syncthreads();
        if (sj != jcur) {  // uniform: stage the job and its table set when the job changes
            jcur = sj;
            stage_job(J, jobs, jcur);
            __syncthreads();
            stage_job(TE, P.tabs, (int)J.tab);
            jbeg = __ldg(P.tile_start + jcur);
            __syncthreads();
        }
        const NttTables &tb = TE.t;
        const int log1 = (TE.log_n + 1) / 2, log2 = TE.log_n / 2;
        const int tile = (int)(u - jbeg);
        const ModInfo mi = tb.mods[J.prime];
        const bool open = mi.q < kOpenBound;
        switch (log2) {
            case 7:
                if (open) keyswitch_up_body<7, 3, true>(tb, log1, log2, tile, J, sm, mi);
                else keyswitch_up_body<7, 3, false>(tb, log1, log2, tile, J, sm, mi);
                break;
            case 8:
                if (open) keyswitch_up_body<8, 3, true>(tb, log1, log2, tile, J, sm, mi);
                else keyswitch_up_body<8, 3, false>(tb, log1, log2, tile, J, sm, mi);
                break;
            default: break;  // refused on the host
        }
    }
}

int persistent_grid(int total, int per_sm) { return std::max(1, std::min(total, sm_count() * per_sm)); }

template <bool INV, bool COL, int MODE>
void run_multi(const MultiParams &P, cudaStream_t st) {
    // the exchange buffer is the same for 128- and 256-point sub-problems
    constexpr size_t smem = COL ? (size_t)256 * 8 * 8 : (size_t)8 * (256 + 16) * 8;
    ntt_pass_multi_kernel<INV, COL, MODE><<<persistent_grid(P.total, kMultiCtas), kThreads, smem, st>>>(P);
}

}  // namespace

int ntt_pass_tiles(int log_n, bool col) {
    TREQUIRE(log_n >= 14 && log_n <= 16, -1, "launches over several ring degrees take log N in [14, 16]");
    const int log1 = (log_n + 1) / 2, log2 = log_n / 2;
    const int logm = col ? log1 : log2, loge = std::min(3, logm);
    const int T = 1 << (logm - loge), nsub = col ? (1 << log2) : (1 << log1);
    const int sub_cta = std::min(kThreads / T, nsub);
    TREQUIRE(sub_cta * T == kThreads, -1, "launches over several ring degrees need full CTAs");
    return nsub / sub_cta;
}

int keyswitch_up_tiles(int log_n) { return ntt_pass_tiles(log_n, false); }

void launch_ntt_pass_multi(bool inverse, int pass, const TabEntry *tabs, const NttJob *jobs_dev,
                           const uint32_t *tile_start, int njobs, int total_tiles, int load_mode, int store_mode,
                           cudaStream_t s) {
    if (njobs <= 0 || total_tiles <= 0) return;
    const MultiParams P{tabs, jobs_dev, tile_start, njobs, total_tiles};
    if (pass == 0) {  // forward: column pass with the load mode; inverse: row pass, plain loads
        if (inverse) {
            TREQUIRE(load_mode == LOAD_PLAIN, -1, "inverse transforms load plain limbs");
            run_multi<true, false, M_PLAIN>(P, s);
        } else if (load_mode == LOAD_CONV_PRE) run_multi<false, true, M_CONVPRE>(P, s);
        else if (load_mode == LOAD_REDUCE) run_multi<false, true, M_REDUCE>(P, s);
        else if (load_mode == LOAD_INT64) run_multi<false, true, M_INT64>(P, s);
        else if (load_mode == LOAD_PIECE) run_multi<false, true, M_PIECE>(P, s);
        else if (load_mode == LOAD_PLAIN) run_multi<false, true, M_PLAIN>(P, s);
        else throw Error(-1, "unsupported load mode");
    } else {  // forward: row pass with the store mode; inverse: column pass
        if (inverse) {
            if (store_mode == STORE_SCALED) run_multi<true, true, M_SCALED>(P, s);
            else if (store_mode == STORE_SCALED_CONV) run_multi<true, true, M_SCALED_CONV>(P, s);
            else if (store_mode == STORE_PLAIN) run_multi<true, true, M_STORE>(P, s);
            else throw Error(-1, "unsupported inverse store mode");
        } else {
            if (store_mode == STORE_COMBINE) run_multi<false, false, M_COMBINE>(P, s);
            else if (store_mode == STORE_PLAIN) run_multi<false, false, M_STORE>(P, s);
            else throw Error(-1, "unsupported forward store mode");
        }
    }
}

void launch_keyswitch_up_multi(const TabEntry *tabs, const KsJob *jobs_dev, const uint32_t *tile_start, int njobs,
                               int total_tiles, cudaStream_t s) {
    if (njobs <= 0 || total_tiles <= 0) return;
    const MultiParams P{tabs, jobs_dev, tile_start, njobs, total_tiles};
    const size_t smem = KsSmem<8, 3>::bytes(kThreads / Geo<8, false, false, 3>::T);  // the same at 128 points
    static std::atomic<uint64_t> opted{0};
    opt_in_smem((const void *)keyswitch_up_multi_kernel, (int)smem, opted);
    keyswitch_up_multi_kernel<<<persistent_grid(total_tiles, kMultiKsCtas), kThreads, smem, s>>>(P);
}

void launch_keyswitch_up(int log_n, const NttTables &t, const KsJob *jobs_dev, int njobs, cudaStream_t s) {
    if (njobs <= 0) return;
    PassParams P{};
    P.t = t;
    P.log1 = (log_n + 1) / 2;
    P.log2 = log_n / 2;
    // the row pass of a forward transform: sub-problems of N2 points, N1 of them
    if (t.loge == 4) keyswitch_up_by_size<4>(P.log2, P, jobs_dev, njobs, s);
    else keyswitch_up_by_size<3>(P.log2, P, jobs_dev, njobs, s);
}

void launch_ntt(bool inverse, int log_n, const NttTables &t, const NttJob *jobs_dev, int njobs, int load_mode,
                int store_mode, cudaStream_t s, int pass) {
    if (njobs <= 0) return;
    PassParams P;
    P.t = t;
    P.jobs = jobs_dev;
    P.log1 = (log_n + 1) / 2;  // rows: N1 >= N2
    P.log2 = log_n / 2;
    if (pass != 1) {
        P.first = 1; P.load_mode = load_mode; P.store_mode = STORE_PLAIN; P.scale_out = 0;
        if (!inverse) first_pass<false>(load_mode, P.log1, P, njobs, s);
        else first_pass<true>(load_mode, P.log2, P, njobs, s);
    }
    if (pass != 0) {
        P.first = 0; P.load_mode = LOAD_PLAIN; P.store_mode = store_mode; P.scale_out = inverse ? 1 : 0;
        if (!inverse) second_pass<false>(store_mode, P.log2, P, njobs, s);
        else second_pass<true>(store_mode, P.log1, P, njobs, s);
    }
}

}  // namespace tetris
