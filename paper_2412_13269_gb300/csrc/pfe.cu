// Private-function-evaluation scoring step (Section 5.4.1; Algorithm 2, the
// loop building ct_i): for every record i,
//   out[i] = sum_j X^{e_ij} U_j   in (Z_q[X] / (X^N + 1))^2, one modulus q,
// where U_j encrypts the scientist's scoring polynomial u_{f_j} and e_ij is the
// record's attribute value in the exponent.  A monomial product is a
// negacyclic rotation: coefficient t of X^k a is a[t - k], negated where the
// index wraps (X^N = -1), so the step is a gather-add with no multiplications.
//
// Ring degrees above 2^12: one CTA per (record, component); a thread owns the
// coefficients t = tid + 256 r, so every warp access (the rotated reads of U_j
// and the write) is coalesced; the inputs are read from L2 for every record.
// Up to 2^12 (the paper's Set I): the staged kernel below.
#include "program.h"

namespace tetris {

namespace {

constexpr int kPfeThreads = 256;
constexpr int kPfeChunk = 16;  // coefficients per thread per pass over the inputs

__global__ void __launch_bounds__(kPfeThreads) pfe_kernel(const u64 *u, const uint32_t *exps, uint32_t m, int log_n,
                                                          u64 q, u64 *out) {
    extern __shared__ uint32_t e[];  // the record's m exponents, reduced mod 2N
    const uint64_t rec = blockIdx.x >> 1;
    const int c = blockIdx.x & 1;
    const int n = 1 << log_n;
    for (uint32_t j = threadIdx.x; j < m; j += blockDim.x) e[j] = exps[rec * m + j] & (uint32_t)(2 * n - 1);
    __syncthreads();
    u64 *dst = out + (rec * 2 + c) * (uint64_t)n;
    for (int t0 = 0; t0 < n; t0 += kPfeThreads * kPfeChunk) {
        u64 acc[kPfeChunk];
#pragma unroll
        for (int r = 0; r < kPfeChunk; r++) acc[r] = 0;
        for (uint32_t j = 0; j < m; j++) {
            const u64 *src = u + ((uint64_t)j * 2 + c) * n;
            int k = (int)e[j];
            const bool neg = k >= n;
            if (neg) k -= n;
#pragma unroll
            for (int r = 0; r < kPfeChunk; r++) {
                const int t = t0 + threadIdx.x + kPfeThreads * r;
                if (t < n) {
                    int s = t - k;
                    bool minus = neg;
                    if (s < 0) {
                        s += n;
                        minus = !minus;
                    }
                    const u64 v = src[s];
                    acc[r] = minus ? sub_mod(acc[r], v, q) : add_mod(acc[r], v, q);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < kPfeChunk; r++) {
            const int t = t0 + threadIdx.x + kPfeThreads * r;
            if (t < n) dst[t] = acc[r];
        }
    }
}

// N <= 2^12: a CTA of kPfeGroups x 256 threads computes kPfeGroups records of
// one component.  Each input polynomial U_j[c] is staged once in shared memory
// for all of them, in negacyclic-extended form ext = (U_j, -U_j) of 2N words,
// so that for any k in [0, 2N) coefficient t of X^k U_j is ext[(t - k) mod 2N]
// (X^N = -1): a read and an add per term, no sign logic.  The m terms are < q
// and summed without reduction (taken when m q < 2^64), then reduced once.
// Double-buffered: the next polynomial is loaded into registers while the
// current one is read.  Thread (g, l) owns coefficients l + 256 r of record g,
// so the rotated shared-memory reads of a warp are consecutive words.  The
// term reads (8 bytes each, from shared memory; a rotated warp read spans three
// wavefronts) bound the kernel.
constexpr int kPfeGroups = 4;
constexpr uint32_t kPfeStagedMaxM = 4096;

template <int LOGN>
__global__ void __launch_bounds__(kPfeThreads * kPfeGroups, 1)
    pfe_staged_kernel(const u64 *u, const uint32_t *exps, uint32_t m, uint64_t p, u64 q, u64 q_one_sh, u64 *out) {
    constexpr int n = 1 << LOGN;
    constexpr int R = n / kPfeThreads;                 // coefficients per thread
    constexpr int NT = kPfeThreads * kPfeGroups;
    constexpr int W = (n + NT - 1) / NT;               // staging words per thread
    extern __shared__ u64 pfe_sm[];                    // [2][2n] staging, then [kPfeGroups][m] exponents
    uint32_t *e = reinterpret_cast<uint32_t *>(pfe_sm + 4 * n);
    const int c = blockIdx.y;
    const uint64_t rec0 = (uint64_t)blockIdx.x * kPfeGroups;
    const int grp = threadIdx.x / kPfeThreads, lane = threadIdx.x % kPfeThreads;
    for (uint32_t i = threadIdx.x; i < kPfeGroups * m; i += NT) {
        const uint64_t r = rec0 + i / m;
        e[i] = r < p ? exps[r * m + i % m] & (uint32_t)(2 * n - 1) : 0;
    }
    auto src = [&](uint32_t j) { return u + ((uint64_t)j * 2 + c) * n; };
    auto stage = [&](u64 *buf, int t, u64 v) {
        buf[t] = v;
        buf[t + n] = v ? q - v : 0;
    };
    u64 nxt[W];
#pragma unroll
    for (int w = 0; w < W; w++) {
        const int t = threadIdx.x + NT * w;
        if (t < n) stage(pfe_sm, t, src(0)[t]);
    }
    u64 acc[R];
#pragma unroll
    for (int r = 0; r < R; r++) acc[r] = 0;
    for (uint32_t j = 0; j < m; j++) {
        __syncthreads();  // stage j is complete (and stage j - 1 is no longer read)
        const u64 *cur = pfe_sm + (j & 1) * 2 * n;
        if (j + 1 < m) {
#pragma unroll
            for (int w = 0; w < W; w++) {
                const int t = threadIdx.x + NT * w;
                if (t < n) nxt[w] = src(j + 1)[t];
            }
        }
        const int k = (int)e[grp * m + j];
#pragma unroll
        for (int r = 0; r < R; r++) acc[r] += cur[(lane + kPfeThreads * r - k) & (2 * n - 1)];
        if (j + 1 < m) {
            u64 *dstbuf = pfe_sm + ((j + 1) & 1) * 2 * n;
#pragma unroll
            for (int w = 0; w < W; w++) {
                const int t = threadIdx.x + NT * w;
                if (t < n) stage(dstbuf, t, nxt[w]);
            }
        }
    }
    const uint64_t rec = rec0 + grp;
    if (rec < p) {
        u64 *dst = out + (rec * 2 + c) * (uint64_t)n;
#pragma unroll
        for (int r = 0; r < R; r++) {
            u64 v = acc[r] - __umul64hi(acc[r], q_one_sh) * q;  // Shoup product with w = 1: [0, 2q)
            dst[lane + kPfeThreads * r] = v >= q ? v - q : v;
        }
    }
}

template <int LOGN>
void run_pfe_staged(const u64 *u, const uint32_t *exps, uint32_t m, uint64_t p, const ModInfo &mi, u64 *out,
                    cudaStream_t s) {
    const size_t stage_bytes = 4 * ((size_t)1 << LOGN) * 8;
    const size_t smem = stage_bytes + (size_t)kPfeGroups * m * 4;
    static std::atomic<uint64_t> opted{0};
    opt_in_smem((const void *)pfe_staged_kernel<LOGN>, (int)(stage_bytes + (size_t)kPfeGroups * kPfeStagedMaxM * 4), opted);
    dim3 grid((unsigned)((p + kPfeGroups - 1) / kPfeGroups), 2);
    pfe_staged_kernel<LOGN><<<grid, kPfeThreads * kPfeGroups, smem, s>>>(u, exps, m, p, mi.q, mi.one_sh, out);
}

}  // namespace

void pfe_scores(Ctx &C, const u64 *u, uint32_t m, const uint32_t *exps, uint64_t p, u64 *out, cudaStream_t s) {
    TREQUIRE(u && exps && out, TETRIS_EINVAL, "pfe: null buffer");
    TREQUIRE(m >= 1 && m <= 4096, TETRIS_EINVAL, "pfe: 1 to 4096 scoring functions");
    TREQUIRE(p >= 1 && p < (1ull << 30), TETRIS_EINVAL, "pfe: 1 to 2^30 - 1 records");  // grid of 2p CTAs
    const bool staged = (u128)m * C.q[0] < ((u128)1 << 64) && m <= kPfeStagedMaxM;  // the unreduced sum fits
    switch (staged ? C.log_n : 0) {
        case 10: run_pfe_staged<10>(u, exps, m, p, C.mods_host[0], out, s); break;
        case 11: run_pfe_staged<11>(u, exps, m, p, C.mods_host[0], out, s); break;
        case 12: run_pfe_staged<12>(u, exps, m, p, C.mods_host[0], out, s); break;
        default:
            pfe_kernel<<<(unsigned)(2 * p), kPfeThreads, m * sizeof(uint32_t), s>>>(u, exps, m, C.log_n, C.q[0], out);
    }
    TCHECK_CUDA(cudaGetLastError());
}

}  // namespace tetris
