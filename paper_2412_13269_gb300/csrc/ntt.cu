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
// memory; each thread holds E = 16 elements in registers and runs four
// butterfly stages per visit (radix-16 groups), so a 256-point sub-problem
// takes two shared-memory round trips.  Stage bit b of a sub-problem of size
// M uses twiddle index (M >> (b+1)) * o + (r >> (b+1)), with o = 1 in the
// column pass and o = N1 + row in the row pass.
//
// Load modes fuse the producer: plain, int64 -> residue, or a fast base
// conversion from up to four source limbs (ModUp / ModDown / rescale), less a
// per-coefficient constant.  The combine store fuses the consumer:
// (extra) + (base - x) * mul.
#include "internal.h"

namespace tetris {

namespace {

constexpr int kThreads = 256;

struct PassParams {
    NttTables t;
    const NttJob *jobs;
    int log1, log2;
    int load_mode, store_mode;
    int scale_out;
    int first;
};

__device__ __forceinline__ u64 load_elem(const NttJob &J, const PassParams &P, size_t g, u64 q) {
    if (!P.first) return J.dst[g];
    if (P.load_mode == LOAD_PLAIN) return J.src[g];
    if (P.load_mode == LOAD_INT64) {
        int64_t x = reinterpret_cast<const int64_t *>(J.src)[g];
        if (x >= 0) return (u64)x % q;
        u64 r = (u64)(-(x + 1)) % q;  // -(x+1) >= 0 avoids overflow at INT64_MIN
        return q - 1 - r;
    }
    // LOAD_CONV
    Acc128 acc = {0, 0};
    for (uint32_t s = 0; s < J.nsrc; s++) {
        const u64 qs = P.t.mods[J.src_prime[s]].q;
        u64 y = add_mod(J.src[s * J.src_stride + g], J.add_s[s], qs);
        y = shoup(y, J.c1[s], J.c1_sh[s], qs);
        acc_mad(acc, y, J.c2[s]);
    }
    return sub_mod(reduce128(acc.hi, acc.lo, P.t.mods[J.prime]), J.conv_sub, q);
}

template <int LOGM, bool INV, bool COL>
__global__ void __launch_bounds__(kThreads) ntt_pass_kernel(PassParams P) {
    constexpr int M = 1 << LOGM;
    constexpr int LOGE = LOGM >= 4 ? 4 : LOGM;
    constexpr int E = 1 << LOGE;
    constexpr int T = M / E;
    constexpr int NG = (LOGM + LOGE - 1) / LOGE;
    extern __shared__ u64 sm[];

    const NttJob &J = P.jobs[blockIdx.y];
    const int N1 = 1 << P.log1, N2 = 1 << P.log2;
    const int nsub = COL ? N2 : N1;
    const int sub_cta = min(kThreads / T, nsub);
    const int sub0 = blockIdx.x * sub_cta;
    const int nthr = sub_cta * T;
    const int tid = threadIdx.x;
    if (tid >= nthr) return;  // never taken for the supported sizes; keeps syncs uniform
    const ModInfo mi = P.t.mods[J.prime];
    const u64 q = mi.q;
    const size_t N = (size_t)N1 * N2;
    const u64 *tw = (INV ? P.t.itw : P.t.tw) + (size_t)J.prime * N;
    const u64 *twsh = (INV ? P.t.itw_sh : P.t.tw_sh) + (size_t)J.prime * N;

    // shared layout: column pass [r][sub], row pass [sub][r] padded every 16 words
    auto smidx = [&](int r, int s) -> int {
        return COL ? r * sub_cta + s : s * (M + M / 16) + r + (r >> 4);
    };
    auto gidx = [&](int r, int s) -> size_t {
        return COL ? (size_t)r * N2 + sub0 + s : (size_t)(sub0 + s) * N2 + r;
    };

    // 1. load the tile
    for (int l = tid; l < M * sub_cta; l += nthr) {
        int r, s;
        if (COL) {
            r = l / sub_cta;
            s = l - r * sub_cta;
        } else {
            s = l >> LOGM;
            r = l & (M - 1);
        }
        sm[smidx(r, s)] = load_elem(J, P, gidx(r, s), q);
    }
    __syncthreads();

    // 2. butterfly groups
    const int s = COL ? tid % sub_cta : tid / T;
    const int t = COL ? tid / sub_cta : tid % T;
    const u64 o = COL ? 1 : (u64)(N1 + sub0 + s);
#pragma unroll
    for (int g = 0; g < NG; g++) {
        int blo, bhi, lo;
        if (!INV) {
            bhi = LOGM - 1 - g * LOGE;
            blo = bhi - LOGE + 1 < 0 ? 0 : bhi - LOGE + 1;
            lo = blo;
        } else {
            blo = g * LOGE;
            bhi = blo + LOGE - 1 > LOGM - 1 ? LOGM - 1 : blo + LOGE - 1;
            lo = blo < LOGM - LOGE ? blo : LOGM - LOGE;
        }
        const int tlow = t & ((1 << lo) - 1);
        const int thigh = (t >> lo) << (lo + LOGE);
        u64 x[E];
#pragma unroll
        for (int k = 0; k < E; k++) x[k] = sm[smidx(tlow | (k << lo) | thigh, s)];
#pragma unroll
        for (int st = 0; st < LOGE; st++) {
            const int b = INV ? blo + st : bhi - st;
            if (INV ? (b > bhi) : (b < blo)) break;
            const int half = 1 << (b - lo);
#pragma unroll
            for (int k = 0; k < E; k++) {
                if (k & half) continue;
                const int r0 = tlow | (k << lo) | thigh;
                const u64 widx = (u64)(M >> (b + 1)) * o + (u64)(r0 >> (b + 1));
                const u64 w = __ldg(tw + widx), wsh = __ldg(twsh + widx);
                const u64 u = x[k], v = x[k | half];
                if (!INV) {
                    const u64 vw = shoup(v, w, wsh, q);
                    x[k] = add_mod(u, vw, q);
                    x[k | half] = sub_mod(u, vw, q);
                } else {
                    x[k] = add_mod(u, v, q);
                    x[k | half] = shoup(sub_mod(u, v, q), w, wsh, q);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < E; k++) sm[smidx(tlow | (k << lo) | thigh, s)] = x[k];
        __syncthreads();
    }

    // 3. store
    for (int l = tid; l < M * sub_cta; l += nthr) {
        int r, ss;
        if (COL) {
            r = l / sub_cta;
            ss = l - r * sub_cta;
        } else {
            ss = l >> LOGM;
            r = l & (M - 1);
        }
        const size_t gi = gidx(r, ss);
        u64 v = sm[smidx(r, ss)];
        if (P.scale_out) v = shoup(v, mi.ninv, mi.ninv_sh, q);
        if (P.store_mode == STORE_COMBINE) {
            v = shoup(sub_mod(J.base[gi], v, q), J.mul, J.mul_sh, q);
            if (J.extra) v = add_mod(v, J.extra[gi], q);
        }
        J.dst[gi] = v;
    }
}

template <int LOGM, bool INV, bool COL>
void run_pass(const PassParams &P, int njobs, cudaStream_t st) {
    constexpr int M = 1 << LOGM;
    constexpr int T = M / (M >= 16 ? 16 : M);
    const int nsub = COL ? (1 << P.log2) : (1 << P.log1);
    const int sub_cta = std::min(kThreads / T, nsub);
    const int threads = sub_cta * T;
    const size_t smem = COL ? (size_t)M * sub_cta * 8 : (size_t)sub_cta * (M + M / 16) * 8;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(ntt_pass_kernel<LOGM, INV, COL>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        attr_set = true;
    }
    for (int j0 = 0; j0 < njobs; j0 += 65535) {
        PassParams Q = P;
        Q.jobs = P.jobs + j0;
        dim3 grid(nsub / sub_cta, std::min(65535, njobs - j0));
        ntt_pass_kernel<LOGM, INV, COL><<<grid, threads, smem, st>>>(Q);
    }
}

template <bool INV, bool COL>
void dispatch(int logm, const PassParams &P, int njobs, cudaStream_t st) {
    switch (logm) {
        case 5: run_pass<5, INV, COL>(P, njobs, st); break;
        case 6: run_pass<6, INV, COL>(P, njobs, st); break;
        case 7: run_pass<7, INV, COL>(P, njobs, st); break;
        case 8: run_pass<8, INV, COL>(P, njobs, st); break;
        default: throw Error(-1, "unsupported NTT pass size");
    }
}

}  // namespace

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
        if (!inverse) dispatch<false, true>(P.log1, P, njobs, s);
        else dispatch<true, false>(P.log2, P, njobs, s);
    }
    if (pass != 0) {
        P.first = 0; P.load_mode = LOAD_PLAIN; P.store_mode = store_mode; P.scale_out = inverse ? 1 : 0;
        if (!inverse) dispatch<false, false>(P.log2, P, njobs, s);
        else dispatch<true, true>(P.log1, P, njobs, s);
    }
}

}  // namespace tetris
