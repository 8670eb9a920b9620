// Elementwise kernels over lists of limbs (each limb = N residues of one
// prime).  All of them stream HBM: a grid-stride loop over (limb, position)
// with 16-byte vector accesses where the operands allow it.
#include "internal.h"

namespace tetris {

namespace {

constexpr int kEwThreads = 256;

// grid-stride kernels: a few resident CTAs per SM
int grid_for(size_t work_items) {
    const int sms = sm_count();
    size_t want = (work_items + kEwThreads - 1) / kEwThreads;
    size_t cap = (size_t)sms * 8;
    return (int)std::max<size_t>(1, std::min(want, cap));
}

// One CTA per (job, chunk of 2 * kEwThreads positions): the descriptor is
// staged in shared memory once and each thread handles one 16-byte pair.
__global__ void __launch_bounds__(kEwThreads) ew_kernel(const EwJob *jobs, int log_n, const ModInfo *mods,
                                                         const TabEntry *tabs) {
    __shared__ EwJob J;
    {
        const u64 *gj = reinterpret_cast<const u64 *>(jobs + blockIdx.y);
        u64 *dj = reinterpret_cast<u64 *>(&J);
        for (int i = threadIdx.x; i < (int)(sizeof(EwJob) / 8); i += blockDim.x) dj[i] = gj[i];
    }
    __syncthreads();
    if (tabs) {  // a job of one of several ring degrees: its own N and primes
        log_n = tabs[J.tab].log_n;
        mods = tabs[J.tab].t.mods;
    }
    const size_t p = ((size_t)blockIdx.x * kEwThreads + threadIdx.x) * 2;
    if (p >= ((size_t)1 << log_n)) return;
    {
        const ModInfo m = mods[J.prime];
        const u64 q = m.q;
        u64 r[2];
        switch (J.op) {
            case EW_ADD: {
                ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(J.a + p);
                ulonglong2 b = *reinterpret_cast<const ulonglong2 *>(J.b + p);
                r[0] = add_mod(a.x, b.x, q); r[1] = add_mod(a.y, b.y, q);
                break;
            }
            case EW_SUB: {
                ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(J.a + p);
                ulonglong2 b = *reinterpret_cast<const ulonglong2 *>(J.b + p);
                r[0] = sub_mod(a.x, b.x, q); r[1] = sub_mod(a.y, b.y, q);
                break;
            }
            case EW_MUL: {
                ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(J.a + p);
                ulonglong2 b = *reinterpret_cast<const ulonglong2 *>(J.b + p);
                r[0] = mul_mod(a.x, b.x, m); r[1] = mul_mod(a.y, b.y, m);
                break;
            }
            case EW_MUL_CONST: {
                ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(J.a + p);
                r[0] = shoup(a.x, J.k, J.k_sh, q); r[1] = shoup(a.y, J.k, J.k_sh, q);
                break;
            }
            case EW_ADD_CONST: {
                ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(J.a + p);
                r[0] = add_mod(a.x, J.k, q); r[1] = add_mod(a.y, J.k, q);
                break;
            }
            case EW_NEG: {
                ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(J.a + p);
                r[0] = a.x ? q - a.x : 0; r[1] = a.y ? q - a.y : 0;
                break;
            }
            case EW_COPY: {
                ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(J.a + p);
                r[0] = a.x; r[1] = a.y;
                break;
            }
            case EW_FMA: {
                ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(J.a + p);
                ulonglong2 b = *reinterpret_cast<const ulonglong2 *>(J.b + p);
                ulonglong2 c = *reinterpret_cast<const ulonglong2 *>(J.c + p);
                r[0] = add_mod(mul_mod(a.x, b.x, m), c.x, q); r[1] = add_mod(mul_mod(a.y, b.y, m), c.y, q);
                break;
            }
            case EW_ADD_MUL_CONST: {  // b + k * a
                ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(J.a + p);
                ulonglong2 b = *reinterpret_cast<const ulonglong2 *>(J.b + p);
                r[0] = add_mod(b.x, shoup(a.x, J.k, J.k_sh, q), q);
                r[1] = add_mod(b.y, shoup(a.y, J.k, J.k_sh, q), q);
                break;
            }
            case EW_REDUCE: {
                ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(J.a + p);
                u64 x = a.x - __umul64hi(a.x, m.one_sh) * q, y = a.y - __umul64hi(a.y, m.one_sh) * q;
                r[0] = x >= q ? x - q : x;
                r[1] = y >= q ? y - q : y;
                break;
            }
            case EW_TENSOR:
            case EW_TENSOR_ACC: {
                ulonglong2 a0 = *reinterpret_cast<const ulonglong2 *>(J.a + p);
                ulonglong2 a1 = *reinterpret_cast<const ulonglong2 *>(J.a1 + p);
                ulonglong2 b0 = *reinterpret_cast<const ulonglong2 *>(J.b + p);
                ulonglong2 b1 = *reinterpret_cast<const ulonglong2 *>(J.b1 + p);
                ulonglong2 d0, d1, d2;
                d0.x = mul_mod(a0.x, b0.x, m); d0.y = mul_mod(a0.y, b0.y, m);
                d2.x = mul_mod(a1.x, b1.x, m); d2.y = mul_mod(a1.y, b1.y, m);
                {
                    Acc128 c = {0, 0};
                    acc_mad(c, a0.x, b1.x); acc_mad(c, a1.x, b0.x);
                    d1.x = reduce128(c.hi, c.lo, m);
                    Acc128 e = {0, 0};
                    acc_mad(e, a0.y, b1.y); acc_mad(e, a1.y, b0.y);
                    d1.y = reduce128(e.hi, e.lo, m);
                }
                if (J.op == EW_TENSOR_ACC) {
                    const ulonglong2 c0 = *reinterpret_cast<const ulonglong2 *>(J.c + p);
                    const ulonglong2 c1 = *reinterpret_cast<const ulonglong2 *>(J.c1 + p);
                    const ulonglong2 c2 = *reinterpret_cast<const ulonglong2 *>(J.c2 + p);
                    d0.x = add_mod(d0.x, c0.x, q); d0.y = add_mod(d0.y, c0.y, q);
                    d1.x = add_mod(d1.x, c1.x, q); d1.y = add_mod(d1.y, c1.y, q);
                    d2.x = add_mod(d2.x, c2.x, q); d2.y = add_mod(d2.y, c2.y, q);
                }
                *reinterpret_cast<ulonglong2 *>(J.dst + p) = d0;
                *reinterpret_cast<ulonglong2 *>(J.d1 + p) = d1;
                *reinterpret_cast<ulonglong2 *>(J.d2 + p) = d2;
                return;
            }
            case EW_RESCALE_COEF: {
                // t = [k2 b + k4]_{q2} (b < q2), then (k a - [t]_q + k5) * k3 modulo q
                const ModInfo m2 = mods[J.prime2];
                ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(J.a + p);
                ulonglong2 b = *reinterpret_cast<const ulonglong2 *>(J.b + p);
                u64 t0 = add_mod(shoup(b.x, J.k2, J.k2_sh, m2.q), J.k4, m2.q);
                u64 t1 = add_mod(shoup(b.y, J.k2, J.k2_sh, m2.q), J.k4, m2.q);
                t0 = t0 - __umul64hi(t0, m.one_sh) * q;
                t1 = t1 - __umul64hi(t1, m.one_sh) * q;
                t0 = t0 >= q ? t0 - q : t0;
                t1 = t1 >= q ? t1 - q : t1;
                r[0] = shoup(add_mod(sub_mod(shoup(a.x, J.k, J.k_sh, q), t0, q), J.k5, q), J.k3, J.k3_sh, q);
                r[1] = shoup(add_mod(sub_mod(shoup(a.y, J.k, J.k_sh, q), t1, q), J.k5, q), J.k3, J.k3_sh, q);
                break;
            }
            default:
                r[0] = r[1] = 0;
        }
        *reinterpret_cast<ulonglong2 *>(J.dst + p) = make_ulonglong2(r[0], r[1]);
    }
}

// Tensor products (and tensor-accumulate) without the generic descriptor
// staging: every thread reads the job's fields through the read-only cache,
// handles two 16-byte pairs with all operand loads issued first, and forms
// a0 b1 + a1 b0 as (a0 + a1)(b0 + b1) - a0 b0 - a1 b1 on 128-bit products
// (three products instead of four; the same residues).
__device__ __forceinline__ void mul128(u64 a, u64 b, u64 &hi, u64 &lo) {
    lo = a * b;
    hi = __umul64hi(a, b);
}
__global__ void __launch_bounds__(kEwThreads, 4) tensor_kernel(const EwJob *jobs, int log_n, const ModInfo *mods,
                                                                const TabEntry *tabs) {
    const EwJob *jp = jobs + blockIdx.y;
    if (tabs) {  // a job of one of several ring degrees: its own N and primes
        const uint32_t tb = __ldg(&jp->tab);
        log_n = tabs[tb].log_n;
        mods = tabs[tb].t.mods;
    }
    const u64 *A0 = (const u64 *)__ldg((const unsigned long long *)&jp->a);
    const u64 *A1 = (const u64 *)__ldg((const unsigned long long *)&jp->a1);
    const u64 *B0 = (const u64 *)__ldg((const unsigned long long *)&jp->b);
    const u64 *B1 = (const u64 *)__ldg((const unsigned long long *)&jp->b1);
    u64 *D0 = (u64 *)__ldg((const unsigned long long *)&jp->dst);
    u64 *D1 = (u64 *)__ldg((const unsigned long long *)&jp->d1);
    u64 *D2 = (u64 *)__ldg((const unsigned long long *)&jp->d2);
    const int op = __ldg(&jp->op);
    const ModInfo m = mods[__ldg(&jp->prime)];
    const u64 q = m.q;
    const size_t n = (size_t)1 << log_n;
    size_t p[2];
    ulonglong2 a0[2], a1[2], b0[2], b1[2];
#pragma unroll
    for (int u = 0; u < 2; u++) {
        p[u] = (((size_t)blockIdx.x * 2 + u) * kEwThreads + threadIdx.x) * 2;
        if (p[u] < n) {
            a0[u] = *reinterpret_cast<const ulonglong2 *>(A0 + p[u]);
            a1[u] = *reinterpret_cast<const ulonglong2 *>(A1 + p[u]);
            b0[u] = *reinterpret_cast<const ulonglong2 *>(B0 + p[u]);
            b1[u] = *reinterpret_cast<const ulonglong2 *>(B1 + p[u]);
        }
    }
    const u64 *C0 = nullptr, *C1 = nullptr, *C2 = nullptr;
    if (op == EW_TENSOR_ACC) {
        C0 = (const u64 *)__ldg((const unsigned long long *)&jp->c);
        C1 = (const u64 *)__ldg((const unsigned long long *)&jp->c1);
        C2 = (const u64 *)__ldg((const unsigned long long *)&jp->c2);
    }
#pragma unroll
    for (int u = 0; u < 2; u++) {
        if (p[u] >= n) break;
        u64 r0[2], r1[2], r2[2];
        const u64 x0[2] = {a0[u].x, a0[u].y}, x1[2] = {a1[u].x, a1[u].y};
        const u64 y0[2] = {b0[u].x, b0[u].y}, y1[2] = {b1[u].x, b1[u].y};
#pragma unroll
        for (int e = 0; e < 2; e++) {
            u64 h0, l0, h2, l2, ht, lt;
            mul128(x0[e], y0[e], h0, l0);
            mul128(x1[e], y1[e], h2, l2);
            mul128(x0[e] + x1[e], y0[e] + y1[e], ht, lt);
            // (t - p0 - p2) as a 128-bit difference (non-negative)
            u64 l1 = lt - l0, h1 = ht - h0 - (lt < l0 ? 1 : 0);
            const u64 l1b = l1;
            l1 -= l2;
            h1 = h1 - h2 - (l1b < l2 ? 1 : 0);
            r0[e] = reduce128(h0, l0, m);
            r1[e] = reduce128(h1, l1, m);
            r2[e] = reduce128(h2, l2, m);
        }
        if (op == EW_TENSOR_ACC) {
            const ulonglong2 c0 = *reinterpret_cast<const ulonglong2 *>(C0 + p[u]);
            const ulonglong2 c1 = *reinterpret_cast<const ulonglong2 *>(C1 + p[u]);
            const ulonglong2 c2 = *reinterpret_cast<const ulonglong2 *>(C2 + p[u]);
            r0[0] = add_mod(r0[0], c0.x, q); r0[1] = add_mod(r0[1], c0.y, q);
            r1[0] = add_mod(r1[0], c1.x, q); r1[1] = add_mod(r1[1], c1.y, q);
            r2[0] = add_mod(r2[0], c2.x, q); r2[1] = add_mod(r2[1], c2.y, q);
        }
        *reinterpret_cast<ulonglong2 *>(D0 + p[u]) = make_ulonglong2(r0[0], r0[1]);
        *reinterpret_cast<ulonglong2 *>(D1 + p[u]) = make_ulonglong2(r1[0], r1[1]);
        *reinterpret_cast<ulonglong2 *>(D2 + p[u]) = make_ulonglong2(r2[0], r2[1]);
    }
}

__global__ void __launch_bounds__(kEwThreads) aut_kernel(const AutJob *jobs, int njobs, int log_n, uint32_t g) {
    const size_t n = (size_t)1 << log_n;
    const size_t total = n * njobs;
    const uint32_t mask2n = (uint32_t)(2 * n - 1);
    for (size_t it = blockIdx.x * (size_t)blockDim.x + threadIdx.x; it < total; it += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(it >> log_n);
        const uint32_t k = (uint32_t)(it & (n - 1));
        // index k holds A(psi^(2 brv(k) + 1)); the image at k is A(psi^(g (2 brv(k) + 1)))
        const uint32_t e = 2 * (__brev(k) >> (32 - log_n)) + 1;
        const uint32_t ge = (uint32_t)(((uint64_t)g * e) & mask2n);
        const uint32_t src = __brev((ge - 1) >> 1) >> (32 - log_n);
        jobs[j].dst[k] = jobs[j].src[src];
    }
}

// Pairs word (r, i, k) of the [rows][nl][n] pairs array with words (r, 0, i, k)
// and (r, 1, i, k) of the [rows][2][nl][n] limbs array, in either direction.
__global__ void __launch_bounds__(kEwThreads) interleave_kernel(u64 *limbs, u64 *pairs, size_t nl, size_t n,
                                                                 size_t total, bool to_pairs) {
    for (size_t it = blockIdx.x * (size_t)blockDim.x + threadIdx.x; it < total; it += (size_t)gridDim.x * blockDim.x) {
        const size_t r = it / (nl * n), rest = it % (nl * n);
        u64 *c0 = limbs + (2 * r) * nl * n + rest;
        u64 *c1 = c0 + nl * n;
        ulonglong2 *pp = reinterpret_cast<ulonglong2 *>(pairs) + it;
        if (to_pairs) {
            *pp = make_ulonglong2(*c0, *c1);
        } else {
            const ulonglong2 v = *pp;
            *c0 = v.x;
            *c1 = v.y;
        }
    }
}

// The automorphism of jobs at several ring degrees: one CTA per (job, chunk of
// kEwThreads positions), each job with its own N and Galois element.
__global__ void __launch_bounds__(kEwThreads) aut_multi_kernel(const AutJob *jobs, const TabEntry *tabs) {
    const AutJob J = jobs[blockIdx.y];
    const int log_n = tabs[J.tab].log_n;
    const uint32_t k = blockIdx.x * kEwThreads + threadIdx.x;
    if (k >= (1u << log_n)) return;
    const uint32_t mask2n = (2u << log_n) - 1;
    const uint32_t e = 2 * (__brev(k) >> (32 - log_n)) + 1;
    const uint32_t ge = (uint32_t)(((uint64_t)J.g * e) & mask2n);
    J.dst[k] = J.src[__brev((ge - 1) >> 1) >> (32 - log_n)];
}

// One CTA per (job, chunk of 2 * kEwThreads positions): the descriptor staged
// in shared memory once, 16-byte pairs, attribute loop unrolled for loads in flight.
__global__ void __launch_bounds__(kEwThreads) lincomb_kernel(const LinJob *jobs, int log_n, const ModInfo *mods) {
    __shared__ LinJob J;
    {
        const u64 *gj = reinterpret_cast<const u64 *>(jobs + blockIdx.y);
        u64 *dj = reinterpret_cast<u64 *>(&J);
        for (int i = threadIdx.x; i < (int)(sizeof(LinJob) / 8); i += blockDim.x) dj[i] = gj[i];
    }
    __syncthreads();
    const size_t p = ((size_t)blockIdx.x * kEwThreads + threadIdx.x) * 2;
    if (p >= ((size_t)1 << log_n)) return;
    const ModInfo m = mods[J.prime];
    Acc128 a0x = {0, 0}, a0y = {0, 0}, a1x = {0, 0}, a1y = {0, 0};
    const int na = (int)J.nattr;
#pragma unroll 4
    for (int a = 0; a < na; a++) {
        const ulonglong2 pt = __ldg(reinterpret_cast<const ulonglong2 *>(J.pt + a * J.pt_stride + p));
        const ulonglong2 w0 = *reinterpret_cast<const ulonglong2 *>(J.w0 + a * J.w_stride + p);
        const ulonglong2 w1 = *reinterpret_cast<const ulonglong2 *>(J.w1 + a * J.w_stride + p);
        acc_mad(a0x, pt.x, w0.x);
        acc_mad(a0y, pt.y, w0.y);
        acc_mad(a1x, pt.x, w1.x);
        acc_mad(a1y, pt.y, w1.y);
    }
    *reinterpret_cast<ulonglong2 *>(J.d0 + p) = make_ulonglong2(reduce128(a0x.hi, a0x.lo, m), reduce128(a0y.hi, a0y.lo, m));
    *reinterpret_cast<ulonglong2 *>(J.d1 + p) = make_ulonglong2(reduce128(a1x.hi, a1x.lo, m), reduce128(a1y.hi, a1y.lo, m));
}

__global__ void __launch_bounds__(kEwThreads) reduce_i64_kernel(const RedJob *jobs, int njobs, int log_n, const ModInfo *mods) {
    const size_t n = (size_t)1 << log_n;
    const size_t total = n * njobs;
    for (size_t it = blockIdx.x * (size_t)blockDim.x + threadIdx.x; it < total; it += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(it >> log_n);
        const size_t p = it & (n - 1);
        const RedJob &J = jobs[j];
        const u64 q = mods[J.prime].q;
        const int64_t x = J.src[p];
        u64 v;
        if (x >= 0) v = (u64)x % q;
        else v = q - 1 - ((u64)(-(x + 1)) % q);
        J.dst[p] = v;
    }
}

// Eight independent chains of lazy Shoup products per thread (the operation
// of a butterfly); the chains never leave registers.
__global__ void __launch_bounds__(kEwThreads) modmul_probe_kernel(u64 *sink, u64 q, u64 w, u64 wsh, int iters) {
    u64 x[8];
#pragma unroll
    for (int k = 0; k < 8; k++) x[k] = (blockIdx.x * 1315423911ull + threadIdx.x * 2654435761ull + k) % q;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < 8; k++) x[k] = shoup_lazy(x[k], w, wsh, q);
    }
    u64 r = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) r ^= x[k];
    if (r == 0x12345) sink[0] = r;  // keeps the chains live; practically never taken
}

}  // namespace

int sm_count() {
    constexpr int kDev = 64;
    static std::atomic<int> sms[kDev];
    int dev = 0;
    TCHECK_CUDA(cudaGetDevice(&dev));
    int v = (dev >= 0 && dev < kDev) ? sms[dev].load(std::memory_order_relaxed) : 0;
    if (v <= 0) {
        TCHECK_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
        TREQUIRE(v > 0, -3, "device reports no SMs");
        if (dev >= 0 && dev < kDev) sms[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

void opt_in_smem(const void *func, int bytes, std::atomic<uint64_t> &done) {
    int dev = 0;
    TCHECK_CUDA(cudaGetDevice(&dev));
    const uint64_t bit = (dev >= 0 && dev < 64) ? 1ull << dev : 0;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return;
    TCHECK_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    if (bit) done.fetch_or(bit, std::memory_order_release);
}

double modmul_peak_probe() {
    const u64 q = 1152921504606584833ull;  // a 60-bit prime = 1 mod 2^17
    const u64 w = 123456789012345ull % q;
    const u64 wsh = (u64)(((u128)w << 64) / q);
    const int sms = sm_count(), blocks = sms * 8, iters = 2048;
    u64 *sink = nullptr;
    TCHECK_CUDA(cudaMalloc(&sink, 8));
    cudaEvent_t a, b;
    TCHECK_CUDA(cudaEventCreate(&a));
    TCHECK_CUDA(cudaEventCreate(&b));
    modmul_probe_kernel<<<blocks, kEwThreads>>>(sink, q, w, wsh, 64);  // warm-up
    TCHECK_CUDA(cudaEventRecord(a));
    modmul_probe_kernel<<<blocks, kEwThreads>>>(sink, q, w, wsh, iters);
    TCHECK_CUDA(cudaEventRecord(b));
    TCHECK_CUDA(cudaEventSynchronize(b));
    float ms = 0;
    TCHECK_CUDA(cudaEventElapsedTime(&ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    return (double)blocks * kEwThreads * iters * 8 / (ms * 1e-3) / 1e9;
}

void launch_ew(const EwJob *jobs, int njobs, int log_n, const ModInfo *mods, cudaStream_t s, const TabEntry *tabs) {
    if (njobs <= 0) return;
    const size_t per_cta = 2 * (size_t)kEwThreads;
    const unsigned chunks = (unsigned)((((size_t)1 << log_n) + per_cta - 1) / per_cta);
    for (int j0 = 0; j0 < njobs; j0 += 65535) {
        dim3 grid(chunks, (unsigned)std::min(65535, njobs - j0));
        ew_kernel<<<grid, kEwThreads, 0, s>>>(jobs + j0, log_n, mods, tabs);
    }
}
void launch_tensor(const EwJob *jobs, int njobs, int log_n, const ModInfo *mods, cudaStream_t s, const TabEntry *tabs) {
    if (njobs <= 0) return;
    const size_t per_cta = 4 * (size_t)kEwThreads;
    const unsigned chunks = (unsigned)((((size_t)1 << log_n) + per_cta - 1) / per_cta);
    for (int j0 = 0; j0 < njobs; j0 += 65535) {
        dim3 grid(chunks, (unsigned)std::min(65535, njobs - j0));
        tensor_kernel<<<grid, kEwThreads, 0, s>>>(jobs + j0, log_n, mods, tabs);
    }
}
void launch_automorphism_multi(const AutJob *jobs, int njobs, const TabEntry *tabs, int max_log_n, cudaStream_t s) {
    if (njobs <= 0) return;
    const unsigned chunks = (unsigned)((((size_t)1 << max_log_n) + kEwThreads - 1) / kEwThreads);
    for (int j0 = 0; j0 < njobs; j0 += 65535) {
        dim3 grid(chunks, (unsigned)std::min(65535, njobs - j0));
        aut_multi_kernel<<<grid, kEwThreads, 0, s>>>(jobs + j0, tabs);
    }
}
void launch_interleave_pairs(u64 *limbs, u64 *pairs, size_t rows, size_t nl, size_t n, bool to_pairs,
                             cudaStream_t s) {
    const size_t total = rows * nl * n;
    if (total == 0) return;
    interleave_kernel<<<grid_for(total), kEwThreads, 0, s>>>(limbs, pairs, nl, n, total, to_pairs);
}
void launch_automorphism(const AutJob *jobs, int njobs, int log_n, uint32_t galois, cudaStream_t s) {
    if (njobs <= 0) return;
    aut_kernel<<<grid_for((size_t)njobs << log_n), kEwThreads, 0, s>>>(jobs, njobs, log_n, galois);
}
void launch_lincomb(const LinJob *jobs, int njobs, int log_n, const ModInfo *mods, cudaStream_t s) {
    if (njobs <= 0) return;
    const size_t per_cta = 2 * (size_t)kEwThreads;
    const unsigned chunks = (unsigned)((((size_t)1 << log_n) + per_cta - 1) / per_cta);
    for (int j0 = 0; j0 < njobs; j0 += 65535) {
        dim3 grid(chunks, (unsigned)std::min(65535, njobs - j0));
        lincomb_kernel<<<grid, kEwThreads, 0, s>>>(jobs + j0, log_n, mods);
    }
}
void launch_reduce_i64(const RedJob *jobs, int njobs, int log_n, const ModInfo *mods, cudaStream_t s) {
    if (njobs <= 0) return;
    reduce_i64_kernel<<<grid_for((size_t)njobs << log_n), kEwThreads, 0, s>>>(jobs, njobs, log_n, mods);
}

}  // namespace tetris
