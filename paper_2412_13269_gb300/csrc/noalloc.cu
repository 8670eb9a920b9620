// Allocation-free rescale on device-resident ciphertexts.
//
// Some callers cannot let a library allocate device memory while they run:
// cudaFree synchronises the whole device (stalling every other stream), and
// cudaMalloc fails or fragments memory once a serving process or another
// framework's caching allocator has reserved the GPU for itself.  This entry
// point therefore takes caller-owned input and output buffers and keeps its
// scratch -- the top limb of every component in the coefficient domain and
// the per-limb job tables of the two transforms -- in one fixed array that
// lives in this file.  The array is resident on every GPU that loads the
// library, until the process exits.
//
// Every call shares that array and it keeps the last call's contents.
// Nothing in it needs to start at zero (each call writes every word it later
// reads), but two calls whose work overlaps on the GPU (different streams,
// or different threads) race on it: callers must serialise them.
#include <mutex>

#include "program.h"

namespace tetris {

namespace {

constexpr size_t kNoAllocMaxComps = 3;
constexpr size_t kNoAllocMaxN = 1u << 16;
constexpr size_t kNoAllocMaxJobs = kNoAllocMaxComps * kMaxPrimes;
constexpr size_t kJobWords = (sizeof(NttJob) + 7) / 8;
constexpr size_t kLimbWords = kNoAllocMaxComps * kNoAllocMaxN;
constexpr size_t kScratchWords = kLimbWords + 2 * kNoAllocMaxJobs * kJobWords;

// The scratch.  In host code this name is only a stand-in for the symbol,
// not a device address: kernels get the address from cudaGetSymbolAddress.
static __device__ __align__(256) u64 g_rescale_scratch[kScratchWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
u64 *g_scratch_addr[kMaxDevices] = {};

// Resolve the scratch address on the current device, once per device.
u64 *scratch_on(int device) {
    TREQUIRE(device >= 0 && device < kMaxDevices, TETRIS_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_rescale_scratch);
        if (e != cudaSuccess) {
            cudaGetLastError();
            throw Error(TETRIS_ECUDA, std::string("cudaGetSymbolAddress of the rescale scratch: ") + cudaGetErrorString(e));
        }
        g_scratch_addr[device] = static_cast<u64 *>(p);
    }
    return g_scratch_addr[device];
}

// The job tables of one call, written on the device from the launch
// parameters alone (nothing is read from host memory after the call returns).
struct NoallocParams {
    const u64 *in;
    u64 *out, *top;
    NttJob *jobs_inv, *jobs_fwd;
    uint32_t N, level, ncomp, pad;
    u64 top_mul, top_mul_sh, top_half;               // N^-1 mod q_l (Shoup pair), floor(q_l/2)
    u64 top_mul_w, top_mul_w_sh;                     // N^-1 psi^-(N/2) mod q_l (the upper half's scale)
    u64 half[kMaxPrimes], mul[kMaxPrimes], mul_sh[kMaxPrimes];  // per q_i, i < l
};

__global__ void noalloc_tables_kernel(NoallocParams p) {
    const size_t N = p.N;
    for (uint32_t c = threadIdx.x; c < p.ncomp; c += blockDim.x) {  // top limb -> coefficient domain
        NttJob j{};
        j.src = p.in + ((size_t)c * (p.level + 1) + p.level) * N;
        j.dst = p.top + (size_t)c * N;
        j.prime = p.level;
        j.mul = p.top_mul;
        j.mul_sh = p.top_mul_sh;
        j.mul_w = p.top_mul_w;
        j.mul_w_sh = p.top_mul_w_sh;
        j.conv_sub = p.top_half;
        p.jobs_inv[c] = j;
    }
    for (uint32_t t = threadIdx.x; t < p.level * p.ncomp; t += blockDim.x) {
        const uint32_t i = t / p.ncomp, c = t % p.ncomp;
        NttJob j{};
        j.prime = i;
        j.conv_sub = p.half[i];
        j.mul = p.mul[i];
        j.mul_sh = p.mul_sh[i];
        j.src = p.top + (size_t)c * N;
        j.base = p.in + ((size_t)c * (p.level + 1) + i) * N;
        j.dst = p.out + ((size_t)c * p.level + i) * N;
        p.jobs_fwd[t] = j;
    }
}

// A caller buffer must be device (or managed) memory of the context's device.
void require_device_buffer(const Ctx &C, const void *ptr, const char *what) {
    cudaPointerAttributes a{};
    cudaError_t e = cudaPointerGetAttributes(&a, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error(TETRIS_EINVAL, std::string("rescale_noalloc: ") + what + " is not a CUDA pointer");
    }
    TREQUIRE((a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == C.device, TETRIS_EINVAL,
             std::string("rescale_noalloc: ") + what + " is not device memory of the context's device");
}

}  // namespace

size_t noalloc_scratch_bytes() { return kScratchWords * 8; }

// Same arithmetic as the recorded rescale (Section 2.5 of the paper):
//   out_i = (a_i + [floor(q_l/2)]_{q_i} - [[a_l + floor(q_l/2)]_{q_l}]_{q_i}) * q_l^-1.
void rescale_ntt_noalloc(Ctx &C, const u64 *in, u64 *out, int level, int ncomp, cudaStream_t s) {
    const size_t N = C.N;
    TREQUIRE(in && out, TETRIS_EINVAL, "rescale_noalloc: null buffer");
    TREQUIRE(level >= 1 && level <= C.L(), TETRIS_ELEVEL, "rescale_noalloc: level must be in [1, L]");
    TREQUIRE(ncomp >= 1 && (size_t)ncomp <= kNoAllocMaxComps, TETRIS_EINVAL,
             "rescale_noalloc: at most 3 components fit the fixed scratch");
    TREQUIRE(N <= kNoAllocMaxN, TETRIS_EINVAL, "rescale_noalloc: ring degree above 2^16");
    const size_t in_words = (size_t)ncomp * (level + 1) * N, out_words = (size_t)ncomp * level * N;
    const bool disjoint = out + out_words <= in || in + in_words <= out;
    TREQUIRE(disjoint, TETRIS_EINVAL, "rescale_noalloc: input and output overlap");
    require_device_buffer(C, in, "input");
    require_device_buffer(C, out, "output");
    u64 *base = scratch_on(C.device);

    NoallocParams p{};
    p.in = in;
    p.out = out;
    p.top = base;                                                  // [ncomp][N] top limbs, coefficient domain
    p.jobs_inv = reinterpret_cast<NttJob *>(base + kLimbWords);
    p.jobs_fwd = p.jobs_inv + kNoAllocMaxJobs;
    p.N = (uint32_t)N;
    p.level = (uint32_t)level;
    p.ncomp = (uint32_t)ncomp;
    const u64 ql = C.q[level], half = (ql - 1) / 2;
    p.top_mul = C.mods_host[level].ninv;
    p.top_mul_sh = C.mods_host[level].ninv_sh;
    p.top_half = half;
    p.top_mul_w = h_mulmod(p.top_mul, ql - h_powmod(C.psi[level], N / 2, ql), ql);
    p.top_mul_w_sh = h_shoup(p.top_mul_w, ql);
    for (int i = 0; i < level; i++) {
        const u64 qi = C.q[i];
        p.half[i] = half % qi;
        p.mul[i] = h_invmod(ql % qi, qi);
        p.mul_sh[i] = h_shoup(p.mul[i], qi);
    }
    noalloc_tables_kernel<<<1, 128, 0, s>>>(p);
    TCHECK_CUDA(cudaGetLastError());
    launch_ntt(true, C.log_n, C.nt, p.jobs_inv, ncomp, LOAD_PLAIN, STORE_SCALED, s);
    launch_ntt(false, C.log_n, C.nt, p.jobs_fwd, level * ncomp, LOAD_REDUCE, STORE_COMBINE, s);
    TCHECK_CUDA(cudaGetLastError());
}

}  // namespace tetris
