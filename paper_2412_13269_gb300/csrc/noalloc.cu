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
    u64 *base = scratch_on(C.device);
    u64 *top = base;                                               // [ncomp][N] top limbs, coefficient domain
    NttJob *jobs_inv = reinterpret_cast<NttJob *>(base + kLimbWords);
    NttJob *jobs_fwd = jobs_inv + kNoAllocMaxJobs;

    const u64 ql = C.q[level], half = (ql - 1) / 2;
    std::vector<NttJob> ji, jf;
    for (int c = 0; c < ncomp; c++) {  // top limb -> [a_l + floor(q_l/2)]_{q_l}, coefficient domain
        NttJob j{};
        j.src = in + ((size_t)c * (level + 1) + level) * N;
        j.dst = top + (size_t)c * N;
        j.prime = level;
        j.mul = C.mods_host[level].ninv;
        j.mul_sh = C.mods_host[level].ninv_sh;
        j.conv_sub = half;
        ji.push_back(j);
    }
    for (int i = 0; i < level; i++) {
        const u64 qi = C.q[i];
        NttJob j{};
        j.prime = i;
        j.conv_sub = half % qi;
        j.mul = h_invmod(ql % qi, qi);
        j.mul_sh = h_shoup(j.mul, qi);
        for (int c = 0; c < ncomp; c++) {
            NttJob jc = j;
            jc.src = top + (size_t)c * N;
            jc.base = in + ((size_t)c * (level + 1) + i) * N;
            jc.dst = out + ((size_t)c * level + i) * N;
            jf.push_back(jc);
        }
    }
    // job tables: copied from pageable host memory (staged before return)
    TCHECK_CUDA(cudaMemcpyAsync(jobs_inv, ji.data(), ji.size() * sizeof(NttJob), cudaMemcpyHostToDevice, s));
    TCHECK_CUDA(cudaMemcpyAsync(jobs_fwd, jf.data(), jf.size() * sizeof(NttJob), cudaMemcpyHostToDevice, s));
    launch_ntt(true, C.log_n, C.nt, jobs_inv, (int)ji.size(), LOAD_PLAIN, STORE_SCALED, s);
    launch_ntt(false, C.log_n, C.nt, jobs_fwd, (int)jf.size(), LOAD_REDUCE, STORE_COMBINE, s);
    TCHECK_CUDA(cudaGetLastError());
}

}  // namespace tetris
