// Ring repacking (Algorithm 1, after Chen-Dai-Kim-Song): n <= N ciphertexts
// whose messages carry x_i in their constant coefficient become one ciphertext
// of sum_i x_i X^i.  Every input is multiplied by N^-1 mod Q; round r
// (r = 0 .. log N - 1) pairs c_j with c_{j+t}, t = N / 2^(r+1), and sets
//     c_j <- (c_j + X^t c_{j+t}) + phi_g(c_j - X^t c_{j+t}),
// phi_g = automorphism X -> X^g and its key switch, g = 2N - 1 first, then
// 5^(2^(r-1)) mod 2N.  The t pairs of a round are independent, so a round is
// one batch of t ciphertexts through every launch (the batched automorphism
// and key switch of the query path).  In the NTT domain X^t c is a pointwise
// product with the transform of X^t, recorded as a transform of the monomial.
#include <cstring>

#include "program.h"

namespace tetris {

namespace {

std::vector<uint32_t> repack_galois(int n) {
    std::vector<uint32_t> g = {(uint32_t)(2 * n - 1)};
    for (int r = 1; (1 << r) < n; r++) g.push_back((uint32_t)h_powmod(5, 1ull << (r - 1), 2 * (u64)n));
    return g;
}

std::unique_ptr<Program> record_repack(Ctx &C, uint32_t count, int level, double scale) {
    auto P = std::make_unique<Program>();
    P->ctx = &C;
    Rec R(C, *P);
    const int n = (int)C.N, nl = level + 1;
    const std::vector<uint32_t> gal = repack_galois(n);
    for (uint32_t g : gal) (void)find_key(C, g);  // every round's rotation key must be loaded
    // staging: N ciphertexts, the first `count` filled by the caller, the rest zero
    CtH x = R.new_ct(n, 2, level);
    x.scale = scale;
    P->hold.push_back(x.buf);
    TCHECK_CUDA(cudaMemsetAsync(x.base, 0, x.bstride * n * 8, C.stream));
    TCHECK_CUDA(cudaStreamSynchronize(C.stream));
    {
        InSlot sl;
        sl.dst = x.base;
        sl.row_words = sl.src_pitch = x.bstride * count;
        P->in_slots.push_back(sl);
    }
    {
        std::vector<NttJob> jobs;
        for (uint32_t b = 0; b < count; b++)
            for (int c = 0; c < 2; c++)
                for (int i = 0; i < nl; i++) {
                    NttJob j{};
                    j.src = j.dst = x.limb(b, c, i);
                    j.prime = i;
                    jobs.push_back(j);
                }
        R.ntt(false, jobs, LOAD_PLAIN, STORE_PLAIN);
    }
    // the monomials X^t, t = N/2, N/4, ..., 1, in the NTT domain (transformed out of place on every run)
    const int rounds = (int)gal.size();
    BufPtr mono = R.pool().alloc((size_t)rounds * nl * n);
    BufPtr mono_ntt = R.pool().alloc((size_t)rounds * nl * n);
    P->hold.push_back(mono);
    P->hold.push_back(mono_ntt);
    {
        std::vector<u64> host((size_t)rounds * nl * n, 0);
        for (int r = 0; r < rounds; r++)
            for (int i = 0; i < nl; i++) host[((size_t)r * nl + i) * n + (n >> (r + 1))] = 1;
        TCHECK_CUDA(cudaMemcpy(mono->ptr, host.data(), host.size() * 8, cudaMemcpyHostToDevice));
        std::vector<NttJob> jobs;
        for (int r = 0; r < rounds; r++)
            for (int i = 0; i < nl; i++) {
                NttJob j{};
                j.src = mono->ptr + ((size_t)r * nl + i) * n;
                j.dst = mono_ntt->ptr + ((size_t)r * nl + i) * n;
                j.prime = i;
                jobs.push_back(j);
            }
        R.ntt(false, jobs, LOAD_PLAIN, STORE_PLAIN);
    }
    // c = N^-1 x (per limb, N^-1 mod q_i)
    CtH c = R.new_ct(n, 2, level);
    c.scale = scale;
    {
        std::vector<EwJob> jobs;
        for (int b = 0; b < n; b++)
            for (int k = 0; k < 2; k++)
                for (int i = 0; i < nl; i++) {
                    EwJob j{};
                    j.op = EW_MUL_CONST;
                    j.prime = i;
                    j.a = x.limb(b, k, i);
                    j.dst = c.limb(b, k, i);
                    j.k = C.mods_host[i].ninv;
                    j.k_sh = C.mods_host[i].ninv_sh;
                    jobs.push_back(j);
                }
        R.ew(jobs);
    }
    for (int r = 0; r < rounds; r++) {
        const int t = n >> (r + 1);
        CtH lo = R.view(c.buf, c.base, t, 2, level, c.bstride, c.cstride, scale);
        CtH hi = R.view(c.buf, c.base + (size_t)t * c.bstride, t, 2, level, c.bstride, c.cstride, scale);
        CtH s = R.mul_plain(hi, mono_ntt->ptr + (size_t)r * nl * n, 0);
        s.scale = scale;
        CtH e = R.add(lo, s);
        CtH d = R.sub(lo, s);
        c = R.add(e, R.rotate(d, gal[r]));
        c.scale = scale;
    }
    CtH o = R.from_ntt(c);
    P->out_buf = o.buf;
    P->out_base = o.base;
    P->out_words = o.bstride;
    P->out_level = level;
    P->out_comps = 2;
    P->out_scale = scale;
    P->finalize();
    return P;
}

}  // namespace

void repack(Ctx &C, const u64 *cts, uint32_t count, int level, double scale, u64 *out, cudaStream_t s, bool device) {
    TREQUIRE(cts && out, TETRIS_EINVAL, "repack: null buffer");
    TREQUIRE(count >= 1 && count <= C.N, TETRIS_EINVAL, "repack: 1 to N ciphertexts");
    TREQUIRE(level >= 0 && level <= C.L(), TETRIS_ELEVEL, "repack: bad level");
    std::string key = "r:" + std::to_string(count) + ":" + std::to_string(level) + ":";
    {
        uint64_t b;
        std::memcpy(&b, &scale, 8);
        key += std::to_string(b);
    }
    auto it = C.programs.find(key);
    if (it == C.programs.end()) it = C.programs.emplace(key, record_repack(C, count, level, scale)).first;
    Program &P = *it->second;
    const cudaMemcpyKind in_kind = device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    P.in_slots[0].copy_from(cts, in_kind, s);
    if (C.profile) P.run_profiled(s, C.stats);
    else if (C.use_graph) P.run_graph(s);
    else P.run(s);
    TCHECK_CUDA(cudaMemcpyAsync(out, P.out_base, P.out_words * 8, device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                s));
    if (!device) TCHECK_CUDA(cudaStreamSynchronize(s));
}

}  // namespace tetris
