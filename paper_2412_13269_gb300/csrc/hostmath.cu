// Host-side modular arithmetic: constants for the device tables, prime and
// root selection.  Pure integer code; the same results on x86-64 and aarch64.
#include <algorithm>

#include "internal.h"

namespace tetris {

u64 h_mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }

u64 h_powmod(u64 a, u64 e, u64 q) {
    u64 r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = h_mulmod(r, a, q);
        a = h_mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}

u64 h_invmod(u64 a, u64 q) { return h_powmod(a, q - 2, q); }  // q prime

u64 h_shoup(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }
// Newton's iteration x <- x (2 - q x) doubles the correct low bits; x = q is
// right to 3 bits for odd q (q^2 = 1 mod 8), five steps reach 96 > 64.
u64 h_inv64(u64 q) {
    u64 x = q;
    for (int i = 0; i < 5; i++) x *= 2 - q * x;
    return x;
}

// Deterministic Miller-Rabin for 64-bit n (first twelve prime bases).
bool h_is_prime(u64 n) {
    static const u64 bases[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (u64 p : bases)
        if (n % p == 0) return n == p;
    u64 d = n - 1;
    int r = 0;
    while ((d & 1) == 0) {
        d >>= 1;
        r++;
    }
    for (u64 a : bases) {
        u64 x = h_powmod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int i = 1; i < r; i++) {
            x = h_mulmod(x, x, n);
            if (x == n - 1) {
                comp = false;
                break;
            }
        }
        if (comp) return false;
    }
    return true;
}

std::vector<u64> h_gen_primes(int bits, int count, int cong_log2, const std::vector<u64> &exclude) {
    TREQUIRE(bits >= 3 && bits <= 62 && cong_log2 >= 1 && cong_log2 < bits, -1, "gen_primes: bad sizes");
    const u64 m = 1ull << cong_log2;
    const u64 top = 1ull << bits, low = 1ull << (bits - 1);
    u64 q = (top - 1) / m * m + 1;
    if (q >= top) q -= m;
    std::vector<u64> out;
    while ((int)out.size() < count) {
        TREQUIRE(q >= low && q > m, -1, "gen_primes: not enough primes of that size");
        if (std::find(exclude.begin(), exclude.end(), q) == exclude.end() && h_is_prime(q)) out.push_back(q);
        q -= m;
    }
    return out;
}

// psi = g^((q-1)/2N) for the least generator g of Z_q^*; the factors of q-1
// are found by trial division of its odd part.
u64 h_primitive_2n_root(u64 q, u64 n) {
    TREQUIRE((q - 1) % (2 * n) == 0, -1, "prime is not 1 mod 2N");
    std::vector<u64> f = {2};
    u64 odd = q - 1;
    while ((odd & 1) == 0) odd >>= 1;
    for (u64 d = 3; d * d <= odd; d += 2)
        if (odd % d == 0) {
            f.push_back(d);
            while (odd % d == 0) odd /= d;
        }
    if (odd > 1) f.push_back(odd);
    for (u64 g = 2;; g++) {
        bool gen = true;
        for (u64 p : f)
            if (h_powmod(g, (q - 1) / p, q) == 1) {
                gen = false;
                break;
            }
        if (gen) {
            u64 psi = h_powmod(g, (q - 1) / (2 * n), q);
            TREQUIRE(h_powmod(psi, n, q) == q - 1, -1, "root check failed");
            return psi;
        }
    }
}

uint32_t bitrev(uint32_t x, int bits) {
    uint32_t r = 0;
    for (int i = 0; i < bits; i++) r |= ((x >> i) & 1u) << (bits - 1 - i);
    return r;
}

}  // namespace tetris
