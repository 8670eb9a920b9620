// Device modular arithmetic on 64-bit residues, q < 2^61.
//
// Fixed multipliers use Shoup's precomputed-quotient multiplication
// (V. Shoup, NTL; D. Harvey, "Faster arithmetic for number-theoretic
// transforms", J. Symb. Comp. 2014): for w < q and w' = floor(w * 2^64 / q),
// a*w - floor(a*w'/2^64)*q lies in [0, 2q) for every 64-bit a.
// A 128-bit value hi*2^64 + lo is reduced as hi*(2^64 mod q) + lo with two
// such products (the second with w = 1, w' = floor(2^64/q)), which keeps
// every step a Shoup product.
#pragma once
#include <cstdint>

typedef uint64_t u64;
typedef unsigned __int128 u128;

struct ModInfo {
    u64 q;
    u64 r64, r64_sh;    // 2^64 mod q and its Shoup companion
    u64 one_sh;         // floor(2^64 / q)
    u64 ninv, ninv_sh;  // N^{-1} mod q
};

__device__ __forceinline__ u64 add_mod(u64 a, u64 b, u64 q) {
    u64 s = a + b;
    return s >= q ? s - q : s;
}
__device__ __forceinline__ u64 sub_mod(u64 a, u64 b, u64 q) {
    return a >= b ? a - b : a + q - b;
}
// a * w mod q in [0, 2q)
__device__ __forceinline__ u64 shoup_lazy(u64 a, u64 w, u64 wsh, u64 q) {
    u64 qt = __umul64hi(a, wsh);
    return a * w - qt * q;
}
__device__ __forceinline__ u64 shoup(u64 a, u64 w, u64 wsh, u64 q) {
    u64 r = shoup_lazy(a, w, wsh, q);
    return r >= q ? r - q : r;
}
// (hi * 2^64 + lo) mod q
__device__ __forceinline__ u64 reduce128(u64 hi, u64 lo, const ModInfo &m) {
    u64 r = shoup_lazy(hi, m.r64, m.r64_sh, m.q) + (lo - __umul64hi(lo, m.one_sh) * m.q);  // < 4q
    u64 q2 = m.q << 1;
    r = r >= q2 ? r - q2 : r;
    return r >= m.q ? r - m.q : r;
}
__device__ __forceinline__ u64 mul_mod(u64 a, u64 b, const ModInfo &m) {
    return reduce128(__umul64hi(a, b), a * b, m);
}
// 128-bit accumulator helpers
struct Acc128 {
    u64 lo, hi;
};
__device__ __forceinline__ void acc_mad(Acc128 &acc, u64 a, u64 b) {
    u64 lo = a * b, hi = __umul64hi(a, b);
    u64 nlo = acc.lo + lo;
    acc.hi += hi + (nlo < lo ? 1 : 0);
    acc.lo = nlo;
}
