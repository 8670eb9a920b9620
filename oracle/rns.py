"""RNS layer of the oracle: ctypes bindings to the C core, prime and root
selection, CRT reconstruction.

TEST INFRASTRUCTURE (see oracle/__init__.py).
"""
from __future__ import annotations

import ctypes as C
from functools import lru_cache

import numpy as np

from . import build as _build

_u64 = C.c_uint64
_p64 = C.POINTER(C.c_uint64)


@lru_cache(maxsize=1)
def lib():
    so = C.CDLL(_build.build())
    sig = {
        "or_mulmod": (_u64, [_u64, _u64, _u64]),
        "or_powmod": (_u64, [_u64, _u64, _u64]),
        "or_ntt": (None, [_p64, _u64, _u64, _u64]),
        "or_intt": (None, [_p64, _u64, _u64, _u64]),
        "or_ntt_direct": (None, [_p64, _p64, _u64, _u64, _u64]),
        "or_polymul": (None, [_p64, _p64, _p64, _u64, _u64, _u64]),
        "or_rns_polymul": (None, [_p64, _p64, _p64, _u64, _u64, _p64, _p64]),
        "or_rns_mul_scalar": (None, [_p64, _p64, _p64, _u64, _u64, _p64]),
        "or_rns_automorphism": (None, [_p64, _p64, _u64, _u64, _p64, _u64]),
        "or_rescale": (None, [_p64, _p64, _u64, _u64, _u64, _p64]),
        "or_base_convert": (None, [_p64, _p64, _u64, _p64, _u64, _u64, _p64]),
        "or_moddown": (None, [_p64, _u64, _u64, _p64, _u64, _p64]),
        "or_keyswitch": (None, [_p64, _u64, _p64, _u64, _u64, _u64, _u64, _p64, _p64, _u64, _p64]),
        "or_num_threads": (C.c_int, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(so, name)
        f.restype = res
        f.argtypes = args
    return so


def ptr(a: np.ndarray):
    assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"], (a.dtype, a.flags)
    return a.ctypes.data_as(_p64)


def u64arr(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.uint64))


# ---------------------------------------------------------------------------
# primes and roots
# ---------------------------------------------------------------------------
_MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)


def is_prime(n: int) -> bool:
    """Deterministic Miller-Rabin for n < 3.3e24 (first twelve prime bases)."""
    if n < 2:
        return False
    for p in _MR_BASES:
        if n % p == 0:
            return n == p
    d, r = n - 1, 0
    while d % 2 == 0:
        d //= 2
        r += 1
    for a in _MR_BASES:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(r - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def gen_primes(bits: int, count: int, congruence_log2: int = 17, exclude=()) -> list[int]:
    """The ``count`` largest primes q < 2^bits with q = 1 mod 2^congruence_log2,
    in descending order, skipping those in ``exclude``. With the default 2^17
    every ring degree N <= 2^16 has a primitive 2N-th root modulo each."""
    m = 1 << congruence_log2
    q = ((1 << bits) - 1) // m * m + 1
    if q >= (1 << bits):
        q -= m
    out = []
    ex = set(int(e) for e in exclude)
    while len(out) < count:
        if q < (1 << (bits - 1)):
            raise ValueError("not enough primes of that size")
        if q not in ex and is_prime(q):
            out.append(q)
        q -= m
    return out


def _factor_small(n: int) -> list[int]:
    fs, d = [], 2
    while d * d <= n:
        if n % d == 0:
            fs.append(d)
            while n % d == 0:
                n //= d
        d += 1
    if n > 1:
        fs.append(n)
    return fs


def primitive_2n_root(q: int, n: int) -> int:
    """The primitive 2N-th root of unity g^((q-1)/2N), g the least generator of Z_q^*."""
    assert (q - 1) % (2 * n) == 0
    # q - 1 = 2^a * odd; factor the odd part by trial division only after
    # removing the large power of two, which keeps it small for NTT primes.
    odd = q - 1
    while odd % 2 == 0:
        odd //= 2
    factors = [2] + (_factor_small(odd) if odd > 1 else [])
    g = 2
    while any(pow(g, (q - 1) // f, q) == 1 for f in factors):
        g += 1
    psi = pow(g, (q - 1) // (2 * n), q)
    assert pow(psi, n, q) == q - 1
    return psi


# ---------------------------------------------------------------------------
# CRT
# ---------------------------------------------------------------------------
def crt(residues: np.ndarray, moduli) -> list[int]:
    """residues[limb][k] -> list of integers in [0, prod moduli)."""
    moduli = [int(q) for q in moduli]
    Q = 1
    for q in moduli:
        Q *= q
    coef = []
    for q in moduli:
        Qh = Q // q
        coef.append(Qh * pow(Qh % q, -1, q))
    out = [0] * residues.shape[1]
    for i, c in enumerate(coef):
        row = residues[i].tolist()
        out = [o + c * int(r) for o, r in zip(out, row)]
    return [o % Q for o in out]


def centered(vals, Q: int) -> list[int]:
    h = Q // 2
    return [v - Q if v > h else v for v in vals]


def to_rns(vals, moduli) -> np.ndarray:
    """Integers (any sign, python ints or int64 array) -> uint64[limbs][N]."""
    if isinstance(vals, np.ndarray) and vals.dtype == np.int64:
        out = np.empty((len(moduli), vals.shape[0]), dtype=np.uint64)
        for i, q in enumerate(moduli):
            out[i] = np.mod(vals, np.int64(q)).astype(np.uint64) if q < (1 << 63) else None
        return out
    out = np.empty((len(moduli), len(vals)), dtype=np.uint64)
    for i, q in enumerate(moduli):
        out[i] = np.array([int(v) % int(q) for v in vals], dtype=np.uint64)
    return out
