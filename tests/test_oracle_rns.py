"""Pins for the oracle's RNS layer against definitions it does not use itself:
Python big-integer arithmetic, sympy's primality test, the O(N^2) sum that
defines the NTT (written here in Python integers), the schoolbook negacyclic
product (Section 2.2: Z_Q[X]/(X^N+1)) and CRT reconstruction."""
import random

import numpy as np
import pytest

from oracle import rns
from oracle.rns import lib, ptr, u64arr

pytestmark = pytest.mark.filterwarnings("ignore")

BITS = [17, 31, 40, 50, 60, 61]


def prime_of(bits):
    return rns.gen_primes(bits, 1, congruence_log2=min(17, bits - 2))[0]


@pytest.mark.parametrize("bits", BITS)
def test_mulmod_powmod_match_bigint(bits):
    q = prime_of(bits)
    rnd = random.Random(bits)
    for _ in range(2000):
        a, b = rnd.randrange(q), rnd.randrange(q)
        assert lib().or_mulmod(a, b, q) == a * b % q
    for _ in range(200):
        a, e = rnd.randrange(q), rnd.randrange(1 << 62)
        assert lib().or_powmod(a, e, q) == pow(a, e, q)
    # edge values
    for a, b in [(q - 1, q - 1), (0, q - 1), (1, q - 1), (q - 2, q - 1)]:
        assert lib().or_mulmod(a, b, q) == a * b % q


def test_is_prime_matches_sympy():
    sympy = pytest.importorskip("sympy")
    rnd = random.Random(5)
    cands = [rnd.randrange(1 << 61) | 1 for _ in range(3000)] + list(range(1, 2000))
    cands += [3215031751, 2152302898747, 3474749660383, 341550071728321]   # strong pseudoprimes to small bases
    for n in cands:
        assert rns.is_prime(n) == bool(sympy.isprime(n)), n


@pytest.mark.parametrize("bits,count", [(50, 20), (60, 3), (40, 11)])
def test_gen_primes(bits, count):
    sympy = pytest.importorskip("sympy")
    ps = rns.gen_primes(bits, count)
    assert len(ps) == count and len(set(ps)) == count
    assert ps == sorted(ps, reverse=True)
    for q in ps:
        assert q.bit_length() == bits and q % (1 << 17) == 1 and sympy.isprime(q)
    # nothing skipped: every candidate between consecutive picks is composite
    top = ((1 << bits) - 1) // (1 << 17) * (1 << 17) + 1
    c = top
    while c > ps[-1]:
        assert (c in ps) == bool(sympy.isprime(c))
        c -= 1 << 17


@pytest.mark.parametrize("bits,logn", [(31, 3), (50, 12), (60, 16)])
def test_primitive_root(bits, logn):
    q = prime_of(bits) if bits != 31 else rns.gen_primes(31, 1)[0]
    n = 1 << logn
    psi = rns.primitive_2n_root(q, n)
    assert pow(psi, n, q) == q - 1 and pow(psi, 2 * n, q) == 1
    for d in range(1, logn + 1):  # order exactly 2N: psi^(2N/2^d) != 1 for the proper divisors
        assert pow(psi, (2 * n) >> d, q) != 1


def ntt_bigint(a, q, psi):
    n = len(a)
    return [sum(a[i] * pow(psi, (2 * k + 1) * i, q) for i in range(n)) % q for k in range(n)]


@pytest.mark.parametrize("logn", [3, 4, 6])
def test_ntt_matches_definition(logn):
    n = 1 << logn
    q = rns.gen_primes(40, 1)[0]
    psi = rns.primitive_2n_root(q, n)
    rnd = random.Random(logn)
    a = [rnd.randrange(q) for _ in range(n)]
    want = ntt_bigint(a, q, psi)
    x = u64arr(a)
    lib().or_ntt(ptr(x), n, q, psi)
    assert x.tolist() == want
    y = np.empty_like(x)
    lib().or_ntt_direct(ptr(u64arr(a)), ptr(y), n, q, psi)
    assert y.tolist() == want
    lib().or_intt(ptr(x), n, q, psi)
    assert x.tolist() == a


def test_ntt_roundtrip_large():
    n = 1 << 12
    q = rns.gen_primes(60, 1)[0]
    psi = rns.primitive_2n_root(q, n)
    a = np.random.default_rng(0).integers(0, q, n, dtype=np.uint64)
    x = a.copy()
    lib().or_ntt(ptr(x), n, q, psi)
    lib().or_intt(ptr(x), n, q, psi)
    assert np.array_equal(x, a)


def negacyclic_schoolbook(a, b, q):
    n = len(a)
    out = [0] * n
    for i in range(n):
        for j in range(n):
            k = i + j
            if k < n:
                out[k] += a[i] * b[j]
            else:
                out[k - n] -= a[i] * b[j]
    return [v % q for v in out]


@pytest.mark.parametrize("logn,bits", [(4, 31), (6, 50), (5, 60)])
def test_polymul_matches_schoolbook(logn, bits):
    n = 1 << logn
    q = rns.gen_primes(bits, 1)[0]
    psi = rns.primitive_2n_root(q, n)
    rnd = random.Random(n)
    a = [rnd.randrange(q) for _ in range(n)]
    b = [rnd.randrange(q) for _ in range(n)]
    out = np.empty(n, dtype=np.uint64)
    lib().or_polymul(ptr(u64arr(a)), ptr(u64arr(b)), ptr(out), n, q, psi)
    assert out.tolist() == negacyclic_schoolbook(a, b, q)


def test_crt_roundtrip():
    mods = rns.gen_primes(50, 4)
    rnd = random.Random(1)
    Q = 1
    for q in mods:
        Q *= q
    vals = [rnd.randrange(Q) for _ in range(64)]
    r = rns.to_rns(vals, mods)
    assert rns.crt(r, mods) == vals
    cen = rns.centered(vals, Q)
    assert all(-Q // 2 <= v <= Q // 2 for v in cen)
    # int64 path of to_rns agrees with the python-int path
    x = np.array([rnd.randrange(-(1 << 60), 1 << 60) for _ in range(64)], dtype=np.int64)
    assert np.array_equal(rns.to_rns(x, mods), rns.to_rns([int(v) for v in x], mods))
