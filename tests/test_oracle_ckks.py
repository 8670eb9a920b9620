"""Pins for the oracle's homomorphic operations on tiny rings, checked with
Python big integers against the statements they implement:

* rescale = round-half-up of c / q_l (Section 2.5) on the CRT value;
* fast base conversion = x + u*Q_D with 0 <= u < |D|, and exactly its
  integer definition sum_i [x_i (Q/q_i)^-1]_{q_i} (Q/q_i) reduced mod p;
* ModDown = floor((c + floor(P/2)) / P) - u with 0 <= u < K (Section 2.4.1),
  and exactly (c + floor(P/2) - V) / P with V that exact conversion;
* automorphism = a(X^g) reduced modulo X^N + 1 (Section 2.2);
* SwitchKeyGen: swk_j[0] + swk_j[1] s = e_j + w_j P s' exactly;
* SwitchKey / relinearisation / rotation: decryption identities with small
  error (Section 2.4.1, Appendix A.2, rotation semantics of Appendix A.1.2);
* 5 has order N/2 modulo 2N and {+-5^j} = Z*_2N (Section 2.2).
"""
import math
import random

import numpy as np
import pytest

import synth
from oracle import ckks, rns
from oracle.rns import lib, ptr, u64arr


def tiny_params(logn=4, nq=4, K=2, qbits=30, pbits=36, scale=2.0 ** 20):
    q = rns.gen_primes(qbits, nq, congruence_log2=logn + 1)
    p = rns.gen_primes(pbits, K, congruence_log2=logn + 1)
    return ckks.Params(logn, q, p, scale)


def rand_rns(rnd, mods, n):
    return u64arr([[rnd.randrange(q) for _ in range(n)] for q in mods])


def test_rescale_is_rounded_division():
    par = tiny_params(nq=4)
    rnd = random.Random(2)
    l = 3
    mods = par.q[: l + 1]
    a = np.stack([rand_rns(rnd, mods, par.N) for _ in range(2)])
    out = ckks.rescale(par, ckks.Ct(a, l, 1.0)).data
    Q = math.prod(mods)
    Qn = math.prod(mods[:l])
    ql = mods[l]
    for c in range(2):
        vals = rns.crt(a[c], mods)
        want = [((v + ql // 2) // ql) % Qn for v in vals]
        assert rns.crt(out[c], mods[:l]) == want


def test_base_convert_excess_bound():
    rnd = random.Random(3)
    src = rns.gen_primes(50, 3)
    dst = rns.gen_primes(60, 2) + rns.gen_primes(40, 2)
    n = 32
    x = rand_rns(rnd, src, n)
    out = np.empty((len(dst), n), dtype=np.uint64)
    lib().or_base_convert(ptr(x), ptr(u64arr(src)), len(src), ptr(u64arr(dst)), len(dst), n, ptr(out))
    Qs = math.prod(src)
    vals = rns.crt(x, src)
    for t, p in enumerate(dst):
        for k in range(n):
            got = int(out[t, k])
            ok = [u for u in range(len(src)) if (vals[k] + u * Qs) % p == got]
            assert ok, (t, k)


def exact_conversion(x_cols, src):
    """sum_i [x_i (Qs/q_i)^-1]_{q_i} (Qs/q_i) as one Python integer, for the
    residues x_cols[i] of one coefficient (the conversion's definition,
    without reduction by the target prime)."""
    Qs = math.prod(src)
    return sum(((int(x) * pow(Qs // qi, -1, qi)) % qi) * (Qs // qi) for x, qi in zip(x_cols, src))


def test_base_convert_exact():
    """The fast base conversion equals its integer definition reduced modulo
    each target prime, for every coefficient; and that integer is x + u Qs with
    the excess u in [0, |src|) determined coefficient by coefficient."""
    rnd = random.Random(13)
    for ns in (1, 2, 3, 4):
        src = rns.gen_primes(50, ns)
        dst = rns.gen_primes(60, 3) + rns.gen_primes(40, 2) + rns.gen_primes(50, 2, exclude=src)
        n = 48
        x = rand_rns(rnd, src, n)
        out = np.empty((len(dst), n), dtype=np.uint64)
        lib().or_base_convert(ptr(x), ptr(u64arr(src)), ns, ptr(u64arr(dst)), len(dst), n, ptr(out))
        Qs = math.prod(src)
        vals = rns.crt(x, src)
        for k in range(n):
            v = exact_conversion(x[:, k], src)
            u, r = divmod(v - vals[k], Qs)
            assert r == 0 and 0 <= u < ns
            for t, p in enumerate(dst):
                assert int(out[t, k]) == v % p, (ns, t, k)


def test_moddown_exact():
    """ModDown (Section 2.4.1's division by P with rounding) equals, modulo
    each q_i, the integer (c + floor(P/2) - V) / P, c the CRT value over Q P
    and V the exact fast conversion of the special residues of c + floor(P/2);
    the division is exact."""
    rnd = random.Random(14)
    for K in (1, 2, 3):
        qs = rns.gen_primes(50, 4)
        ps = rns.gen_primes(60, K)
        n = 40
        mods = qs + ps
        c = rand_rns(rnd, mods, n)
        out = np.empty((len(qs), n), dtype=np.uint64)
        lib().or_moddown(ptr(c), len(qs), K, ptr(u64arr(mods)), n, ptr(out))
        P = math.prod(ps)
        vals = rns.crt(c, mods)
        for k in range(n):
            shifted = [(int(c[len(qs) + j, k]) + P // 2) % pj for j, pj in enumerate(ps)]
            V = exact_conversion(shifted, ps)
            num = vals[k] + P // 2 - V
            assert num % P == 0
            for i, qi in enumerate(qs):
                assert int(out[i, k]) == (num // P) % qi, (K, i, k)


def test_moddown_is_rounded_division_up_to_K():
    rnd = random.Random(4)
    qs = rns.gen_primes(50, 3)
    ps = rns.gen_primes(60, 2)
    n = 32
    mods = qs + ps
    c = rand_rns(rnd, mods, n)
    out = np.empty((len(qs), n), dtype=np.uint64)
    lib().or_moddown(ptr(c), len(qs), len(ps), ptr(u64arr(mods)), n, ptr(out))
    P = math.prod(ps)
    Q = math.prod(qs)
    vals = rns.crt(c, mods)
    got = rns.crt(out, qs)
    for v, g in zip(vals, got):
        base = (v + P // 2) // P
        assert any((base - u) % Q == g for u in range(len(ps)))


def poly_automorphism_bigint(a, g, q):
    n = len(a)
    out = [0] * n
    for i, v in enumerate(a):
        j = i * g % (2 * n)
        if j < n:
            out[j] = (out[j] + v) % q
        else:
            out[j - n] = (out[j - n] - v) % q
    return out


@pytest.mark.parametrize("g", [5, 25, 3, 31, 2 * 16 - 1])
def test_automorphism_definition(g):
    par = tiny_params()
    rnd = random.Random(g)
    a = rand_rns(rnd, par.q, par.N)
    got = ckks.automorphism_poly(a, g, par.q)
    for i, q in enumerate(par.q):
        assert got[i].tolist() == poly_automorphism_bigint(a[i].tolist(), g, q)


def test_galois_group():
    for logn in (3, 4, 8, 12):
        N = 1 << logn
        order = next(k for k in range(1, 2 * N) if pow(5, k, 2 * N) == 1)
        assert order == N // 2
        gens = {pow(5, j, 2 * N) for j in range(N // 2)} | {(-pow(5, j, 2 * N)) % (2 * N) for j in range(N // 2)}
        assert gens == {x for x in range(2 * N) if x % 2 == 1}


def negacyclic(a, b):
    n = len(a)
    out = [0] * n
    for i in range(n):
        if a[i] == 0:
            continue
        for j in range(n):
            k = i + j
            if k < n:
                out[k] += a[i] * b[j]
            else:
                out[k - n] -= a[i] * b[j]
    return out


def test_switch_key_generation_identity():
    par = tiny_params()
    alpha = 2
    dnum = ckks.dnum_for(par.L, alpha)
    s = synth.ternary_secret(synth.stream(7, "s"), par.N, 10)
    s2 = synth.ternary_secret(synth.stream(7, "s2"), par.N, 10)
    d = synth.switch_key_draws(7, "k", dnum, par.moduli, par.N)
    swk = ckks.switch_key(par, s, rns.to_rns(s2, par.moduli), d.a, d.e, alpha)
    P = par.P
    for j in range(dnum):
        group = list(range(j * alpha, min((j + 1) * alpha, par.L + 1)))
        for t, m in enumerate(par.moduli):
            lhs = [(int(x) + y) % m for x, y in zip(swk[j, 0, t], negacyclic([int(v) for v in swk[j, 1, t]], s.tolist()))]
            w = 1 if t in group else 0     # gadget w_j = 1 on its group, 0 elsewhere (and P = 0 mod p_k)
            rhs = [(int(e) + w * P * int(v)) % m for e, v in zip(d.e[j], s2)]
            assert lhs == rhs, (j, t)


def test_encrypt_decrypt_exact():
    par = tiny_params()
    s = synth.ternary_secret(synth.stream(1, "s"), par.N, 8)
    m = np.arange(par.N, dtype=np.int64) * 1000 - 7000
    d = synth.encryption_draws(1, "enc", par.q, par.N)
    ct = ckks.encrypt(par, m, s, d.a, d.e, par.L, 1.0)
    got = ckks.decrypt_int(par, ct, s)
    assert got == [int(a) + int(b) for a, b in zip(m, d.e)]


def ks_setup(logn=5, nq=5, K=2, alpha=2, qbits=40, pbits=60):
    par = tiny_params(logn=logn, nq=nq, K=K, qbits=qbits, pbits=pbits)
    s = synth.ternary_secret(synth.stream(3, "s"), par.N, par.N // 2)
    return par, s, alpha


@pytest.mark.parametrize("alpha,level", [(1, 4), (2, 4), (2, 2), (3, 3)])
def test_keyswitch_decrypts_to_d_times_s_from(alpha, level):
    par, s, _ = ks_setup(alpha=alpha)
    dnum = ckks.dnum_for(par.L, alpha)
    sf = synth.ternary_secret(synth.stream(3, "sf"), par.N, par.N // 2)
    kd = synth.switch_key_draws(3, "k", dnum, par.moduli, par.N)
    swk = ckks.switch_key(par, s, rns.to_rns(sf, par.moduli), kd.a, kd.e, alpha)
    rnd = random.Random(level)
    mods = par.q[: level + 1]
    dpoly = rand_rns(rnd, mods, par.N)
    ks = ckks.keyswitch(par, dpoly, level, swk, alpha)
    Q = math.prod(mods)
    lhs = rns.crt(ks[0], mods)
    c1s = negacyclic(rns.crt(ks[1], mods), s.tolist())
    dval = rns.crt(dpoly, mods)
    want = negacyclic(dval, sf.tolist())
    err = rns.centered([(a + b - w) % Q for a, b, w in zip(lhs, c1s, want)], Q)
    # noise of hybrid keyswitch: (sum_j Q_j e_j)/P + rounding terms; tiny vs Q
    bound = (par.N * 8 * 4 * max(par.q) ** alpha) // par.P + par.N * (par.K + 2)
    assert max(abs(x) for x in err) <= bound, (max(abs(x) for x in err), bound)
    assert Q > (1 << 100) * max(1, bound)


def encode_ct(par, z, s, seed, level=None, scale=None):
    level = par.L if level is None else level
    scale = par.scale if scale is None else scale
    m = ckks.encode_int(par.N, z, scale)
    d = synth.encryption_draws(seed, "enc", par.q[: level + 1], par.N)
    return ckks.encrypt(par, m, s, d.a, d.e, level, scale)


def test_relinearised_product_decrypts_to_slot_product():
    par = tiny_params(logn=5, nq=4, K=2, qbits=40, pbits=60, scale=2.0 ** 30)
    alpha = 2
    s = synth.ternary_secret(synth.stream(4, "s"), par.N, 16)
    dnum = ckks.dnum_for(par.L, alpha)
    kd = synth.switch_key_draws(4, "rlk", dnum, par.moduli, par.N)
    rlk = ckks.relin_key(par, s, kd.a, kd.e, alpha)
    g = np.random.default_rng(4)
    z1, z2 = g.uniform(-1, 1, par.n_slots), g.uniform(-1, 1, par.n_slots)
    a, b = encode_ct(par, z1, s, 1), encode_ct(par, z2, s, 2)
    t = ckks.tensor(par, a, b)
    r = ckks.relinearize(par, t, rlk, alpha)
    # degree-2 decryption equals degree-1 decryption after relinearisation, up to KS noise
    d3 = np.array(ckks.decrypt_int(par, t, s), dtype=object)
    d2 = np.array(ckks.decrypt_int(par, r, s), dtype=object)
    assert max(abs(int(x)) for x in d3 - d2) < 2 ** 20
    rs = ckks.rescale(par, r)
    got = ckks.decrypt_slots(par, rs, s).real
    assert np.max(np.abs(got - z1 * z2)) < 1e-4
    # slot addition (Appendix A.1.2)
    got = ckks.decrypt_slots(par, ckks.add(par, a, b), s).real
    assert np.max(np.abs(got - (z1 + z2))) < 1e-6


@pytest.mark.parametrize("k", [1, 3, 7])
def test_rotation_rotates_slots_left(k):
    par = tiny_params(logn=5, nq=3, K=2, qbits=40, pbits=60, scale=2.0 ** 30)
    alpha = 1
    s = synth.ternary_secret(synth.stream(5, "s"), par.N, 16)
    g = ckks.galois_for_rotation(par.N, k)
    dnum = ckks.dnum_for(par.L, alpha)
    kd = synth.switch_key_draws(5, f"rot{g}", dnum, par.moduli, par.N)
    rk = ckks.rotation_key(par, g, s, kd.a, kd.e, alpha)
    z = np.random.default_rng(k).uniform(-1, 1, par.n_slots)
    ct = encode_ct(par, z, s, 9)
    got = ckks.decrypt_slots(par, ckks.rotate(par, ct, g, rk, alpha), s).real
    assert np.max(np.abs(got - np.roll(z, -k))) < 1e-6
