"""Pins for the base-2^w key-switch decomposition (Table 1, `base2`): with one
piece per digit it is the one-prime-digit hybrid key switch, bit for bit; the
generated keys satisfy the SwitchKeyGen identity exactly; decrypting a key
switch gives d * s_from plus noise well below the undecomposed switch's."""
import numpy as np
import pytest

import synth
from oracle import ckks, query, rns


def params(log_n=8):
    q = rns.gen_primes(50, 1) + rns.gen_primes(40, 2)
    return ckks.Params(log_n, q, rns.gen_primes(45, 1), 2.0 ** 30)


def draws(par, nd, seed):
    g = np.random.default_rng(seed)
    a = np.stack([np.stack([g.integers(0, m, par.N, dtype=np.uint64) for m in par.moduli]) for _ in range(nd)])
    e = np.rint(g.normal(0, 3.2, (nd, par.N))).astype(np.int64)
    return a, e


def test_one_piece_is_the_hybrid_key_switch():
    par = params()
    s = query.secret(par, 1, 2 * par.N // 3)
    s2 = ckks.rns_mul(rns.to_rns(s, par.moduli), rns.to_rns(s, par.moduli), par.moduli, par.psi)
    w = 60                                   # every prime fits one piece
    assert ckks.base2_pieces(par, w) == 1
    a, e = draws(par, par.L + 1, 2)
    k2 = ckks.switch_key_base2(par, s, s2, a, e, w)
    k1 = ckks.switch_key(par, s, s2, a, e, 1)
    assert np.array_equal(k2, k1)
    d = rns.to_rns(np.random.default_rng(3).integers(-2**60, 2**60, par.N, dtype=np.int64), par.q)
    for level in (par.L, 1):
        assert np.array_equal(ckks.keyswitch_base2(par, d, level, k2, w), ckks.keyswitch(par, d, level, k1, 1))


def test_switch_key_generation_identity():
    """b_(i,b) + a_(i,b) s = e_(i,b) + P 2^(w b) s_from on limb i, e_(i,b) elsewhere (exact)."""
    par = params()
    w = 16
    B = ckks.base2_pieces(par, w)
    assert B == 4
    s = query.secret(par, 4, 2 * par.N // 3)
    s_from = rns.to_rns(query.secret(par, 5, 2 * par.N // 3), par.moduli)
    a, e = draws(par, (par.L + 1) * B, 6)
    k = ckks.switch_key_base2(par, s, s_from, a, e, w)
    s_rns = rns.to_rns(s, par.moduli)
    for i in range(par.L + 1):
        for b in range(B):
            j = i * B + b
            lhs = ckks.rns_add(k[j, 0], ckks.rns_mul(k[j, 1], s_rns, par.moduli, par.psi), par.moduli)
            want = rns.to_rns(e[j], par.moduli)
            qi = int(par.moduli[i])
            want[i] = (want[i].astype(object) + s_from[i].astype(object) * ((par.P << (w * b)) % qi)) % qi
            assert np.array_equal(lhs, want.astype(np.uint64)), (i, b)


def test_decomposition_reduces_key_switch_noise():
    par = params()
    s = query.secret(par, 7, 2 * par.N // 3)
    s_rns = rns.to_rns(s, par.moduli)
    s_from = rns.to_rns(query.secret(par, 8, 2 * par.N // 3), par.moduli)
    level = par.L
    mods = par.q[: level + 1]
    d = rns.to_rns(np.random.default_rng(9).integers(-2**62, 2**62, par.N, dtype=np.int64), mods)
    want = ckks.rns_mul(d, s_from[: level + 1], mods, par.psi[: level + 1])

    def noise(ks):
        c = ckks.Ct(ks, level, 1.0)
        got = ckks.rns_add(ks[0], ckks.rns_mul(ks[1], s_rns[: level + 1], mods, par.psi[: level + 1]), mods)
        diff = ckks.rns_sub(got, want, mods)
        vals = rns.centered(rns.crt(diff, mods), int(np.prod([int(m) for m in mods], dtype=object)))
        return max(abs(int(v)) for v in vals)

    a1, e1 = draws(par, par.L + 1, 10)
    plain = noise(ckks.keyswitch(par, d, level, ckks.switch_key(par, s, s_from, a1, e1, 1), 1))
    w = 10
    B = ckks.base2_pieces(par, w)
    a2, e2 = draws(par, (par.L + 1) * B, 11)
    dec = noise(ckks.keyswitch_base2(par, d, level, ckks.switch_key_base2(par, s, s_from, a2, e2, w), w))
    # the undecomposed switch leaves ~ N q_i sigma / P; with 10-bit pieces what is left is
    # mostly the rounding of ModDown
    assert 16 * dec < plain
