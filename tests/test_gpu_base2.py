"""GPU parity of the base-2^w key-switch decomposition (Table 1, `base2`):
with the context option set, generated keys equal the oracle's
`switch_key_base2` and every key-switching primitive (key switch,
relinearisation, rotation, fused relinearisation + rescale) equals the
oracle's `keyswitch_base2` composition bit for bit."""
import numpy as np
import pytest

import synth
from oracle import ckks, query, rns

pytestmark = pytest.mark.gpu

T = pytest.importorskip("paper_2412_13269_gb300")


def rand_ct(par, comps, level, seed):
    g = np.random.default_rng(seed)
    return np.stack([np.stack([g.integers(0, q, par.N, dtype=np.uint64) for q in par.q[: level + 1]]) for _ in range(comps)])


def relin_b2(par, t3, l, key, w):
    ks = ckks.keyswitch_base2(par, t3[2], l, key, w)
    mods = par.q[: l + 1]
    return np.stack([ckks.rns_add(t3[0], ks[0], mods), ckks.rns_add(t3[1], ks[1], mods)])


def rotate_b2(par, a, l, g, key, w):
    t = ckks.automorphism(par, ckks.Ct(a, l, 1.0), g)
    ks = ckks.keyswitch_base2(par, t.data[1], l, key, w)
    return np.stack([ckks.rns_add(t.data[0], ks[0], par.q[: l + 1]), ks[1]])


CASES = {
    # (log N, ciphertext primes, special primes, w): B = ceil(max bits / w) pieces per prime
    "n12_w20": (12, lambda: rns.gen_primes(50, 1) + rns.gen_primes(40, 3), lambda: rns.gen_primes(60, 1), 20),
    "n12_w16_k2": (12, lambda: rns.gen_primes(50, 8), lambda: rns.gen_primes(55, 2), 16),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_base2_keys_and_key_switching(name):
    T.build()
    log_n, qf, pf, w = CASES[name]
    q, p = qf(), pf()
    par = ckks.Params(log_n, q, p, 2.0 ** 40)
    ctx = T.Ctx(log_n, q, p, 2.0 ** 40)
    ctx.set_option(T.OPT_KS_BASE2, w)
    assert ctx.get_option(T.OPT_KS_BASE2) == w
    B = ckks.base2_pieces(par, w)
    nd = (par.L + 1) * B
    assert B >= 2 and nd <= 64
    s = query.secret(par, 3, 2 * par.N // 3)
    s_rns = rns.to_rns(s, par.moduli)
    s2 = ckks.rns_mul(s_rns, s_rns, par.moduli, par.psi)
    d = synth.switch_key_draws(31, "relin", nd, par.moduli, par.N)
    ctx.keygen_relin(s, d.a, d.e, 1)
    rlk = ckks.switch_key_base2(par, s, s2, d.a, d.e, w)
    assert np.array_equal(ctx.get_key(0, nd), rlk)
    g = ckks.galois_for_rotation(par.N, 1)
    dr = synth.switch_key_draws(31, f"rot{g}", nd, par.moduli, par.N)
    ctx.keygen_rotation(g, s, dr.a, dr.e, 1)
    sg = ckks.automorphism_poly(s_rns, g, par.moduli)
    rotk = ckks.switch_key_base2(par, s, sg, dr.a, dr.e, w)
    assert np.array_equal(ctx.get_key(g, nd), rotk)
    for l in sorted({par.L, max(1, par.L - 2), 0}):
        dd = rand_ct(par, 1, l, 30 + l)
        got = ctx.op(T.OP_KEYSWITCH, dd, l, arg=0, out_comps=2)[0]
        assert np.array_equal(got, ckks.keyswitch_base2(par, dd[0], l, rlk, w)), l
        t3 = rand_ct(par, 3, l, 40 + l)
        got = ctx.op(T.OP_RELIN, t3, l, out_comps=2)[0]
        assert np.array_equal(got, relin_b2(par, t3, l, rlk, w)), l
        a = rand_ct(par, 2, l, 50 + l)
        got = ctx.op(T.OP_ROTATE, a, l, arg=g, out_comps=2)[0]
        assert np.array_equal(got, rotate_b2(par, a, l, g, rotk, w)), l
        if l >= 1:
            got, lev, _ = ctx.op(T.OP_RELIN_RESCALE, t3, l, out_comps=2)
            want = ckks.rescale(par, ckks.Ct(relin_b2(par, t3, l, rlk, w), l, 1.0))
            assert lev == l - 1 and np.array_equal(got, want.data), l
    ctx.close()


def test_base2_option_rules():
    """Bad widths are refused, a changed width drops the loaded keys, and the
    decomposition takes one-prime digits only."""
    T.build()
    q, p = rns.gen_primes(50, 1) + rns.gen_primes(40, 3), rns.gen_primes(60, 1)
    par = ckks.Params(12, q, p, 2.0 ** 40)
    ctx = T.Ctx(12, q, p, 2.0 ** 40)
    for bad in (1, 7, 63, 64):
        with pytest.raises(T.TetrisError):
            ctx.set_option(T.OPT_KS_BASE2, bad)
    s = query.secret(par, 5, 2 * par.N // 3)
    ctx.set_option(T.OPT_KS_BASE2, 25)
    nd = (par.L + 1) * ckks.base2_pieces(par, 25)
    d = synth.switch_key_draws(5, "relin", nd, par.moduli, par.N)
    ctx.keygen_relin(s, d.a, d.e, 1)
    t3 = rand_ct(par, 3, par.L, 7)
    ctx.op(T.OP_RELIN, t3, par.L, out_comps=2)
    ctx.set_option(T.OPT_KS_BASE2, 20)       # a new width: the relinearisation key is gone
    with pytest.raises(T.TetrisError):
        ctx.op(T.OP_RELIN, t3, par.L, out_comps=2)
    with pytest.raises(T.TetrisError):       # two-prime digits cannot be split into pieces
        d2 = synth.switch_key_draws(5, "relin", 2 * ckks.base2_pieces(par, 20), par.moduli, par.N)
        ctx.keygen_relin(s, d2.a, d2.e, 2)
    ctx.set_option(T.OPT_KS_BASE2, 0)        # back to the plain hybrid switch
    dh = synth.switch_key_draws(5, "relin", par.L + 1, par.moduli, par.N)
    ctx.keygen_relin(s, dh.a, dh.e, 1)
    got = ctx.op(T.OP_RELIN, t3, par.L, out_comps=2)[0]
    rlk = ckks.relin_key(par, s, dh.a, dh.e, 1)
    assert np.array_equal(got, ckks.relinearize(par, ckks.Ct(t3, par.L, 1.0), rlk, 1).data)
    ctx.close()
