"""Pins for the oracle's InnerSum (the rotate-and-sum count of Algorithm 2):
the rotations by 2^k, k < log2(n), reach every slot offset exactly once, and
the decrypted result holds the sum of all slots in every slot."""
import numpy as np

import synth
from oracle import ckks, query, rns


def test_rotations_cover_every_offset_once():
    for log_n in (5, 8, 12, 16):
        par = ckks.Params(log_n, rns.gen_primes(50, 2), rns.gen_primes(60, 1), 2.0 ** 40)
        gal = query.innersum_galois(par)
        # acc + rot_{2^k}(acc) doubles the set of offsets summed: all of [0, n) once
        offsets = [0]
        for k in range(len(gal)):
            offsets = offsets + [o + (1 << k) for o in offsets]
        assert sorted(offsets) == list(range(par.n_slots))
        assert gal == [ckks.galois_for_rotation(par.N, 1 << k) for k in range(log_n - 1)]


def test_innersum_decrypts_to_total_in_every_slot():
    q = rns.gen_primes(50, 1) + rns.gen_primes(40, 2)
    par = ckks.Params(8, q, rns.gen_primes(60, 1), 2.0 ** 40)
    s = query.secret(par, 4, 2 * par.N // 3)
    keys = query.make_keys(par, s, 4, 1, query.innersum_galois(par))
    z = np.random.default_rng(4).uniform(-1, 1, par.n_slots) / par.n_slots
    m = ckks.encode_int(par.N, z, par.scale)
    d = synth.encryption_draws(4, "x", par.q[:2], par.N)
    ct = ckks.encrypt(par, m, s, d.a, d.e, 1, par.scale)
    plan = query.Plan(S=[par.scale] * (par.L + 1), l_lin=1, l_d=1, l_y=1, l_u=1, l_out=1, pt_scale=1.0,
                      mask_scale=0.0, ragged=False)
    got = ckks.decrypt_slots(par, query.Evaluator(par, keys, plan).innersum(ct), s).real
    assert np.max(np.abs(got - z.sum())) < 1e-7
