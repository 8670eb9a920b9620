"""Pins for the PFE scoring oracle (Section 5.4.1): the monomial product
against the schoolbook negacyclic product and against the oracle's NTT-based
ring product; the constant-coefficient property of the function encoding,
exhaustively; and the decrypted score of an encrypted query against the sum
of the function values."""
import numpy as np
import pytest

import synth
from oracle import ckks, pfe, query, rns


def schoolbook_negacyclic(a, b, q):
    n = len(a)
    out = [0] * n
    for i in range(n):
        for j in range(n):
            if i + j < n:
                out[i + j] += a[i] * b[j]
            else:
                out[i + j - n] -= a[i] * b[j]
    return [x % q for x in out]


@pytest.mark.parametrize("k", [0, 1, 5, 7, 8, 9, 13, 15])
def test_monomial_matches_schoolbook(k):
    q = rns.gen_primes(40, 1)[0]
    g = np.random.default_rng(k)
    a = g.integers(0, q, 8, dtype=np.uint64)
    mono = [0] * 8
    mono[k % 8] = 1 if k < 8 else q - 1     # X^k = -X^(k-8) for 8 <= k < 16
    want = schoolbook_negacyclic([int(x) for x in a], mono, q)
    assert pfe.monomial_mul(a, k, q).tolist() == want


@pytest.mark.parametrize("k", [0, 1, 2047, 4095, 4096, 4097, 8191, 12345])
def test_monomial_matches_ring_product(k):
    """N = 2^12: the rotation equals the oracle's NTT-based product with X^k."""
    par = ckks.Params(12, rns.gen_primes(55, 1), rns.gen_primes(54, 1), 2.0 ** 40)
    q = par.q[0]
    g = np.random.default_rng(k)
    a = g.integers(0, q, par.N, dtype=np.uint64)
    mono = np.zeros(par.N, dtype=np.int64)
    kk = k % (2 * par.N)
    mono[kk % par.N] = 1 if kk < par.N else -1
    want = ckks.rns_mul(a[None], rns.to_rns(mono, [q]), [q], par.psi[:1])[0]
    assert np.array_equal(pfe.monomial_mul(a, k, q), want)


def test_encoding_puts_each_value_in_the_constant_coefficient():
    """X^k u_f has v[k] as its constant coefficient for every k < N (N = 64)."""
    q = rns.gen_primes(40, 1)[0]
    n = 64
    v = np.random.default_rng(3).integers(-1000, 1000, n)
    u = pfe.function_poly(v.astype(np.float64)).astype(np.int64)
    u_res = np.array([x % q for x in u.tolist()], dtype=np.uint64)
    for k in range(n):
        c0 = int(pfe.monomial_mul(u_res, k, q)[0])
        assert (c0 - int(v[k])) % q == 0, k


def test_exponent_discretisation():
    n = 4096
    x = np.array([0.0, 0.5, 1.0 - 1e-9, 1.0, 0.25])
    e = pfe.exponent(x, 0.0, 1.0, n)
    assert e.tolist() == [0, 2048, 4095, 4095, 1024]


def test_decrypted_scores_are_function_sums():
    """Set I shape (N = 2^12, one 55-bit modulus): Enc(u_{f_j}) for 4
    functions, 33 records; the decrypted constant coefficient of ct_i divided by
    Delta is sum_j f_j(x_ij) up to the encryption noise."""
    par = ckks.Params(12, rns.gen_primes(55, 1), rns.gen_primes(54, 1), 2.0 ** 30)
    n, q = par.N, par.q[0]
    s = query.secret(par, 4, 2 * n // 3)
    g = np.random.default_rng(11)
    m, p = 4, 33
    grid = np.arange(n) / n
    tables = [np.sin(2 * np.pi * (j + 1) * grid) for j in range(m)]    # f_j on the discretised domain
    U = []
    for j in range(m):
        coeffs = np.floor(pfe.function_poly(tables[j]) * par.scale + 0.5).astype(np.int64)
        d = synth.encryption_draws(5, f"u{j}", par.q[:1], n)
        U.append(ckks.encrypt(par, coeffs, s, d.a, d.e, 0, par.scale).data[:, 0])   # [2][N]
    U = np.stack(U)
    x = g.uniform(0.0, 1.0, size=(p, m))
    exps = pfe.exponent(x, 0.0, 1.0, n)
    out = pfe.scores(U, exps, q)
    for i in range(p):
        c0 = ckks.decrypt_int(par, ckks.Ct(out[i][:, None, :], 0, par.scale), s)[0]
        want = sum(tables[j][exps[i, j]] for j in range(m))
        assert abs(c0 / par.scale - want) < 1e-5, i


def repack_params(log_n=6):
    q = rns.gen_primes(50, 1) + rns.gen_primes(40, 1)
    return ckks.Params(log_n, q, rns.gen_primes(60, 1), 2.0 ** 30)


def test_repack_galois_elements():
    assert pfe.repack_galois(16) == [31, 5, 25, 17]
    assert pfe.repack_galois(4096)[0] == 8191 and len(pfe.repack_galois(4096)) == 12


@pytest.mark.parametrize("count", [64, 37, 1])
def test_repack_trivial_ciphertexts_exact(count):
    """With c1 = 0 every key switch sees a zero polynomial and returns zero,
    so Algorithm 1 acts on the plaintexts alone: the result is exactly
    sum_i m_i[0] X^i (mod Q) -- the N^-1 premultiplication cancels the log N
    doublings and every other coefficient cancels (Lemma 1)."""
    par = repack_params()
    s = query.secret(par, 2, 2 * par.N // 3)
    keys = query.make_keys(par, s, 2, 1, pfe.repack_galois(par.N))
    g = np.random.default_rng(count)
    mods = par.q[: par.L + 1]
    msgs = [g.integers(-(1 << 20), 1 << 20, par.N) for _ in range(count)]
    cts = [ckks.Ct(np.stack([rns.to_rns(m, mods), np.zeros((par.L + 1, par.N), dtype=np.uint64)]), par.L, 1.0)
           for m in msgs]
    out = pfe.repack(par, cts, keys.rot, 1)
    want = np.zeros(par.N, dtype=np.int64)
    want[:count] = [int(m[0]) for m in msgs]
    assert np.array_equal(out.data[0], rns.to_rns(want, mods))
    assert not out.data[1].any()


def test_repack_decrypts_to_constant_coefficients():
    """Real encryptions: the repacked ciphertext decrypts to sum_i m_i[0] X^i up
    to the key-switching noise (N e_ks after log N rounds, far below Delta)."""
    par = repack_params()
    s = query.secret(par, 3, 2 * par.N // 3)
    keys = query.make_keys(par, s, 3, 1, pfe.repack_galois(par.N))
    g = np.random.default_rng(9)
    vals = g.uniform(-1, 1, par.N)
    cts = []
    for i in range(par.N):
        m = np.round(g.uniform(-1, 1, par.N) * par.scale).astype(np.int64)
        m[0] = int(round(vals[i] * par.scale))
        d = synth.encryption_draws(3, f"r{i}", par.q, par.N)
        cts.append(ckks.encrypt(par, m, s, d.a, d.e, par.L, par.scale))
    out = pfe.repack(par, cts, keys.rot, 1)
    dec = np.array(ckks.decrypt_int(par, out, s), dtype=np.float64) / par.scale
    assert np.max(np.abs(dec - vals)) < 2.0 ** -12
