"""Oracle for the private-function-evaluation scoring step (Section 5.4.1;
Algorithm 2, the loop building ct_i).

TEST INFRASTRUCTURE (see oracle/__init__.py).

The scientist encrypts, per attribute j, the polynomial u_{f_j} of a scoring
function f_j: the value table v_j[k] = f_j(g^-1(k/N)) placed so that
X^k * u_{f_j} has v_j[k] as its constant coefficient (u[0] = v[0],
u[i] = -v[N - i] for i >= 1; Section 5.4.1, with Section 4.3's large-domain
function method).  For each record i the server multiplies each U_j by the
monomial X^{e_ij}, e_ij the record's discretised attribute value, and sums:
    ct_i = sum_j U_j * X^{e_ij}    in (Z_q[X] / (X^N + 1))^2.
A product with a monomial is a negacyclic rotation of the coefficients, which
is what this file writes out (numpy, exact residues below 2^62).
"""
from __future__ import annotations

import numpy as np


def monomial_mul(a: np.ndarray, k: int, q: int) -> np.ndarray:
    """X^k * a in Z_q[X]/(X^N + 1) for any integer k (X^N = -1, X^2N = 1)."""
    a = np.asarray(a, dtype=np.uint64)
    n = a.size
    k %= 2 * n
    neg = k >= n
    if neg:
        k -= n
    out = np.empty_like(a)
    # coefficient i of X^k a is a[i - k] for i >= k, and -a[i - k + N] below k
    out[k:] = a[: n - k]
    wrapped = a[n - k:]
    out[:k] = np.where(wrapped == 0, np.uint64(0), np.uint64(q) - wrapped)
    if neg:
        out = np.where(out == 0, np.uint64(0), np.uint64(q) - out)
    return out


def scores(u: np.ndarray, exps: np.ndarray, q: int) -> np.ndarray:
    """u: uint64 [m][2][N] ciphertexts (one modulus q); exps: [p][m] exponents.
    Returns uint64 [p][2][N] with out[i] = sum_j X^{exps[i][j]} u[j] mod q."""
    u = np.asarray(u, dtype=np.uint64)
    exps = np.asarray(exps)
    m, comps, n = u.shape
    p = exps.shape[0]
    out = np.zeros((p, comps, n), dtype=np.uint64)
    qq = np.uint64(q)
    for i in range(p):
        for j in range(m):
            for c in range(comps):
                out[i, c] = (out[i, c] + monomial_mul(u[j, c], int(exps[i, j]), q)) % qq
    return out


def function_poly(values: np.ndarray) -> np.ndarray:
    """Coefficients (real) of u_f for the value table v[k] = f(g^-1(k/N)),
    k < N: u[0] = v[0], u[i] = -v[N - i]; then X^k u has v[k] in coefficient 0."""
    v = np.asarray(values, dtype=np.float64)
    u = np.empty_like(v)
    u[0] = v[0]
    u[1:] = -v[:0:-1]
    return u


def exponent(x, a: float, b: float, n: int) -> np.ndarray:
    """The record's value in the exponent: round(N g(x)), g(x) = ((2x - b - a)/(b - a) + 1)/2,
    kept below N (g(b) = 1 would wrap to X^N = -1)."""
    g = 0.5 * ((2.0 * np.asarray(x, dtype=np.float64) - b - a) / (b - a) + 1.0)
    return np.minimum(np.floor(n * g + 0.5).astype(np.int64), n - 1)


# ---------------------------------------------------------------------------
# Ring repacking (Algorithm 1, after Chen-Dai-Kim-Song): n <= N ciphertexts
# whose messages carry x_i in their constant coefficient become one ciphertext
# of sum_i x_i X^i.  All inputs are first multiplied by N^-1 mod Q (the log N
# rounds double the coefficients they keep).  Round r (r = 0 .. log N - 1)
# pairs c_j with c_{j+t}, t = N / 2^(r+1), and replaces c_j by
#     (c_j + X^t c_{j+t}) + phi_g(c_j - X^t c_{j+t}),
# phi_g the automorphism X -> X^g followed by its key switch, g = 2N - 1 in the
# first round and 5^(2^(r-1)) mod 2N after it.  Missing inputs are zero.
# ---------------------------------------------------------------------------
def repack_galois(n: int) -> list:
    """The Galois elements the rounds use, in round order."""
    logn = n.bit_length() - 1
    return [2 * n - 1] + [pow(5, 1 << (r - 1), 2 * n) for r in range(1, logn)]


def ct_monomial_mul(ct, t: int, moduli):
    """X^t times every component, limb by limb (a negacyclic rotation)."""
    from .ckks import Ct
    data = np.stack([np.stack([monomial_mul(ct.data[c, i], t, int(moduli[i])) for i in range(ct.level + 1)])
                     for c in range(ct.comps)])
    return Ct(data, ct.level, ct.scale)


def repack(par, cts: list, rot_keys: dict, alpha: int):
    """Algorithm 1 on ciphertexts at one level (coefficient domain)."""
    from . import ckks
    n = par.N
    if not 1 <= len(cts) <= n:
        raise ValueError("repack takes 1 to N ciphertexts")
    level = cts[0].level
    mods = par.q[: level + 1]
    ninv = pow(n, -1, int(np.prod([int(m) for m in mods], dtype=object)))
    zero = ckks.Ct(np.zeros_like(cts[0].data), level, cts[0].scale)
    c = [ckks.mul_int(par, x, ninv) for x in cts] + [zero] * (n - len(cts))
    for r, g in enumerate(repack_galois(n)):
        t = n >> (r + 1)
        for j in range(t):
            s = ct_monomial_mul(c[j + t], t, mods)
            c[j] = ckks.add(par, ckks.add(par, c[j], s),
                            ckks.rotate(par, ckks.sub(par, c[j], s), g, rot_keys[g], alpha))
    return c[0]
