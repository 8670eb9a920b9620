"""Seeded synthetic inputs for the encrypted-query workloads.

This module draws every random number the workloads need and nothing else:
secret-key coefficients, error polynomials, the uniform "a" parts of
encryptions and switching keys, the plaintext database and the query's
cleartext values. It holds none of the RNS-CKKS arithmetic (no reduction of a
key, no ring product, no encoding); the two consumers of these draws, the CPU
oracle and the GPU library, each turn them into keys and ciphertexts on their
own. Both take the same draws, so their ciphertexts can be compared residue by
residue.

Distributions (Section 2.3 of the paper fixes their families; the sizes come
from the workload definitions):
  * secret s: ternary, exactly ``h`` non-zero coefficients in {-1, +1};
  * error e: rounded normal with standard deviation sigma (3.2 by default,
    the paper does not state one);
  * a: uniform residues in [0, q) for each modulus q;
  * database: u8 attribute values, either uniform on [0, 255] or the paper's
    synthetic feature distribution (normal, mean 1, sd 1, bounded to [0, 2),
    Section 5.4.1) quantised as floor(128 * x).
"""
from __future__ import annotations

import zlib
from dataclasses import dataclass

import numpy as np

SIGMA = 3.2


def stream(seed: int, name: str, *index: int) -> np.random.Generator:
    """Independent generator for (seed, purpose name, integer indices)."""
    key = [zlib.crc32(name.encode()) & 0xFFFFFFFF, *[int(i) & 0xFFFFFFFF for i in index]]
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(entropy=int(seed), spawn_key=key)))


def ternary_secret(g: np.random.Generator, n: int, h: int) -> np.ndarray:
    """int64[n] with exactly h entries in {-1,+1}, the rest 0."""
    if not 0 < h <= n:
        raise ValueError("hamming weight out of range")
    s = np.zeros(n, dtype=np.int64)
    pos = g.choice(n, size=h, replace=False)
    s[pos] = g.choice(np.array([-1, 1], dtype=np.int64), size=h)
    return s


def gaussian(g: np.random.Generator, shape, sigma: float = SIGMA) -> np.ndarray:
    """Rounded normal integers, int64."""
    return np.rint(g.normal(0.0, sigma, size=shape)).astype(np.int64)


def uniform_residues(g: np.random.Generator, moduli, n: int) -> np.ndarray:
    """uint64[len(moduli)][n], row i uniform in [0, moduli[i])."""
    out = np.empty((len(moduli), n), dtype=np.uint64)
    for i, q in enumerate(moduli):
        out[i] = g.integers(0, int(q), size=n, dtype=np.uint64, endpoint=False)
    return out


def database(g: np.random.Generator, records: int, attrs: int, dist: str = "uniform") -> np.ndarray:
    """u8[records][attrs]. ``dist``: "uniform", "paper" or "mixed" (first half
    of the columns uniform, second half the paper's distribution)."""
    if dist == "uniform":
        return g.integers(0, 256, size=(records, attrs), dtype=np.uint8)
    if dist == "paper":
        x = g.normal(1.0, 1.0, size=(records, attrs))
        x = np.clip(x, 0.0, np.nextafter(2.0, 0.0))
        return np.floor(128.0 * x).astype(np.uint8)
    if dist == "mixed":
        half = attrs // 2
        a = database(g, records, half, "uniform")
        b = database(g, records, attrs - half, "paper")
        return np.concatenate([a, b], axis=1)
    raise ValueError(dist)


@dataclass
class QueryValues:
    w: np.ndarray        # float64[attrs], linear-combination coefficients in [-1, 1]
    c: np.ndarray        # float64[degree+1], coefficients of f
    t: float             # threshold in [-0.5, 0.5]
    t1: float | None = None  # global threshold, a record count (None: no global threshold)


def query_values(g: np.random.Generator, attrs: int, degree: int) -> QueryValues:
    w = g.uniform(-1.0, 1.0, size=attrs)
    c = g.uniform(-1.0, 1.0, size=degree + 1) / (degree + 1)
    t = float(g.uniform(-0.5, 0.5))
    return QueryValues(w=w, c=c, t=t)


@dataclass
class KeyDraws:
    a: np.ndarray   # uint64[dnum][n_qp][N]
    e: np.ndarray   # int64[dnum][N]


def switch_key_draws(seed: int, name: str, dnum: int, moduli_qp, n: int, sigma: float = SIGMA) -> KeyDraws:
    ga = stream(seed, name + ".a")
    ge = stream(seed, name + ".e")
    a = np.stack([uniform_residues(ga, moduli_qp, n) for _ in range(dnum)])
    e = gaussian(ge, (dnum, n), sigma)
    return KeyDraws(a=a, e=e)


@dataclass
class EncDraws:
    a: np.ndarray   # uint64[level+1][N]
    e: np.ndarray   # int64[N]


def encryption_draws(seed: int, name: str, moduli, n: int, sigma: float = SIGMA) -> EncDraws:
    return EncDraws(a=uniform_residues(stream(seed, name + ".a"), moduli, n),
                    e=gaussian(stream(seed, name + ".e"), n, sigma))
