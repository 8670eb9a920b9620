"""Pins for the oracle's canonical-embedding encoder (Appendix A.1.2):
the FFT route equals the O(N^2) defining sum, decode inverts encode, a
constant vector is the constant polynomial, and slot-wise addition,
multiplication (negacyclic product, schoolbook) and rotation (X -> X^(5^k))
hold on plaintexts."""
import numpy as np
import pytest

from oracle import ckks


@pytest.mark.parametrize("logn", [3, 6, 8])
def test_encode_fft_equals_definition(logn):
    N = 1 << logn
    z = np.random.default_rng(logn).uniform(-1, 1, N // 2) + 1j * np.random.default_rng(logn + 1).uniform(-1, 1, N // 2)
    assert np.allclose(ckks.encode_real(N, z, 1.0), ckks.encode_direct(N, z), atol=1e-12)
    m = np.random.default_rng(logn + 2).uniform(-1, 1, N)
    assert np.allclose(ckks.decode(N, m), ckks.decode_direct(N, m), atol=1e-10)


def test_decode_inverts_encode():
    N = 1 << 12
    z = np.random.default_rng(0).uniform(-1, 1, N // 2)
    assert np.max(np.abs(ckks.decode(N, ckks.encode_real(N, z, 1.0)) - z)) < 1e-12
    # through integer rounding at scale 2^40: error <= N * 2^-41 per slot
    m = ckks.encode_int(N, z, 2.0 ** 40).astype(np.float64) / 2.0 ** 40
    assert np.max(np.abs(ckks.decode(N, m) - z)) < N * 2.0 ** -41


def test_constant_vector_is_constant_polynomial():
    N = 1 << 8
    m = ckks.encode_real(N, np.full(N // 2, 0.37), 1.0)
    assert abs(m[0] - 0.37) < 1e-14 and np.max(np.abs(m[1:])) < 1e-14


def negacyclic_float(a, b):
    N = len(a)
    full = np.convolve(a, b)
    out = full[:N].copy()
    out[: N - 1] -= full[N:]
    return out


def test_slot_arithmetic_identities():
    N = 64
    g = np.random.default_rng(3)
    z1, z2 = g.uniform(-1, 1, N // 2), g.uniform(-1, 1, N // 2)
    m1, m2 = ckks.encode_real(N, z1, 1.0), ckks.encode_real(N, z2, 1.0)
    assert np.allclose(ckks.decode(N, m1 + m2).real, z1 + z2, atol=1e-12)
    assert np.allclose(ckks.decode(N, negacyclic_float(m1, m2)).real, z1 * z2, atol=1e-12)


@pytest.mark.parametrize("k", [1, 2, 5, 31])
def test_rotation_on_plaintext(k):
    N = 128
    z = np.random.default_rng(k).uniform(-1, 1, N // 2)
    m = ckks.encode_real(N, z, 1.0)
    gal = ckks.galois_for_rotation(N, k)
    out = np.zeros(N)
    for i, v in enumerate(m):
        j = i * gal % (2 * N)
        if j < N:
            out[j] += v
        else:
            out[j - N] -= v
    assert np.allclose(ckks.decode(N, out).real, np.roll(z, -k), atol=1e-12)
