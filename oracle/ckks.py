"""RNS-CKKS oracle: encoding, key generation, encryption and the homomorphic
operations of the server path, all in the coefficient domain.

TEST INFRASTRUCTURE (see oracle/__init__.py).

Citations are to the TETRIS paper (arXiv 2412.13269): Section 2.2 (ring,
automorphisms), 2.3 (RLWE encryption), 2.4.1 (SwitchKeyGen / SwitchKey),
2.5 (CKKS scale and rescale), Appendix A.1.2 (canonical-embedding encoding,
slot arithmetic, rotation) and Appendix A.2 (relinearisation, automorphism).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import rns
from .rns import lib, ptr, u64arr


def round_half_up(x: float) -> int:
    """The rounding used wherever a real number becomes an integer: floor(x + 1/2)."""
    return int(math.floor(x + 0.5))


@dataclass
class Params:
    log_n: int
    q: list          # ciphertext primes q_0 .. q_L (q_0 is kept to the end)
    p: list          # special primes p_0 .. p_{K-1} (the modulus P of Section 2.4.1)
    scale: float     # Delta of fresh ciphertexts (Section 2.5)
    psi: list = field(default_factory=list)

    def __post_init__(self):
        self.q = [int(x) for x in self.q]
        self.p = [int(x) for x in self.p]
        if not self.psi:
            self.psi = [rns.primitive_2n_root(m, self.N) for m in self.q + self.p]

    @property
    def N(self) -> int:
        return 1 << self.log_n

    @property
    def n_slots(self) -> int:
        return self.N // 2

    @property
    def L(self) -> int:
        return len(self.q) - 1

    @property
    def K(self) -> int:
        return len(self.p)

    @property
    def moduli(self) -> list:
        return self.q + self.p

    def qmod(self, level: int) -> np.ndarray:
        return u64arr(self.q[: level + 1])

    def qpsi(self, level: int) -> np.ndarray:
        return u64arr(self.psi[: level + 1])

    @property
    def P(self) -> int:
        return math.prod(self.p)


@dataclass
class Ct:
    data: np.ndarray   # uint64[comps][level+1][N], coefficient domain
    level: int
    scale: float

    @property
    def comps(self) -> int:
        return self.data.shape[0]

    def copy(self) -> "Ct":
        return Ct(self.data.copy(), self.level, self.scale)


# ---------------------------------------------------------------------------
# Encoding (Appendix A.1.2): slot j of m is m(zeta^(5^j)), zeta = exp(i pi / N).
# For real slot values z, m_i = (2/N) Re(sum_j z_j zeta^(-i 5^j)).
# ---------------------------------------------------------------------------
def slot_exponents(N: int) -> np.ndarray:
    e = np.empty(N // 2, dtype=np.int64)
    x = 1
    for j in range(N // 2):
        e[j] = x
        x = x * 5 % (2 * N)
    return e


def encode_real(N: int, z, scale: float) -> np.ndarray:
    """Real coefficients m (before scaling) of the polynomial whose slots are z
    (zero padded to N/2), via a length-2N FFT used as a library primitive:
    sum_j z_j zeta^(-i e_j) = FFT_{2N}(v)[i] with v[e_j] = z_j."""
    z = np.asarray(z, dtype=np.complex128)
    v = np.zeros(2 * N, dtype=np.complex128)
    v[slot_exponents(N)[: z.shape[0]]] = z
    return (2.0 / N) * np.fft.fft(v)[:N].real


def encode_direct(N: int, z) -> np.ndarray:
    """The same map written as the O(N^2) sum (the definition)."""
    z = np.asarray(z, dtype=np.complex128)
    e = slot_exponents(N)[: z.shape[0]]
    i = np.arange(N)[:, None]
    zeta = np.exp(-1j * np.pi * ((i * e[None, :]) % (2 * N)) / N)
    return (2.0 / N) * (zeta @ z).real


def decode(N: int, m) -> np.ndarray:
    """Slots of a real polynomial m: z_j = sum_i m_i zeta^(i e_j) = 2N * IFFT_{2N}(m)[e_j]."""
    v = np.zeros(2 * N, dtype=np.complex128)
    v[:N] = np.asarray(m, dtype=np.float64)
    return (2 * N) * np.fft.ifft(v)[slot_exponents(N)]


def decode_direct(N: int, m) -> np.ndarray:
    e = slot_exponents(N)
    i = np.arange(N)[None, :]
    zeta = np.exp(1j * np.pi * ((e[:, None] * i) % (2 * N)) / N)
    return zeta @ np.asarray(m, dtype=np.complex128)


def encode_int(N: int, z, scale: float) -> np.ndarray:
    """round_half_up(scale * m_i) as int64 (the plaintext polynomial)."""
    m = encode_real(N, z, 1.0) * scale
    if np.max(np.abs(m)) >= 2.0 ** 62:
        raise ValueError("encoded coefficient too large")
    return np.floor(m + 0.5).astype(np.int64)


# ---------------------------------------------------------------------------
# Ring helpers over a list of moduli
# ---------------------------------------------------------------------------
def rns_mul(a: np.ndarray, b: np.ndarray, moduli, psis) -> np.ndarray:
    a = np.ascontiguousarray(a)
    b = np.ascontiguousarray(b)
    out = np.empty_like(a)
    lib().or_rns_polymul(ptr(a), ptr(b), ptr(out), a.shape[0], a.shape[1], ptr(u64arr(moduli)), ptr(u64arr(psis)))
    return out


def rns_add(a, b, moduli):
    m = u64arr(moduli)[:, None]
    s = a + b          # < 2^63, no wrap
    return np.where(s >= m, s - m, s)


def rns_sub(a, b, moduli):
    m = u64arr(moduli)[:, None]
    return np.where(a >= b, a - b, a + (m - b))


def rns_neg(a, moduli):
    m = u64arr(moduli)[:, None]
    return np.where(a == 0, a, m - a)


def int_residues(c: int, moduli) -> np.ndarray:
    return u64arr([int(c) % int(q) for q in moduli])


def rns_mul_int(a, c: int, moduli):
    a = np.ascontiguousarray(a)
    out = np.empty_like(a)
    lib().or_rns_mul_scalar(ptr(a), ptr(int_residues(c, moduli)), ptr(out), a.shape[0], a.shape[1], ptr(u64arr(moduli)))
    return out


def automorphism_poly(a: np.ndarray, g: int, moduli) -> np.ndarray:
    a = np.ascontiguousarray(a)
    out = np.empty_like(a)
    lib().or_rns_automorphism(ptr(a), ptr(out), a.shape[0], a.shape[1], ptr(u64arr(moduli)), g)
    return out


# ---------------------------------------------------------------------------
# Keys (Section 2.4.1): swk_j = (-a_j s + e_j + w_j P s_from, a_j) over Q_L P,
# w_j the CRT gadget of the prime group D_j: w_j = 1 mod the primes of D_j and
# 0 mod every other q; mod each special prime P w_j s_from vanishes.
# ---------------------------------------------------------------------------
def dnum_for(level: int, alpha: int) -> int:
    return -(-(level + 1) // alpha)


def switch_key(par: Params, s_to: np.ndarray, s_from_rns: np.ndarray, a: np.ndarray, e: np.ndarray, alpha: int) -> np.ndarray:
    """s_to: int64[N]; s_from_rns: uint64[L+1+K][N]; a: uint64[dnum][L+1+K][N];
    e: int64[dnum][N]. Returns uint64[dnum][2][L+1+K][N]."""
    mods = par.moduli
    nqp = len(mods)
    dnum = dnum_for(par.L, alpha)
    assert a.shape == (dnum, nqp, par.N) and e.shape == (dnum, par.N)
    s_rns = rns.to_rns(s_to, mods)
    Pmod = [par.P % q for q in mods]
    out = np.empty((dnum, 2, nqp, par.N), dtype=np.uint64)
    for j in range(dnum):
        as_ = rns_mul(a[j], s_rns, mods, par.psi)
        b = rns_sub(rns.to_rns(e[j], mods), as_, mods)
        for t in range(j * alpha, min((j + 1) * alpha, par.L + 1)):
            modt = int(mods[t])
            term = rns_mul_int(s_from_rns[t:t + 1], Pmod[t], [modt])
            b[t:t + 1] = rns_add(b[t:t + 1], term, [modt])
        out[j, 0] = b
        out[j, 1] = a[j]
    return out


def relin_key(par: Params, s: np.ndarray, a, e, alpha: int) -> np.ndarray:
    mods = par.moduli
    s_rns = rns.to_rns(s, mods)
    s2 = rns_mul(s_rns, s_rns, mods, par.psi)
    return switch_key(par, s, s2, a, e, alpha)


def rotation_key(par: Params, galois: int, s: np.ndarray, a, e, alpha: int) -> np.ndarray:
    mods = par.moduli
    sg = automorphism_poly(rns.to_rns(s, mods), galois, mods)
    return switch_key(par, s, sg, a, e, alpha)


def galois_for_rotation(N: int, k: int) -> int:
    """phi_(0,k): X -> X^(5^k mod 2N) rotates the slots left by k (Appendix A.1.2)."""
    return pow(5, k % (N // 2), 2 * N)


# ---------------------------------------------------------------------------
# Encryption / decryption (Section 2.3)
# ---------------------------------------------------------------------------
def encrypt(par: Params, m: np.ndarray, s: np.ndarray, a: np.ndarray, e: np.ndarray, level: int, scale: float) -> Ct:
    """(c0, c1) = (-a s + e + m, a) mod Q_level; m: int64 coefficients."""
    mods = par.q[: level + 1]
    psis = par.psi[: level + 1]
    a = np.ascontiguousarray(a[: level + 1])
    c0 = rns_sub(rns_add(rns.to_rns(e, mods), rns.to_rns(m, mods), mods), rns_mul(a, rns.to_rns(s, mods), mods, psis), mods)
    return Ct(np.stack([c0, a]), level, scale)


def decrypt_int(par: Params, ct: Ct, s: np.ndarray) -> list:
    """Centred integer coefficients of c0 + c1 s (+ c2 s^2) mod Q_level."""
    mods = par.q[: ct.level + 1]
    psis = par.psi[: ct.level + 1]
    s_rns = rns.to_rns(s, mods)
    acc = ct.data[0].copy()
    sp = s_rns
    for c in range(1, ct.comps):
        acc = rns_add(acc, rns_mul(ct.data[c], sp, mods, psis), mods)
        sp = rns_mul(sp, s_rns, mods, psis)
    Q = math.prod(mods)
    return rns.centered(rns.crt(acc, mods), Q)


def decrypt_slots(par: Params, ct: Ct, s: np.ndarray) -> np.ndarray:
    coeffs = decrypt_int(par, ct, s)
    m = np.array([float(c) / ct.scale for c in coeffs])
    return decode(par.N, m)


# ---------------------------------------------------------------------------
# Homomorphic operations
# ---------------------------------------------------------------------------
def add(par, a: Ct, b: Ct) -> Ct:
    assert a.level == b.level and a.comps == b.comps
    mods = par.q[: a.level + 1]
    return Ct(np.stack([rns_add(a.data[c], b.data[c], mods) for c in range(a.comps)]), a.level, a.scale)


def sub(par, a: Ct, b: Ct) -> Ct:
    assert a.level == b.level and a.comps == b.comps
    mods = par.q[: a.level + 1]
    return Ct(np.stack([rns_sub(a.data[c], b.data[c], mods) for c in range(a.comps)]), a.level, a.scale)


def add_int_const(par, a: Ct, c: int) -> Ct:
    """Add the constant polynomial c to the message (c0 coefficient 0)."""
    out = a.copy()
    mods = par.q[: a.level + 1]
    for i, q in enumerate(mods):
        out.data[0, i, 0] = np.uint64((int(out.data[0, i, 0]) + c) % q)
    return out


def mul_int(par, a: Ct, c: int) -> Ct:
    mods = par.q[: a.level + 1]
    return Ct(np.stack([rns_mul_int(a.data[k], c, mods) for k in range(a.comps)]), a.level, a.scale)


def mul_plain(par, a: Ct, pt_rns: np.ndarray, pt_scale: float) -> Ct:
    """Plaintext-ciphertext product; pt_rns uint64[>=level+1][N]."""
    mods = par.q[: a.level + 1]
    psis = par.psi[: a.level + 1]
    pt = np.ascontiguousarray(pt_rns[: a.level + 1])
    return Ct(np.stack([rns_mul(a.data[k], pt, mods, psis) for k in range(a.comps)]), a.level, a.scale * pt_scale)


def tensor(par, a: Ct, b: Ct) -> Ct:
    """(a0 b0, a0 b1 + a1 b0, a1 b1): the product of two RLWE ciphertexts,
    a degree-2 ciphertext under (1, s, s^2) (Appendix A.2)."""
    assert a.level == b.level and a.comps == 2 and b.comps == 2
    mods = par.q[: a.level + 1]
    psis = par.psi[: a.level + 1]
    d0 = rns_mul(a.data[0], b.data[0], mods, psis)
    d1 = rns_add(rns_mul(a.data[0], b.data[1], mods, psis), rns_mul(a.data[1], b.data[0], mods, psis), mods)
    d2 = rns_mul(a.data[1], b.data[1], mods, psis)
    return Ct(np.stack([d0, d1, d2]), a.level, a.scale * b.scale)


def keyswitch(par: Params, d: np.ndarray, level: int, evk: np.ndarray, alpha: int) -> np.ndarray:
    """SwitchKey(d, swk) (Section 2.4.1) at the given level -> uint64[2][level+1][N]."""
    d = np.ascontiguousarray(d[: level + 1])
    out = np.empty((2, level + 1, par.N), dtype=np.uint64)
    evk = np.ascontiguousarray(evk)
    lib().or_keyswitch(ptr(d), level, ptr(evk), evk.shape[0], par.L + 1, par.K, alpha,
                       ptr(u64arr(par.moduli)), ptr(u64arr(par.psi)), par.N, ptr(out))
    return out


def relinearize(par, ct: Ct, rlk: np.ndarray, alpha: int, base2: int = 0) -> Ct:
    """SwitchKey(ct[2], swk_{s^2 -> s}) + ct[0:1] (Appendix A.2); base2 = w > 0
    switches with the base-2^w gadget of Table 1 (keys from switch_key_base2)."""
    assert ct.comps == 3
    ks = (keyswitch_base2(par, ct.data[2], ct.level, rlk, base2) if base2
          else keyswitch(par, ct.data[2], ct.level, rlk, alpha))
    mods = par.q[: ct.level + 1]
    return Ct(np.stack([rns_add(ct.data[0], ks[0], mods), rns_add(ct.data[1], ks[1], mods)]), ct.level, ct.scale)


def rescale(par, ct: Ct) -> Ct:
    """Divide by q_level with rounding and drop that prime (Section 2.5)."""
    l = ct.level
    assert l >= 1
    a = np.ascontiguousarray(ct.data)
    out = np.empty((ct.comps, l, par.N), dtype=np.uint64)
    lib().or_rescale(ptr(a), ptr(out), ct.comps, l, par.N, ptr(u64arr(par.q[: l + 1])))
    return Ct(out, l - 1, ct.scale / par.q[l])


def drop_to(ct: Ct, level: int) -> Ct:
    """Keep the residues modulo q_0..q_level (a modulus switch without scaling)."""
    assert level <= ct.level
    return Ct(np.ascontiguousarray(ct.data[:, : level + 1]), level, ct.scale)


def automorphism(par, ct: Ct, g: int) -> Ct:
    mods = par.q[: ct.level + 1]
    return Ct(np.stack([automorphism_poly(ct.data[c], g, mods) for c in range(ct.comps)]), ct.level, ct.scale)


def rotate(par, ct: Ct, g: int, rotk: np.ndarray, alpha: int, base2: int = 0) -> Ct:
    """SwitchKey(phi(c1), swk_{phi(s) -> s}) + (phi(c0), 0) (Appendix A.2);
    base2 as in relinearize."""
    t = automorphism(par, ct, g)
    ks = (keyswitch_base2(par, t.data[1], ct.level, rotk, base2) if base2
          else keyswitch(par, t.data[1], ct.level, rotk, alpha))
    mods = par.q[: ct.level + 1]
    return Ct(np.stack([rns_add(t.data[0], ks[0], mods), ks[1]]), ct.level, ct.scale)


# ---------------------------------------------------------------------------
# Base-2^w decomposition inside the key switch (Table 1, `base2`: needed when P
# cannot grow without lowering security).  One-prime digits: the gadget digit
# (i, b) is q_i's CRT unit times 2^(w b), b < B = ceil(max prime bits / w); the
# polynomial d splits as d_i = sum_b d_(i,b) 2^(w b) with 0 <= d_(i,b) < 2^w, so
# the key inner product multiplies the small pieces (noise ~ 2^w instead of q_i)
# and the pieces need no base conversion (they are the same integers modulo
# every prime).
# ---------------------------------------------------------------------------
def base2_pieces(par: Params, w: int) -> int:
    return max(-(-int(q).bit_length() // w) for q in par.q)


def switch_key_base2(par: Params, s_to: np.ndarray, s_from_rns: np.ndarray, a: np.ndarray, e: np.ndarray,
                     w: int) -> np.ndarray:
    """a: uint64[(L+1) B][L+1+K][N], e: int64[(L+1) B][N] -> uint64[(L+1) B][2][L+1+K][N];
    digit i B + b holds (-a s + e + P 2^(w b) s_from [limb i only], a)."""
    mods = par.moduli
    nqp = len(mods)
    B = base2_pieces(par, w)
    nd = (par.L + 1) * B
    assert a.shape == (nd, nqp, par.N) and e.shape == (nd, par.N)
    s_rns = rns.to_rns(s_to, mods)
    out = np.empty((nd, 2, nqp, par.N), dtype=np.uint64)
    for i in range(par.L + 1):
        qi = int(mods[i])
        for b in range(B):
            j = i * B + b
            as_ = rns_mul(a[j], s_rns, mods, par.psi)
            bj = rns_sub(rns.to_rns(e[j], mods), as_, mods)
            term = rns_mul_int(s_from_rns[i:i + 1], (par.P << (w * b)) % qi, [qi])
            bj[i:i + 1] = rns_add(bj[i:i + 1], term, [qi])
            out[j, 0] = bj
            out[j, 1] = a[j]
    return out


def keyswitch_base2(par: Params, d: np.ndarray, level: int, evk: np.ndarray, w: int) -> np.ndarray:
    """SwitchKey(d, swk) with the base-2^w gadget at the given level: sum over the
    pieces of d_(i,b) * swk_(i,b) over Q_level P, then ModDown by P."""
    nl, K, N = level + 1, par.K, par.N
    B = evk.shape[0] // (par.L + 1)
    tidx = list(range(nl)) + [par.L + 1 + k for k in range(K)]
    tmods = [par.moduli[t] for t in tidx]
    tpsi = [par.psi[t] for t in tidx]
    acc = np.zeros((2, nl + K, N), dtype=np.uint64)
    mask = np.uint64((1 << w) - 1)
    for i in range(nl):
        di = np.asarray(d[i], dtype=np.uint64)
        for b in range(B):
            piece = ((di >> np.uint64(w * b)) & mask).astype(np.int64)
            pr = rns.to_rns(piece, tmods)
            key = evk[i * B + b][:, tidx]
            for c in range(2):
                acc[c] = rns_add(acc[c], rns_mul(pr, np.ascontiguousarray(key[c]), tmods, tpsi), tmods)
    out = np.empty((2, nl, N), dtype=np.uint64)
    for c in range(2):
        o = np.empty((nl, N), dtype=np.uint64)
        lib().or_moddown(ptr(np.ascontiguousarray(acc[c])), nl, K, ptr(u64arr(tmods)), N, ptr(o))
        out[c] = o
    return out
