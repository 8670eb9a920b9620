"""Oracle for the encrypted-query circuit: plan (levels, scales, integer
constants), plain per-block execution, and the FP64 plaintext pipeline the
decrypted result is judged against.

TEST INFRASTRUCTURE (see oracle/__init__.py).

The circuit is the server side of the paper's exploration (Algorithm 2, the
local threshold and InnerSum): a linear combination of attribute columns with
encrypted coefficients (attribute selection, Section 3.3), a private
polynomial with encrypted coefficients, subtraction of an encrypted threshold
(Section 5.4.2), a composite odd sign polynomial mapped to step(x) =
(sign(x)+1)/2 (Section 5.4.2), a sum over ciphertext blocks and InnerSum by
rotations (Appendix A.1.2 rotation semantics).

Scale discipline (a reading; the paper only says scales multiply and rescale
divides, Section 2.5): every ciphertext at level l carries the standard scale
S[l], S[L] = Delta, S[l-1] = S[l]*S[l]/q_l, so the product of two level-l
ciphertexts rescales exactly onto S[l-1]. A ciphertext is moved to a lower
level t by adjust(): keep primes q_0..q_{t+1}, multiply by the integer
floor(a*S[t]*q_{t+1}/scale + 1/2) (which also applies a public factor a), and
rescale by q_{t+1}.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

import synth
from . import ckks, rns
from .ckks import Ct, Params, round_half_up


# ---------------------------------------------------------------------------
# Sign polynomials (Section 5.4.2; the paper composes low-degree polynomials
# after Lee et al. but prints no coefficients).  Default stage: the odd
# degree-7 polynomial f3 with f3(1) = 1 and f3'(x) = 35/16 (1-x^2)^3.
# ---------------------------------------------------------------------------
F3 = (35.0 / 16.0, -35.0 / 16.0, 21.0 / 16.0, -5.0 / 16.0)   # coefficients of x, x^3, x^5, x^7


def odd_poly(coeffs, x):
    x = np.asarray(x, dtype=np.float64)
    return sum(a * x ** (2 * k + 1) for k, a in enumerate(coeffs))


def composite_sign(stages, x):
    for c in stages:
        x = odd_poly(c, x)
    return x


def sign_margin(stages, tol: float, grid: int = 1 << 20) -> float:
    """Smallest a in (0, 1] such that |composite(x) - sign(x)| <= tol for all
    a <= |x| <= 1 on a dense grid (brute force over the grid)."""
    x = np.linspace(0.0, 1.0, grid + 1)[1:]
    err = np.abs(composite_sign(stages, x) - 1.0)
    bad = np.nonzero(err > tol)[0]
    if bad.size == 0:
        return float(x[0])
    if bad[-1] + 1 >= x.size:
        return 1.0
    return float(x[bad[-1] + 1])


# ---------------------------------------------------------------------------
# Query shape and plan
# ---------------------------------------------------------------------------
@dataclass
class QueryShape:
    records: int
    attrs: int
    degree: int
    sign_stages: list            # list of (a0, a1, a2, a3) for x, x^3, x^5, x^7
    norm_records: int = 0        # records the count is normalised by (0: this database's own);
                                 # the total over partitions for a horizontally split database (Section 5.6)
    global_stages: list = field(default_factory=list)   # stages of the global threshold (empty: none)

    def blocks(self, n_slots: int) -> int:
        return -(-self.records // n_slots)


def standard_scales(par: Params) -> list:
    S = [0.0] * (par.L + 1)
    S[par.L] = float(par.scale)
    for l in range(par.L, 0, -1):
        S[l - 1] = (S[l] * S[l]) / float(par.q[l])
    return S


def ceil_log2(k: int) -> int:
    return (k - 1).bit_length()


def poly_schedule(degree: int):
    """Baby-step giant-step form of y = sum_k c_k x^k with encrypted c_k (a
    reading: the paper does not say how the private polynomial is evaluated).

    With g = 2^b baby steps and m = ceil((d+1)/g) giant steps,
      y = s_0 + sum_{i>=1} s_i * x^{g i},  s_i = sum_{j<g} c_{g i + j} x^j,
    every s_i (i >= 1) relinearised once and the degree-2 products of the last
    sum sharing one relinearisation.  Relinearisations: (g - 2) baby powers,
    (m - 1) giant powers, one per s_i with a j >= 1 term, one final.  Depths
    (rescales after x): baby power x^j ceil_log2(j), giant x^{g i}
    b + ceil_log2(i), s_i ceil_log2(g-1) + 1, the final products at
    D_f = max(ceil_log2(g-1) + 1, b + ceil_log2(m-1)).  A schedule is taken
    only if D_f <= ceil_log2(d) (y lands no lower than with plain powers) and it
    needs strictly fewer relinearisations than the d of plain powers; among
    those the fewest relinearisations, then the smallest g.
    Returns None (plain powers) or (g, m, bb, D_f) with bb = ceil_log2(g-1)."""
    best = None
    for b in range(1, ceil_log2(degree + 1) + 1):
        g = 1 << b
        m = -(-(degree + 1) // g)
        if m < 2:
            break
        bb = ceil_log2(g - 1)
        df = max(bb + 1, b + ceil_log2(m - 1))
        if df > ceil_log2(degree):
            continue
        relins = (g - 2) + (m - 1) + sum(1 for i in range(1, m) if g * i + 1 <= degree) + 1
        if relins < degree and (best is None or relins < best[0]):
            best = (relins, g, m, bb, df)
    return None if best is None else best[1:]


@dataclass
class Plan:
    S: list
    l_lin: int          # level of the linear combination x
    l_d: int            # level at which the c_k x^k products are formed (plain powers)
    l_y: int            # level of y = f(x) and z = y - t
    l_u: int            # level after the sign stages and step affine
    l_out: int          # level of the summed step values (scale S[l_out])
    pt_scale: float     # scale of the database plaintexts
    mask_scale: float   # scale of the ragged-block mask plaintext (0 if none)
    ragged: bool
    stage_coeffs: list = field(default_factory=list)   # folded coefficients per stage
    step_const: float = 0.0
    bsgs: tuple | None = None   # poly_schedule(degree): (g, m, bb, D_f) or None
    degree: int = 0
    # level of the returned ciphertext: the sum is dropped to it before InnerSum
    # (a reading: the paper does not fix where the rotations run; at level 1
    # their key switches cover two primes, and |value| <= S[l_out] stays far
    # inside q_0 q_1)
    l_ret: int = 1
    # global threshold (Algorithm 2, last line): step((count - t1 + 1/2) / R) on
    # the InnerSum result at l_out; the 1/2 is the epsilon/2 shift of Section
    # 4.3.2 for integer counts (so the bit is count >= t1); the last stage's
    # coefficients carry the 1/2 of step = (p + 1)/2
    global_coeffs: list = field(default_factory=list)
    records_norm: float = 0.0
    # the circuit starts as low as its depth allows (a reading: Section 2.5
    # only says each rescale consumes a level, not where a circuit starts):
    # the w_j (top level, scale Delta) are dropped to l_lin + 1, and the
    # rescaled sum of their products with the database plaintexts (scale
    # pt_scale, encoded once for any query) has scale
    # x_scale = Delta pt_scale / q_{l_lin+1}, carried through the powers of x
    # by power_scales; the circuit ends at level 1
    x_scale: float = 0.0
    # factor each encrypted coefficient c_k carries after its arrival adjust (a
    # reading, like the schedule): the power x^j it multiplies is only dropped
    # (no rescale) to the product's level lt, so c_k carries S[lt] / S[level of
    # x^j] and the degree-2 product lands on S[lt]^2; 1 where c_k is added
    coef_factors: list = field(default_factory=list)

    def coef_level(self, k: int) -> int:
        """Level at which the encrypted coefficient c_k is used."""
        if k == 0:
            return self.l_y
        if self.bsgs is None:
            return self.l_d
        g, m, bb, df = self.bsgs
        i, j = divmod(k, g)
        if i == 0:
            return self.l_lin - df            # s_0 terms, formed with the final products
        if j >= 1:
            return self.l_lin - bb            # tensors of s_i
        if k + 1 <= self.degree:
            return self.l_lin - bb - 1        # added to s_i after its relinearisation
        return self.l_lin - df                # s_i = c_k alone (k = d)


def stage_depth(co) -> int:
    """Levels a sign stage consumes: odd degree 7 (4 coefficients) in 3, degree 15 (8) in 4."""
    if len(co) not in (4, 8):
        raise ValueError("sign stages are odd polynomials of degree 7 or 15")
    return 3 if len(co) == 4 else 4


def make_plan(par: Params, shape: QueryShape) -> Plan:
    if shape.degree < 1 or shape.attrs < 1 or shape.records < 1 or not shape.sign_stages:
        raise ValueError("empty query")
    L, S = par.L, standard_scales(par)
    n = par.n_slots
    ragged = shape.records % n != 0
    # levels consumed below l_lin: the polynomial, the sign stages, the ragged
    # block's mask, the global threshold
    used = (ceil_log2(shape.degree) + 1 + sum(stage_depth(co) for co in shape.sign_stages) + (1 if ragged else 0)
            + sum(stage_depth(co) for co in shape.global_stages))
    l_lin = min(L - 1, 1 + used)
    l_d = l_lin - ceil_log2(shape.degree)
    l_y = l_d - 1
    l_u = l_y - sum(stage_depth(co) for co in shape.sign_stages)
    l_out = l_u - 1 if ragged else l_u
    if l_out < 1:
        raise ValueError(f"circuit needs more levels: ends at level {l_out}")
    R = float(shape.norm_records if shape.norm_records else shape.records)
    stages = []
    ns = len(shape.sign_stages)
    for s, co in enumerate(shape.sign_stages):
        co = [float(c) for c in co]
        stage_depth(co)
        if s == 0:   # z = (y - t)/2 folded in: a_k -> a_k * 2^-(2k+1)
            co = [c * (0.5 ** (2 * k + 1)) for k, c in enumerate(co)]
        if s == ns - 1:   # step = (p + 1) / 2, normalised by 1/records
            co = [c / (2.0 * R) for c in co]
        stages.append(co)
    gco = []
    for s, co in enumerate(shape.global_stages):
        co = [float(c) for c in co]
        stage_depth(co)
        if s == len(shape.global_stages) - 1:
            co = [c / 2.0 for c in co]
        gco.append(co)
    l_ret = l_out - sum(stage_depth(co) for co in gco) if gco else 1
    if l_ret < 1:
        raise ValueError(f"global threshold needs more levels: ends at level {l_ret}")
    pt_scale = (S[L - 1] * float(par.q[L])) / S[L]
    x_scale = (S[L] * pt_scale) / float(par.q[l_lin + 1])
    bsgs = poly_schedule(shape.degree)
    cf = [1.0] * (shape.degree + 1)
    if bsgs is None:
        sp, _ = power_scales(x_scale, l_lin, shape.degree, par.q)
    else:
        g, m, bb, df = bsgs
        sp, lp = power_scales(x_scale, l_lin, max(g - 1, 1), par.q)
        h = max(g // 2, 1)
        sg, _ = power_scales((sp[h] * sp[h]) / float(par.q[lp[h]]), lp[h] - 1, max(m - 1, 1), par.q)
    for k in range(1, shape.degree + 1):
        if bsgs is None:
            cf[k] = S[l_d] / sp[k]
            continue
        i, j = divmod(k, g)
        l_b, l_f = l_lin - bb, l_lin - df
        if i == 0:
            cf[k] = S[l_f] / sp[j]
            continue
        # s_i multiplies x^(g i) dropped to l_f, and is itself dropped there
        # from l_b - 1 (its terms carry S[l_f] / S[l_b - 1] for that; c_d
        # alone, at l_f, does not)
        fi = S[l_f] / sg[i]
        rb = S[l_f] / S[l_b - 1]
        if j >= 1:
            cf[k] = (fi * (S[l_b] / sp[j])) * rb
        else:
            cf[k] = fi * rb if k < shape.degree else fi
    return Plan(S=S, l_lin=l_lin, l_d=l_d, l_y=l_y, l_u=l_u, l_out=l_out, l_ret=l_ret, global_coeffs=gco,
                records_norm=R, x_scale=x_scale,
                pt_scale=pt_scale,
                mask_scale=((S[l_u - 1] * float(par.q[l_u])) / S[l_u]) if ragged else 0.0,
                ragged=ragged, stage_coeffs=stages, step_const=1.0 / (2.0 * R),
                bsgs=bsgs, degree=shape.degree, coef_factors=cf)


def power_scales(scale: float, level: int, n: int, q) -> tuple:
    """Scales and levels of y^1..y^n formed from y (scale, level) by the power
    rule y^k = y^a y^(k-a), a the largest power of two <= k (a power of two is
    the square of its half), the lower factor dropped to the other's level and
    the relinearisation's rescale removing that level's prime."""
    sc, lv = {1: scale}, {1: level}
    for k in range(2, n + 1):
        a = 1 << (k.bit_length() - 1)
        A, B = (k // 2, k // 2) if a == k else (a, k - a)
        sc[k] = (sc[A] * sc[B]) / float(q[lv[A]])
        lv[k] = lv[A] - 1
    return sc, lv


def adjust_const(plan: Plan, par: Params, lt: int, a: float, scale: float) -> int:
    return round_half_up(((a * plan.S[lt]) * float(par.q[lt + 1])) / scale)


# ---------------------------------------------------------------------------
# Database encoding (Appendix A.1.2): records fill the N/2 slots of each block
# in order; slot values are the normalised attribute / attrs.
# ---------------------------------------------------------------------------
def normalise(vals_u8: np.ndarray) -> np.ndarray:
    return (vals_u8.astype(np.float64) - 127.5) / 127.5


def block_slots(par: Params, vals_u8: np.ndarray, b: int, j: int) -> np.ndarray:
    n = par.n_slots
    rec = vals_u8[b * n:(b + 1) * n, j]
    z = np.zeros(n)
    z[: rec.shape[0]] = normalise(rec) / vals_u8.shape[1]
    return z


@dataclass
class EncodedDB:
    pts: list           # [blocks][attrs] int64[N] coefficients at plan.pt_scale
    mask: object        # int64[N] at plan.mask_scale, or None


def encode_database(par: Params, plan: Plan, vals_u8: np.ndarray) -> EncodedDB:
    R, h = vals_u8.shape
    B = -(-R // par.n_slots)
    pts = [[ckks.encode_int(par.N, block_slots(par, vals_u8, b, j), plan.pt_scale) for j in range(h)] for b in range(B)]
    mask = None
    if plan.ragged:
        live = R - (B - 1) * par.n_slots
        z = np.zeros(par.n_slots)
        z[:live] = 1.0
        mask = ckks.encode_int(par.N, z, plan.mask_scale)
    return EncodedDB(pts=pts, mask=mask)


# ---------------------------------------------------------------------------
# Keys and encrypted query (client side, from the seeded draws)
# ---------------------------------------------------------------------------
def innersum_galois(par: Params) -> list:
    return [pow(5, 1 << k, 2 * par.N) for k in range(par.log_n - 1)]


@dataclass
class Keys:
    alpha: int
    rlk: np.ndarray
    rot: dict           # galois element -> key
    base2: int = 0      # w of the base-2^w gadget (Table 1), 0 for the plain hybrid switch


def secret(par: Params, seed: int, h: int) -> np.ndarray:
    return synth.ternary_secret(synth.stream(seed, "secret"), par.N, h)


def make_keys(par: Params, s: np.ndarray, seed: int, alpha: int, galois=(), base2: int = 0) -> Keys:
    """Relinearisation and rotation keys; base2 = w > 0 makes base-2^w keys
    (one-prime digits, (L+1) B of them, Table 1's base2)."""
    if base2:
        if alpha != 1:
            raise ValueError("the base-2^w gadget takes one-prime digits")
        dnum = (par.L + 1) * ckks.base2_pieces(par, base2)
        mods = par.moduli
        s_rns = rns.to_rns(s, mods)
        gen = lambda s_from, d: ckks.switch_key_base2(par, s, s_from, d.a, d.e, base2)
        d = synth.switch_key_draws(seed, "relin", dnum, mods, par.N)
        rlk = gen(ckks.rns_mul(s_rns, s_rns, mods, par.psi), d)
        rot = {}
        for g in galois:
            d = synth.switch_key_draws(seed, f"rot{g}", dnum, mods, par.N)
            rot[g] = gen(ckks.automorphism_poly(s_rns, g, mods), d)
        return Keys(alpha=1, rlk=rlk, rot=rot, base2=base2)
    dnum = ckks.dnum_for(par.L, alpha)
    d = synth.switch_key_draws(seed, "relin", dnum, par.moduli, par.N)
    rlk = ckks.relin_key(par, s, d.a, d.e, alpha)
    rot = {}
    for g in galois:
        d = synth.switch_key_draws(seed, f"rot{g}", dnum, par.moduli, par.N)
        rot[g] = ckks.rotation_key(par, g, s, d.a, d.e, alpha)
    return Keys(alpha=alpha, rlk=rlk, rot=rot)


def encrypt_value(par: Params, s: np.ndarray, v: float, seed: int, name: str, level=None) -> Ct:
    """Encryption of v in every slot: the constant polynomial round(v * Delta)."""
    level = par.L if level is None else level
    m = np.zeros(par.N, dtype=np.int64)
    m[0] = round_half_up(v * par.scale)
    d = synth.encryption_draws(seed, name, par.q[: level + 1], par.N)
    return ckks.encrypt(par, m, s, d.a, d.e, level, par.scale)


@dataclass
class EncQuery:
    w: list
    c: list
    t: Ct
    t1: Ct | None = None


def encrypt_query(par: Params, s: np.ndarray, qv: synth.QueryValues, seed: int) -> EncQuery:
    return EncQuery(w=[encrypt_value(par, s, float(v), seed, f"w{j}") for j, v in enumerate(qv.w)],
                    c=[encrypt_value(par, s, float(v), seed, f"c{k}") for k, v in enumerate(qv.c)],
                    t=encrypt_value(par, s, float(qv.t), seed, "t"),
                    t1=None if qv.t1 is None else encrypt_value(par, s, float(qv.t1), seed, "t1"))


# ---------------------------------------------------------------------------
# Server-side evaluation
# ---------------------------------------------------------------------------
class Evaluator:
    def __init__(self, par: Params, keys: Keys, plan: Plan):
        self.par, self.keys, self.plan = par, keys, plan

    def adjust(self, ct: Ct, lt: int, a: float = 1.0) -> Ct:
        par, plan = self.par, self.plan
        if ct.level == lt:
            if a != 1.0 or ct.scale != plan.S[lt]:
                raise ValueError("adjust at the same level")
            return ct
        if ct.level < lt:
            raise ValueError("input ciphertext level too low")
        c = adjust_const(plan, par, lt, a, ct.scale)
        out = ckks.rescale(par, ckks.mul_int(par, ckks.drop_to(ct, lt + 1), c))
        out.scale = plan.S[lt]
        return out

    def mul(self, a: Ct, b: Ct) -> Ct:
        assert a.level == b.level
        par = self.par
        out = ckks.rescale(par, ckks.relinearize(par, ckks.tensor(par, a, b), self.keys.rlk, self.keys.alpha, self.keys.base2))
        out.scale = self.plan.S[a.level - 1]
        return out

    def add(self, a: Ct, b: Ct) -> Ct:
        return ckks.add(self.par, a, b)

    def relin_rescale(self, t: Ct, level_out: int) -> Ct:
        par = self.par
        out = ckks.rescale(par, ckks.relinearize(par, t, self.keys.rlk, self.keys.alpha, self.keys.base2))
        out.scale = self.plan.S[level_out]
        return out

    def fold(self, T: Ct, v: Ct, a: float) -> Ct:
        """T + a v for a degree-2 accumulator T at level lt (plaintext scale
        S[lt]^2) and a ciphertext v at level >= lt: v is dropped to lt and
        multiplied by the integer round(a S[lt]^2 / scale(v)), no rescale (the
        relinearisation's rescale that follows covers it).  A reading: the
        paper does not say how the sign polynomial's terms are combined."""
        par, lt = self.par, T.level
        cf = ((a * self.plan.S[lt]) * self.plan.S[lt]) / v.scale
        if not abs(cf) < 2.0 ** 62:
            raise ValueError("fold: coefficient too large for an integer multiple")
        c = round_half_up(cf)
        m = ckks.mul_int(par, ckks.drop_to(v, lt), c)
        mods = par.q[: lt + 1]
        data = T.data.copy()
        data[0] = ckks.rns_add(data[0], m.data[0], mods)
        data[1] = ckks.rns_add(data[1], m.data[1], mods)
        return Ct(data, lt, T.scale)

    def odd7(self, a3u: Ct, a1u: Ct, c2: float, c0: float, u: Ct, u2: Ct, u2d: Ct, u4: Ct, l: int) -> Ct:
        """c0 u + [(a1 u) u^2 + ((a3 u) u^2 + c2 u) u^4] from the adjusts
        a3u (level l-1) and a1u (l-2): c2 u folded into (a3 u) u^2 before its
        relinearisation at l-1, c0 u into the bracket's two degree-2 products
        at l-2, which are relinearised once; ends at level l-3."""
        par = self.par
        inner = self.relin_rescale(self.fold(ckks.tensor(par, a3u, u2), u, c2), l - 2)
        T = ckks.add(par, ckks.tensor(par, a1u, u2d), ckks.tensor(par, inner, u4))
        return self.relin_rescale(self.fold(T, u, c0), l - 3)

    def sign_stage(self, u: Ct, co) -> Ct:
        """p(u) = sum_k a_k u^(2k+1).  Degree 7 (4 coefficients): depth 3,
        four relinearisations.  Degree 15 (8): depth 4 as A(u) + u^8 B(u),
        A and B the degree-7 parts of the low and high coefficients (u^2, u^4
        shared), eight relinearisations, A folded into u^8 B before its
        relinearisation."""
        l = u.level
        u2 = self.mul(u, u)
        u4 = self.mul(u2, u2)
        # u^2 is dropped to l-2 (scale S[l-1]); a1 u carries S[l-2] / S[l-1]
        u2d = ckks.drop_to(u2, l - 2)
        r = self.plan.S[l - 2] / self.plan.S[l - 1]
        A = self.odd7(self.adjust(u, l - 1, co[3]), self.adjust(u, l - 2, co[1] * r), co[2], co[0], u, u2, u2d, u4, l)
        if len(co) == 4:
            return A
        u8 = self.mul(u4, u4)
        B = self.odd7(self.adjust(u, l - 1, co[7]), self.adjust(u, l - 2, co[5] * r), co[6], co[4], u, u2, u2d, u4, l)
        return self.relin_rescale(self.fold(ckks.tensor(self.par, u8, B), A, 1.0), l - 4)

    def per_query(self, q: EncQuery, degree: int):
        """Bring the encrypted coefficients and threshold to their levels (once per query)."""
        p = self.plan
        for w in q.w:
            if w.level != self.par.L or w.scale != p.S[self.par.L]:
                raise ValueError("linear-combination coefficients must be fresh top-level ciphertexts")
        # the w_j at level l_lin + 1, where the linear combination is formed
        self.w_in = [ckks.drop_to(w, p.l_lin + 1) for w in q.w]
        ck = [self.adjust(q.c[k], p.coef_level(k), p.coef_factors[k]) for k in range(degree + 1)]
        return ck, self.adjust(q.t, p.l_y)

    def block(self, pts: list, q: EncQuery, ck: list, tadj: Ct, degree: int, record: dict | None = None) -> Ct:
        """One block's circuit; returns the per-slot step values u / R (after
        the sign stages and their affine map, before the block sum).  With a
        dict ``record`` it also keeps the ciphertexts of the intermediate
        stages: "x" the linear combination, "y" = f(x) (with c_0), "d" = y - t,
        and "u" the result."""
        keep = (lambda k, v: record.__setitem__(k, v)) if record is not None else (lambda k, v: None)
        par, p = self.par, self.plan
        L = par.L
        # linear combination: sum_j pt_j * Enc(w_j) at level l_lin + 1, rescale
        acc = None
        for pt, w in zip(pts, self.w_in):
            prod = ckks.mul_plain(par, w, rns.to_rns(pt, par.q[: p.l_lin + 2]), p.pt_scale)
            acc = prod if acc is None else ckks.add(par, acc, prod)
        x = ckks.rescale(par, acc)
        x.scale = p.x_scale
        keep("x", x)
        # powers x^k, k <= degree; a factor of lower power is dropped (not
        # adjusted) to the other's level, so a power's scale is the product of
        # its factors' over the prime the relinearisation removes (power_scales)
        P = {1: x}

        def power_rule(Q, k):
            # x^k = x^a x^(k-a), a the largest power of two <= k (depth ceil_log2(k))
            a = 1 << (k.bit_length() - 1)
            A, B = (Q[k // 2], Q[k // 2]) if a == k else (Q[a], ckks.drop_to(Q[k - a], Q[a].level))
            out = self.mul(A, B)
            out.scale = (A.scale * B.scale) / float(par.q[A.level])
            return out

        if p.bsgs is None:
            for k in range(2, degree + 1):
                P[k] = power_rule(P, k)
            # y = sum_k c_k x^k: degree-2 products summed, one relinearisation
            T = None
            for k in range(1, degree + 1):
                tk = ckks.tensor(par, ck[k], ckks.drop_to(P[k], p.l_d))
                T = tk if T is None else ckks.add(par, T, tk)
            y = self.relin_rescale(T, p.l_y)
        else:
            g, m, bb, df = p.bsgs
            l_b, l_f = p.l_lin - bb, p.l_lin - df
            for k in range(2, g):
                P[k] = power_rule(P, k)
            G = {1: power_rule({1: P[g // 2]}, 2)}     # giant powers x^(g i)
            for i in range(2, m):
                G[i] = power_rule(G, i)
            # s_i, i >= 1: sum_{j>=1} c_{gi+j} x^j at l_b, relinearised, plus c_{gi}
            T = None
            for j in range(1, g):          # s_0's terms at l_f
                tk = ckks.tensor(par, ck[j], ckks.drop_to(P[j], l_f))
                T = tk if T is None else ckks.add(par, T, tk)
            for i in range(1, m):
                Ti = None
                for j in range(1, g):
                    if g * i + j > degree:
                        break
                    tk = ckks.tensor(par, ck[g * i + j], ckks.drop_to(P[j], l_b))
                    Ti = tk if Ti is None else ckks.add(par, Ti, tk)
                if Ti is None:
                    si = ck[g * i]
                else:
                    si = ckks.drop_to(ckks.add(par, self.relin_rescale(Ti, l_b - 1), ck[g * i]), l_f)
                T = ckks.add(par, T, ckks.tensor(par, si, ckks.drop_to(G[i], l_f)))
            y = self.relin_rescale(T, l_f - 1)
            y = self.adjust(y, p.l_y)
        y = ckks.add(par, y, ck[0])
        keep("y", y)
        # z = y - t (the 1/2 is folded into the first sign stage)
        u = ckks.sub(par, y, tadj)
        keep("d", u)
        for co in p.stage_coeffs:
            u = self.sign_stage(u, co)
        u = ckks.add_int_const(par, u, round_half_up(p.step_const * p.S[u.level]))
        keep("u", u)
        return u

    def global_threshold(self, v: Ct, t1: Ct) -> Ct:
        """step((count - t1 + 1/2) / R) from v = count / R (Algorithm 2, last line)."""
        par, p = self.par, self.plan
        if t1 is None:
            raise ValueError("the global threshold needs an encrypted t1")
        z = ckks.sub(par, v, self.adjust(t1, v.level, 1.0 / p.records_norm))
        z = ckks.add_int_const(par, z, round_half_up(p.S[z.level] / (2.0 * p.records_norm)))
        for co in p.global_coeffs:
            z = self.sign_stage(z, co)
        return ckks.add_int_const(par, z, round_half_up(0.5 * p.S[z.level]))

    def innersum(self, acc: Ct) -> Ct:
        for g in innersum_galois(self.par):
            acc = ckks.add(self.par, acc, ckks.rotate(self.par, acc, g, self.keys.rot[g], self.keys.alpha, self.keys.base2))
        return acc


def evaluate_query(par: Params, keys: Keys, shape: QueryShape, db: EncodedDB, q: EncQuery, blocks=None) -> Ct:
    """The whole circuit; ``blocks`` restricts the block loop (for timing samples)."""
    plan = make_plan(par, shape)
    ev = Evaluator(par, keys, plan)
    ck, tadj = ev.per_query(q, shape.degree)
    B = len(db.pts)
    idx = range(B) if blocks is None else blocks
    full = None
    last = None
    for b in idx:
        u = ev.block(db.pts[b], q, ck, tadj, shape.degree)
        if plan.ragged and b == B - 1:
            last = u
        else:
            full = u if full is None else ckks.add(par, full, u)
    if plan.ragged and last is not None:
        m = ckks.rescale(par, ckks.mul_plain(par, last, rns.to_rns(db.mask, par.q), plan.mask_scale))
        m.scale = plan.S[plan.l_out]
        acc = m if full is None else ckks.add(par, ev.adjust(full, plan.l_out), m)
    else:
        acc = full
    if plan.global_coeffs:
        return ev.global_threshold(ev.innersum(acc), q.t1)
    if acc.level > plan.l_ret:
        acc = ckks.drop_to(acc, plan.l_ret)
    return ev.innersum(acc)


# ---------------------------------------------------------------------------
# FP64 plaintext pipeline
# ---------------------------------------------------------------------------
@dataclass
class Fp64Result:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    u: np.ndarray        # per-record step approximation
    count: float         # sum of u
    exact: int           # number of records with z > 0
    z2: float = 0.0      # global threshold input (count - t1 + 1/2) / R
    bit: float = 0.0     # its step approximation
    exact_bit: int = 0   # 1 iff exact >= t1


def fp64_pipeline(vals_u8: np.ndarray, qv: synth.QueryValues, stages, global_stages=(), records=0) -> Fp64Result:
    h = vals_u8.shape[1]
    x = (normalise(vals_u8) / h) @ np.asarray(qv.w, dtype=np.float64)
    y = sum(c * x ** k for k, c in enumerate(qv.c))
    z = (y - qv.t) / 2.0
    u = (composite_sign(stages, z) + 1.0) / 2.0
    r = Fp64Result(x=x, y=y, z=z, u=u, count=float(u.sum()), exact=int((z > 0).sum()))
    if global_stages:
        R = float(records or vals_u8.shape[0])
        r.z2 = (r.count - qv.t1 + 0.5) / R
        r.bit = float((composite_sign(global_stages, np.array([r.z2]))[0] + 1.0) / 2.0)
        r.exact_bit = int(r.exact >= qv.t1)
    return r
