"""GPU parity, primitive by primitive: every operation of the CUDA library,
called through the C ABI, returns the oracle's residues bit for bit on the
same seeded inputs (coefficient domain at the boundary).  The FP64 encoder is
the one floating-point step: its integer coefficients may differ from the
oracle's by one unit where a product straddles a rounding boundary."""
import numpy as np
import pytest

import synth
from oracle import ckks, query, rns

pytestmark = pytest.mark.gpu

T = pytest.importorskip("paper_2412_13269_gb300")


def brv(k: int, bits: int) -> int:
    return int(format(k, f"0{bits}b")[::-1], 2)


def rand_ct(par, comps, level, seed):
    g = np.random.default_rng(seed)
    return np.stack([np.stack([g.integers(0, q, par.N, dtype=np.uint64) for q in par.q[: level + 1]]) for _ in range(comps)])


class Setup:
    def __init__(self, log_n, q, p, scale, alpha, seed, rot_steps=(1,)):
        self.par = ckks.Params(log_n, q, p, scale)
        self.ctx = T.Ctx(log_n, q, p, scale)
        self.alpha = alpha
        self.s = query.secret(self.par, seed, min(2 * self.par.N // 3, 192 if log_n >= 15 else 2 * self.par.N // 3))
        gal = sorted(set(query.innersum_galois(self.par)) | {ckks.galois_for_rotation(self.par.N, k) for k in rot_steps})
        self.keys = query.make_keys(self.par, self.s, seed, alpha, gal)
        self.ctx.load_relin_key(self.keys.rlk, alpha)
        for g, k in self.keys.rot.items():
            self.ctx.load_rotation_key(g, k, alpha)


@pytest.fixture(scope="module")
def small():
    T.build()
    q = rns.gen_primes(50, 1) + rns.gen_primes(40, 3)
    return Setup(12, q, rns.gen_primes(60, 1), 2.0 ** 40, 1, 21)


@pytest.fixture(scope="module")
def wide():
    """N = 2^12 with three special primes and three-prime digits (alpha = 3), 8 ciphertext primes."""
    T.build()
    q = rns.gen_primes(50, 8)
    return Setup(12, q, rns.gen_primes(60, 3), 2.0 ** 50, 3, 22)


@pytest.fixture(scope="module")
def wide4():
    """As `wide` with four-prime digits (alpha = 4 > K = 3), the benchmark's digit size."""
    T.build()
    q = rns.gen_primes(50, 8)
    return Setup(12, q, rns.gen_primes(60, 3), 2.0 ** 50, 4, 24)


def test_ntt_order_and_values(small):
    par, ctx = small.par, small.ctx
    a = rand_ct(par, 1, 3, 1)
    got, lev, _ = ctx.op(T.OP_NTT, a, 3, out_comps=1)
    for i in range(4):
        x = a[0, i].copy()
        rns.lib().or_ntt(rns.ptr(x), par.N, par.q[i], par.psi[i])
        perm = np.array([brv(k, par.log_n) for k in range(par.N)])
        assert np.array_equal(got[0, i], x[perm]), i


@pytest.mark.parametrize("fx", ["small", "wide", "wide4"])
def test_elementwise(fx, request):
    S = request.getfixturevalue(fx)
    par, ctx = S.par, S.ctx
    l = par.L
    a, b = rand_ct(par, 2, l, 2), rand_ct(par, 2, l, 3)
    A, B = ckks.Ct(a, l, 1.0), ckks.Ct(b, l, 1.0)
    assert np.array_equal(ctx.op(T.OP_ADD, a, l, b=b, b_level=l)[0], ckks.add(par, A, B).data)
    assert np.array_equal(ctx.op(T.OP_SUB, a, l, b=b, b_level=l)[0], ckks.sub(par, A, B).data)
    for c in (3, -7, (1 << 45) + 12345, -(1 << 50) - 3):
        assert np.array_equal(ctx.op(T.OP_MUL_INT, a, l, arg=c)[0], ckks.mul_int(par, A, c).data), c
        assert np.array_equal(ctx.op(T.OP_ADD_INT, a, l, arg=c)[0], ckks.add_int_const(par, A, c).data), c
    assert np.array_equal(ctx.op(T.OP_DROP, a, l, arg=1)[0], ckks.drop_to(A, 1).data)
    for g in (5, 25, 2 * par.N - 1, 3):
        assert np.array_equal(ctx.op(T.OP_AUTOMORPHISM, a, l, arg=g)[0], ckks.automorphism(par, A, g).data), g
    t = ctx.op(T.OP_TENSOR, a, l, b=b, b_level=l)[0]
    assert np.array_equal(t, ckks.tensor(par, A, B).data)
    pt = rand_ct(par, 1, l, 4)
    got = ctx.op(T.OP_MUL_PLAIN, a, l, b=pt, b_level=l)[0]
    assert np.array_equal(got, ckks.mul_plain(par, A, pt[0], 1.0).data)


@pytest.mark.parametrize("fx", ["small", "wide", "wide4"])
def test_rescale(fx, request):
    S = request.getfixturevalue(fx)
    par, ctx = S.par, S.ctx
    for l in range(1, par.L + 1):
        for comps in (2, 3):
            a = rand_ct(par, comps, l, 10 + l)
            got, lev, _ = ctx.op(T.OP_RESCALE, a, l)
            want = ckks.rescale(par, ckks.Ct(a, l, 1.0))
            assert lev == l - 1 and np.array_equal(got, want.data), (l, comps)


@pytest.mark.parametrize("fx", ["small", "wide", "wide4"])
def test_keyswitch_relin_rotate(fx, request):
    S = request.getfixturevalue(fx)
    par, ctx, keys = S.par, S.ctx, S.keys
    for l in sorted({par.L, max(0, par.L - 2), 0}):
        d = rand_ct(par, 1, l, 30 + l)
        got = ctx.op(T.OP_KEYSWITCH, d, l, arg=0, out_comps=2)[0]
        assert np.array_equal(got, ckks.keyswitch(par, d[0], l, keys.rlk, S.alpha)), l
        t3 = rand_ct(par, 3, l, 40 + l)
        got = ctx.op(T.OP_RELIN, t3, l, out_comps=2)[0]
        assert np.array_equal(got, ckks.relinearize(par, ckks.Ct(t3, l, 1.0), keys.rlk, S.alpha).data), l
        g = ckks.galois_for_rotation(par.N, 1)
        a = rand_ct(par, 2, l, 50 + l)
        got = ctx.op(T.OP_ROTATE, a, l, arg=g, out_comps=2)[0]
        assert np.array_equal(got, ckks.rotate(par, ckks.Ct(a, l, 1.0), g, keys.rot[g], S.alpha).data), l


@pytest.mark.parametrize("fx", ["small", "wide", "wide4"])
def test_fused_relin_rescale_and_factor_rescale(fx, request):
    """The fused forms equal the oracle's compositions: rescale(relinearize(t))
    and rescale(mul_int(a, f)), including factors that are not invertible
    modulo a prime of the chain (the unfused fallback)."""
    S = request.getfixturevalue(fx)
    par, ctx, keys = S.par, S.ctx, S.keys
    for l in range(1, par.L + 1):
        t3 = rand_ct(par, 3, l, 80 + l)
        got, lev, _ = ctx.op(T.OP_RELIN_RESCALE, t3, l, out_comps=2)
        want = ckks.rescale(par, ckks.relinearize(par, ckks.Ct(t3, l, 1.0), keys.rlk, S.alpha))
        assert lev == l - 1 and np.array_equal(got, want.data), l
    l = par.L
    a = rand_ct(par, 2, l, 90)
    for f in (1, 3, -7, (1 << 45) + 12345, -(1 << 50) - 3, par.q[0], -par.q[l], 2 * par.q[1]):
        got, lev, _ = ctx.op(T.OP_RESCALE_MUL_INT, a, l, arg=f)
        want = ckks.rescale(par, ckks.mul_int(par, ckks.Ct(a, l, 1.0), f))
        assert lev == l - 1 and np.array_equal(got, want.data), f


def test_innersum(small):
    par, ctx = small.par, small.ctx
    a = rand_ct(par, 2, 1, 60)
    got = ctx.op(T.OP_INNERSUM, a, 1, out_comps=2)[0]
    acc = ckks.Ct(a, 1, 1.0)
    for g in query.innersum_galois(par):
        acc = ckks.add(par, acc, ckks.rotate(par, acc, g, small.keys.rot[g], small.alpha))
    assert np.array_equal(got, acc.data)


@pytest.mark.parametrize("fx", ["small", "wide", "wide4"])
def test_keygen_matches_oracle(fx, request):
    S = request.getfixturevalue(fx)
    par = S.par
    ctx = T.Ctx(par.log_n, par.q, par.p, par.scale)
    dnum = ckks.dnum_for(par.L, S.alpha)
    d = synth.switch_key_draws(77, "relin", dnum, par.moduli, par.N)
    ctx.keygen_relin(S.s, d.a, d.e, S.alpha)
    assert np.array_equal(ctx.get_key(0, dnum), ckks.relin_key(par, S.s, d.a, d.e, S.alpha))
    g = ckks.galois_for_rotation(par.N, 3)
    d = synth.switch_key_draws(77, f"rot{g}", dnum, par.moduli, par.N)
    ctx.keygen_rotation(g, S.s, d.a, d.e, S.alpha)
    assert np.array_equal(ctx.get_key(g, dnum), ckks.rotation_key(par, g, S.s, d.a, d.e, S.alpha))
    ctx.close()


def test_encrypt_matches_oracle(small):
    par, ctx = small.par, small.ctx
    m = ckks.encode_int(par.N, np.linspace(-1, 1, par.n_slots), par.scale)
    for level in (par.L, 1):
        d = synth.encryption_draws(5, "enc", par.q[: level + 1], par.N)
        got = ctx.encrypt(m, small.s, d.a, d.e, level, par.scale)
        want = ckks.encrypt(par, m, small.s, d.a, d.e, level, par.scale)
        assert np.array_equal(got, want.data)


@pytest.mark.parametrize("log_n", [12, 16])
def test_encoder_within_one_unit(log_n):
    T.build()
    q = rns.gen_primes(50, 3)
    ctx = T.Ctx(log_n, q, rns.gen_primes(60, 1), 2.0 ** 50)
    N = 1 << log_n
    z = np.random.default_rng(log_n).uniform(-1, 1, N // 2) / 16
    m_gpu = ctx.encode_real(z)
    m_ref = ckks.encode_real(N, z, 1.0)
    assert np.max(np.abs(m_gpu - m_ref)) < 1e-14
    for scale in (2.0 ** 40, 2.0 ** 50):
        got = ctx.encode(z, scale)
        want = ckks.encode_int(N, z, scale)
        diff = np.abs(got - want)
        assert diff.max() <= 1
        assert (diff > 0).mean() < 0.01
    ctx.close()


def test_full_size_primitives():
    """N = 2^16 with twenty 50-bit primes and three 60-bit special primes:
    NTT, rescale and relinearisation at the top level (alpha = 3)."""
    T.build()
    q, p = rns.gen_primes(50, 20), rns.gen_primes(60, 3)
    par = ckks.Params(16, q, p, 2.0 ** 50)
    ctx = T.Ctx(16, q, p, 2.0 ** 50)
    s = query.secret(par, 9, 192)
    alpha = 3
    dnum = ckks.dnum_for(par.L, alpha)
    d = synth.switch_key_draws(9, "relin", dnum, par.moduli, par.N)
    ctx.keygen_relin(s, d.a, d.e, alpha)
    rlk = ckks.relin_key(par, s, d.a, d.e, alpha)
    assert np.array_equal(ctx.get_key(0, dnum), rlk)
    l = par.L
    a = rand_ct(par, 3, l, 99)
    got = ctx.op(T.OP_RELIN, a, l, out_comps=2)[0]
    assert np.array_equal(got, ckks.relinearize(par, ckks.Ct(a, l, 1.0), rlk, alpha).data)
    got, lev, _ = ctx.op(T.OP_RESCALE, a, l)
    assert np.array_equal(got, ckks.rescale(par, ckks.Ct(a, l, 1.0)).data)
    got, lev, _ = ctx.op(T.OP_RELIN_RESCALE, a, l, out_comps=2)
    want = ckks.rescale(par, ckks.relinearize(par, ckks.Ct(a, l, 1.0), rlk, alpha))
    assert lev == l - 1 and np.array_equal(got, want.data)
    ctx.close()


def test_reduce_sum_device(small):
    torch = pytest.importorskip("torch")
    par, ctx = small.par, small.ctx
    l = par.L
    parts = [rand_ct(par, 2, l, 70 + r) for r in range(4)]
    sums = sum(p.astype(object) for p in parts)
    dev = torch.from_numpy(np.array(sums, dtype=np.uint64).view(np.int64)).cuda()
    ctx.reduce_sum_device(dev, l, 2, 0)
    torch.cuda.synchronize()
    got = dev.cpu().numpy().view(np.uint64)
    acc = ckks.Ct(parts[0], l, 1.0)
    for p_ in parts[1:]:
        acc = ckks.add(par, acc, ckks.Ct(p_, l, 1.0))
    assert np.array_equal(got, acc.data)


def test_full_size_ntt_keyswitch_rotate_alpha4():
    """The benchmark's parameters and digit size (N = 2^16, twenty 50-bit and
    three 60-bit primes, alpha = 4): the forward NTT of every limb against the
    oracle's transform in bit-reversed order, a top-level key switch and
    rotations at the top level and at level 1 (where InnerSum runs), each
    bit-exact against the oracle."""
    T.build()
    q, p = rns.gen_primes(50, 20), rns.gen_primes(60, 3)
    par = ckks.Params(16, q, p, 2.0 ** 50)
    ctx = T.Ctx(16, q, p, 2.0 ** 50)
    s = query.secret(par, 19, 192)
    alpha = 4
    dnum = ckks.dnum_for(par.L, alpha)
    d = synth.switch_key_draws(19, "relin", dnum, par.moduli, par.N)
    ctx.keygen_relin(s, d.a, d.e, alpha)
    rlk = ckks.relin_key(par, s, d.a, d.e, alpha)
    g = ckks.galois_for_rotation(par.N, 1)
    dr = synth.switch_key_draws(19, f"rot{g}", dnum, par.moduli, par.N)
    ctx.keygen_rotation(g, s, dr.a, dr.e, alpha)
    rk = ckks.rotation_key(par, g, s, dr.a, dr.e, alpha)
    assert np.array_equal(ctx.get_key(g, dnum), rk)
    l = par.L
    a = rand_ct(par, 1, l, 7)
    got = ctx.op(T.OP_NTT, a, l, out_comps=1)[0]
    perm = np.array([brv(k, par.log_n) for k in range(par.N)])
    for i in range(l + 1):
        x = a[0, i].copy()
        rns.lib().or_ntt(rns.ptr(x), par.N, par.q[i], par.psi[i])
        assert np.array_equal(got[0, i], x[perm]), i
    got = ctx.op(T.OP_KEYSWITCH, a, l, arg=0, out_comps=2)[0]
    assert np.array_equal(got, ckks.keyswitch(par, a[0], l, rlk, alpha))
    for lv in (l, 1):
        c = rand_ct(par, 2, lv, 70 + lv)
        got = ctx.op(T.OP_ROTATE, c, lv, arg=g, out_comps=2)[0]
        assert np.array_equal(got, ckks.rotate(par, ckks.Ct(c, lv, 1.0), g, rk, alpha).data), lv
    ctx.close()
