"""GPU parity for the PFE scoring step (Section 5.4.1): tetris_pfe_scores
equals the oracle's negacyclic rotate-and-sum residue for residue, through
host and device buffers, with exponents covering 0, N - 1, N, 2N - 1 and
values beyond 2N (taken mod 2N)."""
import numpy as np
import pytest

from oracle import pfe, rns

pytestmark = pytest.mark.gpu

T = pytest.importorskip("paper_2412_13269_gb300")


@pytest.fixture(scope="module")
def set1():
    """The paper's Set I shape: N = 2^12, one 55-bit ciphertext modulus."""
    T.build()
    q, p = rns.gen_primes(55, 1), rns.gen_primes(54, 1)
    return T.Ctx(12, q, p, 2.0 ** 40), q[0]


@pytest.mark.parametrize("m,records", [(1, 1), (5, 257), (16, 96)])
def test_pfe_scores_bit_exact(set1, m, records):
    ctx, q = set1
    n = ctx.N
    g = np.random.default_rng(m * 1000 + records)
    u = g.integers(0, q, (m, 2, n), dtype=np.uint64)
    exps = g.integers(0, 2 * n, (records, m), dtype=np.int64)
    edges = np.array([0, n - 1, n, 2 * n - 1, 1, n + 1], dtype=np.int64)
    exps.reshape(-1)[: min(edges.size, exps.size)] = edges[: min(edges.size, exps.size)]
    want = pfe.scores(u, exps, q)
    assert np.array_equal(ctx.pfe_scores(u, exps.astype(np.uint32)), want)
    # exponents are taken mod 2N
    assert np.array_equal(ctx.pfe_scores(u, (exps + 2 * n * 3).astype(np.uint32)), want)


def test_pfe_scores_device(set1):
    torch = pytest.importorskip("torch")
    ctx, q = set1
    n, m, records = ctx.N, 8, 300
    g = np.random.default_rng(5)
    u = g.integers(0, q, (m, 2, n), dtype=np.uint64)
    exps = g.integers(0, 2 * n, (records, m), dtype=np.int64)
    du = torch.from_numpy(u.view(np.int64)).cuda()
    de = torch.from_numpy(exps.astype(np.int32)).cuda()
    out = torch.empty((records, 2, n), dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    ctx.pfe_scores_device(du, de, out, m, records, stream.cuda_stream)
    stream.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint64), pfe.scores(u, exps, q))


def test_pfe_rejects_bad_sizes(set1):
    ctx, q = set1
    u = np.zeros((0, 2, ctx.N), dtype=np.uint64)
    with pytest.raises(T.TetrisError):
        ctx.pfe_scores(u, np.zeros((3, 0), dtype=np.uint32))


@pytest.fixture(scope="module")
def repack_setup():
    """N = 2^12, a 50-bit and a 40-bit prime and one 60-bit special prime,
    one-prime digits; rotation keys for Algorithm 1's Galois elements."""
    from oracle import ckks, query
    T.build()
    q, p = rns.gen_primes(50, 1) + rns.gen_primes(40, 1), rns.gen_primes(60, 1)
    par = ckks.Params(12, q, p, 2.0 ** 30)
    ctx = T.Ctx(12, q, p, 2.0 ** 30)
    s = query.secret(par, 6, 2 * par.N // 3)
    keys = query.make_keys(par, s, 6, 1, pfe.repack_galois(par.N))
    for g, k in keys.rot.items():
        ctx.load_rotation_key(g, k, 1)
    return par, ctx, s, keys


@pytest.mark.parametrize("count", [4096, 1000])
def test_repack_bit_exact(repack_setup, count):
    """Algorithm 1 on the GPU (each round one batch of t ciphertexts) equals the oracle."""
    from oracle import ckks
    par, ctx, s, keys = repack_setup
    g = np.random.default_rng(count)
    level = par.L
    data = np.stack([np.stack([np.stack([g.integers(0, q, par.N, dtype=np.uint64) for q in par.q])
                               for _ in range(2)]) for _ in range(count)])
    want = pfe.repack(par, [ckks.Ct(d, level, par.scale) for d in data], keys.rot, 1)
    got, lev, sc = ctx.repack(data, level, par.scale)
    assert lev == level and sc == par.scale
    assert np.array_equal(got, want.data)
    if count == 1000:
        torch = pytest.importorskip("torch")
        dc = torch.from_numpy(data.view(np.int64)).cuda()
        out = torch.empty((2, level + 1, par.N), dtype=torch.int64, device="cuda")
        stream = torch.cuda.current_stream()
        ctx.repack_device(dc, count, level, par.scale, out, stream.cuda_stream)
        stream.synchronize()
        assert np.array_equal(out.cpu().numpy().view(np.uint64), want.data)


def test_repack_needs_its_keys():
    T.build()
    q, p = rns.gen_primes(50, 1) + rns.gen_primes(40, 1), rns.gen_primes(60, 1)
    ctx = T.Ctx(12, q, p, 2.0 ** 30)
    with pytest.raises(T.TetrisError):
        ctx.repack(np.zeros((4, 2, 2, ctx.N), dtype=np.uint64), 1, 2.0 ** 30)
    ctx.close()
