"""GPU parity for the PFE scoring step (Section 4.1.1): tetris_pfe_scores
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
