"""The allocation-free rescale (tetris_rescale_ntt_noalloc), for callers that
cannot let the library allocate device memory, returns exactly what the
ordinary rescale returns, on two calls in a row that share its fixed scratch.

It is checked against the existing entry points only: TETRIS_OP_RESCALE on
the coefficient-domain input, brought to the NTT order by TETRIS_OP_NTT."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

T = pytest.importorskip("paper_2412_13269_gb300")
torch = pytest.importorskip("torch")


def rand_ct(q, comps, level, n, seed):
    g = np.random.default_rng(seed)
    return np.stack([np.stack([g.integers(0, m, n, dtype=np.uint64) for m in q[: level + 1]]) for _ in range(comps)])


def test_noalloc_rescale_matches_rescale_on_two_calls():
    T.build()
    q = T.gen_primes(50, 20)
    p = T.gen_primes(60, 3, exclude=q)
    ctx = T.Ctx(16, q, p, 2.0 ** 50)
    n = ctx.N
    stream = torch.cuda.current_stream()
    assert T.lib().tetris_noalloc_scratch_bytes() >= 3 * n * 8
    for call, (level, comps) in enumerate([(19, 3), (7, 2)]):
        a = rand_ct(q, comps, level, n, 100 + call)
        a_ntt = ctx.op(T.OP_NTT, a, level, out_comps=comps)[0]
        want_coef = ctx.op(T.OP_RESCALE, a, level)[0]
        want = ctx.op(T.OP_NTT, want_coef, level - 1, out_comps=comps)[0]
        src = torch.from_numpy(a_ntt.view(np.int64).copy()).cuda()
        dst = torch.empty(comps * level * n, dtype=torch.int64, device="cuda")
        ctx.rescale_ntt_noalloc(src, dst, level, comps, stream.cuda_stream)
        stream.synchronize()
        got = dst.cpu().numpy().view(np.uint64).reshape(comps, level, n)
        assert np.array_equal(got, want), call
    # sizes beyond the fixed scratch are refused with a clear error
    src = torch.zeros(4 * 2 * n, dtype=torch.int64, device="cuda")
    dst = torch.zeros(4 * n, dtype=torch.int64, device="cuda")
    with pytest.raises(T.TetrisError, match="at most 3 components"):
        ctx.rescale_ntt_noalloc(src, dst, 1, 4, stream.cuda_stream)
    ctx.close()
