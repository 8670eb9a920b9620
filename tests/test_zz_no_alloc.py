"""The allocation-free rescale (tetris_rescale_ntt_noalloc) is for callers
that cannot let the library allocate device memory behind their back: a
serving process or another framework that has already reserved the GPU with
its own caching allocator (where cudaMalloc fails or fragments), or a caller
that cannot afford the device-wide synchronisation of cudaFree.  It takes
caller-owned device buffers and keeps its scratch in one fixed array inside
the library.

Checked here on two calls in a row that share that scratch:
  * each result equals what the existing entry points return (TETRIS_OP_RESCALE
    on the coefficient-domain input, brought to the NTT order by TETRIS_OP_NTT)
    and what the oracle's rescale gives (Section 2.5's rounded division by q_l),
    in the same NTT order;
  * a call allocates nothing: the context's held device bytes and the
    device's free memory are the same before and after it;
  * sizes beyond the fixed scratch and host pointers are refused with a clear
    error before any launch.

This file is collected last, so a run that stops at the first failure has
already run every other test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

T = pytest.importorskip("paper_2412_13269_gb300")
torch = pytest.importorskip("torch")

from oracle import ckks  # noqa: E402


def rand_ct(q, comps, level, n, seed):
    g = np.random.default_rng(seed)
    return np.stack([np.stack([g.integers(0, m, n, dtype=np.uint64) for m in q[: level + 1]]) for _ in range(comps)])


def test_noalloc_rescale_matches_rescale_on_two_calls():
    T.build()
    q = T.gen_primes(50, 20)
    p = T.gen_primes(60, 3, exclude=q)
    ctx = T.Ctx(16, q, p, 2.0 ** 50)
    par = ckks.Params(16, q, p, 2.0 ** 50)
    n = ctx.N
    stream = torch.cuda.current_stream()
    assert T.lib().tetris_noalloc_scratch_bytes() >= 3 * n * 8
    cases = [(19, 3), (7, 2)]
    # references first (the ordinary entry points allocate), device buffers next
    refs, bufs = [], []
    for call, (level, comps) in enumerate(cases):
        a = rand_ct(q, comps, level, n, 100 + call)
        a_ntt = ctx.op(T.OP_NTT, a, level, out_comps=comps)[0]
        want_coef = ctx.op(T.OP_RESCALE, a, level)[0]
        oracle_coef = ckks.rescale(par, ckks.Ct(a.copy(), level, 1.0)).data
        assert np.array_equal(want_coef, oracle_coef), call
        want = ctx.op(T.OP_NTT, want_coef, level - 1, out_comps=comps)[0]
        refs.append(want)
        src = torch.from_numpy(a_ntt.view(np.int64).copy()).cuda()
        dst = torch.full((comps * level * n,), -1, dtype=torch.int64, device="cuda")
        bufs.append((src, dst))
    torch.cuda.synchronize()
    for call, ((level, comps), want, (src, dst)) in enumerate(zip(cases, refs, bufs)):
        held = ctx.info().device_bytes
        free = torch.cuda.mem_get_info()[0]
        ctx.rescale_ntt_noalloc(src, dst, level, comps, stream.cuda_stream)
        stream.synchronize()
        assert ctx.info().device_bytes == held, call
        if call > 0:  # the first call on a device may load the library's scratch array itself
            assert torch.cuda.mem_get_info()[0] == free, call
        got = dst.cpu().numpy().view(np.uint64).reshape(comps, level, n)
        assert np.array_equal(got, want), call
    # sizes beyond the fixed scratch are refused with a clear error
    src = torch.zeros(4 * 2 * n, dtype=torch.int64, device="cuda")
    dst = torch.zeros(4 * n, dtype=torch.int64, device="cuda")
    with pytest.raises(T.TetrisError, match="at most 3 components"):
        ctx.rescale_ntt_noalloc(src, dst, 1, 4, stream.cuda_stream)
    # host memory is refused before any launch
    host = np.zeros(2 * 2 * n, dtype=np.uint64)
    with pytest.raises(T.TetrisError, match="not device memory"):
        ctx.rescale_ntt_noalloc(host, dst, 1, 2, stream.cuda_stream)
    with pytest.raises(T.TetrisError, match="not device memory"):
        ctx.rescale_ntt_noalloc(src, np.zeros(2 * n, dtype=np.uint64), 1, 2, stream.cuda_stream)
    ctx.close()
