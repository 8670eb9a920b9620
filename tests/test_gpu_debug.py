"""Debug checks that stand in for a memory sanitizer (compute-sanitizer is
closed on this pool): with TETRIS_OPT_DEBUG_CHECKS every device range each
recorded kernel job will touch is checked on the host against the live
allocations before anything is launched, and with TETRIS_GUARD_WORDS every
device buffer is framed by guard words that tetris_debug_check reads back.

A whole query (batched and plain forms) and the single operations run with
both on: results stay bit-exact with the oracle, the bounds check has
verified ranges and found none outside, no guard word changed; a guard word
overwritten on purpose (an in-bounds write inside the guard) is reported."""
import numpy as np
import pytest

from oracle import ckks, query, rns

pytestmark = pytest.mark.gpu

T = pytest.importorskip("paper_2412_13269_gb300")


def test_bounds_checks_and_guard_words(monkeypatch):
    from test_gpu_query import gpu_query, make_case, upload_encoded
    monkeypatch.setenv("TETRIS_GUARD_WORDS", "1")
    T.build()
    q = rns.gen_primes(50, 1) + rns.gen_primes(40, 11)
    p = rns.gen_primes(60, 1)
    par = ckks.Params(12, q, p, 2.0 ** 40)
    ctx = T.Ctx(12, q, p, 2.0 ** 40)
    ctx.set_option(T.OPT_DEBUG_CHECKS, 1)
    assert ctx.get_option(T.OPT_DEBUG_CHECKS) == 1
    s = query.secret(par, 21, 2 * par.N // 3)
    keys = query.make_keys(par, s, 21, 1, query.innersum_galois(par))
    ctx.load_relin_key(keys.rlk, 1)
    for g, k in keys.rot.items():
        ctx.load_rotation_key(g, k, 1)
    vals, qv, stages, shape, plan, db, eq = make_case(par, s, 3000, 4, 7, 1, 21)
    want = query.evaluate_query(par, keys, shape, db, eq)
    dbh = upload_encoded(ctx, par, plan, db, 3000, 4)
    for bpl in (0, 1):
        ctx.set_option(T.OPT_BLOCKS_PER_LAUNCH, bpl)
        got, lev, sc = gpu_query(ctx, dbh, eq, stages)
        assert lev == want.level and np.array_equal(got, want.data), bpl
    # single operations: rotation (automorphism + key switch) and relinearisation
    g = next(iter(keys.rot))
    a = eq.t
    rot = ctx.op(T.OP_ROTATE, a.data, a.level, arg=g, out_comps=2)[0]
    assert np.array_equal(rot, ckks.rotate(par, a, g, keys.rot[g], 1).data)
    checked = ctx.debug_check()
    assert checked > 1000
    with pytest.raises(T.TetrisError, match="guard words overwritten"):
        ctx.debug_check(plant=True)
    ctx.close()
