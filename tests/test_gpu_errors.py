"""Failure detection without a GPU fault: malformed inputs are refused on the
host before anything is launched, the error is reported as a status with a
message, and the context stays usable with its state unchanged.

* short, oversized, null and out-of-range key buffers, a bad digit size and
  an even Galois element: refused, the keys already loaded still work;
* a rescale at level 0 (level underflow), a query whose coefficients are not
  fresh top-level ciphertexts (scale mismatch) and a query deeper than the
  chain: refused with TETRIS_ELEVEL / TETRIS_EINVAL;
* serving: a queued query withdrawn by tetris_cancel never runs (its ticket
  becomes unknown), a finished one's result is dropped, and the other
  queries still return exactly their alone results."""
import time

import numpy as np
import pytest

import synth
from oracle import ckks, query, rns

pytestmark = pytest.mark.gpu

T = pytest.importorskip("paper_2412_13269_gb300")


@pytest.fixture(scope="module")
def setup():
    T.build()
    q = rns.gen_primes(50, 1) + rns.gen_primes(40, 11)
    p = rns.gen_primes(60, 1)
    par = ckks.Params(12, q, p, 2.0 ** 40)
    s = query.secret(par, 13, 2 * par.N // 3)
    keys = query.make_keys(par, s, 13, 1, query.innersum_galois(par))
    ctx = T.Ctx(12, q, p, 2.0 ** 40)
    ctx.load_relin_key(keys.rlk, 1)
    for g, k in keys.rot.items():
        ctx.load_rotation_key(g, k, 1)
    yield par, s, keys, ctx
    ctx.close()


def relin_matches_oracle(par, s, keys, ctx):
    g = np.random.default_rng(1)
    d = synth.encryption_draws(1, "err", par.q, par.N)
    a = ckks.encrypt(par, ckks.encode_int(par.N, g.uniform(-1, 1, par.n_slots), par.scale), s, d.a, d.e, par.L,
                     par.scale)
    t = ckks.tensor(par, a, a)
    got = ctx.op(T.OP_RELIN, t.data, par.L, out_comps=2)[0]
    return np.array_equal(got, ckks.relinearize(par, t, keys.rlk, 1).data)


def test_malformed_keys_are_refused_and_keys_kept(setup):
    par, s, keys, ctx = setup
    rlk = keys.rlk
    for bad, msg in [(rlk.reshape(-1)[:-1], "wrong size"), (np.concatenate([rlk.reshape(-1), rlk.reshape(-1)[:8]]), "wrong size")]:
        with pytest.raises(T.TetrisError, match=msg):
            ctx.load_relin_key(bad, 1)
    # a digit size the key was not made for: refused before the loaded keys are dropped
    with pytest.raises(T.TetrisError, match="wrong size"):
        ctx.load_relin_key(rlk, 2)
    assert ctx.get_option(T.OPT_KS_ALPHA) == 1
    for alpha in (0, 5):
        with pytest.raises(T.TetrisError, match="alpha"):
            ctx.load_relin_key(rlk, alpha)
    bad = rlk.copy()
    bad[0, 1, 3, 17] = par.moduli[3]            # a residue equal to its prime
    with pytest.raises(T.TetrisError, match="out of range"):
        ctx.load_relin_key(bad, 1)
    g = next(iter(keys.rot))
    with pytest.raises(T.TetrisError, match="odd"):
        ctx.load_rotation_key(g + 1, keys.rot[g], 1)
    rc = T.lib().tetris_load_relin_key(ctx.h, None, rlk.size, 1)
    assert rc == -1 and b"null" in T.lib().tetris_last_error()
    # the context kept its keys: the relinearisation key still gives the oracle's result
    assert relin_matches_oracle(par, s, keys, ctx)
    assert np.array_equal(ctx.get_key(0, rlk.shape[0]), rlk)


def test_level_and_scale_errors(setup):
    par, s, keys, ctx = setup
    a = np.zeros((2, 1, par.N), dtype=np.uint64)
    with pytest.raises(T.TetrisError, match="ELEVEL"):
        ctx.op(T.OP_RESCALE, a, 0)
    db = ctx.upload_database(synth.database(synth.stream(2, "db"), 2048, 4))
    qv = synth.query_values(synth.stream(2, "qv"), 4, 3)
    eq = query.encrypt_query(par, s, qv, 2)
    w = [c.data for c in eq.w]
    good = [(c.level, c.scale) for c in eq.w]
    c = [x.data for x in eq.c]
    cm = [(x.level, x.scale) for x in eq.c]
    stages = np.array([query.F3])
    bad = [(lv, sc * 2) for lv, sc in good]      # not the fresh scale Delta
    with pytest.raises(T.TetrisError, match="fresh top-level"):
        ctx.evaluate_query(db, w, bad, c, cm, eq.t.data, (eq.t.level, eq.t.scale), stages)
    with pytest.raises(T.TetrisError, match="ELEVEL"):  # 3 + 5 stages: deeper than the 12-prime chain
        ctx.evaluate_query(db, w, good, c, cm, eq.t.data, (eq.t.level, eq.t.scale), np.array([query.F3] * 5))
    got, lev, sc = ctx.evaluate_query(db, w, good, c, cm, eq.t.data, (eq.t.level, eq.t.scale), stages)
    want = query.evaluate_query(par, keys, query.QueryShape(2048, 4, 3, [query.F3]),
                                query.encode_database(par, query.make_plan(par, query.QueryShape(2048, 4, 3, [query.F3])),
                                                      synth.database(synth.stream(2, "db"), 2048, 4)), eq)
    z = ckks.decrypt_slots(par, ckks.Ct(got.copy(), lev, sc), s).real
    assert abs(z[0] - ckks.decrypt_slots(par, want, s).real[0]) < 1e-6
    ctx.free_database(db)


def test_cancel_queued_and_running(setup):
    par, s, keys, ctx = setup
    db = ctx.upload_database(synth.database(synth.stream(3, "db"), 2048, 4))
    qs = []
    for i in range(6):
        qv = synth.query_values(synth.stream(600 + i, "qv"), 4, 7)
        qs.append(query.encrypt_query(par, s, qv, 600 + i))

    def args(eq):
        return ([x.data for x in eq.w], [(x.level, x.scale) for x in eq.w], [x.data for x in eq.c],
                [(x.level, x.scale) for x in eq.c], eq.t.data, (eq.t.level, eq.t.scale), np.array([query.F3]))

    alone = [ctx.evaluate_query(db, *args(eq))[0].copy() for eq in qs]
    ctx.serve_start(8 << 30, 1)
    tks = [ctx.submit(db, *args(eq)) for eq in qs]
    ctx.cancel(tks[4])                            # still queued behind four others: withdrawn
    with pytest.raises(T.TetrisError, match="ENOTFOUND"):
        ctx.poll(tks[4], 0)
    with pytest.raises(T.TetrisError, match="ENOTFOUND"):
        ctx.cancel(tks[4])
    for i in (0, 1, 2, 3, 5):
        assert np.array_equal(ctx.poll(tks[i], 30000)[0], alone[i]), i
    st = ctx.serve_stats()
    assert st.cancelled == 1 and st.completed == 5
    # a finished, unpolled result is dropped by cancel
    tk = ctx.submit(db, *args(qs[0]))
    for _ in range(3000):
        if ctx.serve_stats().completed == 6:
            break
        time.sleep(0.01)
    ctx.cancel(tk)
    with pytest.raises(T.TetrisError, match="ENOTFOUND"):
        ctx.poll(tk, 0)
    ctx.serve_stop()
    ctx.free_database(db)
