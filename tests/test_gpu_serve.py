"""Serving (tetris_serve_start / tetris_submit / tetris_poll): queries of
different shapes over different databases, submitted from several threads
while others run, each return exactly the ciphertext the same query returns
when evaluated alone; memory-based admission keeps the device footprint
within the budget; a query that cannot fit is refused."""
import random
import threading
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
    s = query.secret(par, 9, 2 * par.N // 3)
    keys = query.make_keys(par, s, 9, 1, query.innersum_galois(par))

    def new_ctx():
        ctx = T.Ctx(12, q, p, 2.0 ** 40)
        ctx.load_relin_key(keys.rlk, 1)
        for g, k in keys.rot.items():
            ctx.load_rotation_key(g, k, 1)
        return ctx

    return par, s, new_ctx


def make_queries(par, s, n, attrs_of):
    out = []
    rnd = random.Random(3)
    for i in range(n):
        db_i = rnd.randrange(len(attrs_of))
        degree = rnd.choice([1, 3, 7])
        qv = synth.query_values(synth.stream(100 + i, "qv"), attrs_of[db_i], degree)
        eq = query.encrypt_query(par, s, qv, 100 + i)
        out.append((db_i, eq, [query.F3]))
    return out


def args(eq, stages):
    return ([c.data for c in eq.w], [(c.level, c.scale) for c in eq.w], [c.data for c in eq.c],
            [(c.level, c.scale) for c in eq.c], eq.t.data, (eq.t.level, eq.t.scale), np.array(stages))


def test_served_results_equal_alone(setup):
    par, s, new_ctx = setup
    ctx = new_ctx()
    dbs = [ctx.upload_database(synth.database(synth.stream(1, "db"), 2048, 4)),
           ctx.upload_database(synth.database(synth.stream(2, "db"), 3000, 6, "paper"))]
    qs = make_queries(par, s, 12, [4, 6])
    alone = [ctx.evaluate_query(dbs[d], *args(eq, st))[0].copy() for d, eq, st in qs]
    ctx.serve_start(8 << 30, 4)
    tickets = [None] * len(qs)

    def client(idx):
        for i in idx:
            time.sleep(random.random() * 0.01)
            d, eq, st = qs[i]
            tickets[i] = ctx.submit(dbs[d], *args(eq, st))

    ths = [threading.Thread(target=client, args=(list(range(k, len(qs), 3)),)) for k in range(3)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    for i, tk in enumerate(tickets):
        got, lev, sc = ctx.poll(tk, 30000)
        assert np.array_equal(got, alone[i]), i
    st = ctx.serve_stats()
    assert st.completed == len(qs) and st.rejected == 0 and 0 < st.p50_ms <= st.p99_ms
    ctx.serve_stop()
    ctx.close()


def test_admission_respects_budget(setup):
    par, s, new_ctx = setup
    ctx = new_ctx()
    db = ctx.upload_database(synth.database(synth.stream(3, "db"), 2048, 4))
    qs = make_queries(par, s, 4, [4])
    # size one instance of each shape alone, then serve with room for roughly one
    ctx.serve_start(8 << 30, 4)
    sizes = []
    for d, eq, st in qs:
        ctx.poll(ctx.submit(db, *args(eq, st)), 30000)
    big = ctx.serve_stats().peak_device_bytes
    ctx.serve_stop()
    ctx.serve_start(big, 4)
    tks = [ctx.submit(db, *args(eq, st)) for d, eq, st in qs * 2]
    for tk in tks:
        assert ctx.poll(tk, 30000) is not None
    st = ctx.serve_stats()
    assert st.completed == len(tks) and st.peak_device_bytes <= big
    ctx.serve_stop()
    # a budget too small for any query is refused, and the context stays usable
    ctx.serve_start(1, 2)
    d, eq, stg = qs[0]
    tk = ctx.submit(db, *args(eq, stg))
    with pytest.raises(T.TetrisError, match="EBUSY"):
        ctx.poll(tk, 30000)
    ctx.serve_stop()
    got = ctx.evaluate_query(db, *args(eq, stg))
    assert got[1] >= 1
    ctx.close()
