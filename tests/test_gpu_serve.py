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


def shape_queries(par, s, attrs, degrees, seed):
    out = []
    for i, d in enumerate(degrees):
        qv = synth.query_values(synth.stream(seed + i, "qv"), attrs, d)
        out.append((0, query.encrypt_query(par, s, qv, seed + i), [query.F3]))
    return out


def test_admission_respects_budget(setup):
    """Two query shapes whose program instances cannot coexist in the budget:
    alternating them evicts an idle instance for every switch, and the device
    bytes the server's programs hold (measured from their allocations right
    after each new instance) never exceed the budget."""
    par, s, new_ctx = setup
    ctx = new_ctx()
    db = ctx.upload_database(synth.database(synth.stream(3, "db"), 2048, 4))
    a, b = shape_queries(par, s, 4, [1, 7], 300)
    alone = [ctx.evaluate_query(db, *args(eq, st))[0].copy() for _, eq, st in (a, b)]
    sizes = []
    for _, eq, st in (a, b):          # each shape's instance, measured alone
        ctx.serve_start(8 << 30, 1)
        ctx.poll(ctx.submit(db, *args(eq, st)), 30000)
        sizes.append(ctx.serve_stats().peak_device_bytes)
        ctx.serve_stop()
    budget = max(sizes)
    assert sum(sizes) > budget
    ctx.serve_start(budget, 2)
    order = [0, 1, 0, 1, 1, 0]
    for k in order:                   # one at a time: every switch of shape evicts the other
        _, eq, st = (a, b)[k]
        got = ctx.poll(ctx.submit(db, *args(eq, st)), 30000)
        assert np.array_equal(got[0], alone[k])
    st = ctx.serve_stats()
    assert st.completed == len(order) and st.rejected == 0
    assert 0 < st.peak_device_bytes <= budget, (st.peak_device_bytes, budget)
    ctx.serve_stop()
    # a budget too small for any query is refused, and the context stays usable
    ctx.serve_start(1, 2)
    _, eq, stg = a
    tk = ctx.submit(db, *args(eq, stg))
    with pytest.raises(T.TetrisError, match="EBUSY"):
        ctx.poll(tk, 30000)
    ctx.serve_stop()
    got = ctx.evaluate_query(db, *args(eq, stg))
    assert got[1] >= 1
    ctx.close()


def test_poll_timeout_and_small_buffer(setup):
    """A poll whose deadline passes returns TETRIS_ETIMEOUT and keeps the
    ticket; a poll with an output buffer too small is refused and keeps the
    ticket too; the result is then delivered whole."""
    par, s, new_ctx = setup
    ctx = new_ctx()
    db = ctx.upload_database(synth.database(synth.stream(4, "db"), 2048, 4))
    qs = shape_queries(par, s, 4, [7] * 6, 400)
    alone = [ctx.evaluate_query(db, *args(eq, st))[0].copy() for _, eq, st in qs]
    ctx.serve_start(8 << 30, 1)       # one slot: the last ticket waits behind five queries
    tks = [ctx.submit(db, *args(eq, st)) for _, eq, st in qs]
    assert ctx.poll(tks[-1], 0) is None
    for tk, want in zip(tks[:-1], alone):
        assert np.array_equal(ctx.poll(tk, 30000)[0], want)
    with pytest.raises(T.TetrisError, match="too small"):
        ctx.poll(tks[-1], 30000, cap_words=1)
    got = ctx.poll(tks[-1], 30000)
    assert np.array_equal(got[0], alone[-1])
    with pytest.raises(T.TetrisError, match="ENOTFOUND"):
        ctx.poll(tks[-1], 0)
    ctx.serve_stop()
    ctx.close()


def test_served_requests_overlap_on_device(setup):
    """With warm instances and four slots, a burst of requests runs on the
    device at the same time (CUDA-event intervals of completed requests
    overlap), and every result equals the query evaluated alone."""
    par, s, new_ctx = setup
    ctx = new_ctx()
    db = ctx.upload_database(synth.database(synth.stream(5, "db"), 3000, 6, "paper"))
    qs = shape_queries(par, s, 6, [7] * 12, 500)
    alone = [ctx.evaluate_query(db, *args(eq, st))[0].copy() for _, eq, st in qs]
    ctx.serve_start(8 << 30, 4)
    warm = [ctx.submit(db, *args(eq, st)) for _, eq, st in qs[:4]]     # four instances of the shape
    for tk in warm:
        ctx.poll(tk, 30000)
    ctx.serve_stats(reset=True)
    tks = [ctx.submit(db, *args(eq, st)) for _, eq, st in qs]
    for tk, want in zip(tks, alone):
        assert np.array_equal(ctx.poll(tk, 30000)[0], want)
    st = ctx.serve_stats()
    assert st.completed == len(qs)
    assert st.max_admitted >= 2 and st.max_overlap >= 2, (st.max_admitted, st.max_overlap)
    ctx.serve_stop()
    ctx.close()
