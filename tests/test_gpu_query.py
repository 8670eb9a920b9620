"""GPU parity for the whole encrypted query: the CUDA path's output ciphertext
equals the oracle's residue for residue (given the oracle's encoded database),
in batched and plain forms, replayed as a CUDA graph or launched directly,
through host or device buffers; and the decrypted count matches the FP64
plaintext pipeline at the full benchmark size."""
import numpy as np
import pytest

import synth
from oracle import ckks, query, rns

pytestmark = pytest.mark.gpu

T = pytest.importorskip("paper_2412_13269_gb300")


class Chain:
    """Test-only chain at N = 2^12: a 50-bit q_0, n40 primes of 40 bits, one
    60-bit special prime, Delta = 2^40, one-prime digits."""

    def __init__(self, n40=11, seed=5, base2=0):
        T.build()
        q = rns.gen_primes(50, 1) + rns.gen_primes(40, n40)
        p = rns.gen_primes(60, 1)
        self.par = ckks.Params(12, q, p, 2.0 ** 40)
        self.ctx = T.Ctx(12, q, p, 2.0 ** 40)
        self.ctx.set_option(T.OPT_KS_BASE2, base2)
        self.alpha = 1
        self.s = query.secret(self.par, seed, 2 * self.par.N // 3)
        self.keys = query.make_keys(self.par, self.s, seed, 1, query.innersum_galois(self.par), base2)
        self.ctx.load_relin_key(self.keys.rlk, 1)
        for g, k in self.keys.rot.items():
            self.ctx.load_rotation_key(g, k, 1)


@pytest.fixture(scope="module")
def chain():
    return Chain()


def make_case(par, s, records, attrs, degree, nst, seed, dist="uniform"):
    vals = synth.database(synth.stream(seed, "db"), records, attrs, dist)
    qv = synth.query_values(synth.stream(seed, "qv"), attrs, degree)
    stages = [query.F3] * nst
    shape = query.QueryShape(records, attrs, degree, stages)
    plan = query.make_plan(par, shape)
    db = query.encode_database(par, plan, vals)
    eq = query.encrypt_query(par, s, qv, seed)
    return vals, qv, stages, shape, plan, db, eq


def upload_encoded(ctx, par, plan, db, records, attrs):
    coeffs = np.stack([np.stack(blk) for blk in db.pts])
    mask = None
    if plan.ragged:
        live = records - (len(db.pts) - 1) * par.n_slots
        z = np.zeros(par.n_slots)
        z[:live] = 1.0
        mask = ckks.encode_real(par.N, z, 1.0)
    return ctx.upload_database_encoded(coeffs, mask, records, attrs)


def gpu_query(ctx, dbh, eq, stages):
    w = [c.data for c in eq.w]
    c = [x.data for x in eq.c]
    return ctx.evaluate_query(dbh, w, [(x.level, x.scale) for x in eq.w], c, [(x.level, x.scale) for x in eq.c],
                              eq.t.data, (eq.t.level, eq.t.scale), np.array(stages))


@pytest.mark.parametrize("records,attrs,degree,nst", [(2048, 8, 7, 1), (1500, 4, 3, 1), (3000, 3, 2, 1),
                                                     (2048, 4, 12, 1), (2048, 4, 15, 1),
                                                     # degenerate shapes: one record and one attribute with a
                                                     # linear f; a second block holding a single record; one
                                                     # attribute filling exactly one block
                                                     (1, 1, 1, 1), (2049, 2, 1, 2), (2048, 1, 2, 1)])
def test_query_bit_exact(chain, records, attrs, degree, nst):
    par, ctx = chain.par, chain.ctx
    vals, qv, stages, shape, plan, db, eq = make_case(par, chain.s, records, attrs, degree, nst, records)
    want = query.evaluate_query(par, chain.keys, shape, db, eq)
    dbh = upload_encoded(ctx, par, plan, db, records, attrs)
    for bpl, graph in [(0, 1), (1, 0), (0, 0), (1, 1)]:
        ctx.set_option(T.OPT_BLOCKS_PER_LAUNCH, bpl)
        ctx.set_option(T.OPT_USE_GRAPH, graph)
        got, lev, sc = gpu_query(ctx, dbh, eq, stages)
        assert lev == want.level == plan.l_ret
        assert np.array_equal(got, want.data), (bpl, graph)
        assert sc == plan.S[plan.l_out]
    ctx.set_option(T.OPT_BLOCKS_PER_LAUNCH, 0)
    ctx.set_option(T.OPT_USE_GRAPH, 1)
    # decrypts to the FP64 pipeline's normalised count in every slot
    z = ckks.decrypt_slots(par, ckks.Ct(got.copy(), lev, sc), chain.s).real
    ref = query.fp64_pipeline(vals, qv, stages)
    assert np.ptp(z) < 1e-6 and abs(z[0] * records - ref.count) < 0.05
    ctx.free_database(dbh)


def test_query_base2_bit_exact():
    """The whole query with the base-2^w key switch (w = 30, Table 1's Set I)."""
    ch = Chain(n40=9, seed=6, base2=30)
    par, ctx = ch.par, ch.ctx
    vals, qv, stages, shape, plan, db, eq = make_case(par, ch.s, 2048, 4, 7, 1, 77)
    want = query.evaluate_query(par, ch.keys, shape, db, eq)
    dbh = upload_encoded(ctx, par, plan, db, 2048, 4)
    got, lev, sc = gpu_query(ctx, dbh, eq, stages)
    assert lev == want.level and np.array_equal(got, want.data)
    z = ckks.decrypt_slots(par, ckks.Ct(got.copy(), lev, sc), ch.s).real
    ref = query.fp64_pipeline(vals, qv, stages)
    assert abs(z[0] * 2048 - ref.count) < 0.05
    ctx.free_database(dbh)
    ctx.close()


def test_autotune_keeps_results(chain):
    par, ctx = chain.par, chain.ctx
    vals, qv, stages, shape, plan, db, eq = make_case(par, chain.s, 3000, 3, 2, 1, 3000)
    want = query.evaluate_query(par, chain.keys, shape, db, eq)
    dbh = upload_encoded(ctx, par, plan, db, 3000, 3)
    a = ([c.data for c in eq.w], [(c.level, c.scale) for c in eq.w], [c.data for c in eq.c],
         [(c.level, c.scale) for c in eq.c], eq.t.data, (eq.t.level, eq.t.scale), np.array(stages))
    table = ctx.autotune(dbh, *a, reps=2)
    assert sorted((b, g) for b, g, _, p in table) == [(0, 3), (0, 4), (1, 3), (1, 4)]
    assert not any(p for *_, p in table)   # persistent launches take log N >= 14
    best = min(table, key=lambda e: e[2])
    assert (ctx.get_option(T.OPT_BLOCKS_PER_LAUNCH), ctx.get_option(T.OPT_NTT_GROUP)) == best[:2]
    for grp in (3, 4):
        ctx.set_option(T.OPT_NTT_GROUP, grp)
        assert np.array_equal(ctx.evaluate_query(dbh, *a)[0], want.data), grp
    ctx.set_option(T.OPT_NTT_GROUP, 3)
    ctx.set_option(T.OPT_BLOCKS_PER_LAUNCH, 0)
    ctx.free_database(dbh)


def test_partition_normalisation_bit_exact(chain):
    """A partition of a larger database normalised by the total record count
    (the horizontally partitioned database of Section 5.6)."""
    par, ctx = chain.par, chain.ctx
    vals = synth.database(synth.stream(41, "db"), 2048, 4)
    qv = synth.query_values(synth.stream(41, "qv"), 4, 3)
    shape = query.QueryShape(2048, 4, 3, [query.F3], norm_records=6144)
    plan = query.make_plan(par, shape)
    db = query.encode_database(par, plan, vals)
    eq = query.encrypt_query(par, chain.s, qv, 41)
    want = query.evaluate_query(par, chain.keys, shape, db, eq)
    dbh = upload_encoded(ctx, par, plan, db, 2048, 4)
    got = ctx.evaluate_query(dbh, *[v for v in (
        [c.data for c in eq.w], [(c.level, c.scale) for c in eq.w], [c.data for c in eq.c],
        [(c.level, c.scale) for c in eq.c], eq.t.data, (eq.t.level, eq.t.scale), np.array([query.F3]))],
        total_records=6144)[0]
    assert np.array_equal(got, want.data)
    ctx.free_database(dbh)


def test_device_buffers_match_host(chain):
    torch = pytest.importorskip("torch")
    par, ctx = chain.par, chain.ctx
    vals, qv, stages, shape, plan, db, eq = make_case(par, chain.s, 2048, 8, 7, 1, 77)
    dbh = upload_encoded(ctx, par, plan, db, 2048, 8)
    host, lev, sc = gpu_query(ctx, dbh, eq, stages)
    dev = lambda a: torch.from_numpy(a.view(np.int64).copy()).cuda()
    w = [dev(c.data) for c in eq.w]
    c = [dev(x.data) for x in eq.c]
    t = dev(eq.t.data)
    out = torch.empty(2 * (par.L + 1) * par.N, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    lev2, sc2 = ctx.evaluate_query_device(dbh, w, [(x.level, x.scale) for x in eq.w], c, [(x.level, x.scale) for x in eq.c],
                                          t, (eq.t.level, eq.t.scale), np.array(stages), out, stream.cuda_stream)
    stream.synchronize()
    got = out.cpu().numpy().view(np.uint64)[: host.size].reshape(host.shape)
    assert lev2 == lev and np.array_equal(got, host)
    ctx.free_database(dbh)


def test_gpu_encoded_database_decrypts_to_fp64(chain):
    par, ctx = chain.par, chain.ctx
    vals, qv, stages, shape, plan, db, eq = make_case(par, chain.s, 1800, 6, 5, 1, 31, "paper")
    dbh = ctx.upload_database(vals)
    got, lev, sc = gpu_query(ctx, dbh, eq, stages)
    z = ckks.decrypt_slots(par, ckks.Ct(got.copy(), lev, sc), chain.s).real
    ref = query.fp64_pipeline(vals, qv, stages)
    assert abs(z[0] * 1800 - ref.count) < 0.05
    ctx.free_database(dbh)


def test_plan_counts(chain):
    par, ctx = chain.par, chain.ctx
    vals = synth.database(synth.stream(1, "db"), 2048, 8)
    dbh = ctx.upload_database(vals)
    info = ctx.plan(dbh, 7, 1)
    p = query.make_plan(par, query.QueryShape(2048, 8, 7, [query.F3]))
    assert (info.l_lin, info.l_d, info.l_y, info.l_u, info.l_out) == (p.l_lin, p.l_d, p.l_y, p.l_u, p.l_out)
    assert info.l_ret == p.l_ret == 1
    assert info.rotations == par.log_n - 1 and info.relins > 0 and info.kernel_launches > 0
    assert info.pt_scale == p.pt_scale
    ctx.free_database(dbh)


def test_empty_database_refused(chain):
    with pytest.raises(T.TetrisError):
        chain.ctx.upload_database(np.zeros((0, 4), dtype=np.uint8))


def test_errors_leave_context_usable(chain):
    ctx = chain.ctx
    with pytest.raises(T.TetrisError):
        ctx.free_database(12345)
    with pytest.raises(T.TetrisError):
        ctx.op(T.OP_ROTATE, np.zeros((2, 1, ctx.N), dtype=np.uint64), 0, arg=7)   # no key for 7
    a = np.zeros((2, 1, ctx.N), dtype=np.uint64)
    got = ctx.op(T.OP_ADD, a, 0, b=a, b_level=0, out_comps=2)[0]
    assert not got.any()


@pytest.fixture(scope="module")
def full():
    """The benchmark's parameters: N = 2^16, twenty 50-bit primes, three 60-bit special primes, Delta = 2^50, alpha = 4."""
    T.build()
    q, p = rns.gen_primes(50, 20), rns.gen_primes(60, 3)
    par = ckks.Params(16, q, p, 2.0 ** 50)
    ctx = T.Ctx(16, q, p, 2.0 ** 50)
    s = query.secret(par, 8, 192)
    keys = query.make_keys(par, s, 8, 4, query.innersum_galois(par))
    ctx.load_relin_key(keys.rlk, 4)
    for g, k in keys.rot.items():
        ctx.load_rotation_key(g, k, 4)
    return par, ctx, s, keys


def test_full_size_one_block_bit_exact(full):
    par, ctx, s, keys = full
    vals, qv, stages, shape, plan, db, eq = make_case(par, s, 32768, 16, 15, 3, 4, "mixed")
    want = query.evaluate_query(par, keys, shape, db, eq)
    dbh = upload_encoded(ctx, par, plan, db, 32768, 16)
    got, lev, sc = gpu_query(ctx, dbh, eq, stages)
    assert lev == want.level and np.array_equal(got, want.data)
    # persistent launches (resident CTAs walking every limb's tiles) give the same residues
    ctx.set_option(T.OPT_PERSISTENT, 1)
    got, lev, sc = gpu_query(ctx, dbh, eq, stages)
    ctx.set_option(T.OPT_PERSISTENT, 0)
    assert lev == want.level and np.array_equal(got, want.data)
    ctx.free_database(dbh)


def test_full_size_benchmark_workload_decrypts(full):
    """131072 records x 16 attributes (four blocks, as timed by the benchmark): decrypted count vs FP64."""
    par, ctx, s, keys = full
    vals, qv, stages, shape, plan, db, eq = make_case(par, s, 131072, 16, 15, 3, 6, "mixed")
    dbh = ctx.upload_database(vals)
    got, lev, sc = gpu_query(ctx, dbh, eq, stages)
    z = ckks.decrypt_slots(par, ckks.Ct(got.copy(), lev, sc), s).real
    ref = query.fp64_pipeline(vals, qv, stages)
    assert np.ptp(z) < 1e-6
    assert abs(z[0] * 131072 - ref.count) < 0.5
    ctx.free_database(dbh)


@pytest.fixture(scope="module")
def deep():
    """Test-only chain with 18 primes of 40 bits after q_0: room for 3 local and 2 global sign stages."""
    return Chain(n40=18, seed=9)


@pytest.mark.parametrize("p_pos,t1_frac", [(0.9, 0.2), (0.1, 0.8)])
def test_global_threshold_bit_exact(deep, p_pos, t1_frac):
    """Algorithm 2's last line (step((count - t1 + 1/2) / R)) after InnerSum:
    residues equal the oracle's; the decrypted bit is exact."""
    from test_oracle_query import skewed_margin_dataset
    par, ctx = deep.par, deep.ctx
    stages, gstages = [query.F3] * 3, [query.F3] * 2
    R = 2048
    vals, w, side = skewed_margin_dataset(R, 8, 23, p_pos)
    qv = synth.QueryValues(w=w, c=np.array([0.0, 1.0]), t=0.0, t1=float(int(t1_frac * R)))
    shape = query.QueryShape(R, 8, 1, stages, global_stages=gstages)
    plan = query.make_plan(par, shape)
    db = query.encode_database(par, plan, vals)
    eq = query.encrypt_query(par, deep.s, qv, 23)
    want = query.evaluate_query(par, deep.keys, shape, db, eq)
    dbh = upload_encoded(ctx, par, plan, db, R, 8)
    for bpl in (0, 1):
        ctx.set_option(T.OPT_BLOCKS_PER_LAUNCH, bpl)
        got, lev, sc = ctx.evaluate_query(dbh, [c.data for c in eq.w], [(c.level, c.scale) for c in eq.w],
                                          [c.data for c in eq.c], [(c.level, c.scale) for c in eq.c], eq.t.data,
                                          (eq.t.level, eq.t.scale), np.array(stages),
                                          glob=(eq.t1.data, (eq.t1.level, eq.t1.scale), np.array(gstages)))
        assert lev == want.level == plan.l_ret and sc == plan.S[plan.l_ret]
        assert np.array_equal(got, want.data), bpl
    ctx.set_option(T.OPT_BLOCKS_PER_LAUNCH, 0)
    bit = ckks.decrypt_slots(par, ckks.Ct(got.copy(), lev, sc), deep.s).real
    assert np.max(np.abs(bit - (1 if p_pos > 0.5 else 0))) < 2.0 ** -12
    ctx.free_database(dbh)


@pytest.fixture(scope="module")
def chain15():
    """Test-only chain with 15 primes of 40 bits after q_0: three degree-15 stages."""
    return Chain(n40=15, seed=12)


def test_degree15_minimax_stages_bit_exact(chain15):
    """Three degree-15 minimax stages (alpha = 8, the stored Remez coefficients):
    residues equal the oracle's; the count is exact for records within 2^-7.4 of
    the threshold."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "minimax_sign.json")) as f:
        stages = np.array(json.load(f)["alpha8_15x3"]["stages"])
    par, ctx = chain15.par, chain15.ctx
    R = 2048
    v = np.random.default_rng(22).integers(0, 254, R)
    vals = np.where(v >= 127, v + 2, v).astype(np.uint8)[:, None]
    qv = synth.QueryValues(w=np.array([1.0]), c=np.array([0.0, 1.0]), t=0.0)
    shape = query.QueryShape(R, 1, 1, [list(s) for s in stages])
    plan = query.make_plan(par, shape)
    db = query.encode_database(par, plan, vals)
    eq = query.encrypt_query(par, chain15.s, qv, 22)
    want = query.evaluate_query(par, chain15.keys, shape, db, eq)
    dbh = upload_encoded(ctx, par, plan, db, R, 1)
    got, lev, sc = gpu_query(ctx, dbh, eq, stages)
    assert lev == want.level and np.array_equal(got, want.data)
    z = ckks.decrypt_slots(par, ckks.Ct(got.copy(), lev, sc), chain15.s).real
    assert int(np.rint(z[0] * R)) == int((vals[:, 0] > 128).sum())
    ctx.free_database(dbh)


STAGES = [(1, "x"), (2, "y"), (3, "d"), (4, "u")]   # TETRIS_STAGE_X .. TETRIS_STAGE_U


def check_stages(par, ctx, s, keys, vals, qv, stages, seed, bpls=(0,)):
    """Every stage of every block (TETRIS_OPT_QUERY_STAGE): residues equal the
    oracle's stage ciphertexts, and each slot decrypts to the FP64 pipeline's
    value within 2^-12 (x, y = f(x), y - t, and the step values u, which
    leave the block divided by the record count)."""
    records, attrs = vals.shape
    degree = len(qv.c) - 1
    shape = query.QueryShape(records, attrs, degree, stages)
    plan = query.make_plan(par, shape)
    db = query.encode_database(par, plan, vals)
    eq = query.encrypt_query(par, s, qv, seed)
    ev = query.Evaluator(par, keys, plan)
    ck, tadj = ev.per_query(eq, degree)
    recs = []
    for b in range(len(db.pts)):
        rec = {}
        ev.block(db.pts[b], eq, ck, tadj, degree, record=rec)
        recs.append(rec)
    ref = query.fp64_pipeline(vals, qv, stages)
    want_vals = {"x": ref.x, "y": ref.y, "d": ref.y - qv.t, "u": ref.u}
    dbh = upload_encoded(ctx, par, plan, db, records, attrs)
    args = ([c.data for c in eq.w], [(c.level, c.scale) for c in eq.w], [c.data for c in eq.c],
            [(c.level, c.scale) for c in eq.c], eq.t.data, (eq.t.level, eq.t.scale), np.array(stages))
    n, B = par.n_slots, len(db.pts)
    worst = {}
    for bpl in bpls:
        ctx.set_option(T.OPT_BLOCKS_PER_LAUNCH, bpl)
        for stage, name in STAGES:
            got, lev, sc = ctx.query_stage(stage, B, dbh, *args)
            for b in range(B):
                want = recs[b][name]
                assert lev == want.level and sc == want.scale, (name, b)
                assert np.array_equal(got[b], want.data), (bpl, name, b)
                lo, hi = b * n, min(records, (b + 1) * n)
                dec = ckks.decrypt_slots(par, ckks.Ct(got[b].copy(), lev, sc), s).real[: hi - lo]
                if name == "u":
                    dec = dec * plan.records_norm
                err = float(np.max(np.abs(dec - want_vals[name][lo:hi])))
                worst[name] = max(worst.get(name, 0.0), err)
                assert err <= 2.0 ** -12, (name, b, err)
    ctx.set_option(T.OPT_BLOCKS_PER_LAUNCH, 0)
    ctx.free_database(dbh)
    return worst


@pytest.mark.parametrize("records,attrs,degree,nst", [(2048, 8, 7, 1), (3000, 3, 2, 1)])
def test_stage_outputs_bit_exact_per_slot(chain, records, attrs, degree, nst):
    vals = synth.database(synth.stream(50 + degree, "db"), records, attrs)
    qv = synth.query_values(synth.stream(50 + degree, "qv"), attrs, degree)
    check_stages(chain.par, chain.ctx, chain.s, chain.keys, vals, qv, [query.F3] * nst, 50 + degree, bpls=(0, 1))


def test_full_size_stage_outputs_bit_exact_per_slot(full):
    """One 32768-record block of the benchmark workload (degree 15, three f3
    stages, alpha 4): every stage bit-exact and within 2^-12 per slot."""
    par, ctx, s, keys = full
    vals = synth.database(synth.stream(52, "db"), 32768, 16, "mixed")
    qv = synth.query_values(synth.stream(52, "qv"), 16, 15)
    check_stages(par, ctx, s, keys, vals, qv, [query.F3] * 3, 52)
