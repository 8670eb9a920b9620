"""Pins for the oracle's query circuit: the decrypted count matches the FP64
plaintext pipeline (same polynomials, computed in floating point without
encryption); with every record outside the sign margin (the epsilon shift of
Section 5.4.2 keeps records off the threshold) the rounded count is the exact
integer count; InnerSum leaves the total in every slot."""
import numpy as np
import pytest

import synth
from oracle import ckks, query, rns


def chain_params(n_q40: int, log_n: int = 12):
    """Test-only chain: one 50-bit q_0, n_q40 primes of 40 bits, one 60-bit special prime, Delta = 2^40."""
    q = rns.gen_primes(50, 1) + rns.gen_primes(40, n_q40)
    return ckks.Params(log_n, q, rns.gen_primes(60, 1), 2.0 ** 40)


def run(par, vals, qv, stages, seed=1, alpha=1, base2=0):
    shape = query.QueryShape(vals.shape[0], vals.shape[1], len(qv.c) - 1, stages)
    plan = query.make_plan(par, shape)
    s = query.secret(par, seed, 2 * par.N // 3)
    keys = query.make_keys(par, s, seed, alpha, query.innersum_galois(par), base2)
    db = query.encode_database(par, plan, vals)
    eq = query.encrypt_query(par, s, qv, seed)
    out = query.evaluate_query(par, keys, shape, db, eq)
    assert out.level == plan.l_ret == 1
    return ckks.decrypt_slots(par, out, s).real, plan


def test_plan_levels():
    par = chain_params(11)
    p = query.make_plan(par, query.QueryShape(2048, 8, 7, [query.F3]))
    # the circuit starts as low as its depth allows: it ends at level 1
    assert (p.l_lin, p.l_d, p.l_y, p.l_u, p.l_out) == (8, 5, 4, 1, 1)
    q2 = rns.gen_primes(50, 20)
    par2 = ckks.Params(16, q2, rns.gen_primes(60, 3), 2.0 ** 50)
    p2 = query.make_plan(par2, query.QueryShape(131072, 16, 15, [query.F3] * 3))
    assert (p2.l_lin, p2.l_d, p2.l_y, p2.l_u, p2.l_out) == (15, 11, 10, 1, 1)
    p3 = query.make_plan(par2, query.QueryShape(1 << 14, 16, 31, [query.F3] * 3))
    assert p3.ragged and (p3.l_lin, p3.l_u, p3.l_out) == (17, 2, 1)
    # the rescaled linear combination of dropped w_j: Delta pt_scale / q_{l_lin+1}, near S[l_lin]
    for pl in (p2, p3):
        t = pl.l_lin + 1
        assert pl.x_scale == (pl.S[par2.L] * pl.pt_scale) / float(par2.q[t])
        assert abs(pl.x_scale / pl.S[pl.l_lin] - 1) < 1e-3
    # no spare levels: the circuit starts right below the top
    p4 = query.make_plan(par2, query.QueryShape(131072, 16, 15, [query.F3] * 4))
    assert (p4.l_lin, p4.l_out) == (18, 1) and abs(p4.x_scale / p4.S[18] - 1) < 1e-12
    with pytest.raises(ValueError):
        query.make_plan(par, query.QueryShape(2048, 8, 31, [query.F3] * 3))
    # exact standard scales: S[l-1] q_l = S[l]^2 up to one rounding
    for l in range(1, par2.L + 1):
        assert abs(p2.S[l - 1] * par2.q[l] / p2.S[l] ** 2 - 1) < 1e-15


def test_query_matches_fp64_pipeline():
    par = chain_params(11)
    vals = synth.database(synth.stream(11, "db"), 2048, 8)
    qv = synth.query_values(synth.stream(11, "qv"), 8, 7)
    got, plan = run(par, vals, qv, [query.F3])
    ref = query.fp64_pipeline(vals, qv, [query.F3])
    R = vals.shape[0]
    # InnerSum puts the normalised count in every slot
    assert np.ptp(got) < 1e-6
    assert abs(got[0] * R - ref.count) < 0.05


def test_query_base2_matches_fp64_pipeline():
    """With the base-2^w key switch of Table 1's Set I (w = 30, one special
    prime) the whole circuit still decrypts to the FP64 pipeline's count."""
    par = chain_params(9)
    vals = synth.database(synth.stream(12, "db"), 2048, 4)
    qv = synth.query_values(synth.stream(12, "qv"), 4, 3)
    got, plan = run(par, vals, qv, [query.F3], seed=2, base2=30)
    ref = query.fp64_pipeline(vals, qv, [query.F3])
    assert np.ptp(got) < 1e-6
    assert abs(got[0] * vals.shape[0] - ref.count) < 0.05


def test_query_ragged_mask():
    par = chain_params(12)
    vals = synth.database(synth.stream(12, "db"), 1500, 4, "paper")
    qv = synth.query_values(synth.stream(12, "qv"), 4, 3)
    got, plan = run(par, vals, qv, [query.F3])
    assert plan.ragged
    ref = query.fp64_pipeline(vals, qv, [query.F3])
    assert abs(got[0] * 1500 - ref.count) < 0.05


def margin_dataset(records, attrs, seed, margin):
    """Records whose z = (x - t)/2 stays at least ``margin`` from 0 (t = 0, f(x) = x)."""
    g = np.random.default_rng(seed)
    w = g.choice([-1.0, 1.0], size=attrs)
    side = g.choice([-1.0, 1.0], size=records)
    mag = g.uniform(0.75, 1.0, size=(records, attrs))
    xh = side[:, None] * w[None, :] * mag              # normalised values in [-1, 1]
    vals = np.clip(np.rint(xh * 127.5 + 127.5), 0, 255).astype(np.uint8)
    qv = synth.QueryValues(w=w, c=np.array([0.0, 1.0, 0.0, 0.0]), t=0.0)
    return vals, qv, side


def test_exact_count_outside_margin():
    stages = [query.F3] * 3
    tol = 2.0 ** -13
    margin = query.sign_margin(stages, tol)
    vals, qv, side = margin_dataset(2048, 8, 5, margin)
    ref = query.fp64_pipeline(vals, qv, stages)
    assert np.min(np.abs(ref.z)) > margin
    par = chain_params(15)
    got, _ = run(par, vals, qv, stages)
    R = vals.shape[0]
    assert int(np.rint(got[0] * R)) == ref.exact == int((side > 0).sum())


def test_poly_schedule():
    """Baby-step giant-step choice: fewest relinearisations with y no deeper than plain powers."""
    assert all(query.poly_schedule(d) is None for d in (1, 2, 3))
    assert query.poly_schedule(7) == (4, 2, 2, 3)
    assert query.poly_schedule(8) == (4, 3, 2, 3)
    assert query.poly_schedule(12) == (4, 4, 2, 4)
    assert query.poly_schedule(15) == (4, 4, 2, 4)
    assert query.poly_schedule(31) == (8, 4, 3, 5)
    for d in range(1, 64):
        s = query.poly_schedule(d)
        if s is not None:
            g, m, bb, df = s
            assert g * (m - 1) <= d < g * m and df <= query.ceil_log2(d)


@pytest.mark.parametrize("degree,relins", [(12, 8 + 4), (15, 9 + 4), (8, 6 + 4), (3, 3 + 4)])
def test_bsgs_polynomial_matches_fp64(monkeypatch, degree, relins):
    """The polynomial (baby-step giant-step above degree 3, including a last
    block holding one coefficient) and one sign stage: the decrypted count
    matches the FP64 pipeline, and the relinearisations are the schedule's plus
    the stage's four."""
    calls = []
    real = ckks.relinearize
    monkeypatch.setattr(ckks, "relinearize", lambda *a, **k: calls.append(1) or real(*a, **k))
    par = chain_params(12)
    vals = synth.database(synth.stream(degree, "db"), 2048, 4)
    qv = synth.query_values(synth.stream(degree, "qv"), 4, degree)
    got, plan = run(par, vals, qv, [query.F3])
    ref = query.fp64_pipeline(vals, qv, [query.F3])
    assert len(calls) == relins
    assert np.ptp(got) < 1e-6
    assert abs(got[0] * 2048 - ref.count) < 0.05


def skewed_margin_dataset(records, attrs, seed, p_pos):
    """As margin_dataset, with a fraction p_pos of the records on the positive side."""
    g = np.random.default_rng(seed)
    w = g.choice([-1.0, 1.0], size=attrs)
    side = np.where(g.uniform(size=records) < p_pos, 1.0, -1.0)
    mag = g.uniform(0.75, 1.0, size=(records, attrs))
    xh = side[:, None] * w[None, :] * mag
    vals = np.clip(np.rint(xh * 127.5 + 127.5), 0, 255).astype(np.uint8)
    return vals, w, side


@pytest.mark.parametrize("p_pos,t1_frac", [(0.9, 0.2), (0.1, 0.8)])
def test_global_threshold_bit(p_pos, t1_frac):
    """Algorithm 2's last line on the count: with every record outside the
    local sign margin (exact count) and (count - t1 + 1/2)/R outside the
    global margin of two f3 stages at tolerance 2^-12, the decrypted output is
    the exact bit [count >= t1] within 2^-12 in every slot, and matches the FP64
    pipeline's value of the same polynomials."""
    stages, gstages = [query.F3] * 3, [query.F3] * 2
    R = 2048
    vals, w, side = skewed_margin_dataset(R, 8, 17, p_pos)
    t1 = float(int(t1_frac * R))
    qv = synth.QueryValues(w=w, c=np.array([0.0, 1.0]), t=0.0, t1=t1)
    par = chain_params(18)
    shape = query.QueryShape(R, 8, 1, stages, global_stages=gstages)
    plan = query.make_plan(par, shape)
    assert plan.l_ret == plan.l_out - 6 >= 1
    s = query.secret(par, 3, 2 * par.N // 3)
    keys = query.make_keys(par, s, 3, 1, query.innersum_galois(par))
    db = query.encode_database(par, plan, vals)
    eq = query.encrypt_query(par, s, qv, 3)
    out = query.evaluate_query(par, keys, shape, db, eq)
    assert out.level == plan.l_ret
    got = ckks.decrypt_slots(par, out, s).real
    ref = query.fp64_pipeline(vals, qv, stages, gstages)
    assert ref.exact == int((side > 0).sum())
    assert abs(ref.z2) > query.sign_margin(gstages, 2.0 ** -12)
    assert ref.exact_bit == int(ref.exact >= t1) == (1 if p_pos > 0.5 else 0)
    assert np.max(np.abs(got - ref.exact_bit)) < 2.0 ** -12
    assert np.max(np.abs(got - ref.bit)) < 1e-6


def _enc_slots(par, s, z, level, scale, seed):
    m = ckks.encode_int(par.N, z, scale)
    d = synth.encryption_draws(seed, f"v{seed}", par.q[: level + 1], par.N)
    return ckks.encrypt(par, m, s, d.a, d.e, level, scale)


def test_fold_adds_a_times_u_before_the_relinearisation():
    """relin_rescale(tensor(a, b) + fold of c u) decrypts to a b + c u at the
    standard scale of the level below, for u above the product's level (its
    own scale) and positive, negative and tiny c."""
    par = chain_params(6)
    s = query.secret(par, 7, 2 * par.N // 3)
    keys = query.make_keys(par, s, 7, 1)
    S = query.standard_scales(par)
    plan = query.Plan(S=S, l_lin=5, l_d=5, l_y=5, l_u=5, l_out=1, pt_scale=1.0, mask_scale=0.0, ragged=False)
    ev = query.Evaluator(par, keys, plan)
    g = np.random.default_rng(7)
    lt = 4
    za, zb, zu = (g.uniform(-1, 1, par.n_slots) for _ in range(3))
    a = _enc_slots(par, s, za, lt, S[lt], 1)
    b = _enc_slots(par, s, zb, lt, S[lt], 2)
    u = _enc_slots(par, s, zu, 6, S[6], 3)
    for c in (0.75, -2.5, 3e-5):
        t = ev.relin_rescale(ev.fold(ckks.tensor(par, a, b), u, c), lt - 1)
        got = ckks.decrypt_slots(par, t, s).real
        assert np.max(np.abs(got - (za * zb + c * zu))) < 1e-6, c


def test_power_scales_follow_the_power_rule():
    """The planner's tracked scales equal the scales the evaluator's power
    rule leaves on x^k (lower factor dropped, product over the removed prime)."""
    par = chain_params(11)
    S = query.standard_scales(par)
    top = 9
    sc, lv = query.power_scales(S[top] * 1.0001, top, 15, par.q)
    # by hand for the first few powers
    assert lv[2] == top - 1 and sc[2] == (sc[1] * sc[1]) / float(par.q[top])
    assert lv[3] == top - 2 and sc[3] == (sc[2] * sc[1]) / float(par.q[top - 1])
    assert lv[4] == top - 2 and sc[4] == (sc[2] * sc[2]) / float(par.q[top - 1])
    assert lv[12] == top - 4 and sc[12] == (sc[8] * sc[4]) / float(par.q[lv[8]])
    # a standard start keeps the powers of two standard
    st, sl = query.power_scales(S[top], top, 8, par.q)
    for k in (2, 4, 8):
        assert st[k] == S[sl[k]]
