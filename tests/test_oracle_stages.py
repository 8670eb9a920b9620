"""Per-slot pins of the oracle's query stages against the FP64 plaintext
pipeline (the same polynomials evaluated in floating point without
encryption), at the tolerance the method is held to: |error| <= 2^-12 on the
normalised values.  Each stage of a block is decrypted slot by slot -- the
linear combination x (attribute selection, Section 3.3), the private
polynomial y = f(x), y - t (the encrypted threshold, Section 5.4.2) and the
step values u (the composite sign mapped to step(z) = (sign(z) + 1)/2,
Section 5.4.2) -- rather than only through the InnerSum, where per-slot
errors of opposite sign could cancel.  Cases: N = 2^12 test chains (full,
ragged, degree 15 with three stages) and one block of the benchmark
workload (N = 2^16, twenty 50-bit primes, alpha = 4)."""
import numpy as np
import pytest

import synth
from oracle import ckks, query, rns

TOL = 2.0 ** -12


def chain_params(n_q40: int, log_n: int = 12):
    """Test-only chain: one 50-bit q_0, n_q40 primes of 40 bits, one 60-bit special prime, Delta = 2^40."""
    q = rns.gen_primes(50, 1) + rns.gen_primes(40, n_q40)
    return ckks.Params(log_n, q, rns.gen_primes(60, 1), 2.0 ** 40)


def stage_errors(par, vals, qv, stages, seed, alpha, hw, blocks=None):
    """Worst |decrypted - FP64| per stage over the live slots of the blocks."""
    R, h = vals.shape
    degree = len(qv.c) - 1
    shape = query.QueryShape(R, h, degree, stages)
    plan = query.make_plan(par, shape)
    s = query.secret(par, seed, hw)
    keys = query.make_keys(par, s, seed, alpha)          # the relinearisation key is all a block needs
    db = query.encode_database(par, plan, vals)
    eq = query.encrypt_query(par, s, qv, seed)
    ev = query.Evaluator(par, keys, plan)
    ck, tadj = ev.per_query(eq, degree)
    ref = query.fp64_pipeline(vals, qv, stages)
    want = {"x": ref.x, "y": ref.y, "d": ref.y - qv.t, "u": ref.u}
    n = par.n_slots
    worst = {k: 0.0 for k in want}
    for b in range(len(db.pts)) if blocks is None else blocks:
        rec = {}
        u = ev.block(db.pts[b], eq, ck, tadj, degree, record=rec)
        assert rec["u"] is u and set(rec) == set(want)
        lo, hi = b * n, min(R, (b + 1) * n)
        for k, ct in rec.items():
            got = ckks.decrypt_slots(par, ct, s).real[: hi - lo]
            if k == "u":
                got = got * plan.records_norm      # the step values leave the block divided by R
            worst[k] = max(worst[k], float(np.max(np.abs(got - want[k][lo:hi]))))
    return worst, ref


@pytest.mark.parametrize("n_q40,records,attrs,degree,nstages,dist", [
    (11, 2048, 8, 7, 1, "uniform"),
    (12, 1500, 4, 3, 1, "paper"),       # ragged: one block, 1500 live slots
    (17, 2048, 4, 15, 3, "mixed"),
])
def test_stage_values_per_slot_n4096(n_q40, records, attrs, degree, nstages, dist):
    par = chain_params(n_q40)
    vals = synth.database(synth.stream(31 + degree, "db"), records, attrs, dist)
    qv = synth.query_values(synth.stream(31 + degree, "qv"), attrs, degree)
    worst, ref = stage_errors(par, vals, qv, [query.F3] * nstages, seed=4, alpha=1, hw=2 * par.N // 3)
    assert all(v <= TOL for v in worst.values()), worst
    # the check has teeth: the stages differ from one another by far more than the tolerance
    assert np.max(np.abs(ref.y - ref.x)) > 1e-3 and np.max(np.abs(ref.u - 0.5)) > 1e-2


def test_stage_values_per_slot_benchmark_block():
    """One 32768-record block of the benchmark workload: N = 2^16, twenty
    50-bit primes, three 60-bit special primes, Delta = 2^50, alpha = 4,
    16 mixed attributes, degree 15, three f3 stages, h = 192."""
    q = rns.gen_primes(50, 20)
    par = ckks.Params(16, q, rns.gen_primes(60, 3, exclude=q), 2.0 ** 50)
    vals = synth.database(synth.stream(41, "db"), par.n_slots, 16, "mixed")
    qv = synth.query_values(synth.stream(41, "qv"), 16, 15)
    worst, _ = stage_errors(par, vals, qv, [query.F3] * 3, seed=41, alpha=4, hw=192)
    assert all(v <= TOL for v in worst.values()), worst
