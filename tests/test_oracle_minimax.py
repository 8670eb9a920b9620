"""Pins for the composite minimax sign (Table 2's alpha/beta vocabulary): each
Remez stage equioscillates (Chebyshev's alternation theorem: n + 1 alternating
extrema of equal size certify the minimax odd polynomial with n terms), beats
the closed-form f3 on the same interval, and the composite keeps its error on
a dense grid; alpha 8 with three degree-15 stages reaches Table 2's beta of 12;
the stored golden coefficients are what the oracle computes."""
import json
import os

import numpy as np
import pytest

pytest.importorskip("mpmath")
from oracle import query, sign  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "minimax_sign.json")


def alternation(coeffs, a, b, grid=200001):
    x = np.linspace(a, b, grid)
    e = query.odd_poly(coeffs, x) - 1.0
    ext = [0] + [j for j in range(1, grid - 1) if (e[j] - e[j - 1]) * (e[j + 1] - e[j]) <= 0] + [grid - 1]
    seq = []
    for j in ext:
        if seq and np.sign(e[j]) == np.sign(e[seq[-1]]):
            if abs(e[j]) > abs(e[seq[-1]]):
                seq[-1] = j
        else:
            seq.append(j)
    return np.abs(e[seq]), float(np.max(np.abs(e)))


@pytest.mark.parametrize("n_terms,a", [(4, 0.1), (4, 2.0 ** -4), (8, 2.0 ** -8), (8, 0.5)])
def test_stage_equioscillates(n_terms, a):
    c, err = sign.remez_odd(n_terms, a, 1.0)
    mags, emax = alternation(c, a, 1.0)
    assert len(mags) >= n_terms + 1
    top = np.sort(mags)[-(n_terms + 1):]
    assert np.max(top) - np.min(top) <= 1e-6 * max(emax, 1e-12) + 1e-13
    assert abs(emax - err) <= 1e-9 * max(err, 1e-12) + 1e-13


@pytest.mark.parametrize("a", [0.1, 0.25, 0.5])
def test_minimax_beats_f3(a):
    """On [a, 1] the degree-7 minimax error is at most f3's (optimality)."""
    c, err = sign.remez_odd(4, a, 1.0)
    x = np.linspace(a, 1.0, 100001)
    f3err = float(np.max(np.abs(query.odd_poly(query.F3, x) - 1.0)))
    assert err <= f3err + 1e-12


def test_composite_meets_table2_row1():
    """alpha = 8, three degree-15 stages: error E on [2^-8, 1] (dense grid, and by
    oddness on the negative side) with beta = -log2(E/2) >= 12 (Table 2)."""
    stages, err = sign.composite_minimax(8, [15, 15, 15])
    x = np.concatenate([np.linspace(2.0 ** -8, 1.0, 400001), np.geomspace(2.0 ** -8, 2.0 ** -4, 20001)])
    got = np.max(np.abs(query.composite_sign(stages, x) - 1.0))
    assert got <= err * (1 + 1e-6)
    assert np.max(np.abs(query.composite_sign(stages, -x) + 1.0)) <= err * (1 + 1e-6)
    assert sign.beta(err) >= 12


def test_golden_file_matches_oracle():
    with open(GOLDEN) as f:
        gold = json.load(f)
    g = gold["alpha8_15x3"]
    stages, err = sign.composite_minimax(g["alpha"], g["degrees"])
    assert np.allclose(np.array(stages), np.array(g["stages"]), rtol=1e-12, atol=0)
    assert abs(err - g["error"]) <= 1e-12 * err


def load_stages(name):
    with open(GOLDEN) as f:
        return json.load(f)[name]


def test_degree15_stages_exact_count_near_threshold():
    """The query with the alpha = 8 composite (three degree-15 stages, depth 4
    each): one attribute, f(x) = x, t = 0, values avoiding 127-128 so every
    |z| >= 2^-7.4 > 2^-8.  The decrypted count is the exact count -- which
    three f3 stages (margin 2^-1.84 at tolerance 2^-12) cannot give here."""
    import synth
    from oracle import ckks, rns
    g = load_stages("alpha8_15x3")
    stages = g["stages"]
    q = rns.gen_primes(50, 1) + rns.gen_primes(40, 15)
    par = ckks.Params(12, q, rns.gen_primes(60, 1), 2.0 ** 40)
    R = 2048
    rng = np.random.default_rng(21)
    v = rng.integers(0, 254, R)
    vals = np.where(v >= 127, v + 2, v).astype(np.uint8)[:, None]
    qv = synth.QueryValues(w=np.array([1.0]), c=np.array([0.0, 1.0]), t=0.0)
    shape = query.QueryShape(R, 1, 1, stages)
    plan = query.make_plan(par, shape)
    assert plan.l_u == plan.l_y - 12
    s = query.secret(par, 4, 2 * par.N // 3)
    keys = query.make_keys(par, s, 4, 1, query.innersum_galois(par))
    db = query.encode_database(par, plan, vals)
    eq = query.encrypt_query(par, s, qv, 4)
    out = query.evaluate_query(par, keys, shape, db, eq)
    got = ckks.decrypt_slots(par, out, s).real
    ref = query.fp64_pipeline(vals, qv, stages)
    assert np.min(np.abs(ref.z)) > 2.0 ** -8
    assert int(np.rint(got[0] * R)) == ref.exact == int((vals[:, 0] > 128).sum())
    assert abs(got[0] * R - ref.count) < 0.05
    f3 = query.fp64_pipeline(vals, qv, [query.F3] * 3)
    assert abs(f3.count - f3.exact) > 1.0    # f3 stages miss records this close to the threshold
