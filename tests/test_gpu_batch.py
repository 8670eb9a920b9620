"""Batches of independent jobs at uneven ring degrees (N = 2^12, 2^13) and
levels: every schedule (per item, merged launches, automatic) returns the
oracle's ciphertexts residue for residue for the chain
rescale(ct * pt) -> r rotations -> relinearise(y * y)."""
import numpy as np
import pytest

import synth
from oracle import ckks, query, rns

pytestmark = pytest.mark.gpu

T = pytest.importorskip("paper_2412_13269_gb300")


def test_uneven_batch_all_schedules_match_oracle():
    T.build()
    q = rns.gen_primes(50, 1) + rns.gen_primes(40, 6)
    p = rns.gen_primes(60, 1)
    setups = {}
    for log_n in (12, 13):
        par = ckks.Params(log_n, q, p, 2.0 ** 40)
        s = query.secret(par, log_n, 2 * par.N // 3)
        gal = [pow(5, 1 << k, 2 * par.N) for k in range(3)]
        keys = query.make_keys(par, s, log_n, 1, gal)
        ctx = T.Ctx(log_n, q, p, 2.0 ** 40)
        ctx.load_relin_key(keys.rlk, 1)
        for g, k in keys.rot.items():
            ctx.load_rotation_key(g, k, 1)
        setups[log_n] = (par, keys, ctx)
    rnd = np.random.default_rng(5)
    items, want = [], []
    for i in range(8):
        log_n = int(rnd.choice([12, 13]))
        par, keys, ctx = setups[log_n]
        level = int(rnd.integers(2, 7))
        rot = int(rnd.integers(0, 4))
        ct = np.stack([np.stack([rnd.integers(0, m, par.N, dtype=np.uint64) for m in q[: level + 1]]) for _ in range(2)])
        pt = np.stack([rnd.integers(0, m, par.N, dtype=np.uint64) for m in q[: level + 1]])
        items.append((ctx, level, ct, pt, rot))
        y = ckks.rescale(par, ckks.mul_plain(par, ckks.Ct(ct, level, 1.0), pt, 1.0))
        for k in range(rot):
            g = pow(5, 1 << (k % (log_n - 1)), 2 * par.N)
            y = ckks.rotate(par, y, g, keys.rot[g], 1)
        y = ckks.relinearize(par, ckks.tensor(par, y, y), keys.rlk, 1)
        want.append(y.data)
    for sched in (T.SCHED_PER_ITEM, T.SCHED_MERGED, T.SCHED_AUTO):
        outs, used, ms = T.batch_run(items, sched)
        assert ms > 0 and (used == sched or sched == T.SCHED_AUTO)
        for i, (o, w) in enumerate(zip(outs, want)):
            assert np.array_equal(o, w), (sched, i)
    for _, _, ctx in setups.values():
        ctx.close()


def test_fused_batch_across_degrees_matches_oracle():
    """The fused schedule (one launch per stage whatever the ring degree,
    persistent NTT and ModUp/key-inner-product kernels over the jobs' tiles) at
    N = 2^14, 2^15, 2^16 with levels 2..5 and 0..2 rotations: every schedule
    returns the oracle's ciphertexts residue for residue."""
    T.build()
    q = rns.gen_primes(50, 1) + rns.gen_primes(40, 5)
    p = rns.gen_primes(60, 1)
    setups = {}
    for log_n in (14, 15, 16):
        par = ckks.Params(log_n, q, p, 2.0 ** 40)
        s = query.secret(par, log_n, 192)
        gal = [pow(5, 1 << k, 2 * par.N) for k in range(2)]
        keys = query.make_keys(par, s, log_n, 3, gal)
        ctx = T.Ctx(log_n, q, p, 2.0 ** 40)
        ctx.load_relin_key(keys.rlk, 3)
        for g, k in keys.rot.items():
            ctx.load_rotation_key(g, k, 3)
        setups[log_n] = (par, keys, ctx)
    rnd = np.random.default_rng(7)
    items, want = [], []
    for i, log_n in enumerate((14, 15, 16, 16, 14, 15)):
        par, keys, ctx = setups[log_n]
        level = int(rnd.integers(2, 6))
        rot = int(rnd.integers(0, 3))
        ct = np.stack([np.stack([rnd.integers(0, m, par.N, dtype=np.uint64) for m in q[: level + 1]]) for _ in range(2)])
        pt = np.stack([rnd.integers(0, m, par.N, dtype=np.uint64) for m in q[: level + 1]])
        items.append((ctx, level, ct, pt, rot))
        y = ckks.rescale(par, ckks.mul_plain(par, ckks.Ct(ct, level, 1.0), pt, 1.0))
        for k in range(rot):
            g = pow(5, 1 << (k % (log_n - 1)), 2 * par.N)
            y = ckks.rotate(par, y, g, keys.rot[g], 3)
        y = ckks.relinearize(par, ckks.tensor(par, y, y), keys.rlk, 3)
        want.append(y.data)
    for sched in (T.SCHED_FUSED, T.SCHED_PER_ITEM, T.SCHED_MERGED, T.SCHED_AUTO):
        outs, used, ms = T.batch_run(items, sched)
        assert ms > 0 and (used == sched or sched == T.SCHED_AUTO)
        for i, (o, w) in enumerate(zip(outs, want)):
            assert np.array_equal(o, w), (sched, i)
    # degrees the persistent kernels do not take are refused before any launch
    small = T.Ctx(12, q, p, 2.0 ** 40)
    par12 = ckks.Params(12, q, p, 2.0 ** 40)
    ct = np.zeros((2, 3, par12.N), dtype=np.uint64)
    with pytest.raises(T.TetrisError, match="14, 16"):
        T.batch_run([(small, 2, ct, ct[0], 0)], T.SCHED_FUSED)
    small.close()
    for _, _, ctx in setups.values():
        ctx.close()
