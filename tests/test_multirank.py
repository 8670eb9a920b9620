"""Records sharded over two ranks (gloo, CPU): each rank evaluates its
partition with the oracle, normalised by the total record count, and the
ranks' result ciphertexts are summed residue by residue (an integer
all-reduce followed by a reduction mod q).  The sum decrypts to the count
over the whole database (the horizontally partitioned database of
Section 5.6, where the partial counts are added before the final step)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import synth
    from oracle import ckks, query, rns
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    q = rns.gen_primes(50, 1) + rns.gen_primes(40, 11)
    par = ckks.Params(12, q, rns.gen_primes(60, 1), 2.0 ** 40)
    s = query.secret(par, 7, 2 * par.N // 3)
    keys = query.make_keys(par, s, 7, 1, query.innersum_galois(par))   # same client keys on every rank
    per = par.n_slots
    full = synth.database(synth.stream(7, "db"), per * world, 4)
    shard = full[rank * per:(rank + 1) * per]
    qv = synth.query_values(synth.stream(7, "qv"), 4, 3)
    eq = query.encrypt_query(par, s, qv, 7)
    shape = query.QueryShape(per, 4, 3, [query.F3], norm_records=per * world)
    plan = query.make_plan(par, shape)
    out = query.evaluate_query(par, keys, shape, query.encode_database(par, plan, shard), eq)
    t = torch.from_numpy(out.data.view(np.int64).copy())
    dist.all_reduce(t)  # integer sums of residues, each < world * 2^50
    summed = t.numpy().view(np.uint64) % np.array(q[: out.level + 1], dtype=np.uint64)[None, :, None]
    if rank == 0:
        z = ckks.decrypt_slots(par, ckks.Ct(np.ascontiguousarray(summed), out.level, out.scale), s).real
        ref = query.fp64_pipeline(full, qv, [query.F3])
        np.save(os.path.join(out_dir, "result.npy"), np.array([z[0] * per * world, ref.count, np.ptp(z)]))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_records_sum_to_whole_count(tmp_path):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    got, want, spread = np.load(tmp_path / "result.npy")
    assert spread < 1e-6
    assert abs(got - want) < 0.05
