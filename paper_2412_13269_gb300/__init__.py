"""Python binding of the GB300 RNS-CKKS query library (include/tetris.h).

Argument marshalling only: every entry point forwards to the CUDA library
libtetris.so built in-tree by ``build()``; nothing here computes.  Importing
the package does not load the library; the first call does, and it raises
if the library has not been built (there is no CPU fallback).

Functions keep the C names (``tetris_ctx_create`` ...).  ``Ctx`` is a small
convenience wrapper that turns numpy arrays (host) or torch CUDA tensors
(device) into the C structs.
"""
from __future__ import annotations

import ctypes as C
import os
from functools import lru_cache

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libtetris.so")

TETRIS_OK = 0
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ELEVEL", -5: "ENOTFOUND", -6: "ETIMEOUT", -7: "EBUSY"}

OP_ADD, OP_SUB, OP_TENSOR, OP_RELIN, OP_RESCALE, OP_MUL_INT, OP_ADD_INT = 1, 2, 3, 4, 5, 6, 7
OP_AUTOMORPHISM, OP_ROTATE, OP_KEYSWITCH, OP_MUL_PLAIN, OP_NTT, OP_INNERSUM, OP_DROP = 8, 9, 10, 11, 12, 13, 14
OP_RELIN_RESCALE, OP_RESCALE_MUL_INT = 15, 16
OPT_BLOCKS_PER_LAUNCH, OPT_USE_GRAPH, OPT_KS_ALPHA, OPT_PROFILE, OPT_NTT_GROUP, OPT_KS_BASE2 = 1, 2, 3, 4, 5, 6
OPT_QUERY_STAGE, OPT_DEBUG_CHECKS, OPT_PERSISTENT = 7, 8, 9
STAGE_FULL, STAGE_X, STAGE_Y, STAGE_D, STAGE_U = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    from . import buildlib
    return buildlib.build(force=force)


class TetrisError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class CtIn(C.Structure):
    _fields_ = [("level", C.c_uint32), ("ncomp", C.c_uint32), ("scale", C.c_double), ("data", C.c_void_p)]


class CtOut(C.Structure):
    _fields_ = [("level", C.c_uint32), ("ncomp", C.c_uint32), ("scale", C.c_double), ("data", C.c_void_p),
                ("cap_words", C.c_size_t)]


class Query(C.Structure):
    _fields_ = [("n_attrs", C.c_uint32), ("w", C.POINTER(CtIn)), ("f_degree", C.c_uint32),
                ("f_coeffs", C.POINTER(CtIn)), ("threshold", C.POINTER(CtIn)), ("sign_stages", C.c_uint32),
                ("sign_degree", C.c_uint32), ("sign_coeffs", C.POINTER(C.c_double)), ("total_records", C.c_uint64),
                ("global_threshold", C.POINTER(CtIn)), ("global_stages", C.c_uint32),
                ("global_coeffs", C.POINTER(C.c_double))]


class CtxInfo(C.Structure):
    _fields_ = [("log_n", C.c_uint32), ("n_q", C.c_uint32), ("n_p", C.c_uint32), ("scale", C.c_double),
                ("pt_scale", C.c_double), ("device_bytes", C.c_size_t)]


class PlanInfo(C.Structure):
    _fields_ = [("l_lin", C.c_int32), ("l_d", C.c_int32), ("l_y", C.c_int32), ("l_u", C.c_int32),
                ("l_out", C.c_int32), ("ragged", C.c_uint32), ("relins", C.c_uint32), ("rescales", C.c_uint32),
                ("rotations", C.c_uint32), ("kernel_launches", C.c_uint32), ("pt_scale", C.c_double),
                ("mask_scale", C.c_double), ("l_ret", C.c_int32), ("pad", C.c_uint32), ("input_words", C.c_uint64)]


class ServeStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("rejected", C.c_uint64), ("p50_ms", C.c_double),
                ("p99_ms", C.c_double), ("device_bytes", C.c_size_t), ("peak_device_bytes", C.c_size_t),
                ("cancelled", C.c_uint64), ("max_admitted", C.c_uint32), ("max_overlap", C.c_uint32)]


class BatchItem(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("level", C.c_uint32), ("ct", C.c_void_p), ("pt", C.c_void_p),
                ("rotations", C.c_uint32), ("out", C.c_void_p)]


SCHED_PER_ITEM, SCHED_MERGED, SCHED_AUTO, SCHED_FUSED = 0, 1, 2, 3


def batch_run(items, schedule: int = SCHED_AUTO):
    """items: list of (Ctx, level, ct [2][level+1][N] uint64, pt [level+1][N] uint64, rotations).
    Returns (outputs, schedule_used, device_ms)."""
    keep, outs = [], []
    arr = (BatchItem * len(items))()
    for i, (ctx, level, ct, pt, rot) in enumerate(items):
        ct = np.ascontiguousarray(ct, dtype=np.uint64)
        pt = np.ascontiguousarray(pt, dtype=np.uint64)
        out = np.empty((2, level, ctx.N), dtype=np.uint64)
        keep += [ct, pt]
        outs.append(out)
        arr[i] = BatchItem(ctx.h.value if isinstance(ctx.h, C.c_void_p) else ctx.h, level, ct.ctypes.data,
                           pt.ctypes.data, rot, out.ctypes.data)
    used = C.c_int()
    ms = C.c_double()
    check(lib().tetris_batch_run(arr, len(items), schedule, C.byref(used), C.byref(ms)))
    return outs, used.value, ms.value


class TuneEntry(C.Structure):
    _fields_ = [("blocks_per_launch", C.c_int32), ("ntt_group_log2", C.c_int32), ("ms", C.c_double),
                ("persistent", C.c_int32), ("pad", C.c_int32)]


class KernelStat(C.Structure):
    _fields_ = [("kind", C.c_char * 48), ("launches", C.c_uint32), ("total_ms", C.c_double), ("alg_bytes", C.c_double),
                ("alg_modmuls", C.c_double), ("units", C.c_double)]


_vp, _u32, _u64, _i64, _sz, _d = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int64, C.c_size_t, C.c_double
SIGNATURES = {
    "tetris_ctx_create": [C.POINTER(_vp), _u32, _vp, _u32, _vp, _u32, _d, C.c_int],
    "tetris_ctx_destroy": [_vp],
    "tetris_last_error": [],
    "tetris_get_info": [_vp, C.POINTER(CtxInfo)],
    "tetris_standard_scale": [_vp, _u32, C.POINTER(_d)],
    "tetris_gen_primes": [_u32, _u32, _u32, _vp, _u32, _vp],
    "tetris_load_relin_key": [_vp, _vp, _sz, _u32],
    "tetris_load_rotation_key": [_vp, _u32, _vp, _sz, _u32],
    "tetris_get_key": [_vp, _u32, _vp, _sz],
    "tetris_keygen_relin": [_vp, _vp, _vp, _vp, _u32],
    "tetris_keygen_rotation": [_vp, _u32, _vp, _vp, _vp, _u32],
    "tetris_encrypt": [_vp, _vp, _vp, _vp, _vp, _u32, _d, C.POINTER(CtOut)],
    "tetris_upload_database": [_vp, _vp, _u64, _u32, C.POINTER(_u32)],
    "tetris_upload_database_encoded": [_vp, _vp, _vp, _u64, _u32, C.POINTER(_u32)],
    "tetris_free_database": [_vp, _u32],
    "tetris_encode": [_vp, _vp, _u32, _d, _vp],
    "tetris_encode_real": [_vp, _vp, _u32, _vp],
    "tetris_evaluate_query": [_vp, _u32, C.POINTER(Query), C.POINTER(CtOut)],
    "tetris_evaluate_query_device": [_vp, _u32, C.POINTER(Query), C.POINTER(CtOut), _vp],
    "tetris_plan": [_vp, _u32, _u32, _u32, C.POINTER(PlanInfo)],
    "tetris_reduce_sum_device": [_vp, _vp, _u32, _u32, _vp],
    "tetris_batch_run": [C.POINTER(BatchItem), _u32, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double)],
    "tetris_autotune": [_vp, _u32, C.POINTER(Query), _u32, C.POINTER(TuneEntry), _u32, C.POINTER(_u32)],
    "tetris_set_option": [_vp, C.c_int, _i64],
    "tetris_get_option": [_vp, C.c_int, C.POINTER(_i64)],
    "tetris_op": [_vp, C.c_int, C.POINTER(CtIn), C.POINTER(CtIn), _i64, C.POINTER(CtOut)],
    "tetris_modmul_peak": [C.c_int, C.POINTER(C.c_double)],
    "tetris_get_kernel_stats": [_vp, C.POINTER(KernelStat), _u32, C.POINTER(_u32)],
    "tetris_rescale_ntt_noalloc": [_vp, _vp, _vp, _u32, _u32, _vp],
    "tetris_serve_start": [_vp, _sz, _u32],
    "tetris_submit": [_vp, _u32, C.POINTER(Query), C.POINTER(_u64)],
    "tetris_poll": [_vp, _u64, C.POINTER(CtOut), _u32],
    "tetris_serve_stats_get": [_vp, C.POINTER(ServeStats), C.c_int],
    "tetris_cancel": [_vp, _u64],
    "tetris_debug_check": [_vp, C.c_int, C.POINTER(_u64)],
    "tetris_serve_stop": [_vp],
    "tetris_noalloc_scratch_bytes": [],
    "tetris_repack": [_vp, _vp, _u32, _u32, _d, C.POINTER(CtOut)],
    "tetris_repack_device": [_vp, _vp, _u32, _u32, _d, C.POINTER(CtOut), _vp],
    "tetris_pfe_scores": [_vp, _vp, _u32, _vp, _u64, _vp],
    "tetris_pfe_scores_device": [_vp, _vp, _u32, _vp, _u64, _vp, _vp],
}


@lru_cache(maxsize=1)
def lib():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libtetris.so is not built ({LIB_PATH}); run paper_2412_13269_gb300.build()")
    so = C.CDLL(LIB_PATH)
    for name, args in SIGNATURES.items():
        f = getattr(so, name)
        f.argtypes = args
        f.restype = {"tetris_last_error": C.c_char_p, "tetris_ctx_destroy": None,
                     "tetris_noalloc_scratch_bytes": C.c_size_t}.get(name, C.c_int)
    return so


def check(rc: int):
    if rc != TETRIS_OK:
        raise TetrisError(rc, lib().tetris_last_error().decode())


def _ptr(a) -> int:
    """Address of a C-contiguous numpy array or a torch tensor."""
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    return a.data_ptr()


def _is_device(a) -> bool:
    return not isinstance(a, np.ndarray)


def modmul_peak(device: int = 0) -> float:
    """Measured lazy-Shoup modular multiplications per second (G/s)."""
    r = C.c_double()
    check(lib().tetris_modmul_peak(device, C.byref(r)))
    return r.value


def gen_primes(bits: int, count: int, congruence_log2: int = 17, exclude=()) -> list:
    out = np.zeros(count, dtype=np.uint64)
    ex = np.asarray(list(exclude), dtype=np.uint64)
    check(lib().tetris_gen_primes(bits, count, congruence_log2, ex.ctypes.data if ex.size else None, ex.size, out.ctypes.data))
    return [int(x) for x in out]


def ct_in(data, level: int, scale: float, ncomp: int | None = None) -> CtIn:
    nc = ncomp if ncomp is not None else data.shape[0]
    return CtIn(level, nc, float(scale), _ptr(data))


class Ctx:
    """Owns a tetris_ctx; methods marshal numpy/torch buffers into the C calls."""

    def __init__(self, log_n: int, q, p, scale: float, device: int = 0):
        self.log_n, self.N = log_n, 1 << log_n
        self.q, self.p = [int(x) for x in q], [int(x) for x in p]
        self.scale = float(scale)
        qa, pa = np.asarray(self.q, dtype=np.uint64), np.asarray(self.p, dtype=np.uint64)
        h = C.c_void_p()
        check(lib().tetris_ctx_create(C.byref(h), log_n, qa.ctypes.data, len(self.q), pa.ctypes.data, len(self.p),
                                      self.scale, device))
        self.h = h
        self._keep = []

    def close(self):
        if getattr(self, "h", None):
            lib().tetris_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def L(self) -> int:
        return len(self.q) - 1

    def info(self) -> CtxInfo:
        i = CtxInfo()
        check(lib().tetris_get_info(self.h, C.byref(i)))
        return i

    def standard_scale(self, level: int) -> float:
        v = C.c_double()
        check(lib().tetris_standard_scale(self.h, level, C.byref(v)))
        return v.value

    # keys
    def load_relin_key(self, evk: np.ndarray, alpha: int):
        evk = np.ascontiguousarray(evk, dtype=np.uint64)
        check(lib().tetris_load_relin_key(self.h, evk.ctypes.data, evk.size, alpha))

    def load_rotation_key(self, g: int, evk: np.ndarray, alpha: int):
        evk = np.ascontiguousarray(evk, dtype=np.uint64)
        check(lib().tetris_load_rotation_key(self.h, g, evk.ctypes.data, evk.size, alpha))

    def keygen_relin(self, s, a, e, alpha: int):
        s, a, e = (np.ascontiguousarray(x) for x in (s, a, e))
        check(lib().tetris_keygen_relin(self.h, s.ctypes.data, a.ctypes.data, e.ctypes.data, alpha))

    def keygen_rotation(self, g: int, s, a, e, alpha: int):
        s, a, e = (np.ascontiguousarray(x) for x in (s, a, e))
        check(lib().tetris_keygen_rotation(self.h, g, s.ctypes.data, a.ctypes.data, e.ctypes.data, alpha))

    def get_key(self, g: int, dnum: int) -> np.ndarray:
        out = np.empty((dnum, 2, len(self.q) + len(self.p), self.N), dtype=np.uint64)
        check(lib().tetris_get_key(self.h, g, out.ctypes.data, out.size))
        return out

    def encrypt(self, m, s, a, e, level: int, scale: float) -> np.ndarray:
        m, s, e = (np.ascontiguousarray(x, dtype=np.int64) for x in (m, s, e))
        a = np.ascontiguousarray(a[: level + 1], dtype=np.uint64)
        out = np.empty((2, level + 1, self.N), dtype=np.uint64)
        o = CtOut(0, 0, 0.0, out.ctypes.data, out.size)
        check(lib().tetris_encrypt(self.h, m.ctypes.data, s.ctypes.data, a.ctypes.data, e.ctypes.data, level, scale,
                                   C.byref(o)))
        return out

    # database
    def upload_database(self, vals: np.ndarray) -> int:
        vals = np.ascontiguousarray(vals, dtype=np.uint8)
        h = C.c_uint32()
        check(lib().tetris_upload_database(self.h, vals.ctypes.data, vals.shape[0], vals.shape[1], C.byref(h)))
        return h.value

    def upload_database_encoded(self, coeffs: np.ndarray, mask_real, records: int, attrs: int) -> int:
        coeffs = np.ascontiguousarray(coeffs, dtype=np.int64)
        mr = None if mask_real is None else np.ascontiguousarray(mask_real, dtype=np.float64)
        h = C.c_uint32()
        check(lib().tetris_upload_database_encoded(self.h, coeffs.ctypes.data, None if mr is None else mr.ctypes.data,
                                                   records, attrs, C.byref(h)))
        return h.value

    def free_database(self, db: int):
        check(lib().tetris_free_database(self.h, db))

    def encode(self, slots, scale: float) -> np.ndarray:
        z = np.ascontiguousarray(slots, dtype=np.float64)
        out = np.empty(self.N, dtype=np.int64)
        check(lib().tetris_encode(self.h, z.ctypes.data, z.size, scale, out.ctypes.data))
        return out

    def encode_real(self, slots) -> np.ndarray:
        z = np.ascontiguousarray(slots, dtype=np.float64)
        out = np.empty(self.N, dtype=np.float64)
        check(lib().tetris_encode_real(self.h, z.ctypes.data, z.size, out.ctypes.data))
        return out

    # options / plan
    def set_option(self, opt: int, value: int):
        check(lib().tetris_set_option(self.h, opt, value))

    def get_option(self, opt: int) -> int:
        v = C.c_int64()
        check(lib().tetris_get_option(self.h, opt, C.byref(v)))
        return v.value

    def kernel_stats(self) -> dict:
        """{kind: (launches, total_ms, alg_bytes, alg_modmuls, limb jobs)} gathered while OPT_PROFILE is on
        (clears them)."""
        buf = (KernelStat * 256)()
        n = C.c_uint32()
        check(lib().tetris_get_kernel_stats(self.h, buf, 256, C.byref(n)))
        return {buf[i].kind.decode(): (buf[i].launches, buf[i].total_ms, buf[i].alg_bytes, buf[i].alg_modmuls,
                                       buf[i].units) for i in range(n.value)}

    def repack(self, cts: np.ndarray, level: int, scale: float):
        """Ring repacking (Algorithm 1), host arrays: cts uint64 [n][2][level+1][N] ->
        (out [2][level+1][N], level, scale)."""
        cts = np.ascontiguousarray(cts, dtype=np.uint64)
        out = np.empty((2, level + 1, self.N), dtype=np.uint64)
        o = CtOut(0, 0, 0.0, out.ctypes.data, out.size)
        check(lib().tetris_repack(self.h, cts.ctypes.data, cts.shape[0], level, scale, C.byref(o)))
        return out, o.level, o.scale

    def repack_device(self, cts, n: int, level: int, scale: float, out, stream: int = 0):
        """Ring repacking on torch CUDA tensors (cts int64 [n][2][level+1][N], out int64 [2][level+1][N])."""
        o = CtOut(0, 0, 0.0, _ptr(out), out.numel())
        check(lib().tetris_repack_device(self.h, _ptr(cts), n, level, scale, C.byref(o), stream))
        return o.level, o.scale

    def pfe_scores(self, u: np.ndarray, exps: np.ndarray) -> np.ndarray:
        """PFE scoring step, host arrays: u uint64 [m][2][N], exps [p][m] -> uint64 [p][2][N]."""
        u = np.ascontiguousarray(u, dtype=np.uint64)
        e = np.ascontiguousarray(exps, dtype=np.uint32)
        m, p = u.shape[0], e.shape[0]
        out = np.empty((p, 2, self.N), dtype=np.uint64)
        check(lib().tetris_pfe_scores(self.h, u.ctypes.data, m, e.ctypes.data, p, out.ctypes.data))
        return out

    def pfe_scores_device(self, u, exps, out, m: int, p: int, stream: int = 0):
        """PFE scoring step on torch CUDA tensors (u int64 [m][2][N], exps int32 [p][m], out int64 [p][2][N])."""
        check(lib().tetris_pfe_scores_device(self.h, _ptr(u), m, _ptr(exps), p, _ptr(out), stream))

    def rescale_ntt_noalloc(self, src, dst, level: int, ncomp: int, stream: int = 0):
        """Allocation-free rescale of a device-resident NTT-order ciphertext
        (torch CUDA tensors); enqueued on ``stream``."""
        check(lib().tetris_rescale_ntt_noalloc(self.h, _ptr(src), _ptr(dst), level, ncomp, stream))

    def autotune(self, db: int, w, w_meta, c, c_meta, t, t_meta, sign_coeffs, reps: int = 3):
        """Times the query under each candidate schedule, keeps the fastest;
        returns [(blocks_per_launch, ntt_group_log2, ms, persistent)]."""
        q, keep = self._query_struct(w, w_meta, c, c_meta, t, t_meta, sign_coeffs)
        buf = (TuneEntry * 32)()
        n = C.c_uint32()
        check(lib().tetris_autotune(self.h, db, C.byref(q), reps, buf, 32, C.byref(n)))
        return [(buf[i].blocks_per_launch, buf[i].ntt_group_log2, buf[i].ms, buf[i].persistent) for i in range(n.value)]

    def reduce_sum_device(self, data, level: int, ncomp: int = 2, stream: int = 0):
        """In place: residue sums over partitions (torch CUDA int64 tensor) -> residues mod q_i."""
        check(lib().tetris_reduce_sum_device(self.h, _ptr(data), level, ncomp, stream))

    def plan(self, db: int, degree: int, stages: int) -> PlanInfo:
        p = PlanInfo()
        check(lib().tetris_plan(self.h, db, degree, stages, C.byref(p)))
        return p

    # query
    def _query_struct(self, w, w_meta, c, c_meta, t, t_meta, sign_coeffs, total_records=0, glob=None):
        """glob: optional global threshold (t1 ciphertext, (level, scale), stage coefficients)."""
        W = (CtIn * len(w))(*[CtIn(lv, 2, sc, _ptr(x)) for x, (lv, sc) in zip(w, w_meta)])
        Cc = (CtIn * len(c))(*[CtIn(lv, 2, sc, _ptr(x)) for x, (lv, sc) in zip(c, c_meta)])
        T = CtIn(t_meta[0], 2, t_meta[1], _ptr(t))
        sc2 = np.asarray(sign_coeffs, dtype=np.float64)
        ncoef = sc2.shape[-1] if sc2.ndim == 2 else 4      # per stage: 4 (degree 7) or 8 (degree 15)
        sc = np.ascontiguousarray(sc2.reshape(-1))
        q = Query(len(w), W, len(c) - 1, Cc, C.pointer(T), sc.size // ncoef, 2 * ncoef - 1,
                  sc.ctypes.data_as(C.POINTER(C.c_double)), int(total_records))
        keep = [W, Cc, T, sc]
        if glob is not None:
            t1, (lv, scl), gco = glob
            T1 = CtIn(lv, 2, scl, _ptr(t1))
            g = np.ascontiguousarray(np.asarray(gco, dtype=np.float64).reshape(-1))
            q.global_threshold = C.pointer(T1)
            q.global_stages = g.size // ncoef
            q.global_coeffs = g.ctypes.data_as(C.POINTER(C.c_double))
            keep += [T1, g]
        return q, keep

    def evaluate_query(self, db: int, w, w_meta, c, c_meta, t, t_meta, sign_coeffs, out=None, total_records=0,
                       glob=None):
        """Host arrays: w/c/t are [2][level+1][N] uint64; metas are (level, scale);
        glob = (t1, (level, scale), global stage coefficients) adds the global
        threshold.  Returns (out array, level, scale)."""
        q, keep = self._query_struct(w, w_meta, c, c_meta, t, t_meta, sign_coeffs, total_records, glob)
        if out is None:
            out = np.empty(2 * (self.L + 1) * self.N, dtype=np.uint64)
        o = CtOut(0, 0, 0.0, _ptr(out), out.size if isinstance(out, np.ndarray) else out.numel())
        check(lib().tetris_evaluate_query(self.h, db, C.byref(q), C.byref(o)))
        n = 2 * (o.level + 1) * self.N
        return out[:n].reshape(2, o.level + 1, self.N), o.level, o.scale

    def query_stage(self, stage: int, blocks: int, db: int, w, w_meta, c, c_meta, t, t_meta, sign_coeffs,
                    total_records=0):
        """The ciphertexts of one stage of every block (TETRIS_OPT_QUERY_STAGE):
        returns ([blocks][2][level+1][N] uint64, level, scale)."""
        q, keep = self._query_struct(w, w_meta, c, c_meta, t, t_meta, sign_coeffs, total_records)
        out = np.empty(blocks * 2 * (self.L + 1) * self.N, dtype=np.uint64)
        o = CtOut(0, 0, 0.0, out.ctypes.data, out.size)
        prev = self.get_option(OPT_QUERY_STAGE)
        self.set_option(OPT_QUERY_STAGE, stage)
        try:
            check(lib().tetris_evaluate_query(self.h, db, C.byref(q), C.byref(o)))
        finally:
            self.set_option(OPT_QUERY_STAGE, prev)
        n = blocks * 2 * (o.level + 1) * self.N
        return out[:n].reshape(blocks, 2, o.level + 1, self.N), o.level, o.scale

    def evaluate_query_device(self, db: int, w, w_meta, c, c_meta, t, t_meta, sign_coeffs, out, stream: int,
                              total_records=0, glob=None):
        """torch CUDA tensors in and out; enqueued on ``stream`` (a cudaStream_t as int)."""
        q, keep = self._query_struct(w, w_meta, c, c_meta, t, t_meta, sign_coeffs, total_records, glob)
        o = CtOut(0, 0, 0.0, _ptr(out), out.numel())
        check(lib().tetris_evaluate_query_device(self.h, db, C.byref(q), C.byref(o), stream))
        return o.level, o.scale

    # serving
    def serve_start(self, budget_bytes: int, max_inflight: int):
        check(lib().tetris_serve_start(self.h, budget_bytes, max_inflight))

    def submit(self, db: int, w, w_meta, c, c_meta, t, t_meta, sign_coeffs, glob=None) -> int:
        q, keep = self._query_struct(w, w_meta, c, c_meta, t, t_meta, sign_coeffs, 0, glob)
        tk = C.c_uint64()
        check(lib().tetris_submit(self.h, db, C.byref(q), C.byref(tk)))
        return tk.value

    def poll(self, ticket: int, timeout_ms: int = 60000, cap_words: int | None = None):
        """Returns (out array, level, scale), or None if the ticket is still running.
        cap_words: the output capacity to announce (default: the whole buffer)."""
        out = np.empty(2 * (self.L + 1) * self.N, dtype=np.uint64)
        o = CtOut(0, 0, 0.0, out.ctypes.data, out.size if cap_words is None else min(cap_words, out.size))
        rc = lib().tetris_poll(self.h, ticket, C.byref(o), timeout_ms)
        if rc == -6:
            return None
        check(rc)
        n = 2 * (o.level + 1) * self.N
        return out[:n].reshape(2, o.level + 1, self.N), o.level, o.scale

    def debug_check(self, plant: bool = False) -> int:
        """Checks the guard words of every device buffer (TETRIS_GUARD_WORDS);
        returns the ranges the TETRIS_OPT_DEBUG_CHECKS bounds check has verified."""
        n = C.c_uint64()
        check(lib().tetris_debug_check(self.h, 1 if plant else 0, C.byref(n)))
        return n.value

    def cancel(self, ticket: int):
        check(lib().tetris_cancel(self.h, ticket))

    def serve_stats(self, reset: bool = False) -> ServeStats:
        st = ServeStats()
        check(lib().tetris_serve_stats_get(self.h, C.byref(st), 1 if reset else 0))
        return st

    def serve_stop(self):
        check(lib().tetris_serve_stop(self.h))

    # single operations
    def op(self, opcode: int, a: np.ndarray, a_level: int, a_scale: float = 1.0, b: np.ndarray | None = None,
           b_level: int = 0, arg: int = 0, out_comps: int | None = None, out_level: int | None = None):
        a = np.ascontiguousarray(a, dtype=np.uint64)
        A = CtIn(a_level, a.shape[0], a_scale, a.ctypes.data)
        B = None
        if b is not None:
            b = np.ascontiguousarray(b, dtype=np.uint64)
            B = CtIn(b_level, b.shape[0], 1.0, b.ctypes.data)
        comps = out_comps if out_comps is not None else 3
        lev = out_level if out_level is not None else a_level
        out = np.empty((comps, lev + 1, self.N), dtype=np.uint64)
        o = CtOut(0, 0, 0.0, out.ctypes.data, out.size)
        check(lib().tetris_op(self.h, opcode, C.byref(A), C.byref(B) if B is not None else None, arg, C.byref(o)))
        n = o.ncomp * (o.level + 1) * self.N
        return out.reshape(-1)[:n].reshape(o.ncomp, o.level + 1, self.N), o.level, o.scale
