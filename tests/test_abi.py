"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/tetris.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "tetris.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tetris_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def built():
    import paper_2412_13269_gb300 as t
    return t.build()


def test_library_exports_every_declared_symbol(built):
    so = ctypes.CDLL(built)
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing


def test_binding_covers_header():
    import paper_2412_13269_gb300 as t
    assert set(declared_functions()) == set(t.SIGNATURES)


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_2412_13269_gb300 as t
    monkeypatch.setattr(t, "LIB_PATH", str(tmp_path / "missing.so"))
    t.lib.cache_clear()
    try:
        with pytest.raises(ImportError):
            t.lib()
    finally:
        t.lib.cache_clear()


def test_prime_generation_matches_oracle(built):
    import paper_2412_13269_gb300 as t
    from oracle import rns
    for bits, count in [(50, 20), (60, 3), (40, 11)]:
        assert t.gen_primes(bits, count) == rns.gen_primes(bits, count)
    assert t.gen_primes(40, 4, exclude=rns.gen_primes(40, 2)) == rns.gen_primes(40, 4, exclude=rns.gen_primes(40, 2))
