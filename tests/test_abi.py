"""C ABI checks that need no GPU: the library builds, loads, and exports every
function include/kc.h declares; host-only entry points behave."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import kcgen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "kc.h")


@pytest.fixture(scope="module")
def lib():
    import paper_1403_0734_gb300.build as kb
    path = kb.build()
    from paper_1403_0734_gb300 import kc
    kc._load()
    return path


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kc_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["kc_orient", "kc_count", "kc_estimate", "kc_free", "kc_strerror", "kc_build_csr",
                     "kc_count_csr", "kc_estimate_csr", "kc_export", "kc_info"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (kc_[a-z_]+)\b", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    cdll = ctypes.CDLL(lib)
    for f in declared_functions():
        assert hasattr(cdll, f)


def test_strerror_and_version(lib):
    from paper_1403_0734_gb300 import kc
    L = kc._load()
    assert L.kc_strerror(0) == b"ok"
    assert L.kc_strerror(3) == b"count overflow"
    assert b"sm_103a" in L.kc_version()


def test_build_csr_matches_generator_canonicalisation(lib):
    from paper_1403_0734_gb300 import kc
    rng = np.random.default_rng(3)
    n = 300
    e = rng.integers(0, n, size=(4000, 2))
    off, adj, m = kc.build_csr(n, e[:, 0], e[:, 1])
    g = kcgen.from_edges(n, e)
    assert m == g.m
    assert np.array_equal(off, g.off) and np.array_equal(adj, g.adj)


def test_build_csr_rejects_bad_endpoint(lib):
    from paper_1403_0734_gb300 import kc
    with pytest.raises(kc.KcError):
        kc.build_csr(5, [0, 1], [1, 7])


def test_params(lib):
    from paper_1403_0734_gb300 import kc
    assert kc.get_param(kc.KC_PARAM_SMEM_MAX_WORDS) == 32
    kc.set_param(kc.KC_PARAM_SMEM_MAX_WORDS, 4)
    assert kc.get_param(kc.KC_PARAM_SMEM_MAX_WORDS) == 4
    kc.set_param(kc.KC_PARAM_SMEM_MAX_WORDS, 32)
    for bad in (0, 3, 12, 33, 64):  # the queue's group widths only: powers of two up to 32
        with pytest.raises(kc.KcError):
            kc.set_param(kc.KC_PARAM_SMEM_MAX_WORDS, bad)
    with pytest.raises(kc.KcError):
        kc.set_param(99, 1)
    assert kc.get_param(kc.KC_PARAM_ALGO) == kc.KC_ALGO_DFS
    kc.set_param(kc.KC_PARAM_ALGO, kc.KC_ALGO_PIVOT)
    assert kc.get_param(kc.KC_PARAM_ALGO) == kc.KC_ALGO_PIVOT
    kc.set_param(kc.KC_PARAM_ALGO, kc.KC_ALGO_DFS)
    with pytest.raises(kc.KcError):
        kc.set_param(kc.KC_PARAM_ALGO, 7)
    assert kc.get_param(kc.KC_PARAM_TRI) == 1
    kc.set_param(kc.KC_PARAM_TRI, 0)
    assert kc.get_param(kc.KC_PARAM_TRI) == 0
    kc.set_param(kc.KC_PARAM_TRI, 1)
    with pytest.raises(kc.KcError):
        kc.set_param(kc.KC_PARAM_TRI, 2)
    assert kc.get_param(kc.KC_PARAM_COMPLEMENT) == 1
    kc.set_param(kc.KC_PARAM_COMPLEMENT, 0)
    assert kc.get_param(kc.KC_PARAM_COMPLEMENT) == 0
    kc.set_param(kc.KC_PARAM_COMPLEMENT, 1)
    for bad in (-1, 2):
        with pytest.raises(kc.KcError):
            kc.set_param(kc.KC_PARAM_COMPLEMENT, bad)
