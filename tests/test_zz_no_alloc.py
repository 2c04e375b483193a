"""kc_count_static: the allocation-free form of kc_count.

Callers that cannot allocate device memory when they need a count (a
process whose memory manager already owns the device, latency-critical code
that must not wait on cudaMalloc) use kc_count_static; its scratch is a
static array inside the library.  These tests check, through the C ABI, that
it returns exactly kc_count's total, on two calls in a row (the shared array
keeps the previous call's contents, so the second call checks that the
entry point clears what must start at zero), including the path where wide
owners take their bitmap tiles from that static array.

The file is named so that pytest collects it last.
"""
import pytest

import kcgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1403_0734_gb300.build as kb
    kb.build()
    import paper_1403_0734_gb300 as kc
    return kc


def graphs():
    return [kcgen.rmat(12, 16, 0.57, 0.19, 0.19, 1),
            kcgen.chung_lu(20000, 200000, 2.1, 2000.0, 1),
            kcgen.complete_multipartite((10,) * 60, shuffle_seed=5)]


def test_static_count_matches_kc_count_twice(kc):
    for g in graphs():
        G = kc.orient(g.off, g.adj)
        for k in (1, 2, 3, 4, 5):
            expected = kc.count(G, k)[0]
            first = kc.count_static(G, k)
            second = kc.count_static(G, k)
            assert first == expected and second == expected, (g.name, k, first, second, expected)
        G.free()


def test_static_count_with_global_tiles_twice(kc):
    # force every owner wider than 32 into global tiles, carved from the static array
    kc.set_param(kc.KC_PARAM_SMEM_MAX_WORDS, 1)
    try:
        for g in graphs():
            G = kc.orient(g.off, g.adj)
            for k in (3, 4, 5):
                expected = kc.count(G, k)[0]
                assert kc.count_static(G, k) == expected
                assert kc.count_static(G, k) == expected
            G.free()
    finally:
        kc.set_param(kc.KC_PARAM_SMEM_MAX_WORDS, 32)


def test_static_count_device_output_on_a_stream_and_pivot_tiles(kc):
    """Device outputs (two words, low and high) on a torch stream, for k = 1..5
    (k <= 2 written on the stream too), and the pivoting counter with every
    wide owner forced onto global tiles carved from the static array."""
    import ctypes
    import torch
    from paper_1403_0734_gb300 import kc as kcmod
    lib = kcmod._load()
    s = torch.cuda.Stream()
    out = torch.full((2,), -1, dtype=torch.int64, device="cuda")
    for g in graphs():
        G = kc.orient(g.off, g.adj)
        for k in (1, 2, 3, 4, 5):
            expected = kc.count(G, k)[0]
            for _ in range(2):
                out.fill_(-1)
                torch.cuda.synchronize()
                st = lib.kc_count_static(G.handle, k, kc.KC_DEVICE_PTRS, ctypes.c_void_p(out.data_ptr()),
                                         ctypes.c_void_p(s.cuda_stream))
                assert st == 0
                s.synchronize()
                assert int(out[0].item()) == expected and int(out[1].item()) == 0, (g.name, k)
        G.free()
    kc.set_param(kc.KC_PARAM_ALGO, kc.KC_ALGO_PIVOT)
    kc.set_param(kc.KC_PARAM_SMEM_MAX_WORDS, 1)
    try:
        for g in graphs():
            G = kc.orient(g.off, g.adj)
            for k in (4, 5):
                kc.set_param(kc.KC_PARAM_ALGO, kc.KC_ALGO_DFS)
                expected = kc.count(G, k)[0]
                kc.set_param(kc.KC_PARAM_ALGO, kc.KC_ALGO_PIVOT)
                assert kc.count_static(G, k) == expected and kc.count_static(G, k) == expected
            G.free()
    finally:
        kc.set_param(kc.KC_PARAM_SMEM_MAX_WORDS, 32)
        kc.set_param(kc.KC_PARAM_ALGO, kc.KC_ALGO_DFS)


def test_static_count_allocates_nothing(kc):
    """After a warm-up call, repeated calls leave the device's free memory
    unchanged (no allocation by the library, nor by its memory pool)."""
    import torch
    g = kcgen.chung_lu(20000, 200000, 2.1, 2000.0, 1)
    G = kc.orient(g.off, g.adj)
    expected = {k: kc.count(G, k)[0] for k in (3, 4, 5)}
    for k in (3, 4, 5):
        kc.count_static(G, k)  # warm-up: loads the module, commits the static array
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        for k in (3, 4, 5):
            assert kc.count_static(G, k) == expected[k]
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    G.free()
