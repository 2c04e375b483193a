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
