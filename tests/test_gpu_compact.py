"""Compact storage (Section 4.3's graph cost, the 16-bit value setup of
Section 5.4) against the oracle.

16-bit values: the library rounds every document value to the nearest fp16 on
input and builds and searches that rounded collection.  The oracle is given
the same rounded collection (numpy's float16 rounding, ties to even), so the
bars are the fp32 ones: the index is bit-equal, exhaustive ids are exact up to
near-ties with scores within 1e-5 of fp64 (an fp16 value is exact in fp32, so
a score is still an fp32 sum of <= 150 rounded products), and pruned recall is
within 0.005 of the oracle's.

Bit-packed graph: each kappa-NN id takes floor(log2(N - 1)) + 1 bits (one more
when N is a power of two, leaving the all-ones code for a missing neighbour);
the graph read back is the graph installed, and search with it equals the
oracle's expansion over the unpacked graph.
"""
import numpy as np
import pytest

import oracle
import synth
from test_gpu_parity import check_exact_ids, check_scores_only, compare_index, f32

pytestmark = pytest.mark.gpu


def round16(m):
    return synth.CSR(m.indptr.copy(), m.terms.copy(), m.vals.astype(np.float16).astype(np.float32), m.dim)


@pytest.fixture(scope="module")
def half(sz, small):
    docs16 = round16(small["docs"])
    out = {}
    for quant in (True, False):
        ix = sz.seismic_build(small["docs"], lambda_=small["lam"], beta=small["beta"], alpha=small["alpha"],
                              quantize_u8=quant, seed=5, keep_full_lists=True, keep_block_summaries=True,
                              values_fp16=True)
        ox = oracle.Index(docs16, small["lam"], small["beta"], small["alpha"], quant, seed=5)
        out[quant] = (ix, ox)
    yield docs16, out
    for ix, _ in out.values():
        ix.close()


@pytest.mark.parametrize("quant", [True, False])
def test_fp16_index_equals_oracle_on_rounded_collection(sz, small, half, quant):
    docs16, built = half
    ix, ox = built[quant]
    compare_index(sz, ix, ox, docs16.dim, quant)
    inf = sz.seismic_info(ix)
    assert inf["values_fp16"] == 1
    assert inf["nnz"] == int(np.count_nonzero(docs16.vals))


@pytest.mark.parametrize("quant", [True, False])
@pytest.mark.parametrize("cut,k", [(5, 10), (10_000, 10), (3, 100)])
def test_fp16_exhaustive_parity(sz, small, half, quant, cut, k):
    docs16, built = half
    ix, ox = built[quant]
    q = small["queries"]
    gi, gs = sz.seismic_search(ix, q, k=k, cut=cut, exhaustive=True)
    ref = ox.search(q, k, cut=cut, exhaustive=True)
    check_exact_ids(docs16, q, gi, gs, ref["ids"], ref["scores"])


@pytest.mark.parametrize("cut,hf,wave", [(3, 0.8, 1), (5, 0.9, 1), (10, 0.6, 1), (5, 0.9, 16)])
def test_fp16_pruned_recall_parity(sz, small, half, cut, hf, wave):
    docs16, built = half
    ix, ox = built[True]
    q = small["queries"]
    ei, es = oracle.exact_topk(docs16, q, 10)
    gi, gs, st = sz.seismic_search(ix, q, k=10, cut=cut, heap_factor=hf, wave=wave, persistent=True, stats=True)
    ref = ox.search(q, 10, cut=cut, heap_factor=f32(hf))
    rg = oracle.recall_at_k(docs16, q, gi, es, 10).mean()
    ro = oracle.recall_at_k(docs16, q, ref["ids"], es, 10).mean()
    assert abs(rg - ro) <= 0.005, (rg, ro)
    check_scores_only(docs16, q, gi, gs)
    if wave == 1:
        same = (st[:, sz.STATS.index("blocks_evaluated")] == ref["stats"][:, 2]).mean()
        assert same >= 0.95, same


@pytest.mark.parametrize("shape,group", [(1, 8), (2, 8)])
def test_fp16_launch_shapes(sz, small, half, shape, group):
    docs16, built = half
    ix, ox = built[True]
    q = small["queries"]
    gi, gs = sz.seismic_search(ix, q, k=10, cut=5, exhaustive=True, shape=shape, group=group, persistent=True)
    ref = ox.search(q, 10, cut=5, exhaustive=True)
    check_exact_ids(docs16, q, gi, gs, ref["ids"], ref["scores"])


def test_fp16_knn_expansion_and_exact_search(sz, small, half):
    docs16, built = half
    ix, ox = built[True]
    q = small["queries"]
    knn = oracle.knn_exact(docs16, 8)
    sz.seismic_set_knn(ix, knn)
    gi, gs = sz.seismic_search(ix, q, k=10, cut=2, heap_factor=0.9, use_knn=True)
    ref = ox.search(q, 10, cut=2, heap_factor=f32(0.9), knn=knn)
    ei, es = oracle.exact_topk(docs16, q, 10)
    rg = oracle.recall_at_k(docs16, q, gi, es, 10).mean()
    ro = oracle.recall_at_k(docs16, q, ref["ids"], es, 10).mean()
    assert abs(rg - ro) <= 0.005, (rg, ro)
    check_scores_only(docs16, q, gi, gs)
    xi, xs = sz.seismic_search_exact(ix, q, 10)
    check_exact_ids(docs16, q, xi, xs, ei, es)
    # the graph the library builds from its own fp16 rows is the exact graph of the rounded collection
    sz.seismic_build_knn(ix, 6, exact=True)
    g = sz.seismic_get_knn(ix)
    ref6 = oracle.knn_exact(docs16, 6)
    assert (g == ref6).mean() >= 0.999


def test_fp16_input_rules(sz):
    """A value beyond the fp16 range is refused; one that rounds to 0 is dropped."""
    ip = np.array([0, 2, 4], dtype=np.uint64)
    t = np.array([1, 3, 0, 2], dtype=np.uint16)
    v = np.array([1.0, 1e-9, 2.0, 0.5], dtype=np.float32)
    ix = sz.seismic_build(synth.CSR(ip, t, v, 8), lambda_=10, beta=2, values_fp16=True)
    assert sz.seismic_info(ix)["nnz"] == 3
    ix.close()
    v2 = np.array([1.0, 70000.0, 2.0, 0.5], dtype=np.float32)
    with pytest.raises(sz.SeismicError) as e:
        sz.seismic_build(synth.CSR(ip, t, v2, 8), lambda_=10, beta=2, values_fp16=True)
    assert e.value.code == sz.EINVAL and "fp16" in str(e.value)


def _bits(n):
    return int(np.floor(np.log2(n - 1))) + 1 + (1 if n & (n - 1) == 0 else 0)


def test_packed_graph_roundtrip(sz, small, small_built):
    ix, _ = small_built[True]
    n = small["docs"].n_rows
    rng = np.random.default_rng(3)
    g = rng.integers(0, n, size=(n, 7)).astype(np.uint32)
    g[rng.random(g.shape) < 0.05] = oracle.NONE_ID
    sz.seismic_set_knn(ix, g)
    np.testing.assert_array_equal(sz.seismic_get_knn(ix), g)
    inf = sz.seismic_info(ix)
    assert inf["knn_bits"] == _bits(n) == 13  # 8000 docs: floor(log2 7999) + 1
    assert inf["knn_bytes"] <= 4 * ((n * 7 * 13 + 31) // 32 + 1) + 256
    sz.seismic_set_knn(ix, np.zeros((n, 0), dtype=np.uint32))


def test_packed_graph_power_of_two_collection(sz):
    """N = 1024: ids need 10 bits, the missing-neighbour code an 11th."""
    docs = synth.docs(1024, seed=4, d=500, K=8)
    queries = synth.queries(30, seed=4, d=500, K=8)
    ix = sz.seismic_build(docs, lambda_=100, beta=8, alpha=0.5, quantize_u8=True, seed=1)
    ox = oracle.Index(docs, 100, 8, 0.5, True, seed=1)
    knn = oracle.knn_exact(docs, 5)
    knn[::7, 4] = oracle.NONE_ID
    knn[1, :] = [1023, 0, 1022, oracle.NONE_ID, 1]
    sz.seismic_set_knn(ix, knn)
    assert sz.seismic_info(ix)["knn_bits"] == _bits(1024) == 11
    np.testing.assert_array_equal(sz.seismic_get_knn(ix), knn)
    gi, gs = sz.seismic_search(ix, queries, k=10, cut=2, exhaustive=True, use_knn=True)
    ref = ox.search(queries, 10, cut=2, exhaustive=True, knn=knn)
    check_exact_ids(docs, queries, gi, gs, ref["ids"], ref["scores"])
    ix.close()
