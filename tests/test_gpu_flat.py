"""GPU parity of the chunk-flattened CTA scoring path (group = 1) against the
oracle, with the same bars as the other launch shapes: exhaustive ids and
scores (1e-5 relative), pruned recall within 0.005 of the oracle's at wave 1
and the same blocks evaluated for >= 95 % of queries, kappa expansion,
alpha_q, both deduplication sets, waves and learned parameters."""
import numpy as np
import pytest

import oracle
import synth
from test_gpu_parity import NONE, check_exact_ids, check_scores_only, f32

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("quant", [True, False])
@pytest.mark.parametrize("cut,k,warps", [(1, 10, 8), (5, 10, 8), (10_000, 10, 4), (5, 1, 16), (5, 100, 8)])
def test_flat_exhaustive_parity(sz, small, small_built, quant, cut, k, warps):
    ix, ox = small_built[quant]
    for persistent in (False, True):
        gi, gs = sz.seismic_search(ix, small["queries"], k=k, cut=cut, exhaustive=True, shape=1, group=1,
                                   cta_warps=warps, persistent=persistent)
        ref = ox.search(small["queries"], k, cut=cut, exhaustive=True)
        check_exact_ids(small["docs"], small["queries"], gi, gs, ref["ids"], ref["scores"])


@pytest.mark.parametrize("quant", [True, False])
@pytest.mark.parametrize("cut,hf", [(3, 0.8), (5, 0.9), (10, 1.0)])
def test_flat_pruned_parity(sz, small, small_built, quant, cut, hf):
    ix, ox = small_built[quant]
    docs, queries = small["docs"], small["queries"]
    ei, es = oracle.exact_topk(docs, queries, 10)
    gi, gs, gst = sz.seismic_search(ix, queries, k=10, cut=cut, heap_factor=hf, shape=1, group=1, stats=True)
    ref = ox.search(queries, 10, cut=cut, heap_factor=f32(hf))
    rg = oracle.recall_at_k(docs, queries, gi, es, 10).mean()
    ro = oracle.recall_at_k(docs, queries, ref["ids"], es, 10).mean()
    assert abs(rg - ro) <= 0.005, (rg, ro)
    same = (gst[:, sz.STATS.index("blocks_evaluated")] == ref["stats"][:, 2]).mean()
    assert same >= 0.95, same
    same_docs = (gst[:, sz.STATS.index("docs")] == ref["stats"][:, 4]).mean()
    assert same_docs >= 0.95, same_docs
    check_scores_only(docs, queries, gi, gs)


def test_flat_pruned_parity_c1(sz, c1):
    gi, gs = sz.seismic_search(c1["ix"], c1["queries"], k=10, cut=5, heap_factor=0.9, shape=1, group=1,
                               persistent=True)
    ref = c1["ox"].search(c1["queries"], 10, cut=5, heap_factor=f32(0.9))
    rg = oracle.recall_at_k(c1["docs"], c1["queries"], gi, c1["es"], 10).mean()
    ro = oracle.recall_at_k(c1["docs"], c1["queries"], ref["ids"], c1["es"], 10).mean()
    assert abs(rg - ro) <= 0.005, (rg, ro)
    check_scores_only(c1["docs"], c1["queries"], gi, gs)
    gi, gs = sz.seismic_search(c1["ix"], c1["queries"], k=10, cut=10, exhaustive=True, shape=1, group=1,
                               persistent=True)
    ref = c1["ox"].search(c1["queries"], 10, cut=10, exhaustive=True)
    check_exact_ids(c1["docs"], c1["queries"], gi, gs, ref["ids"], ref["scores"])


def test_flat_knn_alpha_q_waves(sz, small, small_built):
    ix, ox = small_built[True]
    docs, queries = small["docs"], small["queries"]
    ei, es = oracle.exact_topk(docs, queries, 10)
    knn = oracle.knn_exact(docs, 10)
    sz.seismic_set_knn(ix, knn)
    gi, gs = sz.seismic_search(ix, queries, k=10, cut=2, heap_factor=0.9, use_knn=True, shape=1, group=1)
    ref = ox.search(queries, 10, cut=2, heap_factor=f32(0.9), knn=knn)
    assert abs(oracle.recall_at_k(docs, queries, gi, es, 10).mean()
               - oracle.recall_at_k(docs, queries, ref["ids"], es, 10).mean()) <= 0.005
    check_scores_only(docs, queries, gi, gs)
    gi, _, st = sz.seismic_search(ix, queries, k=10, alpha_q=0.4, heap_factor=0.9, shape=1, group=1, stats=True)
    ref = ox.search(queries, 10, alpha_q=f32(0.4), heap_factor=f32(0.9))
    np.testing.assert_array_equal(st[:, 0], ref["stats"][:, 0])
    assert abs(oracle.recall_at_k(docs, queries, gi, es, 10).mean()
               - oracle.recall_at_k(docs, queries, ref["ids"], es, 10).mean()) <= 0.005
    for wave in (4, 16):
        gi, gs = sz.seismic_search(ix, queries, k=10, cut=5, heap_factor=0.9, wave=wave, shape=1, group=1,
                                   persistent=True)
        ref = ox.search(queries, 10, cut=5, heap_factor=f32(0.9))
        assert abs(oracle.recall_at_k(docs, queries, gi, es, 10).mean()
                   - oracle.recall_at_k(docs, queries, ref["ids"], es, 10).mean()) <= 0.005
        # the same wave on the lane-group path gives the same ids (up to near-ties)
        a, sa = sz.seismic_search(ix, queries, k=10, cut=5, heap_factor=0.9, wave=wave, shape=1, group=8,
                                  persistent=True)
        check_exact_ids(docs, queries, gi, gs, a, sa.astype(np.float64), tol=2e-5)


def test_flat_edges_and_limits(sz, small, small_built):
    ix, ox = small_built[True]
    d = small["docs"].dim
    q = synth.CSR(np.array([0, 2, 2, 5], np.uint64), np.array([3, 9, 1, 2, 3], np.uint16),
                  np.array([0.0, 0.0, 0.0, 1.5, 0.0], np.float32), d)
    gi, gs = sz.seismic_search(ix, q, k=7, cut=3, heap_factor=0.8, shape=1, group=1)
    assert (gi[0] == NONE).all() and (gi[1] == NONE).all() and np.isneginf(gs[:2]).all()
    ref = ox.search(q, 7, cut=3, heap_factor=f32(0.8))
    check_exact_ids(small["docs"], q, gi, gs, ref["ids"], ref["scores"])
    # long queries (hundreds of nonzeros) and k past the candidate buffer
    rng = np.random.default_rng(4)
    for n in (255, 600):
        t = np.sort(rng.choice(d, size=n, replace=False)).astype(np.uint16)
        qq = synth.CSR(np.array([0, n], np.uint64), t, rng.random(n).astype(np.float32) + 0.1, d)
        gi, gs = sz.seismic_search(ix, qq, k=300, cut=5, exhaustive=True, shape=1, group=1)
        ref = ox.search(qq, 300, cut=5, exhaustive=True)
        check_exact_ids(small["docs"], qq, gi, gs, ref["ids"], ref["scores"])
    # bad input is refused and the index stays usable
    bad = synth.CSR(np.array([0, 1], np.uint64), np.array([d], np.uint16), np.array([1], np.float32), d)
    with pytest.raises(sz.SeismicError):
        sz.seismic_search(ix, bad, k=10, cut=5, shape=1, group=1)
    gi, _ = sz.seismic_search(ix, small["queries"], k=10, cut=5, heap_factor=0.8, shape=1, group=1)
    assert gi.shape == (small["queries"].n_rows, 10)


def test_flat_learned(sz, small, small_built):
    from oracle import mlp
    ix, _ = small_built[True]
    q = small["queries"]
    sz.seismic_set_mlp(ix, (mlp.init(9) * 0.3).astype(np.float32))
    a, sa = sz.seismic_search(ix, q, k=10, cut=5, heap_factor=0.8, learned=True, shape=1, group=8)
    b, sb = sz.seismic_search(ix, q, k=10, cut=5, heap_factor=0.8, learned=True, shape=1, group=1)
    check_exact_ids(small["docs"], q, b, sb, a, sa.astype(np.float64), tol=2e-5)
