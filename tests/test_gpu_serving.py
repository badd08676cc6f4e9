"""The continuous-batching server: every request's result is the same alone
(one query per seismic_search call) and in the served mix, where batches of
different k overlap on several streams; plus the incremental API."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()
    import paper_2509_24815_gb300 as sz
    docs = synth.docs(8000, seed=11, d=4000, K=24)
    ix = sz.seismic_build(docs, lambda_=150, beta=12, alpha=0.4, quantize_u8=True, seed=5)
    q = synth.queries(300, seed=11, d=4000, K=24, uneven=True, stream=synth.SERVE_STREAM)
    return sz, ix, q, docs


@pytest.mark.parametrize("rate,streams,batch", [(2e6, 4, 64), (2e3, 2, 256), (5e4, 3, 16)])
def test_served_results_equal_results_alone(env, rate, streams, batch):
    sz, ix, q, docs = env
    from paper_2509_24815_gb300 import serve
    sp = sz.search_params(cut=5, heap_factor=0.9)
    ids, sc, kq, summ = serve.run_trace(ix, q, rate, search=sp, max_batch=batch, streams=streams)
    assert summ["queries"] == q.n_rows and summ["p99_ms"] >= summ["p50_ms"] > 0
    for i in range(q.n_rows):
        k = int(kq[i])
        a, s = sz.seismic_search(ix, q.take([i]), k=k, cut=5, heap_factor=0.9)
        np.testing.assert_array_equal(ids[i, :k], a[0])
        np.testing.assert_array_equal(sc[i, :k], s[0])
        assert (ids[i, k:] == sz.NONE_ID).all()


def test_incremental_api(env):
    sz, ix, q, docs = env
    srv = sz.Server(ix, sz.search_params(cut=4, heap_factor=0.8), max_batch=8, streams=2)
    tickets = []
    for i in range(20):
        t, v = q.row(i)
        tickets.append((srv.submit(t, v, k=10), i))
    got = {}
    for _ in range(100000):
        srv.progress()
        for tk, i in tickets:
            if i in got:
                continue
            r = srv.result(tk, 10)
            if r is not None:
                got[i] = r
        if len(got) == len(tickets):
            break
    assert len(got) == len(tickets)
    for i, (ids, sc, lat) in got.items():
        a, s = sz.seismic_search(ix, q.take([i]), k=10, cut=4, heap_factor=0.8)
        np.testing.assert_array_equal(ids, a[0])
        assert lat > 0
    with pytest.raises(sz.SeismicError):
        srv.submit(np.array([5, 5], np.uint16), np.array([1, 1], np.float32), k=10)  # terms must increase
    with pytest.raises(sz.SeismicError):
        srv.result(123456789, 10)
    srv.close()


@pytest.mark.parametrize("rate,streams,batch,budget", [(5e4, 3, 32, 16), (2e6, 4, 64, 0)])
def test_served_results_equal_alone_with_graph_and_learned_parameters(env, rate, streams, batch, budget):
    """The configuration the benchmark serves: per-query (cut, heap_factor)
    from the index's MLP and the kappa-NN expansion.  Each request's result is
    the same alone and in the mix, also when a small slot budget (16 queries on
    the device at once) holds arrivals back."""
    import oracle
    sz, ix, q, docs = env
    from paper_2509_24815_gb300 import learn, serve
    sz.seismic_set_knn(ix, oracle.knn_exact(docs, 8))
    rng = np.random.default_rng(5)
    r = rng.standard_normal(2 * 64).astype(np.float32)
    feats = sz.seismic_query_features(ix, q)
    for scale in (0.3, 0.03, 0.003, 0.0003):  # the output layer's scale at which predictions vary per query
        w = learn.init_weights(3)
        w[-2 - 2 * 64:-2] = r * np.float32(scale)
        cut, hf = learn.predict(w, feats)
        if len(np.unique(cut)) > 1 and np.ptp(hf) > 0.01:
            break
    assert len(np.unique(cut)) > 1 and np.ptp(hf) > 0.01
    sz.seismic_set_mlp(ix, w)
    sp = sz.search_params(cut=5, heap_factor=0.9, use_knn=True, learned=True)
    srv = sz.Server(ix, sp, max_batch=batch, streams=streams, slot_budget=budget)
    ids, sc, kq, summ = serve.run_trace(ix, q, rate, search=sp, server=srv)
    srv.close()
    assert summ["queries"] == q.n_rows
    for i in range(q.n_rows):
        k = int(kq[i])
        a, s = sz.seismic_search(ix, q.take([i]), k=k, cut=5, heap_factor=0.9, use_knn=True, learned=True)
        np.testing.assert_array_equal(ids[i, :k], a[0])
        np.testing.assert_array_equal(sc[i, :k], s[0])
