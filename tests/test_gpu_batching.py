"""Batching: the launch autotuner and CUDA-graph capture of the search step.

The result of a search depends on (k, cut, heap_factor, hf_mode, alpha_q, the
kappa expansion) and on `wave`; the kernel shape, lane group, warps per CTA,
L2 prefetch and work-queue order change only the speed (and the fp32
summation order of a score).  So at a fixed wave the autotuner's choice must
return the ids of any other configuration up to near-ties, with scores within
1e-5, and a graph-captured step must return exactly what the same launches
return directly.
"""
import numpy as np
import pytest

import oracle
from test_gpu_parity import check_exact_ids

pytestmark = pytest.mark.gpu

CANDIDATES = [(1, 1, 8, 4, False), (1, 1, 16, 4, True), (1, 8, 8, 4, False), (1, 16, 4, 4, True),
              (1, 32, 16, 4, False)]


def _recall_fn(small, es):
    def fn(i, s):
        return oracle.recall_at_k(small["docs"], small["queries"], i.cpu().numpy().view(np.uint32), es, 10).mean()
    return fn


def test_autotune_choice_equals_fixed_configuration(sz, small, small_built, tmp_path):
    import torch
    from paper_2509_24815_gb300 import autotune
    ix, _ = small_built[True]
    dq = sz.DeviceCSR.from_host(small["queries"])
    _, es = oracle.exact_topk(small["docs"], small["queries"], 10)
    base = dict(k=10, cut=5, heap_factor=0.9)
    cache = str(tmp_path / "tune.json")
    best, table = autotune.autotune(ix, dq, base, recall_fn=_recall_fn(small, es), min_recall=0.0,
                                    candidates=CANDIDATES, reps=2, cache=cache)
    assert best["wave"] == 4 and len(table) == len(CANDIDATES)
    assert all("ms" in t for t in table)
    gi, gs = sz.seismic_search(ix, dq, sz.search_params(max_query_nnz=dq.max_row_nnz, **best))
    ri, rs = sz.seismic_search(ix, dq, sz.search_params(k=10, cut=5, heap_factor=0.9, wave=4, shape=1, group=1,
                                                        cta_warps=8, persistent=True,
                                                        max_query_nnz=dq.max_row_nnz))
    torch.cuda.synchronize()
    ri = ri.cpu().numpy().view(np.uint32)
    rs = rs.cpu().numpy().astype(np.float64)
    check_exact_ids(small["docs"], small["queries"], gi.cpu().numpy().view(np.uint32), gs.cpu().numpy(), ri, rs)
    # the cache answers the same question without timing anything
    best2, table2 = autotune.autotune(ix, dq, base, candidates=CANDIDATES, cache=cache)
    assert best2 == best and table2 == table


def test_autotune_recall_floor(sz, small, small_built):
    from paper_2509_24815_gb300 import autotune
    ix, _ = small_built[True]
    dq = sz.DeviceCSR.from_host(small["queries"])
    _, es = oracle.exact_topk(small["docs"], small["queries"], 10)
    with pytest.raises(RuntimeError):
        autotune.autotune(ix, dq, dict(k=10, cut=5, heap_factor=0.9), recall_fn=_recall_fn(small, es),
                          min_recall=1.01, candidates=CANDIDATES[:2], reps=1)


@pytest.mark.parametrize("use_knn", [False, True])
def test_cuda_graph_replay_equals_direct_launch(sz, small, small_built, use_knn):
    """The whole step (queue reset, work-queue order keys and sort, the
    persistent search, and the expansion) captured once and replayed twice
    gives exactly the direct launch's ids and scores."""
    import torch
    ix, _ = small_built[True]
    if use_knn:
        sz.seismic_set_knn(ix, oracle.knn_exact(small["docs"], 6))
    dq = sz.DeviceCSR.from_host(small["queries"])
    p = sz.search_params(k=10, cut=5, heap_factor=0.9, wave=4, persistent=True, use_knn=use_knn,
                         max_query_nnz=dq.max_row_nnz)
    st = torch.cuda.Stream()
    ids = torch.empty((dq.n_rows, 10), dtype=torch.int32, device="cuda")
    sc = torch.empty((dq.n_rows, 10), dtype=torch.float32, device="cuda")
    sz.seismic_search(ix, dq, p, ids_out=ids, scores_out=sc, stream=st)  # sizes the workspace
    st.synchronize()
    want_i, want_s = ids.clone(), sc.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        sz.seismic_search(ix, dq, p, ids_out=ids, scores_out=sc, stream=st)
    for _ in range(2):
        ids.fill_(-7)
        sc.fill_(float("nan"))
        torch.cuda.synchronize()  # the fills ran on the default stream
        with torch.cuda.stream(st):
            g.replay()
        st.synchronize()
        assert torch.equal(ids, want_i)
        assert torch.equal(sc, want_s)
    if use_knn:
        sz.seismic_set_knn(ix, np.zeros((small["docs"].n_rows, 0), dtype=np.uint32))



@pytest.mark.parametrize("learned", [False, True])
def test_work_queue_orders_change_nothing(sz, small, small_built, learned):
    """Orders 0 (largest term), 1 (input order) and 2 (most lists first) only
    change which CTA takes which query and when: ids and scores are
    bit-identical, with fixed and with learned per-query parameters."""
    import torch
    from paper_2509_24815_gb300 import learn
    ix, _ = small_built[True]
    dq = sz.DeviceCSR.from_host(small["queries"])
    if learned:
        w = learn.init_weights(2)
        w[-2 - 2 * 64:-2] = np.random.default_rng(1).standard_normal(2 * 64).astype(np.float32) * 0.003
        sz.seismic_set_mlp(ix, w)
    out = []
    for order in (0, 1, 2):
        p = sz.search_params(k=10, cut=5, heap_factor=0.9, wave=4, persistent=True, order=order, learned=learned,
                             max_query_nnz=dq.max_row_nnz)
        i, s = sz.seismic_search(ix, dq, p)
        torch.cuda.synchronize()
        out.append((i.cpu(), s.cpu()))
    for i, s in out[1:]:
        assert torch.equal(i, out[0][0]) and torch.equal(s, out[0][1])
