"""seismic_search_noalloc: the search entry point for callers that cannot
allocate device memory while they serve queries (a memory pool fixed at
start-up, no cudaMalloc on the latency path).  It must give the same results
as seismic_search on the same inputs, on two calls in a row (its fixed scratch
array keeps the previous call's contents).  This file is collected last, so a
failure here leaves every other test already run."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
TOL = 1e-5  # the relative score tolerance of the parity tests


@pytest.fixture(scope="module")
def setup():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()
    import paper_2509_24815_gb300 as sz
    docs = synth.docs(6000, seed=21, d=3000, K=16)
    queries = synth.queries(150, seed=21, d=3000, K=16)
    ix = sz.seismic_build(docs, lambda_=150, beta=12, alpha=0.4, quantize_u8=True, seed=3)
    return sz, ix, queries, sz.DeviceCSR.from_host(queries)


@pytest.mark.parametrize("kw", [dict(cut=5, heap_factor=0.9), dict(cut=3, exhaustive=True),
                                dict(cut=4, heap_factor=0.8, wave=4)])
def test_noalloc_matches_search_on_two_calls(setup, kw):
    import torch
    sz, ix, queries, dq = setup
    ref_ids, ref_sc = sz.seismic_search(ix, queries, k=10, persistent=True, shape=1, **kw)
    for _ in range(2):
        ids = torch.full((queries.n_rows, 10), -7, dtype=torch.int32, device="cuda")
        sc = torch.full((queries.n_rows, 10), float("nan"), dtype=torch.float32, device="cuda")
        p = sz.search_params(k=10, persistent=True, shape=1, max_query_nnz=dq.max_row_nnz, **kw)
        sz.seismic_search_noalloc(ix, dq, p, ids, sc)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ids.cpu().numpy().view(np.uint32), ref_ids)
        np.testing.assert_allclose(sc.cpu().numpy(), ref_sc, rtol=TOL, atol=0)


def test_noalloc_rejects_what_needs_memory(setup):
    import torch
    sz, ix, queries, dq = setup
    ids = torch.empty((queries.n_rows, 10), dtype=torch.int32, device="cuda")
    sc = torch.empty((queries.n_rows, 10), dtype=torch.float32, device="cuda")
    p = sz.search_params(k=10, cut=5, heap_factor=0.9)
    s, keep = sz._csr_struct(queries)  # host queries would need a staging copy
    rc = sz._lib.seismic_search_noalloc(ix.handle, sz.ctypes.byref(s), sz.ctypes.byref(p), ids.data_ptr(),
                                        sc.data_ptr(), None)
    assert rc == sz.EINVAL
    s, keep = sz._csr_struct(dq)
    p.max_query_nnz = 0  # measuring the largest query would need a device read-back buffer
    rc = sz._lib.seismic_search_noalloc(ix.handle, sz.ctypes.byref(s), sz.ctypes.byref(p), ids.data_ptr(),
                                        sc.data_ptr(), None)
    assert rc == sz.EINVAL
