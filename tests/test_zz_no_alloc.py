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


# ---------------------------------------------------------------------------
# A collection large enough that the fixed array caps the persistent grid:
# one seen bitmap of ceil(400k / 32) words is 50 KB, so 32 MiB holds 671 of
# them, fewer than the 5 CTAs x 152 SMs the kernel would otherwise launch.
BIG_DOCS, BIG_Q = 400_000, 2000
SCRATCH_BYTES, HEADER_BYTES = 32 << 20, 256


@pytest.fixture(scope="module")
def big():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()
    import paper_2509_24815_gb300 as sz
    docs = synth.docs(BIG_DOCS, seed=23, d=3000, K=16)
    queries = synth.queries(BIG_Q, seed=23, d=3000, K=16, uneven=True)
    ix = sz.seismic_build(docs, lambda_=300, beta=16, alpha=0.4, quantize_u8=True, seed=3)
    yield sz, ix, queries, sz.DeviceCSR.from_host(queries)
    ix.close()


def test_noalloc_allocates_nothing(big):
    """A fresh index has no search workspace; after one warm-up call (which
    looks the fixed array's address up), a further no-allocation call leaves
    the device's free memory unchanged, while seismic_search's first call on
    the same index visibly allocates its seen bitmaps."""
    import torch
    sz, ix, queries, dq = big
    ids = torch.empty((dq.n_rows, 10), dtype=torch.int32, device="cuda")
    sc = torch.empty((dq.n_rows, 10), dtype=torch.float32, device="cuda")
    p = sz.search_params(k=10, cut=5, heap_factor=0.9, persistent=True, shape=1, max_query_nnz=dq.max_row_nnz)
    sz.seismic_search_noalloc(ix, dq, p, ids, sc)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    sz.seismic_search_noalloc(ix, dq, p, ids, sc)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, (free0, free1)
    sz.seismic_search(ix, dq, p, ids_out=ids, scores_out=sc)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] < free1  # the probe does see an allocation


@pytest.mark.parametrize("kw", [dict(cut=5, heap_factor=0.9, wave=16), dict(cut=3, exhaustive=True)])
def test_noalloc_capped_grid_matches_search(big, kw):
    """Here the fixed array, not occupancy, sets the number of persistent CTAs;
    results still equal seismic_search's (full occupancy grid), on two calls."""
    import torch
    sz, ix, queries, dq = big
    words = ((BIG_DOCS + 31) // 32 + 3) & ~3
    assert (SCRATCH_BYTES - HEADER_BYTES) // (4 * words) < 5 * 152  # the cap binds
    p = sz.search_params(k=10, persistent=True, shape=1, max_query_nnz=dq.max_row_nnz, **kw)
    ref_ids, ref_sc = sz.seismic_search(ix, dq, p)
    torch.cuda.synchronize()
    ref_ids, ref_sc = ref_ids.cpu().numpy().view(np.uint32), ref_sc.cpu().numpy()
    for _ in range(2):
        ids = torch.full((dq.n_rows, 10), -7, dtype=torch.int32, device="cuda")
        sc = torch.full((dq.n_rows, 10), float("nan"), dtype=torch.float32, device="cuda")
        sz.seismic_search_noalloc(ix, dq, p, ids, sc)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ids.cpu().numpy().view(np.uint32), ref_ids)
        np.testing.assert_allclose(sc.cpu().numpy(), ref_sc, rtol=TOL, atol=0)


def test_noalloc_refuses_a_collection_beyond_the_array(setup, tmp_path):
    """An index whose seen bitmap alone exceeds the fixed array gets EBUDGET
    before any device work.  The index is the small one saved to a file with
    its document count raised to 300 million (the count sits after the 8-byte
    magic and two u32 fields); the search refuses it on that count alone."""
    import torch
    sz, ix, queries, dq = setup
    path = str(tmp_path / "ix.bin")
    sz.seismic_save(ix, path)
    with open(path, "r+b") as f:
        f.seek(16)
        assert int.from_bytes(f.read(8), "little") == sz.seismic_info(ix)["n_docs"]
        f.seek(16)
        f.write((300_000_000).to_bytes(8, "little"))
    big_ix = sz.seismic_load(path)
    try:
        ids = torch.empty((queries.n_rows, 10), dtype=torch.int32, device="cuda")
        sc = torch.empty((queries.n_rows, 10), dtype=torch.float32, device="cuda")
        p = sz.search_params(k=10, cut=5, heap_factor=0.9, max_query_nnz=dq.max_row_nnz)
        s, keep = sz._csr_struct(dq)
        rc = sz._lib.seismic_search_noalloc(big_ix.handle, sz.ctypes.byref(s), sz.ctypes.byref(p),
                                            ids.data_ptr(), sc.data_ptr(), None)
        assert rc == sz.EBUDGET and "bitmap" in sz.seismic_last_error()
    finally:
        big_ix.close()


def test_noalloc_refuses_the_warp_shape(setup):
    import torch
    sz, ix, queries, dq = setup
    ids = torch.empty((queries.n_rows, 10), dtype=torch.int32, device="cuda")
    sc = torch.empty((queries.n_rows, 10), dtype=torch.float32, device="cuda")
    p = sz.search_params(k=10, cut=5, heap_factor=0.9, shape=2, max_query_nnz=dq.max_row_nnz)
    s, keep = sz._csr_struct(dq)
    rc = sz._lib.seismic_search_noalloc(ix.handle, sz.ctypes.byref(s), sz.ctypes.byref(p), ids.data_ptr(),
                                        sc.data_ptr(), None)
    assert rc == sz.EINVAL and "shape" in sz.seismic_last_error()
