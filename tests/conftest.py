import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 (sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: larger CPU-only case")


@pytest.fixture(scope="session")
def threads():
    return min(16, os.cpu_count() or 1)


# ------------------------------------------------------------------ GPU fixtures (shared by the GPU test files)
def _mk(n_docs, n_q, d, K, seed=11):
    import synth
    return synth.docs(n_docs, seed=seed, d=d, K=K), synth.queries(n_q, seed=seed, d=d, K=K)


@pytest.fixture(scope="session")
def sz():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    import __graft_entry__
    __graft_entry__.build()
    import paper_2509_24815_gb300 as m
    return m


@pytest.fixture(scope="session")
def small(sz):
    docs, queries = _mk(8000, 200, 4000, 24)
    return dict(docs=docs, queries=queries, lam=150, beta=12, alpha=0.4)


@pytest.fixture(scope="session")
def small_built(sz, small):
    import oracle
    out = {}
    for quant in (True, False):
        ix = sz.seismic_build(small["docs"], lambda_=small["lam"], beta=small["beta"], alpha=small["alpha"],
                              quantize_u8=quant, seed=5, keep_full_lists=True, keep_block_summaries=True)
        ox = oracle.Index(small["docs"], small["lam"], small["beta"], small["alpha"], quant, seed=5)
        out[quant] = (ix, ox)
    return out


@pytest.fixture(scope="session")
def c1(sz):
    """The tiny Seismic configuration: 100k docs, lambda=2000, beta=100,
    alpha=0.4, fp32 summaries, 1k queries (seed 0)."""
    import oracle
    import synth
    docs = synth.docs(100_000, seed=0)
    queries = synth.queries(1000, seed=0)
    ix = sz.seismic_build(docs, lambda_=2000, beta=100, alpha=0.4, quantize_u8=False, seed=0,
                          keep_full_lists=True, keep_block_summaries=True)
    ox = oracle.Index(docs, 2000, 100, 0.4, False, seed=0)
    ei, es = oracle.exact_topk(docs, queries, 10)
    return dict(docs=docs, queries=queries, ix=ix, ox=ox, ei=ei, es=es)


