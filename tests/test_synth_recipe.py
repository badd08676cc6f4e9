"""The seeded input generator follows the stated recipe (it stands in for
SPLADE-encoded passages and queries): nnz laws and clips, distinct sorted
terms, the value law |N(0,1)| (1 + exp(-rank/20)), determinism across thread
counts, and disjoint streams."""
import numpy as np

import synth


def _nnz(c):
    return np.diff(c.indptr.astype(np.int64))


def test_document_nnz_law():
    d = synth.docs(20_000, seed=0)
    n = _nnz(d)
    assert n.min() >= 10 and n.max() <= 400
    # round(lognormal) with linear-space mean 120 and sd 40 (clipping barely moves them)
    assert abs(n.mean() - 120.0) < 1.5, n.mean()
    assert abs(n.std() - 40.0) < 1.5, n.std()


def test_query_nnz_laws():
    q = synth.queries(20_000, seed=0)
    n = _nnz(q)
    assert n.min() >= 10 and n.max() <= 150
    assert abs(n.mean() - 40.0) < 1.0, n.mean()
    u = _nnz(synth.queries(20_000, seed=0, uneven=True))
    assert u.min() == 10 and u.max() == 150
    assert abs(u.mean() - 80.0) < 1.0, u.mean()
    h = np.bincount(u - 10, minlength=141)
    assert h.min() > 0.5 * h.mean() and h.max() < 1.5 * h.mean()  # uniform over 10..150


def test_rows_are_sets_of_positive_values():
    d = synth.docs(2000, seed=3, d=5000, K=16)
    for i in range(d.n_rows):
        t, v = d.row(i)
        assert (np.diff(t.astype(np.int64)) > 0).all()  # distinct, ascending terms
        assert (v > 0).all() and np.isfinite(v).all()
        assert t.max(initial=0) < 5000


def test_value_law():
    # |N(0,1)| * (1 + exp(-rank/20)) with rank >= 0: the factor lies in (1, 2]; with
    # Zipf(1) over 30k ranks most entries come from deep ranks, so the mean sits
    # between E|N(0,1)| = 0.798 and twice that, nearer the low end
    v = synth.docs(5000, seed=1).vals.astype(np.float64)
    assert 0.80 < v.mean() < 1.2, v.mean()
    assert np.median(v) > 0.5


def test_deterministic_across_threads_and_streams_disjoint():
    a = synth.docs(3000, seed=5, threads=1)
    b = synth.docs(3000, seed=5, threads=7)
    assert np.array_equal(a.indptr, b.indptr) and np.array_equal(a.terms, b.terms)
    assert np.array_equal(a.vals, b.vals)
    q1 = synth.queries(500, seed=5, uneven=True, stream=synth.TRAIN_STREAM)
    q2 = synth.queries(500, seed=5, uneven=True, stream=synth.HELDOUT_STREAM)
    assert not np.array_equal(q1.terms[:100], q2.terms[:100])
