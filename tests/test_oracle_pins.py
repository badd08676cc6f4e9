"""Pins for the oracle: each test ties an oracle function to something other
than itself -- the paper's worked example (Figure "set-sketch"), a textbook
computation in numpy on small inputs, a published test vector, or an
invariant the paper states.  CPU only."""
import os

import numpy as np
import pytest

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))
NONE = oracle.NONE_ID


def _csr_from_dense(M, dim=None):
    M = np.asarray(M, dtype=np.float32)
    n, d = M.shape
    indptr = np.zeros(n + 1, dtype=np.uint64)
    terms, vals = [], []
    for i in range(n):
        nz = np.nonzero(M[i])[0]
        terms.extend(nz.tolist())
        vals.extend(M[i, nz].tolist())
        indptr[i + 1] = indptr[i] + len(nz)
    return synth.CSR(indptr, np.array(terms, dtype=np.uint16), np.array(vals, dtype=np.float32), dim or d)


def _random_csr(rng, n, d, nnz_lo, nnz_hi, neg=False):
    rows = []
    for _ in range(n):
        k = int(rng.integers(nnz_lo, nnz_hi + 1))
        t = np.sort(rng.choice(d, size=k, replace=False))
        v = rng.exponential(1.0, size=k).astype(np.float32) + np.float32(1e-3)
        if neg:
            v = v * rng.choice([-1.0, 1.0], size=k).astype(np.float32)
        rows.append((t, v))
    indptr = np.zeros(n + 1, dtype=np.uint64)
    for i, (t, _) in enumerate(rows):
        indptr[i + 1] = indptr[i] + len(t)
    terms = np.concatenate([r[0] for r in rows]).astype(np.uint16)
    vals = np.concatenate([r[1] for r in rows]).astype(np.float32)
    return synth.CSR(indptr, terms, vals, d)


def _np_topk(scores_row, k, allowed=None):
    """Textbook ranking: sort by (score desc, id asc); optionally restrict."""
    ids = np.arange(len(scores_row))
    if allowed is not None:
        ids = ids[allowed]
    order = np.lexsort((ids, -scores_row[ids]))
    top = ids[order][:k]
    out = np.full(k, NONE, dtype=np.uint32)
    out[:len(top)] = top
    return out


# ---------------------------------------------------------------- Figure 4
def _read_fig4():
    rows, mode, alpha = {"INPUT": [], "OUTPUT": []}, None, None
    with open(os.path.join(HERE, "golden", "fig4_set_mss.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("ALPHA"):
                alpha = float(line.split()[1])
            elif line in rows:
                mode = line
            else:
                rows[mode].append([float(x) for x in line.split()])
    return alpha, np.array(rows["INPUT"], dtype=np.float32), np.array(rows["OUTPUT"], dtype=np.float32)


def test_fig4_set_alpha_mss():
    """Set alpha-MSS (proportional lambda_i = ceil(alpha * |L_i|)) on the
    paper's toy matrix: columns without ties match the figure exactly, tied
    columns match as multisets of kept values, column 7 is the figure's error."""
    alpha, A, C = _read_fig4()
    docs = _csr_from_dense(A)
    X = oracle.Index(docs, 0, 1, 1.0, False, 0, lambda_frac=alpha, threads=1)
    for col in range(A.shape[1]):
        L = X.list(col)
        kept = np.zeros(A.shape[0], dtype=np.float32)
        kept[L["doc"]] = L["val"]
        n_col = int((A[:, col] != 0).sum())
        assert len(L["doc"]) == int(np.ceil(alpha * n_col))
        one_based = col + 1
        if one_based in (1, 2, 3, 5, 8):
            np.testing.assert_array_equal(kept, C[:, col])
        elif one_based in (4, 6):
            assert sorted(kept[kept != 0].tolist()) == sorted(C[:, col][C[:, col] != 0].tolist())
        else:  # column 7: figure keeps 2 of ceil(0.4*6)=3; its 2 are among ours
            fig = set(np.nonzero(C[:, col])[0].tolist())
            assert len(fig) == 2 and fig <= set(L["doc"].tolist())


# ---------------------------------------------------------------- splitmix64
def test_splitmix64_published_vector():
    """splitmix64 from state 0: the sequence published with the generator."""
    assert oracle.splitmix64(0, 3) == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


# ---------------------------------------------------------------- exact top-k
@pytest.mark.parametrize("neg", [False, True])
def test_exact_topk_matches_dense_numpy(neg):
    rng = np.random.default_rng(3)
    D = _random_csr(rng, 400, 60, 3, 12, neg=neg)
    Q = _random_csr(rng, 25, 60, 1, 8, neg=neg)
    # one query touching a single rare term: zero-score documents must fill in
    Q2 = _csr_from_dense(np.eye(1, 60, 59, dtype=np.float32) * 2.0)
    for queries in (Q, Q2):
        for k in (1, 10, 37):
            ids, sc = oracle.exact_topk(D, queries, k, threads=2)
            S = queries.to_dense() @ D.to_dense().T
            for i in range(queries.n_rows):
                ref = _np_topk(S[i], k)
                np.testing.assert_array_equal(ids[i], ref)
                np.testing.assert_allclose(sc[i], S[i][ref], rtol=1e-12, atol=1e-12)


def test_exact_topk_fewer_docs_than_k():
    D = _csr_from_dense(np.array([[1.0, 0], [0, 2.0]]))
    Q = _csr_from_dense(np.array([[0, 1.0]]))
    ids, sc = oracle.exact_topk(D, Q, 4, threads=1)
    assert ids[0].tolist() == [1, 0, NONE, NONE]
    assert sc[0, 0] == 2.0 and sc[0, 1] == 0.0 and np.isneginf(sc[0, 2:]).all()


# ---------------------------------------------------------------- alpha-MSS
def test_alpha_mss_hand_examples():
    t = np.array([4, 1, 9], dtype=np.uint16)
    v = np.array([0.25, 0.5, 0.25], dtype=np.float32)  # exact binary fractions
    keep, order = oracle.alpha_mss(t, v, 0.5)
    assert keep == 1 and order.tolist() == [1, 0, 2]  # 0.5 >= 0.5 * 1.0; tie -> lower term
    assert oracle.alpha_mss(t, v, 0.6)[0] == 2         # 0.5 < 0.6 <= 0.75
    assert oracle.alpha_mss(t, v, 0.8)[0] == 3
    assert oracle.alpha_mss(t, v, 1.0)[0] == 3
    # |value| orders the entries; a tie on |value| goes to the lower term
    keep, order = oracle.alpha_mss(np.array([7, 3, 5], np.uint16), np.array([-0.4, 0.4, 0.2], np.float32), 0.4)
    assert keep == 1 and order.tolist() == [1, 0, 2]


def test_alpha_mss_mass_and_minimality():
    rng = np.random.default_rng(11)
    for trial in range(200):
        n = int(rng.integers(1, 60))
        t = np.sort(rng.choice(1000, size=n, replace=False)).astype(np.uint16)
        v = (rng.standard_normal(n) * rng.exponential(1.0, n)).astype(np.float32)
        v[v == 0] = 1.0
        alpha = float(rng.uniform(0.05, 1.0))
        keep, order = oracle.alpha_mss(t, v, alpha)
        a = np.abs(v.astype(np.float64))
        # the order is |v| desc, term asc
        ref = np.lexsort((t, -a))
        np.testing.assert_array_equal(order, ref)
        total = a.sum()
        kept_mass = a[order[:keep]].sum()
        assert kept_mass >= alpha * total - 1e-12 * total
        if keep > 1:
            assert a[order[:keep - 1]].sum() < alpha * total + 1e-12 * total


# ---------------------------------------------------------------- index build
@pytest.fixture(scope="module")
def small():
    docs = synth.docs(1500, seed=5, d=300, K=8)
    queries = synth.queries(60, seed=5, d=300, K=8)
    return docs, queries


@pytest.mark.parametrize("alpha,quant", [(0.4, True), (1.0, False), (0.6, False)])
def test_build_invariants(small, alpha, quant):
    docs, _ = small
    lam, beta = 70, 9
    X = oracle.Index(docs, lam, beta, alpha, quant, seed=17, threads=4)
    Dd = docs.to_dense()
    for t in range(docs.dim):
        L = X.list(t)
        col = Dd[:, t]
        full = np.nonzero(col)[0]
        # lists: the top-lambda postings by (value desc, doc asc)
        ref = full[np.lexsort((full, -col[full]))][:lam]
        np.testing.assert_array_equal(L["doc"], ref)
        n = len(ref)
        if n == 0:
            assert len(L["bcent"]) == 0
            continue
        nb = min(beta, n)
        assert len(L["cent"]) == nb and len(set(L["cent"].tolist())) == nb
        assert set(L["cent"].tolist()) <= set(ref.tolist())
        # assignment: argmax over centroids of the full-vector inner product
        dots = Dd[L["doc"]] @ Dd[L["cent"]].T
        best = dots.max(axis=1)
        chosen = dots[np.arange(n), L["assign"]]
        np.testing.assert_allclose(chosen, best, rtol=1e-12, atol=0)
        for i in range(n):  # ties go to the lower centroid index
            assert L["assign"][i] == np.nonzero(dots[i] >= best[i] * (1 - 1e-12))[0][0]
        # blocks: non-empty clusters in centroid order, a partition, members ascending
        nblk = len(L["bcent"])
        assert (np.diff(L["bcent"]) > 0).all()
        mem = [L["bmem"][L["bptr"][b]:L["bptr"][b + 1]] for b in range(nblk)]
        assert all(len(m) > 0 and (np.diff(m.astype(np.int64)) > 0).all() for m in mem)
        assert sorted(np.concatenate(mem).tolist()) == sorted(ref.tolist())
        for b in range(nblk):
            expect = sorted(L["doc"][L["assign"] == L["bcent"][b]].tolist())
            assert mem[b].tolist() == expect
            # summary: coordinate-wise max over the members (Eq. summary) ...
            phi = Dd[mem[b]].max(axis=0)
            nzt = np.nonzero(phi)[0]
            # ... sketched by its alpha-MSS
            a = np.abs(phi[nzt])
            o = np.lexsort((nzt, -a))
            cs = np.cumsum(a[o])
            j = int(np.argmax(cs >= alpha * cs[-1] * (1 - 1e-15))) + 1
            kept_terms = np.sort(nzt[o[:j]])
            s0, s1 = L["sptr"][b], L["sptr"][b + 1]
            np.testing.assert_array_equal(L["sterm"][s0:s1], kept_terms)
            np.testing.assert_array_equal(L["sval"][s0:s1], phi[kept_terms].astype(np.float32))
            if quant and s1 > s0:
                v = L["sval"][s0:s1].astype(np.float64)
                m, size, code = float(L["qm"][b]), float(L["qsz"][b]), L["scode"][s0:s1].astype(np.float64)
                assert m == v.min()
                if size > 0:
                    vhat = m + code * size
                    assert (code >= 0).all() and (code <= 255).all()
                    assert code[np.argmax(v)] == 255
                    # 256 sub-intervals, codes clamped at 255: the top value sits one
                    # interval above its code; size itself is rounded to fp32
                    err = v - vhat
                    assert (err >= -1e-12 * np.abs(v)).all()
                    assert (err <= size * (1 + 2.0 ** -14)).all()
                    assert (np.delete(err, np.argmax(v)) < size * (1 + 2.0 ** -14)).all()
                else:
                    assert (code == 0).all()


def test_pruning_tie_break_across_the_cut():
    """Values rounded to one decimal tie often, so in many lists the lambda-th
    posting sits inside a run of equal values: each list is still the
    top-lambda by (value desc, doc asc) (reading R2), ties at the cut going to
    the lower document ids."""
    docs = synth.docs(1500, seed=6, d=300, K=8)
    vals = np.maximum(np.round(docs.vals, 1), 0.1).astype(np.float32)
    tied = synth.CSR(docs.indptr, docs.terms, vals, docs.dim)
    lam = 70
    X = oracle.Index(tied, lam, 9, 0.4, True, seed=3, threads=4)
    Dd = tied.to_dense()
    straddle = 0
    for t in range(tied.dim):
        col = Dd[:, t]
        full = np.nonzero(col)[0]
        ref = full[np.lexsort((full, -col[full]))][:lam]
        np.testing.assert_array_equal(X.list(t)["doc"], ref, err_msg=f"list {t}")
        if len(full) > lam:
            left_out = np.setdiff1d(full, ref)
            straddle += int(col[left_out].max() == col[ref[-1]])
    assert straddle > 20, straddle


def test_summary_conservative_at_alpha_one(small):
    """Eq. summary: with alpha = 1 and no quantisation, <q, phi(B)> >= <q, u_j>
    for every member j and any non-negative q."""
    docs, _ = small
    X = oracle.Index(docs, 70, 9, 1.0, False, seed=3, threads=4)
    Dd = docs.to_dense()
    rng = np.random.default_rng(0)
    qs = rng.exponential(1.0, size=(20, docs.dim)) * (rng.random((20, docs.dim)) < 0.2)
    for t in range(0, docs.dim, 7):
        L = X.list(t)
        for b in range(len(L["bcent"])):
            s0, s1 = L["sptr"][b], L["sptr"][b + 1]
            phi = np.zeros(docs.dim)
            phi[L["sterm"][s0:s1]] = L["sval"][s0:s1]
            mem = L["bmem"][L["bptr"][b]:L["bptr"][b + 1]]
            assert (qs @ phi >= (qs @ Dd[mem].T).max(axis=1) - 1e-9).all()


def test_quantisation_constant_block():
    # a one-document list: its block summary is constant per kept value set
    A = np.zeros((3, 4), dtype=np.float32)
    A[0, 0] = 0.5
    A[0, 1] = 0.5
    X = oracle.Index(_csr_from_dense(A), 0, 4, 1.0, True, seed=0, threads=1)
    L = X.list(0)
    assert L["qsz"][0] == 0.0 and (L["scode"] == 0).all() and L["qm"][0] == np.float32(0.5)


# ---------------------------------------------------------------- kappa-NN
def test_knn_exact_matches_numpy(small):
    docs, _ = small
    sub = docs.slice(0, 300)
    nb = oracle.knn_exact(sub, 5, threads=4)
    S = sub.to_dense() @ sub.to_dense().T
    for u in range(sub.n_rows):
        allowed = np.ones(sub.n_rows, bool)
        allowed[u] = False
        np.testing.assert_array_equal(nb[u], _np_topk(S[u], 5, allowed))


def test_knn_refine_brute_force(small):
    """One neighbour-of-neighbour pass against dense numpy on a tiny case: the
    candidates of u are its list and its neighbours' lists (self loops and
    missing entries in the input included), u excluded; the new list is their
    kappa best by (score desc, id asc)."""
    docs, _ = small
    sub = docs.slice(0, 120)
    rng = np.random.default_rng(9)
    g = rng.integers(0, sub.n_rows, size=(sub.n_rows, 4)).astype(np.uint32)
    g[rng.random(g.shape) < 0.15] = NONE
    g[3, 0] = 3  # a self loop in the input
    out = oracle.knn_refine(sub, g, threads=3)
    S = sub.to_dense() @ sub.to_dense().T
    for u in range(sub.n_rows):
        cand = set(int(x) for x in g[u] if x != NONE)
        for v in list(cand):
            cand.update(int(x) for x in g[v] if x != NONE)
        cand.discard(u)
        allowed = np.zeros(sub.n_rows, bool)
        allowed[list(cand)] = True
        np.testing.assert_array_equal(out[u], _np_topk(S[u], 4, allowed), err_msg=f"row {u}")


def test_knn_refine_keeps_the_exact_graph_and_improves_others(small):
    """The exact graph is a fixed point (its lists are among the candidates and
    beat every other document); on any other graph each rank's score never
    drops (the old list is among the candidates)."""
    docs, _ = small
    sub = docs.slice(0, 400)
    exact = oracle.knn_exact(sub, 6, threads=4)
    np.testing.assert_array_equal(oracle.knn_refine(sub, exact, threads=4), exact)
    rng = np.random.default_rng(2)
    g = np.stack([rng.permutation(np.delete(np.arange(sub.n_rows), u))[:6] for u in range(sub.n_rows)])
    g = g.astype(np.uint32)
    S = sub.to_dense() @ sub.to_dense().T
    g2 = oracle.knn_refine(sub, g, threads=4)
    old = np.sort(np.take_along_axis(S, g.astype(np.int64), 1), axis=1)[:, ::-1]
    new = np.take_along_axis(S, g2.astype(np.int64), 1)
    assert np.all(new >= old - 1e-12)
    assert (new > old + 1e-12).any()


# ---------------------------------------------------------------- search
def test_exhaustive_equals_brute_force_on_positive_scores(small):
    """With every query term traversed and unpruned lists, exhaustive Seismic is
    brute-force MIPS over the documents that share a term with q."""
    docs, queries = small
    X = oracle.Index(docs, 0, 9, 0.4, True, seed=1, threads=4)
    S = queries.to_dense() @ docs.to_dense().T
    for k in (1, 10):
        res = X.search(queries, k, cut=10_000, exhaustive=True, threads=4)
        for i in range(queries.n_rows):
            ref = _np_topk(S[i], k, allowed=S[i] > 0)
            np.testing.assert_array_equal(res["ids"][i], ref)
            ok = ref != NONE
            np.testing.assert_allclose(res["scores"][i][ok], S[i][ref[ok]], rtol=1e-12)


@pytest.mark.parametrize("cut", [1, 3, 8])
def test_safe_pruning_equals_exhaustive(small, cut):
    """alpha = 1, no quantisation, heap_factor = 1: summaries bound every member
    (Eq. summary), so block skipping is rank-safe in both skip forms."""
    docs, queries = small
    X = oracle.Index(docs, 90, 9, 1.0, False, seed=2, threads=4)
    ex = X.search(queries, 10, cut=cut, exhaustive=True, threads=4)
    for mode in (0, 1):
        pr = X.search(queries, 10, cut=cut, heap_factor=1.0, hf_mode=mode, threads=4)
        np.testing.assert_array_equal(pr["ids"], ex["ids"])
        np.testing.assert_array_equal(pr["scores"], ex["scores"])
        assert pr["stats"][:, 3].sum() > 0  # blocks were actually skipped


def test_hand_worked_visiting_order():
    """Two one-document blocks in list t0 (beta = 2 makes each document its own
    centroid).  q = {t0: 1, t1: 1}.  Summaries (alpha = 1): block(doc0) =
    {t0: 1, t1: 5} scores 6, block(doc1) = {t0: 2, t2: 5} scores 2.  Blocks go
    in decreasing summary score: doc0's block first (theta = <q, doc0> = 6),
    then doc1's block is skipped since 2 < 1.0 * 6."""
    A = np.array([[1.0, 5.0, 0.0], [2.0, 0.0, 5.0]], dtype=np.float32)
    X = oracle.Index(_csr_from_dense(A), 0, 2, 1.0, False, seed=0, threads=1)
    L = X.list(0)
    blocks = {int(L["bmem"][L["bptr"][b]]): b for b in range(2)}
    r = X.block_scores(np.array([0, 1]), np.array([1.0, 1.0], np.float32), 0)
    assert r[blocks[0]] == 6.0 and r[blocks[1]] == 2.0
    Q = _csr_from_dense(np.array([[1.0, 1.0, 0.0]], dtype=np.float32))
    res = X.search(Q, 1, cut=1, heap_factor=1.0, threads=1)
    assert res["ids"][0].tolist() == [0] and res["scores"][0, 0] == 6.0
    st = dict(zip(oracle.STAT_NAMES, res["stats"][0].tolist()))
    assert st["blocks_scored"] == 2 and st["blocks_evaluated"] == 1 and st["blocks_skipped"] == 1
    assert st["docs"] == 1


def test_quantised_block_scores_bound(small):
    """Scalar quantisation (Section 4.1.3) only lowers a summary value, by less
    than one sub-interval: for q >= 0, 0 <= <q, S_b> - r_b <= size_b * sum_i q_i
    over the block's kept terms, where S_b holds the unquantised values."""
    docs, queries = small
    Xq = oracle.Index(docs, 70, 9, 0.4, True, seed=8, threads=4)
    for qi in range(0, queries.n_rows, 6):
        qt, qv = queries.row(qi)
        qd = np.zeros(docs.dim)
        qd[qt] = qv
        for t in qt[:4]:
            L = Xq.list(int(t))
            r = Xq.block_scores(qt, qv, int(t))
            for b in range(len(L["bcent"])):
                s0, s1 = L["sptr"][b], L["sptr"][b + 1]
                exact = float(qd[L["sterm"][s0:s1]] @ L["sval"][s0:s1].astype(np.float64))
                slack = float(L["qsz"][b]) * float(qd[L["sterm"][s0:s1]].sum()) * (1 + 2.0 ** -14)
                assert -1e-9 <= exact - r[b] <= slack + 1e-9


def test_skip_forms_and_direction(small):
    docs, queries = small
    X = oracle.Index(docs, 90, 9, 0.4, True, seed=2, threads=4)
    a = X.search(queries, 10, cut=5, heap_factor=1.0, hf_mode=0, threads=4)
    b = X.search(queries, 10, cut=5, heap_factor=1.0, hf_mode=1, threads=4)
    np.testing.assert_array_equal(a["ids"], b["ids"])  # hf = 1: r < theta either way
    lo = X.search(queries, 10, cut=5, heap_factor=0.5, threads=4)
    # r < hf*theta skips less as hf falls; r < theta/hf skips more
    lo1 = X.search(queries, 10, cut=5, heap_factor=0.5, hf_mode=1, threads=4)
    assert lo["stats"][:, 3].sum() < a["stats"][:, 3].sum() < lo1["stats"][:, 3].sum()


def test_knn_expansion_semantics(small):
    """Final result = top-k of S_+ = union over u in S of {u} and N(u), where S is
    the heap after the list traversal (Algorithm lines for the expansion)."""
    docs, queries = small
    X = oracle.Index(docs, 40, 9, 0.4, True, seed=4, threads=4)
    knn = oracle.knn_exact(docs, 6, threads=4)
    res = X.search(queries, 10, cut=2, heap_factor=1.0, knn=knn, threads=4, want_phase1=True)
    S = queries.to_dense() @ docs.to_dense().T
    grew = 0
    for i in range(queries.n_rows):
        p1 = res["phase1"][i]
        p1 = p1[p1 != NONE]
        cand = set(p1.tolist())
        for u in p1:
            cand |= set(int(v) for v in knn[u] if v != NONE)
        allowed = np.zeros(docs.n_rows, bool)
        allowed[list(cand)] = True
        np.testing.assert_array_equal(res["ids"][i], _np_topk(S[i], 10, allowed))
        grew += int(set(res["ids"][i].tolist()) != set(res["phase1"][i].tolist()))
    assert grew > 0


def test_padding_and_zero_query():
    A = np.zeros((4, 5), dtype=np.float32)
    A[0, 1] = 1.0
    A[2, 1] = 3.0
    A[3, 4] = 1.0
    docs = _csr_from_dense(A)
    X = oracle.Index(docs, 0, 2, 0.4, False, seed=0, threads=1)
    Q = _csr_from_dense(np.array([[0, 2.0, 0, 0, 0], [0, 0, 0, 0, 0]], dtype=np.float32))
    r = X.search(Q, 3, cut=3, heap_factor=0.8, threads=1)
    assert r["ids"][0].tolist() == [2, 0, NONE] and r["scores"][0, :2].tolist() == [6.0, 2.0]
    assert (r["ids"][1] == NONE).all() and np.isneginf(r["scores"][1]).all()


def test_alpha_q_sketch_of_query(small):
    """alpha_q = 1 keeps every query term (the full alpha-MSS), which for
    non-negative queries is the same traversal as cut >= nnz(q)."""
    docs, queries = small
    X = oracle.Index(docs, 90, 9, 0.4, True, seed=2, threads=4)
    a = X.search(queries, 10, alpha_q=1.0, heap_factor=0.9, threads=4)
    b = X.search(queries, 10, cut=10_000, heap_factor=0.9, threads=4)
    np.testing.assert_array_equal(a["ids"], b["ids"])
    c = X.search(queries, 10, alpha_q=0.3, heap_factor=0.9, threads=4)
    assert c["stats"][:, 0].sum() < a["stats"][:, 0].sum()


def test_recall_definition():
    """accuracy@k = |S cap S'| / k (Definition ann-accuracy), with ties at the
    k-th exact score counted as hits."""
    A = np.array([[3.0], [2.0], [2.0], [1.0]], dtype=np.float32)
    docs = _csr_from_dense(A)
    Q = _csr_from_dense(np.array([[1.0]], dtype=np.float32))
    ei, es = oracle.exact_topk(docs, Q, 2, threads=1)
    assert ei[0].tolist() == [0, 1]
    r = oracle.recall_at_k(docs, Q, np.array([[0, 2]], dtype=np.uint32), es, 2)
    assert r[0] == 1.0  # doc 2 ties doc 1
    r = oracle.recall_at_k(docs, Q, np.array([[3, 0]], dtype=np.uint32), es, 2)
    assert r[0] == 0.5
    r = oracle.recall_at_k(docs, Q, np.array([[0, NONE]], dtype=np.uint32), es, 2)
    assert r[0] == 0.5


def test_pair_dots_matches_numpy_on_interleaved_queries():
    """or_pair_dots, the checker behind every GPU score and every recall, against
    a dense numpy product (textbook inner product, fp64) on several queries
    whose pairs come unsorted and interleaved (a query revisited after others),
    with repeated pairs, mixed-sign values and ids past the collection (-inf)."""
    rng = np.random.default_rng(17)
    docs = _random_csr(rng, 60, 90, 1, 25, neg=True)
    queries = _random_csr(rng, 9, 90, 1, 30, neg=True)
    D, Q = docs.to_dense(), queries.to_dense()
    qi = rng.integers(0, queries.n_rows, size=400).astype(np.uint64)
    di = rng.integers(0, docs.n_rows + 5, size=400).astype(np.uint32)  # a few ids past the end
    qi[:6] = [3, 0, 3, 8, 8, 0]
    di[:6] = [7, 7, 7, 2, 2, 61]
    got = oracle.pair_dots(docs, queries, qi, di)
    q64, d64 = qi.astype(np.int64), di.astype(np.int64)
    ok = d64 < docs.n_rows
    want = np.full(len(qi), -np.inf)
    want[ok] = np.einsum("ij,ij->i", Q[q64[ok]], D[d64[ok]])
    assert np.all(np.isneginf(got[~ok]))
    np.testing.assert_allclose(got[ok], want[ok], rtol=1e-12, atol=1e-12)
    assert got[0] == got[2]  # the same pair, with another query scored in between
