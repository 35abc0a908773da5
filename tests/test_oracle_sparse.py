"""The oracle with A in compressed sparse rows (the text corpora of Section 5 are count matrices).

Storage changes only which terms of u = A x and v = A^T y are formed: the sparse products skip
the stored zeros and add the other terms in the dense order, so every result must equal the
dense oracle's bit for bit (the dense oracle is pinned by the tests of test_oracle_am.py).  The
sparse matrix's repeated entries add up, so a matrix built with repeats must give the result of
its summed dense form.  The bag-of-words generator must give canonical, seeded matrices."""
import numpy as np
import pytest

from paper_1212_4137_gb300 import inputs as I

sp = pytest.importorskip("scipy.sparse")


def _bow(n, p, nnz, seed):
    indptr, indices, data = I.bag_of_words(n, p, nnz, seed, topics=3, topic_words=6)
    return sp.csr_matrix((data.astype(np.float64), indices, indptr), shape=(n, p))


@pytest.mark.parametrize("form", range(1, 9))
def test_sparse_solve_equals_dense_bit_for_bit(oracle, form):
    A = _bow(60, 150, 1500, 1)
    G = I.raw_starts(150, 6, 2)
    kw = dict(s=6.0) if form <= 4 else dict(s=6.0, gamma_target=True, calib=5)
    d = oracle.solve(A.toarray(), form, G, max_iter=40, tol=1e-9, **kw)
    s = oracle.solve(A, form, G, max_iter=40, tol=1e-9, **kw)
    assert s.best == d.best
    for name in ("X", "f", "ev", "F", "iters", "status", "gamma"):
        assert np.array_equal(getattr(s, name), getattr(d, name)), name
    assert np.array_equal(np.nan_to_num(s.F_hist, nan=-1), np.nan_to_num(d.F_hist, nan=-1))


def test_sparse_objective_equals_dense(oracle):
    A = _bow(80, 200, 2000, 3)
    x = I.raw_starts(200, 1, 4)[0]
    x[np.abs(x) < 1.0] = 0.0
    for form in range(1, 9):
        assert oracle.objective(A, form, 0.3, x) == oracle.objective(A.toarray(), form, 0.3, x)


def test_repeated_and_unsorted_entries_add_up(oracle):
    # the same matrix entered with repeats and shuffled columns within rows
    rng = np.random.default_rng(5)
    n, p = 30, 40
    rows, cols, vals = [], [], []
    for i in range(n):
        c = rng.choice(p, 8, replace=True)          # repeats within a row
        rows += [i] * 8
        cols += list(c)
        vals += list(rng.integers(1, 5, 8).astype(float))
    A = sp.coo_matrix((vals, (rows, cols)), shape=(n, p))
    # an explicit CSR with the repeats kept and the columns in input order
    order = np.argsort(np.asarray(rows), kind="stable")
    indptr = np.searchsorted(np.asarray(rows)[order], np.arange(n + 1))
    raw = sp.csr_matrix((np.asarray(vals)[order], np.asarray(cols)[order], indptr), shape=(n, p))
    assert not raw.has_canonical_format
    dense = np.zeros((n, p))
    np.add.at(dense, (np.asarray(rows), np.asarray(cols)), vals)
    G = I.raw_starts(p, 3, 6)
    a = oracle.solve(raw, 1, G, s=5.0, max_iter=20, tol=1e-9)
    b = oracle.solve(dense, 1, G, s=5.0, max_iter=20, tol=1e-9)
    assert np.array_equal(a.X, b.X) and np.array_equal(a.f, b.f)


def test_bag_of_words_is_canonical_and_seeded():
    n, p = 500, 900
    ip, ix, v = I.bag_of_words(n, p, 20000, 7, chunk_docs=128)
    ip2, ix2, v2 = I.bag_of_words(n, p, 20000, 7, chunk_docs=4096)
    assert np.array_equal(ip, ip2) and np.array_equal(ix, ix2) and np.array_equal(v, v2)
    assert ip[0] == 0 and ip[-1] == ix.size and np.all(np.diff(ip) >= 1)
    for i in range(n):
        row = ix[ip[i]:ip[i + 1]]
        assert np.all(np.diff(row) > 0)                 # ascending, no repeats
    assert ix.min() >= 0 and ix.max() < p
    assert np.all(v >= 1) and np.array_equal(v, np.rint(v))
    assert 0.7 * 20000 < ix.size < 1.3 * 20000
    ip3, _, _ = I.bag_of_words(n, p, 20000, 8)
    assert not np.array_equal(ip, ip3)


def test_bag_of_words_plants_topics():
    # a planted topic is a small word set drawn together: about topic_share of the documents hold
    # most of one topic's words, while words of equal popularity co-occur far less
    n, p, share = 2000, 3000, 0.1
    ip, ix, v = I.bag_of_words(n, p, 100000, 9, topics=2, topic_words=8, topic_share=share)
    A = sp.csr_matrix((v, ix, ip), shape=(n, p))
    B = (A > 0).astype(np.int32)
    pairs = (B.T @ B).toarray()
    np.fill_diagonal(pairs, 0)
    # the most frequent co-occurring pairs outside the popularity head are topic pairs: their
    # words are in about share * n documents together
    df = np.asarray(B.sum(axis=0)).ravel()
    mid = np.flatnonzero((df > 0.05 * n) & (df < 0.5 * n))
    sub = pairs[np.ix_(mid, mid)].astype(float)
    expect = np.outer(df[mid], df[mid]) / n           # co-occurrence if drawn independently
    lift = sub / np.maximum(expect, 1.0)
    assert lift.max() > 3.0
