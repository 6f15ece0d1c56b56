"""The seeded generators produce the documented shapes and structure."""

import numpy as np
import pytest

import workloads


def _check_csc(p):
    assert p.col_ptr.dtype == np.int64 and p.row_idx.dtype == np.int32 and p.val.dtype == np.float64
    assert p.col_ptr[0] == 0 and np.all(np.diff(p.col_ptr) >= 0) and p.col_ptr[-1] == p.row_idx.size
    for j in range(p.k):
        r = p.row_idx[p.col_ptr[j]:p.col_ptr[j + 1]]
        assert np.all(np.diff(r) > 0) and (r.size == 0 or (r[0] >= 0 and r[-1] < p.n))


def test_config1_shape_and_values():
    p = workloads.config1("logistic")
    assert (p.n, p.k, p.nnz) == (2000, 5000, 100_000)
    assert set(np.unique(p.val)) == {-1.0, 1.0}
    assert set(np.unique(p.y)) == {-1.0, 1.0}
    assert (p.w_star != 0).sum() == 50
    assert np.all(np.diff(p.col_ptr) == 20)
    _check_csc(p)
    q = workloads.config1("logistic")
    assert p.sha256() == q.sha256()  # seeded
    s = workloads.config1("squared")
    assert s.y.dtype == np.float64 and len(np.unique(s.y)) > 100


def test_zipf_counts_hit_the_target():
    c = workloads.synthetic.zipf_counts(4_000_000, 200_000_000, cap=50_000)
    assert abs(c.sum() - 2e8) <= 0.005 * 2e8
    assert c.max() == 50_000 and c.min() >= 1
    assert 400 <= (c == 50_000).sum() <= 800


def test_scaled_zipf_problem_structure():
    p = workloads.config2_scaled(0.002)
    _check_csc(p)
    counts = p.col_nnz()
    assert counts.min() >= 1
    norms = np.sqrt(np.add.reduceat(p.val ** 2, p.col_ptr[:-1]))
    np.testing.assert_allclose(norms, 1.0, rtol=1e-12)
    assert np.all(p.val > 0)
    assert set(np.unique(p.y)) <= {-1.0, 1.0}


def test_distinct_rows_are_uniform_without_replacement():
    rng = np.random.default_rng(0)
    counts = np.array([5, 0, 10, 10])
    rows = workloads.synthetic._distinct_rows(10, counts, rng)
    assert rows[5:15].tolist() == list(range(10))
    assert rows[15:].tolist() == list(range(10))
    with pytest.raises(ValueError):
        workloads.synthetic._distinct_rows(3, np.array([4]), rng)


def test_cv_folds_are_balanced_and_seeded():
    f = workloads.cv_folds(1003, 5, seed=4)
    assert f.dtype == np.uint8 and set(np.unique(f)) == set(range(5))
    assert np.bincount(f).max() - np.bincount(f).min() <= 1
    np.testing.assert_array_equal(f, workloads.cv_folds(1003, 5, seed=4))


def test_row_subset_is_the_dense_row_selection():
    # trailing and inner empty columns, a row subset that empties some columns
    X = np.zeros((7, 6))
    X[0, 0], X[3, 0], X[1, 2], X[6, 2], X[2, 3], X[5, 3] = 1.0, -2.0, 0.5, 1.5, 3.0, -1.0
    y = np.arange(7.0)
    p = workloads.csc_from_dense(X, y, "squared")
    rows = np.array([5, 0, 2, 6])
    s = workloads.row_subset(p, rows)
    np.testing.assert_array_equal(s.to_dense(), X[np.sort(rows)])
    np.testing.assert_array_equal(s.y, y[np.sort(rows)])
    assert s.col_ptr[-1] == s.nnz == int(np.count_nonzero(X[np.sort(rows)]))


def test_lambda_grid_is_log_spaced():
    g = workloads.lambda_grid(2.0, 32, 1e-3)
    assert g.size == 32 and g[0] == 2.0 and abs(g[-1] - 2e-3) < 1e-15
    np.testing.assert_allclose(g[1:] / g[:-1], (1e-3) ** (1 / 31))


def test_generators_draw_no_repeated_row_sets():
    # duplicate columns would make the l1 minimiser non-unique: every
    # generator redraws a column whose row set repeats a lower-index column's
    dup = workloads.synthetic._duplicate_columns
    cp = np.array([0, 1, 3, 4, 6, 9, 10], np.int64)
    ri = np.array([5, 1, 2, 5, 1, 2, 0, 1, 2, 7], np.int32)
    assert dup(10, cp, ri).tolist() == [2, 3]  # planted repeats of columns 0 and 1
    for p in (workloads.config1(), workloads.config3("ones"), workloads.config2_scaled(0.002),
              workloads.uniform_problem(50, 40, 1, values="ones", n_planted=5, seed=3),
              workloads.zipf_problem(5000, 2000, 6000, cap=100, n_planted=5, seed=2)):
        _check_csc(p)
        assert dup(p.n, p.col_ptr, p.row_idx).size == 0, p.name
    # 40 one-entry columns in 50 rows: the first draw repeats rows, the redraws do not
    p = workloads.uniform_problem(50, 40, 1, values="ones", n_planted=5, seed=3)
    assert np.unique(p.row_idx).size == 40
    with pytest.raises(ValueError):
        workloads.uniform_problem(10, 11, 1, values="ones", n_planted=2, seed=0)


def test_no_redraw_leaves_the_first_draw():
    # without repeated row sets the generator's bytes are those of the plain draw
    counts = np.full(300, 20, np.int64)
    a = workloads.synthetic._distinct_rows(2000, counts, workloads.synthetic._rng(5))
    b = workloads.synthetic._distinct_columns(2000, counts, workloads.synthetic._rng(5))
    np.testing.assert_array_equal(a, b)
