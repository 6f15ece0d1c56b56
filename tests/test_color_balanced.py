"""The library's balanced colouring (gencd_color_balanced_csc, host code, no
GPU) against the oracle's (R13): colours are integers, so bit-exact."""

import numpy as np
import pytest

import oracle
import workloads


@pytest.fixture(scope="module")
def gb():
    from paper_1206_6409_gb300 import binding, build

    build.build()
    binding.lib()
    return binding


def _with_empty_columns(p):
    counts = np.concatenate([[0], np.diff(p.col_ptr)[:5], [0, 0], np.diff(p.col_ptr)[5:], [0]])
    col_ptr = np.zeros(counts.size + 1, np.int64)
    np.cumsum(counts, out=col_ptr[1:])
    return workloads.Problem(p.n, counts.size, col_ptr, p.row_idx, p.val, p.y, p.loss, np.zeros(counts.size))


CASES = {
    "cfg1": lambda: workloads.config1("squared"),
    "zipf": lambda: workloads.zipf_problem(2000, 5000, 60_000, cap=400, n_planted=10, seed=2),
    "empty-columns": lambda: _with_empty_columns(workloads.uniform_problem(300, 200, 7, seed=5)),
}


@pytest.mark.parametrize("cap", [0, 1, 7, 10**9])
@pytest.mark.parametrize("name", list(CASES))
def test_balanced_colouring_equals_the_oracle(gb, name, cap):
    p = CASES[name]()
    want, nc_want = oracle.Oracle(p).color_balanced(cap)
    got, nc = gb.gencd_color_balanced_csc(p.n, p.k, p.col_ptr, p.row_idx, cap)
    assert nc == nc_want
    np.testing.assert_array_equal(got, want)


def test_balanced_colouring_rejects_malformed_csc(gb):
    with pytest.raises(gb.GencdError):
        gb.gencd_color_balanced_csc(3, 2, np.array([0, 2, 1]), np.array([0, 1], np.int32))
    with pytest.raises(gb.GencdError):
        gb.gencd_color_balanced_csc(3, 1, np.array([0, 2]), np.array([1, 1], np.int32))
    with pytest.raises(gb.GencdError):
        gb.gencd_color_balanced_csc(3, 1, np.array([0, 1]), np.array([3], np.int32))
