"""The support comparison of the parity tests (parity_tools) on the CPU.

The fragile set is a first-order sensitivity bound: it must cover every
support change between two oracle points at a given KKT accuracy, be empty
when the accuracy is far finer than the problem's margins, and a planted
support change outside it must fail the comparison.
"""

import numpy as np
import pytest

import oracle
import workloads
from parity_tools import assert_support_matches, certified_optimum, fragile_columns, load_optimum


@pytest.fixture(scope="module")
def path():
    # an ill-conditioned sparse logistic problem with k > n
    prob = workloads.uniform_problem(300, 600, 8, values="lognormal", loss="logistic", n_planted=20, seed=6)
    orc = oracle.Oracle(prob)
    lam = 0.02 * orc.lambda_max()
    orc.set_lambda(lam)
    ref, _, _, kkt, _ = orc.solve("ccd", tol_kkt=1e-12, max_iter=10**8)
    assert kkt <= 1e-12
    pts = {tol: orc.solve("ccd", tol_kkt=tol, max_iter=10**8)[0] for tol in (1e-5, 1e-6, 1e-7, 1e-8)}
    return prob, lam, ref, pts


def test_fragile_set_covers_the_support_changes_along_cyclic_cd(path):
    prob, lam, ref, pts = path
    changed = 0
    for tol, w in pts.items():
        eps, nfrag, ndiff = assert_support_matches(prob, lam, w, ref, label=f"ccd {tol}", max_eps=1e-4)
        changed += ndiff
        assert eps >= tol * 0.5  # the point's own KKT level
    assert changed > 0  # the coarser points do differ in support


def test_fragile_set_shrinks_with_the_accuracy(path):
    prob, lam, ref, _ = path
    sizes = [int(fragile_columns(prob, lam, ref, eps).sum()) for eps in (1e-4, 1e-6, 1e-8, 1e-10, 1e-14)]
    assert sizes == sorted(sizes, reverse=True) and sizes[0] > 0 and sizes[-1] == 0


def test_a_planted_support_change_outside_the_fragile_set_fails(path):
    prob, lam, ref, _ = path
    fr = fragile_columns(prob, lam, ref, 1e-9)
    j = int(np.flatnonzero((np.abs(ref) > 1e-3) & ~fr)[0])
    bad = ref.copy()
    bad[j] = 0.0  # a firmly active coefficient dropped
    with pytest.raises(AssertionError, match="outside the fragile set"):
        assert_support_matches(prob, lam, bad, ref, label="planted", eps=1e-9)
    with pytest.raises(AssertionError, match="not comparable"):  # its KKT violation is far above 1e-7
        assert_support_matches(prob, lam, bad, ref, label="planted")


def test_stored_optima_are_certified_by_the_oracle():
    # the fixtures written by tests/golden/make_optima.py satisfy the oracle's
    # KKT conditions to 1e-11 on the problems as generated here
    prob = workloads.config3("pm1", "logistic")
    orc = oracle.Oracle(prob)
    lam = 0.01 * orc.lambda_max()
    w_file, lam_file, meta = load_optimum("cfg3_pm1_logistic")
    assert lam_file == pytest.approx(lam, rel=1e-12)
    orc.set_lambda(lam)
    assert orc.kkt(w_file) <= 1e-11
    w = certified_optimum("cfg3_pm1_logistic", prob, lam)
    np.testing.assert_array_equal(w, w_file)
