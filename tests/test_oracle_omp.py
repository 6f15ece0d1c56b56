"""The OpenMP baseline (Section 4.2's shared-memory design) against the
single-threaded oracle: with one thread its Thread-Greedy and Greedy iterates
are the oracle's bit for bit; with several threads the atomic additions to z
reorder only roundings."""

import numpy as np
import pytest

import oracle
import workloads


@pytest.fixture(scope="module")
def orc():
    prob = workloads.config2_scaled(0.002, "logistic")
    o = oracle.Oracle(prob)
    o.set_lambda(0.05 * o.lambda_max())
    return o


@pytest.mark.parametrize("variant,B", [("thread_greedy", 64), ("thread_greedy", 1024), ("greedy", 1)])
def test_one_thread_equals_the_oracle(orc, variant, B):
    w_cpu, z_cpu, _, st_cpu = orc.run(variant, 12, B=B)
    s = oracle.OmpSolver(orc, threads=1)
    st = s.iterate(12, B=B, greedy=variant == "greedy")
    w, z = s.state()
    np.testing.assert_array_equal(w, w_cpu)
    np.testing.assert_array_equal(z, z_cpu)
    assert st == tuple(int(x) for x in st_cpu)


@pytest.mark.parametrize("threads", [2, 4])
@pytest.mark.parametrize("variant,B", [("thread_greedy", 256), ("greedy", 1)])
def test_threads_reorder_only_roundings(orc, threads, variant, B):
    w_cpu, z_cpu, _, st_cpu = orc.run(variant, 12, B=B)
    s = oracle.OmpSolver(orc, threads=threads)
    st = s.iterate(12, B=B, greedy=variant == "greedy")
    w, z = s.state()
    np.testing.assert_array_equal(w != 0, w_cpu != 0)
    np.testing.assert_allclose(w, w_cpu, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(z, z_cpu, rtol=1e-12, atol=1e-15)
    assert st == tuple(int(x) for x in st_cpu)
    assert s.threads == threads
