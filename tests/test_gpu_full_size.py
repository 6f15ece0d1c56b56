"""Parity at the benchmark's full size (n=1,000,000, k=4,000,000, 2.0e8 nnz,
Zipf(1.1) column lengths up to 50,000), in the launch configuration the
benchmark times.  The oracle computes the sampled columns one by one."""

import os

import numpy as np
import pytest

import oracle
import workloads

from test_gpu_parity import TOL, assert_steps_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1206_6409_gb300 import binding, build

    build.build()
    binding.lib()
    prob = workloads.config2("logistic")
    orc = oracle.Oracle(prob)
    lam_max = orc.lambda_max()
    lam = 0.05 * lam_max
    orc.set_lambda(lam)
    rng = np.random.default_rng(7)
    w = np.zeros(prob.k)
    support = rng.choice(prob.k, 3000, replace=False)
    w[support] = rng.normal(0, 0.3, support.size)
    z = orc.fitted(w)
    counts = np.diff(prob.col_ptr)
    heavy = np.argsort(counts)[-300:]  # the longest columns (up to 50,000 nnz)
    sample = np.unique(np.concatenate([heavy, support[:700], rng.choice(prob.k, 3000, replace=False)]))
    sample = sample.astype(np.int32)
    d_cpu, f_cpu = orc.propose(w, z, sample)
    return binding, prob, lam_max, lam, w, z, sample, d_cpu, f_cpu


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_config2_propose_sampled(full, precision):
    gb, prob, lam_max, lam, w, z, sample, d_cpu, f_cpu = full
    val = prob.val.astype(np.float32) if precision == "f32" else prob.val
    with gb.Problem(n=prob.n, k=prob.k, col_ptr=prob.col_ptr, row_idx=prob.row_idx, val=val, y=prob.y,
                    loss="logistic", precision=precision) as p:
        assert p.lambda_max() == pytest.approx(lam_max, rel=10 * TOL[precision])
        p.set_lambda(lam)
        p.set_params(variant="thread_greedy", blocks=1024)
        p.set_w(w)
        d_all, f_all, _ = p.propose_all()
        assert_steps_close(prob, z, w, lam, sample, d_all[sample], f_all[sample], d_cpu, f_cpu, TOL[precision])
        d_l, f_l = p.propose_at(sample)
        assert_steps_close(prob, z, w, lam, sample, d_l, f_l, d_cpu, f_cpu, TOL[precision])
        # one Thread-Greedy iteration as the benchmark runs it: every accepted
        # column is the best proxy of its partition (FP32 mode ranks with FP32
        # proxies: best up to their rounding), and w moved only there
        p.iterate(1)
        w1 = p.w()
        moved = np.flatnonzero(w1 != w)
        B = 1024
        bounds = (np.arange(B + 1, dtype=np.int64) * prob.k) // B
        part = np.searchsorted(bounds, moved, side="right") - 1
        assert np.unique(part).size == part.size  # at most one update per partition
        for j, b in zip(moved[:50], part[:50]):
            lo, hi = b * prob.k // B, (b + 1) * prob.k // B
            assert lo <= j < hi
            fmin = f_all[lo:hi].min()
            assert f_all[j] < 0
            if precision == "f64":
                assert f_all[j] == fmin
            else:
                assert f_all[j] <= fmin + 1e-4 * abs(fmin)
