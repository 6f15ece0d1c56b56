"""The allocation-free streaming Propose (gencd_propose_all_noalloc) against
the FP64 oracle.

The entry point serves callers that cannot allocate device memory; its
scratch is a fixed device array shared by every call and keeping the last
call's contents.  So the tests call it twice in a row, call it at the largest
size its scratch holds (k = 2^19 columns, nnz = 2^25 non-zeros, with empty
and long columns) and then on a smaller, different problem whose result must
not see the larger call's sums or tile map.  This file is collected last so
that a run stopping at the first failure has run every other test.
"""

import numpy as np
import pytest

import oracle
import workloads
from parity_tools import TOL, assert_steps_close

pytestmark = pytest.mark.gpu

MAX_K = 1 << 19
MAX_NNZ = 1 << 25


@pytest.fixture(scope="module")
def gb():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1206_6409_gb300 import build

    build.build()
    from paper_1206_6409_gb300 import binding

    binding.lib()
    return binding


def _with_empty_columns(prob, every=7):
    """prob with an empty column inserted before every `every`-th column and
    at the end (the tile map's bisection over equal column pointers)."""
    counts = prob.col_nnz()
    new_counts, src = [], []
    for j in range(prob.k):
        if j % every == 0:
            new_counts.append(0)
            src.append(-1)
        new_counts.append(counts[j])
        src.append(j)
    new_counts.append(0)
    src.append(-1)
    cp = np.zeros(len(new_counts) + 1, np.int64)
    np.cumsum(new_counts, out=cp[1:])
    return workloads.Problem(prob.n, len(new_counts), cp, prob.row_idx.copy(), prob.val.copy(), prob.y,
                             prob.loss, np.zeros(len(new_counts)), prob.name + "-empty-cols")


def _max_size_problem(loss, seed=11):
    """Exactly k = 2^19 columns and nnz = 2^25 non-zeros: 64 per column, 4,096
    empty columns (the last one among them), 2,048 of 128 and one long column
    that takes the rest, rows uniform without replacement, log-normal values."""
    rng = np.random.default_rng(seed)
    n = 200_000
    counts = np.full(MAX_K, 64, np.int64)
    perm = rng.permutation(MAX_K - 1)
    counts[perm[:4095]] = 0
    counts[MAX_K - 1] = 0
    counts[perm[4095:4095 + 2048]] = 128
    long_col = perm[4095 + 2048]
    counts[long_col] += MAX_NNZ - counts.sum()
    assert counts.sum() == MAX_NNZ and counts[long_col] <= n
    cp = np.zeros(MAX_K + 1, np.int64)
    np.cumsum(counts, out=cp[1:])
    rows = workloads.synthetic._distinct_rows(n, counts, rng)
    val = rng.lognormal(0.0, 1.0, MAX_NNZ) * np.where(rng.random(MAX_NNZ) < 0.2, -1.0, 1.0)
    y = np.where(rng.random(n) < 0.5, -1.0, 1.0) if loss == "logistic" else rng.normal(size=n)
    return workloads.Problem(n, MAX_K, cp, rows, val, y, loss, np.zeros(MAX_K), "noalloc-max")


def _noalloc(gb, prob, w, z, lam, beta_mode):
    import torch

    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    args = [t(prob.col_ptr), t(prob.row_idx), t(prob.val), t(prob.y), t(z), t(w)]
    delta = torch.full((prob.k,), float("nan"), dtype=torch.float64, device=dev)
    phi = torch.full((prob.k,), float("nan"), dtype=torch.float64, device=dev)
    kkt = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
    gb.gencd_propose_all_noalloc(prob.n, prob.k, prob.nnz, *args, prob.loss, lam, beta_mode, delta, phi, kkt)
    torch.cuda.synchronize()
    return delta.cpu().numpy(), phi.cpu().numpy(), kkt.item()


def _check_against_oracle(gb, prob, lam, beta_mode, w, calls=1):
    orc = oracle.Oracle(prob, lam, beta_mode=beta_mode)
    z = orc.fitted(w)
    J = np.arange(prob.k, dtype=np.int32)
    d_cpu, f_cpu = orc.propose(w, z, J)
    kkt_cpu = orc.kkt(w, z)
    for _ in range(calls):
        d, f, kkt = _noalloc(gb, prob, w, z, lam, beta_mode)
        assert_steps_close(prob, z, w, lam, J, d, f, d_cpu, f_cpu, TOL["f64"], beta_mode=beta_mode)
        assert kkt == pytest.approx(kkt_cpu, rel=1e-9, abs=1e-15)


@pytest.mark.parametrize("beta_mode", [0, 1])
@pytest.mark.parametrize("loss", ["logistic", "squared"])
def test_noalloc_propose_matches_the_oracle(gb, loss, beta_mode):
    # a Zipf problem with heavy and light columns, plus empty columns
    prob = _with_empty_columns(workloads.zipf_problem(120_000, 20_000, 400_000, cap=20_000, n_planted=10,
                                                      loss=loss, seed=7))
    lam = 0.05 * oracle.Oracle(prob, beta_mode=beta_mode).lambda_max()
    w = np.where(np.random.default_rng(8).random(prob.k) < 0.1, 0.3, 0.0)
    _check_against_oracle(gb, prob, lam, beta_mode, w, calls=2)  # two calls in a row share the scratch


def test_noalloc_at_its_size_limit_then_on_a_smaller_problem(gb):
    big = _max_size_problem("logistic")
    lam = 0.05 * oracle.Oracle(big).lambda_max()
    w = np.where(np.random.default_rng(9).random(big.k) < 0.05, -0.2, 0.0)
    _check_against_oracle(gb, big, lam, 0, w)
    # a smaller, different problem right after: stale sums or tile-map entries
    # of the larger call would show here
    small = _with_empty_columns(workloads.config1("squared"), every=5)
    lam_s = 0.05 * oracle.Oracle(small).lambda_max()
    w_s = np.where(np.random.default_rng(10).random(small.k) < 0.1, 0.5, 0.0)
    _check_against_oracle(gb, small, lam_s, 0, w_s, calls=2)


def test_noalloc_rejects_inputs_beyond_its_scratch(gb):
    import torch

    dev = torch.device("cuda")
    one = torch.zeros(1, dtype=torch.float64, device=dev)
    ri = torch.zeros(1, dtype=torch.int32, device=dev)

    def call(n, k, nnz, lam=0.1):
        cp = torch.zeros(k + 1, dtype=torch.int64, device=dev)
        kv = torch.zeros(k, dtype=torch.float64, device=dev)
        gb.gencd_propose_all_noalloc(n, k, nnz, cp, ri, one, one, one, kv, "squared", lam, 0, kv.clone(),
                                     kv.clone(), one)

    with pytest.raises(gb.GencdError) as e:
        call(1, MAX_K + 1, 0)
    assert e.value.code == gb.GENCD_EINVAL and "at most" in str(e.value)
    with pytest.raises(gb.GencdError) as e:
        call(1, 4, MAX_NNZ + 1)
    assert e.value.code == gb.GENCD_EINVAL and "at most" in str(e.value)
    for bad in (float("inf"), float("nan"), -1.0):
        with pytest.raises(gb.GencdError) as e:
            call(1, 4, 0, lam=bad)
        assert e.value.code == gb.GENCD_EINVAL and "lambda" in str(e.value)
