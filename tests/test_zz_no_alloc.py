"""The allocation-free streaming Propose (gencd_propose_all_noalloc) gives the
same steps, proxies and KKT value as gencd_propose_all on the same state.

It serves callers that cannot allocate device memory; its scratch is a fixed
device array shared by all calls, so the test calls it twice in a row (the
second call must not see the first call's sums).  This file is collected
last so that a run stopping at the first failure has run every other test."""

import numpy as np
import pytest

import oracle
import workloads

from test_gpu_parity import TOL, assert_steps_close

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("loss", ["logistic", "squared"])
def test_noalloc_propose_matches_the_problem_entry_point(loss):
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1206_6409_gb300 import binding as gb
    from paper_1206_6409_gb300 import build

    build.build()
    prob = workloads.zipf_problem(120_000, 20_000, 400_000, cap=20_000, n_planted=10, loss=loss, seed=7)
    lam = 0.05 * oracle.Oracle(prob).lambda_max()
    w = np.where(np.random.default_rng(8).random(prob.k) < 0.1, 0.3, 0.0)
    with gb.Problem(prob, precision="f64") as p:
        p.set_lambda(lam)
        p.set_w(w)
        z = p.z()
        d_ref, f_ref, kkt_ref = p.propose_all()
    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    args = [t(prob.col_ptr), t(prob.row_idx), t(prob.val), t(prob.y), t(z), t(w)]
    J = np.arange(prob.k)
    for _ in range(2):  # two calls in a row share the scratch
        delta = torch.full((prob.k,), float("nan"), dtype=torch.float64, device=dev)
        phi = torch.full((prob.k,), float("nan"), dtype=torch.float64, device=dev)
        kkt = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        gb.gencd_propose_all_noalloc(prob.n, prob.k, prob.nnz, *args, loss, lam, 0, delta, phi, kkt)
        torch.cuda.synchronize()
        assert_steps_close(prob, z, w, lam, J, delta.cpu().numpy(), phi.cpu().numpy(), d_ref, f_ref, TOL["f64"])
        assert kkt.item() == pytest.approx(kkt_ref, rel=1e-9, abs=1e-15)


def test_noalloc_rejects_inputs_beyond_its_scratch():
    import torch

    from paper_1206_6409_gb300 import binding as gb

    dev = torch.device("cuda")
    k = (1 << 19) + 1
    one = torch.zeros(1, dtype=torch.float64, device=dev)
    cp = torch.zeros(k + 1, dtype=torch.int64, device=dev)
    ri = torch.zeros(1, dtype=torch.int32, device=dev)
    with pytest.raises(gb.GencdError) as e:
        gb.gencd_propose_all_noalloc(1, k, 0, cp, ri, one, one, one, torch.zeros(k, dtype=torch.float64, device=dev),
                                     "squared", 0.1, 0, torch.zeros(k, dtype=torch.float64, device=dev),
                                     torch.zeros(k, dtype=torch.float64, device=dev), one)
    assert e.value.code == gb.GENCD_EINVAL and "at most" in str(e.value)
