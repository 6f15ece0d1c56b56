"""The serving loop (include/gencd_serve.h) on a stream of small requests:
every response against the same request served alone and, for the smaller
ones, against the oracle's cyclic-CD optimum; admission by the HBM budget."""

import numpy as np
import pytest

import oracle
import workloads
from parity_tools import assert_support_matches

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1206_6409_gb300 import build

    build.build()
    from paper_1206_6409_gb300 import binding

    binding.lib()
    return binding


@pytest.fixture(scope="module")
def stream():
    return workloads.serving_stream(10, rate=500.0, seed=3, n_range=(1_000, 4_000), k_range=(1_000, 8_000))


PARAMS = dict(variant="thread_greedy", blocks=64, tol_kkt=1e-8, max_iter=200_000, check_every=10)


def test_serve_results_are_the_same_alone_and_in_the_mix(gb, stream):
    problems, fracs, arrivals = stream
    mix, w_mix = gb.gencd_serve(problems, fracs, arrivals, workers=4, want_w=True, **PARAMS)
    alone, w_alone = gb.gencd_serve(problems, fracs, arrivals, workers=1, want_w=True, **PARAMS)
    assert max(r["worker"] for r in mix) > 0  # requests ran concurrently
    for q, (a, b) in enumerate(zip(mix, alone)):
        assert a["status"] == 0 and b["status"] == 0, (q, a, b)
        assert a["kkt"] <= 1e-8 and b["kkt"] <= 1e-8
        assert a["lambda_"] == pytest.approx(b["lambda_"], rel=1e-6)
        assert a["objective"] == pytest.approx(b["objective"], rel=1e-7), q
        assert a["end"] >= a["start"] >= a["arrival"] - 1e-6
        # the same support alone and in the mix, outside the columns fragile at
        # the two points' KKT accuracy (FP64 atomics add in arrival order)
        assert_support_matches(oracle.stored_problem(problems[q], "f32"), b["lambda_"], w_mix[q], w_alone[q],
                               label=f"request {q} alone / mix")
    # the smaller requests against the oracle on the same problem
    order = np.argsort([p.nnz for p in problems])[:4]
    for q in order:
        p = problems[q]
        orc = oracle.Oracle(p)
        orc.set_lambda(mix[q]["lambda_"])
        assert mix[q]["lambda_"] == pytest.approx(fracs[q] * orc.lambda_max(), rel=1e-5)
        w_opt, _, _, _, _ = orc.solve("ccd", tol_kkt=1e-11)
        assert mix[q]["objective"] == pytest.approx(orc.objective(w_opt), rel=1e-6), q
        assert orc.kkt(w_mix[q]) <= 5e-8
        assert_support_matches(oracle.stored_problem(p, "f32"), mix[q]["lambda_"], w_mix[q], w_opt,
                               label=f"request {q}")


def test_serve_admits_by_the_hbm_budget(gb, stream):
    # a budget below every request's estimate: each runs alone, in order
    problems, fracs, arrivals = stream
    res, _ = gb.gencd_serve(problems, fracs, arrivals, workers=4, hbm_fraction=1e-9, **PARAMS)
    spans = sorted((r["start"], r["end"]) for r in res)
    assert all(r["status"] == 0 for r in res)
    for (s0, e0), (s1, e1) in zip(spans, spans[1:]):
        assert s1 >= e0 - 1e-3  # no overlap (admission waits for the previous request)
    assert [r["start"] for r in res] == sorted(r["start"] for r in res)  # first come, first served


def test_serve_rejects_bad_streams(gb, stream):
    problems, fracs, arrivals = stream
    with pytest.raises(gb.GencdError):
        gb.gencd_serve(problems[:3], fracs[:3], [0.0, 0.2, 0.1], workers=2, **PARAMS)
    with pytest.raises(gb.GencdError):
        gb.gencd_serve(problems[:2], fracs[:2], arrivals[:2], workers=0, **PARAMS)
