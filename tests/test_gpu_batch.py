"""GPU parity of the batched path (include/gencd_batch.h) against the oracle.

A slot that trains on the rows outside fold f solves the problem of
gencd_create on that row subset, so the oracle runs on
workloads.row_subset(prob, rows outside f): no batched code exists on the CPU
side.  Arithmetic is FP32 (tolerance parity_tools.TOL["f32"]).
"""

import numpy as np
import pytest

import oracle
import workloads
from parity_tools import TOL, _scales, _state, assert_steps_close, assert_support_matches

pytestmark = pytest.mark.gpu

NFOLDS = 4


@pytest.fixture(scope="module")
def gb():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1206_6409_gb300 import build

    build.build()
    from paper_1206_6409_gb300 import binding

    binding.lib()
    return binding


def _problem(loss="squared", seed=3):
    # config-4 law at 1/100: heavy Zipf columns, many one-entry columns; two
    # empty columns and a column living in one fold only are added at the end
    p = workloads.config4(loss, seed=seed, scale=0.01)
    fold = workloads.cv_folds(p.n, NFOLDS, seed=seed)
    rows_f0 = np.flatnonzero(fold == 0)[:3]
    counts = np.concatenate([np.diff(p.col_ptr), [0, rows_f0.size, 0]])
    col_ptr = np.zeros(counts.size + 1, np.int64)
    np.cumsum(counts, out=col_ptr[1:])
    row_idx = np.concatenate([p.row_idx, np.sort(rows_f0).astype(np.int32)])
    val = np.concatenate([p.val, [0.7, -0.4, 1.1]])
    q = workloads.Problem(p.n, counts.size, col_ptr, row_idx, val, p.y, loss, np.zeros(counts.size), p.name)
    return q, fold


def _subset(prob, fold, held_out):
    if held_out < 0:
        return prob
    return workloads.row_subset(prob, np.flatnonzero(fold != held_out))


@pytest.mark.parametrize("loss", ["squared", "logistic"])
def test_batch_lambda_max_matches_oracle(gb, loss):
    prob, fold = _problem(loss)
    with gb.Batch(prob, fold=fold, nfolds=NFOLDS, slots=32) as b:
        for h in range(-1, NFOLDS):
            ref = oracle.Oracle(_subset(prob, fold, h)).lambda_max()
            assert b.lambda_max(h) == pytest.approx(ref, rel=1e-5), h


@pytest.mark.parametrize("slots", [8, 16, 32, 70])
@pytest.mark.parametrize("loss", ["squared", "logistic"])
def test_batch_propose_matches_oracle(gb, loss, slots):
    # every slot its own (training set, lambda, w); some slots stay inactive
    prob, fold = _problem(loss)
    rng = np.random.default_rng(7)
    with gb.Batch(prob, fold=fold, nfolds=NFOLDS, slots=slots) as b:
        S = b.slots
        cases = {}
        for s in range(S):
            if s % 5 == 3:
                continue
            h = int(rng.integers(-1, NFOLDS))
            lam = b.lambda_max(h) * float(rng.choice([0.5, 0.05, 0.01]))
            w = _state(prob, 100 + s, frac=0.05, scale=0.3)
            b.set_slot(s, h, lam, w)
            cases[s] = (h, lam, w)
        d_all, f_all = b.propose()
        obj, kkt = b.objective()
        for s in range(S):
            if s not in cases:
                assert np.all(d_all[s] == 0.0) and np.isnan(obj[s]) and np.isnan(kkt[s])
                continue
            h, lam, w = cases[s]
            sp = _subset(prob, fold, h)
            orc = oracle.Oracle(sp)
            orc.set_lambda(lam)
            z = orc.fitted(w)
            J = np.arange(prob.k, dtype=np.int32)
            d_cpu, f_cpu = orc.propose(w, z, J)
            assert_steps_close(sp, z, w, lam, J, d_all[s], f_all[s], d_cpu, f_cpu, TOL["f32"])
            assert obj[s] == pytest.approx(orc.objective(w), rel=1e-6)
            S_, _ = _scales(sp, z, lam)
            assert abs(kkt[s] - orc.kkt(w, z)) <= TOL["f32"] * (S_.max() + lam) * 10


@pytest.mark.parametrize("B", [1, 7, 256])
def test_batch_step_accepts_each_partitions_best(gb, B):
    # one Thread-Greedy step per slot: in each partition the accepted column
    # has the best proxy up to FP32 rounding, its step is the oracle's FP64
    # Eq. 7 step, and no other coefficient moves
    prob, fold = _problem("logistic", seed=5)
    with gb.Batch(prob, fold=fold, nfolds=NFOLDS, slots=8) as b:
        b.set_params(variant="thread_greedy", blocks=B)
        states = {}
        for s, h in enumerate([-1, 0, 1, 2, 3, -1]):
            lam = b.lambda_max(h) * (0.1 if s % 2 else 0.02)
            w = _state(prob, 200 + s, frac=0.03, scale=0.3)
            b.set_slot(s, h, lam, w)
            states[s] = (h, lam, w)
        _, f_all = b.propose()
        b.iterate(1)
        bounds = (np.arange(B + 1, dtype=np.int64) * prob.k) // B
        for s, (h, lam, w) in states.items():
            w1 = b.w(s)
            moved = np.flatnonzero(w1 != w)
            part = np.searchsorted(bounds, moved, side="right") - 1
            assert moved.size > 0 and np.unique(part).size == part.size
            sp = _subset(prob, fold, h)
            orc = oracle.Oracle(sp)
            orc.set_lambda(lam)
            z = orc.fitted(w)
            d_cpu, _ = orc.propose(w, z, moved.astype(np.int32))
            S_, bj = _scales(sp, z, lam)
            for j, p_, dc in zip(moved, part, d_cpu):
                fmin = f_all[s][bounds[p_]:bounds[p_ + 1]].min()
                assert f_all[s][j] < 0 and f_all[s][j] <= fmin + 1e-4 * abs(fmin)
                sd = abs(dc) + (S_[j] / bj[j] if bj[j] > 0 else abs(w[j]))
                assert abs((w1[j] - w[j]) - dc) <= TOL["f32"] * sd


def test_batch_slot_is_the_same_alone_and_in_the_mix(gb):
    # a slot's iterates do not depend on the other slots
    prob, fold = _problem("squared", seed=9)
    h, w0 = 1, _state(prob, 9, frac=0.02, scale=0.2)
    with gb.Batch(prob, fold=fold, nfolds=NFOLDS, slots=64) as b:
        lam = 0.05 * b.lambda_max(h)
        b.set_slot(0, h, lam, w0)
        b.iterate(6)
        alone = b.w(0)
        b.set_slot(0, h, lam, w0)
        for s in range(1, b.slots):
            hs = s % (NFOLDS + 1) - 1
            b.set_slot(s, hs, b.lambda_max(hs) * 0.03, _state(prob, 300 + s, frac=0.02, scale=0.2))
        b.iterate(6)
        mixed = b.w(0)
    scale = np.abs(alone).max()
    np.testing.assert_allclose(mixed, alone, rtol=0, atol=1e-5 * scale)
    np.testing.assert_array_equal(mixed != 0, alone != 0)


@pytest.mark.parametrize("handoff,slots", [(0.0, 8), (1e-3, 32)])
@pytest.mark.parametrize("loss", ["squared", "logistic"])
def test_batch_path_reaches_every_oracle_optimum(gb, loss, handoff, slots):
    # 3 chains (two folds and all rows) x 5 lambdas from lambda_max to
    # lambda_max / 100, warm started; each solve against the oracle's cyclic
    # CD optimum on its training rows (objective) and the oracle's FP64 KKT
    # value at the GPU's w
    prob, fold = _problem(loss, seed=11)
    chains = [-1, 0, 2]
    with gb.Batch(prob, fold=fold, nfolds=NFOLDS, slots=slots) as b:
        # KKT 1e-8: near the floor of FP32 sums here, and enough for P within 1e-6
        b.set_params(variant="thread_greedy", blocks=64, tol_kkt=1e-8, check_every=5, max_iter=40_000)
        lams = np.stack([workloads.lambda_grid(b.lambda_max(h), 5, 1e-2) for h in chains])
        recs, W, tot = b.path(chains, lams, handoff=handoff, warm=True, want_w=True)
    assert tot.status == 0
    for c, h in enumerate(chains):
        orc = oracle.Oracle(_subset(prob, fold, h))
        for t in range(lams.shape[1]):
            r = recs[c * lams.shape[1] + t]
            assert r["status"] == 0 and r["kkt"] <= 1e-8, (c, t, r)
            orc.set_lambda(lams[c, t])
            w_opt, _, _, kkt, _ = orc.solve("ccd", tol_kkt=1e-11)
            P_opt = orc.objective(w_opt)
            assert r["objective"] == pytest.approx(P_opt, rel=1e-6), (c, t)
            assert orc.objective(W[c, t]) == pytest.approx(P_opt, rel=1e-6), (c, t)
            assert orc.kkt(W[c, t]) <= 5e-8, (c, t)
            # supports equal outside the columns fragile at the compared KKT
            # accuracy (the batch computes in FP32 on FP32-stored values)
            sub = oracle.stored_problem(_subset(prob, fold, h), "f32")
            assert_support_matches(sub, lams[c, t], W[c, t], w_opt, label=f"chain {h} lambda {t}")


def test_batch_rejects_bad_input(gb):
    prob, fold = _problem("squared")
    bad = fold.copy()
    bad[17] = NFOLDS
    with pytest.raises(gb.GencdError) as e:
        gb.Batch(prob, fold=bad, nfolds=NFOLDS, slots=32)
    assert e.value.code == gb.GENCD_EINVAL and "fold[17]" in str(e.value)
    with gb.Batch(prob, fold=fold, nfolds=NFOLDS, slots=32) as b:
        for call in (lambda: b.set_slot(32, -1, 0.1), lambda: b.set_slot(0, NFOLDS, 0.1),
                     lambda: b.set_slot(0, -1, -1.0), lambda: b.copy_slot(1, 2, -1, 0.1),
                     lambda: b.set_params(variant="shotgun")):
            with pytest.raises(gb.GencdError):
                call()


@pytest.mark.parametrize("slots,spmm_kind", [(16, 0), (32, 0), (32, 1), (64, 1)])
def test_every_schedule_proposes_like_the_oracle(gb, slots, spmm_kind):
    # the autotuner's candidates for the X^T U pass compute the same proposals
    prob, fold = _problem("logistic", seed=13)
    with gb.Batch(prob, fold=fold, nfolds=NFOLDS, slots=slots) as b:
        kind, _, tuned = b.schedule()
        assert kind in (0, 1) and "spmm_entries" in tuned or b.slots < 32
        b.set_schedule(spmm_kind, -1)
        assert b.schedule()[0] == spmm_kind
        cases = {}
        for s in range(0, b.slots, 3):
            h = s % (NFOLDS + 1) - 1
            lam = b.lambda_max(h) * 0.05
            w = _state(prob, 400 + s, frac=0.05, scale=0.3)
            b.set_slot(s, h, lam, w)
            cases[s] = (h, lam, w)
        d_all, f_all = b.propose()
        for s, (h, lam, w) in cases.items():
            sp = _subset(prob, fold, h)
            orc = oracle.Oracle(sp)
            orc.set_lambda(lam)
            z = orc.fitted(w)
            J = np.arange(prob.k, dtype=np.int32)
            d_cpu, f_cpu = orc.propose(w, z, J)
            assert_steps_close(sp, z, w, lam, J, d_all[s], f_all[s], d_cpu, f_cpu, TOL["f32"])
    with pytest.raises(gb.GencdError):
        with gb.Batch(prob, fold=fold, nfolds=NFOLDS, slots=16) as b:
            b.set_schedule(1, -1)  # lanes over slots need a multiple of 32 slots


@pytest.mark.parametrize("update_kind", [0, 1])
def test_every_update_schedule_keeps_z_equal_to_xw(gb, update_kind):
    # after steps with either update form, each slot's fitted values are X w
    # (its FP64 objective equals the oracle's at its w, whatever the steps
    # did: plain Thread-Greedy may diverge here); slots share columns (the same
    # training set and lambda in groups of four), so the grouped form's shared
    # walks are taken
    prob, fold = _problem("squared", seed=17)
    with gb.Batch(prob, fold=fold, nfolds=NFOLDS, slots=32) as b:
        b.set_params(variant="thread_greedy", blocks=64)
        b.set_schedule(-1, update_kind)
        cases = {}
        for s in range(b.slots):
            h = (s // 4) % (NFOLDS + 1) - 1
            lam = b.lambda_max(h) * (0.05 if s % 8 < 4 else 0.02)
            b.set_slot(s, h, lam, None)
            cases[s] = (h, lam)
        b.iterate(12)
        obj, _ = b.objective()
        for s, (h, lam) in cases.items():
            orc = oracle.Oracle(oracle.stored_problem(_subset(prob, fold, h), "f32"))  # the batch stores X in FP32
            orc.set_lambda(lam)
            w = b.w(s)
            assert np.count_nonzero(w) > 0
            assert obj[s] == pytest.approx(orc.objective(w), rel=1e-12)


def test_batch_path_to_a_duality_gap(gb):
    # solves that stop at a relative duality gap of 8e-7 (the dual point's
    # scale from FP32 sums, accurate to about 1e-6 relative) are certified by
    # the oracle's FP64 gap to 2e-6
    prob, fold = _problem("logistic", seed=11)
    chains = [-1, 1]
    with gb.Batch(prob, fold=fold, nfolds=NFOLDS, slots=32) as b:
        b.set_params(variant="thread_greedy", blocks=64, tol_kkt=0.0, tol_gap=8e-7, check_every=5, max_iter=100_000)
        lams = np.stack([workloads.lambda_grid(b.lambda_max(h), 4, 1e-2) for h in chains])
        recs, W, tot = b.path(chains, lams, handoff=0.0, warm=True, want_w=True)
    assert tot.status == 0, recs
    for c, h in enumerate(chains):
        sp = oracle.stored_problem(_subset(prob, fold, h), "f32")
        for t in range(lams.shape[1]):
            orc = oracle.Oracle(sp, lams[c, t])
            P = orc.objective(W[c, t])
            assert recs[c * lams.shape[1] + t]["objective"] == pytest.approx(P, rel=1e-9)
            assert orc.duality_gap(W[c, t]) <= 2e-6 * P, (c, t)
