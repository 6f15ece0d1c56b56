"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (step and proxy, from the condition of the sum g_j = (1/n) sum_i
X_ij u_i): with S_j = (1/n) sum_i |X_ij u_i| and sd_j = |delta_j| + S_j/beta_j,
  |delta_gpu - delta_cpu| <= tol * sd_j,
  |phi_gpu - phi_cpu|     <= tol * sd_j * (S_j + beta_j sd_j + lambda),
tol = 1e-12 in FP64 mode and 1e-5 in FP32 mode.  Integer results (colours,
permutations, supports) are compared exactly.
"""

import numpy as np
import pytest

import oracle
import workloads
from parity_tools import (TOL, _scales, _state, _u, assert_steps_close, assert_support_matches,  # noqa: F401
                          certified_optimum)

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


def ragged_problem(loss="logistic", seed=0):
    """Column lengths at the kernel's edges (0, 1, 31..33, tile sizes, 4096,
    50,000), empty rows, a ragged tail."""
    rng = np.random.default_rng(seed)
    n = 60_000
    lengths = [0, 1, 2, 3, 31, 32, 33, 0, 0, 127, 128, 129, 255, 256, 257, 4096, 50_000, 5, 0, 1000,
               7, 1, 0]
    lengths += list(rng.integers(0, 40, size=300))
    lengths += [1, 0, 0, 3]
    counts = np.array(lengths, np.int64)
    col_ptr = np.zeros(counts.size + 1, np.int64)
    np.cumsum(counts, out=col_ptr[1:])
    rows = workloads.synthetic._distinct_rows(n - 100, counts, rng)  # the last 100 rows stay empty
    val = rng.lognormal(0.0, 1.0, rows.size) * np.where(rng.random(rows.size) < 0.3, -1.0, 1.0)
    y = np.where(rng.random(n) < 0.5, -1.0, 1.0) if loss == "logistic" else rng.normal(size=n)
    return workloads.Problem(n, counts.size, col_ptr, rows, val, y, loss, np.zeros(counts.size), "ragged")


PROBLEMS = {
    "cfg1-logistic": lambda: workloads.config1("logistic"),
    "cfg1-squared": lambda: workloads.config1("squared"),
    "ragged-logistic": lambda: ragged_problem("logistic"),
    "ragged-squared": lambda: ragged_problem("squared", 1),
    "zipf-logistic": lambda: workloads.config2_scaled(0.002, "logistic"),
    # several row slabs, heavy and light columns
    "zipf-slabs-squared": lambda: workloads.zipf_problem(120_000, 20_000, 400_000, cap=20_000, n_planted=10,
                                                         loss="squared", seed=5),
}


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_propose_matches_oracle(gb, name, precision):
    prob = PROBLEMS[name]()
    orc = oracle.Oracle(prob)
    lam = 0.05 * orc.lambda_max()
    orc.set_lambda(lam)
    w = _state(prob, 1)
    z = orc.fitted(w)
    rng = np.random.default_rng(2)
    J = np.concatenate([np.arange(prob.k), rng.integers(0, prob.k, 500)]).astype(np.int32)
    d_cpu, f_cpu = orc.propose(w, z, J)
    with gb.Problem(prob, precision=precision) as p:
        p.set_lambda(lam)
        p.set_w(w)
        d_gpu, f_gpu = p.propose_at(J)
        assert_steps_close(prob, z, w, lam, J, d_gpu, f_gpu, d_cpu, f_cpu, TOL[precision])
        # the streaming pass over all columns (Thread-Greedy's Propose)
        d_all, f_all, kkt = p.propose_all()
        Jall = np.arange(prob.k)
        assert_steps_close(prob, z, w, lam, Jall, d_all, f_all, d_cpu[:prob.k], f_cpu[:prob.k],
                           TOL[precision])
        S, _ = _scales(prob, z, lam)
        assert abs(kkt - orc.kkt(w, z)) <= TOL[precision] * (S.max() + lam) * 10


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_lambda_max_and_objective(gb, precision):
    for loss in ("logistic", "squared"):
        prob = workloads.config1(loss)
        orc = oracle.Oracle(prob)
        with gb.Problem(prob, precision=precision) as p:
            lm = p.lambda_max()
            assert lm == pytest.approx(orc.lambda_max(), rel=TOL[precision] * 10)
            lam = 0.02 * orc.lambda_max()
            orc.set_lambda(lam)
            p.set_lambda(lam)
            w = _state(prob, 5)
            p.set_w(w)
            obj, kkt = p.objective()
            assert obj == pytest.approx(orc.objective(w), rel=1e-13 if precision == "f64" else 1e-6)
            np.testing.assert_allclose(p.z(), orc.fitted(w), rtol=0,
                                       atol=1e-12 if precision == "f64" else 1e-5)


def test_permutation_is_bit_exact(gb):
    prob = workloads.config1("logistic")
    with gb.Problem(prob) as p:
        for seed, epoch, m in [(0, 0, 1), (0, 0, 4096), (7, 3, 4097), (2**64 - 1, 11, 100_003),
                               (123, 0, 1_000_000)]:
            np.testing.assert_array_equal(p.permutation(seed, epoch, m), oracle.permutation(seed, epoch, m))


@pytest.mark.parametrize("name", ["cfg1-logistic", "ragged-squared", "zipf-logistic"])
def test_coloring_equals_first_fit(gb, name):
    prob = PROBLEMS[name]()
    colors_cpu, nc_cpu = oracle.Oracle(prob).color()
    with gb.Problem(prob) as p:
        assert p.color() == nc_cpu
        np.testing.assert_array_equal(p.colors(), colors_cpu)


@pytest.mark.parametrize("precision", ["f64"])
@pytest.mark.parametrize("loss", ["logistic", "squared"])
def test_coloring_iterations_match(gb, loss, precision):
    prob = workloads.config1(loss)
    orc = oracle.Oracle(prob)
    lam = 0.05 * orc.lambda_max()
    orc.set_lambda(lam)
    colors, C = orc.color()
    iters = C + C // 2  # crosses an epoch boundary
    w_cpu, z_cpu, _, _ = orc.run("coloring", iters, colors=colors, seed=9)
    with gb.Problem(prob, precision=precision) as p:
        p.set_lambda(lam)
        p.set_colors(colors)
        p.set_params(variant="coloring", seed=9)
        p.iterate(iters)
        w_gpu = p.w()
    np.testing.assert_array_equal(w_gpu != 0, w_cpu != 0)
    np.testing.assert_allclose(w_gpu, w_cpu, rtol=0, atol=1e-10)


@pytest.mark.parametrize("variant,B,P", [("thread_greedy", 64, 0), ("thread_greedy", 5000, 0),
                                          ("greedy", 1, 0), ("shotgun", 0, 200)])
def test_iterations_match(gb, variant, B, P):
    prob = workloads.config1("logistic")
    orc = oracle.Oracle(prob)
    lam = 0.05 * orc.lambda_max()
    orc.set_lambda(lam)
    iters = 40
    w_cpu, z_cpu, _, _ = orc.run(variant, iters, B=B or 1, P=P or 1, seed=4)
    with gb.Problem(prob) as p:
        p.set_lambda(lam)
        p.set_params(variant=variant, blocks=B, P=P, seed=4)
        r = p.iterate(iters)
        w_gpu = p.w()
        assert r.iters == iters and np.isfinite(r.objective)
    np.testing.assert_array_equal(w_gpu != 0, w_cpu != 0)
    np.testing.assert_allclose(w_gpu, w_cpu, rtol=0, atol=1e-10)


@pytest.mark.parametrize("loss", ["logistic", "squared"])
@pytest.mark.parametrize("variant", ["shotgun", "thread_greedy", "coloring"])
def test_solve_reaches_the_oracle_optimum(gb, loss, variant):
    # B = 16 partitions: Thread-Greedy has no convergence guarantee (Section 7)
    # and the oracle itself diverges on this problem for B >= 64.
    prob = workloads.uniform_problem(1000, 2000, 10, values="pm1", loss=loss, n_planted=30, seed=21)
    orc = oracle.Oracle(prob)
    lam = 0.05 * orc.lambda_max()
    orc.set_lambda(lam)
    w_opt, _, _, kkt, _ = orc.solve("ccd", tol_kkt=1e-11)
    assert kkt <= 1e-11
    P_opt = orc.objective(w_opt)
    with gb.Problem(prob) as p:
        p.set_lambda(lam)
        p.set_params(variant=variant, tol_kkt=1e-11, max_iter=400_000, check_every=50, blocks=16)
        r = p.solve()
        assert r.status == 0, r.as_dict()
        w = p.w()
    assert r.objective == pytest.approx(P_opt, rel=1e-6)
    big = (np.abs(w_opt) > 1e-6) | (np.abs(w) > 1e-6)
    np.testing.assert_array_equal(np.sign(w[big]), np.sign(w_opt[big]))
    assert_support_matches(prob, lam, w, w_opt, label=f"{variant} {loss}")


@pytest.mark.parametrize("loss", ["logistic", "squared"])
def test_config1_shotgun_solve_matches_oracle(gb, loss):
    """Plain L1 problem of n=2,000, k=5,000 (20 nnz/column, +-1 values), FP64,
    Shotgun with P* against the oracle's cyclic-CD optimum."""
    prob = workloads.config1(loss)
    orc = oracle.Oracle(prob)
    lam = 0.01 * orc.lambda_max()
    orc.set_lambda(lam)
    if loss == "logistic":  # config 1's logistic problem is config 3's +-1 one: its stored optimum
        w_opt = certified_optimum("cfg3_pm1_logistic", prob, lam)
    else:
        w_opt, _, _, kkt, _ = orc.solve("ccd", tol_kkt=1e-11, max_iter=4 * 10**8)
    P_opt = orc.objective(w_opt)
    with gb.Problem(prob) as p:
        p.set_lambda(lam)
        rho, pstar, _ = p.spectral_radius()
        rho_cpu, _ = orc.spectral_radius()
        assert rho == pytest.approx(rho_cpu, rel=1e-6)
        p.set_params(variant="shotgun", P=0, tol_kkt=1e-10, max_iter=4_000_000, check_every=200)
        r = p.solve()
        assert r.status == 0, r.as_dict()
        w = p.w()
    assert r.objective == pytest.approx(P_opt, rel=1e-6)
    assert_support_matches(prob, lam, w, w_opt, label=f"config 1 shotgun {loss}")


def test_f32_solve_reaches_the_optimum(gb):
    prob = workloads.config2_scaled(0.002, "logistic")
    orc = oracle.Oracle(prob)
    lam = 0.05 * orc.lambda_max()
    orc.set_lambda(lam)
    w_opt, _, _, _, _ = orc.solve("ccd", tol_kkt=1e-11)
    with gb.Problem(prob, precision="f32") as p:
        p.set_lambda(lam)
        p.set_params(variant="thread_greedy", blocks=128, tol_kkt=1e-8, max_iter=100_000, check_every=50)
        r = p.solve()
        assert r.status == 0, r.as_dict()
        w = p.w()
    assert r.objective == pytest.approx(orc.objective(w_opt), rel=1e-6)
    # FP32 storage rounds X: the GPU solves the problem on the stored values,
    # whose optimum is within the fragile margin of the FP64 one
    assert_support_matches(oracle.stored_problem(prob, "f32"), lam, w, w_opt, label="f32 scaled config 2")


@pytest.mark.parametrize("variant,B", [("greedy", 1), ("thread_greedy", 7), ("thread_greedy", 1024)])
def test_f32_accepts_the_best_proxy(gb, variant, B):
    # FP32 mode ranks columns with FP32 proxies and applies the winner's FP64
    # step: each partition's accepted column has the partition's best proxy up
    # to FP32 rounding, its step is the FP64 Eq. 7 step, and nothing else moves
    prob = workloads.config2_scaled(0.01, "logistic")
    orc = oracle.Oracle(prob)
    lam = 0.05 * orc.lambda_max()
    orc.set_lambda(lam)
    w = _state(prob, 11, frac=0.05, scale=0.3)
    z = orc.fitted(w)
    with gb.Problem(prob, precision="f32") as p:
        p.set_lambda(lam)
        p.set_params(variant=variant, blocks=B)
        p.set_w(w)
        _, f_all, _ = p.propose_all()
        p.iterate(1)
        w1 = p.w()
    moved = np.flatnonzero(w1 != w)
    Bp = 1 if variant == "greedy" else B
    bounds = (np.arange(Bp + 1, dtype=np.int64) * prob.k) // Bp
    part = np.searchsorted(bounds, moved, side="right") - 1
    assert moved.size > 0 and np.unique(part).size == part.size
    J = moved.astype(np.int32)
    d_cpu, _ = orc.propose(w, z, J)
    S, bj = _scales(prob, z, lam)
    for j, b, dc in zip(moved, part, d_cpu):
        fmin = f_all[bounds[b]:bounds[b + 1]].min()
        assert f_all[j] < 0 and f_all[j] <= fmin + 1e-4 * abs(fmin)
        sd = abs(dc) + (S[j] / bj[j] if bj[j] > 0 else abs(w[j]))
        assert abs((w1[j] - w[j]) - dc) <= TOL["f32"] * sd


def test_edge_cases(gb):
    # one column, one row, all-empty columns, lambda above lambda_max
    X = np.array([[2.0]])
    p1 = workloads.csc_from_dense(X, np.array([1.0]), "logistic")
    with gb.Problem(p1) as p:
        p.set_lambda(0.01)
        p.set_params(variant="greedy", tol_kkt=1e-12, max_iter=100000, check_every=1)
        r = p.solve()
        assert r.status == 0
        o = oracle.Oracle(p1, 0.01)
        w_opt, _, _, _, _ = o.solve("ccd", tol_kkt=1e-13, max_iter=10**6)
        assert p.w()[0] == pytest.approx(w_opt[0], rel=1e-9)
    empty = workloads.Problem(5, 4, np.zeros(5, np.int64), np.zeros(0, np.int32), np.zeros(0),
                              np.array([1.0, -1, 1, 1, -1]), "logistic", np.zeros(4))
    with gb.Problem(empty) as p:
        assert p.lambda_max() == 0.0
        p.set_lambda(0.1)
        p.set_params(variant="thread_greedy")
        r = p.solve()
        assert r.status == 0 and r.iters == 0
        assert (p.w() == 0).all()
        p.set_w(np.array([1.0, 0.0, -2.0, 0.0]))  # weights on empty columns go to 0 in one step
        p.iterate(1)
        assert (p.w() == 0).all()
    prob = ragged_problem("squared", 3)
    with gb.Problem(prob) as p:
        lm = p.lambda_max()
        p.set_lambda(lm * (1 + 1e-9))
        p.set_params(variant="thread_greedy", tol_kkt=0.0, max_iter=5)
        r = p.solve()
        assert (p.w() == 0).all()


def test_invalid_input_is_rejected(gb):
    good = workloads.uniform_problem(20, 10, 3, seed=1)
    cases = []
    bad = good.row_idx.copy()
    bad[0], bad[1] = bad[1], bad[0]  # unsorted rows in column 0
    cases.append(("rows", dict(row_idx=bad)))
    bad = good.row_idx.copy()
    bad[4] = bad[3]  # duplicate row in column 1
    cases.append(("rows", dict(row_idx=bad)))
    bad = good.row_idx.copy()
    bad[7] = 20  # out of range
    cases.append(("rows", dict(row_idx=bad)))
    bad = good.col_ptr.copy()
    bad[3] = bad[5]  # not monotone
    cases.append(("col_ptr", dict(col_ptr=bad)))
    bad_y = good.y.copy()
    bad_y[2] = 0.5  # logistic labels must be +-1
    cases.append(("label", dict(y=bad_y)))
    bad_v = good.val.copy()
    bad_v[2] = np.nan
    cases.append(("value", dict(val=bad_v)))
    for _, kw in cases:
        args = dict(col_ptr=good.col_ptr, row_idx=good.row_idx, val=good.val, y=good.y)
        args.update(kw)
        with pytest.raises(gb.GencdError) as e:
            gb.gencd_create(good.n, good.k, good.nnz, args["col_ptr"], args["row_idx"], args["val"], args["y"],
                            "logistic", "f64")
        assert e.value.code == gb.GENCD_EINVAL
    with pytest.raises(gb.GencdError):
        gb.gencd_create(good.n, good.k, good.nnz + 1, good.col_ptr, good.row_idx, good.val, good.y)


def test_device_inputs_match_host_inputs(gb):
    import torch

    prob = workloads.config1("logistic")
    dev = dict(col_ptr=torch.from_numpy(prob.col_ptr).cuda(), row_idx=torch.from_numpy(prob.row_idx).cuda(),
               val=torch.from_numpy(prob.val).cuda(), y=torch.from_numpy(prob.y).cuda())
    lam = 0.05 * oracle.Oracle(prob).lambda_max()
    ws = []
    for kw in (dict(prob=prob), dict(n=prob.n, k=prob.k, loss="logistic", **dev)):
        with gb.Problem(**kw) as p:
            p.set_lambda(lam)
            p.set_params(variant="thread_greedy", blocks=100)
            p.iterate(10)
            ws.append(p.w())
    # FP64 atomics combine partial sums of columns cut by lane boundaries in
    # arrival order, so two runs agree to rounding, not bit for bit
    np.testing.assert_allclose(ws[0], ws[1], rtol=1e-13, atol=1e-15)


def test_not_converged_and_diverged_are_reported(gb):
    prob = workloads.config1("logistic")
    with gb.Problem(prob) as p:
        p.set_lambda(1e-4 * p.lambda_max())
        p.set_params(variant="thread_greedy", max_iter=5, tol_kkt=1e-14, check_every=5)
        r = p.solve()
        assert r.status == gb.GENCD_NOT_CONVERGED and r.iters == 5
    # literal beta with columns of norm^2 >> n makes every step overshoot
    X = np.array([[300.0, 0.0], [0.0, 200.0], [100.0, 100.0]])
    big = workloads.csc_from_dense(X, np.array([1.0, -2.0, 0.5]), "squared")
    with gb.Problem(big) as p:
        p.set_lambda(1e-3)
        p.set_params(variant="thread_greedy", beta_mode=1, max_iter=100000, check_every=10, tol_kkt=0.0)
        r = p.solve()
        assert r.status == gb.GENCD_EDIVERGED


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_thread_greedy_backoff_converges_where_plain_thread_greedy_diverges(gb, precision):
    # config-3 shapes, squared loss: Thread-Greedy with B = 16 diverges (the
    # FP64 oracle's too); the solve's accept backoff merges partitions until
    # the iteration converges, to the oracle's cyclic CD optimum
    prob = workloads.config3("lognormal", "squared")
    orc = oracle.Oracle(prob)
    lam = 0.05 * orc.lambda_max()
    orc.set_lambda(lam)
    w_tg, _, _, _ = orc.run("thread_greedy", 200, B=16)[:4]
    assert not orc.objective(w_tg) < orc.objective(np.zeros(prob.k))  # plain Thread-Greedy diverges
    w_opt, _, _, _, _ = orc.solve("ccd", tol_kkt=1e-11)
    with gb.Problem(prob, precision=precision) as p:
        p.set_lambda(lam)
        p.set_params(variant="thread_greedy", blocks=16, tol_kkt=1e-11 if precision == "f64" else 1e-8,
                     max_iter=400_000, check_every=10)
        r = p.solve()
        assert r.status == 0, r.as_dict()
        w = p.w()
    assert r.objective == pytest.approx(orc.objective(w_opt), rel=1e-6)
    assert orc.kkt(w) <= 1e-7
    sp = prob if precision == "f64" else oracle.stored_problem(prob, "f32")
    assert_support_matches(sp, lam, w, w_opt, label=f"backoff {precision}")


@pytest.mark.parametrize("variant,B,P", [("thread_greedy", 64, 0), ("greedy", 1, 0), ("shotgun", 0, 200)])
def test_improve_steps_match_the_oracle(gb, variant, B, P):
    # Improve delta_j (Algorithm 3, reading R11): every accepted increment
    # refined on its own coordinate before the update
    prob = workloads.config1("logistic")
    orc = oracle.Oracle(prob)
    lam = 0.05 * orc.lambda_max()
    orc.set_lambda(lam)
    iters = 15
    w_plain, _, _, _ = orc.run(variant, iters, B=B or 1, P=P or 1, seed=4)
    w_cpu, _, _, _ = orc.run(variant, iters, B=B or 1, P=P or 1, seed=4, improve_steps=500)
    assert np.abs(w_cpu - w_plain).max() > 1e-6  # the step changes the trajectory
    with gb.Problem(prob) as p:
        p.set_lambda(lam)
        p.set_params(variant=variant, blocks=B, P=P, seed=4, improve_steps=500)
        p.iterate(iters)
        w_gpu = p.w()
    np.testing.assert_array_equal(w_gpu != 0, w_cpu != 0)
    np.testing.assert_allclose(w_gpu, w_cpu, rtol=0, atol=1e-9)


@pytest.mark.parametrize("B", [17, 200])
def test_top_greedy_iterations_match(gb, B):
    # Section 7's global top-|J'| Accept (reading R12): the B lowest proxies
    prob = workloads.config1("logistic")
    orc = oracle.Oracle(prob)
    lam = 0.05 * orc.lambda_max()
    orc.set_lambda(lam)
    iters = 15
    w_cpu, _, _, st = orc.run("top_greedy", iters, B=B)
    with gb.Problem(prob) as p:
        p.set_lambda(lam)
        p.set_params(variant="top_greedy", blocks=B)
        p.stats_reset()
        p.iterate(iters)
        w_gpu = p.w()
        assert p.stats().updates == st[0]
    np.testing.assert_array_equal(w_gpu != 0, w_cpu != 0)
    np.testing.assert_allclose(w_gpu, w_cpu, rtol=0, atol=1e-10)


def test_set_loss_switches_the_problem(gb):
    # +-1 labels are valid for both losses: a problem switched to the squared
    # loss equals a problem created with it, in the same state, and back
    prob = workloads.config1("logistic")
    sq = prob.with_loss("squared", prob.y)
    w = _state(prob, 21)
    J = np.arange(prob.k, dtype=np.int32)
    with gb.Problem(prob) as p, gb.Problem(sq) as q:
        lm_logistic = p.lambda_max()
        lam = 0.05 * q.lambda_max()
        for h in (p, q):
            h.set_w(w)
            h.set_lambda(lam)
        p.set_loss("squared")
        assert p.lambda_max() == pytest.approx(q.lambda_max(), rel=1e-14)
        d1, f1 = p.propose_at(J)
        d2, f2 = q.propose_at(J)
        np.testing.assert_allclose(d1, d2, rtol=1e-12, atol=1e-300)
        np.testing.assert_allclose(f1, f2, rtol=1e-12, atol=1e-300)
        assert p.objective()[0] == pytest.approx(q.objective()[0], rel=1e-14)
        p.set_loss("logistic")
        assert p.lambda_max() == pytest.approx(lm_logistic, rel=1e-14)
        orc = oracle.Oracle(prob)
        orc.set_lambda(lam)
        assert p.objective()[0] == pytest.approx(orc.objective(w), rel=1e-13)
    # real-valued labels cannot take the logistic loss; the problem is unchanged
    lasso = workloads.config1("squared")
    with gb.Problem(lasso) as p:
        lm = p.lambda_max()
        with pytest.raises(gb.GencdError) as e:
            p.set_loss("logistic")
        assert e.value.code == gb.GENCD_EINVAL and "-1/+1" in str(e.value)
        assert p.lambda_max() == lm


# --- storage modes: bfloat16 values and index-only binary columns -----------
# The oracle runs on the values the mode stores (oracle.stored_values), so the
# comparison isolates the FP32 arithmetic: the FP32 tolerance applies.

STORAGE_CASES = {
    "cfg3-lognormal-bf16": (lambda: workloads.config3("lognormal"), "bf16"),
    "cfg3-pm1-bf16": (lambda: workloads.config3("pm1", "squared"), "bf16"),
    "ragged-bf16": (lambda: ragged_problem("logistic", 2), "bf16"),
    "zipf-slabs-bf16": (PROBLEMS["zipf-slabs-squared"], "bf16"),
    "cfg3-ones-binary": (lambda: workloads.config3("ones"), "binary"),
    "ragged-binary": (lambda: workloads.binarized(ragged_problem("squared", 3)), "binary"),
    "zipf-binary": (lambda: workloads.binarized(workloads.config2_scaled(0.002, "logistic")), "binary"),
    "zipf-slabs-binary": (lambda: workloads.binarized(PROBLEMS["zipf-slabs-squared"]()), "binary"),
}


@pytest.mark.parametrize("name", list(STORAGE_CASES))
def test_storage_modes_match_oracle(gb, name):
    make, mode = STORAGE_CASES[name]
    prob = make()
    sp = oracle.stored_problem(prob, mode)
    orc = oracle.Oracle(sp)
    lam = 0.05 * orc.lambda_max()
    orc.set_lambda(lam)
    w = _state(prob, 4)
    z = orc.fitted(w)
    rng = np.random.default_rng(6)
    J = np.concatenate([np.arange(prob.k), rng.integers(0, prob.k, 300)]).astype(np.int32)
    d_cpu, f_cpu = orc.propose(w, z, J)
    with gb.Problem(prob, precision=mode) as p:
        assert p.lambda_max() == pytest.approx(orc.lambda_max(), rel=TOL["f32"] * 10)
        p.set_lambda(lam)
        p.set_w(w)
        np.testing.assert_allclose(p.z(), z, rtol=0, atol=1e-5 * max(1.0, np.abs(z).max()))
        d_gpu, f_gpu = p.propose_at(J)
        assert_steps_close(sp, z, w, lam, J, d_gpu, f_gpu, d_cpu, f_cpu, TOL["f32"])
        d_all, f_all, kkt = p.propose_all()
        assert_steps_close(sp, z, w, lam, np.arange(prob.k), d_all, f_all, d_cpu[:prob.k], f_cpu[:prob.k],
                           TOL["f32"])
        S, _ = _scales(sp, z, lam)
        assert abs(kkt - orc.kkt(w, z)) <= TOL["f32"] * (S.max() + lam) * 10
        obj, _ = p.objective()
        assert obj == pytest.approx(orc.objective(w), rel=1e-6)


@pytest.mark.parametrize("mode,values", [("bf16", "lognormal"), ("binary", "ones")])
@pytest.mark.parametrize("loss,variant", [("logistic", "thread_greedy"), ("squared", "coloring")])
def test_storage_solve_reaches_the_stored_optimum(gb, mode, values, loss, variant):
    # Thread-Greedy has no convergence guarantee (Section 7): on the squared
    # loss here the FP64 oracle diverges at B = 16 too.  Coloring converges.
    prob = workloads.config3(values, loss)
    orc = oracle.Oracle(oracle.stored_problem(prob, mode))
    lam = 0.05 * orc.lambda_max()
    orc.set_lambda(lam)
    w_opt, _, _, _, _ = orc.solve("ccd", tol_kkt=1e-11, max_iter=4 * 10**8)
    with gb.Problem(prob, precision=mode) as p:
        p.set_lambda(lam)
        p.set_params(variant=variant, blocks=16, tol_kkt=1e-9, max_iter=200_000, check_every=50)
        r = p.solve()
        assert r.status == 0, r.as_dict()
        w = p.w()
    assert r.objective == pytest.approx(orc.objective(w_opt), rel=1e-6)
    assert_support_matches(oracle.stored_problem(prob, mode), lam, w, w_opt, label=f"{mode} {values} {loss}")


def test_storage_modes_reject_what_they_cannot_hold(gb):
    pm = workloads.config3("pm1")
    with pytest.raises(ValueError) as ref:
        oracle.stored_values(pm, "binary")
    with pytest.raises(gb.GencdError) as e:
        gb.Problem(pm, precision="binary")
    assert e.value.code == gb.GENCD_EINVAL
    col = str(ref.value).split()[1]
    assert f"column {col} " in str(e.value)
    big = workloads.config3("lognormal")
    big.val[7] = 3.4e38
    with pytest.raises(gb.GencdError) as e:
        gb.Problem(big, precision="bf16")
    assert e.value.code == gb.GENCD_EINVAL and "bfloat16" in str(e.value)


# Storage error bound (reading on storage modes): a mode that rounds X
# solves the problem P' on the stored X'.  With P* = P(w*) and P'* <= P'(w*),
#   P(w) - P* = [P(w) - P'(w)] + [P'(w) - P'*] + [P'* - P(w*)]
#             <= [P(w) - P'(w)] + gap'(w) + [P'(w*) - P(w*)],
# gap' the duality gap of w on P' (weak duality bounds P'(w) - P'*).  Every
# term is evaluated by the oracle in FP64.
def _storage_bound(prob, mode, lam, w, w_opt, P_opt):
    orig = oracle.Oracle(prob, lam)
    stored = oracle.Oracle(oracle.stored_problem(prob, mode), lam)
    bound = (orig.objective(w) - stored.objective(w)) + max(stored.duality_gap(w), 0.0) + \
        (stored.objective(w_opt) - orig.objective(w_opt))
    return bound / P_opt


SWEEP = (("pm1", ["f64", "f32", "bf16"]), ("ones", ["f64", "f32", "bf16", "binary"]),
         ("lognormal", ["f64", "f32", "bf16"]))


def test_precision_sweep_config3(gb, capsys):
    # Every storage mode on config 3's shapes (logistic, lambda = 0.01
    # lambda_max), Thread-Greedy B = 16: FP64 to KKT 1e-11, the FP32-arithmetic
    # modes to 1e-9 (the floor of FP32 sums here).  Parity isolates the
    # arithmetic: each mode's w is compared with the oracle's optimum of the
    # problem it stores (objective within 1e-6, supports equal outside the
    # columns that are fragile at the compared KKT accuracy).  The storage
    # error against the original problem is reported and held to the bound
    # above (1e-6 where the mode stores X exactly).
    rows = []
    for values, modes in SWEEP:
        prob = workloads.config3(values, "logistic")
        orc = oracle.Oracle(prob)
        lam = 0.01 * orc.lambda_max()
        orc.set_lambda(lam)
        w_opt = certified_optimum(f"cfg3_{values}_logistic", prob, lam)
        P_opt = orc.objective(w_opt)
        for mode in modes:
            sp = oracle.stored_problem(prob, mode)
            exact = bool(np.array_equal(sp.val, prob.val))
            # the optimum of the stored problem: the original one where the
            # mode stores X exactly or rounds it to FP32 (a KKT perturbation of
            # ~1e-11 here, inside the compared accuracy); bfloat16 of
            # log-normal values has its own stored optimum
            if exact or mode == "f32":
                w_ref = w_opt
            else:
                w_ref = certified_optimum(f"cfg3_{values}_logistic_{mode}", sp, lam)
            o_s = oracle.Oracle(sp, lam)
            P_ref = o_s.objective(w_ref)
            with gb.Problem(prob, precision=mode) as p:
                p.set_lambda(lam)
                p.set_params(variant="thread_greedy", blocks=16, tol_kkt=1e-11 if mode == "f64" else 1e-9,
                             max_iter=3_000_000, check_every=100)
                r = p.solve()
                assert r.status == 0, (values, mode, r.as_dict())
                w = p.w()
            rel_s = (o_s.objective(w) - P_ref) / P_ref
            assert abs(rel_s) <= 1e-6, (values, mode, rel_s)
            eps, nfrag, ndiff = assert_support_matches(sp, lam, w, w_ref, label=f"{values} {mode}")
            rel = (orc.objective(w) - P_opt) / P_opt
            bound = 1e-6 if exact else max(1e-6, _storage_bound(prob, mode, lam, w, w_opt, P_opt))
            assert rel <= bound, (values, mode, rel, bound)
            supp = int(np.sum((np.abs(w) > 1e-6) != (np.abs(w_opt) > 1e-6)))
            rows.append((values, mode, rel, bound, rel_s, np.abs(w - w_opt).max(), supp, ndiff, nfrag, eps,
                         r.iters))
    with capsys.disabled():
        print("\nprecision sweep (config 3 shapes, logistic, lambda = 0.01 lambda_max; Thread-Greedy B = 16)")
        print("  values    mode   vs original: (P(w)-P*)/P*  bound     | vs stored: rel. obj.  support diff "
              "(fragile)  KKT eps   | max|w-w*|  supp diff vs original  iters")
        for values, mode, rel, bound, rel_s, dw, supp, ndiff, nfrag, eps, it in rows:
            print(f"  {values:9s} {mode:6s} {rel:+.3e}  {bound:.1e} | {rel_s:+.2e}  {ndiff:3d} ({nfrag:3d})  "
                  f"{eps:.1e} | {dw:.2e}  {supp:3d}  {it}")


@pytest.mark.parametrize("loss", ["logistic", "squared"])
def test_block_shotgun_matches_the_oracle(gb, loss):
    # Section 7's block Shotgun (reading R14): 7 uneven column blocks, each
    # with its own P*_b from the block's spectral radius; the GPU's P*_b equal
    # the oracle's and 40 iterations follow the oracle's trajectory
    prob = workloads.config1(loss)
    orc = oracle.Oracle(prob)
    lam = 0.05 * orc.lambda_max()
    orc.set_lambda(lam)
    B = 7
    Pb_cpu = orc.block_pstar(B)
    with gb.Problem(prob) as p:
        p.set_lambda(lam)
        Pb, rho = p.block_pstar(B)
        np.testing.assert_array_equal(Pb, Pb_cpu)
        p.set_params(variant="shotgun_blocks", blocks=B, seed=4)
        p.stats_reset()
        p.iterate(40)
        w_gpu = p.w()
        upd = p.stats().updates
    w_cpu, _, _, st = orc.run("shotgun_blocks", 40, B=B, block_P=Pb_cpu, seed=4)
    # the oracle counts every selected column; the library counts the applied
    # (non-zero) steps
    assert 0 < upd <= st[0]
    np.testing.assert_array_equal(w_gpu != 0, w_cpu != 0)
    np.testing.assert_allclose(w_gpu, w_cpu, rtol=0, atol=1e-10)


def test_block_shotgun_solve_reaches_the_optimum(gb):
    prob = workloads.uniform_problem(1000, 2000, 10, values="pm1", loss="logistic", n_planted=30, seed=21)
    orc = oracle.Oracle(prob)
    lam = 0.05 * orc.lambda_max()
    orc.set_lambda(lam)
    w_opt, _, _, kkt, _ = orc.solve("ccd", tol_kkt=1e-11)
    with gb.Problem(prob) as p:
        p.set_lambda(lam)
        p.set_params(variant="shotgun_blocks", blocks=16, tol_kkt=1e-10, max_iter=2_000_000, check_every=100)
        r = p.solve()
        assert r.status == 0, r.as_dict()
        w = p.w()
        with pytest.raises(gb.GencdError):
            p.set_params(variant="shotgun_blocks", blocks=1025)
    assert r.objective == pytest.approx(orc.objective(w_opt), rel=1e-6)
    assert_support_matches(prob, lam, w, w_opt, label="block shotgun")


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("name", ["cfg1-logistic", "cfg1-squared", "ragged-logistic", "zipf-slabs-squared"])
def test_duality_gap_matches_the_oracle(gb, name, precision):
    # the device's duality gap (objective, dual point from the FP64 loss
    # derivative scaled by lambda / max |g|) against the oracle's at the same w
    prob = PROBLEMS[name]()
    orc = oracle.Oracle(prob)
    lam = 0.05 * orc.lambda_max()
    orc.set_lambda(lam)
    w = _state(prob, 31)
    with gb.Problem(prob, precision=precision) as p:
        p.set_lambda(lam)
        p.set_w(w)
        gap, primal, dual = p.duality_gap()
    sp = prob if precision == "f64" else oracle.stored_problem(prob, "f32")
    o_s = oracle.Oracle(sp, lam)
    gap_cpu = o_s.duality_gap(w)
    P = o_s.objective(w)
    assert primal == pytest.approx(P, rel=1e-13 if precision == "f64" else 1e-9)
    # P and D are each accurate to their sums' rounding; the scale of D's
    # dual point comes from max |g| in the problem's arithmetic
    tol = 1e-11 if precision == "f64" else 1e-5
    assert abs(gap - gap_cpu) <= tol * (abs(P) + abs(P - gap_cpu))
    assert gap_cpu >= 0.0


@pytest.mark.parametrize("loss", ["logistic", "squared"])
def test_solve_to_a_duality_gap_certifies_the_objective(gb, loss):
    # stopping at a relative duality gap of 1e-9 bounds (P(w) - P*) / P(w)
    prob = workloads.uniform_problem(1000, 2000, 10, values="pm1", loss=loss, n_planted=30, seed=21)
    orc = oracle.Oracle(prob)
    lam = 0.05 * orc.lambda_max()
    orc.set_lambda(lam)
    w_opt, _, _, kkt, _ = orc.solve("ccd", tol_kkt=1e-11)
    P_opt = orc.objective(w_opt)
    with gb.Problem(prob) as p:
        p.set_lambda(lam)
        p.set_params(variant="thread_greedy", blocks=16, tol_kkt=0.0, tol_gap=1e-9, max_iter=400_000,
                     check_every=50)
        r = p.solve()
        assert r.status == 0, r.as_dict()
        w = p.w()
        gap, primal, _ = p.duality_gap()
    assert gap <= 1e-9 * abs(primal) * (1 + 1e-6)
    assert orc.duality_gap(w) <= 1e-9 * abs(primal) * (1 + 1e-3)
    assert (orc.objective(w) - P_opt) / P_opt <= 1e-9 * (1 + 1e-3)


@pytest.mark.parametrize("loss", ["logistic", "squared"])
def test_top_greedy_solve_reaches_the_optimum(gb, loss):
    # the global top-|J'| Accept has no convergence guarantee either: its solve
    # backs off (|J'| / G accepted, G growing 4x on a rise of the objective)
    # and reaches the oracle's optimum
    prob = workloads.uniform_problem(1000, 2000, 10, values="pm1", loss=loss, n_planted=30, seed=21)
    orc = oracle.Oracle(prob)
    lam = 0.05 * orc.lambda_max()
    orc.set_lambda(lam)
    w_opt, _, _, kkt, _ = orc.solve("ccd", tol_kkt=1e-11)
    with gb.Problem(prob) as p:
        p.set_lambda(lam)
        p.set_params(variant="top_greedy", blocks=64, tol_kkt=1e-10, max_iter=400_000, check_every=50)
        r = p.solve()
        assert r.status == 0, r.as_dict()
        w = p.w()
    assert r.objective == pytest.approx(orc.objective(w_opt), rel=1e-6)
    assert_support_matches(prob, lam, w, w_opt, label=f"top-|J'| {loss}")


@pytest.mark.parametrize("split", [0, 20, 24, 28, 31])
def test_every_propose_schedule_matches_the_oracle(gb, split):
    # the autotuner's candidates (two kernels, or the fused kernel with each
    # split of its warps) compute the same proposals, heavy and light columns
    prob = PROBLEMS["zipf-slabs-squared"]()
    orc = oracle.Oracle(prob)
    lam = 0.05 * orc.lambda_max()
    orc.set_lambda(lam)
    w = _state(prob, 41)
    z = orc.fitted(w)
    J = np.arange(prob.k, dtype=np.int32)
    d_cpu, f_cpu = orc.propose(w, z, J)
    with gb.Problem(prob, precision="f32") as p:
        p.set_lambda(lam)
        p.set_w(w)
        gb.gencd_set_propose_schedule(p.h, split)
        assert gb.gencd_propose_schedule(p.h)[0] == split
        for _ in range(2):  # the light-tile pool's counter is reset between launches
            d_all, f_all, kkt = p.propose_all()
            assert_steps_close(prob, z, w, lam, J, d_all, f_all, d_cpu, f_cpu, TOL["f32"])
        with pytest.raises(gb.GencdError):
            gb.gencd_set_propose_schedule(p.h, 17)


@pytest.mark.parametrize("precision,tol_rel", [("f32", 1e-3), ("f64", 1e-6)])
def test_config2_at_one_percent_solves_to_a_certified_point(gb, precision, tol_rel):
    # config 2's law at 1/100 of its size (n = 10,000, k = 40,000, 2e6 nnz),
    # the benchmark's Thread-Greedy (B = 1024): solved to KKT <= tol_rel lambda,
    # the oracle's FP64 KKT value and duality gap at the GPU's w certify it
    prob = workloads.config2_scaled(0.01, "logistic")
    orc = oracle.Oracle(prob)
    lam = 0.05 * orc.lambda_max()
    orc.set_lambda(lam)
    with gb.Problem(prob, precision=precision) as p:
        p.set_lambda(lam)
        p.set_params(variant="thread_greedy", blocks=1024, tol_kkt=tol_rel * lam, max_iter=200_000, check_every=10)
        r = p.solve()
        assert r.status == 0, r.as_dict()
        w = p.w()
    sp = prob if precision == "f64" else oracle.stored_problem(prob, "f32")
    o_s = oracle.Oracle(sp, lam)
    kkt = o_s.kkt(w)
    # FP32 sums: the oracle's KKT value may exceed the device's by their rounding
    assert kkt <= tol_rel * lam * (1.0 if precision == "f64" else 1.5) + (0 if precision == "f64" else 1e-9), kkt
    P = o_s.objective(w)
    assert o_s.duality_gap(w) <= (1e-5 if precision == "f64" else 1e-2) * P
    assert r.objective == pytest.approx(P, rel=1e-9)
