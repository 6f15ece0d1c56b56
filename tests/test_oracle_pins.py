"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a published
vector, a closed form, a hand-derived optimum, brute force on a tiny problem,
an optimality condition evaluated independently, or an invariant the paper
states.  A dropped term, a wrong sign or a transposed index in the oracle
fails at least one of them.
"""

import itertools
import os

import numpy as np
import pytest

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                parts = line.split()
                rows.setdefault(parts[0], {})[parts[1]] = [float(x) for x in parts[2:]]
    return rows


def _dense_objective(X, y, loss, lam, w):
    t = X @ w
    if loss == "squared":
        f = 0.5 * (y - t) ** 2
    else:
        f = np.logaddexp(0.0, -y * t)
    return f.mean() + lam * np.abs(w).sum()


def _dense_grad(X, y, loss, w):
    t = X @ w
    d = (t - y) if loss == "squared" else -y / (1.0 + np.exp(y * t))
    return X.T @ d / X.shape[0]


# --- selection randomness -------------------------------------------------------

def test_splitmix64_published_vectors():
    with open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for idx, hexval in rows:
        assert oracle.splitmix64(0, int(idx)) == int(hexval, 16)


def test_permutation_sorts_the_keys():
    for seed, epoch, m in [(0, 0, 1), (7, 3, 257), (2**63 + 5, 11, 5000)]:
        perm = oracle.permutation(seed, epoch, m)
        assert sorted(perm.tolist()) == list(range(m))
        s = oracle.splitmix64(seed, epoch)
        keys = [(oracle.splitmix64(s, i) >> 32, i) for i in range(m)]
        assert [i for _, i in sorted(keys)] == perm.tolist()
    assert not np.array_equal(oracle.permutation(1, 0, 100), oracle.permutation(1, 1, 100))


# --- losses and the step -------------------------------------------------------

@pytest.mark.parametrize("loss", ["squared", "logistic"])
def test_dloss_is_the_derivative_in_t(loss):
    h = 1e-5
    for y in (-1.0, 1.0, 0.3):
        if loss == "logistic" and abs(y) != 1.0:
            continue
        for t in (-30.0, -2.0, -0.1, 0.0, 0.7, 5.0, 40.0):
            fd = (oracle.loss(loss, y, t + h) - oracle.loss(loss, y, t - h)) / (2 * h)
            assert oracle.dloss(loss, y, t) == pytest.approx(fd, rel=1e-7, abs=1e-10)


def test_beta_bounds_the_second_derivative():
    # Section 3.2: beta = 1 (squared) and 1/4 (logistic), and it is the supremum.
    assert oracle.beta("squared") == 1.0
    assert oracle.beta("logistic") == 0.25
    h = 1e-4
    ts = np.linspace(-20, 20, 4001)
    for loss in ("squared", "logistic"):
        d2 = [(oracle.dloss(loss, 1.0, t + h) - oracle.dloss(loss, 1.0, t - h)) / (2 * h) for t in ts]
        assert max(d2) <= oracle.beta(loss) + 1e-7
        assert max(d2) >= oracle.beta(loss) - 1e-6


def test_logistic_loss_is_stable_at_large_margins():
    assert oracle.loss("logistic", 1.0, 800.0) == pytest.approx(np.exp(-800.0), abs=1e-300)
    assert oracle.loss("logistic", 1.0, -800.0) == pytest.approx(800.0, rel=1e-15)
    assert oracle.dloss("logistic", -1.0, -800.0) == 0.0 or abs(oracle.dloss("logistic", -1.0, -800.0)) < 1e-300


def test_eq4_clip_form_equals_soft_threshold_form():
    # Section 3.1: -psi(w; (g-l)/H, (g+l)/H) == s_{l/H}(w - g/H) - w.
    rng = np.random.default_rng(1)
    for _ in range(20000):
        g, w = rng.normal(size=2) * rng.choice([1e-3, 1.0, 1e3], size=2)
        lam = abs(rng.normal()) * rng.choice([0.0, 1e-3, 1.0])
        H = abs(rng.normal()) + 1e-3
        d, _ = oracle.step(g, w, lam, H)
        x = w - g / H
        soft = np.sign(x) * max(abs(x) - lam / H, 0.0)
        assert d == pytest.approx(soft - w, rel=1e-12, abs=1e-12 * (abs(w) + abs(g) / H + lam / H))


def test_step_sign_and_proxy_special_cases():
    # w = 0 and |g| <= lambda: no move, proxy 0.
    assert oracle.step(0.3, 0.0, 0.5, 2.0) == (0.0, 0.0)
    # w = 0 and g > lambda: move negative by (g - lambda)/beta.
    d, phi = oracle.step(1.5, 0.0, 0.5, 2.0)
    assert d == -0.5
    assert phi == pytest.approx(0.5 * 2.0 * 0.25 + 1.5 * (-0.5) + 0.5 * 0.5)  # = -0.25
    assert phi == pytest.approx(-0.25)
    # beta_j == 0 (empty column): the exact minimiser of lambda |w + d|.
    assert oracle.step(0.0, 2.0, 0.1, 0.0) == (-2.0, pytest.approx(-0.2))


def _random_state(prob, rng, frac=0.3):
    w = np.where(rng.random(prob.k) < frac, rng.normal(0, 0.5, prob.k), 0.0)
    return w


@pytest.mark.parametrize("seed", [0, 1])
def test_squared_step_is_the_exact_coordinate_minimiser(seed):
    # For squared loss beta_j = c_j = H_jj (Eq. 4 == Eq. 7) and the proxy of
    # Eq. 9 is the exact change of the objective.
    prob = workloads.uniform_problem(60, 40, 6, values="lognormal", loss="squared", seed=seed)
    X = prob.to_dense()
    lam = 0.02
    o = oracle.Oracle(prob, lam)
    rng = np.random.default_rng(seed)
    w = _random_state(prob, rng)
    z = o.fitted(w)
    J = np.arange(prob.k, dtype=np.int32)
    delta, phi = o.propose(w, z, J)
    P0 = _dense_objective(X, prob.y, "squared", lam, w)
    for j in range(prob.k):
        e = np.zeros(prob.k)
        e[j] = 1.0
        f = lambda d: _dense_objective(X, prob.y, "squared", lam, w + d * e)
        # golden-section search on the true objective around the proposal
        a, b = delta[j] - 2.0, delta[j] + 2.0
        gr = (np.sqrt(5) - 1) / 2
        for _ in range(200):
            c, d = b - gr * (b - a), a + gr * (b - a)
            if f(c) < f(d):
                b = d
            else:
                a = c
        # the search resolves the argmin only to ~sqrt(eps) of a flat quadratic
        assert delta[j] == pytest.approx(0.5 * (a + b), abs=1e-6)
        assert f(delta[j]) <= f(0.5 * (a + b)) + 1e-14
        assert phi[j] == pytest.approx(f(delta[j]) - P0, abs=1e-12)


@pytest.mark.parametrize("beta_mode", [0, 1])
def test_logistic_step_never_increases_the_objective(beta_mode):
    # Eq. 5-6: the surrogate bounds F from above, so the true change is <= phi <= 0.
    prob = workloads.uniform_problem(80, 50, 8, values="lognormal", loss="logistic", seed=3)
    X = prob.to_dense()
    lam = 0.003
    o = oracle.Oracle(prob, lam, beta_mode=beta_mode)
    rng = np.random.default_rng(5)
    w = _random_state(prob, rng)
    z = o.fitted(w)
    delta, phi = o.propose(w, z, np.arange(prob.k, dtype=np.int32))
    P0 = _dense_objective(X, prob.y, "logistic", lam, w)
    assert (phi <= 0).all()
    assert (phi < 0).any()
    for j in range(prob.k):
        w2 = w.copy()
        w2[j] += delta[j]
        change = _dense_objective(X, prob.y, "logistic", lam, w2) - P0
        assert change <= phi[j] + 1e-13


def test_gradient_and_col_scale_match_dense_algebra():
    prob = workloads.uniform_problem(50, 30, 7, values="lognormal", loss="logistic", seed=2)
    X = prob.to_dense()
    o = oracle.Oracle(prob, 0.01)
    w = _random_state(prob, np.random.default_rng(2))
    z = o.fitted(w)
    np.testing.assert_allclose(z, X @ w, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(o.gradient(z), _dense_grad(X, prob.y, "logistic", w), rtol=1e-12, atol=1e-16)
    np.testing.assert_allclose(o.col_scale(), (X * X).sum(0) / prob.n, rtol=1e-14)
    assert o.objective(w) == pytest.approx(_dense_objective(X, prob.y, "logistic", 0.01, w), rel=1e-13)


# --- optima --------------------------------------------------------------------

def test_golden_worked_examples():
    g = _golden("worked_examples.txt")
    p = workloads.csc_from_dense(np.array([[1.0, 1.0], [1.0, -1.0]]), np.array([3.0, 1.0]), "squared")
    o = oracle.Oracle(p, 0.5)
    w, z, it, kkt, _ = o.solve("ccd", tol_kkt=1e-14)
    np.testing.assert_allclose(w, g["lasso_orthogonal_2x2"]["w"], rtol=0, atol=1e-14)
    assert o.objective(w) == pytest.approx(g["lasso_orthogonal_2x2"]["objective"][0], rel=1e-15)

    p = workloads.csc_from_dense(np.ones((3, 1)), np.ones(3), "logistic")
    o = oracle.Oracle(p, 0.1)
    w, z, it, kkt, _ = o.solve("ccd", tol_kkt=1e-15, max_iter=100000)
    assert w[0] == pytest.approx(g["logistic_constant_column"]["w"][0], rel=1e-12)
    assert o.objective(w) == pytest.approx(g["logistic_constant_column"]["objective"][0], rel=1e-14)


def test_orthogonal_design_lasso_is_soft_thresholding():
    # Disjoint column supports: the optimum is w_j = s_lambda(X_j^T y / n) / c_j.
    rng = np.random.default_rng(4)
    n, k = 120, 30
    X = np.zeros((n, k))
    rows = rng.permutation(n)
    for j in range(k):
        X[rows[4 * j:4 * j + 4], j] = rng.normal(size=4)
    y = rng.normal(size=n)
    p = workloads.csc_from_dense(X, y, "squared")
    b = X.T @ y / n
    lam = 0.5 * np.abs(b).max()
    o = oracle.Oracle(p, lam)
    w, _, _, kkt, _ = o.solve("ccd", tol_kkt=1e-14)
    c = (X * X).sum(0) / n
    expect = np.sign(b) * np.maximum(np.abs(b) - lam, 0.0) / c
    np.testing.assert_allclose(w, expect, rtol=1e-12, atol=1e-14)
    assert (w == 0).sum() > 0 and (w != 0).sum() > 0


def test_k1_lasso_is_exact_in_one_step():
    rng = np.random.default_rng(6)
    X = rng.normal(size=(40, 1))
    y = rng.normal(size=40) + 2 * X[:, 0]
    p = workloads.csc_from_dense(X, y, "squared")
    lam = 0.1
    o = oracle.Oracle(p, lam)
    w, _, _, _ = o.run("ccd", 1)
    b = X[:, 0] @ y / 40
    c = X[:, 0] @ X[:, 0] / 40
    assert w[0] == pytest.approx(np.sign(b) * max(abs(b) - lam, 0) / c, rel=1e-14)


def test_k1_logistic_matches_bisection_on_the_subgradient():
    rng = np.random.default_rng(7)
    X = rng.normal(size=(50, 1))
    y = np.where(X[:, 0] + rng.normal(size=50) > 0, 1.0, -1.0)
    p = workloads.csc_from_dense(X, y, "logistic")
    lam = 0.02
    o = oracle.Oracle(p, lam)
    w, _, _, kkt, _ = o.solve("ccd", tol_kkt=1e-13, max_iter=10**6)

    def g(v):  # derivative of F along the single coordinate
        return float(np.mean(-y * X[:, 0] / (1.0 + np.exp(y * X[:, 0] * v))))

    assert abs(g(0.0)) > lam  # optimum away from zero
    s = -np.sign(g(0.0))
    lo, hi = 0.0, s * 100.0
    for _ in range(200):  # g(v) + lambda s = 0 on the side of sign s
        mid = 0.5 * (lo + hi)
        if (g(mid) + lam * s) * s < 0:
            lo = mid
        else:
            hi = mid
    assert w[0] == pytest.approx(0.5 * (lo + hi), rel=1e-9)


def _brute_force(X, y, loss, lam):
    """Enumerate sign patterns; solve the smooth restricted problem; keep the
    pattern whose solution is sign-consistent and satisfies the KKT conditions."""
    n, k = X.shape
    best = None
    for pattern in itertools.product((-1, 0, 1), repeat=k):
        s = np.array(pattern, float)
        S = np.flatnonzero(s)
        w = np.zeros(k)
        if S.size:
            XS = X[:, S]
            if loss == "squared":
                A = XS.T @ XS / n
                rhs = XS.T @ y / n - lam * s[S]
                w[S] = np.linalg.solve(A, rhs)
            else:
                # damped Newton on the smooth F(w_S) + lambda s_S^T w_S; this
                # restricted problem may have no minimiser (then skip it)
                def h(v):
                    return np.logaddexp(0.0, -y * (XS @ v)).mean() + lam * s[S] @ v

                v = np.zeros(S.size)
                converged = False
                for _ in range(200):
                    t = XS @ v
                    sig = 0.5 * (1.0 - np.tanh(0.5 * y * t))  # 1 / (1 + e^{y t})
                    grad = XS.T @ (-y * sig) / n + lam * s[S]
                    if np.abs(grad).max() < 1e-10:  # rounding floor is ~1e-13
                        converged = True
                    if np.abs(grad).max() < 1e-15:
                        break
                    Hs = (XS.T * (sig * (1 - sig))) @ XS / n + 1e-300 * np.eye(S.size)
                    try:
                        step = np.linalg.solve(Hs, grad)
                    except np.linalg.LinAlgError:
                        break
                    a = 1.0
                    while h(v - a * step) > h(v) - 1e-4 * a * (grad @ step) and a > 1e-12:
                        a *= 0.5
                    if np.abs(a * step).max() <= 1e-16 * (1 + np.abs(v).max()):
                        break
                    v = v - a * step
                    if np.abs(v).max() > 1e6:
                        converged = False
                        break
                if not converged:
                    continue
                w[S] = v
            if np.any(np.sign(w[S]) != s[S]):
                continue
        g = _dense_grad(X, y, loss, w)
        ok = True
        for j in range(k):
            if s[j] == 0 and abs(g[j]) > lam + 1e-10:
                ok = False
            if s[j] != 0 and abs(g[j] + lam * s[j]) > 1e-8:
                ok = False
        if ok:
            P = _dense_objective(X, y, loss, lam, w)
            if best is None or P < best[0]:
                best = (P, w)
    return best


@pytest.mark.parametrize("loss", ["squared", "logistic"])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tiny_problems_match_brute_force(loss, seed):
    p = workloads.tiny_problem(8, 4, loss=loss, seed=seed)
    X = p.to_dense()
    o = oracle.Oracle(p)
    lam = 0.2 * o.lambda_max()
    o.set_lambda(lam)
    Pbf, wbf = _brute_force(X, p.y, loss, lam)
    w, _, _, kkt, _ = o.solve("ccd", tol_kkt=1e-13, max_iter=10**7)
    assert kkt <= 1e-13
    np.testing.assert_allclose(w, wbf, rtol=1e-7, atol=1e-9)
    assert o.objective(w) == pytest.approx(Pbf, rel=1e-12)
    assert ((w != 0) == (np.abs(wbf) > 0)).all()


def test_lambda_max_is_the_zero_threshold():
    p = workloads.uniform_problem(100, 60, 5, values="lognormal", loss="logistic", seed=9)
    o = oracle.Oracle(p)
    lm = o.lambda_max()
    X = p.to_dense()
    assert lm == pytest.approx(np.abs(_dense_grad(X, p.y, "logistic", np.zeros(p.k))).max(), rel=1e-13)
    o.set_lambda(lm * (1 + 1e-9))
    w, _, it, kkt, _ = o.solve("ccd", tol_kkt=0.0, max_iter=5 * p.k)
    assert (w == 0).all() and kkt == 0.0
    o.set_lambda(lm * 0.999)
    w, _, _, _, _ = o.solve("ccd", tol_kkt=1e-12)
    assert (w != 0).sum() >= 1


@pytest.mark.parametrize("loss", ["squared", "logistic"])
def test_kkt_conditions_hold_at_convergence(loss):
    p = workloads.uniform_problem(300, 400, 10, values="pm1", loss=loss, n_planted=20, seed=11)
    o = oracle.Oracle(p)
    lam = 0.05 * o.lambda_max()
    o.set_lambda(lam)
    w, z, it, kkt, _ = o.solve("ccd", tol_kkt=1e-9)
    g = _dense_grad(p.to_dense(), p.y, loss, w)
    zero = w == 0
    assert np.all(np.abs(g[zero]) <= lam + 1e-9)
    assert np.all(np.abs(g[~zero] + lam * np.sign(w[~zero])) <= 1e-8)
    assert (~zero).sum() > 0


# --- invariants the paper states ------------------------------------------------

@pytest.mark.parametrize("variant", ["ccd", "coloring"])
def test_objective_is_monotone_for_sequential_and_coloring(variant):
    # Section 3.2: the Eq. 7 step never increases the objective; Section 4.1:
    # Coloring behaves like sequential CD.
    p = workloads.uniform_problem(200, 300, 8, values="lognormal", loss="logistic", seed=12)
    o = oracle.Oracle(p)
    o.set_lambda(0.02 * o.lambda_max())
    colors = o.color()[0] if variant == "coloring" else None
    _, _, tr, _ = o.run(variant, 600, colors=colors, seed=3, trace=True)
    P0 = o.objective(np.zeros(p.k))
    seq = np.concatenate([[P0], tr])
    assert np.all(np.diff(seq) <= 1e-15 * np.abs(seq[:-1]))
    assert seq[-1] < P0


def test_coloring_equals_ccd_in_colour_major_order():
    # Section 4.1: updating one colour class == updating its features in sequence.
    p = workloads.uniform_problem(150, 200, 6, values="lognormal", loss="logistic", seed=13)
    o = oracle.Oracle(p)
    o.set_lambda(0.01 * o.lambda_max())
    colors, C = o.color()
    seed = 21
    w_col, z_col, _, _ = o.run("coloring", C, colors=colors, seed=seed)
    order = []
    for c in oracle.permutation(seed, 0, C):
        order.extend(np.flatnonzero(colors == c).tolist())
    assert sorted(order) == list(range(p.k))
    # relabel the columns so that colour-major order becomes index order, then CCD
    X = p.to_dense()[:, order]
    q = workloads.csc_from_dense(X, p.y, "logistic")
    oq = oracle.Oracle(q, o.lam)
    w_ccd, z_ccd, _, _ = oq.run("ccd", p.k)
    assert np.array_equal(w_ccd, w_col[order])
    assert np.array_equal(z_ccd, z_col)


def test_greedy_equals_thread_greedy_with_one_partition():
    p = workloads.uniform_problem(150, 200, 6, values="pm1", loss="logistic", seed=14)
    o = oracle.Oracle(p)
    o.set_lambda(0.05 * o.lambda_max())
    a = o.run("greedy", 40)
    b = o.run("thread_greedy", 40, B=1)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert (a[0] != 0).sum() >= 1


def test_thread_greedy_accepts_the_best_proxy_per_partition():
    p = workloads.uniform_problem(120, 97, 5, values="lognormal", loss="squared", seed=15)
    o = oracle.Oracle(p)
    o.set_lambda(0.1 * o.lambda_max())
    rng = np.random.default_rng(15)
    w0 = _random_state(p, rng, 0.2)
    z0 = o.fitted(w0)
    delta, phi = o.propose(w0, z0, np.arange(p.k, dtype=np.int32))
    for B in (1, 7, 97, 200):
        w, _, _, st = o.run("thread_greedy", 1, w=w0, z=z0, B=B)
        expect = w0.copy()
        accepted = 0
        for b in range(B):
            lo, hi = b * p.k // B, (b + 1) * p.k // B
            if hi > lo:
                j = lo + int(np.argmin(phi[lo:hi]))  # argmin keeps the first minimum
                if phi[j] < 0:
                    expect[j] += delta[j]
                    accepted += 1
        np.testing.assert_array_equal(w, expect)
        assert st[0] == accepted  # a partition whose best proxy is 0 accepts nothing
    assert (phi == 0).any() and (phi < 0).any()


def test_thread_greedy_ties_go_to_the_lower_column():
    # Duplicate columns give identical proxies; the lower index must win.
    rng = np.random.default_rng(19)
    base = rng.normal(size=(40, 3)) * (rng.random((40, 3)) < 0.5)
    X = np.concatenate([base, base], axis=1)[:, [0, 3, 1, 4, 2, 5]]  # pairs (0,1), (2,3), (4,5)
    y = rng.normal(size=40)
    p = workloads.csc_from_dense(X, y, "squared")
    o = oracle.Oracle(p, 0.0)
    for B in (1, 3):
        w, _, _, _ = o.run("thread_greedy", 1, B=B)
        moved = np.flatnonzero(w)
        assert moved.size == B and all(j % 2 == 0 for j in moved)


def test_shotgun_selects_each_column_once_per_epoch():
    p = workloads.uniform_problem(100, 103, 4, values="pm1", loss="squared", seed=16)
    o = oracle.Oracle(p)
    o.set_lambda(0.5 * o.lambda_max())
    P = 10
    perm = oracle.permutation(5, 0, p.k)
    w0 = np.zeros(p.k)
    z0 = o.fitted(w0)
    # one epoch = ceil(103/10) = 11 iterations; the Jacobi step of each chunk
    w, z = w0, z0
    for t in range(11):
        J = np.sort(perm[t * P:(t + 1) * P]).astype(np.int32)
        d, _ = o.propose(w, z, J)
        w = w.copy()
        w[J] += d
        z = o.fitted(w)
    w_run, z_run, _, st = o.run("shotgun", 11, P=P, seed=5)
    np.testing.assert_allclose(w_run, w, rtol=1e-14, atol=1e-16)
    assert st[0] == p.k  # every column proposed and accepted once


def test_coloring_is_a_valid_first_fit_distance2_colouring():
    p = workloads.uniform_problem(90, 150, 5, values="pm1", loss="squared", seed=17)
    o = oracle.Oracle(p)
    colors, C = o.color()
    X = p.to_dense() != 0
    assert colors.min() == 0 and colors.max() == C - 1
    for i in range(p.n):  # columns sharing a row have distinct colours
        cs = colors[X[i]]
        assert len(set(cs.tolist())) == cs.size
    assert C >= X.sum(1).max()
    adj = (X.T.astype(int) @ X.astype(int)) > 0
    for j in range(p.k):  # first-fit: every smaller colour is used by a lower neighbour
        lower = set(colors[:j][adj[j, :j]].tolist())
        assert all(c in lower for c in range(colors[j]))
        assert colors[j] not in lower


def test_spectral_radius_matches_eigvalsh():
    p = workloads.uniform_problem(80, 60, 6, values="lognormal", loss="squared", seed=18)
    scale = np.random.default_rng(18).uniform(0.2, 5.0, p.k)  # columns of different norms
    p.val = p.val * np.repeat(scale, np.diff(p.col_ptr))
    X = p.to_dense()
    d = 1.0 / np.sqrt((X * X).sum(0))
    M = (X * d).T @ (X * d)
    rho_exact = np.linalg.eigvalsh(M)[-1]
    rho, it = oracle.Oracle(p).spectral_radius(max_iter=5000, rel_tol=1e-15)
    assert rho == pytest.approx(rho_exact, rel=1e-9)
    assert oracle.pstar(p.k, rho) == max(1, int(np.floor(p.k / (2 * rho_exact))))


def test_empty_columns_and_rows_are_handled():
    X = np.zeros((6, 5))
    X[0, 0], X[2, 0], X[2, 2], X[5, 2], X[1, 4] = 1.0, -2.0, 0.5, 1.5, 3.0
    y = np.array([1.0, -1.0, 1.0, -1.0, 1.0, 1.0])
    p = workloads.csc_from_dense(X, y, "logistic")
    o = oracle.Oracle(p)
    o.set_lambda(0.05)
    w0 = np.array([0.0, 0.7, 0.0, -0.3, 0.0])  # weights on the empty columns 1 and 3
    w, _, _, _, _ = o.solve("ccd", tol_kkt=1e-12, w=w0)
    assert w[1] == 0.0 and w[3] == 0.0
    assert o.kkt(w) <= 1e-12
    Pbf, wbf = _brute_force(X[:, [0, 2, 4]], y, "logistic", 0.05)
    np.testing.assert_allclose(w[[0, 2, 4]], wbf, atol=1e-8)



def _one_column(vals):
    vals = np.asarray(vals, np.float64)
    return workloads.Problem(1, 1, np.array([0, vals.size], np.int64), np.zeros(vals.size, np.int32), vals,
                             np.ones(1), "squared", np.zeros(1))


def test_stored_values_bf16_rounds_to_nearest_even():
    # R10: bfloat16 keeps 7 mantissa bits of the FP32 value; a halfway case
    # goes to the even neighbour, anything above half rounds away from zero
    h = 2.0 ** -8  # half of bfloat16's last place at 1
    cases = [(1.0, 1.0), (1.0 + h, 1.0), (1.0 + 3 * h, 1.0 + 4 * h), (-(1.0 + h), -1.0),
             (1.0 + h + 2.0 ** -20, 1.0 + 2 * h), (1.0 + h - 2.0 ** -20, 1.0), (0.0, 0.0),
             (2.0 ** -130, 2.0 ** -130), (2.0 ** -140, 0.0), (-(2.0 ** 100) * (1 + 3 * h), -(2.0 ** 100) * (1 + 4 * h)),
             # FP32 rounds first: 1 + h + 2^-30 is 1 + h in FP32, a tie that goes to 1
             (1.0 + h + 2.0 ** -30, 1.0)]
    out = oracle.stored_values(_one_column([c[0] for c in cases]), "bf16")
    np.testing.assert_array_equal(out, [c[1] for c in cases])
    with pytest.raises(ValueError, match="bfloat16 range"):
        oracle.stored_values(_one_column([1.0, 3.4e38]), "bf16")


def test_stored_values_match_library_conversions():
    # FP32 storage is numpy's float32 cast; bfloat16 storage is PyTorch's CPU
    # float32 -> bfloat16 conversion (round to nearest even)
    import torch

    rng = np.random.default_rng(3)
    v = np.concatenate([rng.lognormal(0, 3, 20_000) * np.where(rng.random(20_000) < 0.5, -1, 1),
                        rng.normal(size=1000) * 1e-39])
    p = _one_column(v)
    np.testing.assert_array_equal(oracle.stored_values(p, "f64"), v)
    f32 = v.astype(np.float32)
    np.testing.assert_array_equal(oracle.stored_values(p, "f32"), f32.astype(np.float64))
    ref = torch.from_numpy(f32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(oracle.stored_values(p, "bf16"), ref)


def test_stored_values_binary_needs_one_value_per_column():
    p = workloads.config3("ones")
    np.testing.assert_array_equal(oracle.stored_values(p, "binary"), np.ones(p.nnz))
    b = workloads.binarized(workloads.config2_scaled(0.002))
    np.testing.assert_array_equal(oracle.stored_values(b, "binary"), b.val.astype(np.float32))
    pm = workloads.config3("pm1")
    first_mixed = next(j for j in range(pm.k)
                       if np.unique(pm.val[pm.col_ptr[j]:pm.col_ptr[j + 1]]).size > 1)
    with pytest.raises(ValueError, match=f"column {first_mixed} "):
        oracle.stored_values(pm, "binary")


# --- R11: "Improve delta_j" (Algorithm 3, Section 4.1) ----------------------

def _coordinate_objective(orc, w, j):
    def h(d):
        w2 = w.copy()
        w2[j] += d
        return orc.objective(w2)
    return h


def test_improve_keeps_the_exact_squared_loss_step():
    # squared loss, beta_j = c_j: the Eq. 7 step is the coordinate's exact
    # minimiser (Eq. 4), so the improvement stops at once
    p = workloads.tiny_problem(30, 12, loss="squared", seed=4)
    orc = oracle.Oracle(p)
    orc.set_lambda(0.05 * orc.lambda_max())
    w = np.random.default_rng(4).normal(0, 0.5, p.k)
    z = orc.fitted(w)
    d0, _ = orc.propose(w, z, np.arange(p.k, dtype=np.int32))
    for j in range(p.k):
        assert orc.improve(w, z, j, d0[j], 500) == pytest.approx(d0[j], rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_improve_reaches_the_logistic_coordinate_minimiser(seed):
    from scipy.optimize import minimize_scalar

    p = workloads.tiny_problem(40, 10, loss="logistic", seed=seed)
    orc = oracle.Oracle(p)
    orc.set_lambda(0.02 * orc.lambda_max())
    w = np.random.default_rng(seed).normal(0, 1.0, p.k) * (np.random.default_rng(seed + 9).random(p.k) < 0.5)
    z = orc.fitted(w)
    d0, _ = orc.propose(w, z, np.arange(p.k, dtype=np.int32))
    for j in range(p.k):
        h = _coordinate_objective(orc, w, j)
        d = orc.improve(w, z, j, d0[j], 500)
        span = 10 * abs(d0[j]) + 5.0
        ref = minimize_scalar(h, bounds=(-w[j] - span, -w[j] + span), method="bounded",
                              options={"xatol": 1e-12, "maxiter": 2000})
        assert h(d) <= h(d0[j]) + 1e-15 <= h(0.0) + 2e-15  # never worse than the plain step
        assert h(d) <= ref.fun + 1e-13
        assert d == pytest.approx(ref.x, abs=1e-5)


def test_thread_greedy_applies_the_improved_increments_from_the_start_state():
    # Jacobi (R5): every accepted increment is improved at the start state,
    # then all are applied
    p = workloads.uniform_problem(300, 120, 8, values="lognormal", loss="logistic", seed=6)
    orc = oracle.Oracle(p)
    orc.set_lambda(0.05 * orc.lambda_max())
    w0 = np.random.default_rng(6).normal(0, 0.3, p.k) * (np.random.default_rng(7).random(p.k) < 0.3)
    z0 = orc.fitted(w0)
    w_plain, _, _, _ = orc.run("thread_greedy", 1, w=w0, B=8)
    w_imp, z_imp, _, _ = orc.run("thread_greedy", 1, w=w0, B=8, improve_steps=500)
    moved = np.flatnonzero(w_plain != w0)
    np.testing.assert_array_equal(np.flatnonzero(w_imp != w0), moved)
    for j in moved:
        d = orc.improve(w0, z0, j, w_plain[j] - w0[j], 500)
        assert w_imp[j] - w0[j] == pytest.approx(d, rel=1e-12, abs=1e-15)
    np.testing.assert_allclose(z_imp, orc.fitted(w_imp), rtol=0, atol=1e-12)


def test_cyclic_cd_with_improve_reaches_the_same_optimum():
    p = workloads.config1("logistic")
    orc = oracle.Oracle(p)
    orc.set_lambda(0.05 * orc.lambda_max())
    w_a, _, it_a, kkt_a, _ = orc.solve("ccd", tol_kkt=1e-10)
    w_b, _, it_b, kkt_b, _ = orc.solve("ccd", tol_kkt=1e-10, improve_steps=500)
    assert kkt_a <= 1e-10 and kkt_b <= 1e-10
    assert orc.objective(w_b) == pytest.approx(orc.objective(w_a), rel=1e-10)
    assert it_b <= it_a  # exact coordinate minimisation needs no more sweeps


# --- R12: Thread-Greedy with a global top-|J'| Accept (Section 7) ----------

def test_top_greedy_with_one_accept_is_greedy():
    p = workloads.uniform_problem(200, 80, 6, values="lognormal", loss="logistic", seed=12)
    orc = oracle.Oracle(p)
    orc.set_lambda(0.05 * orc.lambda_max())
    w_a, _, _, _ = orc.run("greedy", 25)
    w_b, _, _, _ = orc.run("top_greedy", 25, B=1)
    np.testing.assert_array_equal(w_a, w_b)


@pytest.mark.parametrize("B", [3, 17, 10_000])
def test_top_greedy_accepts_the_lowest_proxies(B):
    p = workloads.uniform_problem(300, 150, 8, values="pm1", loss="squared", seed=13)
    orc = oracle.Oracle(p)
    orc.set_lambda(0.05 * orc.lambda_max())
    w0 = np.random.default_rng(13).normal(0, 0.2, p.k) * (np.random.default_rng(14).random(p.k) < 0.2)
    z0 = orc.fitted(w0)
    d, f = orc.propose(w0, z0, np.arange(p.k, dtype=np.int32))
    neg = np.flatnonzero(f < 0)
    order = neg[np.lexsort((neg, f[neg]))]  # proxy ascending, then column
    want = np.sort(order[:B])
    w1, _, _, st = orc.run("top_greedy", 1, w=w0, B=B)
    np.testing.assert_array_equal(np.flatnonzero(w1 != w0), want)
    np.testing.assert_allclose(w1[want] - w0[want], d[want], rtol=1e-13, atol=0)
    assert st[0] == want.size


# --- R13: balanced colouring (Section 7) -------------------------------------

def _csc(cols, n):
    """CSC problem from per-column row lists (values 1)."""
    X = np.zeros((n, len(cols)))
    for j, rows in enumerate(cols):
        X[rows, j] = 1.0
    return workloads.csc_from_dense(X, np.ones(n), "squared")


def _valid_distance2(p, colors):
    rows_of = [set(p.row_idx[p.col_ptr[j]:p.col_ptr[j + 1]]) for j in range(p.k)]
    for a in range(p.k):
        for b in range(a + 1, p.k):
            if rows_of[a] & rows_of[b] and colors[a] == colors[b]:
                return False
    return True


def test_balanced_colouring_hand_examples():
    # six columns in separate rows: first-fit needs one colour; the default
    # cap ceil(6/1) keeps them together, a cap of 2 deals them out in order
    free = _csc([[0], [1], [2], [3], [4], [5]], 6)
    o = oracle.Oracle(free)
    assert o.color()[1] == 1
    np.testing.assert_array_equal(o.color_balanced()[0], [0] * 6)
    np.testing.assert_array_equal(o.color_balanced(cap=2)[0], [0, 0, 1, 1, 2, 2])
    # columns 0-2 share row 0, columns 3-5 are free: first-fit gives class
    # sizes 4, 1, 1; the balanced rule (cap ceil(6/3) = 2) gives 2, 2, 2
    tri = _csc([[0, 1], [0, 2], [0, 3], [4], [5], [6]], 7)
    o = oracle.Oracle(tri)
    ff, c0 = o.color()
    np.testing.assert_array_equal(ff, [0, 1, 2, 0, 0, 0])
    bal, c1 = o.color_balanced()
    np.testing.assert_array_equal(bal, [0, 1, 2, 0, 1, 2])
    assert c0 == c1 == 3


def test_balanced_colouring_is_valid_capped_and_flatter():
    p = workloads.zipf_problem(400, 600, 6000, cap=80, n_planted=10, seed=8)
    o = oracle.Oracle(p)
    ff, c0 = o.color()
    bal, c1 = o.color_balanced()
    cap = -(-p.k // c0)
    assert _valid_distance2(p, bal)
    sizes_ff = np.bincount(ff, minlength=c0)
    sizes = np.bincount(bal, minlength=c1)
    assert sizes.max() <= cap and c1 >= c0
    assert sizes.max() < sizes_ff.max() and sizes.std() < sizes_ff.std()


def test_coloring_with_balanced_colours_reaches_the_optimum():
    p = workloads.config1("squared")
    o = oracle.Oracle(p)
    o.set_lambda(0.05 * o.lambda_max())
    bal, _ = o.color_balanced()
    w_ref, _, _, _, _ = o.solve("ccd", tol_kkt=1e-11)
    w, _, _, kkt, _ = o.solve("coloring", tol_kkt=1e-10, colors=bal, seed=3, max_iter=10**6)
    assert kkt <= 1e-10
    assert o.objective(w) == pytest.approx(o.objective(w_ref), rel=1e-9)


# --- R14: block Shotgun, a P*_b per column block (Section 7) ----------------

def test_block_shotgun_with_one_block_is_shotgun_at_pstar():
    p = workloads.uniform_problem(200, 120, 5, values="lognormal", loss="logistic", seed=15)
    o = oracle.Oracle(p)
    o.set_lambda(0.05 * o.lambda_max())
    rho, _ = o.spectral_radius(max_iter=1000, rel_tol=1e-12)
    pstar = oracle.pstar(p.k, rho)
    Pb = o.block_pstar(1, max_iter=1000, rel_tol=1e-12)
    assert list(Pb) == [pstar]
    w_a, _, _, _ = o.run("shotgun", 30, P=pstar, seed=5)
    w_b, _, _, _ = o.run("shotgun_blocks", 30, B=1, block_P=Pb, seed=5)
    np.testing.assert_array_equal(w_a, w_b)


def test_block_pstar_is_each_blocks_own_bound():
    p = workloads.uniform_problem(60, 45, 6, values="pm1", loss="squared", seed=16)
    o = oracle.Oracle(p)
    B = 4
    Pb = o.block_pstar(B, max_iter=5000, rel_tol=1e-14)
    X = p.to_dense()
    for b in range(B):
        lo, hi = p.k * b // B, p.k * (b + 1) // B
        Xb = X[:, lo:hi]
        nb = np.sqrt((Xb * Xb).sum(0))
        M = (Xb / nb).T @ (Xb / nb)
        rho = np.linalg.eigvalsh(M)[-1]
        assert Pb[b] == max(1, int(np.floor((hi - lo) / (2 * rho))))
    # one iteration takes P*_b columns from every block and accepts them all
    o.set_lambda(0.01 * o.lambda_max())
    _, _, _, st = o.run("shotgun_blocks", 1, B=B, block_P=Pb, seed=2)
    assert st[0] == int(np.minimum(Pb, [p.k * (b + 1) // B - p.k * b // B for b in range(B)]).sum())


def test_block_shotgun_converges_on_orthogonal_blocks():
    # block-diagonal X: the blocks are independent problems that share the loss
    rng = np.random.default_rng(17)
    n, kb, B = 240, 40, 3
    X = np.zeros((n, kb * B))
    for b in range(B):
        rows = slice(b * n // B, (b + 1) * n // B)
        Xb = rng.normal(size=(n // B, kb)) * (rng.random((n // B, kb)) < 0.2)
        X[rows, b * kb:(b + 1) * kb] = Xb
    y = X @ (rng.normal(size=kb * B) * (rng.random(kb * B) < 0.1)) + 0.01 * rng.normal(size=n)
    p = workloads.csc_from_dense(X, y, "squared")
    o = oracle.Oracle(p)
    o.set_lambda(0.05 * o.lambda_max())
    Pb = o.block_pstar(B)
    w_ref, _, _, _, _ = o.solve("ccd", tol_kkt=1e-11)
    w, _, _, kkt, _ = o.solve("shotgun_blocks", tol_kkt=1e-10, B=B, block_P=Pb, seed=1, max_iter=10**6)
    assert kkt <= 1e-10
    assert o.objective(w) == pytest.approx(o.objective(w_ref), rel=1e-9)


# --- the duality gap: a certificate of P(w) - P* (the paper has no stopping rule) ----

def _golden_max(f, lo, hi, iters=300):
    """Maximiser of a concave function on [lo, hi] by golden-section search."""
    r = (np.sqrt(5.0) - 1.0) / 2.0
    a, b = lo, hi
    c, d = b - r * (b - a), a + r * (b - a)
    fc, fd = f(c), f(d)
    for _ in range(iters):
        if fc > fd:
            b, d, fd = d, c, fc
            c = b - r * (b - a)
            fc = f(c)
        else:
            a, c, fc = c, d, fd
            d = a + r * (b - a)
            fd = f(d)
    return 0.5 * (a + b)


@pytest.mark.parametrize("loss", ["squared", "logistic"])
def test_conjugate_is_the_sup_over_t(loss):
    # l*(y, v) = sup_t (v t - l(y, t)): the supremum found by search on the
    # concave function of t, for labels and dual values across the domain
    rng = np.random.default_rng(3)
    for _ in range(300):
        if loss == "logistic":
            y = float(rng.choice([-1.0, 1.0]))
            v = -y * float(rng.uniform(1e-3, 1.0 - 1e-3))
        else:
            y, v = float(rng.normal(0, 2)), float(rng.normal(0, 2))
        f = lambda t: v * t - oracle.loss(loss, y, t)
        t_star = _golden_max(f, -60.0, 60.0)
        assert oracle.conjugate(loss, y, v) == pytest.approx(f(t_star), abs=1e-12)
    if loss == "logistic":  # the ends of the domain, and outside it
        assert oracle.conjugate(loss, 1.0, 0.0) == 0.0 and oracle.conjugate(loss, 1.0, -1.0) == 0.0
        assert oracle.conjugate(loss, 1.0, 0.5) == float("inf")
        assert oracle.conjugate(loss, -1.0, -0.1) == float("inf")


@pytest.mark.parametrize("loss", ["squared", "logistic"])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_duality_gap_bounds_the_suboptimality(loss, seed):
    # weak duality: gap(w) >= P(w) - P* for every w, with P* from brute force;
    # and the gap closes at the optimum
    p = workloads.tiny_problem(8, 4, loss=loss, seed=seed)
    X = p.to_dense()
    o = oracle.Oracle(p)
    lam = 0.2 * o.lambda_max()
    o.set_lambda(lam)
    Pbf, wbf = _brute_force(X, p.y, loss, lam)
    rng = np.random.default_rng(seed + 10)
    gaps = []
    for scale in (1e-4, 1e-2, 0.3, 3.0):
        for _ in range(25):
            w = wbf + rng.normal(0, scale, 4) * (rng.random(4) < 0.7)
            gap = o.duality_gap(w)
            sub = _dense_objective(X, p.y, loss, lam, w) - Pbf
            assert gap >= sub - 1e-13, (gap, sub)
            gaps.append(gap)
    assert min(gaps) >= -1e-13
    w, _, _, kkt, _ = o.solve("ccd", tol_kkt=1e-13, max_iter=10**7)
    assert o.duality_gap(w) <= 1e-12


@pytest.mark.parametrize("loss", ["squared", "logistic"])
def test_duality_gap_closes_along_cyclic_cd(loss):
    # a sparse problem with k > n: the gap is non-negative along the solve and
    # shrinks with the KKT violation
    p = workloads.uniform_problem(200, 300, 6, values="lognormal", loss=loss, n_planted=10, seed=4)
    o = oracle.Oracle(p)
    o.set_lambda(0.1 * o.lambda_max())
    last = np.inf
    for tol in (1e-3, 1e-6, 1e-9, 1e-12):
        w, _, _, kkt, _ = o.solve("ccd", tol_kkt=tol, max_iter=10**8)
        gap = o.duality_gap(w)
        assert 0.0 <= gap <= last + 1e-15
        last = gap
    # at KKT violation eps the dual scaling moves D by about eps ||w||_1
    assert last <= 4e-12 * (1.0 + np.abs(w).sum())
