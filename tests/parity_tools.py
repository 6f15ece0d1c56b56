"""Tolerances and helpers shared by the GPU parity tests.

Step and proxy tolerance (the condition of the sum g_j = (1/n) sum_i X_ij u_i):
with S_j = (1/n) sum_i |X_ij u_i| and sd_j = |delta_j| + S_j/beta_j,
  |delta_gpu - delta_cpu| <= tol * sd_j,
  |phi_gpu - phi_cpu|     <= tol * sd_j * (S_j + beta_j sd_j + lambda),
tol = 1e-12 in FP64 mode and 1e-5 in FP32 arithmetic.
"""

import numpy as np

TOL = {"f64": 1e-12, "f32": 1e-5}


def _u(prob, z):
    if prob.loss == "squared":
        return z - prob.y
    return -prob.y / (1.0 + np.exp(prob.y * z))


def _scales(prob, z, lam, beta_mode=0):
    u = _u(prob, z)
    counts = np.diff(prob.col_ptr)
    a = np.abs(prob.val * u[prob.row_idx])
    S = np.zeros(prob.k)
    nz = counts > 0
    S[nz] = np.add.reduceat(a, prob.col_ptr[:-1][nz]) / prob.n
    beta = 1.0 if prob.loss == "squared" else 0.25
    c = np.zeros(prob.k)
    c[nz] = np.add.reduceat(prob.val ** 2, prob.col_ptr[:-1][nz]) / prob.n
    bj = np.full(prob.k, beta) if beta_mode else beta * c
    return S, bj


def assert_steps_close(prob, z, w, lam, J, d_gpu, f_gpu, d_cpu, f_cpu, tol, beta_mode=0):
    S, bj = _scales(prob, z, lam, beta_mode)
    S, bj, wj = S[J], bj[J], w[J]
    sd = np.abs(d_cpu) + np.where(bj > 0, S / np.where(bj > 0, bj, 1.0), np.abs(wj))
    td = tol * sd + 1e-300
    tf = tol * sd * (S + bj * sd + lam) + 1e-300
    bad = np.flatnonzero(np.abs(d_gpu - d_cpu) > td)
    assert bad.size == 0, (bad[:5], d_gpu[bad[:5]], d_cpu[bad[:5]], td[bad[:5]])
    bad = np.flatnonzero(np.abs(f_gpu - f_cpu) > tf)
    assert bad.size == 0, (bad[:5], f_gpu[bad[:5]], f_cpu[bad[:5]], tf[bad[:5]])


def _state(prob, seed, frac=0.1, scale=0.5):
    rng = np.random.default_rng(seed)
    return np.where(rng.random(prob.k) < frac, rng.normal(0, scale, prob.k), 0.0)


# --- support comparison (the "support identical above 1e-6" criterion) ----------
#
# Two points that both satisfy the KKT conditions to within eps can differ in
# support only where the optimum itself is within eps of changing it.  To first
# order, a KKT violation e (|e_j| <= eps) moves the active coefficients S of the
# optimum by dw_S = -H_S^-1 e_S, with H_S = X_S^T D X_S / n and D = l''(y, z*),
# and the gradient of an inactive coordinate j by e_j - (X_j^T D X_S / n) dw_S.
# So an active coefficient can cross the threshold only if
#   | |w*_j| - thresh | <= eps * ||row_j(H_S^-1)||_1,
# and an inactive one can become active only if its slack
#   lambda - |g*_j| <= eps * (1 + ||(X_j^T D X_S / n) H_S^-1||_1).
# Those columns are "fragile at eps"; every other column must have the same
# membership in {|w_j| > thresh} on both sides.

def _csc_matrix(prob):
    import scipy.sparse as sp

    return sp.csc_matrix((prob.val, prob.row_idx, prob.col_ptr), shape=(prob.n, prob.k))


def fragile_columns(prob, lam, w_ref, eps, thresh=1e-6, max_active=6000):
    """Boolean mask of the columns whose support membership is not determined
    at KKT accuracy eps around the optimum w_ref (first-order sensitivity)."""
    X = _csc_matrix(prob)
    n = prob.n
    z = X @ w_ref
    if prob.loss == "squared":
        u, d2 = z - prob.y, np.ones(n)
    else:
        u = -prob.y / (1.0 + np.exp(prob.y * z))
        s = 1.0 / (1.0 + np.exp(-prob.y * z))
        d2 = s * (1.0 - s)
    g = (X.T @ u) / n
    S = np.flatnonzero(w_ref != 0.0)
    I = np.flatnonzero(w_ref == 0.0)
    assert S.size <= max_active, "support too large for the dense sensitivity analysis"
    fr = np.zeros(prob.k, bool)
    if S.size:
        XS = X[:, S].toarray()
        H = (XS.T * d2) @ XS / n
        Hi = np.linalg.pinv(H)
        a = np.abs(Hi).sum(axis=1)
        fr[S] = np.abs(np.abs(w_ref[S]) - thresh) <= eps * a
        XI = X[:, I]
        M = (XI.T @ (XS * d2[:, None])) / n @ Hi
        b = 1.0 + np.abs(M).sum(axis=1)
    else:
        b = np.ones(I.size)
    fr[I] = lam - np.abs(g[I]) <= eps * b
    return fr


def assert_support_matches(prob, lam, w, w_ref, thresh=1e-6, label="", max_eps=1e-7, eps=None):
    """{|w_j| > thresh} equals {|w_ref_j| > thresh} on every column that is not
    fragile at eps = the larger oracle (FP64) KKT violation of the two points,
    which must not exceed max_eps (far from the optimum nothing is
    determined).  `eps` overrides the measured accuracy.  Returns (eps,
    fragile count, differing count)."""
    import oracle

    orc = oracle.Oracle(prob, lam)
    if eps is None:
        eps = max(orc.kkt(w), orc.kkt(w_ref))
        assert eps <= max_eps, f"{label}: KKT violation {eps:.2e} above {max_eps:.1e}: supports are not comparable"
    fr = fragile_columns(prob, lam, w_ref, eps, thresh)
    sw, sr = np.abs(w) > thresh, np.abs(w_ref) > thresh
    bad = np.flatnonzero((sw != sr) & ~fr)
    if bad.size:
        g = orc.gradient(orc.fitted(w_ref))
        detail = [(int(j), float(w[j]), float(w_ref[j]), float(abs(g[j]) - lam)) for j in bad[:8]]
        raise AssertionError(f"{label}: support differs outside the fragile set at eps={eps:.2e}: "
                             f"(j, w_j, w*_j, |g*_j|-lambda) = {detail}")
    return eps, int(fr.sum()), int((sw != sr).sum())


# --- stored optima (tests/golden/optimum_*.txt, written by tests/golden/make_optima.py)

def load_optimum(name):
    """(w, lambda, meta) of a stored oracle optimum; meta holds the header
    fields (problem sha256, lambda/lambda_max, KKT at writing)."""
    import os

    path = os.path.join(os.path.dirname(__file__), "golden", f"optimum_{name}.txt")
    meta, idx, val = {}, [], []
    with open(path) as f:
        for line in f:
            if line.startswith("#"):
                continue
            parts = line.split()
            if parts[0] == "meta":
                meta[parts[1]] = parts[2]
            else:
                idx.append(int(parts[0]))
                val.append(float(parts[1]))
    w = np.zeros(int(meta["k"]))
    w[np.array(idx, np.int64)] = val
    return w, float(meta["lambda"]), meta


def certified_optimum(name, prob, lam, tol=3e-11):
    """The stored optimum of `name` for (prob, lam), re-certified on `prob` as
    generated here: the stored lambda must equal `lam` to 1e-12 (relative)
    and the oracle's FP64 KKT violation at the stored w must be <= tol; else
    the optimum is recomputed by cyclic CD (slow)."""
    import oracle

    orc = oracle.Oracle(prob, lam)
    try:
        w, lam_stored, _ = load_optimum(name)
        if abs(lam - lam_stored) <= 1e-12 * lam and w.size == prob.k and orc.kkt(w) <= tol:
            return w
    except (OSError, KeyError, ValueError):
        pass
    w, _, _, _, _ = orc.solve("ccd", tol_kkt=1e-11, max_iter=4 * 10**8)
    return w
