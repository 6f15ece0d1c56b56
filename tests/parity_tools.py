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
