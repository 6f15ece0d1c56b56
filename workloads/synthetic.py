"""Seeded generators for sparse l1 problems shaped like the paper's workloads.

The paper measures on DOROTHEA (binary, 800 x 100,000, 7.3 nnz/column) and
REUTERS RCV1-v2 (tf-idf, 23,865 x 47,237, 37.2 nnz/column), both with columns
normalised (Section 4.4, Table 3).  Neither data set is available here, so these
generators draw stand-ins with the same structure: sparse column-major X,
binary/+-1 or log-normal values, unit-norm columns, k >> n, a planted sparse
model and noisy labels.

Every generator uses ``numpy.random.Generator(PCG64(seed))`` and a fixed draw
order (documented per function), so the same seed gives the same bytes on any
machine.  Nothing here evaluates the objective, its gradient or a step of the
method.

CSC layout: ``col_ptr`` int64[k+1], ``row_idx`` int32[nnz] (sorted, distinct
within a column), ``val`` float64[nnz]; labels ``y`` float64[n].
"""

from __future__ import annotations

import dataclasses
import hashlib
import os

import numpy as np

SQUARED = "squared"
LOGISTIC = "logistic"


@dataclasses.dataclass
class Problem:
    n: int
    k: int
    col_ptr: np.ndarray
    row_idx: np.ndarray
    val: np.ndarray
    y: np.ndarray
    loss: str
    w_star: np.ndarray
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.col_ptr[-1])

    def col_nnz(self) -> np.ndarray:
        return np.diff(self.col_ptr)

    def sha256(self) -> str:
        h = hashlib.sha256()
        for a in (self.col_ptr, self.row_idx, self.val, self.y):
            h.update(np.ascontiguousarray(a).tobytes())
        return h.hexdigest()

    def to_dense(self) -> np.ndarray:
        X = np.zeros((self.n, self.k))
        for j in range(self.k):
            s, e = self.col_ptr[j], self.col_ptr[j + 1]
            X[self.row_idx[s:e], j] = self.val[s:e]
        return X

    def with_loss(self, loss: str, y: np.ndarray) -> "Problem":
        return dataclasses.replace(self, loss=loss, y=np.ascontiguousarray(y, np.float64))


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _distinct_rows(n: int, counts: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    """Rows for each column, uniform without replacement, sorted per column.

    Draws with replacement, then redraws the duplicates until every column's
    rows are distinct (the result is a uniform draw without replacement).
    Returns the concatenated int32 row indices in column order.
    """
    counts = np.asarray(counts, np.int64)
    if counts.size and counts.max() > n:
        raise ValueError("a column cannot hold more than n distinct rows")
    k = counts.size
    col = np.repeat(np.arange(k, dtype=np.int64), counts)
    key = col * n + rng.integers(0, n, size=col.size, dtype=np.int64)
    key.sort()
    while True:
        dup = np.flatnonzero(key[1:] == key[:-1]) + 1
        if dup.size == 0:
            break
        c = key[dup] // n
        key[dup] = c * n + rng.integers(0, n, size=dup.size, dtype=np.int64)
        key.sort()
    return (key - col * n).astype(np.int32)


def _row_set_hash(col_ptr: np.ndarray, row_idx: np.ndarray) -> np.ndarray:
    """A 64-bit fingerprint of each column's row set (equal sets, equal
    fingerprints), from a SplitMix64-style mix of every row summed per column."""
    with np.errstate(over="ignore"):
        x = row_idx.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15)
        x = (x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        x = (x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        x = x ^ (x >> np.uint64(31))
    counts = np.diff(col_ptr)
    h = np.zeros(counts.size, np.uint64)
    nz = counts > 0
    if nz.any():
        h[nz] = np.add.reduceat(x, col_ptr[:-1][nz])
    return h


def _duplicate_columns(n: int, col_ptr: np.ndarray, row_idx: np.ndarray) -> np.ndarray:
    """Columns whose row set equals that of a lower-index column (ascending)."""
    counts = np.diff(col_ptr)
    h = _row_set_hash(col_ptr, row_idx)
    order = np.lexsort((np.arange(counts.size), h, counts))
    key_c, key_h = counts[order], h[order]
    starts = np.flatnonzero(np.r_[True, (key_c[1:] != key_c[:-1]) | (key_h[1:] != key_h[:-1])])
    ends = np.r_[starts[1:], order.size]
    dups = []
    for a, b in zip(starts[ends - starts > 1], ends[ends - starts > 1]):
        group = order[a:b]  # equal fingerprints, ascending column index
        rows = [row_idx[col_ptr[j]:col_ptr[j + 1]] for j in group]
        for q in range(1, len(group)):
            if any(np.array_equal(rows[q], rows[r]) for r in range(q)):
                dups.append(group[q])
    return np.sort(np.asarray(dups, np.int64))


def _distinct_columns(n: int, counts: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    """Rows of every column as _distinct_rows draws them, then the rows of each
    column whose row set repeats a lower-index column's are drawn again, until
    no two columns share a row set.  Duplicate columns would make the l1
    minimiser non-unique (weight can move freely between them), so the
    generators never produce them.  When no column repeats, no extra draw is
    made: the arrays are those of _distinct_rows."""
    counts = np.asarray(counts, np.int64)
    col_ptr = _col_ptr(counts)
    row_idx = _distinct_rows(n, counts, rng)
    for _ in range(1000):
        dup = _duplicate_columns(n, col_ptr, row_idx)
        if dup.size == 0:
            return row_idx
        fresh = _distinct_rows(n, counts[dup], rng)
        fp = _col_ptr(counts[dup])
        for q, j in enumerate(dup):
            row_idx[col_ptr[j]:col_ptr[j + 1]] = fresh[fp[q]:fp[q + 1]]
    raise ValueError("cannot draw columns with distinct row sets (too many short columns for n rows)")


def _col_ptr(counts: np.ndarray) -> np.ndarray:
    cp = np.zeros(len(counts) + 1, np.int64)
    np.cumsum(counts, out=cp[1:])
    return cp


def _matvec(col_ptr, row_idx, val, n, w) -> np.ndarray:
    """X @ w for the planted model (label generation only)."""
    counts = np.diff(col_ptr)
    contrib = val * np.repeat(w, counts)
    return np.bincount(row_idx, weights=contrib, minlength=n).astype(np.float64)


def _labels(loss: str, t: np.ndarray, noise_sd: float, rng: np.random.Generator) -> np.ndarray:
    eps = rng.normal(0.0, noise_sd, size=t.size)
    if loss == LOGISTIC:
        return np.where(t + eps >= 0.0, 1.0, -1.0)  # sign(0) = +1
    return t + eps


def _normalise_columns(col_ptr, val) -> np.ndarray:
    counts = np.diff(col_ptr)
    nz = counts > 0
    ss = np.zeros(counts.size)
    ss[nz] = np.add.reduceat(val * val, col_ptr[:-1][nz])
    scale = np.where(ss > 0, 1.0 / np.sqrt(np.where(ss > 0, ss, 1.0)), 0.0)
    return val * np.repeat(scale, counts)


def uniform_problem(n, k, nnz_per_col, *, values="pm1", n_planted=50, loss=LOGISTIC,
                    noise_sd=None, seed=0, name="") -> Problem:
    """Every column holds ``nnz_per_col`` distinct rows drawn uniformly.

    Draw order: rows (with redraws of repeated row sets, see
    _distinct_columns), values, planted support, planted weights, label noise.
    ``values``: "pm1" (+-1 at p=1/2), "ones" (binary, DOROTHEA-like) or
    "lognormal" (LogNormal(0,1) then unit-norm columns, tf-idf-like).
    """
    rng = _rng(seed)
    counts = np.full(k, nnz_per_col, np.int64)
    col_ptr = _col_ptr(counts)
    row_idx = _distinct_columns(n, counts, rng)
    nnz = int(col_ptr[-1])
    if values == "pm1":
        val = np.where(rng.random(nnz) < 0.5, -1.0, 1.0)
    elif values == "ones":
        val = np.ones(nnz)
    elif values == "lognormal":
        val = _normalise_columns(col_ptr, rng.lognormal(0.0, 1.0, nnz))
    else:
        raise ValueError(values)
    w_star = np.zeros(k)
    support = rng.choice(k, size=min(n_planted, k), replace=False)
    w_star[support] = rng.normal(0.0, 1.0, support.size)
    t = _matvec(col_ptr, row_idx, val, n, w_star)
    if noise_sd is None:
        noise_sd = 0.1 if loss == LOGISTIC else 0.01
    y = _labels(loss, t, noise_sd, rng)
    return Problem(n, k, col_ptr, row_idx, val.astype(np.float64), y, loss, w_star, name)


def config1(loss=LOGISTIC, seed=0) -> Problem:
    """n=2,000, k=5,000, 20 nnz/column at uniform rows, values +-1; 50 planted
    N(0,1) weights; logistic y = sign(Xw*+N(0,0.1^2)), Lasso y = Xw*+N(0,0.01^2)."""
    return uniform_problem(2000, 5000, 20, values="pm1", n_planted=50, loss=loss,
                           seed=seed, name=f"uniform-2000x5000-20nnz-pm1-{loss}")


def zipf_counts(k, nnz_total, s=1.1, cap=50_000, n=None) -> np.ndarray:
    """Column nnz by rank r: clamp(round(C r^-s), 1, cap), with C found by
    bisection so that the total is nnz_total (to 0.5%)."""
    cap = min(cap, n) if n is not None else cap
    r = np.arange(1, k + 1, dtype=np.float64) ** (-s)

    def total(C):
        return np.clip(np.rint(C * r), 1, cap).sum()

    lo, hi = 0.0, float(nnz_total) * 10.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if total(mid) < nnz_total:
            lo = mid
        else:
            hi = mid
    counts = np.clip(np.rint(hi * r), 1, cap).astype(np.int64)
    if abs(counts.sum() - nnz_total) > 0.005 * nnz_total:
        raise ValueError("cannot meet the nnz target with this cap")
    return counts


def zipf_problem(n, k, nnz_total, *, s=1.1, cap=50_000, n_planted=2000, loss=LOGISTIC,
                 seed=0, name="") -> Problem:
    """Zipf(s) column lengths assigned to columns by a seeded permutation, rows
    uniform without replacement, LogNormal(0,1) values, unit-norm columns.

    Draw order: rank-to-column permutation, rows (with redraws of repeated
    row sets, see _distinct_columns), values, planted support,
    planted weights, label noise.  Labels: y = sign(Xw* + eps) with
    eps ~ N(0, (0.1 rms(Xw*))^2) (logistic), y = Xw* + eps (squared).
    """
    rng = _rng(seed)
    by_rank = zipf_counts(k, nnz_total, s=s, cap=cap, n=n)
    perm = rng.permutation(k)
    counts = np.empty(k, np.int64)
    counts[perm] = by_rank
    col_ptr = _col_ptr(counts)
    row_idx = _distinct_columns(n, counts, rng)
    val = _normalise_columns(col_ptr, rng.lognormal(0.0, 1.0, int(col_ptr[-1])))
    w_star = np.zeros(k)
    support = rng.choice(k, size=min(n_planted, k), replace=False)
    w_star[support] = rng.normal(0.0, 1.0, support.size)
    t = _matvec(col_ptr, row_idx, val, n, w_star)
    rms = float(np.sqrt(np.mean(t * t))) if n else 0.0
    y = _labels(loss, t, 0.1 * rms if rms > 0 else 0.1, rng)
    return Problem(n, k, col_ptr, row_idx, val, y, loss, w_star, name)


def config2(loss=LOGISTIC, seed=0, cache_dir=None) -> Problem:
    """n=1,000,000, k=4,000,000, Zipf(1.1) column nnz capped at 50,000,
    2.00e8 nnz, log-normal unit-norm columns, 2,000 planted weights.

    ``cache_dir`` (default: $GENCD_WORKLOAD_CACHE) keeps the drawn arrays as
    .npy files so that several processes of one session draw them once."""
    name = f"zipf1.1-1Mx4M-200Mnnz-{loss}-seed{seed}"
    cache_dir = cache_dir or os.environ.get("GENCD_WORKLOAD_CACHE")
    if cache_dir:
        base = os.path.join(cache_dir, name)
        files = [base + f".{a}.npy" for a in ("col_ptr", "row_idx", "val", "y", "w_star")]
        if all(os.path.exists(f) for f in files):
            a = [np.load(f, mmap_mode=None) for f in files]
            return Problem(1_000_000, 4_000_000, a[0], a[1], a[2], a[3], loss, a[4], name)
    p = zipf_problem(1_000_000, 4_000_000, 200_000_000, cap=50_000, n_planted=2000,
                     loss=loss, seed=seed, name=name)
    if cache_dir:
        os.makedirs(cache_dir, exist_ok=True)
        for a, f in zip((p.col_ptr, p.row_idx, p.val, p.y, p.w_star), files):
            np.save(f + ".tmp.npy", a)
            os.replace(f + ".tmp.npy", f)
    return p


def config3(values="lognormal", loss=LOGISTIC, seed=0) -> Problem:
    """config1's shapes (n=2,000, k=5,000, 20 nnz/column at uniform rows) with
    one of three value laws: "pm1" (exact in bfloat16), "ones" (binary) or
    "lognormal" (LogNormal(0,1), unit-norm columns: bfloat16 rounds them)."""
    return uniform_problem(2000, 5000, 20, values=values, n_planted=50, loss=loss, seed=seed,
                           name=f"uniform-2000x5000-20nnz-{values}-{loss}")


def binarized(prob: Problem) -> Problem:
    """The same sparsity pattern and labels with binary, unit-norm columns:
    every non-zero of column j becomes 1/sqrt(nnz_j) (no random draws)."""
    counts = prob.col_nnz()
    s = 1.0 / np.sqrt(np.maximum(counts, 1).astype(np.float64))
    return dataclasses.replace(prob, val=np.repeat(s, counts), name=prob.name + "-binary")


def config2_scaled(scale=0.02, loss=LOGISTIC, seed=0) -> Problem:
    """config2's structure at a fraction of its size (rows, columns, nnz and the
    column cap all scaled), for tests that must run in seconds."""
    n = max(1000, int(1_000_000 * scale))
    k = max(1000, int(4_000_000 * scale))
    nnz = int(200_000_000 * scale)
    cap = max(50, int(50_000 * scale))
    return zipf_problem(n, k, nnz, cap=cap, n_planted=max(10, int(2000 * scale)), loss=loss,
                        seed=seed, name=f"zipf1.1-{n}x{k}-{nnz}nnz-{loss}")


def config4(loss=SQUARED, seed=0, scale=1.0) -> Problem:
    """The regularisation-path workload: n=200,000, k=500,000, Zipf(1.1)
    column lengths capped at 10,000 (4.0e7 nnz), LogNormal(0,1) values with
    unit-norm columns, 1,000 planted weights (zipf_problem's law).  ``scale``
    shrinks rows, columns, nnz and the cap together, for tests."""
    n = max(1000, int(200_000 * scale))
    k = max(1000, int(500_000 * scale))
    nnz = int(40_000_000 * scale)
    cap = max(50, int(10_000 * scale))
    return zipf_problem(n, k, nnz, cap=cap, n_planted=max(10, int(1000 * scale)), loss=loss, seed=seed,
                        name=f"zipf1.1-{n}x{k}-{nnz}nnz-{loss}")


def cv_folds(n, nfolds=5, seed=0) -> np.ndarray:
    """Row folds for cross-validation: a seeded permutation of the rows dealt
    round-robin, so fold sizes differ by at most one (uint8[n])."""
    perm = _rng(seed).permutation(n)
    fold = np.empty(n, np.uint8)
    fold[perm] = (np.arange(n) % nfolds).astype(np.uint8)
    return fold


def lambda_grid(lam_max, nlambda=32, ratio=1e-3) -> np.ndarray:
    """nlambda values log-spaced from lam_max down to ratio * lam_max."""
    return lam_max * np.logspace(0.0, np.log10(ratio), nlambda)


def row_subset(prob: Problem, rows) -> Problem:
    """The problem restricted to the given rows (renumbered in increasing
    order), the same columns: the training problem of a cross-validation
    fold."""
    rows = np.sort(np.asarray(rows, np.int64))
    new_id = np.full(prob.n, -1, np.int64)
    new_id[rows] = np.arange(rows.size)
    keep = new_id[prob.row_idx] >= 0
    col_of = np.repeat(np.arange(prob.k), np.diff(prob.col_ptr))
    counts = np.bincount(col_of[keep], minlength=prob.k).astype(np.int64)
    return Problem(int(rows.size), prob.k, _col_ptr(counts), new_id[prob.row_idx[keep]].astype(np.int32),
                   prob.val[keep].copy(), prob.y[rows].copy(), prob.loss, prob.w_star, prob.name + "-rows")


def serving_stream(nreq, rate=200.0, seed=0, n_range=(1_000, 200_000), k_range=(1_000, 1_000_000),
                   nnz_range=(5, 100)):
    """Independent requests arriving as a Poisson process of ``rate`` per
    second: n and k log-uniform over their ranges, a column length uniform in
    ``nnz_range`` (at most n), squared or logistic loss with probability 1/2,
    lambda / lambda_max uniform in [0.01, 0.3]; each X from uniform_problem
    with log-normal unit-norm columns and min(50, k) planted weights.

    Draw order: inter-arrival gaps, then per request n, k, column length,
    loss, lambda fraction and the request's own seed.  Returns (problems,
    lambda_fracs, arrivals in seconds from the first arrival)."""
    rng = _rng(seed)
    gaps = rng.exponential(1.0 / rate, nreq)
    arrivals = np.cumsum(gaps) - gaps[0] if nreq else np.zeros(0)
    problems, fracs = [], []
    for _ in range(nreq):
        n = int(round(np.exp(rng.uniform(np.log(n_range[0]), np.log(n_range[1])))))
        k = int(round(np.exp(rng.uniform(np.log(k_range[0]), np.log(k_range[1])))))
        npc = int(min(n, rng.integers(nnz_range[0], nnz_range[1] + 1)))
        loss = SQUARED if rng.random() < 0.5 else LOGISTIC
        fracs.append(float(rng.uniform(0.01, 0.3)))
        s = int(rng.integers(0, 2**31 - 1))
        problems.append(uniform_problem(n, k, npc, values="lognormal", n_planted=min(50, k), loss=loss, seed=s,
                                        name=f"request-{n}x{k}-{npc}nnz-{loss}"))
    return problems, np.array(fracs), arrivals


def tiny_problem(n, k, density=0.6, loss=LOGISTIC, seed=0, max_tries=1000) -> Problem:
    """A small problem with n >= k and full column rank (so the l1 optimum is
    unique), for brute-force checks.  Values are N(0,1) on a random pattern."""
    rng = _rng(seed)
    for _ in range(max_tries):
        mask = rng.random((n, k)) < density
        vals = rng.normal(0.0, 1.0, (n, k))
        X = np.where(mask, vals, 0.0)
        if np.linalg.matrix_rank(X) < k or (np.abs(X).sum(axis=0) == 0).any():
            continue
        w_star = rng.normal(0.0, 1.0, k) * (rng.random(k) < 0.5)
        t = X @ w_star
        if loss == LOGISTIC:
            y = np.where(t + rng.normal(0.0, 1.0, n) >= 0.0, 1.0, -1.0)
        else:
            y = t + rng.normal(0.0, 0.1, n)
        p = csc_from_dense(X, y, loss)
        p.w_star = w_star
        return p
    raise RuntimeError("could not draw a full-rank tiny problem")


def csc_from_dense(X: np.ndarray, y: np.ndarray, loss: str, name="") -> Problem:
    """CSC arrays of a dense matrix (structural zeros dropped)."""
    X = np.asarray(X, np.float64)
    n, k = X.shape
    cols, rows, vals = [], [], []
    counts = np.zeros(k, np.int64)
    for j in range(k):
        nz = np.flatnonzero(X[:, j])
        counts[j] = nz.size
        rows.append(nz.astype(np.int32))
        vals.append(X[nz, j])
    col_ptr = _col_ptr(counts)
    row_idx = np.concatenate(rows) if rows else np.zeros(0, np.int32)
    val = np.concatenate(vals) if vals else np.zeros(0)
    return Problem(n, k, col_ptr, row_idx.astype(np.int32), val.astype(np.float64),
                   np.asarray(y, np.float64), loss, np.zeros(k), name)
