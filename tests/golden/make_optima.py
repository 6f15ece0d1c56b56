"""Writes the stored oracle optima tests/golden/optimum_<name>.txt.

Each file holds the FP64 oracle's cyclic-CD solution (Section 2.1, run until
the oracle's KKT violation is at most 1e-11) of one seeded problem: config 3's
shapes (n = 2,000, k = 5,000, 20 non-zeros per column) with +-1, all-ones and
log-normal unit-norm values, logistic loss, lambda = 0.01 lambda_max, and the
log-normal problem with its values as bfloat16 storage holds them.  Solving
these ill-conditioned problems to 1e-11 takes the oracle about a minute each,
so the GPU tests load the stored optimum and re-certify it with one oracle KKT
pass (parity_tools.certified_optimum).  Calls only the oracle and the seeded
generators.

    python tests/golden/make_optima.py
"""

import hashlib
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import workloads  # noqa: E402

LAM_FRAC = 0.01


def problems():
    """name -> (problem, lambda); every lambda is 0.01 lambda_max of the
    problem's original (unrounded) values, as the precision sweep sets it."""
    pm1 = workloads.config3("pm1", "logistic")
    ones = workloads.config3("ones", "logistic")
    ln = workloads.config3("lognormal", "logistic")
    lam = {p.name: LAM_FRAC * oracle.Oracle(p).lambda_max() for p in (pm1, ones, ln)}
    return {
        "cfg3_pm1_logistic": (pm1, lam[pm1.name]),
        "cfg3_ones_logistic": (ones, lam[ones.name]),
        "cfg3_lognormal_logistic": (ln, lam[ln.name]),
        "cfg3_lognormal_logistic_bf16": (oracle.stored_problem(ln, "bf16"), lam[ln.name]),
    }


def write(name, prob, lam):
    orc = oracle.Oracle(prob)
    orc.set_lambda(lam)
    w, _, iters, kkt, _ = orc.solve("ccd", tol_kkt=1e-11, max_iter=4 * 10**8)
    assert kkt <= 1e-11, (name, kkt)
    nz = np.flatnonzero(w)
    with open(os.path.join(HERE, f"optimum_{name}.txt"), "w") as f:
        f.write(f"# oracle cyclic-CD optimum of {prob.name} ({name}), logistic loss, lambda = {LAM_FRAC} "
                "lambda_max of the original values\n")
        f.write("# written by tests/golden/make_optima.py (oracle only); lines: column value\n")
        f.write(f"meta k {prob.k}\n")
        f.write(f"meta lambda {float(lam)!r}\n")
        f.write(f"meta lambda_frac {LAM_FRAC!r}\n")
        f.write(f"meta kkt {float(kkt)!r}\n")
        f.write(f"meta iterations {iters}\n")
        f.write(f"meta objective {float(orc.objective(w))!r}\n")
        f.write(f"meta problem_sha256 {prob.sha256()}\n")
        for j in nz:
            f.write(f"{int(j)} {float(w[j])!r}\n")
    print(name, "kkt", kkt, "nonzeros", nz.size, flush=True)


if __name__ == "__main__":
    only = set(sys.argv[1:])
    for name, (prob, lam) in problems().items():
        if not only or name in only:
            write(name, prob, lam)
