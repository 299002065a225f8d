"""Writes tests/golden/oracle_counts.txt: the oracle's own multigrid iteration counts and per-cycle
relative residuals on the benchmark problems at full size. Calls only oracle/ and the seeded input
generators; run it from the repository root: python tests/golden/make_oracle_counts.py"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1402_3545_gb300 import workloads  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_counts.txt")


def main():
    lines = ["# Oracle (plain FP64 C) multigrid solves of the benchmark problems: V(2,2), rho = 0.8,",
             "# 2 coarse smoothing steps, zero initial guess, stop at ||r||/||r0|| < tol (Eq. (10)).",
             "# Written by tests/golden/make_oracle_counts.py, which calls only oracle/."]
    for name, p, tol in [("small", workloads.small(), 1e-6), ("mid", workloads.mid(), 1e-6)]:
        f = p.rhs()
        cx, cy, v = oracle.problem_coefficients(p)
        t0 = time.time()
        u, it, hist, conv = oracle.mg_solve(f, cx, cy, v, p.nlevels, tol=tol, max_iter=100)
        dt = time.time() - t0
        lines.append(f"{name}_iters {it}")
        lines.append(f"{name}_converged {int(conv)}")
        lines.append(f"{name}_final_rel {hist[-1]:.6e}")
        lines.append(f"# {name}: {p.nx}x{p.ny}x{p.nz}, {p.nlevels} levels, history "
                     + " ".join(f"{h:.3e}" for h in hist) + f" ({dt:.1f} s here)")
    with open(OUT, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print("\n".join(lines))


if __name__ == "__main__":
    main()
