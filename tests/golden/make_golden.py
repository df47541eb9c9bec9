"""Writes the oracle-derived golden files.  Calls only oracle/ and workloads/."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as w  # noqa: E402
from oracle import boxmg as bx  # noqa: E402


def main():
    kind, planes, f = w.poisson_problem(127, 1)
    levels = bx.setup(kind, planes)
    _, hist = bx.solve(levels, f, tol=1e-10, maxit=50)
    with open(os.path.join(HERE, "poisson127_history.txt"), "w") as fh:
        fh.write("# FP64 oracle residual history, 127x127 5-point Poisson, RHS seed 1,\n")
        fh.write("# red-black GS V(2,1), 6 levels, tol 1e-10 (written by make_golden.py)\n")
        for v in hist:
            fh.write(f"{v!r}\n")


if __name__ == "__main__":
    main()
