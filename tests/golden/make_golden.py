"""Write the stored expected values under tests/golden/ from the oracle only.

  python tests/golden/make_golden.py

* c1_grad.txt: the two-electron gradient of the c1 workload (2 O + 4 H,
  pairs J(A,A) + K(A,A), c = 1, and K_lr(X,X), omega = 0.3; no screening),
  i.e. terms 4 and 5 of Eq. dE_ao (Sec. II.A) with the density pairs written
  as (A, B, c_J, c_K, c_K_lr, omega), and its canonical quartet count.
* boys.txt: F_m(T) = int_0^1 t^(2m) exp(-T t^2) dt (the Boys function that
  seeds the Hermite R tensor of Sec. II.C) at sample points, from the
  oracle's long-double evaluation.

Nothing here reads the CUDA library."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2407_16586_gb300 import synth  # noqa: E402

BOYS_POINTS = [(0, 0.0), (0, 1.0), (3, 0.5), (5, 12.0), (8, 30.0), (9, 45.0), (16, 2.0)]


def main():
    oracle.build()
    s = synth.config(0)
    g, e, nq = oracle.grad2e(s, tau=0.0, want_energy=True)
    with open(os.path.join(HERE, "c1_grad.txt"), "w") as f:
        f.write("# c1 two-electron gradient (Ha/bohr), Sec. II.A Eq. dE_ao terms 4-5; oracle, tau = 0\n")
        f.write("# quartets %d\n# energy %.17e\n" % (nq, e))
        for row in g:
            f.write("%.17e %.17e %.17e\n" % tuple(row))
    with open(os.path.join(HERE, "boys.txt"), "w") as f:
        f.write("# m T F_m(T), F_m(T) = int_0^1 t^(2m) exp(-T t^2) dt (Sec. II.C); oracle long double\n")
        for m, T in BOYS_POINTS:
            f.write("%d %.17e %.17e\n" % (m, T, oracle.boys(m, T)[m]))


if __name__ == "__main__":
    main()
