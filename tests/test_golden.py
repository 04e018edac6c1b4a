"""Stored expected values (tests/golden/, written by make_golden.py from the
oracle alone) and their checks.

* The Boys values are pinned to mathematics independently of the oracle:
  F_0(T) = sqrt(pi/T) erf(sqrt(T)) / 2, F_m(0) = 1/(2m+1), and the others to
  scipy's adaptive quadrature of the defining integral.
* The c1 gradient is a regression pin of the oracle (it must keep
  reproducing it) and the target of the GPU check, which then needs no
  oracle run; it also satisfies translational invariance (Eq. ti).
"""
import math
import os

import numpy as np
import pytest

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _c1():
    rows, nq = [], None
    with open(os.path.join(HERE, "c1_grad.txt")) as f:
        for line in f:
            if line.startswith("# quartets"):
                nq = int(line.split()[2])
            elif not line.startswith("#"):
                rows.append([float(x) for x in line.split()])
    return np.array(rows), nq


def _boys():
    with open(os.path.join(HERE, "boys.txt")) as f:
        return [(int(a), float(b), float(c)) for a, b, c in (l.split() for l in f if not l.startswith("#"))]


def test_boys_golden_against_mathematics():
    from scipy import integrate
    for m, T, v in _boys():
        if T == 0.0:
            ref = 1.0 / (2 * m + 1)
        elif m == 0:
            ref = 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
        else:
            ref, _ = integrate.quad(lambda t: t ** (2 * m) * math.exp(-T * t * t), 0.0, 1.0,
                                    epsabs=0.0, epsrel=1e-13, limit=200)
        assert abs(v - ref) <= 1e-14 * max(abs(ref), 1e-300) + 1e-300, (m, T, v, ref)


def test_c1_golden_invariants():
    g, nq = _c1()
    assert g.shape == (6, 3) and nq == 45150
    assert np.abs(g.sum(axis=0)).max() <= 1e-10   # Eq. ti


def test_oracle_reproduces_c1_golden(c1):
    import oracle
    g, nq = _c1()
    ref, _, n = oracle.grad2e(c1, tau=0.0)
    assert n == nq
    assert np.abs(ref - g).max() <= 1e-13 * max(1.0, np.abs(g).max())


@pytest.mark.gpu
def test_cuda_path_matches_c1_golden(c1):
    from paper_2407_16586_gb300 import build
    build.build()
    import paper_2407_16586_gb300 as tg
    g, nq = _c1()
    out, st = tg.grad2e(c1, screen_tol=0.0)
    assert st["quartets"] == nq
    assert np.abs(out - g).max() <= 1e-10
