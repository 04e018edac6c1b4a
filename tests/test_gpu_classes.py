"""Per-class parity of every class-kernel form against the oracle restricted
to the same angular class (tg_options.class_mask against the oracle's
qclass filter), in fp64 and in fp32.

Tolerances:
  * fp64: 1e-10 Ha/bohr per gradient component, the plain path's bound.
  * fp32: the fp32 route computes each primitive quartet with fp32 operands
    and products (unit roundoff u = 2^-24 = 6.0e-8) and adds the
    contributions to fp64 accumulators.  A gradient component of one class
    is a sum of products whose longest chain of fp32 roundings (Boys value,
    R recursion of at most 9 levels, one contraction of at most 56 terms, the
    derivative product) holds about 10^2 roundings, so its relative error is
    bounded by about 10^2 u = 6e-6 of the class's largest component.  The
    bound used is max|dg| <= 6e-6 * max|g_class| (+1e-12 for classes whose
    gradient is nearly zero); on this molecule max|g_class| is 0.1..8, so the
    bound is 6e-7..5e-5 Ha/bohr, class by class.
"""
import numpy as np
import pytest

import oracle
from paper_2407_16586_gb300 import synth

pytestmark = pytest.mark.gpu
TOL64 = 1e-10
REL32 = 6e-6
NAMES = ["ssss", "psss", "psps", "ppss", "ppps", "pppp", "dsss", "dsps", "dspp", "dsds", "dpss", "dpps", "dppp",
         "dpds", "dpdp", "ddss", "ddps", "ddpp", "ddds", "dddp", "dddd"]


@pytest.fixture(scope="module")
def tg():
    from paper_2407_16586_gb300 import build
    build.build()
    import paper_2407_16586_gb300 as m
    return m


@pytest.fixture(scope="module")
def system():
    return synth.molecule(14, 3, 3)


@pytest.fixture(scope="module")
def refs(system):
    return {qc: oracle.grad2e(system, tau=0.0, qclass=qc) for qc in range(21)}


@pytest.mark.parametrize("qc", range(21), ids=NAMES)
def test_class_fp64_every_form(tg, system, refs, qc):
    ref, _, nq = refs[qc]
    b = tg.Basis(system)
    assert nq > 0
    for kernel in (1, 2, 3):
        g, st = b.grad2e(system["pairs"], screen_tol=0.0, kernel=kernel, class_mask=1 << qc)
        assert st["quartets"] == nq, (kernel, st["quartets"], nq)
        assert st["class_quartets"][qc] == nq
        assert np.abs(g - ref).max() <= TOL64, (kernel, np.abs(g - ref).max())


@pytest.mark.parametrize("qc", range(21), ids=NAMES)
def test_class_fp32_every_form(tg, system, refs, qc):
    ref, _, nq = refs[qc]
    b = tg.Basis(system)
    scale = float(np.abs(ref).max())
    for kernel in (1, 2, 3):
        g, st = b.grad2e(system["pairs"], screen_tol=0.0, kernel=kernel, class_mask=1 << qc,
                         precision=tg.TG_FP32)
        assert st["quartets"] == nq and st["fp32_quartets"] == nq
        err = float(np.abs(g - ref).max())
        assert err <= REL32 * scale + 1e-12, (kernel, err, scale, err / scale)
