"""Parity of the Fock-type build (tg_fock2e, Sec. II.B: the two-electron part
of eqs. G_2e and zfock) with the oracle's plain definition.

Tolerance: fp64 throughout; every element agrees with the oracle to 1e-11 of
the largest |F| element (rounding of sums of up to 10^5 fp64 terms, added in
scheduling order by fp64 atomics).  The molecules hold s, p and d shells, so
every angular class contributes."""
import numpy as np
import pytest

import oracle
from paper_2407_16586_gb300 import synth

pytestmark = pytest.mark.gpu
REL = 1e-11


@pytest.fixture(scope="module")
def tg():
    from paper_2407_16586_gb300 import build
    build.build()
    import paper_2407_16586_gb300 as m
    return m


def _rand(n, seed):
    return np.random.default_rng(seed).normal(size=(n, n)) / n


def test_fock_every_class_against_the_oracle(tg):
    s = synth.molecule(14, 3, 3)
    n = s["pairs"][0][0].shape[0]
    pairs = [(_rand(n, 1), 2.0, -0.158, -0.842, 0.3), (_rand(n, 2), 0.5, 0.7, 0.0, 0.0)]
    ref = oracle.fock2e(s, pairs)
    F, st = tg.Basis(s).fock2e(pairs, screen_tol=0.0)
    assert st["quartets"] > 0 and all(c > 0 for c in st["class_quartets"])
    assert np.abs(F - ref).max() <= REL * np.abs(ref).max(), np.abs(F - ref).max()


def test_fock_single_terms_and_limits(tg):
    s = synth.molecule(15, 2, 2)
    n = s["pairs"][0][0].shape[0]
    B = _rand(n, 3)
    b = tg.Basis(s)
    for pair in [(B, 1.0, 0.0, 0.0, 0.0), (B, 0.0, 1.0, 0.0, 0.0), (B, 0.0, 0.0, 1.0, 0.3),
                 (B, 0.0, 0.0, 1.0, float("inf"))]:
        ref = oracle.fock2e(s, [pair])
        F, _ = b.fock2e([pair], screen_tol=0.0)
        assert np.abs(F - ref).max() <= REL * np.abs(ref).max(), pair[1:]


def test_zfock_pairs_on_the_gpu(tg):
    """eq. zfock through its pair mapping: the GPU build equals the oracle's."""
    s = synth.molecule(16, 2, 1)
    n = s["pairs"][0][0].shape[0]
    pairs = tg.zfock_pairs(_rand(n, 4), 0.157706, 0.842294, 0.3)
    ref = oracle.fock2e(s, pairs)
    F, _ = tg.Basis(s).fock2e(pairs, screen_tol=0.0)
    assert np.abs(F - ref).max() <= REL * np.abs(ref).max()


def test_fock_screening_stays_within_its_bound(tg):
    s = synth.molecule(17, 3, 4)
    n = s["pairs"][0][0].shape[0]
    pairs = [(s["pairs"][0][0], 2.0, -0.158, -0.842, 0.3)]
    b = tg.Basis(s)
    F0, st0 = b.fock2e(pairs, screen_tol=0.0)
    F1, st1 = b.fock2e(pairs, screen_tol=1e-10)
    assert st1["quartets"] < st0["quartets"]
    assert np.abs(F1 - F0).max() <= 1e-8
