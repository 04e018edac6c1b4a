"""Pins of the oracle's Fock-type build (Sec. II.B: the two-electron part of
eqs. G_2e and zfock),
  F[mu nu] = sum_p sum_{lam sig} B_p[lam sig] (c_J (mu nu|lam sig)
             + c_K (mu lam|nu sig) + c_K_lr (mu lam|nu sig)_w).

Independent routes:
  * trace identity: Tr(A^T F(B)) = sum A_mu_nu F_mu_nu equals the oracle's
    canonical energy E(A, B) = sum (mu nu|lam sig) [c_J A_mu_nu B_lam_sig +
    c_K A_mu_lam B_nu_sig + ...] -- a different code path (8 permutation
    images of canonical quartets, itself pinned by finite differences of its
    gradient) against the plain scatter of the Fock build;
  * element by element: F from the full 4-index integral tensor assembled
    from shell-quartet integrals and contracted with numpy einsum;
  * omega -> infinity: the erf operator's exchange equals the full one.
"""
import numpy as np
import pytest

import oracle
from paper_2407_16586_gb300 import synth


@pytest.fixture(scope="module")
def small():
    return synth.molecule(31, 1, 2)


def _rand(n, seed, sym=False):
    rng = np.random.default_rng(seed)
    m = rng.normal(size=(n, n)) / n
    return m + m.T if sym else m


def test_trace_identity_against_the_canonical_energy(small):
    nbf = small["pairs"][0][0].shape[0]
    A, B = _rand(nbf, 1), _rand(nbf, 2)
    for cJ, cK, cKlr, w in [(1.0, 0.0, 0.0, 0.0), (0.0, 1.0, 0.0, 0.0), (0.0, 0.0, 1.0, 0.3),
                            (2.0, -0.158, -0.842, 0.3)]:
        F = oracle.fock2e(small, [(B, cJ, cK, cKlr, w)])
        e = oracle.grad2e(small, pairs=[(A, B, cJ, cK, cKlr, w)], want_grad=False, want_energy=True)[1]
        tr = float(np.sum(A * F))
        assert tr == pytest.approx(e, rel=1e-12, abs=1e-13), (cJ, cK, cKlr, tr, e)


def _full_eri(s, omega=0.0):
    ls = list(s["shell_l"])
    nc = [(l + 1) * (l + 2) // 2 for l in ls]
    off = np.concatenate([[0], np.cumsum(nc)])
    n = off[-1]
    eri = np.zeros((n, n, n, n))
    ns = len(ls)
    for a in range(ns):
        for b in range(ns):
            for c in range(ns):
                for d in range(ns):
                    eri[off[a]:off[a + 1], off[b]:off[b + 1], off[c]:off[c + 1], off[d]:off[d + 1]] = \
                        oracle.shell_eri(s, a, b, c, d, omega=omega)
    return eri


def test_elements_against_the_integral_tensor():
    s = synth.molecule(32, 1, 1)
    nbf = s["pairs"][0][0].shape[0]
    eri, erl = _full_eri(s), _full_eri(s, 0.3)
    B = _rand(nbf, 3)
    F = oracle.fock2e(s, [(B, 0.7, -0.3, 0.9, 0.3)])
    ref = (0.7 * np.einsum("mnls,ls->mn", eri, B) - 0.3 * np.einsum("mlns,ls->mn", eri, B)
           + 0.9 * np.einsum("mlns,ls->mn", erl, B))
    assert np.abs(F - ref).max() <= 1e-12 * np.abs(ref).max()


def test_omega_infinity_and_symmetry(small):
    nbf = small["pairs"][0][0].shape[0]
    B = _rand(nbf, 4, sym=True)
    Fk = oracle.fock2e(small, [(B, 0.0, 1.0, 0.0, 0.0)])
    Fl = oracle.fock2e(small, [(B, 0.0, 0.0, 1.0, float("inf"))])
    assert np.abs(Fk - Fl).max() <= 1e-12 * np.abs(Fk).max()
    Fj = oracle.fock2e(small, [(B, 1.0, 0.0, 0.0, 0.0)])
    assert np.abs(Fj - Fj.T).max() <= 1e-12 * np.abs(Fj).max()
    assert np.abs(Fk - Fk.T).max() <= 1e-12 * np.abs(Fk).max()


def test_zfock_pair_mapping():
    """The binding's zfock_pairs against eq. zfock written out with the
    4-index integral tensor: sum_{lam sig} B[sig lam] (4 (mu nu|lam sig)
    - alpha ((mu lam|sig nu) + (mu sig|lam nu)) - beta (...)_lr)."""
    import paper_2407_16586_gb300 as tg
    s = synth.molecule(33, 1, 1)
    nbf = s["pairs"][0][0].shape[0]
    eri, erl = _full_eri(s), _full_eri(s, 0.3)
    B = _rand(nbf, 7)
    a, b = 0.157706, 0.842294
    ref = (4 * np.einsum("mnls,sl->mn", eri, B)
           - a * (np.einsum("mlsn,sl->mn", eri, B) + np.einsum("msln,sl->mn", eri, B))
           - b * (np.einsum("mlsn,sl->mn", erl, B) + np.einsum("msln,sl->mn", erl, B)))
    F = oracle.fock2e(s, tg.zfock_pairs(B, a, b, 0.3))
    assert np.abs(F - ref).max() <= 1e-12 * np.abs(ref).max()
