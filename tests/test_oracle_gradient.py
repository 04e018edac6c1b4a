"""Pins for the oracle's two-electron gradient (Sec. II.A eq. dE_ao terms 4-5,
Sec. II.C eqs. deriv, deri, ti, eriupdate; Sec. II.E finite-difference
validation and density-multiplied Schwarz screening).

* central finite differences of E(R) = sum Gamma (mn|ls) with moving centres;
* translational invariance, sum over atoms of g = 0 (eq. ti);
* a single atom has zero gradient (every quartet is one-centre);
* closed forms for two atoms with one s primitive each (Coulomb of two
  Gaussian charges, erf(sqrt(rho) R)/R, and the self-repulsion of their
  overlap charge);
* the paper's Gamma (eq. gamma) contracted directly against derivative
  integrals equals the (A, B, c) pair list;
* plain (all ordered quartets) = canonical (8-fold) mode;
* J(A,B) = J(B,A), K(A,B) = K(B,A); shards sum to the whole; screening."""
import math

import numpy as np
import pytest

import oracle
from paper_2407_16586_gb300 import synth


@pytest.fixture(scope="module")
def small():
    return synth.molecule(3, 1, 2)


@pytest.fixture(scope="module")
def c1_grad(c1):
    g, e, n = oracle.grad2e(c1, want_energy=True)
    return g, e, n


def test_finite_difference(small):
    g, _, _ = oracle.grad2e(small)
    h = 1e-4
    xyz0 = small["xyz"].copy()
    for atom in range(small["natom"]):
        for i in range(3):
            xp = xyz0.copy(); xp[atom, i] += h
            xm = xyz0.copy(); xm[atom, i] -= h
            ep = oracle.grad2e(small, xyz=xp, want_grad=False, want_energy=True)[1]
            em = oracle.grad2e(small, xyz=xm, want_grad=False, want_energy=True)[1]
            fd = (ep - em) / (2 * h)
            assert abs(fd - g[atom, i]) <= 1e-7, (atom, i, fd, g[atom, i])


def test_finite_difference_lr_only(small):
    x = small["pairs"][2][0]
    pairs = [(x, x.T.copy(), 0.0, 0.0, 1.0, 0.3)]
    g, _, _ = oracle.grad2e(small, pairs=pairs)
    h = 1e-4
    xyz0 = small["xyz"].copy()
    for atom, i in [(0, 0), (1, 2), (2, 1)]:
        xp = xyz0.copy(); xp[atom, i] += h
        xm = xyz0.copy(); xm[atom, i] -= h
        ep = oracle.grad2e(small, pairs=pairs, xyz=xp, want_grad=False, want_energy=True)[1]
        em = oracle.grad2e(small, pairs=pairs, xyz=xm, want_grad=False, want_energy=True)[1]
        assert abs((ep - em) / (2 * h) - g[atom, i]) <= 1e-7


def test_translational_invariance(c1_grad):
    g, _, _ = c1_grad
    assert np.abs(g.sum(axis=0)).max() <= 1e-10
    assert np.abs(g).max() > 0.1


def test_single_atom_zero():
    s = synth.molecule(8, 1, 0)
    g, _, _ = oracle.grad2e(s)
    # zero up to the rounding of sum_X d/dX over four explicit centres
    assert np.abs(g).max() <= 1e-11


def _two_s(R, a, b):
    return dict(natom=2, xyz=np.array([[0.0, 0.0, 0.0], [0.3 * R, -0.4 * R, math.sqrt(1 - 0.25) * R]]),
                shell_atom=np.array([0, 1], dtype=np.int32), shell_l=np.zeros(2, dtype=np.int32),
                shell_nprim=np.ones(2, dtype=np.int32), exps=np.array([a, b]), coefs=np.ones(2))


@pytest.mark.parametrize("R,a,b", [(1.7, 0.8, 2.5), (3.0, 0.3, 0.3), (0.9, 5.0, 0.4)])
def test_two_s_primitives_closed_form(R, a, b):
    s = _two_s(R, a, b)
    u = s["xyz"][1] - s["xyz"][0]
    u /= np.linalg.norm(u)
    eye = np.eye(2)
    rho = (2 * a) * (2 * b) / (2 * a + 2 * b)

    def dcoul(k):  # d/dR [erf(k R)/R]
        return 2 * k / math.sqrt(math.pi) * math.exp(-k * k * R * R) / R - math.erf(k * R) / R ** 2

    # J(I, I): E = (11|11) + (22|22) + 2 (11|22), (11|22) = erf(sqrt(rho) R)/R
    g, _, _ = oracle.grad2e(s, pairs=[(eye, eye, 1.0, 0.0, 0.0, 0.0)])
    dEdR = 2 * dcoul(math.sqrt(rho))
    np.testing.assert_allclose(g[1], dEdR * u, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(g[0], -dEdR * u, rtol=1e-12, atol=1e-14)
    w = 0.3
    # K(I, I): E = (11|11) + (22|22) + 2 (12|12); (12|12) = |N1 N2 K12|^2 2 pi^(5/2)/(p^2 sqrt(2p))
    g, _, _ = oracle.grad2e(s, pairs=[(eye, eye, 0.0, 1.0, 0.0, 0.0)])
    p = a + b
    n1 = (2 * a / math.pi) ** 0.75
    n2 = (2 * b / math.pi) ** 0.75
    k12sq = math.exp(-2 * a * b / p * R * R)
    e1212 = (n1 * n2) ** 2 * k12sq * 2 * math.pi ** 2.5 / (p * p * math.sqrt(2 * p))
    dEdR = 2 * e1212 * (-4 * a * b / p * R)
    np.testing.assert_allclose(g[1], dEdR * u, rtol=1e-12, atol=1e-14)
    # lr exchange: erf kernel at zero separation of the overlap charge gives
    # (12|12)_w = (12|12) * theta, theta^2 = w^2/(w^2 + p/2)
    g, _, _ = oracle.grad2e(s, pairs=[(eye, eye, 0.0, 0.0, 1.0, w)])
    th = math.sqrt(w * w / (w * w + p / 2))
    np.testing.assert_allclose(g[1], th * dEdR * u, rtol=1e-12, atol=1e-14)


def _nc(l):
    return (l + 1) * (l + 2) // 2


def test_gamma_mapping_matches_paper_gamma():
    """Gamma and Gamma^lr of eq. gamma contracted with derivative integrals of
    every ordered shell quartet equal the pair list (R,R; 2, -a, -b) +
    (D,P; 1/2, -a/4, -b/4) with D = P + 2 P_delta (P symmetric)."""
    s = synth.molecule(21, 1, 1)
    nbf = s["nbf"]
    rng = np.random.default_rng(4)
    Cm = rng.normal(0, 0.3, size=(nbf, 3))
    P = Cm @ Cm.T
    Cd = rng.normal(0, 0.3, size=(nbf, 3))
    Pd = Cd @ Cd.T - 0.5 * P
    R = rng.normal(size=(nbf, nbf)) / nbf
    D = P + 2 * Pd
    al, be, w = 0.157706, 1 - 0.157706, 0.3
    G = (2 * np.einsum("nm,ls->mnls", R, R) - al * np.einsum("sm,ln->mnls", R, R)
         + 0.5 * (np.einsum("mn,ls->mnls", D, P) - al / 2 * np.einsum("ms,ln->mnls", D, P)))
    Glr = -be * np.einsum("sm,ln->mnls", R, R) - be / 4 * np.einsum("ms,ln->mnls", D, P)
    ns = len(s["shell_l"])
    off = np.concatenate([[0], np.cumsum([_nc(l) for l in s["shell_l"]])])
    g = np.zeros((s["natom"], 3))
    for a in range(ns):
        for b in range(ns):
            for c in range(ns):
                for d in range(ns):
                    sl = tuple(slice(off[x], off[x + 1]) for x in (a, b, c, d))
                    Df = oracle.shell_eri_deriv(s, a, b, c, d)
                    Dl = oracle.shell_eri_deriv(s, a, b, c, d, omega=w)
                    gg = np.einsum("xiabcd,abcd->xi", Df, G[sl]) + np.einsum("xiabcd,abcd->xi", Dl, Glr[sl])
                    for X, sh in enumerate((a, b, c, d)):
                        g[s["shell_atom"][sh]] += gg[X]
    pairs = [(R, R, 2.0, -al, -be, w), (D, P, 0.5, -al / 4, -be / 4, w)]
    g2, _, _ = oracle.grad2e(s, pairs=pairs)
    np.testing.assert_allclose(g2, g, atol=1e-12 * np.abs(g).max(), rtol=0)
    # the binding's helper passes the same Gamma as three pairs, (D, P) split
    # into (P, P) + 2 (P_delta, P)
    from paper_2407_16586_gb300 import tda_pairs
    g3, _, _ = oracle.grad2e(s, pairs=tda_pairs(P, Pd, R, al, be, w))
    np.testing.assert_allclose(g3, g, atol=1e-12 * np.abs(g).max(), rtol=0)


def test_plain_equals_canonical(small):
    g1, e1, _ = oracle.grad2e(small, mode="plain", want_energy=True)
    g2, e2, _ = oracle.grad2e(small, mode="canonical", want_energy=True)
    np.testing.assert_allclose(g1, g2, atol=1e-12, rtol=0)
    assert e1 == pytest.approx(e2, rel=1e-13)


def test_c1_canonical_quartet_count(c1_grad):
    # 24 shells -> 300 shell pairs -> 300*301/2 canonical quartets at tau = 0
    assert c1_grad[2] == 45150


def test_coulomb_exchange_swap_symmetry(small):
    p, pd, x = small["pairs"][0][0], small["pairs"][1][0], small["pairs"][2][0]
    for cj, ck in [(1.0, 0.0), (0.0, 1.0)]:
        ga, _, _ = oracle.grad2e(small, pairs=[(pd, x, cj, ck, 0.0, 0.0)])
        gb, _, _ = oracle.grad2e(small, pairs=[(x, pd, cj, ck, 0.0, 0.0)])
        np.testing.assert_allclose(ga, gb, atol=1e-13, rtol=0)
    # J only sees symmetric parts: J(X, P) = J((X+X^T)/2, P)
    ga, _, _ = oracle.grad2e(small, pairs=[(x, p, 1.0, 0.0, 0.0, 0.0)])
    gb, _, _ = oracle.grad2e(small, pairs=[(0.5 * (x + x.T), p, 1.0, 0.0, 0.0, 0.0)])
    np.testing.assert_allclose(ga, gb, atol=1e-13, rtol=0)
    # K(A, B) = K(A^T, B^T) but not K(A, B^T) for non-symmetric matrices
    ga, _, _ = oracle.grad2e(small, pairs=[(x, pd, 0.0, 1.0, 0.0, 0.0)])
    gb, _, _ = oracle.grad2e(small, pairs=[(x.T.copy(), pd.T.copy(), 0.0, 1.0, 0.0, 0.0)])
    gc, _, _ = oracle.grad2e(small, pairs=[(x, pd.T.copy(), 0.0, 1.0, 0.0, 0.0)])
    np.testing.assert_allclose(ga, gb, atol=1e-13, rtol=0)
    assert np.abs(ga - gc).max() > 1e-8 or np.abs(pd - pd.T).max() == 0


def test_pairs_are_additive(small):
    g, _, _ = oracle.grad2e(small)
    parts = sum(oracle.grad2e(small, pairs=[p])[0] for p in small["pairs"])
    np.testing.assert_allclose(g, parts, atol=1e-12, rtol=0)


def test_shards_sum_to_whole(small):
    g, _, n = oracle.grad2e(small)
    tot = np.zeros_like(g)
    ntot = 0
    for r in range(3):
        gr, _, nr = oracle.grad2e(small, rank=r, nranks=3)
        tot += gr
        ntot += nr
    assert ntot == n
    np.testing.assert_allclose(tot, g, atol=1e-12, rtol=0)


def test_screening_is_rigorous_enough(small):
    g0, _, n0 = oracle.grad2e(small, tau=0.0)
    g1, _, n1 = oracle.grad2e(small, tau=1e-10)
    g2, _, n2 = oracle.grad2e(small, tau=1e-6)
    assert n2 < n1 <= n0
    assert np.abs(g1 - g0).max() <= 1e-9
    assert np.abs(g2 - g0).max() <= 1e-4


def test_class_filter_partitions_the_quartets(c1):
    """The 21 angular classes partition the canonical quartets: the
    class-filtered gradients and quartet counts sum to the whole, and every
    class of c1's s, p, d shells holds quartets."""
    g, _, nq = oracle.grad2e(c1, tau=1e-10)
    tot = np.zeros_like(g)
    n = 0
    for qc in range(21):
        gq, _, nqq = oracle.grad2e(c1, tau=1e-10, qclass=qc)
        assert nqq > 0, qc
        tot += gq
        n += nqq
    assert n == nq
    assert np.abs(tot - g).max() <= 1e-12 * max(1.0, np.abs(g).max())


def test_rigid_translation_leaves_the_gradient_unchanged():
    """The integrals, and so the gradient, depend on the relative positions of
    the centres only (Sec. II.C): shifting the whole molecule by tens of bohr
    changes the c1 gradient by rounding only (the oracle forms P - A, P - Q
    and W - P from centre differences)."""
    s = synth.config(0)
    g0 = oracle.grad2e(s, tau=0.0)[0]
    for shift in ([40.0, 35.0, -30.0], [-120.0, 5.0, 60.0]):
        g1 = oracle.grad2e(s, tau=0.0, xyz=s["xyz"] + np.array(shift))[0]
        assert np.abs(g1 - g0).max() <= 1e-12 * np.abs(g0).max(), shift
