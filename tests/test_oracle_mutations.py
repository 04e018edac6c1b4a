"""The pins have teeth: each plausible mistake planted in the oracle (built
with -DOR_MUTATION=k into a temporary directory, never shipped) must fail the
pin named beside it, while the real oracle passes every pin.

Pins used here (all independent of the oracle's own formulas):
  boys        F_0 closed form and the defining integral by quadrature
  norm        unit self-overlap of a normalised d shell and unit-norm
              primitives under its coefficients, by quadrature
  ssss        closed-form [ss|ss] of both operators (Boys F_0 only)
  quadrature  a (pp|ps) primitive quartet of both operators against the
              Gaussian-geminal quadrature of tests/test_oracle_integrals.py
  fd          central finite differences of E(R) (h = 1e-4 bohr, 1e-7)
  canonical   plain (all ordered quartets) = canonical (8 images/stabiliser)
  gamma       the paper's Gamma (eq. gamma) written as a 4-index tensor and
              contracted with the oracle's derivative integrals = the pair list
  fock        the Fock-type build's trace against the canonical energy
  contraction a (pp|ps) quartet of 2-3-primitive shells of both operators
              against the quadrature of tests/test_oracle_contraction.py, with
              that file's own normalisation
"""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2407_16586_gb300 import synth
from test_oracle_integrals import _cart, _mini_system, geminal_eri
from test_oracle_contraction import contracted_reference, oracle_system, random_shells

MUTATIONS = {
    1: ("derivative rule without its lowering term", "fd"),
    2: ("wrong sign of the electron-transfer term of the vertical recursion", "quadrature"),
    3: ("theta^(2m) instead of theta^(2m+1) for the erf operator", "ssss"),
    4: ("wrong sign in the downward Boys recursion", "boys"),
    5: ("(4 zeta)^l instead of (4 zeta)^(l/2) in the primitive norm", "norm"),
    6: ("one exchange image listed twice, another missing", "canonical"),
    7: ("stabiliser factor of (ab) = (cd) dropped", "canonical"),
    8: ("d/dC added to the atom of D", "fd"),
    9: ("wrong sign of A - B in the horizontal transfer", "quadrature"),
    10: ("transposed first exchange density, A_lm B_ns instead of A_ml B_ns", "gamma"),
    12: ("wrong sign in the upward Boys recursion (large T)", "boys"),
    13: ("coefficient of shell d taken at shell c's primitive index", "contraction"),
    14: ("first primitive's coefficient of shell b used for all its primitives", "contraction"),
    15: ("Fock exchange block read with the density transposed", "fock"),
    16: ("product centres kept as absolute positions (P - A by cancellation)", "translation"),
}


def pin_boys():
    for T in (0.7, 3.0, 12.0, 45.0):
        F = oracle.boys(8, T)
        if abs(F[0] - 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))) > 1e-14:
            return False
        for m in (3, 8):
            ref = integrate.quad(lambda t: t ** (2 * m) * math.exp(-T * t * t), 0.0, 1.0, epsabs=0.0,
                                 epsrel=1e-13)[0]
            if abs(F[m] - ref) > 1e-13 * ref:
                return False
    return True


def pin_norm():
    z = np.array([3.1, 0.9, 0.25])
    s = dict(natom=1, xyz=np.zeros((1, 3)), shell_atom=np.zeros(1, np.int32), shell_l=np.array([2], np.int32),
             shell_nprim=np.array([3], np.int32), exps=z, coefs=np.array([0.3, 0.6, 0.4]))
    c = oracle.normalised_coefs(s)
    tot = 0.0
    for k in range(3):
        for j in range(3):
            zz = z[k] + z[j]
            ix = integrate.quad(lambda x: x ** 4 * math.exp(-zz * x * x), -np.inf, np.inf, epsabs=0, epsrel=1e-13)[0]
            iy = integrate.quad(lambda x: math.exp(-zz * x * x), -np.inf, np.inf, epsabs=0, epsrel=1e-13)[0]
            tot += c[k] * c[j] * ix * iy * iy
    if abs(tot - 1.0) > 1e-11:
        return False
    # the coefficients multiply unit-norm primitives: c_k / d_k = N_c N_k with
    # 1 / N_k^2 the primitive's own norm, so c_k^2 / d_k^2 * norm_k is one constant
    d = s["coefs"]
    r = []
    for k in range(3):
        ix = integrate.quad(lambda x: x ** 4 * math.exp(-2 * z[k] * x * x), -np.inf, np.inf, epsabs=0, epsrel=1e-13)[0]
        iy = integrate.quad(lambda x: math.exp(-2 * z[k] * x * x), -np.inf, np.inf, epsabs=0, epsrel=1e-13)[0]
        r.append((c[k] / d[k]) ** 2 * ix * iy * iy)
    return max(r) - min(r) <= 1e-11 * max(r)


def pin_ssss():
    cen = np.array([[0.0, 0.1, 0.2], [0.9, -0.3, 0.4], [-0.5, 1.1, 0.0], [0.3, 0.8, -0.9]])
    z = np.array([1.3, 0.4, 2.2, 0.7])
    s = _mini_system([0, 0, 0, 0], cen, z)
    c = oracle.normalised_coefs(s)
    p, q = z[0] + z[1], z[2] + z[3]
    P = (z[0] * cen[0] + z[1] * cen[1]) / p
    Q = (z[2] * cen[2] + z[3] * cen[3]) / q
    kab = math.exp(-z[0] * z[1] / p * np.sum((cen[0] - cen[1]) ** 2))
    kcd = math.exp(-z[2] * z[3] / q * np.sum((cen[2] - cen[3]) ** 2))
    rho = p * q / (p + q)
    T = rho * np.sum((P - Q) ** 2)
    for w in (0.0, 0.3):
        th2 = 1.0 if w == 0 else w * w / (w * w + rho)
        Tw = T * th2
        f0 = 0.5 * math.sqrt(math.pi / Tw) * math.erf(math.sqrt(Tw))
        ref = np.prod(c) * 2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * kab * kcd * math.sqrt(th2) * f0
        if abs(oracle.shell_eri(s, 0, 1, 2, 3, omega=w)[0, 0, 0, 0] - ref) > 1e-13 * abs(ref):
            return False
    return True


def pin_quadrature():
    ls = (1, 1, 1, 0)
    cen = np.array([[0.0, 0.2, -0.1], [1.1, -0.4, 0.3], [-0.6, 0.9, 0.5], [0.4, -1.0, 0.8]])
    z = np.array([0.8, 1.9, 0.6, 1.2])
    s = _mini_system(list(ls), cen, z)
    c = np.prod(oracle.normalised_coefs(s))
    comps = [_cart(l) for l in ls]
    for w in (0.0, 0.3):
        got = oracle.shell_eri(s, 0, 1, 2, 3, omega=w)
        for ii in [(0, 0, 0, 0), (1, 2, 0, 0), (2, 1, 1, 0), (0, 2, 2, 0)]:
            prims = [(comps[k][ii[k]], cen[k], z[k]) for k in range(4)]
            ref = c * geminal_eri(prims, 0.0, math.inf if w == 0 else w)
            if abs(got[ii] - ref) > 1e-11 * np.abs(got).max():
                return False
    return True


def _small():
    return synth.molecule(21, 1, 2)


def pin_fd():
    s = _small()
    g, _, _ = oracle.grad2e(s)
    h = 1e-4
    for atom, i in [(0, 0), (1, 1), (2, 2)]:
        xp = s["xyz"].copy()
        xp[atom, i] += h
        xm = s["xyz"].copy()
        xm[atom, i] -= h
        ep = oracle.grad2e(s, xyz=xp, want_grad=False, want_energy=True)[1]
        em = oracle.grad2e(s, xyz=xm, want_grad=False, want_energy=True)[1]
        if abs((ep - em) / (2 * h) - g[atom, i]) > 1e-7:
            return False
    return True


def pin_canonical():
    s = _small()
    a, x = s["pairs"][0][0], s["pairs"][-1][0]
    pairs = [(a, x, 0.7, 0.4, 0.9, 0.3)]
    gp, _, _ = oracle.grad2e(s, pairs=pairs, mode="plain")
    gc, _, _ = oracle.grad2e(s, pairs=pairs, mode="canonical")
    return np.abs(gp - gc).max() <= 1e-12 * max(1.0, np.abs(gp).max())


def pin_gamma():
    """Eq. gamma's Gamma and Gamma^lr as 4-index tensors against the pairs
    (R,R; 2, -a, -b) + (D,P; 1/2, -a/4, -b/4), on a 2-atom s,p / s basis."""
    s = dict(natom=2, xyz=np.array([[0.0, 0.0, 0.0], [0.4, -0.9, 1.2]]), shell_atom=np.array([0, 0, 1], np.int32),
             shell_l=np.array([0, 1, 0], np.int32), shell_nprim=np.array([1, 1, 1], np.int32),
             exps=np.array([1.1, 0.7, 0.5]), coefs=np.ones(3))
    nbf, off = 5, [0, 1, 4, 5]
    rng = np.random.default_rng(11)
    Cm = rng.normal(0, 0.3, size=(nbf, 2))
    P = Cm @ Cm.T
    Pd = 0.3 * P + rng.normal(0, 0.05, size=(nbf, nbf))
    Pd = Pd + Pd.T
    R = rng.normal(size=(nbf, nbf)) / nbf
    D = P + 2 * Pd
    al, be, w = 0.157706, 1 - 0.157706, 0.3
    G = (2 * np.einsum("nm,ls->mnls", R, R) - al * np.einsum("sm,ln->mnls", R, R)
         + 0.5 * (np.einsum("mn,ls->mnls", D, P) - al / 2 * np.einsum("ms,ln->mnls", D, P)))
    Glr = -be * np.einsum("sm,ln->mnls", R, R) - be / 4 * np.einsum("ms,ln->mnls", D, P)
    g = np.zeros((2, 3))
    for a in range(3):
        for b in range(3):
            for c in range(3):
                for d in range(3):
                    sl = tuple(slice(off[x], off[x + 1]) for x in (a, b, c, d))
                    gg = (np.einsum("xiabcd,abcd->xi", oracle.shell_eri_deriv(s, a, b, c, d), G[sl]) +
                          np.einsum("xiabcd,abcd->xi", oracle.shell_eri_deriv(s, a, b, c, d, omega=w), Glr[sl]))
                    for X, sh in enumerate((a, b, c, d)):
                        g[s["shell_atom"][sh]] += gg[X]
    g2, _, _ = oracle.grad2e(s, pairs=[(R, R, 2.0, -al, -be, w), (D, P, 0.5, -al / 4, -be / 4, w)])
    return np.abs(g2 - g).max() <= 1e-12 * np.abs(g).max()


def pin_contraction():
    shells = random_shells((1, 1, 1, 0), (2, 3, 2, 2), seed=77)
    s = oracle_system(shells)
    for w in (0.0, 0.3):
        ref = contracted_reference(shells, w)
        got = oracle.shell_eri(s, 0, 1, 2, 3, omega=w)
        if np.abs(got - ref).max() > 1e-11 * np.abs(ref).max():
            return False
    return True


def pin_fock():
    s = synth.molecule(31, 1, 2)
    n = s["pairs"][0][0].shape[0]
    rng = np.random.default_rng(5)
    A, B = rng.normal(size=(n, n)) / n, rng.normal(size=(n, n)) / n
    F = oracle.fock2e(s, [(B, 0.4, 1.0, 0.6, 0.3)])
    e = oracle.grad2e(s, pairs=[(A, B, 0.4, 1.0, 0.6, 0.3)], want_grad=False, want_energy=True)[1]
    return abs(float(np.sum(A * F)) - e) <= 1e-12 * abs(e)


def pin_translation():
    """The integrals depend on relative positions only: a rigid shift of
    every centre by tens of bohr leaves the c1 gradient unchanged."""
    s = synth.config(0)
    g0 = oracle.grad2e(s, tau=0.0)[0]
    g1 = oracle.grad2e(s, tau=0.0, xyz=s["xyz"] + np.array([40.0, 35.0, -30.0]))[0]
    return float(np.abs(g1 - g0).max()) <= 1e-12 * float(np.abs(g0).max())


PINS = {"translation": pin_translation, "gamma": pin_gamma, "contraction": pin_contraction, "fock": pin_fock, "boys": pin_boys, "norm": pin_norm, "ssss": pin_ssss, "quadrature": pin_quadrature, "fd": pin_fd,
        "canonical": pin_canonical}


def test_real_oracle_passes_every_pin():
    for name, pin in PINS.items():
        assert pin(), name


@pytest.fixture(scope="module")
def variants(tmp_path_factory):
    d = tmp_path_factory.mktemp("oracle_mutants")
    src = os.path.join(os.path.dirname(oracle.__file__), "tdgrad_oracle.c")
    out = {}
    for k in MUTATIONS:
        path = str(d / ("mutant%d.so" % k))
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-D_GNU_SOURCE",
                               "-DOR_MUTATION=%d" % k, src, "-o", path, "-lm"])
        out[k] = path
    return out


@pytest.mark.parametrize("k", sorted(MUTATIONS))
def test_planted_mistake_is_caught(k, variants, monkeypatch):
    what, pin = MUTATIONS[k]
    monkeypatch.setattr(oracle, "_lib", oracle._configure(ctypes.CDLL(variants[k])))
    assert not PINS[pin](), "mutation %d (%s) passed the %s pin" % (k, what, pin)
