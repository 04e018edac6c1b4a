"""Pins of the oracle's Cartesian-to-spherical transform (Sec. II.C: a shell's
2l+1 spherical functions are a spherical transformation of its Cartesian
ones), which the spherical-shell parity tests use.

Independent routes:
  * orthonormality: with the overlap of the x^l-normalised Cartesian
    components of a d shell (a closed form: every component shares the radial
    part, so <c|c'> is a product of 1-D Gaussian moments (n-1)!! over the
    moment of xx), T^T S T is the 5 x 5 identity;
  * purity: every spherical d function is orthogonal to the s-type
    combination r^2 = xx + yy + zz, so the five span the l = 2 space;
  * the energy identity: the energy of spherical-basis densities with the
    integrals transformed to the spherical basis (T on all four indices of the
    shell-quartet integral tensor) equals the oracle's canonical energy of the
    Cartesian densities T A T^T, T B T^T (which is what the library computes
    from; the gradient follows by linearity);
  * a sign or factor planted in a copy of T fails the first two pins.
"""
import numpy as np
import pytest

import oracle
from paper_2407_16586_gb300 import synth

# Cartesian exponents of the d components, order xx xy xz yy yz zz
D_EXP = [(2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2)]


def _moment(n):
    """Integral of x^n exp(-x^2) relative to that of x^0: (n-1)!! / 2^(n/2), 0 for odd n."""
    if n % 2:
        return 0.0
    r = 1.0
    for k in range(1, n, 2):
        r *= k / 2.0
    return r


def _d_overlap():
    """Overlap of the six x^l-normalised d components (xx has norm 1)."""
    S = np.zeros((6, 6))
    for i, a in enumerate(D_EXP):
        for j, b in enumerate(D_EXP):
            S[i, j] = np.prod([_moment(a[k] + b[k]) for k in range(3)])
    return S / S[0, 0]


def _d_block(T, s):
    ls = [int(l) for l in s["shell_l"]]
    i = j = 0
    for l in ls:
        if l == 2:
            return T[i:i + 6, j:j + 5]
        i += (l + 1) * (l + 2) // 2
        j += 2 * l + 1
    raise AssertionError("no d shell")


def _check(d):
    S = _d_overlap()
    orth = np.abs(d.T @ S @ d - np.eye(5)).max()
    r2 = np.array([1.0, 0, 0, 1.0, 0, 1.0])
    pure = np.abs(r2 @ S @ d).max()
    return orth, pure


def test_closed_form_overlap():
    S = _d_overlap()
    # <xx|xx> = 1, <xx|yy> = 1/3, <xy|xy> = 1/3, odd products vanish
    assert S[0, 0] == 1.0 and S[0, 3] == pytest.approx(1 / 3) and S[1, 1] == pytest.approx(1 / 3)
    assert S[0, 1] == 0.0 and S[1, 2] == 0.0


def test_d_functions_are_orthonormal_and_pure():
    s = synth.molecule(32, 1, 1)
    T = oracle.sph_transform(s)
    assert T.shape == (s["nbf"], sum(2 * int(l) + 1 for l in s["shell_l"]))
    orth, pure = _check(_d_block(T, s))
    assert orth <= 1e-15 and pure <= 1e-15


def test_s_and_p_blocks_are_the_identity():
    s = synth.molecule(32, 1, 1)
    T = oracle.sph_transform(s)
    i = j = 0
    for l in [int(x) for x in s["shell_l"]]:
        nc, ns = (l + 1) * (l + 2) // 2, 2 * l + 1
        if l < 2:
            assert np.array_equal(T[i:i + nc, j:j + ns], np.eye(nc))
        # nothing outside the diagonal blocks
        assert not np.any(T[i:i + nc, :j]) and not np.any(T[i:i + nc, j + ns:])
        i += nc
        j += ns


@pytest.mark.parametrize("mutant", ["sign", "factor", "swap"])
def test_planted_mistakes_fail_the_pins(mutant):
    s = synth.molecule(32, 1, 1)
    d = _d_block(oracle.sph_transform(s), s).copy()
    if mutant == "sign":      # (x^2 + y^2) instead of (x^2 - y^2)
        d[3, 4] = -d[3, 4]
    elif mutant == "factor":  # d0 as zz - (xx + yy) without the 1/2
        d[0, 2] = d[3, 2] = -1.0
    else:                     # m = +1 written with yz instead of xz (a copy of m = -1)
        d[2, 3], d[4, 3] = 0.0, d[2, 3]
    orth, pure = _check(d)
    assert max(orth, pure) > 1e-3


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


def test_energy_of_spherical_integrals_equals_the_transformed_densities():
    s = synth.molecule(32, 1, 1)
    T = oracle.sph_transform(s)
    nsph = T.shape[1]
    rng = np.random.default_rng(5)
    A, B = rng.normal(size=(nsph, nsph)) / nsph, rng.normal(size=(nsph, nsph)) / nsph
    eri, erl = _full_eri(s), _full_eri(s, 0.3)
    es = np.einsum("pi,qj,rk,sl,pqrs->ijkl", T, T, T, T, eri, optimize=True)
    el = np.einsum("pi,qj,rk,sl,pqrs->ijkl", T, T, T, T, erl, optimize=True)
    cJ, cK, cKlr = 0.7, -0.3, 0.9
    ref = (cJ * np.einsum("ijkl,ij,kl->", es, A, B) + cK * np.einsum("ijkl,ik,jl->", es, A, B)
           + cKlr * np.einsum("ijkl,ik,jl->", el, A, B))
    Ac, Bc = T @ A @ T.T, T @ B @ T.T
    e = oracle.grad2e(s, pairs=[(Ac, Bc, cJ, cK, cKlr, 0.3)], want_grad=False, want_energy=True)[1]
    assert e == pytest.approx(ref, rel=1e-12, abs=1e-13)
