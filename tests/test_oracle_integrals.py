"""Pins for the oracle's contracted ERIs over Cartesian Gaussians (Sec. II.C,
eq. cartG) for the 1/r operator and the erf(omega r)/r operator of
eq. lreri_k.

The independent route used here never touches a Boys function or a
recursion: the operator is written as a Gaussian-geminal integral
  1/r = (2/sqrt(pi)) int_0^inf exp(-u^2 r^2) du,
  erf(omega r)/r = (2/sqrt(pi)) int_0^omega exp(-u^2 r^2) du,
the geminal integral factorises into x, y, z, and each factor is a 2-D
polynomial-times-Gaussian integral done exactly by Gauss-Hermite quadrature.
The u integral uses Gauss-Legendre panels."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle

GH_X, GH_W = np.polynomial.hermite.hermgauss(14)


def _geminal_1d(u2, prims, axis):
    """prod over one Cartesian axis of the 2-D integral, vectorised over u^2."""
    (la, A, za), (lb, B, zb), (lc, C, zc), (ld, D, zd) = prims
    Ax, Bx, Cx, Dx = A[axis], B[axis], C[axis], D[axis]
    p, q = za + zb, zc + zd
    out = np.empty_like(u2)
    for n, w in enumerate(u2):
        M = np.array([[p + w, -w], [-w, q + w]])
        bvec = np.array([za * Ax + zb * Bx, zc * Cx + zd * Dx])
        const = za * Ax ** 2 + zb * Bx ** 2 + zc * Cx ** 2 + zd * Dx ** 2
        mu = np.linalg.solve(M, bvec)
        c0 = const - bvec @ mu
        L = np.linalg.cholesky(M)
        LiT = np.linalg.inv(L).T
        z1, z2 = np.meshgrid(GH_X, GH_X, indexing="ij")
        x1 = mu[0] + LiT[0, 0] * z1 + LiT[0, 1] * z2
        x2 = mu[1] + LiT[1, 0] * z1 + LiT[1, 1] * z2
        poly = (x1 - Ax) ** la[axis] * (x1 - Bx) ** lb[axis] * (x2 - Cx) ** lc[axis] * (x2 - Dx) ** ld[axis]
        out[n] = math.exp(-c0) / np.prod(np.diag(L)) * np.sum(np.outer(GH_W, GH_W) * poly)
    return out


def _gl_panels(a, b, npanel, nnode):
    x, w = np.polynomial.legendre.leggauss(nnode)
    edges = np.linspace(a, b, npanel + 1)
    xs, ws = [], []
    for lo, hi in zip(edges[:-1], edges[1:]):
        xs.append(0.5 * (hi - lo) * x + 0.5 * (hi + lo))
        ws.append(0.5 * (hi - lo) * w)
    return np.concatenate(xs), np.concatenate(ws)


def geminal_eri(prims, lo=0.0, hi=math.inf):
    """(2/sqrt(pi)) int_lo^hi prod_axis I_axis(u) du for one primitive quartet of
    unnormalised Cartesian Gaussians; prims = [(lxyz, centre, zeta)] * 4."""
    if math.isinf(hi):
        # u = lo + s/(1-s), s in [0, 1)
        s, w = _gl_panels(0.0, 1.0, 24, 40)
        u = lo + s / (1.0 - s)
        w = w / (1.0 - s) ** 2
    else:
        u, w = _gl_panels(lo, hi, 8, 40)
    u2 = u * u
    f = _geminal_1d(u2, prims, 0) * _geminal_1d(u2, prims, 1) * _geminal_1d(u2, prims, 2)
    return 2.0 / math.sqrt(math.pi) * np.sum(w * f)


def _cart(l):
    return [(lx, ly, l - lx - ly) for lx in range(l, -1, -1) for ly in range(l - lx, -1, -1)]


def _mini_system(ls, centres, zetas):
    return dict(natom=4, xyz=np.array(centres, dtype=float), shell_atom=np.arange(4, dtype=np.int32),
                shell_l=np.array(ls, dtype=np.int32), shell_nprim=np.ones(4, dtype=np.int32),
                exps=np.array(zetas, dtype=float), coefs=np.ones(4))


def test_normalisation_unit_self_overlap(c1):
    cn = oracle.normalised_coefs(c1)
    off = 0
    for l, K in zip(c1["shell_l"], c1["shell_nprim"]):
        ex = c1["exps"][off:off + K]
        c = cn[off:off + K]
        tot = 0.0
        for k in range(K):
            for j in range(K):
                z = ex[k] + ex[j]
                ix = integrate.quad(lambda x: x ** (2 * l) * math.exp(-z * x * x), -np.inf, np.inf,
                                    epsabs=0, epsrel=1e-13)[0]
                iy = integrate.quad(lambda x: math.exp(-z * x * x), -np.inf, np.inf, epsabs=0, epsrel=1e-13)[0]
                tot += c[k] * c[j] * ix * iy * iy
        assert tot == pytest.approx(1.0, rel=1e-11)
        off += K


def test_normalisation_primitives_unit_norm(c1):
    """Contraction coefficients multiply unit-norm primitives: c_k / d_k =
    N_c N_k for one N_c per shell, with 1 / N_k^2 the primitive's norm."""
    cn = oracle.normalised_coefs(c1)
    off = 0
    for l, K in zip(c1["shell_l"], c1["shell_nprim"]):
        r = []
        for k in range(K):
            z = c1["exps"][off + k]
            ix = integrate.quad(lambda x: x ** (2 * l) * math.exp(-2 * z * x * x), -np.inf, np.inf,
                                epsabs=0, epsrel=1e-13)[0]
            iy = integrate.quad(lambda x: math.exp(-2 * z * x * x), -np.inf, np.inf, epsabs=0, epsrel=1e-13)[0]
            r.append((cn[off + k] / c1["coefs"][off + k]) ** 2 * ix * iy * iy)
        assert max(r) - min(r) <= 1e-11 * max(r)
        off += K


def test_ssss_closed_form():
    rng = np.random.default_rng(5)
    for _ in range(6):
        cen = rng.normal(size=(4, 3)) * 1.5
        z = np.exp(rng.uniform(np.log(0.1), np.log(50.0), size=4))
        s = _mini_system([0, 0, 0, 0], cen, z)
        c = oracle.normalised_coefs(s)
        p, q = z[0] + z[1], z[2] + z[3]
        P = (z[0] * cen[0] + z[1] * cen[1]) / p
        Q = (z[2] * cen[2] + z[3] * cen[3]) / q
        kab = math.exp(-z[0] * z[1] / p * np.sum((cen[0] - cen[1]) ** 2))
        kcd = math.exp(-z[2] * z[3] / q * np.sum((cen[2] - cen[3]) ** 2))
        rho = p * q / (p + q)
        T = rho * np.sum((P - Q) ** 2)
        f0 = 1.0 if T == 0 else 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
        ref = np.prod(c) * 2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * kab * kcd * f0
        assert oracle.shell_eri(s, 0, 1, 2, 3)[0, 0, 0, 0] == pytest.approx(ref, rel=1e-13)
        # erf operator: rho -> rho w^2/(w^2+rho) in F_0 and in the sqrt(rho) prefactor
        w = 0.3
        th2 = w * w / (w * w + rho)
        Tw = T * th2
        f0w = 1.0 if Tw == 0 else 0.5 * math.sqrt(math.pi / Tw) * math.erf(math.sqrt(Tw))
        refw = np.prod(c) * 2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * kab * kcd * math.sqrt(th2) * f0w
        assert oracle.shell_eri(s, 0, 1, 2, 3, omega=w)[0, 0, 0, 0] == pytest.approx(refw, rel=1e-13)


CLASSES = [(1, 0, 0, 0), (1, 1, 0, 0), (1, 0, 1, 0), (1, 1, 1, 1), (2, 0, 0, 0), (2, 1, 1, 0),
           (2, 2, 1, 0), (0, 2, 1, 2), (2, 2, 2, 2)]


@pytest.mark.parametrize("ls", CLASSES)
@pytest.mark.parametrize("omega", [0.0, 0.3])
def test_primitive_eri_vs_geminal_quadrature(ls, omega):
    rng = np.random.default_rng(abs(hash((ls, omega))) % 2 ** 32)
    cen = rng.normal(size=(4, 3)) * 1.2
    z = np.exp(rng.uniform(np.log(0.15), np.log(6.0), size=4))
    s = _mini_system(list(ls), cen, z)
    got = oracle.shell_eri(s, 0, 1, 2, 3, omega=omega)
    c = np.prod(oracle.normalised_coefs(s))
    comps = [_cart(l) for l in ls]
    idx = list(np.ndindex(*got.shape))
    rng.shuffle(idx)
    for ii in idx[:12]:
        prims = [(comps[k][ii[k]], cen[k], z[k]) for k in range(4)]
        ref = c * geminal_eri(prims, 0.0, math.inf if omega == 0 else omega)
        scale = np.abs(got).max()
        assert abs(got[ii] - ref) <= 1e-11 * scale, (ii, got[ii], ref)


@pytest.mark.parametrize("ls", [(0, 0, 0, 0), (1, 0, 1, 0), (1, 1, 0, 0), (2, 1, 0, 0)])
def test_erfc_complement_vs_quadrature(ls):
    """full - erf = erfc(omega r)/r, computed independently as the geminal
    integral over u in [omega, inf)."""
    rng = np.random.default_rng(7 + sum(ls))
    cen = rng.normal(size=(4, 3)) * 1.2
    z = np.exp(rng.uniform(np.log(0.15), np.log(6.0), size=4))
    s = _mini_system(list(ls), cen, z)
    w = 0.3
    diff = oracle.shell_eri(s, 0, 1, 2, 3) - oracle.shell_eri(s, 0, 1, 2, 3, omega=w)
    c = np.prod(oracle.normalised_coefs(s))
    comps = [_cart(l) for l in ls]
    for ii in list(np.ndindex(*diff.shape))[:6]:
        prims = [(comps[k][ii[k]], cen[k], z[k]) for k in range(4)]
        ref = c * geminal_eri(prims, w, math.inf)
        assert abs(diff[ii] - ref) <= 1e-11 * np.abs(diff).max()


def test_omega_limits(c1):
    rng = np.random.default_rng(3)
    ns = len(c1["shell_l"])
    for _ in range(6):
        a, b, c, d = (int(x) for x in rng.integers(0, ns, 4))
        full = oracle.shell_eri(c1, a, b, c, d)
        big = oracle.shell_eri(c1, a, b, c, d, omega=1e8)
        inf = oracle.shell_eri(c1, a, b, c, d, omega=math.inf)
        small = oracle.shell_eri(c1, a, b, c, d, omega=1e-7)
        sc = np.abs(full).max()
        assert np.abs(big - full).max() <= 1e-13 * sc
        assert np.abs(inf - full).max() <= 1e-14 * sc
        assert np.abs(small).max() <= 1e-5 * sc


def test_permutational_symmetry(c1):
    rng = np.random.default_rng(11)
    ns = len(c1["shell_l"])
    for _ in range(8):
        a, b, c, d = (int(x) for x in rng.integers(0, ns, 4))
        x = oracle.shell_eri(c1, a, b, c, d, omega=0.3)
        sc = np.abs(x).max() + 1e-300
        np.testing.assert_allclose(oracle.shell_eri(c1, b, a, c, d, omega=0.3), x.transpose(1, 0, 2, 3),
                                   atol=1e-13 * sc, rtol=0)
        np.testing.assert_allclose(oracle.shell_eri(c1, c, d, a, b, omega=0.3), x.transpose(2, 3, 0, 1),
                                   atol=1e-13 * sc, rtol=0)
        np.testing.assert_allclose(oracle.shell_eri(c1, a, b, d, c, omega=0.3), x.transpose(0, 1, 3, 2),
                                   atol=1e-13 * sc, rtol=0)


def test_schwarz_bounds_hold(c1):
    """Q bounds sqrt((mn|mn)); max(Q'_ab Q_cd, Q_ab Q'_cd) bounds every
    derivative integral of the quartet (Cauchy-Schwarz for a positive-definite
    kernel, Sec. II.E screening)."""
    Q, Qd = oracle.schwarz(c1)
    ns = len(c1["shell_l"])
    rng = np.random.default_rng(2)
    for _ in range(10):
        a, b = (int(x) for x in rng.integers(0, ns, 2))
        diag = oracle.shell_eri(c1, a, b, a, b)
        na, nb = diag.shape[:2]
        m = max(diag[i, j, i, j] for i in range(na) for j in range(nb))
        assert math.sqrt(m) <= Q[a, b] * (1 + 1e-12)
    for _ in range(10):
        a, b, c, d = (int(x) for x in rng.integers(0, ns, 4))
        D = oracle.shell_eri_deriv(c1, a, b, c, d)
        bound = max(Qd[a, b] * Q[c, d], Q[a, b] * Qd[c, d])
        assert np.abs(D).max() <= bound * (1 + 1e-12)
        Dw = oracle.shell_eri_deriv(c1, a, b, c, d, omega=0.3)
        assert np.abs(Dw).max() <= bound * (1 + 1e-12)
