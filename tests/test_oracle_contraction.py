"""Pin of the oracle's contraction over primitives (Sec. II.C, eq. cartG: a
contracted Cartesian Gaussian is a fixed linear combination of primitives
sharing one centre and one angular part).

Every shell here carries two or three primitives, so a mistake in the
primitive-quartet weights (a coefficient taken at the wrong primitive, a
factor dropped, raw instead of normalised coefficients) changes the result.
The reference value of a contracted integral is computed in this file alone:

  (ab|cd) = sum_{k_a k_b k_c k_d} w_a[k_a] w_b[k_b] w_c[k_c] w_d[k_d] [ab|cd]_prim,

with
  * [ab|cd]_prim the primitive integral of unnormalised Cartesian Gaussians
    by Gaussian-geminal quadrature, 1/r = (2/sqrt(pi)) int_0^inf e^{-u^2 r^2} du
    (erf(omega r)/r: u up to omega), the geminal integral factorised per axis
    and each axis done exactly by 2-D Gauss-Hermite quadrature;
  * w[k] = d_k N_k N_c, where N_k makes the x^l primitive unit-norm and N_c the
    contracted x^l function unit-norm, both from 1-D Gauss-Hermite norms
    (not from the oracle's normalisation routine);
  * derivatives by the chain rule on a primitive (Sec. II.C, eq. deriv):
    d/dA_i [(x_i - A_i)^n e^{-z (x_i - A_i)^2}] = 2 z (x_i - A_i)^{n+1} e - n (x_i - A_i)^{n-1} e,
    i.e. d/dA_i [ab|cd] = 2 z_a [a+1_i b|cd] - a_i [a-1_i b|cd] per primitive.
"""
import math

import numpy as np
import pytest

import oracle

GH_X, GH_W = np.polynomial.hermite.hermgauss(16)
_Z1, _Z2 = np.meshgrid(GH_X, GH_X, indexing="ij")
_Z1, _Z2 = _Z1.ravel(), _Z2.ravel()
_W2 = np.outer(GH_W, GH_W).ravel()


def _gl_panels(a, b, npanel, nnode):
    x, w = np.polynomial.legendre.leggauss(nnode)
    edges = np.linspace(a, b, npanel + 1)
    xs = [0.5 * (hi - lo) * x + 0.5 * (hi + lo) for lo, hi in zip(edges[:-1], edges[1:])]
    ws = [0.5 * (hi - lo) * w for lo, hi in zip(edges[:-1], edges[1:])]
    return np.concatenate(xs), np.concatenate(ws)


def u_nodes(omega):
    """Nodes and weights of the u integral: [0, inf) for 1/r, [0, omega] for
    erf(omega r)/r."""
    if omega <= 0.0:
        s, w = _gl_panels(0.0, 1.0, 24, 40)
        return s / (1.0 - s), w / (1.0 - s) ** 2
    return _gl_panels(0.0, omega, 8, 40)


def axis_table(u, z, X, pmax):
    """T[n, i, j, k, l] = int int (x1-A)^i (x1-B)^j (x2-C)^k (x2-D)^l
    exp(-za(x1-A)^2 - zb(x1-B)^2 - zc(x2-C)^2 - zd(x2-D)^2 - u_n^2 (x1-x2)^2)
    dx1 dx2 along one axis, for i <= pmax[0] ... l <= pmax[3]."""
    za, zb, zc, zd = z
    A, B, C, D = X
    w = u * u
    p, q = za + zb, zc + zd
    b1, b2 = za * A + zb * B, zc * C + zd * D
    det = (p + w) * (q + w) - w * w
    mu1 = ((q + w) * b1 + w * b2) / det
    mu2 = (w * b1 + (p + w) * b2) / det
    c0 = za * A * A + zb * B * B + zc * C * C + zd * D * D - (b1 * mu1 + b2 * mu2)
    # M = L L^T, x = mu + L^{-T} y
    L11 = np.sqrt(p + w)
    L21 = -w / L11
    L22 = np.sqrt(q + w - L21 * L21)
    x1 = mu1[:, None] + _Z1[None, :] / L11[:, None] - (L21 / (L11 * L22))[:, None] * _Z2[None, :]
    x2 = mu2[:, None] + _Z2[None, :] / L22[:, None]
    pa = np.stack([(x1 - A) ** n for n in range(pmax[0] + 1)], -1)
    pb = np.stack([(x1 - B) ** n for n in range(pmax[1] + 1)], -1)
    pc = np.stack([(x2 - C) ** n for n in range(pmax[2] + 1)], -1)
    pd = np.stack([(x2 - D) ** n for n in range(pmax[3] + 1)], -1)
    left = (pa[:, :, :, None] * pb[:, :, None, :]).reshape(len(u), len(_W2), -1)
    right = (pc[:, :, :, None] * pd[:, :, None, :]).reshape(len(u), len(_W2), -1)
    pref = np.exp(-c0) / (L11 * L22)
    t = np.matmul(np.transpose(left * _W2[None, :, None], (0, 2, 1)), right) * pref[:, None, None]
    return t.reshape(len(u), pmax[0] + 1, pmax[1] + 1, pmax[2] + 1, pmax[3] + 1)


def cart(l):
    return [(lx, ly, l - lx - ly) for lx in range(l, -1, -1) for ly in range(l - lx, -1, -1)]


def _moment(n, z):
    """int x^n e^{-z x^2} dx over the real line by Gauss-Hermite (exact)."""
    if n % 2:
        return 0.0
    return float(np.sum(GH_W * (GH_X / math.sqrt(z)) ** n)) / math.sqrt(z)


def effective_coefs(l, zetas, d):
    """w_k = d_k N_k N_c for the x^l component (unit-norm primitives, unit-norm
    contracted function)."""
    nk = np.array([1.0 / math.sqrt(_moment(2 * l, 2 * zk) * _moment(0, 2 * zk) ** 2) for zk in zetas])
    s = 0.0
    for k in range(len(zetas)):
        for j in range(len(zetas)):
            zz = zetas[k] + zetas[j]
            s += d[k] * d[j] * nk[k] * nk[j] * _moment(2 * l, zz) * _moment(0, zz) ** 2
    return np.asarray(d) * nk / math.sqrt(s)


def contracted_reference(shells, omega, deriv=False):
    """Contracted integrals of shells = [(l, centre, zetas, coefs)] * 4 by
    quadrature: array [na, nb, nc, nd], or with deriv [4, 3, na, nb, nc, nd]
    (d/dA_i ... d/dD_i)."""
    u, uw = u_nodes(omega)
    ls = [s[0] for s in shells]
    comps = [cart(l) for l in ls]
    dims = [len(c) for c in comps]
    pmax = [l + (1 if deriv else 0) for l in ls]
    wts = [effective_coefs(s[0], s[2], s[3]) for s in shells]
    cen = [np.asarray(s[1], dtype=float) for s in shells]
    out = np.zeros(([4, 3] if deriv else []) + dims)
    idx = list(np.ndindex(*dims))
    for ka in range(len(shells[0][2])):
        for kb in range(len(shells[1][2])):
            for kc in range(len(shells[2][2])):
                for kd in range(len(shells[3][2])):
                    ks = (ka, kb, kc, kd)
                    z = [shells[x][2][ks[x]] for x in range(4)]
                    w = 2.0 / math.sqrt(math.pi) * wts[0][ka] * wts[1][kb] * wts[2][kc] * wts[3][kd]
                    tab = [axis_table(u, z, [cen[x][ax] for x in range(4)], pmax) for ax in range(3)]

                    def prim(pw):  # pw[x][ax] powers; None where a power is negative
                        f = uw.copy()
                        for ax in range(3):
                            f = f * tab[ax][:, pw[0][ax], pw[1][ax], pw[2][ax], pw[3][ax]]
                        return float(np.sum(f))

                    for ii in idx:
                        pw = [list(comps[x][ii[x]]) for x in range(4)]
                        if not deriv:
                            out[ii] += w * prim(pw)
                            continue
                        for X in range(4):
                            for i in range(3):
                                up = [list(v) for v in pw]
                                up[X][i] += 1
                                val = 2.0 * z[X] * prim(up)
                                n = pw[X][i]
                                if n > 0:
                                    dn = [list(v) for v in pw]
                                    dn[X][i] -= 1
                                    val -= n * prim(dn)
                                out[(X, i) + ii] += w * val
    return out


def oracle_system(shells):
    """The same four shells as an oracle basis: one shell per atom."""
    return dict(natom=4, xyz=np.array([s[1] for s in shells], dtype=float),
                shell_atom=np.arange(4, dtype=np.int32), shell_l=np.array([s[0] for s in shells], dtype=np.int32),
                shell_nprim=np.array([len(s[2]) for s in shells], dtype=np.int32),
                exps=np.concatenate([np.asarray(s[2], dtype=float) for s in shells]),
                coefs=np.concatenate([np.asarray(s[3], dtype=float) for s in shells]))


def random_shells(ls, nprims, seed):
    rng = np.random.default_rng(seed)
    cen = rng.normal(size=(4, 3)) * 1.1
    shells = []
    for x in range(4):
        z = np.sort(np.exp(rng.uniform(np.log(0.2), np.log(5.0), size=nprims[x])))[::-1]
        d = rng.uniform(0.2, 1.0, size=nprims[x])
        shells.append((ls[x], cen[x], z, d))
    return shells


CASES = [((1, 0, 0, 0), (3, 2, 2, 2)), ((1, 1, 1, 0), (2, 3, 2, 2)), ((2, 0, 1, 1), (2, 2, 3, 2)),
         ((2, 1, 2, 0), (2, 2, 2, 3)), ((2, 2, 2, 1), (2, 2, 2, 2))]


@pytest.mark.parametrize("ls,nprims", CASES)
@pytest.mark.parametrize("omega", [0.0, 0.3])
def test_contracted_eri_vs_quadrature(ls, nprims, omega):
    shells = random_shells(ls, nprims, seed=1000 + 10 * sum(ls) + int(10 * omega))
    got = oracle.shell_eri(oracle_system(shells), 0, 1, 2, 3, omega=omega)
    ref = contracted_reference(shells, omega)
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("ls,nprims", [((1, 1, 1, 0), (2, 3, 2, 2)), ((2, 1, 2, 0), (2, 2, 2, 3))])
@pytest.mark.parametrize("omega", [0.0, 0.3])
def test_contracted_eri_derivatives_vs_quadrature(ls, nprims, omega):
    shells = random_shells(ls, nprims, seed=2000 + 10 * sum(ls) + int(10 * omega))
    got = oracle.shell_eri_deriv(oracle_system(shells), 0, 1, 2, 3, omega=omega)
    ref = contracted_reference(shells, omega, deriv=True)
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


def test_quadrature_reference_reduces_to_one_primitive():
    """With one primitive per shell and d = 1 the reference is N_a N_b N_c N_d
    times one primitive integral, and the closed form [ss|ss] holds."""
    cen = np.array([[0.0, 0.1, 0.2], [0.9, -0.3, 0.4], [-0.5, 1.1, 0.0], [0.3, 0.8, -0.9]])
    z = [1.3, 0.4, 2.2, 0.7]
    shells = [(0, cen[x], np.array([z[x]]), np.array([1.0])) for x in range(4)]
    ref = contracted_reference(shells, 0.0)[0, 0, 0, 0]
    p, q = z[0] + z[1], z[2] + z[3]
    P = (z[0] * cen[0] + z[1] * cen[1]) / p
    Q = (z[2] * cen[2] + z[3] * cen[3]) / q
    kab = math.exp(-z[0] * z[1] / p * np.sum((cen[0] - cen[1]) ** 2))
    kcd = math.exp(-z[2] * z[3] / q * np.sum((cen[2] - cen[3]) ** 2))
    rho = p * q / (p + q)
    T = rho * np.sum((P - Q) ** 2)
    f0 = 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
    norm = np.prod([(2 * zz / math.pi) ** 0.75 for zz in z])
    closed = norm * 2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * kab * kcd * f0
    assert ref == pytest.approx(closed, rel=1e-12)
