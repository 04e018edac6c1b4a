"""Spherical shells (tg_grad2e_sph): the gradient of the integrals over
spherical functions, computed by the library as the Cartesian gradient of
T A T^T, against the oracle's Cartesian gradient of the densities that the
oracle's own transform (pinned in test_oracle_spherical.py) produces.

Tolerances: fp64 1e-10 Ha/bohr per component (the plain path's bound); the
mixed route within its mixed_tol of the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2407_16586_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def tg():
    from paper_2407_16586_gb300 import build
    build.build()
    import paper_2407_16586_gb300 as m
    return m


def _pairs(nsph, seed):
    rng = np.random.default_rng(seed)
    c = rng.normal(0.0, 0.3, size=(nsph, 5))
    P = c @ c.T
    X = rng.normal(size=(nsph, nsph))
    X /= np.linalg.norm(X)
    Q = rng.normal(size=(nsph, nsph)) / nsph
    return [(P, P, 1.0, 0.157706, 0.0, 0.0), (X, X, 0.0, 0.0, 1.0, 0.3), (Q, P, 0.5, -0.25, -0.75, 0.3)]


def _cart(T, pairs):
    return [(T @ a @ T.T, T @ b @ T.T, cj, ck, cl, om) for (a, b, cj, ck, cl, om) in pairs]


@pytest.mark.parametrize("system", ["c1", "chain"])
def test_spherical_gradient_against_the_oracle(tg, system):
    s = synth.config(0) if system == "c1" else synth.molecule(31, 1, 2)
    T = oracle.sph_transform(s)
    b = tg.Basis(s)
    assert b.nsph == T.shape[1] and b.nbf == T.shape[0]
    pairs = _pairs(b.nsph, 7)
    ref, _, nq = oracle.grad2e(s, pairs=_cart(T, pairs), tau=0.0)
    g, st = b.grad2e(pairs, screen_tol=0.0, spherical=True)
    assert st["quartets"] == nq
    assert np.abs(g - ref).max() <= TOL
    gm, stm = b.grad2e(pairs, screen_tol=0.0, spherical=True, precision=tg.TG_MIXED_BOUND, mixed_tol=1e-6)
    assert np.abs(gm - ref).max() <= 1e-6


def test_spherical_device_pointers_match_host(tg):
    import torch
    s = synth.config(0)
    b = tg.Basis(s)
    pairs = _pairs(b.nsph, 8)
    gh, _ = b.grad2e(pairs, screen_tol=1e-12, spherical=True)
    dev = [(torch.from_numpy(a).cuda(), torch.from_numpy(c).cuda(), cj, ck, cl, om)
           for (a, c, cj, ck, cl, om) in pairs]
    gd, _ = b.grad2e(dev, screen_tol=1e-12, spherical=True)
    torch.cuda.synchronize()
    assert np.array_equal(gd.cpu().numpy(), gh)
