"""Seeded synthetic inputs for the two-electron TDA gradient term.

This module only draws random numbers: geometries, a split-valence-like
Cartesian Gaussian basis, and density-like matrices.  It holds none of the
integral or gradient arithmetic, so both the CUDA path and the CPU oracle can
take their inputs from it without sharing any of the method.

Workloads (shaped like the paper's GFP / def2-SVP application, Sec. III, which
is not available here):

* ``c1``: 2 O + 4 H placed sequentially at 0.95-3.0 A distances; J(A,A)+K(A,A)
  full range with unit coefficients plus K_lr(X,X) at omega = 0.3 bohr^-1.
* ``c2``: 32-atom C/N/O/H chain (19 H), three density pairs
  [(P,P), (P_delta,P), (X,X)] with c_J = 1, c_K = 0.157706, c_K_lr = 1,
  omega = 0.3.
* ``c3``: 64 independent chain molecules of 20-120 atoms, same pairs.
* ``c4``: 300-atom compact core + water cluster.
* ``c5``: 1500-atom compact core + water shells.

Heavy atoms carry 3s2p1d contracted shells (exponents log-uniform in
[0.15, 2000]), H carries 2s1p (exponents in [0.1, 20]); 1-6 primitives per
shell, sorted descending, contraction coefficients U[0.2, 1.0] that multiply
normalised primitives.  One basis is drawn per element, as a basis-set
library would hold it.  Coordinates are returned in bohr.
"""
from __future__ import annotations

import numpy as np

BOHR_PER_ANG = 1.0 / 0.529177210903  # CODATA 2018

HEAVY_SHELLS = (0, 0, 0, 1, 1, 2)  # 3s2p1d
H_SHELLS = (0, 0, 1)               # 2s1p

OMEGA_WB97X = 0.3
CK_WB97X = 0.157706
SEED_BASE = 16586


def _draw_element_basis(rng, heavy):
    shells = HEAVY_SHELLS if heavy else H_SHELLS
    lo, hi = (0.15, 2000.0) if heavy else (0.1, 20.0)
    out = []
    for l in shells:
        k = int(rng.integers(1, 7))
        ex = np.sort(np.exp(rng.uniform(np.log(lo), np.log(hi), size=k)))[::-1]
        co = rng.uniform(0.2, 1.0, size=k)
        out.append((l, ex.copy(), co))
    return out


def _unit(rng):
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def place_sequential(rng, elements, dmin=0.95, dmax=3.0):
    """Each new atom sits d ~ U[dmin, dmax] A from a random placed atom in a
    random direction; rejected if closer than dmin to any placed atom."""
    pos = [np.zeros(3)]
    for _ in elements[1:]:
        for _try in range(10000):
            j = int(rng.integers(0, len(pos)))
            p = pos[j] + rng.uniform(dmin, dmax) * _unit(rng)
            if min(np.linalg.norm(p - q) for q in pos) >= dmin:
                pos.append(p)
                break
        else:
            raise RuntimeError("placement failed")
    return np.array(pos)


def _chain(rng, nheavy, nh, radius=None, heavy_kinds=("C", "C", "C", "N", "O")):
    """Heavy-atom chain with 1.2-1.6 A bonds, then X-H bonds of 1.0-1.1 A.
    With ``radius`` the chain is kept inside a sphere (compact core)."""
    for _restart in range(200):
        pos = [np.zeros(3)]
        ok = True
        for i in range(1, nheavy):
            for _try in range(2000):
                p = pos[-1] + rng.uniform(1.2, 1.6) * _unit(rng)
                if radius is not None and np.linalg.norm(p) > radius:
                    continue
                if all(np.linalg.norm(p - q) >= 2.0 for q in pos[:-1]):
                    pos.append(p)
                    break
            else:
                ok = False
                break
        if not ok:
            continue
        hpos = []
        for i in range(nh):
            for _try in range(5000):
                j = int(rng.integers(0, nheavy))
                p = pos[j] + rng.uniform(1.0, 1.1) * _unit(rng)
                if all(np.linalg.norm(p - q) >= 1.7 for k, q in enumerate(pos) if k != j) and \
                        all(np.linalg.norm(p - q) >= 1.4 for q in hpos):
                    hpos.append(p)
                    break
            else:
                ok = False
                break
        if ok:
            kinds = [heavy_kinds[int(rng.integers(0, len(heavy_kinds)))] for _ in range(nheavy)]
            return kinds + ["H"] * nh, np.array(pos + hpos)
    raise RuntimeError("chain placement failed")


def _water_shell(rng, core_xyz, nwater, r_in):
    """Waters (O-H 0.96 A, 104.5 deg) at 0.0334 molecules/A^3 in a shell
    around the core; min O-O 2.5 A, min O-core 2.4 A."""
    vol = nwater / 0.0334
    r_out = (r_in ** 3 + 3.0 * vol / (4.0 * np.pi)) ** (1.0 / 3.0)
    ox = []
    tries = 0
    while len(ox) < nwater:
        tries += 1
        if tries > 2000000:
            raise RuntimeError("water placement failed")
        if tries % 200000 == 0:
            r_out *= 1.03
        p = _unit(rng) * (rng.uniform(r_in ** 3, r_out ** 3) ** (1.0 / 3.0))
        if len(ox) and np.min(np.linalg.norm(np.array(ox) - p, axis=1)) < 2.5:
            continue
        if len(core_xyz) and np.min(np.linalg.norm(core_xyz - p, axis=1)) < 2.4:
            continue
        ox.append(p)
    half = np.deg2rad(104.5) / 2.0
    els, xyz = [], []
    for o in ox:
        u = _unit(rng)
        w = _unit(rng)
        w = w - u * np.dot(u, w)
        w /= np.linalg.norm(w)
        h1 = o + 0.96 * (np.cos(half) * u + np.sin(half) * w)
        h2 = o + 0.96 * (np.cos(half) * u - np.sin(half) * w)
        els += ["O", "H", "H"]
        xyz += [o, h1, h2]
    return els, np.array(xyz)


def _cluster(rng, natom):
    """Compact core (half H) at ~1.35 g/cm^3 plus water at 1.0 g/cm^3; about
    58 % of the atoms are in the core, which gives ~43 % heavy atoms."""
    ncore = int(round(0.58 * natom))
    nwater = (natom - ncore) // 3
    ncore = natom - 3 * nwater
    nheavy = ncore // 2
    nh = ncore - nheavy
    # 1.35 g/cm^3 with a mean atomic mass ~7.3 amu -> 0.111 atoms / A^3
    r_core = (3.0 * ncore / (4.0 * np.pi * 0.111)) ** (1.0 / 3.0)
    els, xyz = _chain(rng, nheavy, nh, radius=r_core * 1.15)
    wel, wxyz = _water_shell(rng, xyz, nwater, r_core + 1.0)
    return els + wel, np.vstack([xyz, wxyz])


def _basis_for(elements, rng):
    lib = {}
    for el in ("H", "C", "N", "O"):
        lib[el] = _draw_element_basis(rng, heavy=(el != "H"))
    shell_atom, shell_l, shell_nprim, exps, coefs = [], [], [], [], []
    for ia, el in enumerate(elements):
        for (l, ex, co) in lib[el]:
            shell_atom.append(ia)
            shell_l.append(l)
            shell_nprim.append(len(ex))
            exps.append(ex)
            coefs.append(co)
    return dict(shell_atom=np.array(shell_atom, dtype=np.int32),
                shell_l=np.array(shell_l, dtype=np.int32),
                shell_nprim=np.array(shell_nprim, dtype=np.int32),
                exps=np.concatenate(exps).astype(np.float64),
                coefs=np.concatenate(coefs).astype(np.float64))


def nbf_of(shell_l):
    l = np.asarray(shell_l)
    return int(np.sum((l + 1) * (l + 2) // 2))


def _density(rng, nbf):
    c = rng.normal(0.0, 0.3, size=(nbf, 5))
    return np.ascontiguousarray(c @ c.T)


def _transition(rng, nbf):
    x = rng.normal(size=(nbf, nbf))
    return np.ascontiguousarray(x / np.linalg.norm(x))


def _system(elements, xyz_ang, rng, pairs_kind):
    basis = _basis_for(elements, rng)
    nbf = nbf_of(basis["shell_l"])
    if pairs_kind == "c1":
        a = _density(rng, nbf)
        x = _transition(rng, nbf)
        pairs = [(a, a, 1.0, 1.0, 0.0, 0.0), (x, x, 0.0, 0.0, 1.0, OMEGA_WB97X)]
    else:
        p = _density(rng, nbf)
        pd = _density(rng, nbf)
        x = _transition(rng, nbf)
        pairs = [(m1, m2, 1.0, CK_WB97X, 1.0, OMEGA_WB97X)
                 for (m1, m2) in ((p, p), (pd, p), (x, x))]
    return dict(elements=list(elements), natom=len(elements),
                xyz=np.ascontiguousarray(np.asarray(xyz_ang, dtype=np.float64) * BOHR_PER_ANG),
                nbf=nbf, pairs=pairs, **basis)


def molecule(seed, nheavy, nh, pairs_kind="c2"):
    """A chain molecule with ``nheavy`` heavy atoms and ``nh`` hydrogens."""
    rng = np.random.default_rng(seed)
    els, xyz = _chain(rng, nheavy, nh)
    return _system(els, xyz, rng, pairs_kind)


def config(index):
    """The five workloads: ``config(0)`` .. ``config(4)`` = c1 .. c5.
    ``config(2)`` returns a list of 64 molecules."""
    rng = np.random.default_rng(SEED_BASE + index)
    if index == 0:
        els = ["O", "O", "H", "H", "H", "H"]
        xyz = place_sequential(rng, els)
        return _system(els, xyz, rng, "c1")
    if index == 1:
        els, xyz = _chain(rng, 13, 19)
        return _system(els, xyz, rng, "c2")
    if index == 2:
        mols = []
        for _ in range(64):
            n = int(rng.integers(20, 121))
            nheavy = int(round(0.4 * n))
            els, xyz = _chain(rng, nheavy, n - nheavy)
            mols.append(_system(els, xyz, rng, "c2"))
        return mols
    if index == 3:
        els, xyz = _cluster(rng, 300)
        return _system(els, xyz, rng, "c2")
    if index == 4:
        els, xyz = _cluster(rng, 1500)
        return _system(els, xyz, rng, "c2")
    raise ValueError(index)


def router_cluster(i, natom=None):
    """Training clusters for the learned router: seed 20240716 + i, 30-80 atoms."""
    rng = np.random.default_rng(20240716 + i)
    n = int(rng.integers(30, 81)) if natom is None else natom
    els, xyz = _cluster(rng, n)
    return _system(els, xyz, rng, "c2")
