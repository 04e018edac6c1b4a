"""The seeded synthetic workloads follow their stated recipe (CPU only).

They stand in for the paper's GFP / def2-SVP application (Sec. III), which
is not available: split-valence-like Cartesian shells (3s2p1d on C/N/O, 2s1p
on H), exponents log-uniform in [0.15, 2000] (heavy) or [0.1, 20] (H), 1-6
primitives per shell sorted descending, coefficients in [0.2, 1], one basis
per element; c1 placed sequentially at 0.95-3.0 A; chains with 1.2-1.6 A
heavy-atom bonds and 1.0-1.1 A X-H bonds; clusters of a compact core and
rigid waters (O-H 0.96 A, 104.5 degrees, O-O >= 2.5 A); densities
A = C C^T with C of nbf x 5 normal entries (sigma 0.3) and a transition
density X with |X|_F = 1."""
import numpy as np
import pytest

from paper_2407_16586_gb300 import synth

ANG = synth.BOHR_PER_ANG
SHELLS = {"H": [0, 0, 1], "C": [0, 0, 0, 1, 1, 2], "N": [0, 0, 0, 1, 1, 2], "O": [0, 0, 0, 1, 1, 2]}


def _atom_shells(s):
    """Per atom: list of (l, exponents, coefficients)."""
    out = [[] for _ in range(s["natom"])]
    off = 0
    for a, l, n in zip(s["shell_atom"], s["shell_l"], s["shell_nprim"]):
        out[a].append((int(l), s["exps"][off:off + n], s["coefs"][off:off + n]))
        off += n
    assert off == len(s["exps"])
    return out


def _check_basis(s):
    per_el = {}
    for el, shells in zip(s["elements"], _atom_shells(s)):
        assert [l for l, _, _ in shells] == SHELLS[el]
        lo, hi = (0.1, 20.0) if el == "H" else (0.15, 2000.0)
        for l, ex, co in shells:
            assert 1 <= len(ex) <= 6
            assert np.all(ex >= lo) and np.all(ex <= hi)
            assert np.all(np.diff(ex) <= 0)  # sorted descending
            assert np.all(co >= 0.2) and np.all(co <= 1.0)
        key = tuple(np.concatenate([np.concatenate([ex, co]) for _, ex, co in shells]))
        assert per_el.setdefault(el, key) == key  # one basis per element


def _check_densities(s):
    n = s["nbf"]
    mats = {id(m): m for p in s["pairs"] for m in p[:2]}
    sym = [m for m in mats.values() if np.allclose(m, m.T)]
    nonsym = [m for m in mats.values() if not np.allclose(m, m.T)]
    assert len(nonsym) == 1 and abs(np.linalg.norm(nonsym[0]) - 1.0) < 1e-12
    for m in sym:
        assert m.shape == (n, n)
        w = np.linalg.eigvalsh(m)
        assert w.min() > -1e-10 * w.max() and np.sum(w > 1e-8 * w.max()) == 5
        # trace(C C^T) / 0.09 is chi-square with 5n degrees of freedom (C ~ N(0, 0.3^2)):
        # within 5 standard deviations of its mean 5n
        assert abs(np.trace(m) / (5 * n * 0.09) - 1.0) < 5.0 * np.sqrt(2.0 / (5 * n))


def _dist(xyz):
    return np.linalg.norm(xyz[:, None, :] - xyz[None, :, :], axis=-1)


def test_c1_recipe():
    s = synth.config(0)
    assert sorted(s["elements"]) == ["H"] * 4 + ["O"] * 2
    d = _dist(s["xyz"] / ANG)
    np.fill_diagonal(d, np.inf)
    assert d.min() >= 0.95 - 1e-12
    assert np.all(d.min(axis=1) <= 3.0 + 1e-12)  # each atom within 3 A of another
    _check_basis(s)
    (A, A2, *ca), (X, X2, *cx) = s["pairs"]
    assert ca == [1.0, 1.0, 0.0, 0.0] and cx == [0.0, 0.0, 1.0, 0.3]
    assert A is A2 and X is X2
    _check_densities(s)


def test_c2_chain_recipe():
    s = synth.config(1)
    els = s["elements"]
    assert len(els) == 32 and els.count("H") == 19
    assert set(els) <= {"C", "N", "O", "H"}
    xyz = s["xyz"] / ANG
    heavy = [i for i, e in enumerate(els) if e != "H"]
    for i, j in zip(heavy[:-1], heavy[1:]):
        assert 1.2 - 1e-12 <= np.linalg.norm(xyz[i] - xyz[j]) <= 1.6 + 1e-12
    for i, e in enumerate(els):
        if e == "H":
            dh = min(np.linalg.norm(xyz[i] - xyz[j]) for j in heavy)
            assert 1.0 - 1e-12 <= dh <= 1.1 + 1e-12
    _check_basis(s)
    _check_densities(s)


def test_c4_cluster_recipe():
    s = synth.config(3)
    els = s["elements"]
    assert len(els) == 300
    assert abs(sum(e != "H" for e in els) / 300 - 0.43) < 0.03
    xyz = s["xyz"] / ANG
    # the waters are the trailing O, H, H triples
    nw = 0
    i = len(els) - 3
    while i >= 0 and els[i:i + 3] == ["O", "H", "H"]:
        o, h1, h2 = xyz[i], xyz[i + 1], xyz[i + 2]
        r1, r2 = np.linalg.norm(h1 - o), np.linalg.norm(h2 - o)
        ang = np.degrees(np.arccos(np.dot(h1 - o, h2 - o) / (r1 * r2)))
        if abs(r1 - 0.96) > 1e-9 or abs(r2 - 0.96) > 1e-9 or abs(ang - 104.5) > 1e-6:
            break
        nw += 1
        i -= 3
    assert nw >= 35
    ox = xyz[[len(els) - 3 * (k + 1) for k in range(nw)]]
    d = _dist(ox)
    np.fill_diagonal(d, np.inf)
    assert d.min() >= 2.5 - 1e-9
    _check_basis(s)
    _check_densities(s)


def test_c3_molecules_are_chains_of_the_c2_recipe():
    mols = synth.config(2)
    assert len({m["natom"] for m in mols}) > 20  # uneven sizes
    for m in mols[:4]:
        assert m["elements"].count("H") == m["natom"] - int(round(0.4 * m["natom"]))
        _check_basis(m)
        _check_densities(m)


@pytest.mark.slow
def test_c5_sizes():
    s = synth.config(4)
    assert (s["natom"], s["nbf"], len(s["shell_l"])) == (1500, 13950, 6435)
    assert abs(sum(e != "H" for e in s["elements"]) / 1500 - 0.43) < 0.02
