"""Host-side logic that needs no GPU: the workload generator's structure, the
bench's class table and bookkeeping, and the router's budget calibration
(against a fake of the library, on the CPU)."""
import glob
import os

import numpy as np
import pytest

import bench
from paper_2407_16586_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("index,natom,nbf,nshell,npair", [(0, 6, 50, 24, 2), (1, 32, 290, 135, 3),
                                                         (3, 300, 2790, 1287, 3)])
def test_workload_sizes(index, natom, nbf, nshell, npair):
    s = synth.config(index)
    assert (s["natom"], s["nbf"], len(s["shell_l"]), len(s["pairs"])) == (natom, nbf, nshell, npair)
    assert max(s["shell_l"]) == 2
    # basis functions counted from the shells (Cartesian: 1, 3, 6)
    assert sum((l + 1) * (l + 2) // 2 for l in s["shell_l"]) == nbf


def test_workloads_are_seeded():
    a, b = synth.config(1), synth.config(1)
    assert np.array_equal(a["xyz"], b["xyz"]) and np.array_equal(a["exps"], b["exps"])
    for (A1, B1, *c1), (A2, B2, *c2) in zip(a["pairs"], b["pairs"]):
        assert np.array_equal(A1, A2) and np.array_equal(B1, B2) and c1 == c2


def test_c2_pairs_follow_the_reading():
    """[(P,P), (P_delta,P), (X,X)], c_J = 1, c_K = 0.157706, c_K_lr = 1, omega = 0.3;
    P symmetric positive semidefinite of rank 5, X normalised to |X|_F = 1."""
    s = synth.config(1)
    (P, P2, *c0), (Pd, P3, *c1), (X, X2, *c2) = s["pairs"]
    assert P is P2 or np.array_equal(P, P2)
    assert np.array_equal(P3, P)
    assert np.array_equal(X, X2)
    for c in (c0, c1, c2):
        assert c == [1.0, 0.157706, 1.0, 0.3]
    assert np.allclose(P, P.T)
    w = np.linalg.eigvalsh(P)
    assert w.min() > -1e-10 and np.sum(w > 1e-8 * w.max()) == 5
    assert abs(np.linalg.norm(X) - 1.0) < 1e-12


def test_c3_batch_sizes():
    mols = synth.config(2)
    assert len(mols) == 64
    assert all(20 <= m["natom"] <= 120 for m in mols)


def test_class_table_matches_the_kernels():
    """bench.class_ls() index = the library's class index = the class file number."""
    names = "spd"
    files = sorted(os.path.basename(f) for f in glob.glob(os.path.join(ROOT, "paper_2407_16586_gb300", "csrc",
                                                                        "class_*.cu")))
    assert len(files) == 21
    for qc, (la, lb, lc, ld) in enumerate(bench.class_ls()):
        assert files[qc] == "class_%02d_%s%s%s%s.cu" % (qc, names[la], names[lb], names[lc], names[ld])
        assert la >= lb and lc >= ld


def test_flop_model_is_monotone_in_angular_momentum():
    from paper_2407_16586_gb300 import build
    import paper_2407_16586_gb300 as tg
    build.build()
    ls = bench.class_ls()
    f = {c: sum(tg.tg_class_flops(qc)) for qc, c in enumerate(ls)}
    assert f[(2, 2, 2, 2)] > f[(2, 2, 2, 1)] > f[(2, 2, 1, 1)] > f[(1, 1, 1, 1)] > f[(0, 0, 0, 0)]
    # one operator costs less than two
    assert tg.tg_class_flops(5, 1)[0] < tg.tg_class_flops(5, 2)[0]


def test_workload_names():
    s, name = bench.workload("chain:5:6:6")
    assert s["natom"] == 12 and "6 heavy + 6 H" in name
    assert bench.workload("c1")[0]["natom"] == 6
    with pytest.raises(ValueError):
        bench.workload("c9")


def test_clock_summary():
    rows = ["0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "1, 1000, 2070, 100.0, 0x0, Active, Not Active, Not Active, Not Active"]
    c = bench._clocks_summary(rows, 0)
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"]
    assert bench._clocks_summary([], 0)["sm_mhz"] is None


class _FakeRouter:
    def __init__(self):
        self.calib = np.array([1.0, 1e-6, 1.0], np.float32)

    def get(self):
        return None, None, None, self.calib.copy()

    def set(self, calib=None, **kw):
        self.calib = np.asarray(calib, np.float32)


def test_budget_calibration_keeps_the_last_safe_margin(monkeypatch):
    """A fake library whose mixed-route error grows by 3x per 0.5 of margin
    lowered: calibrate_budget must stop at the first margin over
    mixed_tol / safety and keep the one before it."""
    from paper_2407_16586_gb300 import router
    r = _FakeRouter()

    class FakeBasis:
        def __init__(self, s):
            pass

        def grad2e(self, pairs, screen_tol=1e-10, precision=0, router=None, mixed_tol=1e-6, **kw):
            g = np.zeros((2, 3))
            if precision == router_mod.TG_MIXED_LEARNED:
                m = float(router.calib[0])
                g[0, 0] = 1e-8 * 3.0 ** ((1.0 - m) / 0.5)
            return g, {"fp32_quartets": 1, "quartets": 2}

        def close(self):
            pass

    router_mod = router.tg
    monkeypatch.setattr(router_mod, "Basis", FakeBasis)
    log = router.calibrate_budget(r, [{"pairs": []}], mixed_tol=1e-6, safety=5.0, step=0.5)
    errs = [e for _, e, _, _ in log]
    assert all(b > a for a, b in zip(errs, errs[1:]))
    assert errs[-1] > 2e-7 and errs[-2] <= 2e-7
    assert float(r.calib[0]) == pytest.approx(log[-2][0])
    assert float(r.calib[1]) == pytest.approx(1e-6)


def _fake_stats(ms64, ms32, pq64, pq32):
    z = [0.0] * 21
    st = {"class_ms": list(z), "class_ms_fp32": list(z), "class_prim_quartets": [0] * 21,
          "class_prim_quartets_fp32": [0] * 21, "class_bra_prims": [0] * 21, "class_bra_prims_fp32": [0] * 21}
    for qc, v in ms64.items():
        st["class_ms"][qc] = v
    for qc, v in ms32.items():
        st["class_ms_fp32"][qc] = v
    for qc, v in pq64.items():
        st["class_prim_quartets"][qc] = v
    for qc, v in pq32.items():
        st["class_prim_quartets_fp32"][qc] = v
    return st


def test_roofline_of_the_dominant_kernel():
    """achieved = algorithmic FLOPs of the longest class launch (per primitive
    quartet and per bra primitive pair, tg_class_flops) / its time; frac
    against the derived fp64 (or fp32) ALU peak; frac_mixed = the time all
    class launches would take at their peaks / their summed time."""
    import paper_2407_16586_gb300 as tg
    ls = bench.class_ls()
    dppp, dddd = ls.index((2, 1, 1, 1)), ls.index((2, 2, 2, 2))
    st = _fake_stats({dppp: 600.0, 0: 5.0}, {dddd: 100.0}, {dppp: 4_850_000, 0: 10_000}, {dddd: 20_000})
    st["class_bra_prims"][dppp] = 400_000
    st["class_bra_prims"][0] = 1_000
    st["class_bra_prims_fp32"][dddd] = 5_000
    r = bench.roofline_entry(st)
    a, b = tg.tg_class_flops(dppp)
    flops = 4_850_000 * a + 400_000 * b
    assert r["kernel"] == "(dp|pp) fp64"
    assert r["achieved"] == pytest.approx(flops / 0.6 / 1e12)
    assert r["peak"] == pytest.approx(152 * 2 * 2 * 2.07e9 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["traffic"] is None
    a0, b0 = tg.tg_class_flops(0)
    a20, b20 = tg.tg_class_flops(dddd)
    f64 = flops + 10_000 * a0 + 1_000 * b0
    f32 = 20_000 * a20 + 5_000 * b20
    ideal = f64 / (r["peak"] * 1e12) + f32 / (152 * 128 * 2 * 2.07e9)
    assert r["frac_mixed"] == pytest.approx(ideal / 0.705)
    assert r["fp64_frac"] == pytest.approx(f64 / 0.605 / 1e12 / r["peak"])
    # an fp32 launch that dominates: its own peak
    st = _fake_stats({dppp: 50.0}, {dddd: 100.0}, {dppp: 1000}, {dddd: 20_000})
    r = bench.roofline_entry(st)
    assert r["kernel"] == "(dd|dd) fp32"
    assert r["peak"] == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"



def _flop_model(la, lb, lc, ld, nops):
    """The algorithmic count of the class kernels' evaluation, enumerated here
    term by term: per primitive quartet the Boys orders (6 Taylor FMAs and a
    base product each), the Hermite R recursion, E^{cd} over the index boxes,
    W = E^{cd} R over the boxes of cd, z = F R over the derivative boxes of cd
    and the d/dC products; per bra primitive pair E^{ab}, F = Gamma E^{ab},
    Y = Gamma W over the derivative boxes of ab and the d/dA, d/dA + d/dB
    products (an FMA counts 2)."""
    def nh(L):
        return 0 if L < 0 else (L + 1) * (L + 2) * (L + 3) // 6

    def cart(l):
        return [(l - s, s - z, z) for s in range(l + 1) for z in range(s + 1)]

    def ext(l1, l2):
        return [tuple(a[i] + b[i] for i in range(3)) for a in cart(l1) for b in cart(l2)]

    def box(n):
        return (n[0] + 1) * (n[1] + 1) * (n[2] + 1)

    def dboxes(n):
        out = []
        for t in range(n[0] + 2):
            for u in range(n[1] + 2):
                for v in range(n[2] + 2):
                    ix, iy, iz = t <= n[0], u <= n[1], v <= n[2]
                    g = (t <= n[0] + 1 and iy and iz) + (ix and u <= n[1] + 1 and iz) + (ix and iy and v <= n[2] + 1)
                    if g:
                        out.append(g)
        return out

    L1, L2 = la + lb, lc + ld
    L = L1 + L2
    r = 0
    for n in range(L + 1):
        for k in range(1, L + 2 - n):
            for t in range(k + 1):
                for u in range(k - t + 1):
                    v = k - t - u
                    two = (t > 1) if t > 0 else ((u > 1) if u > 0 else (v > 1))
                    r += 3 if two else 1
    ab, cd = ext(la, lb), ext(lc, ld)
    pq = nops * r + nops * (L + 2) * 14 + 2 * sum(box(n) for n in cd)
    pq += nops * sum(box(n) for n in cd) * nh(L1 + 1) * 2 + nops * sum(len(dboxes(n)) for n in cd) * nh(L1) * 2
    pq += sum(7 * g for n in cd for g in dboxes(n))
    p = 2 * sum(box(n) for n in ab) + nops * len(cd) * sum(box(n) for n in ab) * 2
    p += nops * len(cd) * sum(len(dboxes(n)) for n in ab) * 2 + sum(11 * g for n in ab for g in dboxes(n))
    return pq, p


def test_class_flop_model_matches_the_enumeration():
    from paper_2407_16586_gb300 import build
    import paper_2407_16586_gb300 as tg
    build.build()
    pcs = [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2)]
    qc = 0
    for P in range(6):
        for Q in range(P + 1):
            for nops in (1, 2):
                got = tg.tg_class_flops(qc, nops)
                assert got == _flop_model(*pcs[P], *pcs[Q], nops), (qc, nops)
            qc += 1
    # (dp|pp): the index boxes cut the full-tetrahedron count several times
    assert tg.tg_class_flops(12)[0] == 15104


def test_tile_shards_cover_every_tile_once():
    """TG_SHARD_TILES: the ranks' tiles of a launch list partition it, and the
    counts differ by at most one (the list is ordered by decreasing cost, so
    the cyclic deal also balances cost)."""
    from paper_2407_16586_gb300 import build
    import paper_2407_16586_gb300 as tg
    build.build()
    for n in (0, 1, 7, 128, 1001):
        for nr in (1, 2, 3, 8):
            seen = []
            counts = []
            for r in range(nr):
                first, count, stride = tg.tg_tile_shard(n, r, nr)
                seen += [first + k * stride for k in range(count)]
                counts.append(count)
            assert sorted(seen) == list(range(n))
            assert max(counts) - min(counts) <= 1
    with pytest.raises(tg.TGError):
        tg.tg_tile_shard(10, 3, 3)


def test_shard_estimate_counts_the_plan_once():
    """A tile shard's step is its plan (of the whole system) plus 1/N of the
    class kernels: the whole-gradient estimate adds the plan once."""
    assert bench.shard_full_estimate(1000.0, 0.0, 32) == pytest.approx(32.0)
    assert bench.shard_full_estimate(46356.5, 30875.0, 4096) == pytest.approx(30.875 + 4096 * 15.4815)
    # one shard is the whole gradient
    assert bench.shard_full_estimate(1234.0, 200.0, 1) == pytest.approx(1.234)
