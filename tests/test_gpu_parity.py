"""Parity of the CUDA path (through the C-ABI) with the CPU oracle.

Tolerance: the plain fp64 path must match the fp64 oracle within 1e-10
Ha/bohr per gradient component.  Quartet counts are integers and must match
exactly.  Inputs are the seeded synthetic systems of synth.py; C1 and the
small molecules span several 16x8 quartet tiles of every class with ragged
tails; C2 is checked at full size on shards (the launch configuration is the
full one, the shard filter keeps 1/nranks of the quartets) so the oracle
finishes in seconds."""
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


def test_c1_unscreened(tg, c1):
    g, st = tg.grad2e(c1, screen_tol=0.0)
    ref, _, nq = oracle.grad2e(c1, tau=0.0)
    assert st["quartets"] == nq == 45150
    assert np.abs(g - ref).max() <= TOL, np.abs(g - ref).max()


@pytest.mark.parametrize("seed,nheavy,nh", [(11, 2, 3), (12, 3, 1), (13, 1, 4)])
def test_small_molecules(tg, seed, nheavy, nh):
    s = synth.molecule(seed, nheavy, nh)
    g, st = tg.grad2e(s, screen_tol=0.0)
    ref, _, nq = oracle.grad2e(s, tau=0.0)
    assert st["quartets"] == nq
    assert np.abs(g - ref).max() <= TOL


def test_kernel_kinds(tg):
    """Both class-kernel forms (one quartet per thread; a thread group per
    quartet, with tiles cut into quartet chunks and bra-primitive splits) give
    the oracle's gradient, and the same quartet and primitive-quartet counts."""
    s = synth.molecule(14, 3, 3)
    b = tg.Basis(s)
    ref, _, nq = oracle.grad2e(s, tau=0.0)
    pqs = []
    for kernel in (1, 2):
        g, st = b.grad2e(s["pairs"], screen_tol=0.0, kernel=kernel)
        assert st["quartets"] == nq
        assert np.abs(g - ref).max() <= TOL, (kernel, np.abs(g - ref).max())
        pqs.append(st["prim_quartets"])
    assert pqs[0] == pqs[1]


def test_screening_follows_the_defined_bound(tg, c1):
    for tau in (1e-10, 1e-7, 1e-4):
        g, st = tg.grad2e(c1, screen_tol=tau)
        ref, _, nq = oracle.grad2e(c1, tau=tau)
        assert st["quartets"] == nq
        assert np.abs(g - ref).max() <= TOL


def test_shards(tg):
    s = synth.molecule(14, 2, 2)
    whole, stw = tg.grad2e(s, screen_tol=0.0)
    tot = np.zeros_like(whole)
    nq = 0
    for r in range(3):
        g, st = tg.grad2e(s, screen_tol=0.0, rank=r, nranks=3)
        ref, _, n = oracle.grad2e(s, tau=0.0, rank=r, nranks=3)
        assert st["quartets"] == n
        assert np.abs(g - ref).max() <= TOL
        tot += g
        nq += st["quartets"]
    assert nq == stw["quartets"]
    assert np.abs(tot - whole).max() <= 1e-12


def test_c2_full_size_shards(tg):
    s = synth.config(1)
    for rank in (7, 1234):
        g, st = tg.grad2e(s, screen_tol=1e-10, rank=rank, nranks=3000)
        ref, _, nq = oracle.grad2e(s, tau=1e-10, rank=rank, nranks=3000)
        assert st["quartets"] == nq and nq > 0
        assert np.abs(g - ref).max() <= TOL


def test_c4_full_size_shard(tg):
    """The 300-atom core + water cluster (2790 basis functions) at full size:
    every tile of every class is launched, the shard filter keeps 1/50000 of
    the canonical quartets, and the oracle evaluates the same shard."""
    s = synth.config(3)
    g, st = tg.grad2e(s, screen_tol=1e-10, rank=11, nranks=50000)
    ref, _, nq = oracle.grad2e(s, tau=1e-10, rank=11, nranks=50000)
    assert st["quartets"] == nq and nq > 1000
    assert np.abs(g - ref).max() <= TOL


def test_omega_infinity_is_the_full_operator(tg):
    """erf(omega r)/r -> 1/r as omega -> inf: an lr exchange pair at omega = +inf
    gives the full-range exchange gradient."""
    s = synth.molecule(15, 2, 2)
    A = s["pairs"][0][0]
    X = s["pairs"][-1][0]
    b = tg.Basis(s)
    g_lr, st1 = b.grad2e([(A, X, 0.0, 0.0, 1.0, float("inf"))], screen_tol=0.0)
    g_full, st2 = b.grad2e([(A, X, 0.0, 1.0, 0.0, 0.0)], screen_tol=0.0)
    assert st1["quartets"] == st2["quartets"]
    assert np.abs(g_lr - g_full).max() <= 1e-12 * max(1.0, np.abs(g_full).max())


def test_single_atom_has_zero_gradient(tg):
    """Every quartet of one atom is one-centre; its derivative integrals sum to
    zero over the centres (eq. ti)."""
    s = synth.molecule(16, 1, 0)
    assert s["natom"] == 1
    g, st = tg.grad2e(s, screen_tol=0.0)
    assert st["quartets"] > 0
    assert np.abs(g).max() <= 1e-10


def test_eight_pairs(tg):
    """The largest pair list (TG_MAX_PAIRS = 8), mixed coefficients and
    operators, against the oracle."""
    s = synth.molecule(11, 2, 3)
    P, X = s["pairs"][0][0], s["pairs"][-1][0]
    rng = np.random.default_rng(3)
    mats = [P, X, X.T.copy(), P + X]
    pairs = []
    for k in range(8):
        A, B = mats[k % 4], mats[(k + 1) % 4]
        cj, ck, cl = (float(v) for v in rng.uniform(-1.0, 1.0, 3))
        pairs.append((A, B, cj, ck, cl, 0.3))
    b = tg.Basis(s)
    g, st = b.grad2e(pairs, screen_tol=0.0)
    ref, _, nq = oracle.grad2e(s, pairs=pairs, tau=0.0)
    assert st["quartets"] == nq
    assert np.abs(g - ref).max() <= TOL


def test_bitwise_deterministic(tg, c1):
    g1, _ = tg.grad2e(c1, screen_tol=1e-12)
    g2, _ = tg.grad2e(c1, screen_tol=1e-12)
    assert np.array_equal(g1, g2)


def test_device_pointers_match_host(tg, c1):
    torch = pytest.importorskip("torch")
    dev = [(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), cj, ck, cl, om)
           for (a, b, cj, ck, cl, om) in c1["pairs"]]
    basis = tg.Basis(c1)
    gd, _ = basis.grad2e(dev, screen_tol=1e-12)
    gh, _ = basis.grad2e(c1["pairs"], screen_tol=1e-12)
    torch.cuda.synchronize()
    assert np.array_equal(gd.cpu().numpy(), gh)


def test_error_codes(tg, c1):
    bad = dict(c1)
    bad["exps"] = c1["exps"].copy()
    bad["exps"][3] = -1.0
    with pytest.raises(tg.TGError) as e:
        tg.Basis(bad)
    assert e.value.status == tg.TG_EINVAL
    bad = dict(c1)
    bad["shell_l"] = c1["shell_l"].copy()
    bad["shell_l"][0] = 3
    with pytest.raises(tg.TGError) as e:
        tg.Basis(bad)
    assert e.value.status == tg.TG_EUNSUPPORTED
    a = c1["pairs"][0][0]
    basis = tg.Basis(c1)
    with pytest.raises(tg.TGError) as e:
        basis.grad2e([(a, a, 0, 0, 1.0, 0.3), (a, a, 0, 0, 1.0, 0.4)])
    assert e.value.status == tg.TG_EUNSUPPORTED
    with pytest.raises(tg.TGError) as e:
        basis.grad2e([(a, a, 1, 0, 0, 0)] * 9)
    assert e.value.status == tg.TG_EUNSUPPORTED
    with pytest.raises(tg.TGError) as e:
        basis.grad2e([(a, a, 1, 0, 0, 0)], rank=2, nranks=2)
    assert e.value.status == tg.TG_EINVAL
    # named options out of range
    for kw in (dict(kernel=4), dict(shard_mode=2), dict(class_mask=1 << 21), dict(autotune=3)):
        out = np.full((c1["natom"], 3), 5.0)
        with pytest.raises(tg.TGError) as e:
            basis.grad2e([(a, a, 1, 0, 0, 0)], out=out, **kw)
        assert e.value.status == tg.TG_EINVAL, kw
        assert np.all(out == 5.0)


def test_fp32_route_close_to_fp64(tg, c1):
    g64, _ = tg.grad2e(c1, screen_tol=1e-12)
    g32, st = tg.grad2e(c1, screen_tol=1e-12, precision=tg.TG_FP32)
    assert st["fp32_quartets"] == st["quartets"]
    assert np.abs(g32 - g64).max() <= 1e-4


def test_mixed_bound_meets_tolerance(tg, c1):
    ref, _, _ = oracle.grad2e(c1, tau=1e-10)
    g, st = tg.grad2e(c1, screen_tol=1e-10, precision=tg.TG_MIXED_BOUND)
    assert np.abs(g - ref).max() <= 1e-6


def test_batch_matches_single_calls(tg):
    """Several uneven molecules in one planned batch (persistent class
    launches over all of them, replayed from a captured CUDA graph) give the
    single-molecule results; replays are bitwise identical."""
    systems = [synth.molecule(40 + i, n, h) for i, (n, h) in enumerate([(1, 2), (3, 2), (2, 4), (4, 1)])]
    batch = tg.Batch(systems, screen_tol=1e-10)
    g1, st = batch.run()
    g2, _ = batch.run()
    for s, a, b in zip(systems, g1, g2):
        ref, _ = tg.grad2e(s, screen_tol=1e-10)
        assert np.abs(a - ref).max() <= 1e-12
        assert np.array_equal(a, b)
    tuned = tg.Batch(systems, screen_tol=1e-10, autotune=True)
    g3, _ = tuned.run()
    for a, c in zip(g1, g3):
        assert np.abs(a - c).max() <= 1e-12
    ref0, _, _ = oracle.grad2e(systems[0], tau=1e-10)
    assert np.abs(g1[0] - ref0).max() <= TOL


@pytest.mark.parametrize("tau", [0.0, 1e-10, 1e-6])
def test_device_tile_lists_match_the_host_planner(tg, tau):
    """The device block screen (tg_grad2e) keeps exactly the tiles of the host
    planner (the batch path) for one molecule: same tile count, same quartets,
    same gradient to rounding."""
    s = synth.molecule(17, 3, 4)
    g, st = tg.grad2e(s, screen_tol=tau)
    batch = tg.Batch([s], screen_tol=tau)
    gb, stb = batch.run()
    assert st["tiles"] == stb["tiles"] and st["tiles"] > 0
    assert st["quartets"] == stb["quartets"]
    assert np.abs(g - gb[0]).max() <= 1e-12
    ref, _, nq = oracle.grad2e(s, tau=tau)
    assert st["quartets"] == nq
    assert np.abs(g - ref).max() <= TOL


def test_device_routing_meets_the_budget(tg):
    """The device router's histogram cut-off sends tiles to fp32 while the
    summed error estimate stays within the budget: the gradient stays within
    mixed_tol of the oracle, and some tiles do go to fp32."""
    s = synth.molecule(18, 4, 4)
    ref, _, _ = oracle.grad2e(s, tau=1e-10)
    for tol in (1e-6, 1e-8):
        g, st = tg.grad2e(s, screen_tol=1e-10, precision=tg.TG_MIXED_BOUND, mixed_tol=tol)
        assert np.abs(g - ref).max() <= tol
        assert 0 < st["fp32_quartets"] < st["quartets"]


def test_tile_shards_sum_to_the_whole(tg):
    """Tile-cyclic shards (every class list dealt round-robin to the ranks):
    the ranks' quartet counts and partial gradients sum to the whole call."""
    s = synth.molecule(19, 3, 3)
    b = tg.Basis(s)
    whole, stw = b.grad2e(s["pairs"], screen_tol=1e-10)
    tot = np.zeros_like(whole)
    nq = 0
    for r in range(3):
        g, st = b.grad2e(s["pairs"], screen_tol=1e-10, rank=r, nranks=3, shard_mode=tg.TG_SHARD_TILES)
        assert 0 < st["quartets"] < stw["quartets"]
        tot += g
        nq += st["quartets"]
    assert nq == stw["quartets"]
    assert np.abs(tot - whole).max() <= 1e-12


def test_tile_shards_hold_the_same_tiles_at_every_precision(tg):
    """The tile shard is dealt before the fp32 / fp64 split and the route is the
    whole call's: a rank's mixed partial covers the same quartets as its fp64
    partial and stays within the whole call's mixed_tol of it, and the ranks'
    fp32 quartets add up to the whole call's."""
    s = synth.molecule(18, 4, 4)
    b = tg.Basis(s)
    tol = 1e-6
    _, stw = b.grad2e(s["pairs"], screen_tol=1e-10, precision=tg.TG_MIXED_BOUND, mixed_tol=tol)
    assert 0 < stw["fp32_quartets"] < stw["quartets"]
    n32 = 0
    for r in range(3):
        kw = dict(screen_tol=1e-10, rank=r, nranks=3, shard_mode=tg.TG_SHARD_TILES)
        g64, s64 = b.grad2e(s["pairs"], **kw)
        gm, sm = b.grad2e(s["pairs"], precision=tg.TG_MIXED_BOUND, mixed_tol=tol, **kw)
        assert sm["quartets"] == s64["quartets"]
        assert sm["prim_quartets"] == s64["prim_quartets"]
        assert np.abs(gm - g64).max() <= tol
        n32 += sm["fp32_quartets"]
    assert n32 == stw["fp32_quartets"]


def test_allocation_failure_leaves_the_output_untouched(tg, monkeypatch):
    """With the host-side hook TDGRAD_FAIL_ALLOC=1 every growth of the work
    areas fails as an out-of-memory would: the call returns TG_ENOMEM and the
    output keeps its contents; without the hook the same basis works."""
    s = synth.molecule(20, 1, 2)
    b = tg.Basis(s)  # fresh basis: its work areas are still empty
    out = np.full((s["natom"], 3), 7.0)
    monkeypatch.setenv("TDGRAD_FAIL_ALLOC", "1")
    with pytest.raises(tg.TGError) as e:
        b.grad2e(s["pairs"], screen_tol=1e-10, out=out)
    assert e.value.status == tg.TG_ENOMEM
    assert np.all(out == 7.0)
    monkeypatch.delenv("TDGRAD_FAIL_ALLOC")
    g, _ = b.grad2e(s["pairs"], screen_tol=1e-10, out=out)
    ref, _, _ = oracle.grad2e(s, tau=1e-10)
    assert np.abs(g - ref).max() <= TOL


def test_autotuned_single_calls(tg):
    """tg_grad2e with autotune = 1 tunes the launches of every class list on the
    basis's first such call and reuses them.  On full-size c2 (lists of more
    than 152 tiles, so the tuner runs): a pair-key shard stays within the plain
    bound of the oracle's shard, a second tuned call repeats the first bitwise,
    a re-tune (autotune = 2) stays within the bound, and the whole tuned
    gradient equals the untuned one up to summation order."""
    s = synth.config(1)
    ref, _, nq = oracle.grad2e(s, tau=1e-10, rank=7, nranks=3000)
    b = tg.Basis(s)
    kw = dict(screen_tol=1e-10, rank=7, nranks=3000)
    g1, st1 = b.grad2e(s["pairs"], autotune=1, **kw)
    assert st1["quartets"] == nq and nq > 0
    assert np.abs(g1 - ref).max() <= TOL
    g2, _ = b.grad2e(s["pairs"], autotune=1, **kw)
    assert np.array_equal(g1, g2)
    g3, _ = b.grad2e(s["pairs"], autotune=2, **kw)
    assert np.abs(g3 - ref).max() <= TOL
    whole, stw = b.grad2e(s["pairs"], screen_tol=1e-10)
    tuned, stt = b.grad2e(s["pairs"], screen_tol=1e-10, autotune=1)
    assert stt["quartets"] == stw["quartets"]
    assert np.abs(tuned - whole).max() <= 1e-11
