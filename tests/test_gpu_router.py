"""Learned router: GPU forward/backward against the fp64 CPU backprop
(oracle/mlp.py), training, and the gain over the rigorous-bound router at
the same accuracy target."""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2407_16586_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tg():
    from paper_2407_16586_gb300 import build
    build.build()
    import paper_2407_16586_gb300 as m
    return m


def test_router_gradient_matches_cpu_backprop(tg):
    rng = np.random.default_rng(3)
    r = tg.Router(seed=11)
    p, mu, sd, _ = r.get()
    X = rng.normal(size=(3000, 16)).astype(np.float32)
    y = rng.normal(size=3000).astype(np.float32)
    for q in (0.5, 0.9):
        L, g = r.loss_grad(X, y, q=q)
        Lr, gr = mlp.loss_and_grad(p.astype(np.float64), (X - mu) / sd, y, q)
        assert abs(L - Lr) <= 1e-4 * abs(Lr)
        assert np.abs(g - gr).max() <= 1e-4 * np.abs(gr).max()


def test_router_prediction_matches_cpu_forward(tg):
    rng = np.random.default_rng(4)
    r = tg.Router(seed=5)
    p, mu, sd, _ = r.get()
    X = rng.normal(size=(500, 16)).astype(np.float32)
    ref, _ = mlp.forward(p.astype(np.float64), (X - mu) / sd)
    assert np.abs(r.predict(X) - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())


def test_router_training_decreases_loss(tg):
    rng = np.random.default_rng(5)
    X = rng.normal(size=(20000, 16)).astype(np.float32)
    y = (np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2] - X[:, 3] ** 2).astype(np.float32)
    r = tg.Router(seed=1)
    hist = r.train(X, y, epochs=300, lr=1e-2, q=0.5)
    assert hist[-1] < 0.1 * hist[0]
    assert np.all(np.isfinite(hist))


def test_router_save_load_roundtrip(tg, tmp_path):
    r = tg.Router(seed=9)
    r.set(calib=[0.5, 1e-6, 1.0])
    f = tmp_path / "r.bin"
    r.save(str(f))
    r2 = tg.Router(path=str(f))
    for a, b in zip(r.get(), r2.get()):
        assert np.array_equal(a, b)


def test_learned_router_gain_over_bound_router(tg):
    """Trained on four seeded clusters, tested on a held-out molecule: at
    max|dg| <= 1e-6 against fp64 the learned router sends more quartets to
    fp32 than the rigorous-bound router."""
    from paper_2407_16586_gb300 import router
    train = [synth.router_cluster(i, natom=30) for i in range(4)]
    X, y, e = router.collect(train, stride=5, cap=40000)
    r, info = router.fit(X, y, e, epochs=300)
    assert info["loss_last"] < info["loss_first"]
    s = synth.molecule(31, 4, 6)
    b = tg.Basis(s)
    g64, _ = b.grad2e(s["pairs"], screen_tol=1e-10)
    gb, sb = b.grad2e(s["pairs"], screen_tol=1e-10, precision=tg.TG_MIXED_BOUND)
    gl, sl = b.grad2e(s["pairs"], screen_tol=1e-10, precision=tg.TG_MIXED_LEARNED, router=r)
    assert np.abs(gb - g64).max() <= 1e-6
    assert np.abs(gl - g64).max() <= 1e-6
    assert sl["fp32_quartets"] > sb["fp32_quartets"]
    # measured budget calibration on another molecule: more fp32, still within tolerance
    log = router.calibrate_budget(r, [synth.router_cluster(50, natom=20)], safety=10.0, max_steps=8)
    assert log[0][1] <= 1e-6 / 10
    g2, s2 = b.grad2e(s["pairs"], screen_tol=1e-10, precision=tg.TG_MIXED_LEARNED, router=r)
    assert np.abs(g2 - g64).max() <= 1e-6
    assert s2["fp32_quartets"] >= sl["fp32_quartets"]


def test_learned_mode_needs_a_trained_router(tg, c1):
    b = tg.Basis(c1)
    with pytest.raises(tg.TGError) as e:
        b.grad2e(c1["pairs"], precision=tg.TG_MIXED_LEARNED)
    assert e.value.status == tg.TG_EROUTER
