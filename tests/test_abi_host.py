"""Host-side behaviour of the C-ABI, run without a GPU: argument checks that
return a status before any CUDA call, the router handle's host functions
(initialisation, get/set, the file format), and the absence of a CPU
fallback (with no CUDA device a valid basis is refused with TG_ECUDA).
No compute call is made."""
import ctypes
import struct

import numpy as np
import pytest

import paper_2407_16586_gb300 as tg
from paper_2407_16586_gb300 import build, synth

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_fp = ctypes.POINTER(ctypes.c_float)


@pytest.fixture(scope="module")
def lib():
    build.build()
    return tg.lib()


def _create(lib, s, **over):
    """tg_basis_create on the arrays of a synthetic system, with overrides;
    returns (status, handle)."""
    a = {"natom": int(s["natom"]), "xyz": np.ascontiguousarray(s["xyz"], np.float64),
         "nshell": len(s["shell_l"]), "shell_atom": np.ascontiguousarray(s["shell_atom"], np.int32),
         "shell_l": np.ascontiguousarray(s["shell_l"], np.int32),
         "shell_nprim": np.ascontiguousarray(s["shell_nprim"], np.int32),
         "exps": np.ascontiguousarray(s["exps"], np.float64), "coefs": np.ascontiguousarray(s["coefs"], np.float64)}
    a.update(over)
    ptr = lambda x, t: None if x is None else x.ctypes.data_as(t)
    h = ctypes.c_void_p(12345)
    rc = lib.tg_basis_create(a["natom"], ptr(a["xyz"], _dp), a["nshell"], ptr(a["shell_atom"], _ip),
                             ptr(a["shell_l"], _ip), ptr(a["shell_nprim"], _ip), ptr(a["exps"], _dp),
                             ptr(a["coefs"], _dp), ctypes.byref(h))
    return rc, h.value


def test_basis_argument_checks(lib):
    s = synth.molecule(3, 1, 2)
    bad = {
        "natom": 0,
        "nshell": 0,
        "xyz": None,
        "exps": None,
        "shell_atom": np.full(len(s["shell_l"]), s["natom"], np.int32),
        "shell_nprim": np.zeros(len(s["shell_l"]), np.int32),
    }
    for k, v in bad.items():
        rc, h = _create(lib, s, **{k: v})
        assert rc == tg.TG_EINVAL, k
        assert h is None, k  # *out is cleared on error
    nprim17 = np.array(s["shell_nprim"], np.int32)
    nprim17[0] = 17
    assert _create(lib, s, shell_nprim=nprim17)[0] == tg.TG_EINVAL
    lneg = np.array(s["shell_l"], np.int32)
    lneg[1] = -1
    assert _create(lib, s, shell_l=lneg)[0] == tg.TG_EINVAL
    lf = np.array(s["shell_l"], np.int32)
    lf[1] = 3
    assert _create(lib, s, shell_l=lf)[0] == tg.TG_EUNSUPPORTED
    for bad_exp in (0.0, -1.0, np.nan, np.inf):
        e = np.array(s["exps"], np.float64)
        e[2] = bad_exp
        assert _create(lib, s, exps=e)[0] == tg.TG_EINVAL
    c = np.array(s["coefs"], np.float64)
    c[0] = np.nan
    assert _create(lib, s, coefs=c)[0] == tg.TG_EINVAL
    x = np.array(s["xyz"], np.float64)
    x[0, 1] = np.inf
    assert _create(lib, s, xyz=x)[0] == tg.TG_EINVAL


def test_no_cpu_fallback_without_a_device(lib):
    """A valid basis needs the GPU: without one the library returns
    TG_ECUDA instead of computing anything on the host."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    rc, h = _create(lib, synth.molecule(3, 1, 2))
    assert rc == tg.TG_ECUDA
    assert h is None


def test_null_handles_are_rejected(lib):
    g = np.zeros(3)
    st = tg.tg_stats()
    opt = tg.tg_options_default()
    arr = (tg.tg_pair * 1)()
    assert lib.tg_grad2e(None, 1, arr, ctypes.byref(opt), g.ctypes.data_as(_dp), ctypes.byref(st)) == tg.TG_EINVAL
    assert lib.tg_grad2e_sph(None, 1, arr, ctypes.byref(opt), g.ctypes.data_as(_dp),
                             ctypes.byref(st)) == tg.TG_EINVAL
    assert lib.tg_basis_nbf(None) == tg.TG_EINVAL
    assert lib.tg_basis_natom(None) == tg.TG_EINVAL
    assert lib.tg_basis_nsph(None) == tg.TG_EINVAL
    lib.tg_basis_destroy(None)  # no-op
    out = ctypes.c_void_p()
    assert lib.tg_batch_create(0, None, None, None, None, ctypes.byref(out)) == tg.TG_EINVAL
    assert lib.tg_batch_run(None, None, None, None) == tg.TG_EINVAL
    n = ctypes.c_int(-1)
    f = np.zeros(16, np.float32)
    assert lib.tg_tile_samples(None, 1, arr, None, 1, 1, f.ctypes.data_as(_fp), f.ctypes.data_as(_fp),
                               f.ctypes.data_as(_fp), ctypes.byref(n)) == tg.TG_EINVAL


def test_noalloc_entry_point_checks_sizes_before_any_device_call(lib):
    fn = lib.tg_router_loss_grad_noalloc
    fn.argtypes = [ctypes.c_int] + [ctypes.c_void_p] * 5 + [ctypes.c_float] + [ctypes.c_void_p] * 3
    fn.restype = ctypes.c_int
    p = ctypes.c_void_p(16)  # never dereferenced: the checks return first
    assert fn(0, p, p, p, p, p, 0.9, p, p, None) == tg.TG_EINVAL
    assert fn(10, p, p, p, p, p, 1.5, p, p, None) == tg.TG_EINVAL
    assert fn(10, None, p, p, p, p, 0.9, p, p, None) == tg.TG_EINVAL
    assert fn(65537, p, p, p, p, p, 0.9, p, p, None) == tg.TG_EUNSUPPORTED


def test_router_initialisation_is_seeded_xavier():
    """16-32-32-1 perceptron: W1[32][16], b1, W2[32][32], b2, w3[32], b3 with
    Xavier-uniform weights in +-sqrt(6/(fan_in+fan_out)) and zero biases."""
    assert tg.lib().tg_router_nparam() == 16 * 32 + 32 + 32 * 32 + 32 + 32 + 1
    p1 = tg.Router(seed=7).get()[0]
    p2 = tg.Router(seed=7).get()[0]
    p3 = tg.Router(seed=8).get()[0]
    assert np.array_equal(p1, p2) and not np.array_equal(p1, p3)
    o = 0
    for fin, fout in ((16, 32), (32, 32), (32, 1)):
        w = p1[o:o + fin * fout]
        o += fin * fout
        b = p1[o:o + fout]
        o += fout
        lim = np.sqrt(6.0 / (fin + fout))
        assert np.abs(w).max() <= lim and np.abs(w).max() > 0.5 * lim
        assert abs(float(w.mean())) < 0.25 * lim
        assert np.all(b == 0)
    _, mu, sd, cal = tg.Router(seed=7).get()
    assert np.all(mu == 0) and np.all(sd == 1) and cal[2] == 0  # untrained


def test_router_set_validates_before_changing_anything():
    r = tg.Router(seed=3)
    before = [a.copy() for a in r.get()]
    p = before[0].copy()
    p[5] = np.nan
    sd = np.ones(16, np.float32)
    sd[4] = 0.0
    for kw in ({"params": p}, {"sd": sd}, {"params": before[0] + 1, "sd": sd},
               {"calib": [np.inf, 1e-6, 1]}, {"calib": [0.0, -1.0, 1]}, {"mu": np.full(16, np.nan)}):
        with pytest.raises(tg.TGError) as e:
            r.set(**kw)
        assert e.value.status == tg.TG_EINVAL
        for a, b in zip(before, r.get()):
            assert np.array_equal(a, b)
    r.set(params=before[0] * 2, calib=[0.25, 2e-6, 1.0])
    p2, _, _, cal = r.get()
    assert np.array_equal(p2, before[0] * 2)
    assert cal[0] == np.float32(0.25) and cal[1] == np.float32(2e-6) and cal[2] == 1


def test_router_file_format(tmp_path):
    r = tg.Router(seed=21)
    mu = np.linspace(-1, 1, 16).astype(np.float32)
    sd = np.linspace(0.5, 2, 16).astype(np.float32)
    r.set(mu=mu, sd=sd, calib=[-0.5, 3e-6, 1.0])
    f = tmp_path / "r.bin"
    r.save(str(f))
    raw = f.read_bytes()
    n = tg.lib().tg_router_nparam()
    assert len(raw) == 16 + 4 * (n + 16 + 16 + 3)
    assert struct.unpack("<4i", raw[:16]) == (0x54524754, 1, 16, 32)
    vals = np.frombuffer(raw[16:], dtype="<f4")
    p, mu2, sd2, cal = r.get()
    assert np.array_equal(vals[:n], p)
    assert np.array_equal(vals[n:n + 16], mu) and np.array_equal(vals[n + 16:n + 32], sd)
    assert np.array_equal(vals[n + 32:], cal)
    r2 = tg.Router(path=str(f))
    for a, b in zip(r.get(), r2.get()):
        assert np.array_equal(a, b)


def test_router_load_rejects_foreign_files(tmp_path):
    good = tmp_path / "good.bin"
    tg.Router(seed=2).save(str(good))
    raw = bytearray(good.read_bytes())
    cases = {
        "missing": None,
        "short": bytes(raw[:100]),
        "magic": b"XXXX" + bytes(raw[4:]),
        "version": bytes(raw[:4]) + struct.pack("<i", 2) + bytes(raw[8:]),
        "width": bytes(raw[:12]) + struct.pack("<i", 64) + bytes(raw[16:]),
    }
    n = tg.lib().tg_router_nparam()
    nanp = bytearray(raw)
    nanp[16 + 4 * 7:16 + 4 * 8] = struct.pack("<f", float("nan"))
    cases["nan weight"] = bytes(nanp)
    zsd = bytearray(raw)
    zsd[16 + 4 * (n + 16):16 + 4 * (n + 17)] = struct.pack("<f", 0.0)
    cases["zero sd"] = bytes(zsd)
    for name, data in cases.items():
        f = tmp_path / ("bad_%s.bin" % name.replace(" ", "_"))
        if data is not None:
            f.write_bytes(data)
        h = ctypes.c_void_p(99)
        rc = tg.lib().tg_router_load(str(f).encode(), ctypes.byref(h))
        assert rc == tg.TG_EROUTER, name
        assert h.value is None, name


def test_shipped_router_loads_and_is_trained():
    import json
    import os
    d = os.path.join(os.path.dirname(tg.__file__), "data")
    r = tg.Router(path=os.path.join(d, "router.bin"))
    p, mu, sd, cal = r.get()
    info = json.load(open(os.path.join(d, "router.bin.json")))
    assert cal[2] == 1
    assert abs(float(cal[0]) - info["margin"]) <= 1e-6
    assert abs(float(cal[1]) - info["eps_rel"]) <= 1e-6 * info["eps_rel"]
    assert np.all(np.isfinite(p)) and np.all(sd > 0)


def test_every_status_has_its_own_message(lib):
    codes = [tg.TG_OK, tg.TG_EINVAL, tg.TG_EUNSUPPORTED, tg.TG_ENOMEM, tg.TG_ECUDA, tg.TG_ETIMEOUT, tg.TG_EROUTER]
    msgs = [tg.tg_strerror(c) for c in codes]
    assert len(set(msgs)) == len(codes)
    assert not any("unknown" in m for m in msgs)
