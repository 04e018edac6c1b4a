"""tdgrad: the two-electron term of the TDA-TDDFT nuclear gradient on GB300.

Thin ctypes binding of libtdgrad.so (C-ABI in include/tdgrad.h).  It only
marshals arguments: every step of the gradient runs in the library's CUDA
kernels.  There is no CPU fallback; a missing library raises.

The functions keep the C names (tg_basis_create, tg_grad2e, ...).  ``Basis``
and ``grad2e`` are conveniences over them for dict-shaped systems such as
those returned by ``paper_2407_16586_gb300.synth``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtdgrad.so")

TG_OK = 0
TG_EINVAL = -1
TG_EUNSUPPORTED = -2
TG_ENOMEM = -3
TG_ECUDA = -4
TG_ETIMEOUT = -5
TG_EROUTER = -6

TG_FP64 = 0
TG_MIXED_BOUND = 1
TG_MIXED_LEARNED = 2
TG_FP32 = 3
TG_MAX_PAIRS = 8
TG_SHARD_PAIR_KEY = 0
TG_SHARD_TILES = 1

EXPORTS = ("tg_options_default", "tg_abi_version", "tg_class_flops", "tg_tile_shard", "tg_fock2e", "tg_basis_create", "tg_basis_nbf", "tg_basis_natom", "tg_basis_nsph", "tg_basis_destroy",
           "tg_grad2e", "tg_grad2e_sph", "tg_strerror", "tg_tile_samples", "tg_router_nparam", "tg_router_create",
           "tg_router_destroy", "tg_router_get", "tg_router_set", "tg_router_train", "tg_router_loss_grad",
           "tg_router_predict", "tg_router_save", "tg_router_load", "tg_batch_create", "tg_batch_run",
           "tg_batch_destroy")
NFEAT = 16


class tg_pair(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("B", ctypes.c_void_p), ("c_J", ctypes.c_double),
                ("c_K", ctypes.c_double), ("c_K_lr", ctypes.c_double), ("omega", ctypes.c_double)]


class tg_fpair(ctypes.Structure):
    _fields_ = [("B", ctypes.c_void_p), ("c_J", ctypes.c_double), ("c_K", ctypes.c_double),
                ("c_K_lr", ctypes.c_double), ("omega", ctypes.c_double)]


class tg_options(ctypes.Structure):
    _fields_ = [("screen_tol", ctypes.c_double), ("precision", ctypes.c_int), ("router", ctypes.c_void_p),
                ("mixed_tol", ctypes.c_double), ("device_ptrs", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("rank", ctypes.c_int), ("nranks", ctypes.c_int), ("timing", ctypes.c_int),
                ("autotune", ctypes.c_int), ("kernel_kind", ctypes.c_int), ("deterministic", ctypes.c_int),
                ("class_mask", ctypes.c_uint), ("shard_mode", ctypes.c_int), ("reserved", ctypes.c_int * 3)]


class tg_stats(ctypes.Structure):
    _fields_ = [("seconds", ctypes.c_double), ("quartets", ctypes.c_longlong), ("prim_quartets", ctypes.c_longlong),
                ("fp32_quartets", ctypes.c_longlong), ("pairs", ctypes.c_longlong), ("tiles", ctypes.c_longlong),
                ("launches", ctypes.c_int), ("grid", ctypes.c_int), ("class_ms", ctypes.c_double * 21),
                ("class_ms_fp32", ctypes.c_double * 21), ("class_quartets", ctypes.c_longlong * 21),
                ("class_prim_quartets", ctypes.c_longlong * 21),
                ("class_prim_quartets_fp32", ctypes.c_longlong * 21), ("class_bra_prims", ctypes.c_longlong * 21),
                ("class_bra_prims_fp32", ctypes.c_longlong * 21), ("plan_ms", ctypes.c_double),
                ("fp64_flop", ctypes.c_double), ("fp32_flop", ctypes.c_double),
                ("fp64_frac_peak", ctypes.c_double), ("fp32_frac_peak", ctypes.c_double)]

    def as_dict(self):
        out = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            out[k] = list(v) if hasattr(v, "_length_") else v
        return out


class TGError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s failed: %s (%d)" % (where, tg_strerror(status), status))


_lib = None


def lib():
    """The loaded libtdgrad.so.  Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libtdgrad.so is not built (run paper_2407_16586_gb300.build.build()); "
                               "there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        vp, ip, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
        L.tg_options_default.argtypes = [ctypes.POINTER(tg_options)]
        L.tg_options_default.restype = None
        L.tg_basis_create.argtypes = [ctypes.c_int, dp, ctypes.c_int, ip, ip, ip, dp, dp, ctypes.POINTER(vp)]
        L.tg_basis_create.restype = ctypes.c_int
        L.tg_basis_nbf.argtypes = [vp]
        L.tg_basis_nbf.restype = ctypes.c_int
        L.tg_basis_natom.argtypes = [vp]
        L.tg_basis_natom.restype = ctypes.c_int
        L.tg_basis_destroy.argtypes = [vp]
        L.tg_basis_destroy.restype = None
        L.tg_grad2e.argtypes = [vp, ctypes.c_int, ctypes.POINTER(tg_pair), ctypes.POINTER(tg_options), vp,
                                ctypes.POINTER(tg_stats)]
        L.tg_grad2e.restype = ctypes.c_int
        L.tg_grad2e_sph.argtypes = L.tg_grad2e.argtypes
        L.tg_grad2e_sph.restype = ctypes.c_int
        L.tg_basis_nsph.argtypes = [vp]
        L.tg_basis_nsph.restype = ctypes.c_int
        L.tg_strerror.argtypes = [ctypes.c_int]
        L.tg_strerror.restype = ctypes.c_char_p
        fp = ctypes.POINTER(ctypes.c_float)
        L.tg_tile_samples.argtypes = [vp, ctypes.c_int, ctypes.POINTER(tg_pair), ctypes.POINTER(tg_options),
                                      ctypes.c_int, ctypes.c_int, fp, fp, fp, ctypes.POINTER(ctypes.c_int)]
        L.tg_router_nparam.argtypes = []
        L.tg_router_create.argtypes = [ctypes.c_ulonglong, ctypes.POINTER(vp)]
        L.tg_router_destroy.argtypes = [vp]
        L.tg_router_destroy.restype = None
        L.tg_router_get.argtypes = [vp, fp, fp, fp, fp]
        L.tg_router_set.argtypes = [vp, fp, fp, fp, fp]
        L.tg_router_train.argtypes = [vp, ctypes.c_int, fp, fp, ctypes.c_int, ctypes.c_float, ctypes.c_float, fp]
        L.tg_router_loss_grad.argtypes = [vp, ctypes.c_int, fp, fp, ctypes.c_float, fp, fp]
        L.tg_router_predict.argtypes = [vp, ctypes.c_int, fp, fp]
        L.tg_router_save.argtypes = [vp, ctypes.c_char_p]
        L.tg_router_load.argtypes = [ctypes.c_char_p, ctypes.POINTER(vp)]
        L.tg_batch_create.argtypes = [ctypes.c_int, ctypes.POINTER(vp), ip, ctypes.POINTER(ctypes.POINTER(tg_pair)),
                                      ctypes.POINTER(tg_options), ctypes.POINTER(vp)]
        L.tg_batch_run.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(tg_options), ctypes.POINTER(tg_stats)]
        L.tg_batch_destroy.argtypes = [vp]
        L.tg_batch_destroy.restype = None
        for n in ("tg_batch_create", "tg_batch_run", "tg_tile_samples", "tg_router_nparam", "tg_router_create", "tg_router_get", "tg_router_set",
                  "tg_router_train", "tg_router_loss_grad", "tg_router_predict", "tg_router_save",
                  "tg_router_load"):
            getattr(L, n).restype = ctypes.c_int
        _lib = L
    return _lib


def tg_class_flops(qc, nops=2):
    """(FLOPs per primitive quartet, FLOPs per bra primitive pair) of angular
    class qc in the library's algorithmic count."""
    a, b = ctypes.c_double(0.0), ctypes.c_double(0.0)
    L = lib()
    L.tg_class_flops.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_double)]
    L.tg_class_flops.restype = ctypes.c_int
    rc = L.tg_class_flops(int(qc), int(nops), ctypes.byref(a), ctypes.byref(b))
    if rc != TG_OK:
        raise TGError(rc, "tg_class_flops")
    return a.value, b.value


def tg_tile_shard(ntiles, rank, nranks):
    """(first, count, stride) of the tiles of a list of ntiles that rank
    evaluates under TG_SHARD_TILES."""
    L = lib()
    ll = ctypes.c_longlong
    L.tg_tile_shard.argtypes = [ll, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ll), ctypes.POINTER(ll),
                                ctypes.POINTER(ll)]
    L.tg_tile_shard.restype = ctypes.c_int
    a, b, c = ll(0), ll(0), ll(0)
    rc = L.tg_tile_shard(int(ntiles), int(rank), int(nranks), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    if rc != TG_OK:
        raise TGError(rc, "tg_tile_shard")
    return a.value, b.value, c.value


def tg_strerror(status):
    return lib().tg_strerror(int(status)).decode()


def tg_options_default():
    o = tg_options()
    lib().tg_options_default(ctypes.byref(o))
    return o


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def tg_basis_create(natom, xyz, nshell, shell_atom, shell_l, shell_nprim, exps, coefs):
    xyz, shell_atom, shell_l = _c(xyz, np.float64), _c(shell_atom, np.int32), _c(shell_l, np.int32)
    shell_nprim, exps, coefs = _c(shell_nprim, np.int32), _c(exps, np.float64), _c(coefs, np.float64)
    h = ctypes.c_void_p()
    dp, ip = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    rc = lib().tg_basis_create(int(natom), xyz.ctypes.data_as(dp), int(nshell), shell_atom.ctypes.data_as(ip),
                               shell_l.ctypes.data_as(ip), shell_nprim.ctypes.data_as(ip), exps.ctypes.data_as(dp),
                               coefs.ctypes.data_as(dp), ctypes.byref(h))
    if rc != TG_OK:
        raise TGError(rc, "tg_basis_create")
    return h


def tg_basis_nbf(h):
    return lib().tg_basis_nbf(h)


def tg_basis_natom(h):
    return lib().tg_basis_natom(h)


def tg_basis_nsph(h):
    return lib().tg_basis_nsph(h)


def tg_basis_destroy(h):
    lib().tg_basis_destroy(h)


def tg_grad2e(h, pairs, options=None, grad_ptr=None, natom=None, spherical=False):
    """pairs: list of (A_ptr, B_ptr, c_J, c_K, c_K_lr, omega) with raw pointers
    (host or device per options.device_ptrs).  grad_ptr: raw output pointer;
    spherical: the matrices are over spherical functions (tg_grad2e_sph).
    Returns (status, tg_stats)."""
    arr = (tg_pair * len(pairs))()
    for i, (a, b, cj, ck, cl, om) in enumerate(pairs):
        arr[i] = tg_pair(a, b, cj, ck, cl, om)
    st = tg_stats()
    opt = options if options is not None else tg_options_default()
    fn = lib().tg_grad2e_sph if spherical else lib().tg_grad2e
    rc = fn(h, len(pairs), arr, ctypes.byref(opt), grad_ptr, ctypes.byref(st))
    return rc, st


class Basis:
    """Owns a tg_basis handle built from a dict-shaped system."""

    def __init__(self, system):
        self.natom = int(system["natom"])
        self.nshell = len(system["shell_l"])
        self.h = tg_basis_create(self.natom, system["xyz"], self.nshell, system["shell_atom"], system["shell_l"],
                                 system["shell_nprim"], system["exps"], system["coefs"])
        self.nbf = tg_basis_nbf(self.h)
        self.nsph = tg_basis_nsph(self.h)

    def close(self):
        if self.h is not None:
            tg_basis_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _plist(self, pairs):
        keep, plist = [], []
        for (a, b, cj, ck, cl, om) in pairs:
            a, b = _c(a, np.float64), _c(b, np.float64)
            keep += [a, b]
            plist.append((a.ctypes.data, b.ctypes.data, float(cj), float(ck), float(cl), float(om)))
        return keep, plist

    def tile_samples(self, pairs, stride=50, cap=100000, screen_tol=1e-10):
        """Router training data: (features [n,16], log10 max|fp64 contribution|,
        log10 max|fp32 - fp64|) for every stride-th screened tile."""
        keep, plist = self._plist(pairs)
        arr = (tg_pair * len(plist))(*[tg_pair(*p) for p in plist])
        opt = tg_options_default()
        opt.screen_tol = float(screen_tol)
        X = np.zeros((cap, NFEAT), dtype=np.float32)
        y = np.zeros(cap, dtype=np.float32)
        e = np.zeros(cap, dtype=np.float32)
        n = ctypes.c_int(0)
        f = ctypes.POINTER(ctypes.c_float)
        rc = lib().tg_tile_samples(self.h, len(plist), arr, ctypes.byref(opt), int(stride), int(cap),
                                   X.ctypes.data_as(f), y.ctypes.data_as(f), e.ctypes.data_as(f), ctypes.byref(n))
        if rc != TG_OK:
            raise TGError(rc, "tg_tile_samples")
        return X[:n.value].copy(), y[:n.value].copy(), e[:n.value].copy()

    def fock2e(self, pairs, screen_tol=0.0, timing=False, stream=None):
        """Fock-type matrix (nbf x nbf) of host pairs [(B, c_J, c_K, c_K_lr, omega)]
        (tg_fock2e) and the call's statistics."""
        L = lib()
        L.tg_fock2e.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(tg_fpair), ctypes.POINTER(tg_options),
                                ctypes.c_void_p, ctypes.POINTER(tg_stats)]
        L.tg_fock2e.restype = ctypes.c_int
        opt = tg_options_default()
        opt.screen_tol = float(screen_tol)
        opt.timing = 1 if timing else 0
        if stream is not None:
            opt.stream = ctypes.c_void_p(stream)
        keep = [_c(b, np.float64) for (b, *_r) in pairs]
        arr = (tg_fpair * len(pairs))(*[tg_fpair(k.ctypes.data, float(cj), float(ck), float(cl), float(om))
                                        for k, (_b, cj, ck, cl, om) in zip(keep, pairs)])
        n = keep[0].shape[0]
        F = np.zeros((n, n))
        st = tg_stats()
        rc = L.tg_fock2e(self.h, len(pairs), arr, ctypes.byref(opt), ctypes.c_void_p(F.ctypes.data), ctypes.byref(st))
        if rc != TG_OK:
            raise TGError(rc, "tg_fock2e")
        return F, st.as_dict()

    def grad2e(self, pairs, screen_tol=1e-10, precision=TG_FP64, rank=0, nranks=1, stream=None, out=None,
               timing=False, router=None, mixed_tol=1e-6, kernel=0, class_mask=0, shard_mode=0, autotune=0,
               spherical=False):
        """Gradient (natom x 3) of host numpy pairs [(A, B, c_J, c_K, c_K_lr, omega)], or of
        torch CUDA tensors (then the densities and ``out`` stay on the device).  ``kernel``
        picks the class kernels: 0 per-class default, 1 one quartet per thread, 2 a thread
        group per quartet where compiled, 3 a warp per quartet where compiled.  ``class_mask``
        (0 = all) keeps the angular classes whose bits are set.  ``autotune`` 1 tunes the
        launches of every class list on this basis's first such call and reuses them, 2
        tunes again (tg_options.autotune).  ``spherical``: the matrices are nsph x nsph over
        spherical functions (tg_grad2e_sph)."""
        opt = tg_options_default()
        opt.kernel_kind = int(kernel)
        opt.autotune = int(autotune)
        opt.class_mask = int(class_mask)
        opt.shard_mode = int(shard_mode)
        opt.screen_tol = float(screen_tol)
        opt.precision = int(precision)
        opt.rank, opt.nranks = int(rank), int(nranks)
        opt.timing = 1 if timing else 0
        opt.mixed_tol = float(mixed_tol)
        if router is not None:
            opt.router = router.h
        dev = hasattr(pairs[0][0], "is_cuda") and pairs[0][0].is_cuda
        keep = []
        plist = []
        for (a, b, cj, ck, cl, om) in pairs:
            if dev:
                a, b = a.contiguous(), b.contiguous()
                keep += [a, b]
                plist.append((a.data_ptr(), b.data_ptr(), float(cj), float(ck), float(cl), float(om)))
            else:
                a, b = _c(a, np.float64), _c(b, np.float64)
                keep += [a, b]
                plist.append((a.ctypes.data, b.ctypes.data, float(cj), float(ck), float(cl), float(om)))
        if dev:
            import torch
            opt.device_ptrs = 1
            opt.stream = ctypes.c_void_p(stream if stream is not None else torch.cuda.current_stream().cuda_stream)
            g = out if out is not None else torch.empty((self.natom, 3), dtype=torch.float64, device=pairs[0][0].device)
            rc, st = tg_grad2e(self.h, plist, opt, ctypes.c_void_p(g.data_ptr()), spherical=spherical)
        else:
            g = out if out is not None else np.zeros((self.natom, 3))
            if stream is not None:
                opt.stream = ctypes.c_void_p(stream)
            rc, st = tg_grad2e(self.h, plist, opt, ctypes.c_void_p(g.ctypes.data), spherical=spherical)
        if rc != TG_OK:
            raise TGError(rc, "tg_grad2e_sph" if spherical else "tg_grad2e")
        return g, st.as_dict()


def zfock_pairs(B, alpha, beta, omega):
    """The Z-vector's Fock-type matrix of eq. zfock (Sec. II.B, without the XC
    kernel term) as tg_fock2e pairs: sum_{lam sig} B[sig lam] [4 (mu nu|lam sig)
    - alpha ((mu lam|sig nu) + (mu sig|lam nu)) - beta (same)_lr] is the pair
    (B^T; 4, -alpha, -beta) plus (B; 0, -alpha, -beta)."""
    return [(np.ascontiguousarray(np.asarray(B).T), 4.0, -alpha, -beta, omega), (B, 0.0, -alpha, -beta, omega)]


def tda_pairs(P, P_delta, R, alpha, beta, omega):
    """The density pairs of the TDA excited-state gradient's two-electron
    term (Sec. II.A, eq. gamma): Gamma holds 2 R R (Coulomb-like), -alpha R R
    and -beta R R through the full and erf(omega r)/r operators (exchange-
    like), and the ground-state and relaxed-difference densities through
    D = P + 2 P_delta paired with P, with a factor 1/2 and exchange weights
    -alpha/4, -beta/4.  P is the ground-state density, P_delta the relaxed
    difference density and R the transition density (X in the AO basis),
    each nbf x nbf row-major, numpy arrays or torch CUDA tensors.

    Pairs are bilinear in their first matrix, so (D, P) is passed as
    (P, P) + 2 (P_delta, P): the list holds three pairs and the helper does no
    arithmetic on the matrices."""
    a, b = float(alpha), float(beta)
    return [(R, R, 2.0, -a, -b, omega),
            (P, P, 0.5, -a / 4.0, -b / 4.0, omega),
            (P_delta, P, 1.0, -a / 2.0, -b / 2.0, omega)]


def grad2e(system, pairs=None, **kw):
    """One-shot gradient of a dict-shaped system (builds and frees a Basis)."""
    b = Basis(system)
    try:
        return b.grad2e(system["pairs"] if pairs is None else pairs, **kw)
    finally:
        b.close()


class Router:
    """Owns a tg_router handle (16-32-32-1 tanh MLP trained on the GPU)."""

    def __init__(self, seed=0, path=None):
        self.h = ctypes.c_void_p()
        if path is not None:
            rc = lib().tg_router_load(os.fsencode(path), ctypes.byref(self.h))
            if rc != TG_OK:
                raise TGError(rc, "tg_router_load")
        else:
            rc = lib().tg_router_create(int(seed), ctypes.byref(self.h))
            if rc != TG_OK:
                raise TGError(rc, "tg_router_create")
        self.nparam = lib().tg_router_nparam()

    def close(self):
        if self.h is not None:
            lib().tg_router_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _f(a):
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))

    def get(self):
        p = np.zeros(self.nparam, np.float32)
        mu = np.zeros(NFEAT, np.float32)
        sd = np.zeros(NFEAT, np.float32)
        cal = np.zeros(3, np.float32)
        rc = lib().tg_router_get(self.h, self._f(p), self._f(mu), self._f(sd), self._f(cal))
        if rc != TG_OK:
            raise TGError(rc, "tg_router_get")
        return p, mu, sd, cal

    def set(self, params=None, mu=None, sd=None, calib=None):
        c = lambda a: None if a is None else np.ascontiguousarray(a, np.float32)
        params, mu, sd, calib = c(params), c(mu), c(sd), c(calib)
        nul = ctypes.POINTER(ctypes.c_float)()
        rc = lib().tg_router_set(self.h, *[nul if a is None else self._f(a) for a in (params, mu, sd, calib)])
        if rc != TG_OK:
            raise TGError(rc, "tg_router_set")

    def train(self, X, y, epochs=300, lr=1e-2, q=0.9):
        X = np.ascontiguousarray(X, np.float32)
        y = np.ascontiguousarray(y, np.float32)
        hist = np.zeros(epochs, np.float32)
        rc = lib().tg_router_train(self.h, len(y), self._f(X), self._f(y), int(epochs), float(lr), float(q),
                                   self._f(hist))
        if rc != TG_OK:
            raise TGError(rc, "tg_router_train")
        return hist

    def loss_grad(self, X, y, q=0.9):
        X = np.ascontiguousarray(X, np.float32)
        y = np.ascontiguousarray(y, np.float32)
        g = np.zeros(self.nparam, np.float32)
        L = np.zeros(1, np.float32)
        rc = lib().tg_router_loss_grad(self.h, len(y), self._f(X), self._f(y), float(q), self._f(L), self._f(g))
        if rc != TG_OK:
            raise TGError(rc, "tg_router_loss_grad")
        return float(L[0]), g

    def predict(self, X):
        X = np.ascontiguousarray(X, np.float32)
        out = np.zeros(len(X), np.float32)
        rc = lib().tg_router_predict(self.h, len(X), self._f(X), self._f(out))
        if rc != TG_OK:
            raise TGError(rc, "tg_router_predict")
        return out

    def save(self, path):
        rc = lib().tg_router_save(self.h, os.fsencode(path))
        if rc != TG_OK:
            raise TGError(rc, "tg_router_save")


class Batch:
    """Planned evaluation of many independent molecules (tg_batch_*): every
    molecule keeps its own Basis; run() replays one captured CUDA graph."""

    def __init__(self, systems, screen_tol=1e-10, precision=TG_FP64, router=None, mixed_tol=1e-6, autotune=False,
                 device=None):
        self.bases = [Basis(s) for s in systems]
        self.natoms = [int(s["natom"]) for s in systems]
        self._keep = []
        opt = tg_options_default()
        opt.screen_tol = float(screen_tol)
        opt.precision = int(precision)
        opt.mixed_tol = float(mixed_tol)
        if router is not None:
            opt.router = router.h
        if autotune:
            opt.autotune = 1
        parrs = []
        for s, b in zip(systems, self.bases):
            keep, plist = b._plist(s["pairs"])
            self._keep.append(keep)
            parrs.append((tg_pair * len(plist))(*[tg_pair(*p) for p in plist]))
        self._parrs = parrs
        n = len(systems)
        hs = (ctypes.c_void_p * n)(*[b.h for b in self.bases])
        npair = np.array([len(s["pairs"]) for s in systems], dtype=np.int32)
        pp = (ctypes.POINTER(tg_pair) * n)(*[ctypes.cast(a, ctypes.POINTER(tg_pair)) for a in parrs])
        self.h = ctypes.c_void_p()
        rc = lib().tg_batch_create(n, hs, npair.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), pp, ctypes.byref(opt),
                                   ctypes.byref(self.h))
        if rc != TG_OK:
            raise TGError(rc, "tg_batch_create")

    def run(self, stream=None):
        outs = [np.zeros((n, 3)) for n in self.natoms]
        ptrs = (ctypes.c_void_p * len(outs))(*[o.ctypes.data for o in outs])
        opt = tg_options_default()
        if stream is not None:
            opt.stream = ctypes.c_void_p(stream)
        st = tg_stats()
        rc = lib().tg_batch_run(self.h, ptrs, ctypes.byref(opt), ctypes.byref(st))
        if rc != TG_OK:
            raise TGError(rc, "tg_batch_run")
        return outs, st.as_dict()

    def close(self):
        if self.h is not None:
            lib().tg_batch_destroy(self.h)
            self.h = None
        for b in self.bases:
            b.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
