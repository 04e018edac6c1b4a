"""CPU oracle for the two-electron TDA gradient term (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It wraps ``tdgrad_oracle.c`` (plain fp64 C,
OpenMP) through ctypes.  It shares no code with the CUDA library and the
product never calls it.

Functions follow the paper's Sec. II.C (Cartesian Gaussians eq. cartG, the
derivative rule eq. deriv, the centre decomposition eq. deri) and the AO
gradient's two-electron terms (eq. dE_ao with eq. gamma as (A, B, c) pairs).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tdgrad_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force=False):
    """Compile the oracle with gcc (OpenMP).  Idempotent."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-D_GNU_SOURCE",
           _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _configure(lib):
    """Declare the C signatures on a loaded build of tdgrad_oracle.c."""
    lib.or_boys.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp]
    lib.or_normalise.argtypes = [ctypes.c_int, _ip, _ip, _dp, _dp, _dp]
    basis_args = [ctypes.c_int, _dp, ctypes.c_int, _ip, _ip, _ip, _dp, _dp]
    lib.or_shell_eri.argtypes = basis_args + [ctypes.c_int] * 4 + [ctypes.c_double, _dp]
    lib.or_shell_eri_deriv.argtypes = basis_args + [ctypes.c_int] * 4 + [ctypes.c_double, _dp]
    lib.or_schwarz.argtypes = basis_args + [_dp, _dp]
    lib.or_grad2e.argtypes = basis_args + [
        ctypes.c_int, ctypes.POINTER(_dp), ctypes.POINTER(_dp), _dp, _dp, _dp, _dp,
        ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
        ctypes.c_int, _dp, _dp, ctypes.POINTER(ctypes.c_longlong), ctypes.c_int]
    lib.or_grad2e.restype = ctypes.c_int
    lib.or_fock2e.argtypes = basis_args + [
        ctypes.c_int, ctypes.POINTER(_dp), _dp, _dp, _dp, _dp, ctypes.c_int, _dp]
    lib.or_fock2e.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _configure(ctypes.CDLL(_LIB))
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _i(a):
    return a.ctypes.data_as(_ip)


class _Basis:
    def __init__(self, s):
        self.natom = int(s["natom"])
        self.xyz = np.ascontiguousarray(s["xyz"], dtype=np.float64)
        self.sh_atom = np.ascontiguousarray(s["shell_atom"], dtype=np.int32)
        self.sh_l = np.ascontiguousarray(s["shell_l"], dtype=np.int32)
        self.sh_nprim = np.ascontiguousarray(s["shell_nprim"], dtype=np.int32)
        self.exps = np.ascontiguousarray(s["exps"], dtype=np.float64)
        self.coefs = np.ascontiguousarray(s["coefs"], dtype=np.float64)

    def args(self):
        return [self.natom, _d(self.xyz), len(self.sh_l), _i(self.sh_atom), _i(self.sh_l),
                _i(self.sh_nprim), _d(self.exps), _d(self.coefs)]


def boys(mmax, T, branch=0):
    """[F_0(T) .. F_mmax(T)]; branch 1 = series+downward, 2 = erf+upward."""
    out = np.zeros(mmax + 1)
    _load().or_boys(mmax, float(T), branch, _d(out))
    return out


def normalised_coefs(s):
    b = _Basis(s)
    out = np.zeros_like(b.exps)
    _load().or_normalise(len(b.sh_l), _i(b.sh_l), _i(b.sh_nprim), _d(b.exps), _d(b.coefs), _d(out))
    return out


def _nc(l):
    return (l + 1) * (l + 2) // 2


def sph_transform(s):
    """Cartesian-to-spherical matrix T (ncart x nsph) of the basis, block
    diagonal over shells (Sec. II.C: the 2l+1 spherical functions of a shell
    follow from its Cartesian ones by a spherical transformation).  Column m
    of a shell's block holds the coefficients of spherical function m in its
    Cartesian components (x^l normalised, order xx xy xz yy yz zz for d):
      s: 1;  p: x, y, z;
      d: m = -2: sqrt3 xy, -1: sqrt3 yz, 0: zz - (xx + yy) / 2,
         +1: sqrt3 xz, +2: sqrt3 / 2 (xx - yy),
    the real solid harmonics r^2 Y_2m written in Cartesian monomials and
    scaled to unit norm.  A spherical-basis density A enters the Cartesian
    integrals as T A T^T."""
    ls = [int(l) for l in s["shell_l"]]
    nc = sum(_nc(l) for l in ls)
    ns = sum(2 * l + 1 for l in ls)
    T = np.zeros((nc, ns))
    r3 = np.sqrt(3.0)
    d = np.zeros((6, 5))
    # columns m = -2, -1, 0, +1, +2; rows xx, xy, xz, yy, yz, zz
    d[1, 0] = r3
    d[4, 1] = r3
    d[5, 2], d[0, 2], d[3, 2] = 1.0, -0.5, -0.5
    d[2, 3] = r3
    d[0, 4], d[3, 4] = r3 / 2.0, -r3 / 2.0
    i = j = 0
    for l in ls:
        if l < 2:
            T[i:i + _nc(l), j:j + 2 * l + 1] = np.eye(_nc(l))
        elif l == 2:
            T[i:i + 6, j:j + 5] = d
        else:
            raise ValueError("l > 2")
        i += _nc(l)
        j += 2 * l + 1
    return T


def shell_eri(s, a, b, c, d, omega=0.0):
    """Contracted (ab|cd) for one shell quartet; omega>0 selects erf(omega r)/r."""
    bs = _Basis(s)
    dims = [_nc(int(bs.sh_l[x])) for x in (a, b, c, d)]
    out = np.zeros(int(np.prod(dims)))
    _load().or_shell_eri(*bs.args(), a, b, c, d, float(omega), _d(out))
    return out.reshape(dims)


def shell_eri_deriv(s, a, b, c, d, omega=0.0):
    """d(ab|cd)/dX_i for X = a, b, c, d: array [4, 3, na, nb, nc, nd]."""
    bs = _Basis(s)
    dims = [_nc(int(bs.sh_l[x])) for x in (a, b, c, d)]
    out = np.zeros(12 * int(np.prod(dims)))
    _load().or_shell_eri_deriv(*bs.args(), a, b, c, d, float(omega), _d(out))
    return out.reshape([4, 3] + dims)


def schwarz(s):
    """(Q, Q') over all shell pairs, each nshell x nshell."""
    bs = _Basis(s)
    n = len(bs.sh_l)
    Q = np.zeros((n, n))
    Qd = np.zeros((n, n))
    _load().or_schwarz(*bs.args(), _d(Q), _d(Qd))
    return Q, Qd


def grad2e(s, pairs=None, mode="canonical", tau=0.0, rank=0, nranks=1, nthreads=0,
           want_grad=True, want_energy=False, xyz=None, qclass=-1):
    """Two-electron gradient (natom x 3, Ha/bohr) of the pair list.

    Returns (grad, energy, nquartets).  mode "plain" loops over all ordered
    shell quartets; "canonical" uses the 8-fold symmetry and supports
    screening (tau) and shards (rank, nranks).  qclass >= 0 keeps only the
    quartets of one angular class (0..20: the pair classes ss ps pp ds dp dd
    numbered 0..5, class P(P+1)/2 + Q for bra pair class P >= ket class Q)."""
    s2 = dict(s)
    if xyz is not None:
        s2["xyz"] = xyz
    bs = _Basis(s2)
    pairs = s["pairs"] if pairs is None else pairs
    npair = len(pairs)
    mats = [(np.ascontiguousarray(p[0], dtype=np.float64), np.ascontiguousarray(p[1], dtype=np.float64))
            for p in pairs]
    Ap = (_dp * max(npair, 1))(*[_d(m[0]) for m in mats])
    Bp = (_dp * max(npair, 1))(*[_d(m[1]) for m in mats])
    cJ = np.array([p[2] for p in pairs] + [0.0])
    cK = np.array([p[3] for p in pairs] + [0.0])
    cKlr = np.array([p[4] for p in pairs] + [0.0])
    om = np.array([p[5] for p in pairs] + [0.0])
    grad = np.zeros((bs.natom, 3))
    e = ctypes.c_double(0.0)
    nq = ctypes.c_longlong(0)
    rc = _load().or_grad2e(*bs.args(), npair, Ap, Bp, _d(cJ), _d(cK), _d(cKlr), _d(om),
                           0 if mode == "plain" else 1, float(tau), int(rank), int(nranks),
                           int(nthreads), 1 if want_grad else 0, _d(grad),
                           ctypes.byref(e) if want_energy else None, ctypes.byref(nq), int(qclass))
    if rc != 0:
        raise ValueError("oracle rejected its arguments")
    return grad, (e.value if want_energy else None), nq.value


def fock2e(s, pairs=None, nthreads=0):
    """Fock-type matrix (nbf x nbf) of the pair list [(B, c_J, c_K, c_K_lr, omega)]:
    F[mu nu] = sum_p sum_{lam sig} B[lam sig] (c_J (mu nu|lam sig) + c_K (mu lam|nu sig)
    + c_K_lr (mu lam|nu sig)_omega), the two-electron part of eqs. G_2e and zfock
    (Sec. II.B).  Plain definition over all ordered shell quartets."""
    bs = _Basis(s)
    npair = len(pairs)
    mats = [np.ascontiguousarray(p[0], dtype=np.float64) for p in pairs]
    nbf = mats[0].shape[0]
    Bp = (_dp * max(npair, 1))(*[_d(m) for m in mats])
    cJ = np.array([p[1] for p in pairs] + [0.0])
    cK = np.array([p[2] for p in pairs] + [0.0])
    cKlr = np.array([p[3] for p in pairs] + [0.0])
    om = np.array([p[4] for p in pairs] + [0.0])
    F = np.zeros((nbf, nbf))
    rc = _load().or_fock2e(*bs.args(), npair, Bp, _d(cJ), _d(cK), _d(cKlr), _d(om), int(nthreads), _d(F))
    if rc != 0:
        raise ValueError("oracle rejected its arguments")
    return F
