"""The C-ABI library loads here (no GPU) and exports every symbol that
include/tdgrad.h declares; no compute call is made."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tdgrad.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tg_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_api():
    names = _declared()
    for n in ("tg_basis_create", "tg_grad2e", "tg_strerror", "tg_options_default", "tg_basis_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2407_16586_gb300 import build
    import paper_2407_16586_gb300 as tg
    build.build()
    lib = ctypes.CDLL(tg.LIB_PATH)
    for n in _declared():
        assert hasattr(lib, n), n
    assert set(tg.EXPORTS) <= set(_declared())


def test_strerror_and_defaults_without_gpu():
    import paper_2407_16586_gb300 as tg
    o = tg.tg_options_default()
    assert o.screen_tol == 1e-10 and o.nranks == 1 and o.precision == tg.TG_FP64
    assert tg.tg_strerror(tg.TG_EINVAL) == "invalid argument"
    assert "unknown" in tg.tg_strerror(-99)


def test_abi_version_and_named_option_defaults():
    import paper_2407_16586_gb300 as tg
    src = open(os.path.join(ROOT, "include", "tdgrad.h")).read()
    ver = int(re.search(r"#define TG_ABI_VERSION (\d+)", src).group(1))
    L = tg.lib()
    L.tg_abi_version.restype = ctypes.c_int
    assert L.tg_abi_version() == ver
    o = tg.tg_options_default()
    assert o.deterministic == 1 and o.class_mask == 0 and o.kernel_kind == 0 and o.autotune == 0
    assert list(o.reserved) == [0, 0, 0] and o.shard_mode == 0
