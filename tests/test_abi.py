"""The C-ABI library builds, loads and exports every entry point that
include/jsim.h declares (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

from paper_1911_04200_gb300 import build_native, jsim

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        names |= set(re.findall(r"JSIM_API\s+[\w\s\*]+?\b(jsim_\w+)\s*\(", text))
    return names


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ("jsim_create", "jsim_destroy", "jsim_all_pairs", "jsim_pack", "jsim_product", "jsim_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol():
    path = build_native.build()
    lib = ctypes.CDLL(path)
    missing = [s for s in sorted(declared_symbols()) if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_covers_header():
    assert set(jsim.SIGNATURES) == declared_symbols()


def test_host_only_entry_points():
    lib = jsim.load()
    assert lib.jsim_version().decode().startswith("jsim")
    assert lib.jsim_strerror(0) == b"ok"
    assert b"sorted" in lib.jsim_strerror(2)
    o = jsim.Options()
    lib.jsim_default_options(ctypes.byref(o))
    assert o.word_bits == 64 and o.count_bits == 32 and o.id_bits == 64 and o.variant == 0


def test_bad_options_rejected_before_any_device_call():
    lib = jsim.load()
    o = jsim.Options()
    lib.jsim_default_options(ctypes.byref(o))
    o.word_bits = 48
    h = ctypes.c_void_p()
    assert lib.jsim_create(ctypes.byref(h), ctypes.byref(o)) == 1
    lib.jsim_default_options(ctypes.byref(o))
    o.batch_rows = 100  # not a multiple of 64
    assert lib.jsim_create(ctypes.byref(h), ctypes.byref(o)) == 1
