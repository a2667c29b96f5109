"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/pf.h declares (no compute calls: this runs without a GPU)."""
import re
import subprocess

import pytest

from paper_2304_07338_b300 import _lib, build


def test_library_builds_and_exports_header():
    path = build.build()
    L = _lib.load(path)
    decl = set(re.findall(r"\b(pf_[a-z0-9_]+)\s*\(", open(build.INC + "/pf.h").read()))
    assert len(decl) >= 20
    syms = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in syms.splitlines() if " T " in l}
    assert decl <= exported, decl - exported
    assert decl == set(_lib.SIGNATURES), decl ^ set(_lib.SIGNATURES)
    for name in decl:
        assert getattr(L, name) is not None


def test_struct_layouts_match_header():
    import ctypes as C
    assert C.sizeof(_lib.PfVolume) == 80   # sizes as laid out by a C compiler for pf.h
    assert C.sizeof(_lib.PfLight) == 28
    assert C.sizeof(_lib.PfCamera) == 48
    assert C.sizeof(_lib.PfFieldDesc) == 56
    assert C.sizeof(_lib.PfTrainDesc) == 128
    assert _lib.PfCacheInfo.tally.offset == 48


def test_create_rejects_bad_device_without_gpu():
    import ctypes as C
    L = _lib.load()
    h = C.c_void_p()
    assert L.pf_create(C.byref(h), -1, None) == _lib.PF_ERR_INVALID_ARG
    assert not h.value
    assert L.pf_destroy(None) == _lib.PF_OK
