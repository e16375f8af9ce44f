"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports every function that
include/sq.h declares (no compute calls: there may be no GPU here)."""
import ctypes
import os
import re

import pytest

from paper_2011_13517_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(sq_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["sq_build_hamiltonian", "sq_density", "sq_fermi_level", "sq_energy", "sq_nonlocal_force"]:
        assert required in names


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu():
    lib = ctypes.CDLL(build.build())
    lib.sq_status_string.restype = ctypes.c_char_p
    for code in range(10):
        assert lib.sq_status_string(code)
    assert b"unknown" in lib.sq_status_string(99)


def test_binding_names_match_the_abi():
    from paper_2011_13517_gb300 import sq
    for name in declared_functions():
        if name in ("sq_status_string", "sq_last_error", "sq_get_moments"):
            continue
        assert hasattr(sq, name), name
