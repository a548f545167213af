"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports
every entry point include/kmv.h declares.  No compute call is made."""
import ctypes
import os
import re

import pytest

from paper_2412_20884_gb300 import build as kb

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "kmv.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*([a-z_][a-z_0-9]*)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def so():
    return ctypes.CDLL(kb.build_library())


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["kmv_forward", "kmv_backward", "leapfrog_step", "kmv_cg_solve", "kmv_energy",
              "kmv_create", "kmv_destroy", "kmv_status_string", "kmv_last_error"]:
        assert n in names, n


def test_library_exports_every_declared_symbol(so):
    for n in declared_functions():
        assert hasattr(so, n), f"libkmv.so does not export {n}"


def test_status_strings(so):
    so.kmv_status_string.restype = ctypes.c_char_p
    assert so.kmv_status_string(0) == b"ok"
    assert so.kmv_status_string(1) == b"invalid argument"
    assert so.kmv_status_string(99) == b"unknown status"


def test_binding_signatures_cover_header():
    from paper_2412_20884_gb300 import binding
    for n in declared_functions():
        assert n in binding._SIGS, n
