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


def _declaration_arities():
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for m in re.finditer(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*([a-z_][a-z_0-9]*)\s*\(([^)]*)\)\s*;", text, flags=re.M):
        args = m.group(2).strip()
        out[m.group(1)] = 0 if args in ("", "void") else args.count(",") + 1
    return out


def test_binding_argument_counts_match_header():
    from paper_2412_20884_gb300 import binding
    for name, n in _declaration_arities().items():
        assert len(binding._SIGS[name][1]) == n, (name, len(binding._SIGS[name][1]), n)


def test_struct_layouts_match_ctypes(tmp_path):
    """kmv_points and kmv_nystrom as the C compiler lays them out (gcc on the
    header) against the binding's ctypes structures: field order, offsets, size."""
    import shutil
    import subprocess
    from paper_2412_20884_gb300 import binding
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"kmv_points": binding._Points, "kmv_nystrom": binding._Nystrom}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "kmv.h"', "int main(void) {"]
    for cname, ct in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in ct._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        cname, field, val = line.split()
        got[(cname, field)] = int(val)
    for cname, ct in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(ct), cname
        for fname, _ in ct._fields_:
            assert got[(cname, fname)] == getattr(ct, fname).offset, (cname, fname)


def test_argument_errors_need_no_device(so):
    """Entry points reject bad arguments before any CUDA call (no GPU needed)."""
    from paper_2412_20884_gb300 import binding
    for name, (res, args) in binding._SIGS.items():
        getattr(so, name).restype = res
        getattr(so, name).argtypes = args
    EINVAL = 1
    # a NULL handle
    assert so.kmv_forward(None, None, 1, None, None, 1, None, None, None, 0, None) == EINVAL
    assert so.kmv_set_preconditioner(None, None) == EINVAL
    assert so.kmv_profile_enable(None, 1) == EINVAL
    # handle-free calls with bad sizes
    assert so.kmv_accept(4, 0, None, None, None, None, None, None, None, None) == EINVAL
    assert so.kmv_accept(4, 3, None, None, None, None, None, None, None, None) == EINVAL
    assert so.kmv_status_merge(-1, None, None, None) == EINVAL
    assert so.kmv_backward_noalloc(None, 1, None, None, None, 1, None, None, None) == EINVAL


def test_noalloc_applies_the_common_point_rules(so):
    """kmv_backward_noalloc checks the point set by the same rules as the
    handle-based entry points (before any CUDA call): too many systems
    (n_inst * chains > 2^30), too many rows, decreasing offsets; and the tile
    calls reject a NULL handle."""
    from paper_2412_20884_gb300 import binding
    f = so.kmv_backward_noalloc
    f.restype, f.argtypes = binding._SIGS["kmv_backward_noalloc"]
    EINVAL = 1
    dummy = ctypes.c_void_p(16)   # never dereferenced: the checks fail first

    def pts(offsets, d=2):
        arr = (ctypes.c_int64 * len(offsets))(*offsets)
        p = binding._Points(len(offsets) - 1, ctypes.cast(arr, ctypes.POINTER(ctypes.c_int64)), d, 1, dummy, 0)
        return p, arr

    # 2^15 empty instances x 2^15 + 1 chains: more than 2^30 systems, yet tiny scratch
    n_inst = 1 << 15
    p, keep = pts([0] * (n_inst + 1))
    assert f(ctypes.byref(p), (1 << 15) + 1, dummy, dummy, dummy, 1, dummy, None, None) == EINVAL
    p, keep = pts([0, 10, 5])
    assert f(ctypes.byref(p), 1, dummy, dummy, dummy, 1, dummy, None, None) == EINVAL
    p, keep = pts([0, (1 << 40) + 1])
    assert f(ctypes.byref(p), 1, dummy, dummy, dummy, 1, dummy, None, None) == EINVAL
    for name in ("kmv_set_tiles", "kmv_get_tiles"):
        g = getattr(so, name)
        g.restype, g.argtypes = binding._SIGS[name]
        assert g(None, 0, None) == EINVAL
    so.kmv_autotune.restype, so.kmv_autotune.argtypes = binding._SIGS["kmv_autotune"]
    assert so.kmv_autotune(None, None, 1, None, 1, None, None) == EINVAL
