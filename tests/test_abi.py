"""C-ABI boundary checks that need no GPU: the library loads, exports every entry point the
public header declares, and rejects invalid arguments before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nudft2_hss.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nudft2_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def cdll():
    from paper_2607_00928_b300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ["nudft2_hss_build", "nudft2_hss_factor", "nudft2_hss_solve", "nudft2_hss_apply", "nudft2_hss_free"]:
        assert f in names


def test_library_exports_every_declared_symbol(cdll):
    missing = [f for f in declared_functions() if not hasattr(cdll, f)]
    assert not missing, missing


def test_invalid_arguments_are_rejected_on_the_host(cdll):
    from paper_2607_00928_b300.binding import EINVAL, ESTATE, Opts
    cdll.nudft2_hss_build.restype = ctypes.c_int
    cdll.nudft2_hss_factor.restype = ctypes.c_int
    cdll.nudft2_last_error.restype = ctypes.c_char_p
    h = ctypes.c_void_p()
    # NULL points
    assert cdll.nudft2_hss_build(None, None, ctypes.c_int64(512), 16, 16, None, None, ctypes.byref(h)) == EINVAL
    # M < N (checked before any device access)
    fake = ctypes.c_void_p(1)
    assert cdll.nudft2_hss_build(fake, fake, ctypes.c_int64(100), 16, 16, None, None, ctypes.byref(h)) == EINVAL
    assert b"M >= N" in cdll.nudft2_last_error()
    # eps outside (0, 1)
    o = Opts(2.0, 0, 64, 0, 1e-8, 4, 0)
    assert cdll.nudft2_hss_build(fake, fake, ctypes.c_int64(512), 16, 16, ctypes.byref(o), None,
                                 ctypes.byref(h)) == EINVAL
    # factor on a NULL handle is an ordering error
    assert cdll.nudft2_hss_factor(None, None) == ESTATE


def test_batched_entry_points_reject_bad_arguments_on_the_host(cdll):
    from paper_2607_00928_b300.binding import EINVAL
    cdll.nudft2_hss_build_batched.restype = ctypes.c_int
    cdll.nudft2_hss_solve_batched.restype = ctypes.c_int
    cdll.nudft2_last_error.restype = ctypes.c_char_p
    assert cdll.nudft2_hss_build_batched(0, None, None, None, None, None, None, 1, 4, None, None, None) == EINVAL
    assert b"build_batched" in cdll.nudft2_last_error()
    assert cdll.nudft2_hss_solve_batched(3, None, None, None, None, None, None, 4, None, None) == EINVAL
    assert b"solve_batched" in cdll.nudft2_last_error()


def test_header_is_plain_c(tmp_path):
    """The boundary header compiles as C99 on its own (no C++ or torch types leak into it)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_header.c"
    src.write_text('#include "nudft2_hss.h"\nint main(void) { return 0; }\n')
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-fsyntax-only", "-I", inc, str(src)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_factor_store_header_is_checked_on_the_host(cdll, tmp_path):
    """nudft2_hss_load validates the file header before any device work: a missing file, a file
    that is not a factor store, one of another version and a truncated header are all EINVAL, and
    *out stays NULL."""
    import struct
    from paper_2607_00928_b300.binding import EINVAL
    cdll.nudft2_hss_load.restype = ctypes.c_int
    cdll.nudft2_hss_load.argtypes = [ctypes.c_char_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    out = ctypes.c_void_p()
    assert cdll.nudft2_hss_load(str(tmp_path / "missing.bin").encode(), None, ctypes.byref(out)) == EINVAL
    junk = tmp_path / "junk.bin"
    junk.write_bytes(b"not a factor store at all" * 4)
    assert cdll.nudft2_hss_load(str(junk).encode(), None, ctypes.byref(out)) == EINVAL
    magic = struct.pack("<II", 0x4644554E, 0x53483254)
    other = tmp_path / "other.bin"
    other.write_bytes(magic + struct.pack("<II", 999, 48) + bytes(64))
    assert cdll.nudft2_hss_load(str(other).encode(), None, ctypes.byref(out)) == EINVAL
    short = tmp_path / "short.bin"
    short.write_bytes(magic + struct.pack("<I", 1))
    assert cdll.nudft2_hss_load(str(short).encode(), None, ctypes.byref(out)) == EINVAL
    assert out.value is None
