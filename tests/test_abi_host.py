"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function ``include/tsm2.h`` declares, and rejects bad arguments before
touching the device."""
import ctypes
import os
import re

import pytest

import paper_2002_03258_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include"))) if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b([A-Za-z_][A-Za-z0-9_]*)\s*\(", text):
            name = m.group(1)
            if name.startswith("tsm2") and name not in names:
                names.append(name)
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2002_03258_gb300 import build
    build.build()
    return pkg.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("tsm2r_d", "tsm2r_s", "tsm2l_d", "tsm2l_s", "tsm2_get_last_error_string",
                     "tsm2_get_device_status", "tsm2_shutdown"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


FAKE = 1 << 20  # never dereferenced: every call below fails or returns before any launch


@pytest.mark.parametrize("fn", ["tsm2r_d", "tsm2r_s", "tsm2l_d", "tsm2l_s",
                                "tsm2r_s_host", "tsm2r_d_host", "tsm2l_s_host", "tsm2l_d_host"])
@pytest.mark.parametrize("args,why", [
    ((-1, 4, 2, FAKE, 4, FAKE * 2, 4, FAKE * 3, 4), "negative m"),
    ((4, -4, 2, FAKE, 4, FAKE * 2, 4, FAKE * 3, 4), "negative n"),
    ((4, 4, -2, FAKE, 4, FAKE * 2, 4, FAKE * 3, 4), "negative k"),
    ((8, 4, 2, FAKE, 7, FAKE * 2, 4, FAKE * 3, 8), "lda < m"),
    ((8, 4, 2, FAKE, 8, FAKE * 2, 3, FAKE * 3, 8), "ldb < n"),
    ((8, 4, 2, FAKE, 8, FAKE * 2, 4, FAKE * 3, 7), "ldc < m"),
    ((8, 4, 2, 0, 8, FAKE * 2, 4, FAKE * 3, 8), "A NULL"),
    ((8, 4, 2, FAKE, 8, 0, 4, FAKE * 3, 8), "B NULL"),
    ((8, 4, 2, FAKE, 8, FAKE * 2, 4, 0, 8), "C NULL"),
    ((8, 4, 2, FAKE, 8, FAKE * 2, 4, FAKE + 16, 8), "C overlaps A"),
    ((0, 0, 2, FAKE, 0, FAKE * 2, 0, FAKE * 3, 1), "lda 0"),
])
def test_invalid_arguments(lib, fn, args, why):
    st = getattr(pkg, fn)(*args, 0)
    assert st == pkg.ERR_INVALID_VALUE, why
    assert pkg.tsm2_get_last_error_string() != "no error"


@pytest.mark.parametrize("fn", ["tsm2r_d", "tsm2r_s", "tsm2l_d", "tsm2l_s",
                                "tsm2r_s_host", "tsm2r_d_host", "tsm2l_s_host", "tsm2l_d_host"])
def test_quick_returns_without_device(lib, fn):
    # m == 0 or k == 0: nothing to do, no CUDA call is made.
    assert getattr(pkg, fn)(0, 5, 3, 0, 1, FAKE, 5, 0, 1, 0) == pkg.SUCCESS
    assert getattr(pkg, fn)(5, 5, 0, FAKE, 5, FAKE * 2, 5, 0, 5, 0) == pkg.SUCCESS


@pytest.mark.parametrize("fn", ["tsm2l_d", "tsm2l_s", "tsm2l_s_host", "tsm2l_d_host"])
def test_tsm2l_takes_any_inner_dimension(lib, fn):
    # n > 64 (B staged instead of resident) and k > 64 (column chunks) are
    # accepted: with m == 0 the call returns before touching the device.
    assert getattr(pkg, fn)(0, 500, 100, 0, 1, FAKE, 500, 0, 1, 0) == pkg.SUCCESS


def test_error_string_is_thread_local(lib):
    import threading
    pkg.tsm2r_s(-1, 1, 1, FAKE, 1, FAKE, 1, FAKE, 1, 0)
    msg_main = pkg.tsm2_get_last_error_string()
    other = {}

    def worker():
        other["msg"] = pkg.tsm2_get_last_error_string()

    t = threading.Thread(target=worker)
    t.start()
    t.join()
    assert "negative" in msg_main
    assert other["msg"] == "no error"


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    import importlib
    monkeypatch.setattr(pkg, "_lib", None)
    monkeypatch.setattr(pkg, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="not built"):
        pkg.lib()


@pytest.mark.parametrize("elem,m,n,k,want", [
    (4, 1 << 20, 256, 16, "l"), (4, 1 << 20, 257, 16, "r"), (4, 15360, 64, 16, "l"), (4, 15360, 65, 16, "r"),
    (4, 15360, 128, 32, "l"), (4, 15360, 129, 32, "r"), (8, 1 << 17, 64, 16, "l"), (8, 1 << 17, 65, 16, "r"),
    (8, 1 << 20, 256, 17, "l"), (8, 1000, 32, 8, "l"), (8, 1000, 33, 8, "r"), (8, 1000, 64, 20, "l"),
    (4, 30720, 30720, 16, "r"), (4, 1 << 23, 8, 8, "l"),
])
def test_tsm2x_schedule_choice(lib, elem, m, n, k, want):
    assert pkg.tsm2x_choice(elem, m, n, k) == want


def test_tsm2x_choice_rejects_bad_arguments(lib):
    assert pkg.tsm2x_choice(2, 10, 10, 10) == ""
    assert pkg.tsm2x_choice(4, -1, 10, 10) == ""


def test_debug_build_flag_exported(lib):
    """The release library reports no bounds checks; the debug variant (when
    built) reports them.  No device is needed for either call."""
    assert lib.tsm2_debug_checks() == 0
    import ctypes
    import os
    from paper_2002_03258_gb300 import build as b
    if os.path.exists(b.DEBUG_LIB):
        dbg = ctypes.CDLL(b.DEBUG_LIB)
        dbg.tsm2_debug_checks.restype = ctypes.c_int
        assert dbg.tsm2_debug_checks() == 1
