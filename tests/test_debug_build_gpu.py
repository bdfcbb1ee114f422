"""The bounds-checking build (libtsm2_debug.so, -DTSM2_DEBUG) on the GPU.

In it, every hand-computed global address of the bulk-copy, batched and
backward kernels (C rows and columns, B rows, workspace slots, arrival
counters) is checked against its operand's extents before the access; an
out-of-range access would be skipped and reported as TSM2_ERR_BOUNDS.  The
memory checker is closed on this machine, so this build stands in for it: the
parity cases of tests/debug_build_cases.py (single products of every path,
the allocation-free and backward entry points, batched plans of every tile
variant in both launch modes) run against it in a child process and must
match the oracle with a clean status.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_parity_cases_under_bounds_checks():
    pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    from paper_2002_03258_gb300 import build as b
    b.build(debug=True)
    env = dict(os.environ, TSM2_DEBUG="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_build_cases.py")], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "DEBUG-BUILD-OK" in r.stdout, r.stdout[-2000:]


def test_release_build_has_no_checks():
    pytest.importorskip("torch")
    import paper_2002_03258_gb300 as pkg
    if pkg.DEBUG:
        pytest.skip("this process runs the debug build")
    assert pkg.lib().tsm2_debug_checks() == 0
