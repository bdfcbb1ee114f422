"""Batches of uneven TSM2R / TSM2L problems (binary32): Python wrapper over
the ``tsm2_batch_plan_*`` C ABI.

A plan groups the problems into tile classes of one compiled tile variant.
By default the whole batch runs as ONE persistent kernel launch whose blocks
walk their share of every class in turn; the classes can also run one after
another (one launch each, on all SMs) or concurrently on SM shares.  Any mode
can be replayed as one CUDA graph launch.
"""
from __future__ import annotations

import ctypes

from . import _load, check

WIDE_L = 1  # accepted and ignored
MERGE_R = 2
MERGE_L = 4

CONCURRENT = 0
SERIAL = 1
SINGLE_LAUNCH = 2
MODES = {"concurrent": CONCURRENT, "serial": SERIAL, "single": SINGLE_LAUNCH}


def variant_flag(v: int) -> int:
    """Plan flag selecting tile variant ``v``."""
    return int(v) << 8


def num_variants() -> int:
    return int(_load().tsm2_batch_num_variants())


def variant_info(v: int) -> dict:
    """Tile parameters of compiled variant ``v``."""
    lib = _load()
    name = ctypes.c_char_p()
    st, rows, inner = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    check(lib.tsm2_batch_variant_info(v, ctypes.byref(name), ctypes.byref(st), ctypes.byref(rows),
                                      ctypes.byref(inner)))
    return {"variant": v, "name": name.value.decode(), "stages": st.value, "rows_per_lane": rows.value,
            "inner_per_warp": inner.value}


class Problem(ctypes.Structure):
    """Mirror of ``tsm2_problem_s``: C(m x k) = A(m x n) B(n x k), column-major."""
    _fields_ = [("op", ctypes.c_char), ("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int64),
                ("A", ctypes.c_void_p), ("lda", ctypes.c_int64), ("B", ctypes.c_void_p), ("ldb", ctypes.c_int64),
                ("C", ctypes.c_void_p), ("ldc", ctypes.c_int64)]


def problem(op, m, n, k, A, lda, B, ldb, C, ldc) -> Problem:
    return Problem(op.encode() if isinstance(op, str) else op, m, n, k, A, lda, B, ldb, C, ldc)


class BatchPlan:
    def __init__(self, problems, flags: int = 0):
        lib = _load()
        arr = (Problem * len(problems))(*problems)
        self._arr = arr  # keep alive while creating
        out = ctypes.c_void_p()
        check(lib.tsm2_batch_plan_create_s(len(problems), ctypes.cast(arr, ctypes.c_void_p), flags, ctypes.byref(out)))
        self.handle = out
        self.flags = flags
        self.variant = (flags >> 8) & 0xFF

    def execute(self, stream=0):
        check(_load().tsm2_batch_plan_execute(self.handle, stream))

    def execute_class(self, cls: int, stream=0):
        check(_load().tsm2_batch_plan_execute_class(self.handle, cls, stream))

    def graph_launch(self, stream=0):
        check(_load().tsm2_batch_plan_graph_launch(self.handle, stream))

    def classes(self):
        lib = _load()
        out = []
        for i in range(lib.tsm2_batch_plan_num_classes(self.handle)):
            name = ctypes.c_char_p()
            nbytes = ctypes.c_double()
            grid = ctypes.c_int()
            nprob = ctypes.c_int()
            check(lib.tsm2_batch_plan_class_info(self.handle, i, ctypes.byref(name), ctypes.byref(nbytes),
                                                 ctypes.byref(grid), ctypes.byref(nprob)))
            out.append({"name": name.value.decode(), "bytes": nbytes.value, "grid": grid.value, "nprob": nprob.value})
        return out

    def set_grids(self, grids):
        arr = (ctypes.c_int * len(grids))(*[int(g) for g in grids])
        check(_load().tsm2_batch_plan_set_grids(self.handle, len(grids), arr))

    def set_serial(self, serial: bool):
        check(_load().tsm2_batch_plan_set_serial(self.handle, int(bool(serial))))

    def set_mode(self, mode):
        """``mode``: SINGLE_LAUNCH, SERIAL, CONCURRENT or one of their names."""
        check(_load().tsm2_batch_plan_set_mode(self.handle, MODES.get(mode, mode)))

    def set_single_grid(self, grid: int):
        check(_load().tsm2_batch_plan_set_single_grid(self.handle, int(grid)))

    def num_launches(self) -> int:
        return int(_load().tsm2_batch_plan_num_launches(self.handle))

    def close(self):
        if self.handle:
            _load().tsm2_batch_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
