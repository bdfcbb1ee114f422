"""bfloat16 storage of A on the tensor cores (tsm2r_bf16) and the split
helper (tsm2_split_bf16), against the CPU oracle.

The oracle side forms A_hi / A_lo with its own bit-level round-to-nearest-even
(pinned against torch on the CPU) and evaluates the plain product of the
bfloat16-represented A with binary32 B in binary64.  The componentwise bound
|C - A_eff B| <= f |A_eff||B| takes f from ``bf16_bound``, which derives it
from the kernel's structure (B-piece truncation, one drain group of tensor-core
sums, binary32 adds across groups and stream-K partials); at 32768^2 it is
about 5e-5 (plain) and 7e-5 (hi+lo), tight enough that a lost pipeline stage
fails (tests/test_bf16_bound_host.py).  Small-integer inputs make every product
and partial sum exact: bit equality.
"""
import numpy as np
import pytest

import bf16_bound as bb
import oracle
import tsm2_inputs as ti

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev_colmajor(a, ld=None, dtype=None):
    rows, cols = a.shape
    ld = ld or rows
    t = torch.full((cols, ld), float("nan") if dtype is None else 0, dtype=dtype or torch.float32, device="cuda")
    v = t.t()[:rows]
    if dtype is None:
        v.copy_(torch.from_numpy(np.ascontiguousarray(a)).cuda())
    else:
        v.copy_(torch.from_numpy(np.ascontiguousarray(a).view(np.int16)).cuda())
    return t, v


def split_host(X32):
    hi = oracle.bf16_rne(X32)
    r = (X32 - oracle.bf16_to_float(hi)).astype(np.float32)  # exact in binary32
    lo = oracle.bf16_rne(r)
    return hi, lo


def launch_grid(grid):
    """The grid the bound assumes: the override, else the SM count (the
    library never launches more blocks than SMs by default, and a larger grid
    only loosens the bound)."""
    return grid if grid > 0 else torch.cuda.get_device_properties(0).multi_processor_count


def run(m, n, k, hilo, lda=None, gen="logmag", seed=0, grid=0):
    import paper_2002_03258_gb300 as pkg
    pkg.tsm2_set_grid(grid)
    lda = lda or (m + 7) // 8 * 8
    if gen == "logmag":
        X = ti.logmag(seed, ti.MID_A, m, n, np.float32)
        B = ti.uniform_pm1(seed, ti.MID_B, n, k, np.float32)
    else:
        X = ti.int_small(seed, ti.MID_A, m, n, np.float32)
        B = ti.int_small(seed, ti.MID_B, n, k, np.float32)
    hi, lo = split_host(np.asfortranarray(X))
    thi, vhi = dev_colmajor(hi, lda, torch.int16)
    tlo, vlo = dev_colmajor(lo, lda, torch.int16)
    tB, vB = dev_colmajor(B)
    tC = torch.full((k, m + 5), -9.0, device="cuda")
    st = pkg.tsm2r_bf16(m, n, k, thi.data_ptr(), tlo.data_ptr() if hilo else None, lda, vB.data_ptr(), n,
                        tC.data_ptr(), m + 5, 0)
    assert st == 0, pkg.tsm2_get_last_error_string()
    torch.cuda.synchronize()
    assert pkg.tsm2_get_device_status(0) == 0
    cfg = pkg.tsm2_last_config()
    pkg.tsm2_set_grid(0)
    Cfull = tC.t().cpu().numpy()
    assert np.all(Cfull[m:] == -9.0)
    Aeff = oracle.bf16_to_float(hi).astype(np.float64)
    if hilo:
        Aeff = Aeff + oracle.bf16_to_float(lo).astype(np.float64)
    return Cfull[:m].astype(np.float64), np.asfortranarray(Aeff), B.astype(np.float64), cfg


def check(C, Aeff, B, hilo, cfg, grid=0, m=None, exact=False):
    ref = oracle.gemm(Aeff, B)
    if exact:
        assert np.array_equal(C, ref)
        return 0.0
    S = oracle.absgemm(Aeff, B)
    n = Aeff.shape[1]
    m = C.shape[0] if m is None else m
    bound = bb.factor(cfg, m, n, hilo, launch_grid(grid)) * S
    err = np.abs(C - ref)
    assert np.all(err <= bound), float(np.max(err / np.maximum(bound, 1e-300)))
    return float(np.max(err / np.maximum(S, 1e-300)))


@pytest.mark.parametrize("hilo", [False, True])
@pytest.mark.parametrize("m,n,k", [(128, 64, 16), (1000, 1000, 16), (1031, 777, 5), (300, 4100, 1),
                                   (4096, 2048, 16), (257, 63, 20), (2000, 3000, 8)])
def test_tensor_core_parity(m, n, k, hilo):
    C, Aeff, B, cfg = run(m, n, k, hilo)
    assert cfg.startswith("tc_bf16"), cfg
    check(C, Aeff, B, hilo, cfg)


@pytest.mark.parametrize("hilo", [False, True])
def test_tensor_core_integers_bit_exact(hilo):
    C, Aeff, B, cfg = run(2048, 4096, 16, hilo, gen="int")
    assert cfg.startswith("tc_bf16")
    check(C, Aeff, B, hilo, cfg, exact=True)


@pytest.mark.parametrize("hilo", [False, True])
@pytest.mark.parametrize("grid", [1, 3, 50])
def test_tensor_core_any_grid(grid, hilo):
    C, Aeff, B, cfg = run(1500, 2500, 12, hilo, grid=grid)
    check(C, Aeff, B, hilo, cfg, grid=grid)


def test_elementwise_path_unaligned_lda():
    C, Aeff, B, cfg = run(999, 500, 7, True, lda=1001)
    assert cfg == "simple_bf16", cfg
    check(C, Aeff, B, True, cfg)


def test_split_matches_oracle_rounding():
    import paper_2002_03258_gb300 as pkg
    rows, cols, ld = 1003, 37, 1008
    X = np.asfortranarray(ti.logmag(5, 9, rows, cols, np.float32))
    X[0, 0] = 1.0 + 2.0 ** -8  # a tie
    tX, vX = dev_colmajor(X, ld)
    th = torch.zeros((cols, ld), dtype=torch.int16, device="cuda")
    tl = torch.zeros((cols, ld), dtype=torch.int16, device="cuda")
    assert pkg.tsm2_split_bf16(rows, cols, vX.data_ptr(), ld, th.data_ptr(), tl.data_ptr(), ld, 0) == 0
    torch.cuda.synchronize()
    hi, lo = split_host(X)
    assert np.array_equal(th.t()[:rows].cpu().numpy().view(np.uint16), hi)
    assert np.array_equal(tl.t()[:rows].cpu().numpy().view(np.uint16), lo)
    # hi + lo carries about 16 significant bits
    rec = oracle.bf16_to_float(hi).astype(np.float64) + oracle.bf16_to_float(lo)
    assert np.all(np.abs(rec - X) <= 2.0 ** -16 * np.abs(X))


def test_config5_fullsize_sampled():
    """32768 x 32768 A (log-uniform magnitudes), k = 16: device-generated and
    device-split A, sampled rows against the oracle on host-regenerated A."""
    import paper_2002_03258_gb300 as pkg
    lib = pkg.lib()
    m = n = 32768
    k = 16
    X = torch.empty((n, m), dtype=torch.float32, device="cuda").t()
    assert lib.tsm2_fill_logmag_s(m, n, 0, ti.MID_A, X.data_ptr(), m, 0) == 0
    B = torch.empty((k, n), dtype=torch.float32, device="cuda").t()
    assert lib.tsm2_fill_uniform_s(n, k, 0, ti.MID_B, B.data_ptr(), n, 0) == 0
    hi = torch.empty((n, m), dtype=torch.int16, device="cuda")
    lo = torch.empty((n, m), dtype=torch.int16, device="cuda")
    assert pkg.tsm2_split_bf16(m, n, X.data_ptr(), m, hi.data_ptr(), lo.data_ptr(), m, 0) == 0
    del X
    rows = np.array(bb.CONFIG5_ROWS)
    Xr = ti.logmag(0, ti.MID_A, m, n, np.float32, row_idx=rows)
    Bh = ti.uniform_pm1(0, ti.MID_B, n, k, np.float32)
    hih, loh = split_host(np.asfortranarray(Xr))
    for hilo in (False, True):
        C = torch.empty((k, m), dtype=torch.float32, device="cuda").t()
        st = pkg.tsm2r_bf16(m, n, k, hi.data_ptr(), lo.data_ptr() if hilo else None, m, B.data_ptr(), n,
                            C.data_ptr(), m, 0)
        assert st == 0, pkg.tsm2_get_last_error_string()
        assert pkg.tsm2_get_device_status(0) == 0
        cfg = pkg.tsm2_last_config()
        assert cfg.startswith("tc_bf16")
        got = C.cpu().numpy()[rows].astype(np.float64)
        Aeff = oracle.bf16_to_float(hih).astype(np.float64)
        if hilo:
            Aeff = Aeff + oracle.bf16_to_float(loh)
        check(got, np.asfortranarray(Aeff), Bh.astype(np.float64), hilo, cfg, m=m)
