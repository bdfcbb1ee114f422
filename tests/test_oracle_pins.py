"""Pins for the CPU oracle against facts fixed by the mathematics and the paper.

The oracle computes C = A B as the plain definition (Sec. 2.1; Algorithms 2,
4, 5 accumulate exactly this).  None of these checks re-types that formula in
floating point: each compares against exact rational arithmetic, integer
arithmetic, a structural identity, or a value the paper prints, chosen so that
a dropped term, a wrong sign or index, a transposed operand or a mishandled
leading dimension fails at least one of them.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import tsm2_inputs as ti

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def exact_product(A, B):
    """Exact rational C and S = |A||B| for tiny float matrices."""
    m, n = A.shape
    k = B.shape[1]
    Af = [[Fraction(float(A[i, j])) for j in range(n)] for i in range(m)]
    Bf = [[Fraction(float(B[j, c])) for c in range(k)] for j in range(n)]
    C = [[sum((Af[i][j] * Bf[j][c] for j in range(n)), Fraction(0)) for c in range(k)] for i in range(m)]
    S = [[sum((abs(Af[i][j] * Bf[j][c]) for j in range(n)), Fraction(0)) for c in range(k)] for i in range(m)]
    return C, S


@pytest.mark.parametrize("dtype,u", [(np.float64, oracle.U_FP64), (np.float32, oracle.U_FP32)])
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (3, 5, 2), (7, 4, 3), (5, 9, 1), (2, 13, 4), (6, 6, 6)])
def test_exact_rational(m, n, k, dtype, u):
    A = ti.uniform_pm1(11, ti.MID_A, m, n, dtype)
    B = ti.uniform_pm1(11, ti.MID_B, n, k, dtype)
    C = oracle.gemm(A, B)
    Ce, Se = exact_product(A, B)
    # The oracle sums in binary64 whatever the input precision.
    g = oracle.gamma(n, oracle.U_FP64)
    for i in range(m):
        for c in range(k):
            err = abs(Fraction(float(C[i, c])) - Ce[i][c])
            assert err <= Fraction(g) * Se[i][c], (i, c, float(err), float(Se[i][c]))


def test_exact_rational_catches_transpose():
    """A non-square case where A^T-style indexing would give different sums."""
    A = ti.uniform_pm1(3, ti.MID_A, 4, 3, np.float64)
    B = ti.uniform_pm1(3, ti.MID_B, 3, 4, np.float64)
    C = oracle.gemm(A, B)
    Ce, _ = exact_product(A, B)
    Ct, _ = exact_product(B.T.copy(order="F"), A.T.copy(order="F"))  # (A B)^T = B^T A^T
    for i in range(4):
        for c in range(4):
            assert Ct[c][i] == Ce[i][c]
    assert abs(float(C[1, 2]) - float(Ce[1][2])) < 1e-15
    assert abs(float(C[1, 2]) - float(Ce[2][1])) > 1e-6


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_identity_gives_b_exactly(dtype):
    n, k = 37, 5
    lda, ldb = 41, 40
    Abuf = ti.padded(np.eye(n, dtype=dtype, order="F"), lda)
    Bbuf = ti.padded(ti.uniform_pm1(5, ti.MID_B, n, k, dtype), ldb)
    A = Abuf[:n, :]
    B = Bbuf[:n, :]
    C = oracle.gemm(A, B)
    assert np.array_equal(C, B.astype(np.float64))


def test_permutation_gives_pb_exactly():
    n, k = 50, 7
    perm = np.argsort(ti.uniform_pm1(9, 99, n, 1)[:, 0])
    P = np.zeros((n, n), order="F")
    P[np.arange(n), perm] = 1.0
    B = ti.uniform_pm1(9, ti.MID_B, n, k)
    C = oracle.gemm(P, B)
    assert np.array_equal(C, B[perm, :])


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_all_ones_gives_column_sums(dtype):
    m, n, k = 9, 300, 4
    A = np.ones((m, n), dtype=dtype, order="F")
    B = ti.uniform_pm1(21, ti.MID_B, n, k, dtype)
    C = oracle.gemm(A, B)
    for i in range(1, m):
        assert np.array_equal(C[i], C[0])  # identical sums in identical order
    g = oracle.gamma(n, oracle.U_FP64)
    for c in range(k):
        col = [float(x) for x in B[:, c]]
        exact = math.fsum(col)  # correctly rounded sum
        s = math.fsum(abs(x) for x in col)
        assert abs(C[0, c] - exact) <= g * s + abs(exact) * oracle.U_FP64


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_small_integers_exact(dtype):
    m, n, k = 123, 301, 16
    A = ti.int_small(4, ti.MID_A, m, n, dtype)
    B = ti.int_small(4, ti.MID_B, n, k, dtype)
    C = oracle.gemm(A, B)
    Ci = A.astype(np.int64) @ B.astype(np.int64)  # integer arithmetic, exact
    assert np.array_equal(C, Ci.astype(np.float64))
    assert set(np.unique(A)).issubset(set(range(-4, 5)))


def test_rank_one():
    m, n, k = 6, 48, 3
    u = ti.uniform_pm1(8, 50, m, 1)[:, 0]
    v = ti.uniform_pm1(8, 51, n, 1)[:, 0]
    A = np.asfortranarray(np.outer(u, v))
    B = ti.uniform_pm1(8, ti.MID_B, n, k)
    C = oracle.gemm(A, B)
    Ce, Se = exact_product(A, B)
    g = oracle.gamma(n, oracle.U_FP64)
    for i in range(m):
        for c in range(k):
            assert abs(Fraction(float(C[i, c])) - Ce[i][c]) <= Fraction(g) * Se[i][c]
    # and the structure: rows are proportional to u
    w = oracle.gemm(v[None, :].copy(order="F"), B)[0]
    np.testing.assert_allclose(C, np.outer(u, w), rtol=0, atol=4 * g * float(np.max(np.abs(Se_to_np(Se)))))


def Se_to_np(S):
    return np.array([[float(x) for x in row] for row in S])


def test_long_double_agrees():
    m, n, k = 17, 64, 16
    A = ti.uniform_pm1(2, ti.MID_A, m, n)
    B = ti.uniform_pm1(2, ti.MID_B, n, k)
    C = oracle.gemm(A, B)
    Cl = oracle.gemm_ld(A, B)
    S = oracle.absgemm(A, B)
    assert oracle.long_double_mant_dig() >= 64
    g = oracle.gamma(n, oracle.U_FP64)
    assert np.all(np.abs(C.astype(np.longdouble) - Cl) <= g * S * 1.0000001)
    # long double vs exact on a tiny corner
    Ce, Se = exact_product(A[:3, :], B[:, :2])
    gl = oracle.gamma(n, 2.0 ** -oracle.long_double_mant_dig())
    for i in range(3):
        for c in range(2):
            assert abs(Fraction(*Cl[i, c].as_integer_ratio()) - Ce[i][c]) <= Fraction(gl) * Se[i][c] * 2


def test_absgemm_exact_on_integers():
    A = ti.int_small(6, ti.MID_A, 20, 30)
    B = ti.int_small(6, ti.MID_B, 30, 4)
    assert np.array_equal(oracle.absgemm(A, B), (np.abs(A).astype(np.int64) @ np.abs(B).astype(np.int64)).astype(float))


def test_strides_and_padding_not_read():
    m, n, k = 10, 12, 3
    A = ti.uniform_pm1(1, ti.MID_A, m, n)
    B = ti.uniform_pm1(1, ti.MID_B, n, k)
    Abuf = ti.padded(A, 16, np.nan)
    Bbuf = ti.padded(B, 13, np.nan)
    C1 = oracle.gemm(A, B)
    C2 = oracle.gemm(Abuf[:m], Bbuf[:n])
    assert np.array_equal(C1, C2)
    # transposed views: (A B)^T computed as B^T A^T matches exactly in value
    # structure (same products, same order of j)
    C3 = oracle.gemm(B.T, A.T)
    assert np.array_equal(C3.T, C1)


def test_empty_inner_dimension_gives_zero():
    A = np.zeros((5, 0), order="F")
    B = np.zeros((0, 3), order="F")
    C = oracle.gemm(A, B)
    assert C.shape == (5, 3) and np.all(C == 0)
    assert oracle.gemm(np.zeros((0, 4), order="F"), np.zeros((4, 2), order="F")).shape == (0, 2)


def test_nan_inf_propagate():
    A = ti.uniform_pm1(3, ti.MID_A, 6, 8)
    B = ti.uniform_pm1(3, ti.MID_B, 8, 3)
    A[2, 5] = np.nan
    B[1, 1] = np.inf
    C = oracle.gemm(A, B)
    assert np.all(np.isnan(C[2, :]))
    # column 1 picks up inf * A[i,1] (finite nonzero) -> +-inf, or NaN in row 2
    assert np.all(~np.isfinite(C[:, 1]))
    assert np.all(np.isfinite(np.delete(C, 2, axis=0)[:, [0, 2]]))


def test_threaded_bitwise_equal():
    A = ti.uniform_pm1(5, ti.MID_A, 301, 77, np.float32)
    B = ti.uniform_pm1(5, ti.MID_B, 77, 8, np.float32)
    assert np.array_equal(oracle.gemm(A, B), oracle.gemm_threaded(A, B, 4))


def test_bf16_rne_against_torch_and_specials():
    torch = pytest.importorskip("torch")
    x = ti.logmag(7, 1, 4000, 1, np.float32)[:, 0]
    specials = np.array([0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, 3.4028235e38, 1e-45, -1e-45,
                         # exact ties: 1 + 2^-8 -> 1 (even); 1 + 3*2^-8 -> 1 + 2^-6 (even)
                         1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -8 + 2.0 ** -20],
                        dtype=np.float32)
    x = np.concatenate([x, specials])
    h = oracle.bf16_rne(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(h, ref)
    assert oracle.bf16_to_float(oracle.bf16_rne(np.array([1.0 + 2.0 ** -8], np.float32)))[0] == 1.0
    assert oracle.bf16_to_float(oracle.bf16_rne(np.array([1.0 + 3 * 2.0 ** -8], np.float32)))[0] == 1.0 + 2.0 ** -6
    assert np.isinf(oracle.bf16_to_float(oracle.bf16_rne(np.array([3.4028235e38], np.float32)))[0])
    nan = oracle.bf16_to_float(oracle.bf16_rne(np.array([np.nan], np.float32)))[0]
    assert np.isnan(nan)


def test_splitmix64_known_answer():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64_kat.txt")) if l.strip() and not l.startswith("#")]
    idx = np.array([int(r[0]) for r in rows])
    want = [int(r[1]) for r in rows]
    got = [int(x) for x in ti.draws(1234567, idx)]
    assert got == want


def test_input_distributions_and_random_access():
    A = ti.uniform_pm1(0, ti.MID_A, 300, 200)
    assert A.min() >= -1.0 and A.max() < 1.0
    assert abs(A.mean()) < 0.01 and abs(A.var() - 1 / 3) < 0.01
    sub = ti.uniform_pm1(0, ti.MID_A, 300, 200, row_idx=[5, 17, 299], col_idx=[0, 199])
    assert np.array_equal(sub, A[[5, 17, 299]][:, [0, 199]])
    Z = ti.normal_ih(0, ti.MID_A, 400, 300, scale=0.5)
    assert abs(Z.mean()) < 0.01 and abs(Z.std() - 0.5) < 0.01
    L = ti.logmag(0, ti.MID_A, 500, 100)
    e = np.floor(np.log2(np.abs(L)))
    assert e.min() == -10 and e.max() == 9
    f32 = ti.uniform_pm1(0, ti.MID_A, 300, 200, np.float32)
    assert np.array_equal(f32, A.astype(np.float32))


def test_absgemm_s_exact_on_float32_integers():
    """Binary32 magnitude matrix S = |A||B| (Sec. 2.1 definition on absolute
    values) equals integer arithmetic exactly; negative entries in both
    operands make a dropped fabs on either side fail."""
    A = ti.int_small(6, ti.MID_A, 33, 47, np.float32)
    B = ti.int_small(6, ti.MID_B, 47, 5, np.float32)
    assert (A < 0).any() and (B < 0).any()
    S = oracle.absgemm(A, B)
    Si = np.abs(A).astype(np.int64) @ np.abs(B).astype(np.int64)
    assert S.dtype == np.float64
    assert np.array_equal(S, Si.astype(np.float64))
    # a signed product differs from S wherever the signs mix
    assert not np.array_equal(S, (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64))


@pytest.mark.parametrize("m,n,k", [(3, 5, 2), (4, 11, 3), (2, 17, 4)])
def test_absgemm_s_matches_exact_rational(m, n, k):
    """S for binary32 uniform inputs: every binary32 value widens exactly to
    binary64 and all terms are non-negative, so the binary64 sum is within
    gamma_n(2^-53) * S of the exact rational sum of |a||b|.  A widening that
    rounded through a narrower type (an error of about 2^-24 per term) or a
    lost term fails this."""
    A = ti.uniform_pm1(13, ti.MID_A, m, n, np.float32)
    B = ti.uniform_pm1(13, ti.MID_B, n, k, np.float32)
    S = oracle.absgemm(A, B)
    _, Se = exact_product(A, B)
    g = oracle.gamma(n, oracle.U_FP64)
    for i in range(m):
        for c in range(k):
            err = abs(Fraction(float(S[i, c])) - Se[i][c])
            assert err <= Fraction(g) * Se[i][c], (i, c, float(err))
            # much tighter than one binary32 ulp of S: the widening is exact
            assert float(err) < 2.0 ** -40 * float(Se[i][c])


def test_absgemm_s_strided_and_transposed():
    """Padded leading dimensions are not read and a transposed view (A^T
    with row stride lda) gives the transposed magnitude matrix."""
    m, n, k = 9, 14, 3
    A = ti.int_small(2, ti.MID_A, m, n, np.float32)
    B = ti.int_small(2, ti.MID_B, n, k, np.float32)
    Abuf = ti.padded(A, 12, np.nan)
    S1 = oracle.absgemm(A, B)
    S2 = oracle.absgemm(Abuf[:m], B)
    assert np.array_equal(S1, S2)
    S3 = oracle.absgemm(B.T, A.T)
    assert np.array_equal(S3.T, S1)
