"""Componentwise error bound of tsm2r_bf16, derived from how the kernel sums.

The reference is the exact product of the bfloat16-represented A (A_hi, or
A_hi + A_lo) with binary32 B, so A's own representation error is not part of
it.  Per output C(i, c), with S = sum_j |A(i, j)| |B(j, c)| (the magnitude
matrix of Sec. 2.1's definition):

1. B pieces.  B is split into bfloat16 pieces, each the round-to-nearest-even
   of the remainder.  For b in [2^e, 2^(e+1)) the first remainder is at most
   2^(e-8) and lies below bit e-8; the second is at most 2^(e-17).  Plain A
   uses two pieces, so |b - b1 - b2| <= 2^-17 |b|.  hi+lo uses three, and the
   third remainder has at most 7 significant bits, so b1 + b2 + b3 = b exactly.
2. Tensor-core sums.  One drain group covers G inner indices (plain: 4 stages
   of 64, G = 256; hi+lo: one stage of 32, G = 32) accumulated in TMEM by
   s = G/16 MMA steps per piece (hi+lo: two steps per 16 indices, A_hi then
   A_lo).  Each step adds 16 exact products to the accumulator.  The model is
   the one Fasi, Higham, Mikaitis and Pranesh (2021, "Numerical behavior of
   NVIDIA tensor cores") measured on earlier parts: the 17 addends are aligned
   to the largest exponent with truncation to a 24-bit window, then the sum is
   normalised by truncation.  Each addend then loses less than 2^-23 times
   the largest magnitude and the normalisation as much again, so one step
   errs by at most 18 * 2^-23 times the sum of its addends' magnitudes, which
   the group's share of S bounds.
3. Piece sum.  The epilogue adds the NP pieces of a group in binary32
   round-to-nearest: gamma_{NP-1}(2^-24).
4. Carry.  Group sums are added in binary32 round-to-nearest in one chain per
   block, and the stream-K partial sums of a row block in a fixed order.  A
   block's range ends groups early at most once per partial, so the chain
   has at most ceil(units_per_row_block / group) + P rounded adds, where P
   bounds the partials that cover one row block.

Piece magnitudes add at most a factor 1 + 2^-6 to the group shares; the
final factor 1.04 covers that and the second-order terms.

The element-wise path (unaligned operands) is a binary32 FMA chain over n:
gamma_n(2^-24) S.
"""
U32 = 2.0 ** -24
TC_STEP = 18 * 2.0 ** -23
BM = 512  # rows per unit of the tensor-core kernel


def gamma(n, u=U32):
    nu = n * u
    return float("inf") if nu >= 1 else nu / (1 - nu)


def geometry(hilo):
    """(inner columns per stage, stages per drain group, B pieces, MMA steps per group)."""
    bk = 32 if hilo else 64
    group = 1 if hilo else 4
    npieces = 3 if hilo else 2
    steps = group * (bk // 16) * (2 if hilo else 1)
    return bk, group, npieces, steps


def max_partials(m, n, hilo, grid):
    """Upper bound on the stream-K partial sums that cover one row block when
    the kernel runs on ``grid`` blocks (a larger grid only raises it)."""
    bk, _, _, _ = geometry(hilo)
    upr = -(-n // bk)
    ngroups = -(-m // BM) * upr
    grid = max(1, min(grid, ngroups))
    per_block = max(1, ngroups // grid)
    return min(grid, -(-(upr - 1) // per_block) + 1)


def tc_factor(m, n, hilo, grid):
    """Bound on |C - C_ref| / S for the tensor-core path."""
    bk, group, npieces, steps = geometry(hilo)
    upr = -(-n // bk)
    e_b = 0.0 if hilo else 2.0 ** -17
    e_tc = steps * TC_STEP
    e_piece = gamma(npieces - 1)
    n_carry = -(-upr // group) + max_partials(m, n, hilo, grid)
    return 1.04 * (e_b + e_tc + e_piece + gamma(n_carry))


def simple_factor(n):
    """Bound on |C - C_ref| / S for the element-wise path."""
    return gamma(n)


def factor(cfg, m, n, hilo, grid):
    if cfg.startswith("tc_bf16"):
        return tc_factor(m, n, hilo, grid)
    if cfg == "simple_bf16":
        return simple_factor(n)
    raise ValueError(f"unknown bfloat16 configuration {cfg!r}")


def stage_columns(n, hilo):
    """Inner-index ranges of the kernel's pipeline stages."""
    bk = geometry(hilo)[0]
    return [(j0, min(n, j0 + bk)) for j0 in range(0, n, bk)]


# Rows of the 32768 x 32768 x 16 bfloat16 workload that the full-size GPU
# test checks against the oracle (first, second, tile edges, interior, last).
CONFIG5_ROWS = (0, 1, 127, 128, 4095, 20000, 32767)
