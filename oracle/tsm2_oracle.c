/*
 * CPU oracle for tall-and-skinny matrix multiplication (TSM2R / TSM2L).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header or constant with the CUDA
 * library.
 *
 * What it computes.  TSM2R and TSM2L (Sec. 2.1 of the paper: a large regular
 * matrix times a tall-and-skinny one, and a tall-and-skinny matrix times a
 * small square one) both compute the plain matrix product
 *
 *     C(i, c) = sum_{j = 0}^{n-1} A(i, j) * B(j, c),   0 <= i < m, 0 <= c < k,
 *
 * (Algorithms 2, 4 and 5 accumulate exactly this; the outer-product order of
 * Algorithm 2 only changes the loop nest, not the sums).  Here A is m x n,
 * B is n x k and C is m x k, matching the library's naming (the paper names
 * the inner dimension k and the skinny one n).  The oracle is that definition
 * written out: every output is a left-to-right sum over j = 0, 1, ..., n-1 of
 * rounded products, in IEEE binary64 (the translation unit is compiled with
 * -ffp-contract=off, so no fused multiply-adds), for every input precision.
 *
 * Matrices are addressed through explicit row and column strides, so one
 * routine serves column-major operands with any leading dimension as well as
 * transposed views (A^T: row stride lda, column stride 1), which is what the
 * backward products dB = A^T dC and dA = dC B^T need.
 *
 * Parity pins (tests/test_oracle_pins.py): exact rational arithmetic on tiny
 * inputs, identity and permutation A (C = P B exactly), all-ones A (every row
 * equal to the column sums of B, bitwise equal across rows), small-integer
 * inputs (exact; compared with integer arithmetic), rank-one A, and the
 * long-double variant below.  The magnitude matrix S = |A||B| is pinned for
 * binary64 and binary32 inputs alike: exact integer arithmetic on signed
 * small integers (a dropped fabs on either operand fails) and the exact
 * rational sum of |a||b| on uniform binary32 inputs (a widening through a
 * narrower type fails).
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#include <math.h>

#define AT(P, i, j, rs, cs) (P)[(int64_t)(i) * (rs) + (int64_t)(j) * (cs)]

/* C = A B in binary64; A, B, C binary64. C is overwritten. */
void oracle_gemm_d(int64_t m, int64_t n, int64_t k,
                   const double *A, int64_t a_rs, int64_t a_cs,
                   const double *B, int64_t b_rs, int64_t b_cs,
                   double *C, int64_t c_rs, int64_t c_cs)
{
    for (int64_t c = 0; c < k; ++c) {
        for (int64_t i = 0; i < m; ++i) AT(C, i, c, c_rs, c_cs) = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            const double b = AT(B, j, c, b_rs, b_cs);
            for (int64_t i = 0; i < m; ++i)
                AT(C, i, c, c_rs, c_cs) = AT(C, i, c, c_rs, c_cs) + AT(A, i, j, a_rs, a_cs) * b;
        }
    }
}

/* Binary32 inputs, widened exactly to binary64; sums in binary64. */
void oracle_gemm_s(int64_t m, int64_t n, int64_t k,
                   const float *A, int64_t a_rs, int64_t a_cs,
                   const float *B, int64_t b_rs, int64_t b_cs,
                   double *C, int64_t c_rs, int64_t c_cs)
{
    for (int64_t c = 0; c < k; ++c) {
        for (int64_t i = 0; i < m; ++i) AT(C, i, c, c_rs, c_cs) = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            const double b = (double)AT(B, j, c, b_rs, b_cs);
            for (int64_t i = 0; i < m; ++i)
                AT(C, i, c, c_rs, c_cs) = AT(C, i, c, c_rs, c_cs) + (double)AT(A, i, j, a_rs, a_cs) * b;
        }
    }
}

/* S = |A| |B| (the magnitude matrix of the componentwise error bound). */
void oracle_absgemm_d(int64_t m, int64_t n, int64_t k,
                      const double *A, int64_t a_rs, int64_t a_cs,
                      const double *B, int64_t b_rs, int64_t b_cs,
                      double *S, int64_t s_rs, int64_t s_cs)
{
    for (int64_t c = 0; c < k; ++c) {
        for (int64_t i = 0; i < m; ++i) AT(S, i, c, s_rs, s_cs) = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            const double b = fabs(AT(B, j, c, b_rs, b_cs));
            for (int64_t i = 0; i < m; ++i)
                AT(S, i, c, s_rs, s_cs) = AT(S, i, c, s_rs, s_cs) + fabs(AT(A, i, j, a_rs, a_cs)) * b;
        }
    }
}

void oracle_absgemm_s(int64_t m, int64_t n, int64_t k,
                      const float *A, int64_t a_rs, int64_t a_cs,
                      const float *B, int64_t b_rs, int64_t b_cs,
                      double *S, int64_t s_rs, int64_t s_cs)
{
    for (int64_t c = 0; c < k; ++c) {
        for (int64_t i = 0; i < m; ++i) AT(S, i, c, s_rs, s_cs) = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            const double b = fabs((double)AT(B, j, c, b_rs, b_cs));
            for (int64_t i = 0; i < m; ++i)
                AT(S, i, c, s_rs, s_cs) = AT(S, i, c, s_rs, s_cs) + fabs((double)AT(A, i, j, a_rs, a_cs)) * b;
        }
    }
}

/* The same definition accumulated in long double (80-bit x87 on x86-64,
 * binary128 on AArch64), for checking the binary64 oracle itself. */
void oracle_gemm_ld(int64_t m, int64_t n, int64_t k,
                    const double *A, int64_t a_rs, int64_t a_cs,
                    const double *B, int64_t b_rs, int64_t b_cs,
                    long double *C, int64_t c_rs, int64_t c_cs)
{
    for (int64_t c = 0; c < k; ++c)
        for (int64_t i = 0; i < m; ++i) {
            long double acc = 0.0L;
            for (int64_t j = 0; j < n; ++j)
                acc += (long double)AT(A, i, j, a_rs, a_cs) * (long double)AT(B, j, c, b_rs, b_cs);
            AT(C, i, c, c_rs, c_cs) = acc;
        }
}

int oracle_long_double_mant_dig(void) { return __LDBL_MANT_DIG__; }

/*
 * Binary32 -> bfloat16, round to nearest, ties to even, written from the
 * format definitions: bfloat16 keeps the sign, the 8 exponent bits and the
 * top 7 fraction bits of binary32.  The discarded low 16 bits decide the
 * rounding: above half an ulp rounds up, below rounds down, exactly half
 * rounds to the even neighbour.  Adding 0x7FFF plus the kept lowest bit to
 * the bit pattern implements exactly that, and a carry out of the fraction
 * correctly bumps the exponent (up to infinity).  NaNs stay NaN (quiet).
 */
static uint16_t bf16_rne_one(float x)
{
    uint32_t u;
    memcpy(&u, &x, sizeof u);
    if ((u & 0x7F800000u) == 0x7F800000u && (u & 0x007FFFFFu) != 0u)
        return (uint16_t)((u >> 16) | 0x0040u);
    const uint32_t keep_lsb = (u >> 16) & 1u;
    u += 0x7FFFu + keep_lsb;
    return (uint16_t)(u >> 16);
}

void oracle_bf16_rne(int64_t count, const float *x, uint16_t *out)
{
    for (int64_t t = 0; t < count; ++t) out[t] = bf16_rne_one(x[t]);
}

float oracle_bf16_to_float(uint16_t h)
{
    uint32_t u = (uint32_t)h << 16;
    float f;
    memcpy(&f, &u, sizeof f);
    return f;
}

void oracle_bf16_to_float_n(int64_t count, const uint16_t *h, float *out)
{
    for (int64_t t = 0; t < count; ++t) out[t] = oracle_bf16_to_float(h[t]);
}
