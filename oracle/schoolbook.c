/*
 * Oracle: plain CPU schoolbook multiplication of unsigned integers.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this code.  The library's product
 * path never calls it.
 *
 * The product w = u v that every Toom-Cook variant must reach exactly
 * (Section 1: u = U(2^b), v = V(2^b), w = W(2^b) = u v) has a plain
 * definition, and this file writes that definition out: the integer
 * product computed limb by limb, one row a[i] * b[0..nb) at a time, with a
 * 64-bit accumulator.  No blocking, no reordering, no tricks.
 *
 * Limbs are little-endian uint32: limb i carries bits [32 i, 32 i + 32).
 * The result has exactly na + nb limbs (leading zeros kept).
 */
#include <stdint.h>
#include <stddef.h>

/* out[0 .. na+nb) = a[0 .. na) * b[0 .. nb).  out must not alias a or b. */
void oracle_schoolbook(const uint32_t *a, size_t na,
                       const uint32_t *b, size_t nb,
                       uint32_t *out)
{
    size_t i, j;
    for (i = 0; i < na + nb; ++i)
        out[i] = 0;
    for (i = 0; i < na; ++i) {
        uint64_t carry = 0;
        for (j = 0; j < nb; ++j) {
            /* (2^32-1)^2 + 2 (2^32-1) = 2^64 - 1: never overflows. */
            uint64_t t = (uint64_t)a[i] * (uint64_t)b[j]
                       + (uint64_t)out[i + j] + carry;
            out[i + j] = (uint32_t)t;
            carry = t >> 32;
        }
        out[i + nb] = (uint32_t)carry;
    }
}

/* Batched form: count independent products laid out back to back.
 * a_off/b_off/out_off are limb offsets into A/B/OUT; lengths in a_len/b_len;
 * product k occupies OUT[out_off[k] .. out_off[k] + a_len[k] + b_len[k]). */
void oracle_schoolbook_batch(size_t count,
                             const uint32_t *A, const int64_t *a_off, const int64_t *a_len,
                             const uint32_t *B, const int64_t *b_off, const int64_t *b_len,
                             uint32_t *OUT, const int64_t *out_off)
{
    size_t k;
    for (k = 0; k < count; ++k)
        oracle_schoolbook(A + a_off[k], (size_t)a_len[k],
                          B + b_off[k], (size_t)b_len[k],
                          OUT + out_off[k]);
}
