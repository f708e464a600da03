/*
 * scan_oracle.h -- plain sequential CPU scan used ONLY as test infrastructure.
 *
 * This is the correctness authority for the GPU scan library.  It shares no
 * code, header, table or helper with the CUDA path.  Only tests, the smoke
 * check and the benchmark's CPU-baseline leg may load it.
 *
 * Definition followed (LightScan, Section 1): for an associative operator (+)
 * and input x_0..x_{N-1}, the inclusive scan is y_j = x_0 (+) ... (+) x_j and
 * the exclusive scan is y_j = x_0 (+) ... (+) x_{j-1}, with y_0 = identity.
 *
 * Precision of the oracle (the paper fixes none; the readings are stated):
 *   int32 add : accumulated in 64-bit unsigned arithmetic, emitted mod 2^32
 *               (two's-complement wrap), i.e. the exact result of wrapping
 *               int32 addition.
 *   fp32/bf16 add : every input converted exactly to double and accumulated
 *               sequentially in double; the double is the reference value.
 *   int64 add : accumulated in 64-bit unsigned arithmetic (wrap mod 2^64).
 *   double add : accumulated sequentially in double-double arithmetic (a
 *               (hi, lo) pair updated with Knuth's two-sum, TAOCP vol. 2,
 *               4.2.2, and renormalised with Dekker's fast-two-sum), so the
 *               running sum carries ~106 bits; the reference value is
 *               hi + lo rounded to double.
 *   max       : exact; ties keep the EARLIER element (result bits are those of
 *               the first occurrence of the maximum).  Identity INT32_MIN /
 *               INT64_MIN for integers, -infinity for floats.  NaN inputs
 *               are outside the contract.
 *   bf16      : a bf16 value is the upper 16 bits of an IEEE binary32, so the
 *               decode is exact (bits << 16).
 *
 * Batched (segmented) scans: segment s is x[offsets[s] .. offsets[s+1]), each
 * scanned independently by the definition above.
 */
#ifndef SCAN_ORACLE_H
#define SCAN_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* op codes */
#define ORACLE_OP_ADD 0
#define ORACLE_OP_MAX 1
/* dtype codes */
#define ORACLE_I32  0
#define ORACLE_F32  1
#define ORACLE_BF16 2
#define ORACLE_I64  3
#define ORACLE_F64  4

/* Returns 0 on success, -1 on an unknown (op, dtype) or n < 0.
 * Output element type:
 *   (ADD, I32)  -> int32_t
 *   (ADD, F32)  -> double   (FP64 reference value)
 *   (ADD, BF16) -> double   (FP64 reference value)
 *   (MAX, I32)  -> int32_t
 *   (MAX, F32)  -> float    (bits of the selected element)
 *   (MAX, BF16) -> uint16_t (bits of the selected element)
 *   (ADD, I64)  -> int64_t
 *   (ADD, F64)  -> double   (double-double sum rounded to double)
 *   (MAX, I64)  -> int64_t
 *   (MAX, F64)  -> double   (bits of the selected element)            */
int oracle_scan(int op, int dtype, const void *x, void *y, int64_t n,
                int inclusive);

/* Same as oracle_scan for each segment [offsets[s], offsets[s+1]).
 * offsets has n_seg+1 entries, offsets[0] = 0, non-decreasing. */
int oracle_segscan(int op, int dtype, const void *x, void *y,
                   const int64_t *offsets, int64_t n_seg, int inclusive);

/* S_j = sum_{i<=j} |x_i| (inclusive) or sum_{i<j} |x_i| (exclusive), in double,
 * for float dtypes; used by the float error bound |err_j| <= c * S_j. */
int oracle_abs_prefix(int dtype, const void *x, double *s, int64_t n,
                      int inclusive);

/* Segmented version of oracle_abs_prefix. */
int oracle_abs_segprefix(int dtype, const void *x, double *s,
                         const int64_t *offsets, int64_t n_seg, int inclusive);

/* Stream compaction (a consumer of the scan; not in the paper): copies, in
 * order, every element x[j] (elem_size bytes) whose flag[j] is nonzero to
 * y[0..count) and returns count (-1 on bad arguments).  The output index of
 * a selected element is the exclusive prefix sum of the flags. */
int64_t oracle_select_flagged(const void *x, const uint8_t *flags, void *y,
                              int64_t n, int elem_size);

/* Radix-sort digit offsets (a consumer of the scan; not in the paper).
 * keys: n unsigned integers of key_bytes (4 or 8) bytes.  Digit p of a key
 * (p = 0 .. P-1, P = ceil(8 * key_bytes / digit_bits), lowest digit first)
 * is (key >> (p * digit_bits)) & (2^digit_bits - 1).  With B = 2^digit_bits,
 * offsets[p * B + v] is the number of keys whose digit p is less than v: the
 * exclusive prefix sum over v of the digit-p histogram, i.e. where bucket v
 * starts in a stable counting-sort pass on digit p.  Returns 0, or -1 on bad
 * arguments (key_bytes not 4 or 8, digit_bits outside 1..8, n < 0). */
int oracle_radix_offsets(const void *keys, int key_bytes, int64_t n,
                         int digit_bits, int64_t *offsets);

/* bf16 bit pattern -> double (exact). */
double oracle_bf16_to_double(uint16_t bits);

#ifdef __cplusplus
}
#endif
#endif
