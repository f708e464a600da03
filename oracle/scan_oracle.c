/*
 * scan_oracle.c -- plain sequential CPU scan (TEST INFRASTRUCTURE ONLY).
 *
 * Every function is the definition of scan from LightScan Section 1 written
 * out as one sequential loop: acc starts at the identity of the operator; for
 * j = 0..n-1 the exclusive result is acc before the update and the inclusive
 * result is acc after acc = acc (+) x_j.  There is no blocking, tiling or
 * reordering.  The paper fixes no precision; the accumulation types are
 * stated in scan_oracle.h.
 *
 * Nothing in the GPU library includes or links this file.
 */
#include "scan_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

double oracle_bf16_to_double(uint16_t bits) {
    /* bf16 is the high half of an IEEE binary32 word. */
    uint32_t w = ((uint32_t)bits) << 16;
    float f;
    memcpy(&f, &w, sizeof f);
    return (double)f;
}

static double f32_to_double(float v) { return (double)v; }

/* ---- int32 add: wrapping two's-complement sum ------------------------ */
static void scan_i32_add(const int32_t *x, int32_t *y, int64_t n, int incl) {
    uint64_t acc = 0; /* identity of + ; unsigned so overflow is defined */
    for (int64_t j = 0; j < n; ++j) {
        if (!incl) y[j] = (int32_t)(uint32_t)acc;
        acc += (uint64_t)(int64_t)x[j];
        if (incl) y[j] = (int32_t)(uint32_t)acc;
    }
}

/* ---- int32 max ----------------------------------------------------- */
static void scan_i32_max(const int32_t *x, int32_t *y, int64_t n, int incl) {
    int32_t acc = INT32_MIN; /* identity of max */
    for (int64_t j = 0; j < n; ++j) {
        if (!incl) y[j] = acc;
        if (x[j] > acc) acc = x[j]; /* tie keeps the earlier value */
        if (incl) y[j] = acc;
    }
}

/* ---- fp32 add: exact widening, FP64 sequential sum ------------------ */
static void scan_f32_add(const float *x, double *y, int64_t n, int incl) {
    double acc = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        if (!incl) y[j] = acc;
        acc += f32_to_double(x[j]);
        if (incl) y[j] = acc;
    }
}

/* ---- fp32 max: first occurrence of the maximum ---------------------- */
static void scan_f32_max(const float *x, float *y, int64_t n, int incl) {
    float acc = -INFINITY;
    for (int64_t j = 0; j < n; ++j) {
        if (!incl) y[j] = acc;
        if (x[j] > acc) acc = x[j]; /* strict: a tie keeps the earlier bits */
        if (incl) y[j] = acc;
    }
}

/* ---- bf16 add: exact widening, FP64 sequential sum ------------------ */
static void scan_bf16_add(const uint16_t *x, double *y, int64_t n, int incl) {
    double acc = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        if (!incl) y[j] = acc;
        acc += oracle_bf16_to_double(x[j]);
        if (incl) y[j] = acc;
    }
}

/* ---- bf16 max: compare decoded values, emit the selected bits ------- */
static void scan_bf16_max(const uint16_t *x, uint16_t *y, int64_t n, int incl) {
    const uint16_t neg_inf_bits = 0xFF80u; /* bf16 -infinity */
    uint16_t acc_bits = neg_inf_bits;
    double acc = -INFINITY;
    for (int64_t j = 0; j < n; ++j) {
        if (!incl) y[j] = acc_bits;
        double v = oracle_bf16_to_double(x[j]);
        if (v > acc) {
            acc = v;
            acc_bits = x[j];
        }
        if (incl) y[j] = acc_bits;
    }
}

/* ---- int64 add: wrapping two's-complement sum ------------------------ */
static void scan_i64_add(const int64_t *x, int64_t *y, int64_t n, int incl) {
    uint64_t acc = 0; /* unsigned: overflow wraps mod 2^64, defined in C */
    for (int64_t j = 0; j < n; ++j) {
        if (!incl) y[j] = (int64_t)acc;
        acc += (uint64_t)x[j];
        if (incl) y[j] = (int64_t)acc;
    }
}

/* ---- int64 max ----------------------------------------------------- */
static void scan_i64_max(const int64_t *x, int64_t *y, int64_t n, int incl) {
    int64_t acc = INT64_MIN;
    for (int64_t j = 0; j < n; ++j) {
        if (!incl) y[j] = acc;
        if (x[j] > acc) acc = x[j];
        if (incl) y[j] = acc;
    }
}

/* ---- double add: sequential double-double accumulation --------------- */
static void scan_f64_add(const double *x, double *y, int64_t n, int incl) {
    double hi = 0.0, lo = 0.0; /* the running sum is hi + lo */
    for (int64_t j = 0; j < n; ++j) {
        if (!incl) y[j] = hi + lo;
        /* two-sum: s + e == hi + x_j exactly */
        double s = hi + x[j];
        double bb = s - hi;
        double e = (hi - (s - bb)) + (x[j] - bb);
        /* fold the error into lo, then renormalise (fast-two-sum, |s| >= |lo|) */
        lo += e;
        double t = s + lo;
        lo = lo - (t - s);
        hi = t;
        if (incl) y[j] = hi + lo;
    }
}

/* ---- double max: first occurrence of the maximum -------------------- */
static void scan_f64_max(const double *x, double *y, int64_t n, int incl) {
    double acc = -INFINITY;
    for (int64_t j = 0; j < n; ++j) {
        if (!incl) y[j] = acc;
        if (x[j] > acc) acc = x[j]; /* strict: a tie keeps the earlier bits */
        if (incl) y[j] = acc;
    }
}

static int out_size(int op, int dtype) {
    if (op == ORACLE_OP_ADD) {
        if (dtype == ORACLE_I32) return 4;
        if (dtype == ORACLE_F32 || dtype == ORACLE_BF16) return 8;
        if (dtype == ORACLE_I64 || dtype == ORACLE_F64) return 8;
    } else if (op == ORACLE_OP_MAX) {
        if (dtype == ORACLE_I32 || dtype == ORACLE_F32) return 4;
        if (dtype == ORACLE_BF16) return 2;
        if (dtype == ORACLE_I64 || dtype == ORACLE_F64) return 8;
    }
    return 0;
}

static int in_size(int dtype) {
    if (dtype == ORACLE_I32 || dtype == ORACLE_F32) return 4;
    if (dtype == ORACLE_BF16) return 2;
    if (dtype == ORACLE_I64 || dtype == ORACLE_F64) return 8;
    return 0;
}

int oracle_scan(int op, int dtype, const void *x, void *y, int64_t n,
                int inclusive) {
    if (n < 0 || out_size(op, dtype) == 0) return -1;
    int incl = inclusive != 0;
    if (op == ORACLE_OP_ADD && dtype == ORACLE_I32)
        scan_i32_add((const int32_t *)x, (int32_t *)y, n, incl);
    else if (op == ORACLE_OP_MAX && dtype == ORACLE_I32)
        scan_i32_max((const int32_t *)x, (int32_t *)y, n, incl);
    else if (op == ORACLE_OP_ADD && dtype == ORACLE_F32)
        scan_f32_add((const float *)x, (double *)y, n, incl);
    else if (op == ORACLE_OP_MAX && dtype == ORACLE_F32)
        scan_f32_max((const float *)x, (float *)y, n, incl);
    else if (op == ORACLE_OP_ADD && dtype == ORACLE_BF16)
        scan_bf16_add((const uint16_t *)x, (double *)y, n, incl);
    else if (op == ORACLE_OP_MAX && dtype == ORACLE_BF16)
        scan_bf16_max((const uint16_t *)x, (uint16_t *)y, n, incl);
    else if (op == ORACLE_OP_ADD && dtype == ORACLE_I64)
        scan_i64_add((const int64_t *)x, (int64_t *)y, n, incl);
    else if (op == ORACLE_OP_MAX && dtype == ORACLE_I64)
        scan_i64_max((const int64_t *)x, (int64_t *)y, n, incl);
    else if (op == ORACLE_OP_ADD && dtype == ORACLE_F64)
        scan_f64_add((const double *)x, (double *)y, n, incl);
    else
        scan_f64_max((const double *)x, (double *)y, n, incl);
    return 0;
}

int oracle_segscan(int op, int dtype, const void *x, void *y,
                   const int64_t *offsets, int64_t n_seg, int inclusive) {
    int isz = in_size(dtype), osz = out_size(op, dtype);
    if (n_seg < 0 || osz == 0 || offsets[0] != 0) return -1;
    for (int64_t s = 0; s < n_seg; ++s) {
        int64_t a = offsets[s], b = offsets[s + 1];
        if (b < a) return -1;
        const char *xs = (const char *)x + a * isz;
        char *ys = (char *)y + a * osz;
        if (oracle_scan(op, dtype, xs, ys, b - a, inclusive) != 0) return -1;
    }
    return 0;
}

int64_t oracle_select_flagged(const void *x, const uint8_t *flags, void *y,
                              int64_t n, int elem_size) {
    if (n < 0 || elem_size <= 0) return -1;
    int64_t k = 0; /* selected so far = exclusive prefix sum of the flags */
    for (int64_t j = 0; j < n; ++j) {
        if (flags[j] != 0) {
            memcpy((char *)y + k * elem_size, (const char *)x + j * elem_size,
                   (size_t)elem_size);
            ++k;
        }
    }
    return k;
}

int oracle_radix_offsets(const void *keys, int key_bytes, int64_t n,
                         int digit_bits, int64_t *offsets) {
    if ((key_bytes != 4 && key_bytes != 8) || digit_bits < 1 || digit_bits > 8 ||
        n < 0)
        return -1;
    const int key_bits = 8 * key_bytes;
    const int P = (key_bits + digit_bits - 1) / digit_bits;
    const int B = 1 << digit_bits;
    const uint64_t mask = (uint64_t)B - 1u;
    /* histogram of every digit position ... */
    int64_t *count = (int64_t *)calloc((size_t)P * (size_t)B, sizeof(int64_t));
    if (count == NULL) return -1;
    for (int64_t j = 0; j < n; ++j) {
        const uint64_t k = key_bytes == 4 ? (uint64_t)((const uint32_t *)keys)[j]
                                          : ((const uint64_t *)keys)[j];
        for (int p = 0; p < P; ++p)
            ++count[(size_t)p * B + ((k >> (p * digit_bits)) & mask)];
    }
    /* ... then its exclusive scan over the digit values (Section 1) */
    for (int p = 0; p < P; ++p) {
        int64_t acc = 0;
        for (int v = 0; v < B; ++v) {
            offsets[(size_t)p * B + v] = acc;
            acc += count[(size_t)p * B + v];
        }
    }
    free(count);
    return 0;
}

int oracle_abs_prefix(int dtype, const void *x, double *s, int64_t n,
                      int inclusive) {
    if (n < 0) return -1;
    double acc = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        double v;
        if (dtype == ORACLE_F32)
            v = f32_to_double(((const float *)x)[j]);
        else if (dtype == ORACLE_BF16)
            v = oracle_bf16_to_double(((const uint16_t *)x)[j]);
        else if (dtype == ORACLE_I32)
            v = (double)((const int32_t *)x)[j];
        else if (dtype == ORACLE_F64)
            v = ((const double *)x)[j];
        else
            return -1;
        if (!inclusive) s[j] = acc;
        acc += fabs(v);
        if (inclusive) s[j] = acc;
    }
    return 0;
}

int oracle_abs_segprefix(int dtype, const void *x, double *s,
                         const int64_t *offsets, int64_t n_seg, int inclusive) {
    int isz = in_size(dtype);
    if (n_seg < 0 || isz == 0 || offsets[0] != 0) return -1;
    for (int64_t k = 0; k < n_seg; ++k) {
        int64_t a = offsets[k], b = offsets[k + 1];
        if (b < a) return -1;
        if (oracle_abs_prefix(dtype, (const char *)x + a * isz, s + a, b - a,
                              inclusive) != 0)
            return -1;
    }
    return 0;
}
