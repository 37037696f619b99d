/*
 * CPU oracle for Onesweep LSD radix sorting (Adinets and Merrill,
 * "Onesweep: A Faster Least Significant Digit Radix Sort for GPUs",
 * arXiv 2206.01784).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library. The product path never
 * calls it, and it shares no code, header, table or helper with the CUDA
 * path: everything below is written out plainly from the paper.
 *
 * What it computes, and where the paper defines it:
 *  - the problem: ascending, stable sort of k-bit keys (optionally with
 *    payload values) by d-bit digit places, least significant place first,
 *    p = ceil(k/d) places (Section 1, "As a lexicographic sorting method ...";
 *    stability: Section 1, "LSD variants are necessarily stable");
 *  - signed / floating-point keys are first mapped to unsigned integers by an
 *    order-preserving ("magnitude-preserving") conversion, and mapped back on
 *    output (Section 3, chained scan digit-binning kernel): for two's
 *    complement keys the sign bit is inverted;
 *  - per-place digit histograms over the whole input (Section 3, phase 1 and
 *    Figure 5) and their exclusive prefix sums, the global bin offsets
 *    (Section 2 "Prefix sum", Section 3 phase 2);
 *  - one digit-binning pass: every key goes to its bin's global offset plus
 *    the number of earlier keys of the input with the same digit (Section 2,
 *    the flag prefix-sum example; Section 3, "Global bin offset" plus
 *    "bin-relative block offset");
 *  - per-tile digit counts, whose running sums over tiles are the values the
 *    chained scan leaves in its status counters (Section 3, Figure 7f).
 *
 * The oracle is slow on purpose: one key at a time, in input order, with
 * 64-bit counters and 64-bit working keys for every key type.
 *
 * Readings where the paper is silent (the same readings bind the CUDA path):
 *  - float keys: bijective sign-flip. A key with the sign bit set is bitwise
 *    inverted; otherwise only the sign bit is flipped. So -0.0 sorts before
 *    +0.0, and NaNs sort by bit pattern (negative NaNs first, positive last).
 *    Output keys carry the input bits unchanged;
 *  - a bit range [begin_bit, end_bit): places start at begin_bit and go
 *    upward; when (end_bit - begin_bit) is not a multiple of d the last (most
 *    significant) place is narrower;
 *  - equal keys keep their input order;
 *  - descending order (the paper sorts ascending only, Section 4): equal
 *    keys still keep their input order, and every place bins by the
 *    complement of its digit within the place (largest digit first), which is
 *    the ascending sort of the complemented field.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_U32 = 0, ORC_U64 = 1, ORC_F32 = 2, ORC_F64 = 3, ORC_I32 = 4, ORC_I64 = 5 };

/* Key width in bits for a key type. */
int orc_key_bits(int key_type) {
    return (key_type == ORC_U64 || key_type == ORC_F64 || key_type == ORC_I64) ? 64 : 32;
}

/*
 * Order-preserving map of a key's bits to an unsigned integer (Section 3:
 * "magnitude-preserving conversion to unsigned integer values").
 * Unsigned keys map to themselves. For IEEE-754 keys, a set sign bit means a
 * negative number, whose magnitude order is reversed, so all bits are
 * inverted; a clear sign bit only gets the sign bit set, which places every
 * non-negative number above every negative one.
 */
uint64_t orc_to_ordered(int key_type, uint64_t bits) {
    /* two's-complement keys: inverting the sign bit puts negative numbers
       below non-negative ones and keeps the order within each */
    if (key_type == ORC_I32) return (uint32_t)bits ^ 0x80000000u;
    if (key_type == ORC_I64) return bits ^ 0x8000000000000000ULL;
    if (key_type == ORC_F32) {
        uint32_t b = (uint32_t)bits;
        return (b & 0x80000000u) ? (uint32_t)~b : (b | 0x80000000u);
    }
    if (key_type == ORC_F64) {
        uint64_t sign = 0x8000000000000000ULL;
        return (bits & sign) ? ~bits : (bits | sign);
    }
    return bits;
}

/* Inverse of orc_to_ordered (applied when keys are written out). */
uint64_t orc_from_ordered(int key_type, uint64_t u) {
    if (key_type == ORC_I32) return (uint32_t)u ^ 0x80000000u;
    if (key_type == ORC_I64) return u ^ 0x8000000000000000ULL;
    if (key_type == ORC_F32) {
        uint32_t v = (uint32_t)u;
        return (v & 0x80000000u) ? (v & 0x7FFFFFFFu) : (uint32_t)~v;
    }
    if (key_type == ORC_F64) {
        uint64_t sign = 0x8000000000000000ULL;
        return (u & sign) ? (u & ~sign) : ~u;
    }
    return u;
}

/* Number of digit places p = ceil((end_bit - begin_bit) / d) (Section 1). */
int orc_num_places(int begin_bit, int end_bit, int radix_bits) {
    int k = end_bit - begin_bit;
    if (k <= 0) return 0;
    return (k + radix_bits - 1) / radix_bits;
}

/* First bit and width of digit place `place` (place 0 = least significant). */
static void place_bits(int begin_bit, int end_bit, int radix_bits, int place, int *shift, int *width) {
    *shift = begin_bit + place * radix_bits;
    int w = end_bit - *shift;
    *width = w < radix_bits ? w : radix_bits;
}

/* The digit of an ordered key at the place starting at `shift`, `width` bits wide. */
static uint64_t digit_of(uint64_t u, int shift, int width) {
    uint64_t mask = (width >= 64) ? ~0ULL : ((1ULL << width) - 1ULL);
    return (u >> shift) & mask;
}

/* The digit a pass bins by: the digit itself, or for a descending sort its
   complement within the place (2^width - 1 - digit). */
static uint64_t sort_digit(uint64_t u, int shift, int width, int descending) {
    uint64_t d = digit_of(u, shift, width);
    return descending ? ((1ULL << width) - 1ULL) - d : d;
}

static uint64_t load_key(int key_type, const void *keys, uint64_t i) {
    if (orc_key_bits(key_type) == 64) return ((const uint64_t *)keys)[i];
    return ((const uint32_t *)keys)[i];
}

static void store_key(int key_type, void *keys, uint64_t i, uint64_t bits) {
    if (orc_key_bits(key_type) == 64)
        ((uint64_t *)keys)[i] = bits;
    else
        ((uint32_t *)keys)[i] = (uint32_t)bits;
}

/*
 * Exclusive prefix sum (Section 2, "Prefix sum"): out[i] = in[0] + ... + in[i-1].
 * Example from the paper: <8,6,7,5,3,0,9,2> -> <0,8,14,21,26,29,29,38>.
 */
void orc_exclusive_sum(const uint64_t *in, int64_t count, uint64_t *out) {
    uint64_t running = 0;
    for (int64_t i = 0; i < count; ++i) {
        uint64_t v = in[i];
        out[i] = running;
        running += v;
    }
}

/*
 * Digit histograms of every digit place over the whole input (Section 3,
 * phase 1, "Histograms of global digit counts"; Figure 5).
 * hist is [p][2^radix_bits], row `place` counts the digits of that place.
 */
void orc_histograms_ex(int key_type, const void *keys, uint64_t n, int begin_bit, int end_bit,
                       int radix_bits, int descending, uint64_t *hist) {
    int p = orc_num_places(begin_bit, end_bit, radix_bits);
    uint64_t r = 1ULL << radix_bits;
    memset(hist, 0, sizeof(uint64_t) * (size_t)(p * r));
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t u = orc_to_ordered(key_type, load_key(key_type, keys, i));
        for (int place = 0; place < p; ++place) {
            int shift, width;
            place_bits(begin_bit, end_bit, radix_bits, place, &shift, &width);
            hist[place * r + sort_digit(u, shift, width, descending)] += 1;
        }
    }
}

void orc_histograms(int key_type, const void *keys, uint64_t n, int begin_bit, int end_bit,
                    int radix_bits, uint64_t *hist) {
    orc_histograms_ex(key_type, keys, n, begin_bit, end_bit, radix_bits, 0, hist);
}

/*
 * Global bin offsets of every place: the exclusive prefix sum of each place's
 * histogram (Section 3, phase 2, "Prefix sums of global digit counts").
 */
void orc_bin_offsets_ex(int key_type, const void *keys, uint64_t n, int begin_bit, int end_bit,
                        int radix_bits, int descending, uint64_t *offsets) {
    int p = orc_num_places(begin_bit, end_bit, radix_bits);
    uint64_t r = 1ULL << radix_bits;
    uint64_t *hist = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(p * r + 1));
    orc_histograms_ex(key_type, keys, n, begin_bit, end_bit, radix_bits, descending, hist);
    for (int place = 0; place < p; ++place) orc_exclusive_sum(hist + place * r, (int64_t)r, offsets + place * r);
    free(hist);
}

void orc_bin_offsets(int key_type, const void *keys, uint64_t n, int begin_bit, int end_bit,
                     int radix_bits, uint64_t *offsets) {
    orc_bin_offsets_ex(key_type, keys, n, begin_bit, end_bit, radix_bits, 0, offsets);
}

/*
 * One digit-binning pass over ordered keys (Section 2 "Prefix sum" and
 * Section 3 "High-level description"): a key's output index is its digit's
 * global bin offset plus the count of keys before it in the input with the
 * same digit. Walking the input in order and bumping a per-digit cursor
 * computes exactly that; values follow their keys.
 */
static void binning_pass(const uint64_t *in, const uint32_t *vin, uint64_t n, int shift, int width,
                         int descending, uint64_t *out, uint32_t *vout) {
    uint64_t r = 1ULL << width;
    uint64_t *count = (uint64_t *)calloc((size_t)r, sizeof(uint64_t));
    uint64_t *cursor = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)r);
    for (uint64_t i = 0; i < n; ++i) count[sort_digit(in[i], shift, width, descending)] += 1;
    orc_exclusive_sum(count, (int64_t)r, cursor);
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t d = sort_digit(in[i], shift, width, descending);
        uint64_t dst = cursor[d]++;
        out[dst] = in[i];
        if (vin) vout[dst] = vin[i];
    }
    free(count);
    free(cursor);
}

/*
 * LSD radix sort (Section 1; Section 3 phase 3): p binning passes, least
 * significant place first. vals_in / vals_out may be NULL (keys only).
 * keys_out receives the input key bits in stable ascending (descending != 0:
 * stable descending) order of the ordered field bits [begin_bit, end_bit).
 * Returns 0, or -1 on bad arguments.
 */
int orc_sort_ex(int key_type, const void *keys_in, const uint32_t *vals_in, uint64_t n, int begin_bit,
                int end_bit, int radix_bits, int descending, void *keys_out, uint32_t *vals_out) {
    int kbits = orc_key_bits(key_type);
    if (begin_bit < 0 || end_bit > kbits || begin_bit > end_bit || radix_bits < 1 || radix_bits > 16) return -1;
    if ((vals_in == NULL) != (vals_out == NULL)) return -1;
    int p = orc_num_places(begin_bit, end_bit, radix_bits);
    uint64_t *a = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n + 1));
    uint64_t *b = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n + 1));
    uint32_t *va = NULL, *vb = NULL;
    if (vals_in) {
        va = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n + 1));
        vb = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n + 1));
        memcpy(va, vals_in, sizeof(uint32_t) * (size_t)n);
    }
    for (uint64_t i = 0; i < n; ++i) a[i] = orc_to_ordered(key_type, load_key(key_type, keys_in, i));
    for (int place = 0; place < p; ++place) {
        int shift, width;
        place_bits(begin_bit, end_bit, radix_bits, place, &shift, &width);
        binning_pass(a, va, n, shift, width, descending, b, vb);
        uint64_t *t = a; a = b; b = t;
        uint32_t *tv = va; va = vb; vb = tv;
    }
    for (uint64_t i = 0; i < n; ++i) store_key(key_type, keys_out, i, orc_from_ordered(key_type, a[i]));
    if (vals_out) memcpy(vals_out, va, sizeof(uint32_t) * (size_t)n);
    free(a); free(b); free(va); free(vb);
    return 0;
}

int orc_sort(int key_type, const void *keys_in, const uint32_t *vals_in, uint64_t n, int begin_bit,
             int end_bit, int radix_bits, void *keys_out, uint32_t *vals_out) {
    return orc_sort_ex(key_type, keys_in, vals_in, n, begin_bit, end_bit, radix_bits, 0, keys_out, vals_out);
}

/*
 * The input after the first `passes` binning passes only (passes <= p), in
 * the original key bits. With passes = 1 this is the output of one
 * digit-binning iteration over place 0.
 */
int orc_sort_passes(int key_type, const void *keys_in, const uint32_t *vals_in, uint64_t n, int begin_bit,
                    int end_bit, int radix_bits, int passes, void *keys_out, uint32_t *vals_out) {
    int p = orc_num_places(begin_bit, end_bit, radix_bits);
    if (passes < 0 || passes > p) return -1;
    int end = begin_bit + passes * radix_bits;
    if (end > end_bit) end = end_bit;
    return orc_sort(key_type, keys_in, vals_in, n, begin_bit, end, radix_bits, keys_out, vals_out);
}

/* Segmented form: each segment [offsets[s], offsets[s+1]) sorted on its own. */
int orc_sort_segments_ex(int key_type, const void *keys_in, const uint32_t *vals_in, const uint64_t *offsets,
                         int64_t num_segments, int begin_bit, int end_bit, int radix_bits, int descending,
                         void *keys_out, uint32_t *vals_out) {
    size_t kb = (size_t)orc_key_bits(key_type) / 8;
    for (int64_t s = 0; s < num_segments; ++s) {
        uint64_t lo = offsets[s], hi = offsets[s + 1];
        if (hi < lo) return -1;
        int rc = orc_sort_ex(key_type, (const char *)keys_in + lo * kb, vals_in ? vals_in + lo : NULL, hi - lo,
                             begin_bit, end_bit, radix_bits, descending, (char *)keys_out + lo * kb,
                             vals_out ? vals_out + lo : NULL);
        if (rc) return rc;
    }
    return 0;
}

int orc_sort_segments(int key_type, const void *keys_in, const uint32_t *vals_in, const uint64_t *offsets,
                      int64_t num_segments, int begin_bit, int end_bit, int radix_bits, void *keys_out,
                      uint32_t *vals_out) {
    return orc_sort_segments_ex(key_type, keys_in, vals_in, offsets, num_segments, begin_bit, end_bit, radix_bits,
                                0, keys_out, vals_out);
}

/*
 * Per-tile digit counts of one place over the input of that pass (tiles of
 * `tile` consecutive keys; the last one may be short): counts[t][digit].
 * In the chained scan, tile t's status counter for a digit ends holding the
 * inclusive sum of these counts over tiles 0..t (Section 3, Figure 7f).
 */
int orc_tile_digit_counts(int key_type, const void *keys, uint64_t n, int shift, int width, uint64_t tile,
                          uint64_t *counts) {
    if (tile == 0) return -1;
    uint64_t r = 1ULL << width;
    uint64_t tiles = (n + tile - 1) / tile;
    memset(counts, 0, sizeof(uint64_t) * (size_t)(tiles * r));
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t u = orc_to_ordered(key_type, load_key(key_type, keys, i));
        counts[(i / tile) * r + digit_of(u, shift, width)] += 1;
    }
    return 0;
}
