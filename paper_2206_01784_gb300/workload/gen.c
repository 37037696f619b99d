/*
 * Seeded synthetic workloads for the Onesweep radix sort (arXiv 2206.01784).
 *
 * This module only draws inputs. It holds none of the sort's arithmetic and is
 * the one piece of code that both the CUDA path and the CPU oracle are fed
 * from. Every draw is counter-based, so element i of any array can be
 * produced independently of the others (and in parallel).
 *
 * Random source: SplitMix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), written from its published
 * definition: the state advances by the golden-ratio Weyl increment and each
 * output is the state passed through the variant-13 finaliser.
 *
 * Key distributions follow the paper's evaluation (Section 4):
 *  - Thearling-Smith entropy bands: a key is the bitwise AND of q independent
 *    uniform words, so each bit is set with probability 2^-q (Table 1 gives
 *    the resulting Shannon entropy per bit);
 *  - all-equal keys (the degenerate one-bin case);
 *  - float keys drawn N(0,1) with a few signed zeros and duplicates, to
 *    exercise the order-preserving float transform.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>

#define WL_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t wl_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Output number i (0-based) of the SplitMix64 generator seeded with `seed`. */
uint64_t wl_splitmix64(uint64_t seed, uint64_t i) {
    return wl_mix(seed + (i + 1) * WL_GAMMA);
}

/* Seed of independent stream `stream` derived from a user seed. */
uint64_t wl_stream_seed(uint64_t seed, uint64_t stream) {
    return wl_splitmix64(seed ^ 0x6A09E667F3BCC909ULL, stream);
}

/* Uniform double in [0,1) with 53 random bits. */
static inline double wl_unit(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

/* out[i] = AND of q uniform 32-bit words (upper halves of stream w = 0..q-1). */
void wl_u32_and(uint32_t *out, uint64_t n, uint64_t seed, int q) {
    uint64_t s[64];
    if (q < 1) q = 1;
    if (q > 64) q = 64;
    for (int w = 0; w < q; ++w) s[w] = wl_stream_seed(seed, (uint64_t)w);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) {
        uint32_t k = 0xFFFFFFFFu;
        for (int w = 0; w < q; ++w) k &= (uint32_t)(wl_splitmix64(s[w], (uint64_t)i) >> 32);
        out[i] = k;
    }
}

/* out[i] = AND of q uniform 64-bit words. */
void wl_u64_and(uint64_t *out, uint64_t n, uint64_t seed, int q) {
    uint64_t s[64];
    if (q < 1) q = 1;
    if (q > 64) q = 64;
    for (int w = 0; w < q; ++w) s[w] = wl_stream_seed(seed, (uint64_t)w);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) {
        uint64_t k = ~0ULL;
        for (int w = 0; w < q; ++w) k &= wl_splitmix64(s[w], (uint64_t)i);
        out[i] = k;
    }
}

/* All-equal keys: every element is the first draw of the seed's stream 0. */
void wl_u32_const(uint32_t *out, uint64_t n, uint64_t seed) {
    uint32_t k = (uint32_t)(wl_splitmix64(wl_stream_seed(seed, 0), 0) >> 32);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) out[i] = k;
}

void wl_u64_const(uint64_t *out, uint64_t n, uint64_t seed) {
    uint64_t k = wl_splitmix64(wl_stream_seed(seed, 0), 0);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) out[i] = k;
}

/* Box-Muller normal deviate number i of the pair of streams (s0, s1). */
static inline double wl_normal_at(uint64_t s0, uint64_t s1, uint64_t i) {
    double u1 = 1.0 - wl_unit(wl_splitmix64(s0, i)); /* (0,1] so log is finite */
    double u2 = wl_unit(wl_splitmix64(s1, i));
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925 * u2);
}

/*
 * Float keys drawn N(0,1) with structure for the sign-flip transform:
 * a uniform draw u per element picks
 *   u < 0.005        -> -0.0
 *   0.005 <= u < 0.01 -> +0.0
 *   0.01  <= u < 0.02 -> the normal value of a uniformly chosen other element
 *                        (a duplicate)
 *   otherwise         -> the element's own normal value.
 * Written as raw IEEE-754 bits.
 */
void wl_f32_normal(uint32_t *out_bits, uint64_t n, uint64_t seed) {
    uint64_t s0 = wl_stream_seed(seed, 0), s1 = wl_stream_seed(seed, 1);
    uint64_t s2 = wl_stream_seed(seed, 2), s3 = wl_stream_seed(seed, 3);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) {
        double u = wl_unit(wl_splitmix64(s2, (uint64_t)i));
        union { float f; uint32_t b; } v;
        if (u < 0.005) {
            v.f = -0.0f;
        } else if (u < 0.01) {
            v.f = 0.0f;
        } else {
            uint64_t src = (uint64_t)i;
            if (u < 0.02 && n > 0) src = wl_splitmix64(s3, (uint64_t)i) % n;
            v.f = (float)wl_normal_at(s0, s1, src);
        }
        out_bits[i] = v.b;
    }
}

/* Same recipe in double precision (raw bits). */
void wl_f64_normal(uint64_t *out_bits, uint64_t n, uint64_t seed) {
    uint64_t s0 = wl_stream_seed(seed, 0), s1 = wl_stream_seed(seed, 1);
    uint64_t s2 = wl_stream_seed(seed, 2), s3 = wl_stream_seed(seed, 3);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) {
        double u = wl_unit(wl_splitmix64(s2, (uint64_t)i));
        union { double f; uint64_t b; } v;
        if (u < 0.005) {
            v.f = -0.0;
        } else if (u < 0.01) {
            v.f = 0.0;
        } else {
            uint64_t src = (uint64_t)i;
            if (u < 0.02 && n > 0) src = wl_splitmix64(s3, (uint64_t)i) % n;
            v.f = wl_normal_at(s0, s1, src);
        }
        out_bits[i] = v.b;
    }
}

/* out[i] = i (the index payload used to check stability). */
void wl_iota_u32(uint32_t *out, uint64_t n) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) out[i] = (uint32_t)i;
}

/* Uniform doubles in [0,1) from stream `stream` of `seed`. */
void wl_uniform01(double *out, uint64_t n, uint64_t seed, uint64_t stream) {
    uint64_t s = wl_stream_seed(seed, stream);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) out[i] = wl_unit(wl_splitmix64(s, (uint64_t)i));
}

/* Standard normal doubles (Box-Muller) from streams (2*stream, 2*stream+1). */
void wl_normal(double *out, uint64_t n, uint64_t seed, uint64_t stream) {
    uint64_t s0 = wl_stream_seed(seed, 2 * stream), s1 = wl_stream_seed(seed, 2 * stream + 1);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) out[i] = wl_normal_at(s0, s1, (uint64_t)i);
}
