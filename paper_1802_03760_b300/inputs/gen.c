/*
 * Seeded synthetic inputs for the subgraph-query workloads: directed
 * Erdos-Renyi edge sets, R-MAT edge samples (Chakrabarti, Zhan, Faloutsos,
 * SDM 2004) with a seeded vertex relabelling, planted hub vertices, and the
 * uniform index draws used by update streams.
 *
 * This module only produces inputs. It holds no part of the join method:
 * no index building, no prefix extension, no counting. Both the CPU oracle
 * and the CUDA path consume its output, and neither is imported here.
 *
 * Randomness is counter based: every draw is a pure function of
 * (seed, counter) through the SplitMix64 output function (Steele, Lea,
 * Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014),
 * so results do not depend on the thread count.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN 0x9e3779b97f4a7c15ULL

static inline uint64_t sm64_out(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* The ctr-th output of a SplitMix64 stream started at state `seed`. */
uint64_t gjin_rand(uint64_t seed, uint64_t ctr) {
    return sm64_out(seed + (ctr + 1) * GOLDEN);
}

/* Uniform integer in [0, bound) from a 64-bit draw (multiply-high). */
static inline uint64_t below(uint64_t r, uint64_t bound) {
    return (uint64_t)(((unsigned __int128)r * bound) >> 64);
}

/*
 * Directed Erdos-Renyi edge set: draws (u, v) pairs uniformly from
 * [0,n)^2 until m distinct pairs with u != v have been seen, in draw order.
 * Returns m, or -1 if m > n(n-1) or memory runs out.
 */
int64_t gjin_er(uint32_t n, uint64_t m, uint64_t seed, uint32_t* src, uint32_t* dst) {
    if (n < 2 || m > (uint64_t)n * (n - 1)) return -1;
    uint64_t nbits = (uint64_t)n * n;
    uint64_t* seen = (uint64_t*)calloc((nbits + 63) / 64, sizeof(uint64_t));
    if (!seen) return -1;
    uint64_t got = 0, ctr = 0;
    while (got < m) {
        uint64_t r = gjin_rand(seed, ctr++);
        /* two 32-bit halves, each scaled to [0, n) by multiply-high */
        uint32_t u = (uint32_t)(((r & 0xffffffffULL) * (uint64_t)n) >> 32);
        uint32_t v = (uint32_t)(((r >> 32) * (uint64_t)n) >> 32);
        if (u == v) continue;
        uint64_t bit = (uint64_t)u * n + v;
        if (seen[bit >> 6] & (1ULL << (bit & 63))) continue;
        seen[bit >> 6] |= 1ULL << (bit & 63);
        src[got] = u;
        dst[got] = v;
        got++;
    }
    free(seen);
    return (int64_t)got;
}

/* Seeded uniform permutation of [0, n) (Fisher-Yates, Knuth Algorithm P). */
void gjin_permutation(uint32_t n, uint64_t seed, uint32_t* perm) {
    for (uint32_t i = 0; i < n; i++) perm[i] = i;
    for (uint32_t i = n; i > 1; i--) {
        uint32_t j = (uint32_t)below(gjin_rand(seed, i), i);
        uint32_t t = perm[i - 1];
        perm[i - 1] = perm[j];
        perm[j] = t;
    }
}

/*
 * R-MAT samples number first .. first+count-1 of the stream `seed` on
 * 2^scale vertices with quadrant probabilities (a, b, c, 1-a-b-c). At each
 * of the `scale` recursion levels, a 53-bit uniform picks the quadrant; the
 * first level decides the most significant bit. No noise is added. If perm
 * is not NULL, both endpoints are relabelled through it. Duplicates and
 * self-loops are kept: they are raw samples.
 */
void gjin_rmat(uint32_t scale, uint64_t first, uint64_t count, uint64_t seed,
               double a, double b, double c, const uint32_t* perm,
               uint32_t* src, uint32_t* dst) {
    const double ab = a + b, abc = a + b + c;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)count; i++) {
        uint64_t e = first + (uint64_t)i;
        uint32_t u = 0, v = 0;
        for (uint32_t l = 0; l < scale; l++) {
            uint64_t r = gjin_rand(seed, e * 64 + l);
            double x = (double)(r >> 11) * (1.0 / 9007199254740992.0);
            uint32_t bu, bv;
            if (x < a) { bu = 0; bv = 0; }
            else if (x < ab) { bu = 0; bv = 1; }
            else if (x < abc) { bu = 1; bv = 0; }
            else { bu = 1; bv = 1; }
            u = (u << 1) | bu;
            v = (v << 1) | bv;
        }
        if (perm) { u = perm[u]; v = perm[v]; }
        src[i] = u;
        dst[i] = v;
    }
}

/*
 * Planted hubs: for hub h (h = 0..nhubs-1, id hub_ids[h]) writes deg
 * distinct out-neighbours and deg distinct in-neighbours drawn uniformly
 * from [0, n) without the hub itself. Output layout: hub h's out-edges at
 * [2*h*deg, 2*h*deg + deg), its in-edges right after. Returns 0, or -1 if
 * deg >= n or memory runs out.
 */
int gjin_hubs(uint32_t n, uint32_t nhubs, uint64_t deg, uint64_t seed,
              const uint32_t* hub_ids, uint32_t* src, uint32_t* dst) {
    if (deg >= n) return -1;
    int err = 0;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < 2 * (int64_t)nhubs; t++) {
        uint32_t h = (uint32_t)(t / 2);
        int in_dir = (int)(t % 2);
        uint64_t* seen = (uint64_t*)calloc(((uint64_t)n + 63) / 64, sizeof(uint64_t));
        if (!seen) { err = -1; continue; }
        uint32_t hub = hub_ids[h];
        seen[hub >> 6] |= 1ULL << (hub & 63);
        uint64_t base = 2 * (uint64_t)h * deg + (in_dir ? deg : 0);
        uint64_t got = 0, ctr = 0;
        uint64_t s2 = seed ^ (0x5bd1e995ULL * (uint64_t)(t + 1));
        while (got < deg) {
            uint32_t x = (uint32_t)below(gjin_rand(s2, ctr++), n);
            if (seen[x >> 6] & (1ULL << (x & 63))) continue;
            seen[x >> 6] |= 1ULL << (x & 63);
            if (in_dir) { src[base + got] = x; dst[base + got] = hub; }
            else { src[base + got] = hub; dst[base + got] = x; }
            got++;
        }
        free(seen);
    }
    return err;
}

/* count uniform draws in [0, bound): out[i] = below(rand(seed, first+i), bound). */
void gjin_uniform(uint64_t bound, uint64_t first, uint64_t count, uint64_t seed, uint64_t* out) {
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)count; i++)
        out[i] = below(gjin_rand(seed, first + (uint64_t)i), bound);
}
