/*
 * Seeded synthetic graph inputs shared by the oracle and the CUDA engine.
 *
 * This file generates INPUTS only: edge lists, the destination-sorted
 * compressed-sparse-column (CSC) layout that the engine's boundary takes,
 * SSSP edge weights and traversal roots.  It holds none of the method's
 * arithmetic (no frontier, no transform, no pull step, no application).
 *
 * Random numbers come from one counter-based generator: the n-th output of
 * SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014) started at state `seed`, i.e.
 *     rand(seed, n) = mix64(seed + (n + 1) * 0x9E3779B97F4A7C15)
 * with mix64 the SplitMix64 output function.  Because every draw is addressed
 * by its counter, the parallel loops below give the same bytes for any
 * number of threads.
 *
 * Workloads:
 *  - R-MAT (Chakrabarti, Zhan, Faloutsos, SDM 2004): ef * 2^scale edge
 *    samples, one quadrant choice per bit level, most significant bit first,
 *    quadrant probabilities a (0,0), b (0,1), c (1,0), d = 1-a-b-c (1,1) with
 *    the row bit giving the source and the column bit the destination.  Each
 *    64-bit draw serves two levels (two 32-bit halves compared against
 *    thresholds floor(p * 2^32)).  No noise, no vertex permutation.
 *  - 2D grid: n x n vertices, id = row * n + col, undirected 4-neighbour
 *    edges; each undirected edge is rewired with probability p by replacing
 *    its far endpoint with a uniform vertex (Watts-Strogatz style); both
 *    directions are then emitted.
 *  - Self-loops and duplicate edges are removed; E is counted after that.
 *  - SSSP weights: w(u,v) = 1 + (fmix32(u*0x9E3779B1 ^ rotl32(v*0x85EBCA77,15)
 *    ^ seed) mod W) where fmix32 is the MurmurHash3 32-bit finaliser; for
 *    undirected inputs (u,v) is taken as (min,max) so that w(u,v) = w(v,u).
 *    The paper only says its weights come from a multiplicative hash
 *    (Section 5, "Applications"); this formula is our reading of that.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GOLDEN64 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* n-th output of SplitMix64 seeded with `seed` (n counts from 0). */
uint64_t gg_rand(uint64_t seed, uint64_t n) {
    return mix64(seed + (n + 1) * GOLDEN64);
}

static inline uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85EBCA6BU;
    h ^= h >> 13;
    h *= 0xC2B2AE35U;
    h ^= h >> 16;
    return h;
}

static inline uint32_t rotl32(uint32_t x, int r) { return (x << r) | (x >> (32 - r)); }

uint32_t gg_weight(uint32_t u, uint32_t v, uint32_t seed, uint32_t wmax) {
    uint32_t h = fmix32((u * 0x9E3779B1U) ^ rotl32(v * 0x85EBCA77U, 15) ^ seed);
    return 1U + h % wmax;
}

static inline int quadrant(uint32_t r, uint32_t ta, uint32_t tab, uint32_t tabc) {
    if (r < ta) return 0;
    if (r < tab) return 1;
    if (r < tabc) return 2;
    return 3;
}

/* Writes m = ef << scale keys (dst << 32 | src), duplicates and self-loops
 * included.  ta/tab/tabc are the cumulative thresholds floor(p * 2^32). */
void gg_rmat_keys(int scale, uint64_t m, uint32_t ta, uint32_t tab, uint32_t tabc,
                  uint64_t seed, uint64_t* keys) {
    const uint64_t draws = (uint64_t)((scale + 1) / 2);
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < (int64_t)m; ++i) {
        uint32_t u = 0, v = 0;
        int level = 0;
        for (uint64_t j = 0; j < draws; ++j) {
            uint64_t r = gg_rand(seed, (uint64_t)i * draws + j);
            for (int h = 0; h < 2 && level < scale; ++h, ++level) {
                uint32_t r32 = (uint32_t)(h == 0 ? (r >> 32) : r);
                int q = quadrant(r32, ta, tab, tabc);
                u = (u << 1) | (uint32_t)(q >> 1);
                v = (v << 1) | (uint32_t)(q & 1);
            }
        }
        keys[i] = ((uint64_t)v << 32) | u;
    }
}

/* n x n grid.  p_thresh = floor(p * 2^64) as the rewiring test on a 64-bit
 * draw (0 means never).  Writes both directions of each undirected edge into
 * keys (capacity 4 * n * n) and returns the number written. */
uint64_t gg_grid_keys(uint32_t n, uint64_t p_thresh, uint64_t seed, uint64_t* keys) {
    const uint64_t V = (uint64_t)n * n;
    int64_t id;
#pragma omp parallel for schedule(static)
    for (id = 0; id < (int64_t)V; ++id) {
        uint32_t r = (uint32_t)(id / n), c = (uint32_t)(id % n);
        for (int dir = 0; dir < 2; ++dir) {
            uint64_t e = 2 * (uint64_t)id + dir;
            uint64_t slot = 2 * e;
            int exists = dir == 0 ? (c + 1 < n) : (r + 1 < n);
            if (!exists) {
                keys[slot] = keys[slot + 1] = ~0ULL; /* placeholder, dropped later */
                continue;
            }
            uint32_t a = (uint32_t)id;
            uint32_t b = dir == 0 ? (uint32_t)(id + 1) : (uint32_t)(id + n);
            if (p_thresh != 0 && gg_rand(seed, 2 * e) < p_thresh)
                b = (uint32_t)(gg_rand(seed, 2 * e + 1) % V);
            keys[slot] = ((uint64_t)b << 32) | a;
            keys[slot + 1] = ((uint64_t)a << 32) | b;
        }
    }
    return 4 * V;
}

/* Appends the reverse of every key: keys has capacity 2n; returns 2n. */
uint64_t gg_add_reverse(uint64_t* keys, uint64_t n) {
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < (int64_t)n; ++i) {
        uint64_t k = keys[i];
        keys[n + i] = k == ~0ULL ? ~0ULL : ((k << 32) | (k >> 32));
    }
    return 2 * n;
}

/* Stable LSD radix sort of 64-bit keys on their low `bits` bits, 16-bit
 * digits, per-thread histograms.  tmp has n entries.  Result in keys. */
static void radix_sort(uint64_t* keys, uint64_t* tmp, uint64_t n, int bits) {
    enum { D = 16, R = 1 << D };
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    uint64_t* hist = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)R * nthreads);
    uint64_t* src = keys;
    uint64_t* dst = tmp;
    for (int shift = 0; shift < bits; shift += D) {
        memset(hist, 0, sizeof(uint64_t) * (size_t)R * nthreads);
#pragma omp parallel num_threads(nthreads)
        {
            int t = 0;
#ifdef _OPENMP
            t = omp_get_thread_num();
#endif
            uint64_t lo = n * (uint64_t)t / nthreads, hi = n * (uint64_t)(t + 1) / nthreads;
            uint64_t* h = hist + (size_t)R * t;
            for (uint64_t i = lo; i < hi; ++i) h[(src[i] >> shift) & (R - 1)]++;
#pragma omp barrier
#pragma omp single
            {
                uint64_t sum = 0;
                for (int d = 0; d < R; ++d)
                    for (int tt = 0; tt < nthreads; ++tt) {
                        uint64_t c = hist[(size_t)R * tt + d];
                        hist[(size_t)R * tt + d] = sum;
                        sum += c;
                    }
            }
            for (uint64_t i = lo; i < hi; ++i) dst[h[(src[i] >> shift) & (R - 1)]++] = src[i];
        }
        uint64_t* s = src;
        src = dst;
        dst = s;
    }
    if (src != keys) memcpy(keys, src, sizeof(uint64_t) * n);
    free(hist);
}

/* Sorts keys (dst << 32 | src) by (dst, src), drops placeholders (~0),
 * self-loops and duplicates in place; returns the new count.  Vertex ids
 * must be < 2^vbits. */
uint64_t gg_sort_unique(uint64_t* keys, uint64_t* tmp, uint64_t n, int vbits) {
    /* compress to (dst << vbits | src) so the sort only touches 2*vbits bits;
       placeholders map to the all-ones value of that width and sort last */
    const uint64_t vmask = (vbits >= 32) ? 0xFFFFFFFFULL : ((1ULL << vbits) - 1);
    const uint64_t ones = (2 * vbits >= 64) ? ~0ULL : ((1ULL << (2 * vbits)) - 1);
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < (int64_t)n; ++i) {
        uint64_t k = keys[i];
        keys[i] = k == ~0ULL ? ones : (((k >> 32) & vmask) << vbits) | (k & vmask);
    }
    radix_sort(keys, tmp, n, 2 * vbits);
    uint64_t out = 0;
    for (uint64_t j = 0; j < n; ++j) {
        uint64_t k = keys[j];
        if (k == ones && vbits < 32) break;
        uint64_t s = k & vmask, d = k >> vbits;
        if (s == d) continue;
        uint64_t full = (d << 32) | s;
        if (out > 0 && keys[out - 1] == full) continue;
        keys[out++] = full;
    }
    return out;
}

/* Sorted unique keys -> CSC: offsets[V+1], src[E]. */
void gg_keys_to_csc(const uint64_t* keys, uint64_t E, uint32_t V, uint32_t* offsets, uint32_t* src) {
    uint64_t e = 0;
    for (uint32_t v = 0; v < V; ++v) {
        offsets[v] = (uint32_t)e;
        while (e < E && (uint32_t)(keys[e] >> 32) == v) {
            src[e] = (uint32_t)keys[e];
            ++e;
        }
    }
    offsets[V] = (uint32_t)e;
}

/* Edge weights in CSC order. */
void gg_csc_weights(const uint32_t* offsets, const uint32_t* src, uint32_t V, uint32_t seed,
                    uint32_t wmax, int symmetric, uint32_t* w) {
    int64_t v;
#pragma omp parallel for schedule(dynamic, 4096)
    for (v = 0; v < (int64_t)V; ++v) {
        for (uint32_t e = offsets[v]; e < offsets[v + 1]; ++e) {
            uint32_t a = src[e], b = (uint32_t)v;
            if (symmetric && a > b) {
                uint32_t t = a;
                a = b;
                b = t;
            }
            w[e] = gg_weight(a, b, seed, wmax);
        }
    }
}

/* Out-degree of every vertex from the CSC source array. */
void gg_outdeg(const uint32_t* src, uint64_t E, uint32_t V, uint32_t* outdeg) {
    memset(outdeg, 0, sizeof(uint32_t) * V);
    for (uint64_t e = 0; e < E; ++e) outdeg[src[e]]++;
}

/* `count` roots drawn uniformly (with replacement) among vertices whose
 * out-degree is positive: draw j picks the (rand(seed, j) mod K)-th such
 * vertex in id order, K their number. */
void gg_roots(const uint32_t* outdeg, uint32_t V, uint64_t seed, uint32_t count, uint32_t* roots) {
    uint32_t* cand = (uint32_t*)malloc(sizeof(uint32_t) * (V ? V : 1));
    uint32_t K = 0;
    for (uint32_t v = 0; v < V; ++v)
        if (outdeg[v]) cand[K++] = v;
    for (uint32_t j = 0; j < count; ++j) roots[j] = K ? cand[gg_rand(seed, j) % K] : 0;
    free(cand);
}

int gg_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
