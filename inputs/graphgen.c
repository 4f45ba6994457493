/*
 * Seeded synthetic graph inputs: R-MAT and Erdos-Renyi edge streams, CSR/CSC
 * assembly with duplicate removal, and the symmetric per-edge weight draw.
 *
 * This file holds input tooling only. It computes nothing of the
 * vertex-centric method itself; both the CPU oracle and the GPU library
 * consume the CSR/CSC arrays it produces.
 *
 * Random numbers: every draw is counter based. The mixing function is the
 * SplitMix64 output function (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014). Edge i of a stream uses the
 * SplitMix64 sequence started at state_i = mix(mix(seed) + i * GOLDEN), so
 * the edge list does not depend on the thread count.
 *
 * R-MAT (Chakrabarti, Zhan and Faloutsos, SDM 2004): for each of `scale`
 * levels, from the most significant bit down, one uniform draw picks a
 * quadrant: [0,a) -> (src bit 0, dst bit 0), [a,a+b) -> (0,1),
 * [a+b,a+b+c) -> (1,0), otherwise (1,1). No noise and no vertex permutation
 * (the permuted variant relabels the vertices afterwards, see gg_random_keys).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GOLDEN 0x9e3779b97f4a7c15ULL

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static inline double u01(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

int gg_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

uint64_t gg_mix64(uint64_t z) { return mix64(z); }

/* key[i] = a counter-based 64-bit draw for item i (stream `seed`): sorting the
 * items by key gives a seeded uniform random permutation. */
void gg_random_keys(int64_t n, uint64_t seed, uint64_t* key) {
    const uint64_t base = mix64(seed ^ 0x5065726d75746521ULL);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) key[i] = mix64(base + (uint64_t)i * GOLDEN);
}

/* R-MAT edge stream: edges [0, m) written to src/dst. */
void gg_rmat_edges(int scale, int64_t m, double a, double b, double c, uint64_t seed,
                   uint32_t* src, uint32_t* dst) {
    const uint64_t base = mix64(seed);
    const double ab = a + b, abc = a + b + c;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        uint64_t st = mix64(base + (uint64_t)i * GOLDEN);
        uint32_t u = 0, v = 0;
        for (int l = 0; l < scale; ++l) {
            st += GOLDEN;
            double r = u01(mix64(st));
            uint32_t bit = 1u << (scale - 1 - l);
            if (r < a) {
            } else if (r < ab) {
                v |= bit;
            } else if (r < abc) {
                u |= bit;
            } else {
                u |= bit;
                v |= bit;
            }
        }
        src[i] = u;
        dst[i] = v;
    }
}

/* Erdos-Renyi G(n, m) edge stream: m uniform ordered pairs (duplicates are
 * removed later by the CSR assembly). */
void gg_er_edges(uint32_t n, int64_t m, uint64_t seed, uint32_t* src, uint32_t* dst) {
    const uint64_t base = mix64(seed ^ 0x5851f42d4c957f2dULL);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        uint64_t st = mix64(base + (uint64_t)i * GOLDEN);
        uint64_t x = mix64(st + GOLDEN), y = mix64(st + 2 * GOLDEN);
        src[i] = (uint32_t)(((x >> 32) * (uint64_t)n) >> 32);
        dst[i] = (uint32_t)(((y >> 32) * (uint64_t)n) >> 32);
    }
}

/* Pack (src, dst) into 64-bit keys src<<32|dst; with symmetrize, also the
 * reversed pair. keys must hold m (or 2m) entries. Returns the key count. */
int64_t gg_pack_keys(int64_t m, const uint32_t* src, const uint32_t* dst, int symmetrize,
                     uint64_t* keys) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        keys[i] = ((uint64_t)src[i] << 32) | dst[i];
        if (symmetrize) keys[m + i] = ((uint64_t)dst[i] << 32) | src[i];
    }
    return symmetrize ? 2 * m : m;
}

/* Stable LSD radix sort of 64-bit keys, 16-bit digits; tmp has n entries.
 * Digit passes in which every key has the same digit are skipped. The sorted
 * result is left in keys. */
void gg_radix_sort64(uint64_t* keys, uint64_t* tmp, int64_t n) {
    if (n <= 1) return;
    int nt = 1;
#ifdef _OPENMP
    nt = omp_get_max_threads();
#endif
    const int R = 1 << 16;
    int64_t* hist = (int64_t*)malloc(sizeof(int64_t) * (size_t)nt * R);
    uint64_t* in = keys;
    uint64_t* out = tmp;
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = pass * 16;
        memset(hist, 0, sizeof(int64_t) * (size_t)nt * R);
#pragma omp parallel num_threads(nt)
        {
            int t = 0;
#ifdef _OPENMP
            t = omp_get_thread_num();
#endif
            int64_t lo = n * t / nt, hi = n * (t + 1) / nt;
            int64_t* h = hist + (size_t)t * R;
            for (int64_t i = lo; i < hi; ++i) h[(in[i] >> shift) & 0xFFFF]++;
        }
        /* skip the pass when one digit value holds every key */
        int64_t maxc = 0;
        for (int d = 0; d < R; ++d) {
            int64_t s = 0;
            for (int t = 0; t < nt; ++t) s += hist[(size_t)t * R + d];
            if (s > maxc) maxc = s;
        }
        if (maxc == n) continue;
        int64_t run = 0;
        for (int d = 0; d < R; ++d)
            for (int t = 0; t < nt; ++t) {
                int64_t c = hist[(size_t)t * R + d];
                hist[(size_t)t * R + d] = run;
                run += c;
            }
#pragma omp parallel num_threads(nt)
        {
            int t = 0;
#ifdef _OPENMP
            t = omp_get_thread_num();
#endif
            int64_t lo = n * t / nt, hi = n * (t + 1) / nt;
            int64_t* h = hist + (size_t)t * R;
            for (int64_t i = lo; i < hi; ++i) out[h[(in[i] >> shift) & 0xFFFF]++] = in[i];
        }
        uint64_t* sw = in;
        in = out;
        out = sw;
    }
    if (in != keys) memcpy(keys, in, sizeof(uint64_t) * (size_t)n);
    free(hist);
}

/* Remove adjacent duplicates from sorted keys in place; returns the new count. */
int64_t gg_unique_sorted(uint64_t* keys, int64_t n) {
    if (n == 0) return 0;
    int64_t w = 1;
    for (int64_t i = 1; i < n; ++i)
        if (keys[i] != keys[w - 1]) keys[w++] = keys[i];
    return w;
}

/* CSR from sorted unique keys: row_ptr has n+1 entries, col has e. */
void gg_keys_to_csr(uint32_t n, const uint64_t* keys, int64_t e, uint32_t* row_ptr, uint32_t* col) {
    memset(row_ptr, 0, sizeof(uint32_t) * ((size_t)n + 1));
    for (int64_t i = 0; i < e; ++i) row_ptr[(keys[i] >> 32) + 1]++;
    for (uint32_t v = 0; v < n; ++v) row_ptr[v + 1] += row_ptr[v];
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < e; ++i) col[i] = (uint32_t)keys[i];
}

/* Stable transposition (counting sort by destination). Within each in-list
 * the sources come out in increasing order because the CSR rows are scanned
 * in increasing source order. w / wt may be NULL. cursor has n entries. */
void gg_transpose(uint32_t n, const uint32_t* row_ptr, const uint32_t* col, const uint32_t* w,
                  uint32_t* t_ptr, uint32_t* t_idx, uint32_t* t_w, uint32_t* cursor) {
    const int64_t e = row_ptr[n];
    memset(t_ptr, 0, sizeof(uint32_t) * ((size_t)n + 1));
    for (int64_t i = 0; i < e; ++i) t_ptr[col[i] + 1]++;
    for (uint32_t v = 0; v < n; ++v) t_ptr[v + 1] += t_ptr[v];
    memcpy(cursor, t_ptr, sizeof(uint32_t) * (size_t)n);
    for (uint32_t u = 0; u < n; ++u)
        for (uint32_t k = row_ptr[u]; k < row_ptr[u + 1]; ++k) {
            uint32_t pos = cursor[col[k]]++;
            t_idx[pos] = u;
            if (w && t_w) t_w[pos] = w[k];
        }
}

/* Symmetric weight draw in [1, 255]: one value per unordered pair {u, v},
 * so w(u,v) == w(v,u). */
static inline uint32_t sym_weight(uint64_t wbase, uint32_t u, uint32_t v) {
    uint32_t lo = u < v ? u : v, hi = u < v ? v : u;
    return 1u + (uint32_t)(mix64(wbase ^ (((uint64_t)lo << 32) | hi)) % 255u);
}

void gg_sym_weights(uint32_t n, const uint32_t* row_ptr, const uint32_t* col, uint64_t seed,
                    uint32_t* w) {
    const uint64_t wbase = mix64(seed * GOLDEN + 0x2545f4914f6cdd1dULL);
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t u = 0; u < (int64_t)n; ++u)
        for (uint32_t k = row_ptr[u]; k < row_ptr[u + 1]; ++k) w[k] = sym_weight(wbase, (uint32_t)u, col[k]);
}

/* Uniform vertex draws (e.g. batched SSSP sources). */
void gg_uniform_vertices(uint32_t n, int64_t k, uint64_t seed, uint32_t* out) {
    const uint64_t base = mix64(seed ^ 0x6a09e667f3bcc909ULL);
    for (int64_t i = 0; i < k; ++i) {
        uint64_t x = mix64(base + (uint64_t)(i + 1) * GOLDEN);
        out[i] = (uint32_t)(((x >> 32) * (uint64_t)n) >> 32);
    }
}

/* Log-uniform integer draws in [lo, hi] (batched instance sizes). */
void gg_loguniform(int64_t k, double lo, double hi, uint64_t seed, uint32_t* out);
#include <math.h>
void gg_loguniform(int64_t k, double lo, double hi, uint64_t seed, uint32_t* out) {
    const uint64_t base = mix64(seed ^ 0xbb67ae8584caa73bULL);
    const double llo = log(lo), lhi = log(hi);
    for (int64_t i = 0; i < k; ++i) {
        double r = u01(mix64(base + (uint64_t)(i + 1) * GOLDEN));
        double x = exp(llo + r * (lhi - llo));
        uint32_t v = (uint32_t)(x + 0.5);
        if (v < (uint32_t)lo) v = (uint32_t)lo;
        if (v > (uint32_t)hi) v = (uint32_t)hi;
        out[i] = v;
    }
}
