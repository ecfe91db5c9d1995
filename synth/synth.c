/*
 * Seeded synthetic text generators shared by the tests and the benchmark.
 *
 * This file holds no wavelet tree / matrix arithmetic: it only draws symbols.
 * Both the oracle and the CUDA library consume the bytes it writes.
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014).  Output i (0-based) of the
 * stream seeded with s is mix(s + (i + 1) * 0x9E3779B97F4A7C15), mix being the
 * published 64-bit finaliser.  A uniform double in [0, 1) is (x >> 11) * 2^-53.
 * Because each output depends only on (seed, i), streams split across threads
 * give the same bytes as one thread.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN 0x9E3779B97F4A7C15ull

static uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t synth_splitmix64(uint64_t seed, uint64_t i) { return mix64(seed + (i + 1) * GOLDEN); }

static double unit_double(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

static uint64_t below(uint64_t x, uint64_t k) { return (uint64_t)(unit_double(x) * (double)k); }

static void put(void *out, int w, uint64_t i, uint32_t v)
{
    if (w == 1) ((uint8_t *)out)[i] = (uint8_t)v;
    else if (w == 2) ((uint16_t *)out)[i] = (uint16_t)v;
    else ((uint32_t *)out)[i] = v;
}

/* Seeded Fisher-Yates shuffle of [0, k). */
int synth_permutation(uint64_t seed, uint32_t k, uint32_t *perm)
{
    for (uint32_t i = 0; i < k; ++i) perm[i] = i;
    uint64_t c = 0;
    for (uint32_t i = k; i-- > 1;) {
        uint32_t j = (uint32_t)below(synth_splitmix64(seed, c++), (uint64_t)i + 1);
        uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    return 0;
}

/* ---- parallel fill ------------------------------------------------------ */

typedef struct {
    int kind;                  /* 0 uniform, 1 zipf */
    uint64_t seed, off, begin, end;
    uint32_t k;
    const double *cdf;         /* zipf: cdf[r] = P(rank <= r+1) */
    const uint32_t *perm;
    void *out; int w;
} job_t;

static uint32_t zipf_rank(const double *cdf, uint32_t k, double u)
{
    uint32_t lo = 0, hi = k - 1;            /* smallest r with cdf[r] > u */
    while (lo < hi) {
        uint32_t mid = lo + (hi - lo) / 2;
        if (cdf[mid] > u) hi = mid; else lo = mid + 1;
    }
    return lo;
}

static void *fill_worker(void *arg)
{
    job_t *j = (job_t *)arg;
    for (uint64_t i = j->begin; i < j->end; ++i) {
        uint64_t x = synth_splitmix64(j->seed, j->off + i);
        uint32_t v;
        if (j->kind == 0) v = (uint32_t)below(x, j->k);
        else v = j->perm[zipf_rank(j->cdf, j->k, unit_double(x))];
        put(j->out, j->w, i, v);
    }
    return NULL;
}

static int run_parallel(job_t base, uint64_t n, int threads)
{
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    if ((uint64_t)threads > n / 65536 + 1) threads = (int)(n / 65536 + 1);
    pthread_t tid[256];
    job_t jobs[256];
    for (int t = 0; t < threads; ++t) {
        jobs[t] = base;
        jobs[t].begin = n * (uint64_t)t / (uint64_t)threads;
        jobs[t].end = n * (uint64_t)(t + 1) / (uint64_t)threads;
    }
    for (int t = 1; t < threads; ++t)
        if (pthread_create(&tid[t], NULL, fill_worker, &jobs[t]) != 0) return -3;
    fill_worker(&jobs[0]);
    for (int t = 1; t < threads; ++t) pthread_join(tid[t], NULL);
    return 0;
}

/* out[i] = floor(u_{off+i} * k), i in [0, n). */
int synth_uniform(uint64_t seed, uint64_t off, uint64_t n, uint32_t k, void *out, int w,
                  int threads)
{
    if (k == 0 || (w != 1 && w != 2 && w != 4)) return -1;
    job_t b = {0, seed, off, 0, 0, k, NULL, NULL, out, w};
    return run_parallel(b, n, threads);
}

/* Zipf(s) over k ranks (P(r) proportional to r^-s, r = 1..k), inverse CDF by
 * binary search, rank r mapped to symbol perm[r-1] of a seeded permutation. */
int synth_zipf(uint64_t seed, uint64_t perm_seed, uint64_t n, uint32_t k, double s,
               void *out, int w, int threads)
{
    if (k == 0 || (w != 1 && w != 2 && w != 4)) return -1;
    double *cdf = malloc((size_t)k * sizeof(double));
    uint32_t *perm = malloc((size_t)k * sizeof(uint32_t));
    if (!cdf || !perm) { free(cdf); free(perm); return -3; }
    double acc = 0.0;
    for (uint32_t r = 0; r < k; ++r) {
        acc += (s == 1.0) ? 1.0 / (double)(r + 1) : pow((double)(r + 1), -s);
        cdf[r] = acc;
    }
    for (uint32_t r = 0; r < k; ++r) cdf[r] /= acc;
    cdf[k - 1] = 2.0;                       /* every u < 1 lands inside */
    synth_permutation(perm_seed, k, perm);
    job_t b = {1, seed, 0, 0, 0, k, cdf, perm, out, w};
    int rc = run_parallel(b, n, threads);
    free(cdf); free(perm);
    return rc;
}

/* Order-1 Markov chain over [0, k), k a power of two.  State x has 64
 * successors succ(x, j) = mix(seed_succ ^ (x * 64 + j)) mod k; the next state
 * is succ(cur, j) with j drawn uniformly from [0, 64) by stream seed_step. */
int synth_markov(uint64_t seed_step, uint64_t seed_succ, uint64_t n, uint32_t k,
                 uint32_t start, void *out, int w)
{
    if (k == 0 || (k & (k - 1)) || (w != 1 && w != 2 && w != 4)) return -1;
    uint32_t cur = start & (k - 1);
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t j = synth_splitmix64(seed_step, i) >> 58;   /* top 6 bits */
        cur = (uint32_t)(mix64(seed_succ ^ ((uint64_t)cur * 64u + j)) & (uint64_t)(k - 1));
        put(out, w, i, cur);
    }
    return 0;
}
