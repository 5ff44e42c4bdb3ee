/*
 * Seeded synthetic graph workloads shared by the tests, the oracle checks and
 * the benchmark.  Nothing here computes any part of BOBA; it only produces
 * inputs: R-MAT, 2D grid and Erdos-Renyi COO edge lists with randomly relabelled
 * vertices and shuffled edge order, and uniform fp32 vectors.
 *
 * Randomness is counter based, so any output index can be produced on its own
 * and the result does not depend on the number of threads:
 *   - SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
 *     generators", OOPSLA 2014): the i-th output of a stream with key k is
 *     mix64(k + (i + 1) * 0x9E3779B97F4A7C15);
 *   - permutations of [0, N) are 4-round balanced Feistel networks on the next
 *     even number of bits, with cycle walking back into [0, N) (Black and
 *     Rogaway, "Ciphers with arbitrary finite domains", CT-RSA 2002).
 * R-MAT (Chakrabarti, Zhan, Faloutsos, SDM 2004) picks one quadrant per level
 * from a 32-bit draw compared with integer thresholds floor(a*2^32),
 * floor((a+b)*2^32), floor((a+b+c)*2^32); quadrant a = (src bit 0, dst bit 0),
 * b = (0, 1), c = (1, 0), d = (1, 1), most significant bit first.
 *
 * Plain C with POSIX threads; no architecture-specific code.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define GOLDEN 0x9E3779B97F4A7C15ull

static inline uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static inline uint64_t sm_at(uint64_t key, uint64_t i) { return mix64(key + (i + 1) * GOLDEN); }

uint64_t synth_stream_key(uint64_t seed, uint64_t stream)
{
    return mix64(seed * GOLDEN + 0xD1B54A32D192ED03ull * (stream + 1));
}

uint64_t synth_splitmix_at(uint64_t key, uint64_t i) { return sm_at(key, i); }

/* ---------------- Feistel permutation of [0, N) ---------------- */
typedef struct {
    uint64_t N;
    int half;        /* bits per Feistel half */
    uint64_t mask;
    uint64_t k[4];
} feistel_t;

static void feistel_init(feistel_t *f, uint64_t key, uint64_t N)
{
    int bits = 2;
    while (bits < 64 && (1ull << bits) < N) bits++;
    if (bits & 1) bits++;
    f->N = N;
    f->half = bits / 2;
    f->mask = (1ull << f->half) - 1;
    for (int r = 0; r < 4; ++r) f->k[r] = sm_at(key, (uint64_t)r);
}

static inline uint64_t feistel_once(const feistel_t *f, uint64_t x)
{
    uint64_t L = x >> f->half, R = x & f->mask;
    for (int r = 0; r < 4; ++r) {
        uint64_t t = L ^ (mix64(R ^ f->k[r]) & f->mask);
        L = R;
        R = t;
    }
    return (L << f->half) | R;
}

static inline uint64_t feistel_apply(const feistel_t *f, uint64_t x)
{
    uint64_t y = feistel_once(f, x);
    while (y >= f->N) y = feistel_once(f, y);
    return y;
}

/* ---------------- generators ---------------- */
enum { KIND_RMAT = 0, KIND_GRID = 1, KIND_ER = 2 };

typedef struct {
    int kind;
    uint64_t ekey;           /* edge stream */
    int scale;               /* R-MAT levels */
    uint32_t ta, tab, tabc;  /* R-MAT thresholds */
    int64_t n, m, side;
    int shuffle, relabel;
    feistel_t shuf, lab;
    int32_t *src, *dst;      /* out[i - base] for output index i */
    int64_t base;
    int64_t lo, hi;
} job_t;

static void rmat_edge(const job_t *J, uint64_t j, int64_t *pu, int64_t *pv)
{
    const int words = (J->scale + 1) / 2;
    for (uint64_t attempt = 0; attempt < 256; ++attempt) {
        uint64_t base = ((j << 8) | attempt) * (uint64_t)words;
        int64_t u = 0, v = 0;
        uint64_t w = 0;
        for (int l = 0; l < J->scale; ++l) {
            if ((l & 1) == 0) w = sm_at(J->ekey, base + (uint64_t)(l >> 1));
            uint32_t r = (l & 1) ? (uint32_t)(w >> 32) : (uint32_t)w;
            int sb = 0, db = 0;
            if (r < J->ta) { sb = 0; db = 0; }
            else if (r < J->tab) { sb = 0; db = 1; }
            else if (r < J->tabc) { sb = 1; db = 0; }
            else { sb = 1; db = 1; }
            u = (u << 1) | sb;
            v = (v << 1) | db;
        }
        if (u < J->n && v < J->n) { *pu = u; *pv = v; return; }
    }
    /* practically unreachable for n > 2^(scale-1); keep the result defined */
    *pu = (int64_t)(sm_at(J->ekey, j) % (uint64_t)J->n);
    *pv = (int64_t)(sm_at(J->ekey ^ 1, j) % (uint64_t)J->n);
}

static void grid_edge(const job_t *J, uint64_t j, int64_t *pu, int64_t *pv)
{
    const int64_t s = J->side, per = s * (s - 1);
    int64_t d = (int64_t)j / per, t = (int64_t)j % per;
    int64_t a, b;
    if (d < 2) {                /* horizontal pair (r, c) - (r, c+1) */
        int64_t r = t / (s - 1), c = t % (s - 1);
        a = r * s + c; b = r * s + c + 1;
    } else {                    /* vertical pair (r, c) - (r+1, c) */
        int64_t c = t / (s - 1), r = t % (s - 1);
        a = r * s + c; b = (r + 1) * s + c;
    }
    if (d & 1) { int64_t x = a; a = b; b = x; }
    *pu = a; *pv = b;
}

static void er_edge(const job_t *J, uint64_t j, int64_t *pu, int64_t *pv)
{
    uint64_t w = sm_at(J->ekey, j);
    *pu = (int64_t)(((w & 0xFFFFFFFFull) * (uint64_t)J->n) >> 32);
    *pv = (int64_t)(((w >> 32) * (uint64_t)J->n) >> 32);
}

static void *run_job(void *arg)
{
    const job_t *J = (const job_t *)arg;
    for (int64_t i = J->lo; i < J->hi; ++i) {
        uint64_t j = J->shuffle ? feistel_apply(&J->shuf, (uint64_t)i) : (uint64_t)i;
        int64_t u, v;
        if (J->kind == KIND_RMAT) rmat_edge(J, j, &u, &v);
        else if (J->kind == KIND_GRID) grid_edge(J, j, &u, &v);
        else er_edge(J, j, &u, &v);
        if (J->relabel) {
            u = (int64_t)feistel_apply(&J->lab, (uint64_t)u);
            v = (int64_t)feistel_apply(&J->lab, (uint64_t)v);
        }
        J->src[i - J->base] = (int32_t)u;
        J->dst[i - J->base] = (int32_t)v;
    }
    return NULL;
}

static int run_parallel(job_t *proto, int64_t lo, int64_t hi, int nthreads)
{
    if (lo < 0 || hi > proto->m || lo > hi) return 1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (hi - lo < 65536) nthreads = 1;
    job_t jobs[256];
    pthread_t th[256];
    int64_t chunk = (hi - lo + nthreads - 1) / nthreads;
    int started = 0;
    proto->base = lo;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = *proto;
        jobs[t].lo = lo + (int64_t)t * chunk;
        jobs[t].hi = jobs[t].lo + chunk < hi ? jobs[t].lo + chunk : hi;
        if (jobs[t].lo >= jobs[t].hi) continue;
        if (nthreads == 1) { run_job(&jobs[t]); continue; }
        if (pthread_create(&th[started], NULL, run_job, &jobs[t]) != 0) {
            run_job(&jobs[t]);
        } else {
            started++;
        }
    }
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    return 0;
}

static void common_init(job_t *J, uint64_t seed, int64_t n, int64_t m, int shuffle,
                        int relabel, int32_t *src, int32_t *dst)
{
    memset(J, 0, sizeof(*J));
    J->ekey = synth_stream_key(seed, 1);
    J->n = n;
    J->m = m;
    J->shuffle = shuffle;
    J->relabel = relabel;
    J->src = src;
    J->dst = dst;
    feistel_init(&J->lab, synth_stream_key(seed, 2), (uint64_t)(n > 0 ? n : 1));
    feistel_init(&J->shuf, synth_stream_key(seed, 3), (uint64_t)(m > 0 ? m : 1));
}

/* R-MAT on 2^scale IDs; IDs >= n are redrawn (n <= 2^scale).  Returns 0 / 1 bad arg. */
/* Output edges [lo, hi) of the m-edge list go to src[0 .. hi-lo), dst[...]. */
int synth_rmat(uint64_t seed, int scale, int64_t n, int64_t m, double a, double b, double c,
               int shuffle, int relabel, int64_t lo, int64_t hi, int32_t *src, int32_t *dst,
               int nthreads)
{
    if (scale < 1 || scale > 31 || n < 1 || n > (1ll << scale) || m < 0) return 1;
    if (a < 0 || b < 0 || c < 0 || a + b + c > 1.0) return 1;
    job_t J;
    common_init(&J, seed, n, m, shuffle, relabel, src, dst);
    J.kind = KIND_RMAT;
    J.scale = scale;
    double s1 = a, s2 = a + b, s3 = a + b + c;
    J.ta = s1 >= 1.0 ? 0xFFFFFFFFu : (uint32_t)floor(s1 * 4294967296.0);
    J.tab = s2 >= 1.0 ? 0xFFFFFFFFu : (uint32_t)floor(s2 * 4294967296.0);
    J.tabc = s3 >= 1.0 ? 0xFFFFFFFFu : (uint32_t)floor(s3 * 4294967296.0);
    return run_parallel(&J, lo, hi, nthreads);
}

/* 4-neighbour side x side grid, both directions: m = 4 * side * (side - 1). */
int synth_grid(uint64_t seed, int64_t side, int shuffle, int relabel, int64_t lo, int64_t hi,
               int32_t *src, int32_t *dst, int nthreads)
{
    if (side < 2 || side * side > 2147483647ll) return 1;
    job_t J;
    common_init(&J, seed, side * side, 4 * side * (side - 1), shuffle, relabel, src, dst);
    J.kind = KIND_GRID;
    J.side = side;
    return run_parallel(&J, lo, hi, nthreads);
}

/* Erdos-Renyi style: m edges with independent uniform endpoints. */
int synth_er(uint64_t seed, int64_t n, int64_t m, int shuffle, int relabel, int64_t lo,
             int64_t hi, int32_t *src, int32_t *dst, int nthreads)
{
    if (n < 1 || n > 2147483647ll || m < 0) return 1;
    job_t J;
    common_init(&J, seed, n, m, shuffle, relabel, src, dst);
    J.kind = KIND_ER;
    return run_parallel(&J, lo, hi, nthreads);
}

/* out[i] = the Feistel permutation of [0, N) under key(seed, stream) at i. */
int synth_permutation(uint64_t seed, uint64_t stream, int64_t N, int64_t *out)
{
    if (N < 1) return 1;
    feistel_t f;
    feistel_init(&f, synth_stream_key(seed, stream), (uint64_t)N);
    for (int64_t i = 0; i < N; ++i) out[i] = (int64_t)feistel_apply(&f, (uint64_t)i);
    return 0;
}

/* out[i] = uniform fp32 in [0, 1) with 24 random bits: (draw >> 40) * 2^-24. */
int synth_uniform_f32(uint64_t seed, uint64_t stream, int64_t n, float *out)
{
    uint64_t key = synth_stream_key(seed, stream);
    for (int64_t i = 0; i < n; ++i)
        out[i] = (float)(sm_at(key, (uint64_t)i) >> 40) * (1.0f / 16777216.0f);
    return 0;
}

/* out[i] = raw 64-bit draws (used to derive per-graph sizes of a batch). */
int synth_draws(uint64_t seed, uint64_t stream, int64_t n, uint64_t *out)
{
    uint64_t key = synth_stream_key(seed, stream);
    for (int64_t i = 0; i < n; ++i) out[i] = sm_at(key, (uint64_t)i);
    return 0;
}
