/*
 * Seeded synthetic inputs for pospopcnt tests and benchmarks.
 *
 * This module holds no pospopcnt arithmetic.  It only turns (seed, index)
 * pairs into bytes, so the same input can be handed to the CPU oracle and,
 * through a host->device copy, to the GPU path.
 *
 * Random numbers come from a counter-based form of SplitMix64 (Steele, Lea
 * and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014;
 * the finaliser constants are Stafford's "Mix13"):
 *
 *     draw(seed, i) = mix(mix(seed) + (i + 1) * 0x9E3779B97F4A7C15)
 *     mix(z): z ^= z >> 30; z *= 0xBF58476D1CE4E5B9;
 *             z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31
 *
 * Every generator below is a pure function of (seed, index), so the work is
 * split over threads by index range and the output does not depend on the
 * thread count.
 */
#include <pthread.h>
#include <stdint.h>
#include <stddef.h>
#include <string.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ULL;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBULL;
  z ^= z >> 31;
  return z;
}

static inline uint64_t draw(uint64_t key, uint64_t i) { return mix64(key + (i + 1) * GOLDEN); }

static inline uint64_t key_of(uint64_t seed) { return mix64(seed); }

uint64_t synth_draw(uint64_t seed, uint64_t i) { return draw(key_of(seed), i); }

/* ---- parallel-for over an index range -------------------------------- */

typedef void (*range_fn)(void* ctx, uint64_t lo, uint64_t hi);

typedef struct {
  range_fn fn;
  void* ctx;
  uint64_t lo, hi;
} job_t;

static void* run_job(void* p) {
  job_t* j = (job_t*)p;
  if (j->hi > j->lo) j->fn(j->ctx, j->lo, j->hi);
  return NULL;
}

static void parallel_for(range_fn fn, void* ctx, uint64_t n, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 64) nthreads = 64;
  if (n < (1u << 16)) nthreads = 1;
  pthread_t th[64];
  int live[64] = {0};
  job_t jobs[64];
  uint64_t chunk = (n + (uint64_t)nthreads - 1) / (uint64_t)nthreads;
  for (int t = 0; t < nthreads; ++t) {
    uint64_t lo = chunk * (uint64_t)t;
    uint64_t hi = lo + chunk;
    if (lo > n) lo = n;
    if (hi > n) hi = n;
    jobs[t].fn = fn;
    jobs[t].ctx = ctx;
    jobs[t].lo = lo;
    jobs[t].hi = hi;
    if (t == 0) continue;
    if (pthread_create(&th[t], NULL, run_job, &jobs[t]) == 0)
      live[t] = 1;
    else
      run_job(&jobs[t]); /* no thread available: do it inline */
  }
  run_job(&jobs[0]);
  for (int t = 1; t < nthreads; ++t)
    if (live[t]) pthread_join(th[t], NULL);
}

/* ---- uniform random bits ---------------------------------------------- */

typedef struct {
  uint64_t key;
  unsigned char* out;
  uint64_t nbytes;
} uniform_ctx;

/* Byte j is byte (j mod 8) of draw j/8, little-endian. */
static void uniform_range(void* p, uint64_t lo, uint64_t hi) {
  uniform_ctx* c = (uniform_ctx*)p;
  for (uint64_t w = lo; w < hi; ++w) {
    uint64_t x = draw(c->key, w);
    uint64_t b0 = w * 8;
    if (b0 + 8 <= c->nbytes) {
      for (int b = 0; b < 8; ++b) c->out[b0 + b] = (unsigned char)(x >> (8 * b));
    } else {
      for (uint64_t b = 0; b0 + b < c->nbytes; ++b) c->out[b0 + b] = (unsigned char)(x >> (8 * b));
    }
  }
}

void synth_uniform_bits(uint64_t seed, void* out, uint64_t nbytes, int nthreads) {
  uniform_ctx c = {key_of(seed), (unsigned char*)out, nbytes};
  parallel_for(uniform_range, &c, (nbytes + 7) / 8, nthreads);
}

/* ---- little-endian store of one word ------------------------------------ */

static inline void store_le(unsigned char* p, int nbytes, uint64_t v) {
  for (int b = 0; b < nbytes; ++b) p[b] = (unsigned char)(v >> (8 * b));
}

/* ---- one-hot words with a categorical position --------------------------
 * Word i takes the 32-bit uniform u = draw(i) >> 32 and picks the smallest
 * position j with u < cdf[j], where cdf[] holds cumulative probabilities
 * scaled to 2^32 (cdf[width-1] must be 2^32).  The word is 1 << j.
 * Optionally the chosen positions are written to pos_out (one byte each). */

typedef struct {
  uint64_t key;
  int width;
  const uint64_t* cdf;
  unsigned char* out;
  unsigned char* pos_out;
} onehot_ctx;

static inline int pick(const uint64_t* cdf, int m, uint64_t u) {
  int j = 0;
  while (j < m - 1 && u >= cdf[j]) ++j;
  return j;
}

static void onehot_range(void* p, uint64_t lo, uint64_t hi) {
  onehot_ctx* c = (onehot_ctx*)p;
  int wb = c->width / 8;
  for (uint64_t i = lo; i < hi; ++i) {
    uint64_t u = draw(c->key, i) >> 32;
    int j = pick(c->cdf, c->width, u);
    store_le(c->out + i * (uint64_t)wb, wb, 1ULL << j);
    if (c->pos_out) c->pos_out[i] = (unsigned char)j;
  }
}

int synth_one_hot(uint64_t seed, int width, const uint64_t* cdf, void* out, uint64_t n,
                  unsigned char* pos_out, int nthreads) {
  if (width != 8 && width != 16 && width != 32 && width != 64) return -1;
  onehot_ctx c = {key_of(seed), width, cdf, (unsigned char*)out, pos_out};
  parallel_for(onehot_range, &c, n, nthreads);
  return 0;
}

/* ---- sparse words: every bit set independently with probability thr/2^24 --
 * Bit p of word i uses 24 bits of draw(i * (width / 2) + p / 2): bits 0..23
 * for even p, bits 24..47 for odd p. */

typedef struct {
  uint64_t key;
  int width;
  uint32_t thr;
  unsigned char* out;
} sparse_ctx;

static void sparse_range(void* p, uint64_t lo, uint64_t hi) {
  sparse_ctx* c = (sparse_ctx*)p;
  int wb = c->width / 8;
  uint64_t per = (uint64_t)(c->width / 2);
  for (uint64_t i = lo; i < hi; ++i) {
    uint64_t w = 0;
    for (uint64_t q = 0; q < per; ++q) {
      uint64_t x = draw(c->key, i * per + q);
      if ((x & 0xFFFFFFULL) < c->thr) w |= 1ULL << (2 * q);
      if (((x >> 24) & 0xFFFFFFULL) < c->thr) w |= 1ULL << (2 * q + 1);
    }
    store_le(c->out + i * (uint64_t)wb, wb, w);
  }
}

int synth_sparse(uint64_t seed, int width, uint32_t thr24, void* out, uint64_t n, int nthreads) {
  if (width != 8 && width != 16 && width != 32 && width != 64) return -1;
  sparse_ctx c = {key_of(seed), width, thr24, (unsigned char*)out};
  parallel_for(sparse_range, &c, n, nthreads);
  return 0;
}

/* ---- segmented one-hot words ---------------------------------------------
 * Segment s covers words [offsets[s], offsets[s+1]).  Its words are one-hot
 * with position (pick(cdf, u) + rot[s]) mod width, u = draw(i) >> 32 for the
 * global word index i, so each segment has its own skew. */

typedef struct {
  uint64_t key;
  int width;
  const uint64_t* cdf;
  const int64_t* offsets;
  const uint32_t* rot;
  uint64_t nseg;
  unsigned char* out;
} seg_ctx;

static void seg_range(void* p, uint64_t lo, uint64_t hi) {
  seg_ctx* c = (seg_ctx*)p;
  int wb = c->width / 8;
  for (uint64_t s = lo; s < hi; ++s) {
    uint64_t a = (uint64_t)c->offsets[s], b = (uint64_t)c->offsets[s + 1];
    for (uint64_t i = a; i < b; ++i) {
      uint64_t u = draw(c->key, i) >> 32;
      int j = (pick(c->cdf, c->width, u) + (int)c->rot[s]) % c->width;
      store_le(c->out + i * (uint64_t)wb, wb, 1ULL << j);
    }
  }
}

int synth_segmented_one_hot(uint64_t seed, int width, const uint64_t* cdf, const int64_t* offsets,
                            const uint32_t* rot, uint64_t nseg, void* out, int nthreads) {
  if (width != 8 && width != 16 && width != 32 && width != 64) return -1;
  seg_ctx c = {key_of(seed), width, cdf, offsets, rot, nseg, (unsigned char*)out};
  parallel_for(seg_range, &c, nseg, nthreads);
  return 0;
}

/* ---- categorical ids ------------------------------------------------------
 * Id i takes the 32-bit uniform u = draw(i) >> 32 and is the smallest j with
 * u < cdf[j] (cdf over m categories scaled to 2^32), stored little-endian in
 * id_bytes bytes. */

typedef struct {
  uint64_t key;
  int m, id_bytes;
  const uint64_t* cdf;
  unsigned char* out;
} ids_ctx;

static void ids_range(void* p, uint64_t lo, uint64_t hi) {
  ids_ctx* c = (ids_ctx*)p;
  for (uint64_t i = lo; i < hi; ++i) {
    uint64_t u = draw(c->key, i) >> 32;
    store_le(c->out + i * (uint64_t)c->id_bytes, c->id_bytes, (uint64_t)pick(c->cdf, c->m, u));
  }
}

int synth_categorical_ids(uint64_t seed, int m, const uint64_t* cdf, int id_bytes, void* out, uint64_t n,
                          int nthreads) {
  if (m < 1 || (id_bytes != 1 && id_bytes != 2 && id_bytes != 4)) return -1;
  ids_ctx c = {key_of(seed), m, id_bytes, cdf, (unsigned char*)out};
  parallel_for(ids_range, &c, n, nthreads);
  return 0;
}
