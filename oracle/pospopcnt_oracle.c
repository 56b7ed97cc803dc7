/*
 * pospopcnt ORACLE -- test infrastructure only.
 *
 * A plain, slow, obviously correct CPU implementation of the positional
 * population count of Klarqvist, Mula and Lemire, "Efficient Computation of
 * Positional Population Counts Using SIMD Instructions" (arXiv 1911.02696).
 * Only the test suite, the package's smoke check and the benchmark's CPU
 * baseline may load it.  It shares no code, header or table with the CUDA
 * library: it includes nothing but libc and pthreads.
 *
 * Contents
 *   oracle_pospopcnt_add / oracle_pospopcnt
 *       The definition (Abstract; §1 around Fig. 1; §4): for k-bit words
 *       w_0..w_{n-1}, counts[p] = sum_i ((w_i >> p) & 1), p = 0..k-1, taken
 *       word by word and bit by bit with a shift, a mask and an add (the
 *       scalar routine of §4, Fig. 6).  The paper's routine adds into the
 *       caller's counters; oracle_pospopcnt_add keeps that, and
 *       oracle_pospopcnt zeroes first.
 *   oracle_pospopcnt_mt
 *       The same loop run over contiguous chunks on several threads, chunk
 *       sums added (additivity of the definition).  Used to time the CPU
 *       baseline on all host cores.
 *   oracle_pospopcnt_segments
 *       One definition per segment [offsets[s], offsets[s+1]).
 *   oracle_popcount
 *       The number of set bits of a byte array, bit by bit: the single sum
 *       that pospopcnt generalises (Abstract, §2).
 *   oracle_onehot_counts
 *       Categorical ids one-hot encoded, then positionally counted: the
 *       frequency histogram that motivates the paper (§1, Table 1).
 *   oracle_csa_*
 *       The paper's own method, step by step in its order: the carry-save
 *       adder (§2, Fig. 3), the recursive Harley-Seal circuit F_N built from
 *       two F_{N-1} and one more CSA (§2, Fig. 4), run over 512-bit registers
 *       (§3, §4.1), the top register flushed into positional counters with
 *       its weight deferred (§4.1), the remaining B_l flushed with weights 2^l
 *       at the end and the residual words counted by the scalar routine
 *       (§4.1).  It reaches the definition exactly; the tests pin it there.
 *
 * Word layout: word i occupies bytes [i*k/8, (i+1)*k/8) of the input and is
 * read little-endian byte by byte, so the result does not depend on the
 * host's byte order.  Bit p of a word is (w >> p) & 1.
 *
 * Parity is pinned in tests/test_oracle_pins.py (worked example of Table 1,
 * exhaustive closed forms, numpy brute force, popcount invariant, one-hot
 * histogram, cross-width identities, CSA truth tables of Table 2 and the
 * circuit sizes of §2/§4.1).
 */
#include <pthread.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int width_ok(int k) { return k == 8 || k == 16 || k == 32 || k == 64; }

/* Little-endian load of one k-bit word from its bytes. */
static uint64_t load_word(const unsigned char* p, int k) {
  uint64_t w = 0;
  for (int b = 0; b < k / 8; ++b) w |= (uint64_t)p[b] << (8 * b);
  return w;
}

/* counts[p] += sum over the n words of ((w >> p) & 1)  (§4, Fig. 6). */
int oracle_pospopcnt_add(int k, const void* in, uint64_t n, uint64_t* counts) {
  if (!width_ok(k) || (n && !in) || !counts) return -1;
  const unsigned char* bytes = (const unsigned char*)in;
  for (uint64_t i = 0; i < n; ++i) {
    uint64_t w = load_word(bytes + i * (uint64_t)(k / 8), k);
    for (int p = 0; p < k; ++p) counts[p] += (w >> p) & 1u;
  }
  return 0;
}

int oracle_pospopcnt(int k, const void* in, uint64_t n, uint64_t* counts) {
  if (!width_ok(k) || !counts) return -1;
  memset(counts, 0, sizeof(uint64_t) * (size_t)k);
  return oracle_pospopcnt_add(k, in, n, counts);
}

/* Population count of a byte array (the single sum that pospopcnt
 * generalises, Abstract and §2): the number of set bits, bit by bit. */
int oracle_popcount(const void* in, uint64_t nbytes, uint64_t* count) {
  if ((nbytes && !in) || !count) return -1;
  const unsigned char* b = (const unsigned char*)in;
  uint64_t c = 0;
  for (uint64_t i = 0; i < nbytes; ++i)
    for (int j = 0; j < 8; ++j) c += (b[i] >> j) & 1u;
  *count = c;
  return 0;
}

/* The pipeline that motivates the paper (§1, Table 1): categorical ids are
 * one-hot encoded -- id v becomes the word with only bit v set (ids >= k map
 * to the empty word) -- and the words' positional counts are the frequency
 * histogram.  Written in that order: encode a word, then count its bits.
 * ids: n unsigned little-endian integers of id_bytes (1, 2 or 4) bytes;
 * counts: k values, 1 <= k <= 64. */
int oracle_onehot_counts(const void* ids, uint64_t n, int id_bytes, int k, uint64_t* counts) {
  if ((id_bytes != 1 && id_bytes != 2 && id_bytes != 4) || k < 1 || k > 64 || (n && !ids) || !counts)
    return -1;
  const unsigned char* b = (const unsigned char*)ids;
  memset(counts, 0, sizeof(uint64_t) * (size_t)k);
  for (uint64_t i = 0; i < n; ++i) {
    uint64_t v = 0;
    for (int j = 0; j < id_bytes; ++j) v |= (uint64_t)b[i * (uint64_t)id_bytes + (uint64_t)j] << (8 * j);
    const uint64_t word = v < (uint64_t)k ? (uint64_t)1 << v : 0; /* one-hot encoding */
    for (int p = 0; p < k; ++p) counts[p] += (word >> p) & 1u;       /* positional count */
  }
  return 0;
}

/* ---- the same definition over contiguous chunks on threads -------------- */

typedef struct {
  int k;
  const unsigned char* in;
  uint64_t n;
  uint64_t counts[64];
} chunk_t;

static void* chunk_run(void* p) {
  chunk_t* c = (chunk_t*)p;
  oracle_pospopcnt(c->k, c->in, c->n, c->counts);
  return NULL;
}

/* Returns the number of threads used (>= 1), or -1 on bad arguments. */
int oracle_pospopcnt_mt(int k, const void* in, uint64_t n, uint64_t* counts, int nthreads) {
  if (!width_ok(k) || (n && !in) || !counts) return -1;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if ((uint64_t)nthreads > n) nthreads = n ? (int)n : 1;
  chunk_t* ch = (chunk_t*)calloc((size_t)nthreads, sizeof(chunk_t));
  pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
  int* live = (int*)calloc((size_t)nthreads, sizeof(int));
  if (!ch || !th || !live) {
    free(ch), free(th), free(live);
    return -1;
  }
  uint64_t per = n / (uint64_t)nthreads, extra = n % (uint64_t)nthreads, at = 0;
  for (int t = 0; t < nthreads; ++t) {
    uint64_t len = per + ((uint64_t)t < extra ? 1 : 0);
    ch[t].k = k;
    ch[t].in = (const unsigned char*)in + at * (uint64_t)(k / 8);
    ch[t].n = len;
    at += len;
    if (t > 0 && pthread_create(&th[t], NULL, chunk_run, &ch[t]) == 0) live[t] = 1;
    else if (t > 0) chunk_run(&ch[t]);
  }
  chunk_run(&ch[0]);
  int used = 1;
  for (int t = 1; t < nthreads; ++t)
    if (live[t]) pthread_join(th[t], NULL), ++used;
  memset(counts, 0, sizeof(uint64_t) * (size_t)k);
  for (int t = 0; t < nthreads; ++t)
    for (int p = 0; p < k; ++p) counts[p] += ch[t].counts[p];
  free(ch), free(th), free(live);
  return used;
}

/* ---- one definition per segment ----------------------------------------- */

/* Segment s covers words [offsets[s], offsets[s+1]) of `in`; its counts go
 * to counts[s*k .. s*k+k-1].  Offsets must be nondecreasing and >= 0. */
int oracle_pospopcnt_segments(int k, const void* in, const int64_t* offsets, uint64_t nseg,
                              uint64_t* counts) {
  if (!width_ok(k) || (nseg && (!offsets || !counts))) return -1;
  for (uint64_t s = 0; s < nseg; ++s)
    if (offsets[s] < 0 || offsets[s + 1] < offsets[s]) return -1;
  for (uint64_t s = 0; s < nseg; ++s) {
    const unsigned char* base = (const unsigned char*)in + (uint64_t)offsets[s] * (uint64_t)(k / 8);
    int rc = oracle_pospopcnt(k, base, (uint64_t)(offsets[s + 1] - offsets[s]), counts + s * (uint64_t)k);
    if (rc) return rc;
  }
  return 0;
}

/* ---- the paper's CSA / Harley-Seal method ------------------------------- */

/* A 512-bit register (§3: one AVX-512 register), as eight 64-bit lanes.
 * Bit j of the register is bit (j mod 64) of q[j / 64]. */
typedef struct {
  uint64_t q[8];
} reg512;

static long g_csa_calls; /* CSA invocations made by the last circuit run */

/* Carry-save adder (§2, Fig. 3): h = majority(a,b,c), l = a ^ b ^ c, with the
 * a ^ b term shared, bit by bit over the whole register. */
static void csa(reg512* h, reg512* l, reg512 a, reg512 b, reg512 c) {
  for (int i = 0; i < 8; ++i) {
    uint64_t u = a.q[i] ^ b.q[i];
    h->q[i] = (a.q[i] & b.q[i]) | (u & c.q[i]);
    l->q[i] = u ^ c.q[i];
  }
  ++g_csa_calls;
}

/* The recursive circuit F_N of §2: takes 2^N input registers d[] and the
 * running sums B[0..N-1] (updated in place) and returns the new top register
 * B_N, whose bits carry weight 2^N.  F_1 is one CSA of (B_0, d0, d1);
 * F_N runs F_{N-1} on each half of the inputs and joins the two carries with
 * B_{N-1} in one more CSA, hence 2^N - 1 CSAs for 2^N inputs. */
static reg512 circuit(int N, const reg512* d, reg512* B) {
  reg512 h;
  if (N == 1) {
    csa(&h, &B[0], B[0], d[0], d[1]);
    return h;
  }
  reg512 x = circuit(N - 1, d, B);
  reg512 y = circuit(N - 1, d + (1 << (N - 1)), B);
  csa(&h, &B[N - 1], B[N - 1], x, y);
  return h;
}

static uint64_t bit_of(const reg512* r, int j) { return (r->q[j / 64] >> (j % 64)) & 1u; }

/* Flush (§4.1): for every bit j of the register, counter (j mod k) gains the
 * bit; the caller applies the register's weight. */
static void flush(const reg512* r, int k, uint64_t* acc) {
  for (int j = 0; j < 512; ++j) acc[j % k] += bit_of(r, j);
}

static reg512 load_reg(const unsigned char* p) {
  reg512 r;
  for (int i = 0; i < 8; ++i) {
    uint64_t v = 0;
    for (int b = 0; b < 8; ++b) v |= (uint64_t)p[8 * i + b] << (8 * b);
    r.q[i] = v;
  }
  return r;
}

/* pospopcnt by the method of §4.1 with a circuit of 2^N registers
 * (N = 2, 3, 4 are the paper's 256 B, 512 B and 1 kB circuits; any
 * 1 <= N <= 8 is accepted).  Blocks of 2^N * 64 bytes go through F_N; the
 * top register's count is kept unweighted and multiplied by 2^N once at the
 * end (the deferred multiplication of §4.1); B_0..B_{N-1} are flushed with
 * weights 1, 2, 4, ...; the residual words that do not fill a block are
 * counted by the scalar routine.  Returns the CSA calls made, or -1. */
long oracle_csa_pospopcnt(int k, const void* in, uint64_t n, int N, uint64_t* counts) {
  if (!width_ok(k) || N < 1 || N > 8 || (n && !in) || !counts) return -1;
  const unsigned char* bytes = (const unsigned char*)in;
  uint64_t block = (uint64_t)64 << N; /* bytes per circuit run */
  uint64_t nbytes = n * (uint64_t)(k / 8);
  uint64_t nblocks = nbytes / block;
  reg512 B[9];
  memset(B, 0, sizeof B);
  uint64_t top[64] = {0};
  uint64_t regs_per = (uint64_t)1 << N;
  reg512* d = (reg512*)malloc(sizeof(reg512) * (size_t)regs_per);
  if (!d) return -1;
  g_csa_calls = 0;
  for (uint64_t blk = 0; blk < nblocks; ++blk) {
    for (uint64_t r = 0; r < regs_per; ++r) d[r] = load_reg(bytes + blk * block + r * 64);
    reg512 hi = circuit(N, d, B);
    flush(&hi, k, top);
  }
  free(d);
  memset(counts, 0, sizeof(uint64_t) * (size_t)k);
  for (int p = 0; p < k; ++p) counts[p] = top[p] << N;
  for (int l = 0; l < N; ++l) {
    uint64_t acc[64] = {0};
    flush(&B[l], k, acc);
    for (int p = 0; p < k; ++p) counts[p] += acc[p] << l;
  }
  uint64_t done_words = nblocks * block / (uint64_t)(k / 8);
  oracle_pospopcnt_add(k, bytes + nblocks * block, n - done_words, counts);
  return g_csa_calls;
}

/* The truth table of one CSA output as the 8-bit immediate of a three-input
 * logic instruction (§3, Table 2): bit (1a + 2b + 4c) of the result is the
 * output for inputs (a, b, c).  which = 0 gives l (sum bit), 1 gives h. */
int oracle_csa_truth(int which) {
  int imm = 0;
  for (int idx = 0; idx < 8; ++idx) {
    reg512 a, b, c, h, l;
    memset(&a, 0, sizeof a), memset(&b, 0, sizeof b), memset(&c, 0, sizeof c);
    a.q[0] = (uint64_t)(idx & 1);
    b.q[0] = (uint64_t)((idx >> 1) & 1);
    c.q[0] = (uint64_t)((idx >> 2) & 1);
    csa(&h, &l, a, b, c);
    uint64_t bit = (which ? h.q[0] : l.q[0]) & 1u;
    imm |= (int)bit << idx;
  }
  return imm;
}

/* CSA calls made by one run of F_N (the circuit-size claim of §2). */
long oracle_csa_circuit_size(int N) {
  if (N < 1 || N > 12) return -1;
  uint64_t regs = (uint64_t)1 << N;
  reg512* d = (reg512*)calloc((size_t)regs, sizeof(reg512));
  reg512 B[13];
  if (!d) return -1;
  memset(B, 0, sizeof B);
  g_csa_calls = 0;
  (void)circuit(N, d, B);
  free(d);
  return g_csa_calls;
}
