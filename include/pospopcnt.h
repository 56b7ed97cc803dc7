/*
 * pospopcnt for GB300 (sm_103a) -- public C ABI.
 *
 * The positional population count of Klarqvist, Mula and Lemire, "Efficient
 * Computation of Positional Population Counts Using SIMD Instructions"
 * (arXiv 1911.02696): given a stream of k-bit words w_0..w_{n-1}, return the
 * k sums counts[p] = sum_i ((w_i >> p) & 1), p = 0..k-1 (Abstract; §1; the
 * scalar shift-mask-add routine of §4, Fig. 6).  For one-hot words the
 * counts are the frequency histogram (§1, Table 1).
 *
 * Conventions shared by every entry point
 *   - Words are little-endian; bit p of a word is (w >> p) & 1, so
 *     counts[0] belongs to the least significant bit.
 *   - n counts WORDS, not bytes.  Offsets are in words relative to d_in.
 *   - d_in must be aligned to the word size (1, 2, 4 or 8 bytes); any such
 *     start is valid: words before the first 16-byte boundary and after the
 *     last whole 16-byte vector are counted one by one (§4.1 counts the
 *     residual that does not fill a SIMD block with the scalar routine).
 *   - Results overwrite d_counts (the paper's routine adds into its
 *     counters; the *_accumulate entry point keeps that form).  Counts are
 *     exact uint64 values; every result is bit-exact.
 *   - Entry points taking a cudaStream_t are asynchronous on that stream:
 *     they enqueue at most a memset of the outputs and one counting kernel,
 *     copy nothing between host and device and never synchronise.  A plain
 *     count overwrites its outputs without a memset: a count that fits one
 *     CTA stores them, a larger one adds into an accumulator bound to the
 *     stream and its last block writes them (while the stream is being
 *     captured into a CUDA graph, and on cudaStreamPerThread, the outputs
 *     are zeroed by a memset first, so a graph may be replayed on any
 *     stream).  The batched and one-hot forms zero their outputs with a
 *     memset; the checked batched form adds a small offsets check.  The
 *     caller owns every buffer; the library never frees, retains or writes
 *     d_in.
 *   - The first call on a device allocates the library's per-device
 *     workspace (error word, work-queue slots, per-stream accumulators);
 *     pospopcnt_init() does that up front, after which the asynchronous
 *     calls allocate nothing.
 *   - Errors are returned as pospopcnt_status values before anything is
 *     enqueued; a failing CUDA call yields POSPOPCNT_ERR_CUDA and its
 *     cudaError_t is kept for pospopcnt_last_cuda_error().
 */
#ifndef POSPOPCNT_GB300_H
#define POSPOPCNT_GB300_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  POSPOPCNT_OK = 0,
  POSPOPCNT_ERR_INVALID = 1,         /* null pointer with n > 0, bad width, bad config */
  POSPOPCNT_ERR_MISALIGNED = 2,      /* d_in not aligned to the word size */
  POSPOPCNT_ERR_CUDA = 3,            /* a CUDA runtime call failed */
  POSPOPCNT_ERR_NOT_INITIALIZED = 4, /* no CUDA device / library state */
  POSPOPCNT_ERR_TIMEOUT = 5,         /* a bounded device-side wait gave up */
  POSPOPCNT_ERR_TOO_LARGE = 6        /* a size beyond a documented limit */
} pospopcnt_status;

/* Kernel families for the single-stream count (pospopcnt_count). */
typedef enum {
  POSPOPCNT_KERNEL_AUTO = 0,   /* the tuned choice for this width and size */
  POSPOPCNT_KERNEL_CSA = 1,    /* 128-bit loads + per-thread carry-save circuit + popc flush */
  POSPOPCNT_KERNEL_TMA = 2,    /* bulk async copies into an mbarrier ring, same circuit */
  POSPOPCNT_KERNEL_BALLOT = 3  /* __ballot_sync bit transpose + popc (comparison kernel) */
} pospopcnt_kernel;

/* Launch configuration of the single-stream count. Zero fields take the
 * library default.  threads: CTA size for CSA/BALLOT (128, 256 or 512);
 * unroll: 16-byte vectors per thread per loop trip for CSA (2, 4 or 8; the
 * carry-save circuit then spans 4*unroll 32-bit registers) and BALLOT
 * (1, 2 or 4); blocks_per_sm: resident CTAs per SM the grid is sized for;
 * stages / chunk_bytes: ring depth and bytes per stage for TMA
 * (chunk_bytes a multiple of 16384, stages*chunk_bytes <= 196608). */
typedef struct {
  int kernel;
  int threads;
  int unroll;
  int blocks_per_sm;
  int stages;
  int chunk_bytes;
  int flags;  /* POSPOPCNT_FLAG_* bits (0: none) */
} pospopcnt_config;

/* TMA family: the bulk copies carry an L2 evict-first policy (every input
 * byte is read exactly once, so its lines need not stay in L2). */
#define POSPOPCNT_FLAG_EVICT_FIRST 1

/* Creates the per-device state of `device` (error word, queue slots,
 * per-stream accumulators of the plain count, SM count).  Idempotent.  Makes `device` current only for the duration of
 * the call. */
int pospopcnt_init(int device);

/* pospopcnt over n 8-, 16- or 32-bit words at d_in (device memory); writes
 * 8, 16 or 32 uint64 counts to d_counts (device memory, 8-byte aligned).
 * The definition is that of the Abstract and §4 (Fig. 6); the method is
 * the carry-save (Harley-Seal) circuit of §2-§4.1 run per GPU thread over
 * 32-bit registers, flushed with popc.  n == 0 writes zero counts. */
int pospopcnt_u8(const void* d_in, size_t n, uint64_t* d_counts, cudaStream_t stream);
int pospopcnt_u16(const void* d_in, size_t n, uint64_t* d_counts, cudaStream_t stream);
int pospopcnt_u32(const void* d_in, size_t n, uint64_t* d_counts, cudaStream_t stream);

/* The same for 64-bit words (64 counts; d_in 8-byte aligned).  Wider words
 * are narrower streams side by side (§4): in each 16-byte vector the 32-bit
 * registers alternate between positions 0..31 and 32..63, and each thread
 * runs one carry-save circuit per class.  pospopcnt_count / _config /
 * _accumulate / _count_host also take width 64 (CSA and TMA families);
 * the batched and serving forms take 8, 16 or 32. */
int pospopcnt_u64(const void* d_in, size_t n, uint64_t* d_counts, cudaStream_t stream);

/* pospopcnt_u8/u16/u32/u64 for width 8, 16, 32 or 64 with an explicit
 * kernel family (pospopcnt_kernel; width 64: CSA or TMA). */
int pospopcnt_count(int width, int kernel, const void* d_in, size_t n, uint64_t* d_counts,
                    cudaStream_t stream);

/* The same with an explicit launch configuration (validated; see
 * pospopcnt_config). */
int pospopcnt_count_config(int width, const pospopcnt_config* cfg, const void* d_in, size_t n,
                           uint64_t* d_counts, cudaStream_t stream);

/* Accumulate form, the paper's convention (§4, Fig. 6 adds into its
 * counters): d_counts[p] += counts[p].  Nothing is zeroed, so a stream can
 * be counted in chunks over several calls. */
int pospopcnt_count_accumulate(int width, const void* d_in, size_t n, uint64_t* d_counts,
                               cudaStream_t stream);

/* Array popcount: the number of set bits in nbytes bytes at d_in, written
 * to *d_count (device memory, one uint64).  This is the single sum that the
 * positional count generalises (Abstract; the Harley-Seal popcount of §2):
 * the same carry-save circuit with one counter, whose flush is one popc of
 * the top register.  Any start address; asynchronous on `stream`. */
int pospopcnt_popcount(const void* d_in, size_t nbytes, uint64_t* d_count, cudaStream_t stream);

/* Fused one-hot encode + count: the frequency histogram of n categorical
 * ids (unsigned, id_bytes = 1, 2 or 4 bytes each, little-endian, d_ids
 * aligned to id_bytes) over k categories, 1 <= k <= 32: d_counts[v] = the
 * number of ids equal to v, for v < k (k uint64 values, overwritten); ids
 * >= k are not counted.  This is the pipeline that motivates the paper (§1,
 * Table 1: values one-hot encoded, then positionally counted), with the
 * one-hot words built in registers and never written to memory.
 * Asynchronous on `stream`. */
int pospopcnt_onehot_counts(const void* d_ids, size_t n, int id_bytes, int k, uint64_t* d_counts,
                            cudaStream_t stream);

/* pospopcnt of HOST memory (n words at h_in); writes the width uint64
 * counts to h_counts (host memory).  Synchronous: returns when h_counts is
 * written.  If the whole range is pinned host memory mapped into the
 * device's address space (cudaHostAlloc / cudaHostRegister with mapping),
 * the kernel reads it in place across the CPU-GPU link; otherwise the bytes
 * are copied to the device in chunks through the library's staging buffers,
 * overlapping the copies with counting on two streams.  The first call on a
 * device allocates the staging buffers (2 x 64 MiB) and two streams. */
int pospopcnt_count_host(int width, const void* h_in, size_t n, uint64_t* h_counts);

/* 1 if pospopcnt_count_host would read [h_in, h_in + nbytes) in place
 * (the whole range is pinned host memory mapped into the current device's
 * address space), 0 if it would copy it through the staging buffers. */
int pospopcnt_host_is_mapped(const void* h_in, size_t nbytes);

/* Segmented pospopcnt (one persistent launch over all segments).
 * Segment s covers words [d_offsets[s], d_offsets[s+1]) of d_in; row s of
 * d_counts (width uint64 values, row-major, nseg rows) receives its counts.
 * d_offsets: nseg+1 int64 values in device memory, nondecreasing, >= 0
 * (d_offsets[0] may be > 0; validity is the caller's contract).
 * width: 8, 16 or 32 (bits).  nseg == 0 is a no-op.  Uses one of the
 * device's queue slots, chosen per stream: launches on one stream never
 * share a slot concurrently; a CUDA graph captured from a stream keeps that
 * stream's slot and must not be replayed concurrently with itself or with
 * batched calls on that stream. */
int pospopcnt_batched(const void* d_in, const int64_t* d_offsets, size_t nseg, int width,
                      uint64_t* d_counts, cudaStream_t stream);

/* Launch parameters of the batched form, per device and width.  unit_bytes:
 * the scheduling unit the warps claim from the work queue (4 KiB .. 1 MiB, a
 * multiple of 128); blocks_per_sm: CTAs per SM of the persistent grid (0: as
 * many as fit; more than fit is clamped); ring_stages: depth of each warp's
 * bulk-copy ring, 2, 3 or 4 stages (0: 2); vectors_per_lane: 16-byte words
 * each lane takes from a stage per trip, 4, 8 or 16 (0: 8), so a stage holds
 * 2, 4 or 8 KiB and a trip runs the carry-save circuit over 16 or 32
 * registers per lane (16: twice over 32) -- the analogue of the paper's
 * 256 B / 512 B / 1 kB circuit choice (§4.1); 16 takes at most 3 stages.
 * Defaults: 32 KiB, 2, 2, 8.  The paper's method has no launch parameters;
 * these tune the segmented form (§5 notes that fixed costs dominate small
 * inputs, which these trade against load balance). */
typedef struct {
  int unit_bytes;
  int blocks_per_sm;
  int ring_stages;
  int vectors_per_lane;
} pospopcnt_batched_config;

/* The configuration pospopcnt_batched (and its checked and graph forms)
 * uses for `width` on the current device. */
int pospopcnt_batched_get_config(int width, pospopcnt_batched_config* cfg);
/* Installs cfg for `width` on the current device (NULL: back to the
 * default).  POSPOPCNT_ERR_INVALID for an out-of-range field. */
int pospopcnt_batched_set_config(int width, const pospopcnt_batched_config* cfg);
/* Times every unit size in {4, 8, 16, 32, 64} KiB x CTAs per SM in {1, 2,
 * as many as fit} x ring depth in {2, 3, 4} x vectors per lane in {4, 8,
 * 16} (the valid combinations, 120) on the caller's own layout (on
 * `stream`, synchronous): three rounds interleaved across the candidates,
 * about 2 ms of back-to-back calls per round, median round.  Checks that all
 * of them produce identical rows (POSPOPCNT_ERR_INVALID and nothing
 * installed if not), installs the fastest for `width` on the current device
 * and returns it (and its time per call in ms if best_ms is not NULL).
 * d_counts receives the rows. */
int pospopcnt_batched_autotune(const void* d_in, const int64_t* d_offsets, size_t nseg, int width,
                               uint64_t* d_counts, pospopcnt_batched_config* best, float* best_ms,
                               cudaStream_t stream);

/* Returns the work-queue slot that batched calls on `stream` hold on the
 * current device (the library binds one of its 256 slots per device to
 * each stream on that stream's first batched call), and the accumulator its
 * plain counts hold (one of 1024; a stream that finds none free counts
 * through a memset instead).  Call it before destroying a stream that made
 * such calls, once none of its work is in flight; a later call on the
 * stream binds them again.  OK if the stream holds none.  (pospopcnt_graph_destroy releases its graph's slot
 * itself.)  Not in the paper: bookkeeping of the segmented form. */
int pospopcnt_release_stream(cudaStream_t stream);

/* A pospopcnt_batched call (its memset and its kernel) captured once into
 * an instantiated CUDA graph; each pospopcnt_graph_launch recounts the same
 * buffers (their contents may change between launches) with a single graph
 * launch on `stream`.  The graph owns a work-queue slot: launches of one
 * graph must not overlap each other on the GPU.  create() allocates the
 * library workspace if needed, then captures; it is synchronous. */
typedef struct pospopcnt_graph pospopcnt_graph;
int pospopcnt_batched_graph_create(const void* d_in, const int64_t* d_offsets, size_t nseg, int width,
                                   uint64_t* d_counts, pospopcnt_graph** out);
int pospopcnt_graph_launch(pospopcnt_graph* graph, cudaStream_t stream);
int pospopcnt_graph_destroy(pospopcnt_graph* graph);

/* pospopcnt_batched with the offsets checked on the device first: d_in
 * holds n_words words; unless offsets[0] >= 0, the offsets are
 * nondecreasing and offsets[nseg] <= n_words, nothing is counted (the rows
 * stay zero) and the device error word records it, so that
 * pospopcnt_check_device_error reports POSPOPCNT_ERR_INVALID.  Bad offsets
 * thus become an error status instead of reads outside d_in.  Costs one
 * small extra kernel over the offsets. */
int pospopcnt_batched_checked(const void* d_in, size_t n_words, const int64_t* d_offsets, size_t nseg,
                              int width, uint64_t* d_counts, cudaStream_t stream);

/* pospopcnt_batched for callers that cannot allocate device memory (their
 * memory belongs to another runtime's pool allocator, or they must not
 * allocate once running).  The paper has no counterpart: this is a property
 * of the library, not of the method.  Same arguments, layout and result as
 * pospopcnt_batched; it calls no cudaMalloc, cudaFree or other allocating
 * routine, and needs no pospopcnt_init.  Its scratch (the work-queue state
 * of one launch and a word where a bounded device wait records that it gave
 * up, 24 bytes in all) lives in a 256-byte static device array that every
 * GPU which loads the library holds until the process exits; a call whose
 * scratch need exceeded 256 bytes would be rejected with
 * POSPOPCNT_ERR_TOO_LARGE (the need does not grow with the input, so every
 * input size fits).  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress, with that device current): make
 * that first call before any stream capture.  Every call on a device shares
 * the one array and clears all of it on its stream before launching, so
 * calls that overlap on the GPU (calls on different streams, for instance)
 * race and give wrong counts: serialise them.  A wait that gave up is
 * reported by pospopcnt_check_device_error(stream), which allocates nothing
 * either, if it is called before the next call of this form on the device
 * clears the word. */
int pospopcnt_batched_noalloc(const void* d_in, const int64_t* d_offsets, size_t nseg, int width,
                              uint64_t* d_counts, cudaStream_t stream);

/* The per-segment alternative to pospopcnt_batched, for offsets known on
 * the host: one plain count (memset + kernel) per segment, issued in order
 * on `stream` from a host loop.  h_offsets: nseg+1 int64 word offsets in
 * host memory; d_counts as for pospopcnt_batched.  Asynchronous. */
int pospopcnt_plain_segments(const void* d_in, const int64_t* h_offsets, size_t nseg, int width,
                             uint64_t* d_counts, cudaStream_t stream);

/* ---- serving: continuous batching of jobs on one GPU ----------------------
 * Not in the paper (whose experiments count one buffer at a time): a runtime
 * that counts many independent jobs of mixed widths and sizes as they
 * arrive.  A worker thread admits jobs oldest first while the payload bytes
 * admitted and not yet completed stay within hbm_budget_bytes, launches up
 * to max_batch_jobs pending jobs of one width as one segmented count (the
 * job table travels in the kernel's parameters), keeps up to max_inflight
 * batches on the GPU on separate streams, and lets jobs that arrive
 * meanwhile join the next batch as soon as a slot frees (continuous
 * batching).  Each job's payload stays where the caller put it in device
 * memory; the GPU writes each job's counts to pinned host memory and flags
 * that job complete as soon as its own last piece is counted, so a job never
 * waits for the rest of its batch.
 * Jobs of at least large_job_bytes are launched on their own with the
 * tuned plain count (the bulk-copy ring from 64 MiB, as served payloads are
 * read-only; added into a row kept at zero, then published through
 * the same flag by a one-warp kernel).  per_request = 1 launches every job
 * that way (one plain count per job), the comparison the batched form is
 * measured against. */
typedef struct pospopcnt_server pospopcnt_server;

typedef struct {
  uint64_t hbm_budget_bytes; /* admission budget in payload bytes (0: 64 GiB) */
  int max_inflight;          /* batches (jobs, per_request) on the GPU at once, 1..256 (0: 16 or 64) */
  int max_batch_jobs;        /* jobs per batch, 1..240 (0: 240; per_request: 1) */
  int per_request;           /* 1: one plain launch per job */
  uint64_t large_job_bytes;  /* jobs at least this large get their own plain launch (0: 4 MiB) */
  int max_large_inflight;    /* such jobs on the GPU at once (0: no limit); a large job launched
                                alone gets the whole HBM bandwidth instead of sharing it */
} pospopcnt_server_config;

typedef struct {
  uint64_t tag;      /* the caller's tag (submit) or request index (trace) */
  int status;        /* POSPOPCNT_OK or the error the job met */
  int width;
  uint64_t n;        /* words */
  double t_arrival, t_admit, t_launch, t_done; /* seconds on the runtime's monotonic clock */
  uint64_t counts[32];
} pospopcnt_result;

typedef struct {
  uint64_t submitted, completed, rejected, batches, jobs_in_batches, max_batch, deferrals;
  uint64_t bytes_completed, max_bytes_in_flight;
} pospopcnt_server_stats;

/* Creates a server on `device` (allocates its slots: per slot a stream,
 * device rows and counters, and pinned mapped result and flag buffers that
 * the GPU writes) and starts its worker thread.  cfg may be NULL for the
 * defaults. */
int pospopcnt_server_create(int device, const pospopcnt_server_config* cfg, pospopcnt_server** out);

/* Waits for every submitted job, stops the worker and frees the server. */
int pospopcnt_server_destroy(pospopcnt_server* server);

/* Submits one job: n words of `width` bits at d_in (device memory, aligned
 * to the word size, unchanged until the job completes); arrival time = now.
 * POSPOPCNT_ERR_TOO_LARGE if the job alone exceeds the budget. */
int pospopcnt_server_submit(pospopcnt_server* server, int width, const void* d_in, size_t n, uint64_t tag);

/* Moves up to max completed jobs into out (non-blocking); *n_out = count. */
int pospopcnt_server_poll(pospopcnt_server* server, pospopcnt_result* out, int max, int* n_out);

/* Replays an open-loop arrival trace: request i (width[i], nwords[i] words at
 * device address d_addr[i]) is submitted at t_arrival[i] seconds after the
 * start (nondecreasing), stamped with that scheduled time, whatever the
 * state of the GPU.  Returns when every request has completed:
 * latency_out[i] = completion seen on the host - scheduled arrival (s);
 * counts_out (optional, n x 32 uint64) and status_out (optional) per
 * request.  Jobs submitted earlier finish first. */
int pospopcnt_server_run_trace(pospopcnt_server* server, size_t n, const double* t_arrival, const int* width,
                               const uint64_t* d_addr, const uint64_t* nwords, double* latency_out,
                               uint64_t* counts_out, int* status_out);

/* pospopcnt_server_run_trace that also records where each request's time
 * went: stages_out (optional, n x 3 doubles) receives, per request, the
 * seconds from its scheduled arrival to its admission (payload within the
 * HBM budget), to the launch that carries it, and to its completion seen on
 * the host.  Entries of requests that did not complete stay NaN. */
int pospopcnt_server_run_trace_timed(pospopcnt_server* server, size_t n, const double* t_arrival, const int* width,
                                     const uint64_t* d_addr, const uint64_t* nwords, double* latency_out,
                                     uint64_t* counts_out, int* status_out, double* stages_out);

int pospopcnt_server_get_stats(pospopcnt_server* server, pospopcnt_server_stats* out);

/* The server's admission policy on a mock clock (host only, no device): jobs
 * arrive at t_arrival[i] (nondecreasing) with bytes[i] of payload, are
 * admitted oldest first while the bytes admitted and not yet completed fit
 * in `budget`, and complete service_s[i] seconds after admission.  Writes
 * each job's admission time (NaN if rejected) and status
 * (POSPOPCNT_ERR_TOO_LARGE for a job larger than the budget). */
int pospopcnt_admission_simulate(uint64_t budget, size_t n, const double* t_arrival, const uint64_t* bytes,
                                 const double* service_s, double* t_admit_out, int* status_out);

/* Synchronises `stream`, reads and clears the device error words (set by
 * a bounded wait that gave up, or by the offsets check of
 * pospopcnt_batched_checked): the word of the library workspace, if the
 * workspace exists on the current device, and the word of the
 * allocation-free batched form, if that form has run there.  Allocates
 * nothing (a word that does not exist holds no error).  Returns
 * POSPOPCNT_OK, POSPOPCNT_ERR_INVALID (bad offsets only) or
 * POSPOPCNT_ERR_TIMEOUT. */
int pospopcnt_check_device_error(cudaStream_t stream);

/* Host-only planning of the head/body/tail split (§4.1 residual handling):
 * for n words of `width` bits starting at address addr, the words before the
 * first 16-byte boundary (head), the whole 16-byte vectors (body) and the
 * words after them (tail).  Touches no device. */
int pospopcnt_plan_split(int width, uint64_t addr, size_t n, size_t* head_words,
                         size_t* body_vectors, size_t* tail_words);

/* The launch configuration the library uses for (width, n) on the current
 * device, and a way to replace it for a size class (size_class =
 * floor(log4(bytes)), 0..20; -1 = every class). */
int pospopcnt_get_config(int width, size_t n, pospopcnt_config* cfg);
int pospopcnt_set_config(int width, int size_class, const pospopcnt_config* cfg);

/* Times every candidate configuration on the caller's device buffer d_in
 * (n words) with CUDA events -- each candidate in three rounds interleaved
 * with the others, each round about 2 ms of back-to-back calls (5 to 200),
 * its median round kept -- checks that all candidates produce the same
 * counts (POSPOPCNT_ERR_INVALID and nothing installed otherwise), installs
 * the fastest for that width and size class, and returns it in best (and
 * its time per call in *best_ms).  d_scratch_counts: device memory for width
 * uint64 values.  Synchronous. */
int pospopcnt_autotune(int width, const void* d_in, size_t n, uint64_t* d_scratch_counts,
                       pospopcnt_config* best, float* best_ms);

/* Self-test of the bounded-wait path used by the TMA ring: launches one warp
 * that waits on an mbarrier no one will ever complete, gives up after
 * limit_ns nanoseconds (at most 10^9), sets the device error word and
 * returns normally.  pospopcnt_check_device_error(stream) then reports
 * POSPOPCNT_ERR_TIMEOUT and clears the word.  Nothing faults or traps. */
int pospopcnt_selftest_timeout(uint64_t limit_ns, cudaStream_t stream);

/* Message for a status code, and the cudaError_t of the last CUDA failure
 * seen by this thread. */
const char* pospopcnt_strerror(int status);
int pospopcnt_last_cuda_error(void);

/* Number of kernels this library has launched in this process (all devices);
 * lets a caller count launches inside a timed region. */
uint64_t pospopcnt_launch_count(void);

/* Bytes of device memory the library currently holds from its own
 * cudaMalloc calls in this process (all devices: per-device workspaces,
 * host-path staging buffers, servers' slot buffers).  Lets a caller check
 * that a sequence of calls allocated nothing.  Not in the paper. */
uint64_t pospopcnt_device_bytes_allocated(void);

#ifdef __cplusplus
}
#endif

#endif /* POSPOPCNT_GB300_H */
