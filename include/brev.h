/*
 * brev.h -- C ABI of the GB300 (sm_103a) bit-reversed permutation library.
 *
 * The operation (paper: "Practically efficient methods for performing
 * bit-reversed permutation in C++11 on the x86-64 architecture",
 * Introduction, definition of the bit-reversed permutation and its n = 8
 * worked example): for an array of n = 2^k elements, the element at index
 * i moves to index rev_k(i), the k-bit reversal of i.  Elements are opaque
 * blobs of elem_bytes bytes (1, 2, 4, 8 or 16: uint8 ... complex<double>);
 * they are moved, never interpreted, so every bit pattern (NaN, -0.0) is
 * preserved and results are exact.
 *
 * General conventions
 *   - log2n is k, 0 <= k <= 34; n = 2^k elements.  k = 0 and k = 1 are the
 *     identity.
 *   - Data pointers are DEVICE pointers (cudaMalloc / torch CUDA tensors).
 *     Host or unregistered pointers are rejected with BREV_ERR_INVALID_ARG
 *     before anything is launched.  Each pointer must be aligned to
 *     elem_bytes (else BREV_ERR_ALIGNMENT).  Pointers that are also 16-byte
 *     aligned take the 16-byte vector path; others take an element-wide path
 *     on the GPU.  There is no CPU fallback.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  All
 *     calls are stream-ordered and asynchronous: they enqueue work and
 *     return; the caller synchronises.  Only brev_autotune and
 *     brev_permute_host (see there) block the calling thread.
 *   - The caller owns every data buffer.  The library owns only its small
 *     device workspaces (batch descriptors, ticket counters, host-path
 *     staging), plans and the tuning table.  Workspaces are stream-ordered
 *     allocations from a memory pool the library creates per device on
 *     first use; it keeps up to 32 MiB reserved across synchronisations
 *     (so a call right after a synchronise does not map memory again) and
 *     lives until the process exits.  The device's default memory pool is
 *     not touched.
 *   - Every call returns a brev_status.  On failure nothing was enqueued
 *     (except for BREV_ERR_CUDA raised by the launch itself), and
 *     brev_last_error() returns a message for the calling thread.
 *   - Calls are thread-safe.
 */
#ifndef BREV_H
#define BREV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define BREV_API __attribute__((visibility("default")))
#else
#define BREV_API
#endif

#define BREV_VERSION 1000 /* 1.0.0 */
#define BREV_MAX_LOG2N 34

typedef enum brev_status {
    BREV_OK = 0,
    BREV_ERR_INVALID_ARG = 1, /* bad k / elem_bytes / count / null or host pointer */
    BREV_ERR_ALIGNMENT = 2,   /* pointer not aligned to elem_bytes */
    BREV_ERR_OVERLAP = 3,     /* out-of-place source and destination partly overlap */
    BREV_ERR_OOM = 4,         /* a library workspace could not be allocated */
    BREV_ERR_CUDA = 5,        /* a CUDA runtime call failed (see brev_last_error) */
    BREV_ERR_UNSUPPORTED = 6  /* a valid request this build does not handle */
} brev_status;

/* ---------------------------------------------------------------- single */

/* Out-of-place permutation dst[rev_k(i)] = src[i] (Introduction, the
 * definition; Introduction, "Bit reversal using a matrix buffer": the
 * kernel is the matrix-buffer method with a 2^bx x 2^bz shared-memory
 * buffer per tile, index = x y z, destination rev(z) rev(y) rev(x)).
 * dst and src: device pointers to 2^log2n elements each.  src == dst is
 * allowed and means in-place (the pair-swap form below).  Partial overlap
 * returns BREV_ERR_OVERLAP. */
BREV_API brev_status brev_permute_to(void *dst, const void *src, int log2n, int elem_bytes,
                            void *stream);

/* Single-pointer form.  in_place != 0: `data` holds 2^log2n elements and is
 * permuted in place (Introduction, Listing 1: each index swaps with its
 * reverse once; here each tile swaps with its partner tile rev(y), and
 * self-paired tiles are permuted inside one CTA).  in_place == 0: `data`
 * holds 2n elements laid out as [src | dst]; the first n are read and the
 * permutation is written to the second n. */
BREV_API brev_status brev_permute(void *data, int log2n, int elem_bytes, int in_place,
                         void *stream);

/* ---------------------------------------------------------------- batched */

/* In-place permutation of `count` independent arrays in ONE persistent
 * kernel launch (a work queue over tiles; no counterpart in the paper,
 * whose methods handle one array).  ptr_array[i] is a device pointer to
 * 2^log2n_array[i] elements of elem_bytes bytes.  ptr_array and
 * log2n_array are HOST arrays, read before the call returns.  Arrays must
 * not overlap one another.  count == 0 is a no-op.  The call uploads the
 * batch's descriptors from pageable host memory into stream-ordered
 * workspace, so it cannot be captured into a CUDA graph: capture a plan
 * (brev_plan_create) instead. */
BREV_API brev_status brev_permute_batched(void *const *ptr_array, const int *log2n_array,
                                 int count, int elem_bytes, void *stream);

/* The same with a per-array element size (mixed complex<float> and
 * complex<double> batches in one launch).  elem_bytes_array is a host
 * array of count entries, each in {1,2,4,8,16}. */
BREV_API brev_status brev_permute_batched_mixed(void *const *ptr_array, const int *log2n_array,
                                       const int *elem_bytes_array, int count,
                                       void *stream);

/* A batch captured once into a CUDA graph (ticket reset + persistent
 * kernel) and replayed by brev_plan_launch.  The arrays' pointers and
 * sizes are fixed at creation; their contents may change between
 * launches.  Each launch permutes every array in place once (so two
 * launches restore the input).  elem_bytes_array may be NULL with
 * elem_bytes giving one size for all arrays.  Creation allocates the
 * plan's device workspace and may synchronise the device. */
typedef struct brev_plan brev_plan;
BREV_API brev_status brev_plan_create(void *const *ptr_array, const int *log2n_array,
                             const int *elem_bytes_array, int elem_bytes, int count,
                             brev_plan **out_plan);
BREV_API brev_status brev_plan_launch(brev_plan *plan, void *stream);
BREV_API void brev_plan_destroy(brev_plan *plan);

/* No-allocation form of brev_permute_batched_mixed.  The paper has no
 * counterpart: it exists for callers that cannot allocate device memory --
 * code whose device memory is entirely handed to another allocator (a
 * framework's caching pool, a fixed arena), or latency-critical loops in
 * which a cudaMalloc, which can synchronise the device and can fail under
 * fragmentation, is not acceptable.  Same arguments and result as
 * brev_permute_batched_mixed, but the call allocates nothing: its scratch
 * (ticket counter and per-array descriptors) is a fixed device array inside
 * the library of 256 + BREV_NOALLOC_MAX_ARRAYS * 48 bytes (about 48 KiB),
 * which every GPU that loads the library holds until the process exits.
 *   - count > BREV_NOALLOC_MAX_ARRAYS returns BREV_ERR_INVALID_ARG.
 *   - The first call on a device looks up the array's device address (once
 *     per device, with that device current); make that first call before
 *     any stream capture.
 *   - Every call on a device shares that device's one array and overwrites
 *     the previous call's contents (descriptors uploaded and counter zeroed
 *     on `stream`), so calls ordered on one stream are safe, while calls
 *     that overlap on the GPU (for example on two streams) race.
 *   - Arrays of 1- or 2-byte elements, or not 16-byte aligned, are permuted
 *     by single-array launches within the call (these allocate no device
 *     memory either). */
#define BREV_NOALLOC_MAX_ARRAYS 1024
BREV_API brev_status brev_permute_batched_noalloc(void *const *ptr_array, const int *log2n_array,
                                                  const int *elem_bytes_array, int count,
                                                  void *stream);

/* ------------------------------------------- one array over several GPUs */

/* The permutation of one array of 2^log2n elements held by G = 2^log2_ranks
 * ranks (one GPU each), rank p holding the consecutive block of elements
 * [p 2^(log2n - log2_ranks), (p + 1) 2^(log2n - log2_ranks)).  By the
 * concatenation identity of the paper's Introduction (rev(x y z) =
 * rev(z) rev(y) rev(x)), element (p, m, l) -- rank, middle and low log2_ranks
 * bits of its index -- goes to rank rev(l) at local offset
 * rev(m) 2^log2_ranks + rev(p).  Three steps per rank, each block of
 * 2^(log2n - log2_ranks) elements:
 *   1. brev_dist_pack: a local pass into the send buffer, whose segment q
 *      (2^(log2n - 2 log2_ranks) elements) is what rank q needs;
 *   2. the caller's exchange: segment q of every rank p's send buffer to
 *      segment p of rank q's receive buffer (an all-to-all of equal parts;
 *      brev_dist_plan gives the offsets in elements);
 *   3. brev_dist_finish: a local pass from the receive buffer into the
 *      block, which then holds the block's part of the permuted array.
 * Constraints: 2 log2_ranks <= log2n, blocks of at most 2^34 elements,
 * log2_ranks <= BREV_DIST_MAX_LOG2_RANKS and, for the finish, at most 5
 * (16-byte elements), 5 (8), 6 (4), 7 (2), 8 (1).  Buffers are device
 * memory of the calling rank's current device, aligned to elem_bytes.
 * Errors: BREV_ERR_INVALID_ARG, BREV_ERR_ALIGNMENT, BREV_ERR_OVERLAP,
 * BREV_ERR_UNSUPPORTED, BREV_ERR_CUDA, as brev_permute_to. */
#define BREV_DIST_MAX_LOG2_RANKS 10

/* Offsets (in elements) of the exchange on rank `rank`: segment q of the
 * send buffer starts at send_offsets[q] and goes to rank q; the segment
 * from rank q lands at recv_offsets[q]; every segment holds
 * *segment_elems elements.  send_offsets and recv_offsets hold
 * 2^log2_ranks entries.  Host-only (no GPU needed). */
BREV_API brev_status brev_dist_plan(int log2n, int log2_ranks, int elem_bytes, int rank,
                                    uint64_t *send_offsets, uint64_t *recv_offsets,
                                    uint64_t *segment_elems);
/* Step 1: send = the (log2n - log2_ranks)-bit permutation of block (send may
 * equal block: in place). */
BREV_API brev_status brev_dist_pack(void *send, const void *block, int log2n, int log2_ranks,
                                    int elem_bytes, void *stream);
/* Step 3: block[r 2^log2_ranks + rev(p)] = recv[p 2^(log2n - 2 log2_ranks) + r]
 * (a transposition with the rows taken in bit-reversed order); block and
 * recv must not overlap. */
BREV_API brev_status brev_dist_finish(void *block, const void *recv, int log2n, int log2_ranks,
                                      int elem_bytes, void *stream);

/* A batch of independent arrays split across `world` ranks by array: owner[i]
 * receives the rank that permutes array i.  Arrays go largest first to the
 * rank with the fewest bytes so far, so every rank's share of the bytes is
 * within one array of the mean.  Host-only; the same inputs give the same
 * owners on every rank (no communication needed).  Errors:
 * BREV_ERR_INVALID_ARG. */
BREV_API brev_status brev_shard_batch(const int *log2n_array, const int *elem_bytes_array,
                                      int count, int world, int *owner);

/* ---------------------------------------------------------------- transpositions */

/* Transposition of a row-major 2^log2_rows x 2^log2_cols matrix of
 * elem_bytes elements: dst[j * 2^log2_rows + i] = src[i * 2^log2_cols + j].
 * The paper (Introduction) reads the Stockham even-odd step as such a
 * transposition.  Same tile machinery as the permutation (staged through
 * shared memory, whole rows moved in 16-byte vectors), with identity index
 * maps.  dst == src is allowed for square matrices only (in place, tile
 * pairs swapped); a non-square matrix in place returns
 * BREV_ERR_UNSUPPORTED. */
BREV_API brev_status brev_transpose(void *dst, const void *src, int log2_rows, int log2_cols,
                                    int elem_bytes, void *stream);

/* Even-odd step of the Stockham auto-sort (Introduction): the even-indexed
 * elements in order, then the odd-indexed ones; the transposition of the
 * n/2 x 2 matrix.  Out of place only (dst == src only for n <= 4). */
BREV_API brev_status brev_even_odd(void *dst, const void *src, int log2n, int elem_bytes,
                                   void *stream);

/* Perfect (faro) shuffle, the inverse of the even-odd step: the two halves
 * interleaved; the transposition of the 2 x n/2 matrix. */
BREV_API brev_status brev_perfect_shuffle(void *dst, const void *src, int log2n,
                                          int elem_bytes, void *stream);

/* In-place bit reversal of each of 2^log2_segments contiguous segments of
 * 2^log2_seglen elements (one launch for all segments).  The small,
 * contiguous bit reversals of the paper's recursive method (Methods,
 * cache-oblivious recursive bit-reversed permutation). */
BREV_API brev_status brev_permute_segments(void *data, int log2_segments, int log2_seglen,
                                           int elem_bytes, void *stream);

/* The paper's recursive method with one level of recursion, in place, as a
 * multi-pass comparison point for the one-pass tile kernel (Methods,
 * cache-oblivious recursive bit-reversed permutation; Results, the GPU
 * variant): for even k, index = x y with k/2 bits each, reverse every
 * contiguous block (x rev(y)), transpose the square matrix (rev(y) x),
 * reverse every block again (rev(y) rev(x)) -- three read+write passes.  Odd
 * k takes the even-odd step first (Methods, odd number of bits) into
 * stream-ordered device workspace, permutes each half, and copies back.
 * Same result as brev_permute(data, log2n, elem_bytes, 1, stream). */
BREV_API brev_status brev_permute_recursive(void *data, int log2n, int elem_bytes,
                                            void *stream);

/* ---------------------------------------------------------------- fused FFT stages */

/* The bit-reversed permutation fused with the first `stages` radix-2
 * decimation-in-time FFT stages (Introduction: after the permutation, every
 * level of the Cooley-Tukey recursion finds its even-odd split already
 * done).  dst = stages 1..S applied to the permuted src, where stage s
 * combines, in each block of m = 2^s consecutive elements, a[j] and
 * a[j + m/2] (j < m/2) with w = exp(-2 pi i j / m) (the conjugate when
 * inverse != 0): (a[j], a[j+m/2]) <- (a[j] + w a[j+m/2], a[j] - w a[j+m/2]).
 * elem_bytes 8 = complex<float> (float arithmetic) or 16 = complex<double>
 * (double arithmetic); arrays 16-byte aligned; dst == src runs in place.
 * The butterflies run on the shared-memory tile between load and store, so
 * permutation and stages take one HBM round trip.  stages = 0 is the plain
 * permutation; stages up to 6 are supported for every size (up to log2n
 * when the whole array fits one CTA); more return BREV_ERR_UNSUPPORTED.
 * Results are floating point: they match a double-precision reference to
 * within rounding (see the tests for the bound).  complex<double> arrays
 * with more 2^5 x 2^5 tiles (or tile pairs, in place) than the device has
 * resident CTA slots for them (log2n >= 20 out of place and >= 21 in
 * place on GB300, stages <= 5) run one CTA per slot, which
 * claim tiles from a 16-byte counter taken from the library's workspace
 * pool in stream order (BREV_ERR_OOM if it cannot be had); the results are
 * the same bit for bit as with one CTA per tile.  Everything the call
 * enqueues (that allocation, a memset, the kernel, the release) can be
 * captured into a CUDA graph; a GPU test captures and replays it. */
BREV_API brev_status brev_fft_stages(void *dst, const void *src, int log2n, int elem_bytes,
                                     int stages, int inverse, void *stream);

/* ---------------------------------------------------------------- serving */

/* A native serving loop (no counterpart in the paper): requests for the
 * in-place permutation of arrays of different sizes arrive over time and
 * are served by continuous batching.
 *   - Admission: first in, first out, when a slot is free and a first-fit
 *     pool over the caller's device arena can hold the request's
 *     2^k * elem_bytes bytes (admission by free HBM, the pool's own
 *     accounting).
 *   - Launch: every loop iteration puts all admitted requests (at most
 *     max_batch) into ONE launch -- single-array for one request, the
 *     persistent batched kernel for more -- on an idle stream, round robin
 *     over n_streams, so requests arriving while others run overlap with
 *     them on the device.
 *   - Completion: a CUDA event per batch; when the serving thread sees it
 *     complete, the batch's requests are complete (latency = that time -
 *     arrival) and their memory and slots are released.
 * Resident mode (resident = 1) replaces the launches: one kernel stays on
 * the GPU for the whole run and takes requests from a ring in page-locked
 * host memory (NVLink-C2C), so no request pays a kernel launch:
 *   - admission is the same (FIFO head, slots, pool), plus room in the ring
 *     (4096 requests) and in the kernel's ticket window (2^22 tickets);
 *   - each admitted request is written into the ring and published at once;
 *     the kernel spreads its tile units over all CTAs (~64 KiB tickets, or
 *     256 KiB while 16 or more requests are in flight), so
 *     requests in flight overlap on the device;
 *   - the kernel writes a completion word per request into host memory;
 *   - element sizes 4, 8 and 16 only (BREV_ERR_UNSUPPORTED otherwise);
 *     max_batch and n_streams are not used.
 *   The kernel's waits are bounded: if the run stalls for 2 s with nothing
 *   to do (no request and no end of run), it exits, the waits are counted
 *   in brev_wait_timeouts, and the run returns BREV_ERR_CUDA.  While it
 *   runs it holds every SM (other kernels on the device wait); after 0.5 s
 *   with nothing in flight the host stops it and relaunches it at the next
 *   request.
 * The arena is a caller-owned device buffer (256-byte aligned); the server
 * owns its streams and events. */
typedef struct brev_server brev_server;
typedef struct brev_server_config {
    int max_slots; /* requests admitted at once (resident: at most 4096) */
    int max_batch; /* requests per launch */
    int n_streams; /* streams with a batch in flight, 1..64 */
    int resident;  /* 1: resident kernel fed through host memory, 0: launches */
    int idle_stop_ms; /* resident: stop the kernel after this long with nothing
                       * in flight or waiting (0 = 500 ms); above 2000 the
                       * kernel's own idle limit ends it first, and the run
                       * fails with BREV_ERR_CUDA at the next request */
} brev_server_config;
typedef struct brev_server_stats {
    uint64_t offered, completed, batches, launches;
    double p50_us, p99_us, max_us, mean_us; /* completion seen by the serving
                                             * thread - arrival (what a client
                                             * waits), both modes */
    double queue_p99_us;                    /* launch or publication - arrival */
    double req_per_s, gbs, wall_s;          /* gbs: 2 n E bytes per request / wall time */
    uint64_t peak_pool_bytes;
    int max_inflight;
    double device_p50_us, device_p99_us;    /* launches: completion event on the
                                             * device clock - arrival (read
                                             * against a reference event, which
                                             * completed slightly before the run's
                                             * host clock started, so biased
                                             * high by that gap); resident:
                                             * equal to p50_us, p99_us */
} brev_server_stats;
typedef struct brev_server_request {
    uint64_t offset; /* byte offset of the request's buffer in the arena */
    int log2n, elem_bytes, batch;
    double arrival_us, launch_us, done_us; /* since the run started; launch: host
                                            * time of the enqueue (publication
                                            * when resident), done: completion on
                                            * the device clock (launches) or seen
                                            * by the serving thread (resident) */
    double seen_us; /* completion seen by the serving thread (both modes): the
                     * latency p50_us / p99_us count, seen_us - arrival_us */
} brev_server_request;

BREV_API brev_status brev_server_create(const brev_server_config *cfg, void *arena,
                                        uint64_t arena_bytes, brev_server **out);
BREV_API void brev_server_destroy(brev_server *srv);

/* Serve a seeded Poisson stream in the calling thread (after waiting for all
 * earlier work on the device, so the arena may be written on any stream
 * beforehand; the call returns when every request has completed):
 * exponential gaps of
 * mean 1/rate_per_s over `seconds`, k uniform in [k_min, k_max], element
 * size uniform over elem_bytes[0..n_elem_bytes).  Each request permutes, in
 * place, the arena bytes the pool gave it (whatever they hold).
 * hold_results != 0 keeps every completed request's buffer reserved until
 * the run ends, so that the arena afterwards holds all results (needs an
 * arena large enough for the whole stream).  trace, if not NULL, receives
 * up to trace_capacity per-request records in arrival order. */
BREV_API brev_status brev_server_run_poisson(brev_server *srv, uint64_t seed, double rate_per_s,
                                             double seconds, int k_min, int k_max,
                                             const int *elem_bytes, int n_elem_bytes,
                                             int hold_results, brev_server_request *trace,
                                             uint64_t trace_capacity, brev_server_stats *out);

/* ---------------------------------------------------------------- host path */

/* End-to-end form for host buffers: permutes src_host (2^log2n elements)
 * into dst_host (which may equal src_host) on `stream`, then waits for the
 * stream.  When both buffers are page-locked (cudaHostAlloc /
 * cudaHostRegister) and the driver confirms that each whole range lies in
 * its allocation, the tile kernel reads and writes the host memory
 * directly over the CPU-GPU link (no device copy).  Otherwise the source is
 * copied to stream-ordered device workspace, permuted there, and copied
 * back.  The buffers must hold 2^log2n elements each. */
BREV_API brev_status brev_permute_host(void *dst_host, const void *src_host, int log2n,
                              int elem_bytes, void *stream);

/* ---------------------------------------------------------------- tuning */

/* Tile shape used for (log2n, elem_bytes, in_place): bx high bits and bz
 * low bits per tile (the matrix-buffer side lengths 2^bx, 2^bz); bx = bz =
 * 0 means the whole array is staged in one CTA (small arrays).  order is
 * how the tiles are run: 0 = tile y by CTA y, 1 = blocked (consecutive
 * CTAs take 8 x 8 blocks of (high, low) bits of y, so that both the tiles
 * and their destinations come in runs of 8 adjacent tiles), 2 = the TMA
 * pipeline (in place only: persistent CTAs take tickets of tile pairs and
 * stage their rows by bulk copies; element sizes 4, 8, 16).  Host-only
 * query, no GPU needed. */
BREV_API brev_status brev_tile_shape(int log2n, int elem_bytes, int in_place, int *bx, int *bz,
                                     int *order);

/* Tile exponent b the batched kernel uses for an array of 2^log2n elements
 * of elem_bytes (square 2^b x 2^b tiles staged by bulk copies; b = 0 means
 * the whole array is staged in one unit).  The tuned value when the tuner
 * or a loaded cache set one for (log2n, elem_bytes), else the built-in
 * choice.  BREV_ERR_UNSUPPORTED: such an array is not run by the batched
 * kernel (element sizes 1 and 2, or log2n <= 1, which is the identity);
 * the batched calls permute it with a single-array launch instead.
 * Host-only query, no GPU needed. */
BREV_API brev_status brev_batched_shape(int log2n, int elem_bytes, int *b);

/* Run the permutation with a forced tile shape and launch order (tests and
 * the tuner).  Out-of-place accepts bx != bz; in-place requires bx == bz.
 * Shapes that are not compiled in return BREV_ERR_UNSUPPORTED.  src == dst
 * means in-place. */
BREV_API brev_status brev_permute_shape(void *dst, const void *src, int log2n, int elem_bytes,
                                        int bx, int bz, int order, void *stream);

/* Number of compiled 16-byte-path (tile shape, launch order) pairs for
 * (elem_bytes, in_place), including the TMA pipeline's tile exponents (order
 * 2) for in place, and the i-th one (host-only; the tuner's candidates). */
BREV_API int brev_shape_count(int elem_bytes, int in_place);
BREV_API brev_status brev_shape_at(int elem_bytes, int in_place, int i, int *bx, int *bz,
                                   int *order);

/* Time every compiled shape for k in [k_min, k_max] (out-of-place and
 * in-place; in place also the TMA pipeline, order 2, so the choice between
 * the LSU tile kernels and bulk-copy staging is measured per (k, E)), keep
 * the fastest in the library's table, and, if cache_path
 * is not NULL, write the table as JSON.  For elem_bytes 4, 8 and 16 it also
 * times the batched kernel's tile exponent b for each k up to 24 on a
 * batch of equal arrays (up to 4096 arrays, about 256 MiB), and keeps the
 * fastest (brev_batched_shape).  Allocates and frees its own device
 * buffers; blocks the calling thread. */
BREV_API brev_status brev_autotune(int k_min, int k_max, int elem_bytes, const char *cache_path);

/* Load a table written by brev_autotune.  Entries whose device name or SM
 * count differ from the current device are ignored.  Host-only apart from
 * the device-name query. */
BREV_API brev_status brev_load_tune_cache(const char *cache_path);

/* Forget tuned shapes and batched tile exponents (back to the built-in
 * defaults). */
BREV_API void brev_reset_tuning(void);

/* ---------------------------------------------------------------- info */

typedef struct brev_device_info {
    int sm_count;
    int l2_bytes;
    int mem_clock_khz;   /* peak memory clock */
    int mem_bus_bits;    /* global memory bus width */
    double nominal_gbs;  /* mem_clock_khz * 2 (DDR) * mem_bus_bits / 8 */
    int max_smem_per_block;
    char name[96];
} brev_device_info;

/* Properties of the current device (needs a GPU). */
BREV_API brev_status brev_get_device_info(brev_device_info *out);

/* Measured FP64 fused multiply-add rate of the current device, in TFLOP/s
 * (2 flops per FMA): the ceiling of the complex<double> FFT stages of
 * brev_fft_stages, whose time is their FP64 arithmetic.  The paper has no
 * counterpart; it is the denominator of that roofline.  Runs a kernel of
 * independent FMA chains on every SM for about 10 ms, four times on a
 * stream of its own, and returns the best of the last three; blocks the
 * calling thread.  Errors: BREV_ERR_INVALID_ARG (NULL), BREV_ERR_CUDA. */
BREV_API brev_status brev_fp64_fma_tflops(double *tflops);

/* Measured rate (GB/s, read + write bytes) of a plain copy kernel that reads
 * `bytes` of page-locked host memory at src_host and writes them to
 * page-locked host memory at dst_host -- the same route the host-buffer
 * permutation takes (the SMs load and store host memory over the CPU-GPU
 * link) with no permutation: the ceiling of brev_permute_host.  The paper
 * has no counterpart.  Both pointers 16-byte aligned, bytes a multiple of 16,
 * no overlap.  Four copies on a stream of its own, best of the last three;
 * blocks the calling thread.  Errors: BREV_ERR_INVALID_ARG (NULL, not
 * page-locked), BREV_ERR_ALIGNMENT, BREV_ERR_OVERLAP, BREV_ERR_CUDA. */
BREV_API brev_status brev_host_link_gbs(void *dst_host, const void *src_host, uint64_t bytes,
                                        double *gbs);

/* Number of kernel launches the library has issued on this process (all
 * entry points); lets callers count launches inside a timed region. */
BREV_API uint64_t brev_launch_count(void);

/* Device memory of the library's workspace pool on the current device:
 * *reserved = bytes the pool holds from the device, *used = bytes of it in
 * use by work not yet released (both 0 before the first call that needs
 * workspace on this device).  The pool keeps up to 32 MiB reserved across
 * synchronisations.  Host-side query; it creates nothing.  Errors:
 * BREV_ERR_INVALID_ARG (a NULL output), BREV_ERR_CUDA. */
BREV_API brev_status brev_workspace_bytes(uint64_t *reserved, uint64_t *used);

/* Number of times a CTA of the batched kernel gave up waiting for its own
 * bulk copies into shared memory (about one second with the copies not
 * complete), on the current device since the library was loaded.  Each
 * such CTA stops early, so some arrays of that batch are left partly
 * permuted; the count is 0 on a healthy device.  Waits for all earlier work
 * on the device (a synchronous read).  Errors: BREV_ERR_INVALID_ARG (out is
 * NULL), BREV_ERR_CUDA. */
BREV_API brev_status brev_wait_timeouts(uint64_t *out);

BREV_API const char *brev_status_string(brev_status s);
/* Message of the last failing call on this thread ("" if none). */
BREV_API const char *brev_last_error(void);
BREV_API int brev_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BREV_H */
