// Host-side declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/brev.h"

namespace brev {

// One compiled tile kernel.  kind: 0 = out-of-place tile (grid = 2^(k-bx-bz)),
// 1 = in-place pair/self units (grid = count_lt(w) + count_self(w)).
struct ShapeEntry {
  int E;        // element bytes
  int W;        // access width: 16 (vector path) or E (element-wide path)
  int bx, bz;   // tile = 2^bx source rows x 2^bz elements
  int kind;
  int order;    // 0: tile y = CTA index; 1: blocked order (runs of 8 tiles)
  const void* kernel;
  unsigned smem;   // dynamic shared memory per CTA
  int threads;     // CTA size
};

// Tables defined in brev_shapes_*.cu.
extern const ShapeEntry g_shapes_e16[];
extern const int g_shapes_e16_n;
extern const ShapeEntry g_shapes_e8[];
extern const int g_shapes_e8_n;
extern const ShapeEntry g_shapes_e4[];
extern const int g_shapes_e4_n;
extern const ShapeEntry g_shapes_e21[];
extern const int g_shapes_e21_n;

// Small-array kernel for element size E (brev_shapes_e21.cu).
const void* small_kernel(int E);

// Smallest square tile exponent whose rows are >= 128 bytes.
inline int b_min_for(int E) {
  int b = 0;
  while ((E << b) < 128) ++b;
  return b;
}

// Launch bookkeeping (brev_api.cu).
void note_launch(uint64_t n = 1);
void note_launch_adjust(int64_t delta);
brev_status set_error(brev_status s, const char* fmt, ...);
brev_status cuda_error(cudaError_t e, const char* what);
// Raise the dynamic shared-memory limit of `kernel` to `smem` on the
// current device (once per kernel and device).
cudaError_t ensure_smem(const void* kernel, unsigned smem);
// Kernel launch with programmatic stream serialisation, for kernels that
// call pdl_wait before their first global access (all but the batched
// kernel, whose launch follows its ticket reset in the stream).
cudaError_t launch_pdl(const void* kern, unsigned grid, unsigned threads, void** args,
                       unsigned smem, cudaStream_t stream);
int current_device_sm_count();
// Stream-ordered workspace from the library's own memory pool on the current
// device (brev_api.cu); released with ws_free on a stream.  Capturable.
cudaError_t ws_alloc(void** p, size_t bytes, cudaStream_t stream);
void ws_free(void* p, cudaStream_t stream);
// Validate a device range (device or managed memory, inside one allocation).
brev_status check_device_range(const void* p, uint64_t bytes, const char* what);

// Batched work (brev_batched.cu).
struct BatchItem {
  void* ptr;
  int k;
  int E;
};
brev_status batched_launch(const BatchItem* items, int count, cudaStream_t stream);
// The same launch with a caller-owned device workspace of ws_bytes >=
// batched_ws_bytes(count) (free for reuse once the stream has passed the
// launch); allocates nothing.
size_t batched_ws_bytes(int count);
brev_status batched_launch_into(const BatchItem* items, int count, void* ws, size_t ws_bytes,
                                cudaStream_t stream);
// Choices of a batched launch imposed on it (the tuner's candidates): tile
// exponent b for every array (-1: the usual choice; each array must accept
// b, see batched_candidates), pipeline stages (0: usual), tile rows staged
// as bulk copies (0) or per-thread chunks (1) (-1: usual), and consumer
// warps per CTA, 4 or 8 (0: usual).
struct BatchForce {
  int b = -1;
  int stages = 0;
  int copy = -1;
  int warps = 0;
};
brev_status batched_launch_forced(const BatchItem* items, int count, const BatchForce& f,
                                  cudaStream_t stream);
// Stage counts the batched kernel can run with stages of the array (k, E)
// at tile exponent b, into out[0..return).
int batched_stage_candidates(int k, int E, int b, int* out);
// Tile exponents the batched kernel can use for an array (k, E), into
// out[0..return); the built-in choice in *def.  0 candidates: the array is
// not run by the batched kernel.
int batched_candidates(int k, int E, int* out, int* def);
// In-place transposition of a square 2^a x 2^a matrix through the
// pipelined batched kernel (one descriptor); needs E in {4, 8, 16}, 16-byte
// alignment and a >= transpose_pipelined_b(E).
int transpose_pipelined_b(int E);
brev_status transpose_inplace_pipelined(void* data, int a, int E, cudaStream_t stream);
// ---- resident serving (kernel in brev_batched.cu, host loop in brev_serve.cu)
// One request, written by the host into page-locked memory before it
// publishes the request count.
struct ServeHostReq {
  char* ptr;
  unsigned units;  // work units (tile pairs, self tiles, or 1 whole array)
  unsigned grain;  // units per ticket
  int k, E, b, pad_;
  unsigned long long seq;           // request number (the slot is seq % ring)
  unsigned long long first_ticket;  // tickets [first_ticket, + ceil(units / grain))
};
// Host-written control words (page-locked).
struct ServeHostCtl {
  unsigned long long requests;  // requests published so far
  int stop;                     // 1: no more requests; the kernel drains and exits
  int pad_;
};
struct ResidentState {
  // page-locked host memory, read and written by the running kernel
  ServeHostReq* h_ring = nullptr;
  ServeHostCtl* h_ctl = nullptr;
  unsigned long long* h_done = nullptr;  // per slot: seq + 1 of its last completed request
  // device memory: descriptor ring, per-slot unit counters, ticket table,
  // ticket counters
  void* d_mem = nullptr;
  unsigned ring = 0, ticket_table = 0;
  int ctas = 0;  // resident CTAs of the kernel (SMs x occupancy)
};
// Allocate the state for `ring` request slots and a ticket table of
// `ticket_table` entries (both powers of two).
brev_status resident_alloc(ResidentState* st, unsigned ring, unsigned ticket_table);
void resident_free(ResidentState* st);
// Reset the counters and control words (stream-ordered for the device
// part) and launch the resident kernel on `stream`; it runs until the host
// sets h_ctl->stop (or until idle_ns pass with no new request, counted as a
// wait timeout).
brev_status resident_launch(ResidentState* st, cudaStream_t stream, unsigned long long idle_ns);
// Units, grain and tile exponent of a request in the resident kernel;
// false if it cannot run there (elem sizes 1, 2; k <= 1).
// backlog: many requests are already in flight (larger tickets then).
bool resident_shape(int k, int E, int ctas, bool backlog, int* b, unsigned* units,
                    unsigned* grain);
// Requests in flight from which new ones are admitted with backlog-sized
// tickets.
int resident_backlog_requests();
// Single arrays on the pipeline (launch order 2): valid tile exponents,
// the list of them for E, and the launch.
bool pipeline_shape_ok(int k, int E, int b);
int pipeline_shapes(int E, int* out);
brev_status bitrev_inplace_pipelined(void* data, int k, int E, int b, cudaStream_t stream);
// Tuned batched tile exponent for (k, E), or -1, and tuned stage count of
// a batch whose largest stage is this array's, or 0 (brev_api.cu).
int tuned_batched_b(int k, int E);
int tuned_batched_stages(int k, int E);
// Tuned consumer warps per CTA of a batch whose largest stage is an array
// (k, E), or 0.
int tuned_batched_warps(int k, int E);
// Tuned staging of the array's tile rows (0 bulk, 1 chunks), or -1.
int tuned_batched_copy(int k, int E);
// Argument checks of a batch (sizes, alignment, device ranges, no overlap).
brev_status validate_batch_items(const BatchItem* items, int count);
// Transposition of a 2^g x 2^c matrix whose source row x becomes
// destination column rev_g(x) (out of place, no argument checks), and the
// largest g it takes for element size E (brev_transpose.cu).
brev_status transpose_rowrev_launch(void* dst, const void* src, int g, int c, int E,
                                    cudaStream_t stream);
int transpose_rowrev_max_g(int E);
// Launch one permutation without argument checks (src == dst: in-place).
brev_status launch_single(void* dst, const void* src, int k, int E, cudaStream_t stream);
// Load the kernel that launch_single would use for (k, E, in place) -- with
// lazy module loading a kernel is otherwise loaded at its first launch.
void preload_single(int k, int E, bool inplace);
// The same for the batched kernel.
void preload_batched();

}  // namespace brev
