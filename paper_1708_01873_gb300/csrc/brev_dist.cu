// One array's bit-reversed permutation spread over G = 2^g ranks (one GPU
// each) that hold consecutive blocks of 2^(k-g) elements, with one
// all-to-all exchange between two local passes.
//
// With the index split i = p m l (|p| = |l| = g, |m| = k - 2g; p is the
// rank holding i, and the concatenation identity of the paper's
// Introduction, rev(x y z) = rev(z) rev(y) rev(x)):
//     rev_k(i) = rev(l) rev(m) rev(p),
// so element (p, m, l) goes to rank q = rev_g(l), at local offset
// rev(m) 2^g + rev_g(p) there.
//   pack (on rank p):   the (k-g)-bit permutation of the block, m l ->
//                       rev(l) rev(m): segment q = rev(l) of 2^(k-2g)
//                       elements is what rank q needs, ordered by rev(m);
//   exchange:           segment q of rank p -> segment p of rank q's
//                       receive buffer (equal sizes; an all-to-all);
//   finish (on rank q): receive segment p, element r -> local offset
//                       r 2^g + rev_g(p): a 2^g x 2^(k-2g) transposition
//                       with the rows taken in bit-reversed order.
// Each pass moves every local element once; the exchange moves all but the
// 1/G that stays on its rank.  The exchange itself belongs to the caller's
// collective library (NCCL send/recv or an all-to-all).
#include "brev_internal.h"
#include "brev_trace.h"

using namespace brev;

namespace {

brev_status check_dist(int log2n, int log2_ranks, int elem_bytes) {
  if (!(elem_bytes == 1 || elem_bytes == 2 || elem_bytes == 4 || elem_bytes == 8 ||
        elem_bytes == 16))
    return set_error(BREV_ERR_INVALID_ARG, "elem_bytes=%d", elem_bytes);
  if (log2_ranks < 0 || log2_ranks > BREV_DIST_MAX_LOG2_RANKS)
    return set_error(BREV_ERR_INVALID_ARG, "log2_ranks=%d outside [0, %d]", log2_ranks,
                     BREV_DIST_MAX_LOG2_RANKS);
  if (log2n < 2 * log2_ranks || log2n - log2_ranks > BREV_MAX_LOG2N)
    return set_error(BREV_ERR_INVALID_ARG,
                     "log2n=%d: needs 2 log2_ranks <= log2n and blocks of at most 2^%d",
                     log2n, BREV_MAX_LOG2N);
  return BREV_OK;
}

uint32_t rev_g(uint32_t v, int g) {
  uint32_t r = 0;
  for (int i = 0; i < g; ++i) r |= ((v >> i) & 1u) << (g - 1 - i);
  return r;
}

}  // namespace

extern "C" {

brev_status brev_dist_plan(int log2n, int log2_ranks, int elem_bytes, int rank,
                           uint64_t* send_offsets, uint64_t* recv_offsets,
                           uint64_t* segment_elems) {
  brev_status s = check_dist(log2n, log2_ranks, elem_bytes);
  if (s != BREV_OK) return s;
  const int G = 1 << log2_ranks;
  if (rank < 0 || rank >= G) return set_error(BREV_ERR_INVALID_ARG, "rank=%d of %d", rank, G);
  if (!send_offsets || !recv_offsets || !segment_elems)
    return set_error(BREV_ERR_INVALID_ARG, "NULL output");
  const uint64_t R = 1ull << (log2n - 2 * log2_ranks);
  for (int q = 0; q < G; ++q) {
    send_offsets[q] = (uint64_t)q * R;  // pack output segment q -> rank q
    recv_offsets[q] = (uint64_t)q * R;  // from rank q -> receive segment q
  }
  *segment_elems = R;
  return BREV_OK;
}

brev_status brev_dist_pack(void* send, const void* block, int log2n, int log2_ranks,
                           int elem_bytes, void* stream) {
  BREV_TRACE("brev_dist_pack");
  brev_status s = check_dist(log2n, log2_ranks, elem_bytes);
  if (s != BREV_OK) return s;
  // the local pass is the (k-g)-bit permutation of the block
  return brev_permute_to(send, block, log2n - log2_ranks, elem_bytes, stream);
}

brev_status brev_dist_finish(void* block, const void* recv, int log2n, int log2_ranks,
                             int elem_bytes, void* stream) {
  BREV_TRACE("brev_dist_finish");
  brev_status s = check_dist(log2n, log2_ranks, elem_bytes);
  if (s != BREV_OK) return s;
  const int E = elem_bytes, g = log2_ranks, c = log2n - 2 * log2_ranks;
  if (!block || !recv) return set_error(BREV_ERR_INVALID_ARG, "NULL data pointer");
  if ((uintptr_t)block % E || (uintptr_t)recv % E)
    return set_error(BREV_ERR_ALIGNMENT, "pointers must be aligned to elem_bytes=%d", E);
  const uint64_t bytes = (uint64_t)E << (log2n - g);
  const uint64_t d = (uintptr_t)block, r = (uintptr_t)recv;
  if (d < r + bytes && r < d + bytes)
    return set_error(BREV_ERR_OVERLAP, "block and receive buffer overlap");
  if (g > transpose_rowrev_max_g(E))
    return set_error(BREV_ERR_UNSUPPORTED, "log2_ranks=%d above %d for elem_bytes=%d", g,
                     transpose_rowrev_max_g(E), E);
  s = check_device_range(recv, bytes, "receive buffer");
  if (s == BREV_OK) s = check_device_range(block, bytes, "block");
  if (s != BREV_OK) return s;
  if (g == 0) {  // one rank: the receive buffer already holds the result
    cudaError_t e = cudaMemcpyAsync(block, recv, bytes, cudaMemcpyDeviceToDevice,
                                    (cudaStream_t)stream);
    return e == cudaSuccess ? BREV_OK : cuda_error(e, "copy");
  }
  return transpose_rowrev_launch(block, recv, g, c, E, (cudaStream_t)stream);
}

}  // extern "C"

// ------------------------------------------- batches sharded by array --
#include <algorithm>
#include <vector>

extern "C" brev_status brev_shard_batch(const int* log2n_array, const int* elem_bytes_array,
                                        int count, int world, int* owner) {
  if (count < 0 || world < 1) return set_error(BREV_ERR_INVALID_ARG, "count=%d world=%d", count, world);
  if (count > 0 && (!log2n_array || !elem_bytes_array || !owner))
    return set_error(BREV_ERR_INVALID_ARG, "NULL array");
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) {
    const int k = log2n_array[i], E = elem_bytes_array[i];
    if (k < 0 || k > BREV_MAX_LOG2N || E < 1 || E > 16)
      return set_error(BREV_ERR_INVALID_ARG, "array %d: log2n=%d elem_bytes=%d", i, k, E);
    order[i] = i;
  }
  auto bytes = [&](int i) { return (uint64_t)elem_bytes_array[i] << log2n_array[i]; };
  // largest arrays first, each to the rank with the fewest bytes so far
  // (ties: the lower rank); equal sizes keep their input order
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return bytes(a) > bytes(b); });
  std::vector<uint64_t> load(world, 0);
  for (int i : order) {
    const int r = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    owner[i] = r;
    load[r] += bytes(i);
  }
  return BREV_OK;
}
