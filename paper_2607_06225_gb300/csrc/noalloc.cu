// noalloc.cu -- filtr_align_batch_noalloc: the batched tiled kernel, score
// only, with its scratch (work-queue counter and per-warp strip buffers) in a
// fixed file-scope device array instead of a context workspace.
//
// Some callers cannot call cudaMalloc: code running inside a host framework
// that owns all device memory and forbids further allocation, and
// latency-critical paths that cannot afford cudaMalloc's implicit device-wide
// synchronisation.  This entry point allocates nothing: no cudaMalloc, no
// cudaFree, no allocating library routine; the caller passes inputs and
// outputs, and the library's scratch is the array below, which every GPU that
// loads the library holds until the process exits.
#include <algorithm>
#include <cstdlib>
#include <mutex>

#include "filtr_ctx.h"

namespace filtr {
namespace {

// 32 MiB: 256 bytes of counters, then int2 strip buffers of (max_ref_len + 2)
// entries per resident warp.
constexpr size_t NOALLOC_SCRATCH_BYTES = 32u << 20;
constexpr size_t NOALLOC_HEADER = 256;
constexpr int NOALLOC_R = 16;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mu;
void *g_scratch_addr[MAX_DEVICES] = {};
int g_sms[MAX_DEVICES] = {};

// Set-up, once per device, with that device current: the host-side name of a
// __device__ array is only a stand-in, so the device address is looked up.
filtr_status scratch_for_current_device(void **ptr, int *sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= MAX_DEVICES) {
    set_error("device %d is beyond the %d devices this entry point tracks", dev, MAX_DEVICES);
    return FILTR_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    g_scratch_addr[dev] = p;
    g_sms[dev] = n;
  }
  *ptr = g_scratch_addr[dev];
  *sms = g_sms[dev];
  return FILTR_OK;
}

}  // namespace
}  // namespace filtr

using namespace filtr;

extern "C" {

filtr_status filtr_align_batch_noalloc(const filtr_params *params, uint32_t n_pairs,
                                       const uint8_t *q_seq, const uint64_t *q_off,
                                       const uint32_t *q_len, const uint8_t *r_seq,
                                       const uint64_t *r_off, const uint32_t *r_len,
                                       uint32_t max_query_len, uint32_t max_ref_len,
                                       filtr_result *out, void *stream) {
  ScoreParams sp;
  filtr_status rc = to_score_params(params, &sp);
  if (rc != FILTR_OK) return rc;
  if (sp.traceback) {
    set_error("filtr_align_batch_noalloc computes scores only (traceback must be 0)");
    return FILTR_ERR_UNSUPPORTED;
  }
  if (sp.use_xdrop) {
    set_error("filtr_align_batch_noalloc supports the full matrix and bands, not X-drop");
    return FILTR_ERR_UNSUPPORTED;
  }
  if (n_pairs == 0) return FILTR_OK;
  if (!q_seq || !q_off || !q_len || !r_seq || !r_off || !r_len || !out) {
    set_error("filtr_align_batch_noalloc: NULL pointer");
    return FILTR_ERR_INVALID;
  }
  // the strip buffers must hold at least one CTA's warps
  const uint64_t per_warp = ((uint64_t)max_ref_len + 2) * sizeof(int2);
  const uint64_t max_warps = (NOALLOC_SCRATCH_BYTES - NOALLOC_HEADER) / per_warp;
  if (max_ref_len == 0 || max_query_len == 0) {
    set_error("filtr_align_batch_noalloc: max_query_len and max_ref_len must be >= 1");
    return FILTR_ERR_INVALID;
  }
  if (max_query_len >= (1u << 30)) {
    set_error("max_query_len %u: queries are limited to fewer than 2^30 residues", max_query_len);
    return FILTR_ERR_UNSUPPORTED;
  }
  if (max_warps < (uint64_t)FULL_WARPS) {
    set_error("max_ref_len %u: the strip buffers of the fixed %zu-byte scratch hold references "
              "of at most %zu residues",
              max_ref_len, NOALLOC_SCRATCH_BYTES,
              (size_t)((NOALLOC_SCRATCH_BYTES - NOALLOC_HEADER) / (FULL_WARPS * sizeof(int2)) - 2));
    return FILTR_ERR_UNSUPPORTED;
  }
  if (!score_range_ok(sp, max_query_len, max_ref_len)) {
    set_error("scores could exceed 2^28 (2^26 for local alignments) for these lengths and penalties");
    return FILTR_ERR_UNSUPPORTED;
  }
  void *scratch = nullptr;
  int sms = 0;
  rc = scratch_for_current_device(&scratch, &sms);
  if (rc != FILTR_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char *base = static_cast<unsigned char *>(scratch);
  uint32_t *counter = reinterpret_cast<uint32_t *>(base);       // work queue cursor
  uint32_t *bad = reinterpret_cast<uint32_t *>(base + 64);      // invalid residue count

  // residue codes: an out-of-alphabet code would index past the score tables
  cudaError_t e = cudaMemsetAsync(base, 0, NOALLOC_HEADER, st);
  BatchDev b{q_seq, r_seq, q_off, r_off, q_len, r_len};
  if (e == cudaSuccess) e = launch_validate_pairs(b, n_pairs, sp.alphabet, bad, st);
  uint32_t h_bad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_bad, bad, sizeof h_bad, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "filtr_align_batch_noalloc: validation");
  if (h_bad) {
    set_error("%u residue codes are >= the alphabet size %d", h_bad, sp.alphabet);
    return FILTR_ERR_INVALID;
  }

  FullArgs fa{};
  fa.b = b;
  fa.sp = sp;
  fa.order = nullptr;  // pairs in input order
  fa.n_order = n_pairs;
  fa.counter = counter;
  fa.out = out;
  fa.fwd = nullptr;
  fa.tb = nullptr;
  fa.tbl = nullptr;
  fa.strip_buf = reinterpret_cast<int2 *>(base + NOALLOC_HEADER);
  fa.strip_stride = max_ref_len + 2;
  fa.max_n = max_ref_len;
  fa.max_m = max_query_len;
  fa.ck = nullptr;
  const int bps = std::max(1, full_max_blocks_per_sm(NOALLOC_R, sp, sp.alphabet));
  int64_t grid = std::min<int64_t>((int64_t)sms * bps, (int64_t)(max_warps / FULL_WARPS));
  grid = std::min<int64_t>(grid, ((int64_t)n_pairs + FULL_WARPS - 1) / FULL_WARPS);
  e = launch_full(fa, NOALLOC_R, (int)std::max<int64_t>(grid, 1), st);
  if (e != cudaSuccess) return cuda_fail(e, "filtr_align_batch_noalloc: launch");
  return FILTR_OK;
}

}  // extern "C"
