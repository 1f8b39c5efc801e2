// spgemm_scan_counts_noalloc: the a3 scan (per-row counts -> row pointers) with its scratch in a fixed
// device array instead of a caller workspace, for callers that can neither allocate device memory nor
// lend a workspace at call time.
//
// The scratch is one file-scope __device__ array: a 256-byte header (a Counters record: the tile
// ticket, the status bits and the total) followed by one look-back state word per scan tile.  It
// is sized for SPGEMM_NOALLOC_MAX_ROWS rows; every device that runs this code holds it (about
// 256 KiB) until the process exits.  Nothing here calls cudaMalloc, cudaFree or any routine that
// allocates device memory.
#include "internal.h"
#include "spgemm_gb300.h"

namespace spg {
namespace {

constexpr size_t NOALLOC_HEADER_BYTES = 256;
constexpr long long NOALLOC_MAX_N = (long long)SPGEMM_NOALLOC_MAX_ROWS + 1;   // row_ptr entries
static_assert(sizeof(Counters) <= NOALLOC_HEADER_BYTES, "scratch header must hold the counters");
static_assert(NOALLOC_HEADER_BYTES % 256 == 0, "tile states must stay 256-byte aligned");

// Fixed scratch: header, then the tile states for the largest accepted size.  The public constant
// SPGEMM_NOALLOC_SCRATCH_BYTES states the same size; the assertion below keeps the two equal.
constexpr size_t SCRATCH_WORDS = NOALLOC_HEADER_BYTES / 8 + (size_t)((NOALLOC_MAX_N + 2047) / 2048);
static __device__ __align__(256) unsigned long long g_scan_scratch[SCRATCH_WORDS];
static_assert(sizeof(g_scan_scratch) == SPGEMM_NOALLOC_SCRATCH_BYTES, "stated scratch size out of date");

// Device address of g_scan_scratch in the current context.  It is looked up on every call, with
// the caller's device current: the address belongs to the context that loaded this module, and a
// context made later on the same device (after a device reset, or a driver context of the
// caller's own) loads the module at another address.  The lookup allocates nothing.
cudaError_t scratch_for_current_device(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_scan_scratch);
  if (e != cudaSuccess) return e;
  if (!p) return cudaErrorInvalidSymbol;
  *out = p;
  return cudaSuccess;
}

}  // namespace
}  // namespace spg

extern "C" spgemm_status_t spgemm_scan_counts_noalloc(int32_t* row_ptr, int64_t rows, int64_t* total, void* stream) {
  using namespace spg;
  // size and argument checks come first and touch no CUDA state
  if (!row_ptr || rows < 0) return SPGEMM_ERR_INVALID;
  if (rows > SPGEMM_NOALLOC_MAX_ROWS) return SPGEMM_ERR_SCRATCH_LIMIT;
  const long long n = rows + 1;
  if (NOALLOC_HEADER_BYTES + scan_tile_state_bytes(n) > sizeof(g_scan_scratch)) return SPGEMM_ERR_SCRATCH_LIMIT;
  cudaStream_t s = (cudaStream_t)stream;
  void* scratch = nullptr;
  if (scratch_for_current_device(&scratch) != cudaSuccess) return SPGEMM_ERR_CUDA;
  Counters* ctr = (Counters*)scratch;
  unsigned long long* tile_state = (unsigned long long*)((unsigned char*)scratch + NOALLOC_HEADER_BYTES);
  // the ticket, the status bits, the total and the tile states this call uses must start at zero
  if (cudaMemsetAsync(scratch, 0, NOALLOC_HEADER_BYTES + scan_tile_state_bytes(n), s) != cudaSuccess)
    return SPGEMM_ERR_CUDA;
  launch_scan(row_ptr, n, tile_state, ctr, &ctr->nnzC, s);
  if (cudaGetLastError() != cudaSuccess) return SPGEMM_ERR_CUDA;
  Counters h;
  if (cudaMemcpyAsync(&h, ctr, sizeof(Counters), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SPGEMM_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return SPGEMM_ERR_CUDA;
  if (h.status & ST_TIMEOUT) return SPGEMM_ERR_TIMEOUT;
  if (total) *total = h.nnzC;   // 64-bit, exact even when it overflows int32
  return (h.status & ST_OVERFLOW) ? SPGEMM_ERR_OVERFLOW : SPGEMM_OK;
}
