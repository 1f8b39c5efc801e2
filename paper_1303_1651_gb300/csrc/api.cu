// C ABI of the SpGEMM library: plan object, workspace layout, call sequencing.
// See include/spgemm_gb300.h for the contract of every entry point.
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "internal.h"
#include "spgemm_gb300.h"

using namespace spg;

namespace {

constexpr size_t ALIGN = 256;
inline size_t up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

struct Layout {
  size_t ctr, cls, list_w, list_b, list_g, scan, fused, slabs, total;
};

Layout layout(int m, int ncols, int nslabs) {
  Layout L{};
  size_t o = 0;
  L.ctr = o; o += up(sizeof(Counters));
  L.cls = o; o += up((size_t)std::max(m, 1));
  L.list_w = o; o += up(4 * (size_t)std::max(m, 1));
  L.list_b = o; o += up(4 * (size_t)std::max(m, 1));
  L.list_g = o; o += up(4 * (size_t)std::max(m, 1));
  L.scan = o; o += up(scan_tile_state_bytes((long long)m + 1) + 64);
  L.fused = o; o += up(fused_tile_state_bytes(m) + 64);
  L.slabs = o; o += (size_t)nslabs * dense_slab_bytes(ncols);
  L.total = o;
  return L;
}

Limits limits_from(const spgemm_options_t* o) {
  Limits l{8, 32, 64, 1024, 4096};
  if (o) {
    if (o->merge_max_k > 0) l.merge_k = std::min(o->merge_max_k, 8);
    if (o->m1_max_u > 0) l.m1_u = std::min(o->m1_max_u, 32);
    if (o->m2_max_u > 0) l.m2_u = std::min(o->m2_max_u, 64);
    if (o->warp_max_u > 0) l.warp_u = std::min(o->warp_max_u, 1024);
    if (o->block_max_u > 0) l.block_u = std::min(o->block_max_u, 4096);
    if (o->m1_max_u < 0) l.m1_u = -1;     // negative: class disabled (testing hook)
    if (o->m2_max_u < 0) l.m2_u = -1;
    if (o->warp_max_u < 0) l.warp_u = -1;
    if (o->block_max_u < 0) l.block_u = -1;
  }
  l.m2_u = std::max(l.m2_u, l.m1_u);
  return l;
}

int slabs_from(const spgemm_options_t* o) { return (o && o->dense_slabs > 0) ? o->dense_slabs : 2; }

bool desc_ok(const spgemm_csr_t* M) {
  if (!M || M->rows < 0 || M->cols < 0 || M->nnz < 0 || M->nnz > INT32_MAX) return false;
  if (!M->row_ptr && M->rows > 0) return false;
  if (!M->col_idx && M->nnz > 0) return false;
  return true;
}

DevCsr to_dev(const spgemm_csr_t& M) {
  return DevCsr{M.rows, M.cols, (long long)M.nnz, M.row_ptr, M.col_idx, M.val};
}

spgemm_status_t status_from_bits(unsigned bits) {
  if (bits & ST_INVALID) return SPGEMM_ERR_INVALID;
  if (bits & ST_OVERFLOW) return SPGEMM_ERR_OVERFLOW;
  if (bits & ST_UNSORTED) return SPGEMM_ERR_UNSORTED;
  if (bits & ST_TABLE_FULL) return SPGEMM_ERR_TABLE_FULL;
  if (bits & ST_TIMEOUT) return SPGEMM_ERR_TIMEOUT;
  if (bits & ST_MISMATCH) return SPGEMM_ERR_MISMATCH;
  return SPGEMM_OK;
}

}  // namespace

// a small CSR validation pass (optional): monotone row pointers, ends, column range
namespace spg {
__global__ void k_validate(DevCsr M, Counters* ctr) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  bool bad = false;
  for (long long r = tid; r < M.rows; r += stride) bad |= M.rp[r] > M.rp[r + 1];
  if (tid == 0) bad |= (M.rows >= 0 && (M.rp[0] != 0 || M.rp[M.rows] != M.nnz));
  for (long long p = tid; p < M.nnz; p += stride) bad |= (unsigned)M.col[p] >= (unsigned)M.cols;
  if (bad) atomicOr(&ctr->status, ST_INVALID);
}
}  // namespace spg

namespace {

// Counters are read back to the host after every synchronising call.  Through pinned memory
// that is one DMA; through pageable memory the CUDA driver stages the copy.  A small pinned buffer,
// allocated once per process on first use, gives each live plan a slot while slots last (plans
// beyond that read into their own pageable copy).
constexpr int PINNED_SLOTS = 256;
std::mutex g_pin_mu;
Counters* g_pin_base = nullptr;
bool g_pin_tried = false;
std::vector<int> g_pin_free;

Counters* pinned_take() {
  std::lock_guard<std::mutex> lock(g_pin_mu);
  if (!g_pin_tried) {
    g_pin_tried = true;
    void* b = nullptr;
    if (cudaHostAlloc(&b, PINNED_SLOTS * sizeof(Counters), cudaHostAllocPortable) == cudaSuccess) {
      g_pin_base = (Counters*)b;
      for (int i = PINNED_SLOTS - 1; i >= 0; --i) g_pin_free.push_back(i);
    } else {
      cudaGetLastError();   // no pinned buffer: every plan reads into pageable memory
    }
  }
  if (!g_pin_base || g_pin_free.empty()) return nullptr;
  const int i = g_pin_free.back();
  g_pin_free.pop_back();
  return g_pin_base + i;
}

void pinned_give(Counters* c) {
  if (!c) return;
  std::lock_guard<std::mutex> lock(g_pin_mu);
  g_pin_free.push_back((int)(c - g_pin_base));
}

}  // namespace

struct spgemm_plan_s {
  DevCsr A{}, B{};
  Limits lim{};
  int nslabs = 0;
  int values_mode = 0;          // merge classes: 0 automatic, 1 values read from B, 2 staged
  Layout L{};
  unsigned char* ws = nullptr;
  Counters* ctr = nullptr;
  Counters h{};                 // host copy of the counters after the last synchronising call
  int state = 0;                // 1 planned, 2 symbolic done
  int32_t* C_rp = nullptr;
  int32_t* C_col = nullptr;     // set by numeric / compute (the backward reads C's structure)
  bool slabs_clean = false;
  const void* transposed_ws = nullptr;   // backward workspace holding A's transpose, once built
  const void* replay_map = nullptr;      // position map recorded for this plan's C, if any
  cudaEvent_t ev_start = nullptr, ev_stop = nullptr;   // optional, recorded around the compute kernels
  Counters* pinned = nullptr;   // this plan's slot of the pinned read-back buffer, if it got one
  ~spgemm_plan_s() { pinned_give(pinned); }
};

namespace {
// Read the device counters into p->h: enqueue the copy, synchronise the stream.
cudaError_t read_counters(spgemm_plan_s* p, cudaStream_t s) {
  Counters* dst = p->pinned ? p->pinned : &p->h;
  cudaMemcpyAsync(dst, p->ctr, sizeof(Counters), cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess && p->pinned) p->h = *p->pinned;
  return e;
}
}  // namespace

extern "C" {

int32_t spgemm_version(void) { return 10000; }

const char* spgemm_error_string(int code) {
  switch (code) {
    case SPGEMM_OK: return "ok";
    case SPGEMM_ERR_INVALID: return "invalid argument or input matrix";
    case SPGEMM_ERR_ALLOC: return "workspace too small";
    case SPGEMM_ERR_OVERFLOW: return "count exceeds int32 (nnz(C) or a row's products)";
    case SPGEMM_ERR_TABLE_FULL: return "hash table full";
    case SPGEMM_ERR_CUDA: return "CUDA error";
    case SPGEMM_ERR_TIMEOUT: return "bounded device wait timed out";
    case SPGEMM_ERR_STATE: return "calls out of order";
    case SPGEMM_ERR_UNSORTED: return "reserved: unsorted input";
    case SPGEMM_ERR_MISMATCH: return "structure changed between symbolic and numeric";
    case SPGEMM_ERR_SCRATCH_LIMIT: return "size exceeds the fixed scratch of a no-allocation entry point";
    default: return "unknown status";
  }
}

spgemm_status_t spgemm_workspace_size(const spgemm_csr_t* A, const spgemm_csr_t* B, const spgemm_options_t* opt,
                                      size_t* bytes) {
  if (!bytes || !desc_ok(A) || !desc_ok(B) || A->cols != B->rows) return SPGEMM_ERR_INVALID;
  *bytes = layout(A->rows, B->cols, slabs_from(opt)).total;
  return SPGEMM_OK;
}

spgemm_status_t spgemm_plan(spgemm_plan_t* out, const spgemm_csr_t* A, const spgemm_csr_t* B,
                            const spgemm_options_t* opt, void* workspace, size_t workspace_bytes, void* stream) {
  if (!out) return SPGEMM_ERR_INVALID;
  *out = nullptr;
  if (!desc_ok(A) || !desc_ok(B) || A->cols != B->rows) return SPGEMM_ERR_INVALID;
  if (!workspace || ((uintptr_t)workspace % ALIGN) != 0) return SPGEMM_ERR_INVALID;
  const int nslabs = slabs_from(opt);
  const Layout L = layout(A->rows, B->cols, nslabs);
  if (workspace_bytes < L.total) return SPGEMM_ERR_ALLOC;
  cudaStream_t s = (cudaStream_t)stream;
  spgemm_plan_s* p = new (std::nothrow) spgemm_plan_s();
  if (!p) return SPGEMM_ERR_ALLOC;
  p->pinned = pinned_take();
  p->A = to_dev(*A);
  p->B = to_dev(*B);
  p->lim = limits_from(opt);
  p->nslabs = nslabs;
  p->values_mode = (opt && opt->merge_values >= 0 && opt->merge_values <= 2) ? opt->merge_values : 0;
  p->L = L;
  p->ws = (unsigned char*)workspace;
  p->ctr = (Counters*)(p->ws + L.ctr);
  cudaMemsetAsync(p->ctr, 0, sizeof(Counters), s);
  if (opt && opt->validate) {
    const int grid = num_sms() * 4;
    if (p->A.rp) k_validate<<<grid, 256, 0, s>>>(p->A, p->ctr);
    if (p->B.rp) k_validate<<<grid, 256, 0, s>>>(p->B, p->ctr);
  }
  int* lists[NUM_CLS] = {nullptr, nullptr, (int*)(p->ws + L.list_w), (int*)(p->ws + L.list_b),
                         (int*)(p->ws + L.list_g)};
  launch_bin(p->A, p->B, p->lim, p->ws + L.cls, lists, p->ctr, s);
  if (read_counters(p, s) != cudaSuccess) {
    delete p;
    return SPGEMM_ERR_CUDA;
  }
  const spgemm_status_t st = status_from_bits(p->h.status);
  if (st != SPGEMM_OK) {
    delete p;
    return st;
  }
  p->state = 1;
  *out = p;
  return SPGEMM_OK;
}

spgemm_status_t spgemm_symbolic(spgemm_plan_t p, int32_t* C_row_ptr, int64_t* nnz_c, void* stream) {
  if (!p || p->state < 1) return SPGEMM_ERR_STATE;
  if (!C_row_ptr || !nnz_c) return SPGEMM_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  const Layout& L = p->L;
  const int m = p->A.rows;
  // scan ticket and tile states start from zero
  cudaMemsetAsync(&p->ctr->ticket, 0, sizeof(unsigned), s);
  cudaMemsetAsync(p->ws + L.scan, 0, scan_tile_state_bytes((long long)m + 1), s);
  const int* cnt = p->h.count;
  uint8_t* cls = p->ws + L.cls;
  if (cnt[CLS_G] > 0 && !p->slabs_clean) {
    cudaMemsetAsync(p->ws + L.slabs, 0, (size_t)p->nslabs * dense_slab_bytes(p->B.cols), s);
    p->slabs_clean = true;
  }
  const int wide = p->h.max_u_merge > 32;
  if (cnt[CLS_M1] + cnt[CLS_M2] > 0) launch_merge_symbolic(wide, p->A, p->B, cls, C_row_ptr, p->ctr, s);
  if (cnt[CLS_W] > 0)
    launch_hash_symbolic(CLS_W, p->A, p->B, (const int*)(p->ws + L.list_w), cnt[CLS_W], C_row_ptr, p->ctr, s, p->h.max_u_w);
  if (cnt[CLS_B] > 0)
    launch_hash_symbolic(CLS_B, p->A, p->B, (const int*)(p->ws + L.list_b), cnt[CLS_B], C_row_ptr, p->ctr, s);
  if (cnt[CLS_G] > 0)
    launch_dense_symbolic(p->A, p->B, (const int*)(p->ws + L.list_g), cnt[CLS_G], p->ws + L.slabs, p->nslabs,
                          C_row_ptr, p->ctr, s);
  launch_scan(C_row_ptr, (long long)m + 1, (unsigned long long*)(p->ws + L.scan), p->ctr, &p->ctr->nnzC, s);
  // until a structure pass succeeds, no numeric pass may use a row pointer
  p->state = 1;
  if (read_counters(p, s) != cudaSuccess) return SPGEMM_ERR_CUDA;
  const spgemm_status_t st = status_from_bits(p->h.status);
  if (st != SPGEMM_OK) return st;
  p->C_rp = C_row_ptr;
  p->state = 2;
  *nnz_c = p->h.nnzC;
  return SPGEMM_OK;
}

spgemm_status_t spgemm_numeric(spgemm_plan_t p, const double* A_val, const double* B_val, int32_t* C_col,
                               double* C_val, void* stream) {
  if (!p || p->state < 2) return SPGEMM_ERR_STATE;
  if ((!A_val && p->A.nnz > 0) || (!B_val && p->B.nnz > 0)) return SPGEMM_ERR_INVALID;
  if ((!C_col || !C_val) && p->h.nnzC > 0) return SPGEMM_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  DevCsr A = p->A, B = p->B;
  A.val = A_val;
  B.val = B_val;
  const Layout& L = p->L;
  const int* cnt = p->h.count;
  uint8_t* cls = p->ws + L.cls;
  const int wide = p->h.max_u_merge > 32;
  if (p->ev_start) cudaEventRecord(p->ev_start, s);
  if (cnt[CLS_M1] + cnt[CLS_M2] > 0)
    launch_merge_numeric(wide, p->values_mode, A, B, cls, p->C_rp, C_col, C_val, p->ctr, s);
  if (cnt[CLS_W] > 0)
    launch_hash_numeric(CLS_W, A, B, (const int*)(p->ws + L.list_w), cnt[CLS_W], p->C_rp, C_col, C_val, p->ctr, s, p->h.max_u_w);
  if (cnt[CLS_B] > 0)
    launch_hash_numeric(CLS_B, A, B, (const int*)(p->ws + L.list_b), cnt[CLS_B], p->C_rp, C_col, C_val, p->ctr, s);
  if (cnt[CLS_G] > 0)
    launch_dense_numeric(A, B, (const int*)(p->ws + L.list_g), cnt[CLS_G], p->ws + L.slabs, p->nslabs, p->C_rp,
                         C_col, C_val, p->ctr, s);
  if (p->ev_stop) cudaEventRecord(p->ev_stop, s);
  if (cudaGetLastError() != cudaSuccess) return SPGEMM_ERR_CUDA;
  p->C_col = C_col;
  return SPGEMM_OK;
}

static spgemm_status_t compute_enqueue(spgemm_plan_t p, const double* A_val, const double* B_val, int32_t* C_row_ptr,
                                       int32_t* C_col, double* C_val, int64_t capacity, cudaStream_t s) {
  if (!p || p->state < 1) return SPGEMM_ERR_STATE;
  if (!C_row_ptr || capacity < 0) return SPGEMM_ERR_INVALID;
  if ((!A_val && p->A.nnz > 0) || (!B_val && p->B.nnz > 0)) return SPGEMM_ERR_INVALID;
  if ((!C_col || !C_val) && capacity > 0) return SPGEMM_ERR_INVALID;
  const Layout& L = p->L;
  const int m = p->A.rows;
  DevCsr A = p->A, B = p->B;
  A.val = A_val;
  B.val = B_val;
  if (m == 0) {
    cudaMemsetAsync(C_row_ptr, 0, sizeof(int32_t), s);
    cudaMemsetAsync(&p->ctr->nnzC, 0, sizeof(long long), s);
  } else {
    const int* cnt = p->h.count;
    uint8_t* cls = p->ws + L.cls;
    cudaMemsetAsync(&p->ctr->ticket, 0, sizeof(unsigned), s);
    cudaMemsetAsync(p->ws + L.fused, 0, fused_tile_state_bytes(m), s);
    // rows of the hash and dense classes: counts first (the fused pass places every row)
    if (cnt[CLS_G] > 0 && !p->slabs_clean) {
      cudaMemsetAsync(p->ws + L.slabs, 0, (size_t)p->nslabs * dense_slab_bytes(p->B.cols), s);
      p->slabs_clean = true;
    }
    if (p->ev_start) cudaEventRecord(p->ev_start, s);
    if (cnt[CLS_W] > 0)
      launch_hash_symbolic(CLS_W, A, B, (const int*)(p->ws + L.list_w), cnt[CLS_W], C_row_ptr, p->ctr, s, p->h.max_u_w);
    if (cnt[CLS_B] > 0)
      launch_hash_symbolic(CLS_B, A, B, (const int*)(p->ws + L.list_b), cnt[CLS_B], C_row_ptr, p->ctr, s);
    if (cnt[CLS_G] > 0)
      launch_dense_symbolic(A, B, (const int*)(p->ws + L.list_g), cnt[CLS_G], p->ws + L.slabs, p->nslabs,
                            C_row_ptr, p->ctr, s);
    const int wide = p->h.max_u_merge > 32;
    launch_merge_fused(wide, p->values_mode, A, B, cls, C_row_ptr, C_col, C_val, capacity,
                       (unsigned long long*)(p->ws + L.fused), p->ctr, s);
    if (cnt[CLS_W] > 0)
      launch_hash_numeric(CLS_W, A, B, (const int*)(p->ws + L.list_w), cnt[CLS_W], C_row_ptr, C_col, C_val, p->ctr, s, p->h.max_u_w);
    if (cnt[CLS_B] > 0)
      launch_hash_numeric(CLS_B, A, B, (const int*)(p->ws + L.list_b), cnt[CLS_B], C_row_ptr, C_col, C_val, p->ctr, s);
    if (cnt[CLS_G] > 0)
      launch_dense_numeric(A, B, (const int*)(p->ws + L.list_g), cnt[CLS_G], p->ws + L.slabs, p->nslabs, C_row_ptr,
                           C_col, C_val, p->ctr, s);
    if (p->ev_stop) cudaEventRecord(p->ev_stop, s);
  }
  if (cudaGetLastError() != cudaSuccess) return SPGEMM_ERR_CUDA;
  p->C_rp = C_row_ptr;
  p->C_col = C_col;
  p->state = 2;
  return SPGEMM_OK;
}

spgemm_status_t spgemm_compute(spgemm_plan_t p, const double* A_val, const double* B_val, int32_t* C_row_ptr,
                               int32_t* C_col, double* C_val, int64_t capacity, int64_t* nnz_c, void* stream) {
  if (!nnz_c) return SPGEMM_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  const spgemm_status_t e = compute_enqueue(p, A_val, B_val, C_row_ptr, C_col, C_val, capacity, s);
  if (e != SPGEMM_OK) return e;
  if (read_counters(p, s) != cudaSuccess) { p->state = 1; return SPGEMM_ERR_CUDA; }
  const spgemm_status_t st = status_from_bits(p->h.status);
  if (st != SPGEMM_OK) { p->state = 1; return st; }
  *nnz_c = p->h.nnzC;
  return SPGEMM_OK;
}

spgemm_status_t spgemm_compute_async(spgemm_plan_t p, const double* A_val, const double* B_val, int32_t* C_row_ptr,
                                     int32_t* C_col, double* C_val, int64_t capacity, int64_t* nnz_c_device,
                                     void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const spgemm_status_t e = compute_enqueue(p, A_val, B_val, C_row_ptr, C_col, C_val, capacity, s);
  if (e != SPGEMM_OK) return e;
  if (nnz_c_device) cudaMemcpyAsync(nnz_c_device, &p->ctr->nnzC, sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
  if (cudaGetLastError() != cudaSuccess) return SPGEMM_ERR_CUDA;
  return SPGEMM_OK;
}

spgemm_status_t spgemm_replay_size(spgemm_plan_t p, size_t* bytes) {
  if (!p || p->state < 1) return SPGEMM_ERR_STATE;
  if (!bytes) return SPGEMM_ERR_INVALID;
  *bytes = replay_map_bytes(p->A.rows, p->h.max_u_merge);
  return SPGEMM_OK;
}

spgemm_status_t spgemm_replay_record(spgemm_plan_t p, const int32_t* C_col, void* map, size_t map_bytes,
                                     void* stream) {
  if (!p || p->state < 2 || !p->C_rp) return SPGEMM_ERR_STATE;
  if (!map || ((uintptr_t)map % ALIGN) != 0 || (!C_col && p->h.nnzC > 0)) return SPGEMM_ERR_INVALID;
  if (map_bytes < replay_map_bytes(p->A.rows, p->h.max_u_merge)) return SPGEMM_ERR_ALLOC;
  cudaStream_t s = (cudaStream_t)stream;
  p->replay_map = nullptr;
  if (p->A.rows > 0)
    launch_replay_record(p->A, p->B, p->ws + p->L.cls, p->C_rp, C_col, map,
                         (unsigned long long*)(p->ws + p->L.scan), p->ctr, s);
  if (read_counters(p, s) != cudaSuccess) return SPGEMM_ERR_CUDA;
  const spgemm_status_t st = status_from_bits(p->h.status);
  if (st != SPGEMM_OK) return st;
  p->replay_map = map;
  return SPGEMM_OK;
}

spgemm_status_t spgemm_replay(spgemm_plan_t p, const double* A_val, const double* B_val, const void* map,
                              int32_t* C_col, double* C_val, void* stream) {
  if (!p || p->state < 2 || !map || map != p->replay_map) return SPGEMM_ERR_STATE;
  if ((!A_val && p->A.nnz > 0) || (!B_val && p->B.nnz > 0)) return SPGEMM_ERR_INVALID;
  if ((!C_col || !C_val) && p->h.nnzC > 0) return SPGEMM_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  DevCsr A = p->A, B = p->B;
  A.val = A_val;
  B.val = B_val;
  const Layout& L = p->L;
  const int* cnt = p->h.count;
  if (p->ev_start) cudaEventRecord(p->ev_start, s);
  if (cnt[CLS_M1] + cnt[CLS_M2] > 0) launch_replay(p->h.max_u_merge > 32, A, B, p->ws + L.cls, p->C_rp, map, C_val, s);
  if (cnt[CLS_W] > 0)
    launch_hash_numeric(CLS_W, A, B, (const int*)(p->ws + L.list_w), cnt[CLS_W], p->C_rp, C_col, C_val, p->ctr, s, p->h.max_u_w);
  if (cnt[CLS_B] > 0)
    launch_hash_numeric(CLS_B, A, B, (const int*)(p->ws + L.list_b), cnt[CLS_B], p->C_rp, C_col, C_val, p->ctr, s);
  if (cnt[CLS_G] > 0)
    launch_dense_numeric(A, B, (const int*)(p->ws + L.list_g), cnt[CLS_G], p->ws + L.slabs, p->nslabs, p->C_rp,
                         C_col, C_val, p->ctr, s);
  if (p->ev_stop) cudaEventRecord(p->ev_stop, s);
  if (cudaGetLastError() != cudaSuccess) return SPGEMM_ERR_CUDA;
  return SPGEMM_OK;
}

spgemm_status_t spgemm_backward_workspace_size(const spgemm_csr_t* A, const spgemm_csr_t* B, size_t* bytes) {
  if (!bytes || !desc_ok(A) || !desc_ok(B) || A->cols != B->rows) return SPGEMM_ERR_INVALID;
  *bytes = transpose_bytes(A->cols, A->nnz);
  return SPGEMM_OK;
}

spgemm_status_t spgemm_backward(spgemm_plan_t p, const double* A_val, const double* B_val, const double* dC_val,
                                double* dA_val, double* dB_val, void* workspace, size_t workspace_bytes,
                                void* stream) {
  if (!p || p->state < 2 || !p->C_rp || (!p->C_col && p->h.nnzC > 0)) return SPGEMM_ERR_STATE;
  if (!dC_val && p->h.nnzC > 0) return SPGEMM_ERR_INVALID;
  if (dA_val && !B_val && p->B.nnz > 0) return SPGEMM_ERR_INVALID;
  if (dB_val) {
    if (!A_val && p->A.nnz > 0) return SPGEMM_ERR_INVALID;
    if (!workspace || workspace_bytes < transpose_bytes(p->A.cols, p->A.nnz) || ((uintptr_t)workspace % ALIGN) != 0)
      return SPGEMM_ERR_ALLOC;
  }
  cudaStream_t s = (cudaStream_t)stream;
  DevCsr A = p->A, B = p->B;
  A.val = A_val;
  B.val = B_val;
  if (p->ev_start) cudaEventRecord(p->ev_start, s);
  if (dA_val) launch_grad_a(A, B, p->C_rp, p->C_col, dC_val, dA_val, p->ctr, s);
  if (dB_val) {
    if (p->transposed_ws != workspace) {
      launch_transpose(A, workspace, p->ctr, s);
      p->transposed_ws = workspace;
    }
    launch_grad_b(A, B, workspace, p->C_rp, p->C_col, dC_val, dB_val, p->ctr, s);
  }
  if (p->ev_stop) cudaEventRecord(p->ev_stop, s);
  if (cudaGetLastError() != cudaSuccess) return SPGEMM_ERR_CUDA;
  return SPGEMM_OK;
}

spgemm_status_t spgemm_status(spgemm_plan_t p, void* stream) {
  if (!p) return SPGEMM_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  if (read_counters(p, s) != cudaSuccess) return SPGEMM_ERR_CUDA;
  return status_from_bits(p->h.status);
}

spgemm_status_t spgemm_plan_info(spgemm_plan_t p, spgemm_info_t* info) {
  if (!p || !info) return SPGEMM_ERR_INVALID;
  std::memset(info, 0, sizeof(*info));
  info->products = (int64_t)p->h.F;
  info->nnz_c = p->state >= 2 ? p->h.nnzC : -1;
  info->max_row_products = p->h.max_u;
  for (int i = 0; i < NUM_CLS; ++i) info->rows_per_class[i] = p->h.count[i];
  return SPGEMM_OK;
}

spgemm_status_t spgemm_plan_set_events(spgemm_plan_t p, void* start_event, void* stop_event) {
  if (!p || ((start_event == nullptr) != (stop_event == nullptr))) return SPGEMM_ERR_INVALID;
  p->ev_start = (cudaEvent_t)start_event;
  p->ev_stop = (cudaEvent_t)stop_event;
  return SPGEMM_OK;
}

spgemm_status_t spgemm_free(spgemm_plan_t p) {
  delete p;
  return SPGEMM_OK;
}

}  // extern "C"
