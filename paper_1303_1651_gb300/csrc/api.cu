// C ABI of the SpGEMM library: plan object, workspace layout, call sequencing.
// See include/spgemm_gb300.h for the contract of every entry point.
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "internal.h"
#include "spgemm_gb300.h"

using namespace spg;

namespace {

constexpr size_t ALIGN = 256;
inline size_t up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

// Workspace pieces.  conv/cval/cgrad exist for an operand given in compressed columns: its
// structure converted to rows (row pointers, column indices and, per entry, its position in the
// given arrays: the transpose's output), its values gathered into that order for each call, and
// its gradient before it is scattered back (spgemm_backward).
struct Layout {
  size_t ctr, cls, list_w, list_b, list_g, scan, fused, slabs, total;
  size_t conv[2], cval[2], cgrad[2];
};

Layout layout(const spgemm_csr_t& A, const spgemm_csr_t& B, int nslabs, const bool csc[2]) {
  const int m = A.rows;
  Layout L{};
  size_t o = 0;
  L.ctr = o; o += up(sizeof(Counters));
  L.cls = o; o += up((size_t)std::max(m, 1));
  L.list_w = o; o += up(4 * (size_t)std::max(m, 1));
  L.list_b = o; o += up(4 * (size_t)std::max(m, 1));
  L.list_g = o; o += up(4 * (size_t)std::max(m, 1));
  L.scan = o; o += up(scan_tile_state_bytes((long long)m + 1) + 64);
  L.fused = o; o += up(fused_tile_state_bytes(m) + 64);
  L.slabs = o; o += (size_t)nslabs * dense_slab_bytes(B.cols);
  const spgemm_csr_t* M[2] = {&A, &B};
  for (int i = 0; i < 2; ++i) {
    if (!csc[i]) continue;
    const size_t n = (size_t)std::max(M[i]->nnz, (int64_t)1);
    L.conv[i] = o; o += up(transpose_bytes(M[i]->rows, M[i]->nnz));
    L.cval[i] = o; o += up(8 * n);
    L.cgrad[i] = o; o += up(8 * n);
  }
  L.total = o;
  return L;
}

Limits limits_from(const spgemm_options_t* o) {
  // Class W takes rows of up to 256 products by default: longer rows run faster in class B's
  // bit-vector blocks (measured on the batched workload and on the 0.1 % fill rows).
  Limits l{8, 32, 64, 256, 0};
  if (o) {
    if (o->merge_max_k > 0) l.merge_k = std::min(o->merge_max_k, 8);
    if (o->m1_max_u > 0) l.m1_u = std::min(o->m1_max_u, 32);
    if (o->m2_max_u > 0) l.m2_u = std::min(o->m2_max_u, 64);
    if (o->warp_max_u > 0) l.warp_u = std::min(o->warp_max_u, 1024);
    if (o->block_max_u > 0) l.block_u = o->block_max_u;   // clamped by block_limit
    if (o->m1_max_u < 0) l.m1_u = -1;     // negative: class disabled (testing hook)
    if (o->m2_max_u < 0) l.m2_u = -1;
    if (o->warp_max_u < 0) l.warp_u = -1;
    if (o->block_max_u < 0) l.block_u = -1;
  }
  l.m2_u = std::max(l.m2_u, l.m1_u);
  return l;
}

// Dense accumulators of class G, one per CTA: the caller's number, else as many as fit 128 MB
// (at least 2, at most one per SM).
WarpOrder wopts_from(const spgemm_options_t* o) {
  WarpOrder w;
  if (o && o->warp_bitvec_ratio > 0) w.bitvec_ratio = std::min(o->warp_bitvec_ratio, 128);
  if (o && o->warp_order >= 0 && o->warp_order <= 3) w.order = o->warp_order;
  return w;
}

// Class B takes up to BB_MAX_U products per row (the sums of its bit-vector windows).
void block_limit(Limits& l) {
  if (l.block_u > 0) l.block_u = std::min(l.block_u, BB_MAX_U);
  else if (l.block_u == 0) l.block_u = BB_MAX_U;
}

int slabs_from(const spgemm_options_t* o, int ncols) {
  if (o && o->dense_slabs > 0) return o->dense_slabs;
  const size_t fit = ((size_t)128 << 20) / dense_slab_bytes(ncols);
  return (int)std::max<size_t>(2, std::min<size_t>(fit, (size_t)num_sms()));
}

bool csc_of(const spgemm_options_t* o, int i) { return o && (i == 0 ? o->a_storage : o->b_storage) == 1; }

bool storage_ok(const spgemm_options_t* o) {
  return !o || ((o->a_storage == 0 || o->a_storage == 1) && (o->b_storage == 0 || o->b_storage == 1));
}

// A descriptor in compressed rows, or (csc) in compressed columns: then row_ptr has cols + 1 entries.
bool desc_ok(const spgemm_csr_t* M, bool csc = false) {
  if (!M || M->rows < 0 || M->cols < 0 || M->nnz < 0 || M->nnz > INT32_MAX) return false;
  if (!M->row_ptr && (csc ? M->cols : M->rows) > 0) return false;
  if (!M->col_idx && M->nnz > 0) return false;
  if (M->nnz > 0 && (M->rows == 0 || M->cols == 0)) return false;   // entries need a row and a column
  return true;
}

DevCsr to_dev(const spgemm_csr_t& M) {
  return DevCsr{M.rows, M.cols, (long long)M.nnz, M.row_ptr, M.col_idx, M.val};
}

// Host-side fault injection for tests of the error paths, read from the environment at each call:
// SPGEMM_FAULT=alloc makes spgemm_plan report a workspace that is too small; SPGEMM_FAULT=nnz_overflow
// makes spgemm_symbolic report nnz(C) past INT32_MAX and the single-pass product run with no room
// for C (its device overflow path).  Nothing is injected on the device.
bool fault_is(const char* name) {
  const char* f = std::getenv("SPGEMM_FAULT");
  return f && std::strcmp(f, name) == 0;
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
  DevCsr A{}, B{};              // in compressed rows (converted in the workspace when given by columns)
  bool csc[2] = {false, false}; // A, B given in compressed columns
  const int* perm[2] = {nullptr, nullptr};   // converted entry -> position in the given arrays
  double* cval[2] = {nullptr, nullptr};      // values gathered into row order
  double* cgrad[2] = {nullptr, nullptr};     // gradients in row order, before the scatter
  int spin_limit = 0;           // look-back bound of the single-pass product (0: default)
  int drop_tile = -1;           // testing: a fused tile that publishes nothing (-1: none)
  Limits lim{};
  int nslabs = 0;
  int values_mode = 0;          // merge classes: 0 automatic, 1 values read from B, 2 staged
  WarpOrder wopt{};             // ordering of the class-W rows
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

namespace {
// Values of A and B as the kernels read them: the caller's arrays, or for an operand given by
// columns its values gathered into the converted row order.
void prepare_values(spgemm_plan_s* p, const double* A_val, const double* B_val, DevCsr& A, DevCsr& B,
                    cudaStream_t s) {
  A = p->A;
  B = p->B;
  A.val = A_val;
  B.val = B_val;
  if (p->csc[0] && A_val) { launch_gather(p->perm[0], A_val, p->cval[0], p->A.nnz, s); A.val = p->cval[0]; }
  if (p->csc[1] && B_val) { launch_gather(p->perm[1], B_val, p->cval[1], p->B.nnz, s); B.val = p->cval[1]; }
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
  if (!bytes || !storage_ok(opt)) return SPGEMM_ERR_INVALID;
  const bool csc[2] = {csc_of(opt, 0), csc_of(opt, 1)};
  if (!desc_ok(A, csc[0]) || !desc_ok(B, csc[1]) || A->cols != B->rows) return SPGEMM_ERR_INVALID;
  *bytes = layout(*A, *B, slabs_from(opt, B->cols), csc).total;
  return SPGEMM_OK;
}

// Checks of spgemm_plan's arguments (host only); on success fills csc, nslabs and the layout.
static spgemm_status_t plan_args(const spgemm_csr_t* A, const spgemm_csr_t* B, const spgemm_options_t* opt,
                                 void* workspace, size_t workspace_bytes, bool csc[2], int* nslabs, Layout* L) {
  if (!storage_ok(opt)) return SPGEMM_ERR_INVALID;
  csc[0] = csc_of(opt, 0);
  csc[1] = csc_of(opt, 1);
  if (!desc_ok(A, csc[0]) || !desc_ok(B, csc[1]) || A->cols != B->rows) return SPGEMM_ERR_INVALID;
  if (!workspace || ((uintptr_t)workspace % ALIGN) != 0) return SPGEMM_ERR_INVALID;
  *nslabs = slabs_from(opt, B->cols);
  *L = layout(*A, *B, *nslabs, csc);
  if (workspace_bytes < L->total || fault_is("alloc")) return SPGEMM_ERR_ALLOC;
  return SPGEMM_OK;
}

// Enqueue the plan's device work (conversion of operands given by columns, optional validation,
// binning) on s; the counters stay on the device.
// zero_fused: the binning kernel also clears the single-pass product's tile states.
static void plan_enqueue(spgemm_plan_s* p, const spgemm_csr_t* A, const spgemm_csr_t* B, const spgemm_options_t* opt,
                         void* workspace, const bool csc[2], int nslabs, const Layout& L, cudaStream_t s,
                         bool zero_fused = false) {
  p->A = to_dev(*A);
  p->B = to_dev(*B);
  p->lim = limits_from(opt);
  block_limit(p->lim);
  p->nslabs = nslabs;
  p->values_mode = (opt && opt->merge_values >= 0 && opt->merge_values <= 2) ? opt->merge_values : 0;
  p->wopt = wopts_from(opt);
  p->spin_limit = (opt && opt->debug_spin_limit > 0) ? opt->debug_spin_limit : 0;
  p->drop_tile = (opt && opt->debug_drop_tile > 0) ? opt->debug_drop_tile - 1 : -1;
  p->L = L;
  p->ws = (unsigned char*)workspace;
  p->ctr = (Counters*)(p->ws + L.ctr);
  cudaMemsetAsync(p->ctr, 0, sizeof(Counters), s);
  // An operand given by columns is first read as the compressed rows of its transpose (the given
  // arrays as they are), checked in that form, and transposed into the workspace: its rows in
  // CSR, with each entry's position in the given arrays (Section IV-A's storage-order conversion).
  DevCsr given[2] = {p->A, p->B};
  for (int i = 0; i < 2; ++i) {
    if (!csc[i]) continue;
    const spgemm_csr_t* M = i == 0 ? A : B;
    given[i] = DevCsr{M->cols, M->rows, (long long)M->nnz, M->row_ptr, M->col_idx, nullptr};
  }
  if (opt && opt->validate) {
    const int grid = num_sms() * 4;
    if (given[0].rp) k_validate<<<grid, 256, 0, s>>>(given[0], p->ctr);
    if (given[1].rp) k_validate<<<grid, 256, 0, s>>>(given[1], p->ctr);
  }
  for (int i = 0; i < 2; ++i) {
    if (!csc[i]) continue;
    DevCsr& X = i == 0 ? p->A : p->B;
    unsigned char* conv = p->ws + L.conv[i];
    launch_transpose(given[i], conv, p->ctr, s);
    TransposeView tv = transpose_view(conv, X.rows, X.nnz);
    X.rp = tv.T_cp;
    X.col = tv.T_row;
    X.val = nullptr;
    p->csc[i] = true;
    p->perm[i] = tv.T_src;
    p->cval[i] = (double*)(p->ws + L.cval[i]);
    p->cgrad[i] = (double*)(p->ws + L.cgrad[i]);
  }
  int* lists[NUM_CLS] = {nullptr, nullptr, (int*)(p->ws + L.list_w), (int*)(p->ws + L.list_b),
                         (int*)(p->ws + L.list_g)};
  launch_bin(p->A, p->B, p->lim, p->ws + L.cls, lists, p->ctr, s,
             zero_fused ? (unsigned long long*)(p->ws + L.fused) : nullptr,
             (long long)(fused_tile_state_bytes(p->A.rows) / sizeof(unsigned long long)));
}

spgemm_status_t spgemm_plan(spgemm_plan_t* out, const spgemm_csr_t* A, const spgemm_csr_t* B,
                            const spgemm_options_t* opt, void* workspace, size_t workspace_bytes, void* stream) {
  if (!out) return SPGEMM_ERR_INVALID;
  *out = nullptr;
  bool csc[2];
  int nslabs = 0;
  Layout L{};
  const spgemm_status_t a = plan_args(A, B, opt, workspace, workspace_bytes, csc, &nslabs, &L);
  if (a != SPGEMM_OK) return a;
  cudaStream_t s = (cudaStream_t)stream;
  spgemm_plan_s* p = new (std::nothrow) spgemm_plan_s();
  if (!p) return SPGEMM_ERR_ALLOC;
  p->pinned = pinned_take();
  plan_enqueue(p, A, B, opt, workspace, csc, nslabs, L, s);
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

// spgemm_multiply: binning and the single-pass product enqueued together.  The host does not know
// the row classes yet, so every class kernel is launched over an upper bound of rows and reads its
// row count on the device (a class with no rows costs an empty launch), the dense slabs are cleared
// by their kernel, and both tile forms of the fused pass are launched (the one the binning did not
// choose returns at once).  The counters are read back once, at the end.
// Side streams and events of spgemm_multiply_async, one set per host thread and device (calls from
// several threads never share an event).  The class kernels that do not depend on one another (the
// three structure passes, the two tile forms, the three value passes) go to separate streams joined
// by events, so a CUDA graph captured from the call holds them side by side instead of in a chain.
// Created on the thread's first call on a device and kept until the thread ends.
struct ForkSet {
  cudaStream_t side[2] = {nullptr, nullptr};
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  bool ok = false;
  ForkSet() = default;
  ForkSet(const ForkSet&) = delete;
  ForkSet& operator=(const ForkSet&) = delete;
  ~ForkSet() {
    for (cudaEvent_t e : ev) if (e) cudaEventDestroy(e);
    for (cudaStream_t t : side) if (t) cudaStreamDestroy(t);
  }
};

static ForkSet* fork_set() {
  thread_local std::map<int, ForkSet> sets;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  ForkSet& f = sets[dev];
  if (!f.ok) {
    bool good = true;
    for (cudaStream_t& t : f.side)
      if (!t) good = good && cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking) == cudaSuccess;
    for (cudaEvent_t& e : f.ev)
      if (!e) good = good && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    f.ok = good;
    if (!good) return nullptr;   // the call then runs on one stream
  }
  return &f;
}

// n side streams wait for the work enqueued on s so far (fork), or s waits for them (join).
static void fork_to(ForkSet* f, int n, cudaStream_t s) {
  if (!f) return;
  cudaEventRecord(f->ev[0], s);
  for (int i = 0; i < n; ++i) cudaStreamWaitEvent(f->side[i], f->ev[0], 0);
}
static void join_from(ForkSet* f, int n, cudaStream_t s) {
  if (!f) return;
  for (int i = 0; i < n; ++i) {
    cudaEventRecord(f->ev[1 + i], f->side[i]);
    cudaStreamWaitEvent(s, f->ev[1 + i], 0);
  }
}

// Enqueue spgemm_multiply's work on s (p: a plan object on the caller's stack, holding no pinned
// slot unless the caller gave it one).  Host checks only; nothing is read back.  fork: independent
// class kernels on side streams (above).
static spgemm_status_t multiply_enqueue(spgemm_plan_s& p, const spgemm_csr_t* A, const spgemm_csr_t* B,
                                        const spgemm_options_t* opt, void* workspace, size_t workspace_bytes,
                                        int32_t* C_row_ptr, int32_t* C_col, double* C_val, int64_t capacity,
                                        cudaStream_t s, bool fork = false) {
  if (!C_row_ptr || capacity < 0) return SPGEMM_ERR_INVALID;
  if ((!C_col || !C_val) && capacity > 0) return SPGEMM_ERR_INVALID;
  bool csc[2];
  int nslabs = 0;
  Layout L{};
  const spgemm_status_t a = plan_args(A, B, opt, workspace, workspace_bytes, csc, &nslabs, &L);
  if (a != SPGEMM_OK) return a;
  if ((!A->val && A->nnz > 0) || (!B->val && B->nnz > 0)) return SPGEMM_ERR_INVALID;
  if (fault_is("nnz_overflow")) capacity = 0;
  // the fused pass's tile states and ticket are cleared by the binning kernel (after any
  // conversion of an operand given by columns, whose scan takes tickets too)
  plan_enqueue(&p, A, B, opt, workspace, csc, nslabs, L, s, true);
  const int m = p.A.rows;
  if (m == 0) {
    cudaMemsetAsync(C_row_ptr, 0, sizeof(int32_t), s);
  } else {
    DevCsr Av, Bv;
    prepare_values(&p, A->val, B->val, Av, Bv, s);
    ForkSet* f = fork ? fork_set() : nullptr;
    cudaStream_t s1 = f ? f->side[0] : s, s2 = f ? f->side[1] : s;
    const int* cnt_dev = p.ctr->count;
    const int* lw = (const int*)(p.ws + L.list_w);
    const int* lb = (const int*)(p.ws + L.list_b);
    const int* lg = (const int*)(p.ws + L.list_g);
    const Limits& lim = p.lim;
    fork_to(f, 2, s);
    if (lim.warp_u > 0)
      launch_hash_symbolic(CLS_W, Av, Bv, lw, m, C_row_ptr, p.ctr, s, lim.warp_u, p.wopt, cnt_dev + CLS_W);
    if (lim.block_u > 0) launch_hash_symbolic(CLS_B, Av, Bv, lb, m, C_row_ptr, p.ctr, s1, lim.block_u, p.wopt, cnt_dev + CLS_B);
    launch_dense_symbolic(Av, Bv, lg, m, p.ws + L.slabs, p.nslabs, C_row_ptr, p.ctr, s2, cnt_dev + CLS_G, true);
    join_from(f, 2, s);
    fork_to(f, 1, s);
    for (int wide = 0; wide < 2; ++wide)
      launch_merge_fused(wide, p.values_mode, Av, Bv, p.ws + L.cls, C_row_ptr, C_col, C_val, capacity,
                         (unsigned long long*)(p.ws + L.fused), p.ctr, wide ? s1 : s, p.spin_limit, p.drop_tile,
                         &p.ctr->max_u_merge);
    join_from(f, 1, s);
    fork_to(f, 2, s);
    if (lim.warp_u > 0)
      launch_hash_numeric(CLS_W, Av, Bv, lw, m, C_row_ptr, C_col, C_val, p.ctr, s, lim.warp_u, p.wopt, cnt_dev + CLS_W);
    if (lim.block_u > 0)
      launch_hash_numeric(CLS_B, Av, Bv, lb, m, C_row_ptr, C_col, C_val, p.ctr, s1, lim.block_u, p.wopt, cnt_dev + CLS_B);
    launch_dense_numeric(Av, Bv, lg, m, p.ws + L.slabs, p.nslabs, C_row_ptr, C_col, C_val, p.ctr, s2, cnt_dev + CLS_G);
    join_from(f, 2, s);
  }
  return cudaGetLastError() == cudaSuccess ? SPGEMM_OK : SPGEMM_ERR_CUDA;
}

spgemm_status_t spgemm_multiply(const spgemm_csr_t* A, const spgemm_csr_t* B, const spgemm_options_t* opt,
                                void* workspace, size_t workspace_bytes, int32_t* C_row_ptr, int32_t* C_col,
                                double* C_val, int64_t capacity, int64_t* nnz_c, int64_t* products, void* stream) {
  if (!nnz_c || !products) return SPGEMM_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  spgemm_plan_s p;
  p.pinned = pinned_take();
  const spgemm_status_t e = multiply_enqueue(p, A, B, opt, workspace, workspace_bytes, C_row_ptr, C_col, C_val,
                                             capacity, s);
  if (e != SPGEMM_OK) return e;
  if (read_counters(&p, s) != cudaSuccess) return SPGEMM_ERR_CUDA;
  *products = (int64_t)p.h.F;
  *nnz_c = p.A.rows == 0 ? 0 : p.h.nnzC;
  return status_from_bits(p.h.status);
}

spgemm_status_t spgemm_multiply_async(const spgemm_csr_t* A, const spgemm_csr_t* B, const spgemm_options_t* opt,
                                      void* workspace, size_t workspace_bytes, int32_t* C_row_ptr, int32_t* C_col,
                                      double* C_val, int64_t capacity, void* stream) {
  spgemm_plan_s p;
  return multiply_enqueue(p, A, B, opt, workspace, workspace_bytes, C_row_ptr, C_col, C_val, capacity,
                          (cudaStream_t)stream, true);
}

spgemm_status_t spgemm_multiply_result(const void* workspace, int64_t* nnz_c, int64_t* products, void* stream) {
  if (!workspace || ((uintptr_t)workspace % ALIGN) != 0 || !nnz_c || !products) return SPGEMM_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  spgemm_plan_s p;
  p.pinned = pinned_take();
  p.ws = (unsigned char*)const_cast<void*>(workspace);
  p.ctr = (Counters*)p.ws;   // the counters open every workspace (Layout::ctr is 0)
  if (read_counters(&p, s) != cudaSuccess) return SPGEMM_ERR_CUDA;
  *products = (int64_t)p.h.F;
  *nnz_c = p.h.nnzC;
  return status_from_bits(p.h.status);
}

spgemm_status_t spgemm_symbolic(spgemm_plan_t p, int32_t* C_row_ptr, int64_t* nnz_c, void* stream) {
  if (!p || p->state < 1) return SPGEMM_ERR_STATE;
  if (!C_row_ptr || !nnz_c) return SPGEMM_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  const Layout& L = p->L;
  const int m = p->A.rows;
  // each structure pass reports its own errors; the scan ticket and tile states start from zero
  cudaMemsetAsync(&p->ctr->status, 0, sizeof(unsigned), s);
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
    launch_hash_symbolic(CLS_W, p->A, p->B, (const int*)(p->ws + L.list_w), cnt[CLS_W], C_row_ptr, p->ctr, s, p->h.max_u_w,
                           p->wopt);
  if (cnt[CLS_B] > 0)
    launch_hash_symbolic(CLS_B, p->A, p->B, (const int*)(p->ws + L.list_b), cnt[CLS_B], C_row_ptr, p->ctr, s,
                         p->h.max_u_b);
  if (cnt[CLS_G] > 0)
    launch_dense_symbolic(p->A, p->B, (const int*)(p->ws + L.list_g), cnt[CLS_G], p->ws + L.slabs, p->nslabs,
                          C_row_ptr, p->ctr, s);
  launch_scan(C_row_ptr, (long long)m + 1, (unsigned long long*)(p->ws + L.scan), p->ctr, &p->ctr->nnzC, s);
  // until a structure pass succeeds, no numeric pass may use a row pointer
  p->state = 1;
  if (read_counters(p, s) != cudaSuccess) return SPGEMM_ERR_CUDA;
  const spgemm_status_t st = fault_is("nnz_overflow") ? SPGEMM_ERR_OVERFLOW : status_from_bits(p->h.status);
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
  const Layout& L = p->L;
  const int* cnt = p->h.count;
  uint8_t* cls = p->ws + L.cls;
  const int wide = p->h.max_u_merge > 32;
  if (p->ev_start) cudaEventRecord(p->ev_start, s);
  DevCsr A, B;
  prepare_values(p, A_val, B_val, A, B, s);
  if (cnt[CLS_M1] + cnt[CLS_M2] > 0)
    launch_merge_numeric(wide, p->values_mode, A, B, cls, p->C_rp, C_col, C_val, p->ctr, s);
  if (cnt[CLS_W] > 0)
    launch_hash_numeric(CLS_W, A, B, (const int*)(p->ws + L.list_w), cnt[CLS_W], p->C_rp, C_col, C_val, p->ctr, s, p->h.max_u_w,
                        p->wopt);
  if (cnt[CLS_B] > 0)
    launch_hash_numeric(CLS_B, A, B, (const int*)(p->ws + L.list_b), cnt[CLS_B], p->C_rp, C_col, C_val, p->ctr, s,
                        p->h.max_u_b);
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
  if (fault_is("nnz_overflow")) capacity = 0;
  const Layout& L = p->L;
  const int m = p->A.rows;
  DevCsr A = p->A, B = p->B;
  cudaMemsetAsync(&p->ctr->status, 0, sizeof(unsigned), s);   // each structure pass reports its own errors
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
    prepare_values(p, A_val, B_val, A, B, s);
    if (cnt[CLS_W] > 0)
      launch_hash_symbolic(CLS_W, A, B, (const int*)(p->ws + L.list_w), cnt[CLS_W], C_row_ptr, p->ctr, s, p->h.max_u_w,
                           p->wopt);
    if (cnt[CLS_B] > 0)
      launch_hash_symbolic(CLS_B, A, B, (const int*)(p->ws + L.list_b), cnt[CLS_B], C_row_ptr, p->ctr, s,
                           p->h.max_u_b);
    if (cnt[CLS_G] > 0)
      launch_dense_symbolic(A, B, (const int*)(p->ws + L.list_g), cnt[CLS_G], p->ws + L.slabs, p->nslabs,
                            C_row_ptr, p->ctr, s);
    const int wide = p->h.max_u_merge > 32;
    launch_merge_fused(wide, p->values_mode, A, B, cls, C_row_ptr, C_col, C_val, capacity,
                       (unsigned long long*)(p->ws + L.fused), p->ctr, s, p->spin_limit, p->drop_tile);
    if (cnt[CLS_W] > 0)
      launch_hash_numeric(CLS_W, A, B, (const int*)(p->ws + L.list_w), cnt[CLS_W], C_row_ptr, C_col, C_val, p->ctr, s, p->h.max_u_w,
                        p->wopt);
    if (cnt[CLS_B] > 0)
      launch_hash_numeric(CLS_B, A, B, (const int*)(p->ws + L.list_b), cnt[CLS_B], C_row_ptr, C_col, C_val, p->ctr, s,
                          p->h.max_u_b);
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
  const Layout& L = p->L;
  const int* cnt = p->h.count;
  if (p->ev_start) cudaEventRecord(p->ev_start, s);
  DevCsr A, B;
  prepare_values(p, A_val, B_val, A, B, s);
  if (cnt[CLS_M1] + cnt[CLS_M2] > 0) launch_replay(p->h.max_u_merge > 32, A, B, p->ws + L.cls, p->C_rp, map, C_val, s);
  if (cnt[CLS_W] > 0)
    launch_hash_numeric(CLS_W, A, B, (const int*)(p->ws + L.list_w), cnt[CLS_W], p->C_rp, C_col, C_val, p->ctr, s, p->h.max_u_w,
                        p->wopt);
  if (cnt[CLS_B] > 0)
    launch_hash_numeric(CLS_B, A, B, (const int*)(p->ws + L.list_b), cnt[CLS_B], p->C_rp, C_col, C_val, p->ctr, s,
                        p->h.max_u_b);
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
  if (p->ev_start) cudaEventRecord(p->ev_start, s);
  DevCsr A, B;
  prepare_values(p, dB_val ? A_val : nullptr, dA_val ? B_val : nullptr, A, B, s);
  // gradients of an operand given by columns are formed in row order, then scattered back
  double* dA_rows = (dA_val && p->csc[0]) ? p->cgrad[0] : dA_val;
  double* dB_rows = (dB_val && p->csc[1]) ? p->cgrad[1] : dB_val;
  if (dA_val) launch_grad_a(A, B, p->C_rp, p->C_col, dC_val, dA_rows, p->ctr, s);
  if (dB_val) {
    if (p->transposed_ws != workspace) {
      launch_transpose(A, workspace, p->ctr, s);
      p->transposed_ws = workspace;
    }
    launch_grad_b(A, B, workspace, p->C_rp, p->C_col, dC_val, dB_rows, p->ctr, s);
  }
  if (dA_rows != dA_val) launch_scatter(p->perm[0], dA_rows, dA_val, p->A.nnz, s);
  if (dB_rows != dB_val) launch_scatter(p->perm[1], dB_rows, dB_val, p->B.nnz, s);
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
