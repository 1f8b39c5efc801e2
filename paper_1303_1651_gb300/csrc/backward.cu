// Backward of C = A * B for a loss L with dL/dC = W given on C's structure:
//   dA_ij = sum over x in row j of B of  B_jx * W_ix          (W restricted to A's structure: SDDMM)
//   dB_jx = sum over i with (i, j) in A of  A_ij * W_ix        (W restricted to B's structure)
// Both are sampled products: every term a product of the forward pass, read back through C's
// structure.  W_ix is found by binary search in row i of C (sorted, unique columns).
//
// dA: one thread per entry of A, looping over row j of B in storage order.
// dB: one thread per entry of B, looping over column j of A in row order, through the transpose
//     of A's structure (the CSR -> CSC conversion of Section IV-A), built once per plan.
// Accumulation is acc = fma(term factor, W, acc) starting from +0.0, in the oracle's order.
#include "internal.h"

namespace spg {

constexpr int BW_THREADS = 256;

// position of column x in the sorted columns [lo, hi) of C, or -1
__device__ __forceinline__ int find_col(const int* __restrict__ col, int lo, int hi, int x) {
  const int end = hi;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const int v = __ldg(col + mid);
    if (v < x) lo = mid + 1; else hi = mid;
  }
  return (lo < end && __ldg(col + lo) == x) ? lo : -1;
}

// row of A's entry p: the last r with rp[r] <= p (rows may be empty)
__device__ __forceinline__ int row_of(const int* __restrict__ rp, int rows, int p) {
  int lo = 0, hi = rows;   // answer in [0, rows)
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(rp + mid) <= p) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(BW_THREADS)
k_grad_a(DevCsr A, DevCsr B, const int* __restrict__ C_rp, const int* __restrict__ C_col,
         const double* __restrict__ W, double* __restrict__ dA, Counters* __restrict__ ctr) {
  const long long stride = (long long)gridDim.x * BW_THREADS;
  bool miss = false;
  for (long long pl = (long long)blockIdx.x * BW_THREADS + threadIdx.x; pl < A.nnz; pl += stride) {
    const int p = (int)pl;
    const int i = row_of(A.rp, A.rows, p);
    const int j = __ldg(A.col + p);
    const int c0 = __ldg(C_rp + i), c1 = __ldg(C_rp + i + 1);
    const int q0 = __ldg(B.rp + j), q1 = __ldg(B.rp + j + 1);
    double acc = 0.0;
    for (int q = q0; q < q1; ++q) {
      const int pos = find_col(C_col, c0, c1, __ldg(B.col + q));
      if (pos < 0) { miss = true; continue; }
      acc = __fma_rn(__ldg(B.val + q), __ldg(W + pos), acc);
    }
    dA[p] = acc;
  }
  if (__any_sync(FULL, miss) && (threadIdx.x & 31) == 0) atomicOr(&ctr->status, ST_MISMATCH);
}

// Transposed structure of A: T_cp (A.cols + 1), T_row (nnzA), T_src (nnzA: position in A).  The
// operand may come straight from the caller, before any validation: an index outside [0, A.cols)
// is counted in the last column, so every entry of T_row and T_src is still written (nothing is
// addressed out of range), and the status reports SPGEMM_ERR_INVALID.
__device__ __forceinline__ int clamp_col(int j, int ncols) { return j < 0 ? 0 : (j >= ncols ? ncols - 1 : j); }

__global__ void k_count_cols(DevCsr A, int* __restrict__ cnt, Counters* __restrict__ ctr) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  bool bad = false;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < A.nnz; p += stride) {
    const int j = __ldg(A.col + p);
    bad = bad || (unsigned)j >= (unsigned)A.cols;
    atomicAdd(&cnt[clamp_col(j, A.cols)], 1);
  }
  if (bad) atomicOr(&ctr->status, ST_INVALID);
}

__global__ void k_scatter_cols(DevCsr A, const int* __restrict__ T_cp, int* __restrict__ next,
                               int* __restrict__ T_row, int* __restrict__ T_src) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long pl = (long long)blockIdx.x * blockDim.x + threadIdx.x; pl < A.nnz; pl += stride) {
    const int p = (int)pl;
    const int j = clamp_col(__ldg(A.col + p), A.cols);   // as counted by k_count_cols
    const int d = __ldg(T_cp + j) + atomicAdd(&next[j], 1);
    T_row[d] = row_of(A.rp, A.rows, p);
    T_src[d] = p;
  }
}

// Order every column's entries by (row, position in A): one thread per column, insertion sort
// (columns are short; the scatter above places them in arbitrary order).
__global__ void k_sort_cols(int ncols, const int* __restrict__ T_cp, int* __restrict__ T_row, int* __restrict__ T_src) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long jl = (long long)blockIdx.x * blockDim.x + threadIdx.x; jl < ncols; jl += stride) {
    const int j = (int)jl;
    const int a = T_cp[j], b = T_cp[j + 1];
    for (int x = a + 1; x < b; ++x) {
      const int rk = T_row[x], sk = T_src[x];
      int y = x - 1;
      while (y >= a && (T_row[y] > rk || (T_row[y] == rk && T_src[y] > sk))) {
        T_row[y + 1] = T_row[y];
        T_src[y + 1] = T_src[y];
        --y;
      }
      T_row[y + 1] = rk;
      T_src[y + 1] = sk;
    }
  }
}

__global__ void __launch_bounds__(BW_THREADS)
k_grad_b(DevCsr A, DevCsr B, const int* __restrict__ T_cp, const int* __restrict__ T_row,
         const int* __restrict__ T_src, const int* __restrict__ C_rp, const int* __restrict__ C_col,
         const double* __restrict__ W, double* __restrict__ dB, Counters* __restrict__ ctr) {
  const long long stride = (long long)gridDim.x * BW_THREADS;
  bool miss = false;
  for (long long ql = (long long)blockIdx.x * BW_THREADS + threadIdx.x; ql < B.nnz; ql += stride) {
    const int q = (int)ql;
    const int j = row_of(B.rp, B.rows, q);
    const int x = __ldg(B.col + q);
    const int t0 = __ldg(T_cp + j), t1 = __ldg(T_cp + j + 1);
    double acc = 0.0;
    for (int t = t0; t < t1; ++t) {
      const int i = __ldg(T_row + t);
      const int pos = find_col(C_col, __ldg(C_rp + i), __ldg(C_rp + i + 1), x);
      if (pos < 0) { miss = true; continue; }
      acc = __fma_rn(__ldg(A.val + __ldg(T_src + t)), __ldg(W + pos), acc);
    }
    dB[q] = acc;
  }
  if (__any_sync(FULL, miss) && (threadIdx.x & 31) == 0) atomicOr(&ctr->status, ST_MISMATCH);
}

// Transpose workspace: T_cp (nrows_t + 1), next (nrows_t), T_row (nnz), T_src (nnz), all int, then
// the scan's tile states; 256-aligned pieces.
static size_t up256(size_t x) { return (x + 255) / 256 * 256; }

size_t transpose_bytes(int nrows_t, long long nnz) {
  return up256(4 * ((size_t)nrows_t + 1)) + up256(4 * (size_t)std::max(nrows_t, 1)) +
         2 * up256(4 * (size_t)std::max(nnz, 1LL)) + up256(scan_tile_state_bytes((long long)nrows_t + 1) + 64);
}

TransposeView transpose_view(void* ws, int nrows_t, long long nnz) {
  unsigned char* b = (unsigned char*)ws;
  TransposeView v;
  v.T_cp = (int*)b;
  v.T_row = (int*)(b + up256(4 * ((size_t)nrows_t + 1)) + up256(4 * (size_t)std::max(nrows_t, 1)));
  v.T_src = (int*)((unsigned char*)v.T_row + up256(4 * (size_t)std::max(nnz, 1LL)));
  return v;
}

void launch_transpose(const DevCsr& A, void* ws, Counters* ctr, cudaStream_t s) {
  unsigned char* b = (unsigned char*)ws;
  const TransposeView v = transpose_view(ws, A.cols, A.nnz);
  int* T_cp = v.T_cp;
  int* next = (int*)(b + up256(4 * ((size_t)A.cols + 1)));
  int* T_row = v.T_row;
  int* T_src = v.T_src;
  unsigned long long* scan_state = (unsigned long long*)((unsigned char*)T_src + up256(4 * (size_t)std::max(A.nnz, 1LL)));
  cudaMemsetAsync(T_cp, 0, 4 * ((size_t)A.cols + 1), s);
  cudaMemsetAsync(next, 0, 4 * (size_t)std::max(A.cols, 1), s);
  const int grid = num_sms() * 8;
  // (a matrix with entries but no columns has no column to count them in: the plan rejects it)
  if (A.nnz > 0 && A.cols > 0) k_count_cols<<<grid, 256, 0, s>>>(A, T_cp, ctr);
  // counts sit in T_cp[0..cols-1]; the scan turns them into column pointers
  cudaMemsetAsync(&ctr->ticket, 0, sizeof(unsigned), s);
  cudaMemsetAsync(scan_state, 0, scan_tile_state_bytes((long long)A.cols + 1), s);
  launch_scan(T_cp, (long long)A.cols + 1, scan_state, ctr, nullptr, s);
  if (A.nnz > 0 && A.cols > 0) {
    k_scatter_cols<<<grid, 256, 0, s>>>(A, T_cp, next, T_row, T_src);
    k_sort_cols<<<std::max(1, std::min(grid, (A.cols + 255) / 256)), 256, 0, s>>>(A.cols, T_cp, T_row, T_src);
  }
}

void launch_grad_a(const DevCsr& A, const DevCsr& B, const int* C_rp, const int* C_col, const double* W, double* dA,
                   Counters* ctr, cudaStream_t s) {
  if (A.nnz <= 0) return;
  const long long need = (A.nnz + BW_THREADS - 1) / BW_THREADS;
  const int grid = (int)std::min<long long>(need, (long long)num_sms() * 16);
  k_grad_a<<<grid, BW_THREADS, 0, s>>>(A, B, C_rp, C_col, W, dA, ctr);
}

void launch_grad_b(const DevCsr& A, const DevCsr& B, const void* tws, const int* C_rp, const int* C_col,
                   const double* W, double* dB, Counters* ctr, cudaStream_t s) {
  if (B.nnz <= 0) return;
  const TransposeView v = transpose_view(const_cast<void*>(tws), A.cols, A.nnz);
  const int* T_cp = v.T_cp;
  const int* T_row = v.T_row;
  const int* T_src = v.T_src;
  const long long need = (B.nnz + BW_THREADS - 1) / BW_THREADS;
  const int grid = (int)std::min<long long>(need, (long long)num_sms() * 16);
  k_grad_b<<<grid, BW_THREADS, 0, s>>>(A, B, T_cp, T_row, T_src, C_rp, C_col, W, dB, ctr);
}

// Values of an operand given by columns, moved between the given order and the converted row
// order: gather dst[d] = src[perm[d]], scatter dst[perm[d]] = src[d] (perm is a permutation).
__global__ void k_gather(const int* __restrict__ perm, const double* __restrict__ src, double* __restrict__ dst,
                         long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long d = (long long)blockIdx.x * blockDim.x + threadIdx.x; d < n; d += stride) {
    const int q = __ldg(perm + d);
    dst[d] = (unsigned long long)(unsigned)q < (unsigned long long)n ? __ldg(src + q) : 0.0;   // in range
  }
}

__global__ void k_scatter(const int* __restrict__ perm, const double* __restrict__ src, double* __restrict__ dst,
                          long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long d = (long long)blockIdx.x * blockDim.x + threadIdx.x; d < n; d += stride) {
    const int q = __ldg(perm + d);
    if ((unsigned long long)(unsigned)q < (unsigned long long)n) dst[q] = __ldg(src + d);   // in range
  }
}

void launch_gather(const int* perm, const double* src, double* dst, long long n, cudaStream_t s) {
  if (n <= 0) return;
  const int grid = (int)std::min<long long>((n + 255) / 256, (long long)num_sms() * 8);
  k_gather<<<grid, 256, 0, s>>>(perm, src, dst, n);
}

void launch_scatter(const int* perm, const double* src, double* dst, long long n, cudaStream_t s) {
  if (n <= 0) return;
  const int grid = (int)std::min<long long>((n + 255) / 256, (long long)num_sms() * 8);
  k_scatter<<<grid, 256, 0, s>>>(perm, src, dst, n);
}

}  // namespace spg
