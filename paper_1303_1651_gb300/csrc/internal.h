// Host-side launchers between the C-ABI layer (api.cu) and the kernel files.
#pragma once
#include <cstddef>
#include <cuda_runtime.h>
#include "common.cuh"

namespace spg {

// a1: per-row product counts, row classes, class lists, F, max row count (binning).
// zero / nzero: when given, the kernel also clears nzero 64-bit words there (the single-pass
// product's tile states) and the counters' ticket, so that no separate memset precedes that pass.
void launch_bin(const DevCsr& A, const DevCsr& B, const Limits& lim, uint8_t* cls, int* const lists[NUM_CLS],
                Counters* ctr, cudaStream_t s, unsigned long long* zero = nullptr, long long nzero = 0);

// a3: exclusive scan, in place, of counts[0..n-2] into row_ptr[0..n-1] (n = rows + 1).
size_t scan_tile_state_bytes(long long n);
// The total (rp[n-1]) is also stored at total_out when it is not NULL.
void launch_scan(int* rp, long long n, unsigned long long* tile_state, Counters* ctr, long long* total_out,
                 cudaStream_t s);

// a2/a4, merge classes (M1 and M2 together): warp tiles of 32 consecutive rows.  `wide` selects the
// 64-product sort (needed when some merge-class row has more than 32 products).  values_mode:
// 0 = automatic (values read from B in the reduce for 32-product tiles, staged for 64), 1 = read
// from B (C written from the reduce), 2 = staged in shared memory (C written by a coalesced pass).
void launch_merge_symbolic(int wide, const DevCsr& A, const DevCsr& B, const uint8_t* rowcls, int* counts,
                           Counters* ctr, cudaStream_t s);
void launch_merge_numeric(int wide, int values_mode, const DevCsr& A, const DevCsr& B, const uint8_t* rowcls,
                          const int* rp, int* C_col, double* C_val, Counters* ctr, cudaStream_t s);
// Fused single pass: numeric for merge-class rows, C's row pointer for every row (rows of other classes
// bring their counts in rp), entries written into C_col/C_val of `capacity` entries.  Uses ctr->ticket.
// spin_limit: rounds of re-reads before a look-back gives up (0: the default bound); drop_tile:
// testing only, a tile that publishes nothing (-1: none).  max_u_dev: when not NULL, the launch runs
// only if (*max_u_dev > 32) == wide on the device (both forms are launched before the host knows).
void launch_merge_fused(int wide, int values_mode, const DevCsr& A, const DevCsr& B, const uint8_t* rowcls, int* rp,
                        int* C_col, double* C_val, long long capacity, unsigned long long* tile_state, Counters* ctr,
                        cudaStream_t s, int spin_limit = 0, int drop_tile = -1, const int* max_u_dev = nullptr);
size_t fused_tile_state_bytes(int rows);

// Ordering of the rows of class W (the per-row choice of Section IV-B's "Combined" kernel):
// bitvec_ratio: the bit vector is taken when the row's column range is at most this many columns
// per product (1..128); order: 0 automatic, 1 bit vector whenever it fits, 2 register sort
// whenever its keys fit, 3 hash table.
struct WarpOrder {
  int bitvec_ratio = 128;
  int order = 0;
};

// a2/a4, classes W (warp per row) and B (block per row), rows from a list.  umax: the longest row
// of the class (W: sizes the W kernel's shared memory; B: the sums of its bit-vector windows, at
// most BB_MAX_U, and the block size).  Class B orders each row by a bit vector over windows of
// columns (all of B when B has at most 2^18 columns, else 2^16 columns per window).
constexpr int BB_MAX_U = 8192;
void launch_hash_symbolic(int cls, const DevCsr& A, const DevCsr& B, const int* list, int count, int* counts,
                          Counters* ctr, cudaStream_t s, int umax = 1024, WarpOrder wo = WarpOrder(),
                          const int* count_dev = nullptr);
void launch_hash_numeric(int cls, const DevCsr& A, const DevCsr& B, const int* list, int count, const int* rp,
                         int* C_col, double* C_val, Counters* ctr, cudaStream_t s, int umax = 1024,
                         WarpOrder wo = WarpOrder(), const int* count_dev = nullptr);

// a2/a4, class G: dense accumulator slabs in global memory (one slab per CTA).
size_t dense_slab_bytes(int ncols);
// zero_slabs: every slab in use is cleared first (when the caller does not know them to be clear).
void launch_dense_symbolic(const DevCsr& A, const DevCsr& B, const int* list, int count, void* slabs, int nslabs,
                           int* counts, Counters* ctr, cudaStream_t s, const int* count_dev = nullptr,
                           bool zero_slabs = false);
void launch_dense_numeric(const DevCsr& A, const DevCsr& B, const int* list, int count, void* slabs, int nslabs,
                          const int* rp, int* C_col, double* C_val, Counters* ctr, cudaStream_t s,
                          const int* count_dev = nullptr);

// Transpose of A's structure (workspace of transpose_bytes(A.cols, A.nnz)): the compressed rows of
// A^T -- T_cp (A.cols + 1), T_row (nnz: the row of A of each entry) and T_src (nnz: its position
// in A) -- each row ordered by (T_row, T_src).  Used by the backward (dB) and to convert an operand
// given in compressed columns into compressed rows.
size_t transpose_bytes(int nrows_t, long long nnz);
void launch_transpose(const DevCsr& A, void* ws, Counters* ctr, cudaStream_t s);
struct TransposeView {
  int* T_cp;
  int* T_row;
  int* T_src;
};
TransposeView transpose_view(void* ws, int nrows_t, long long nnz);
// dst[d] = src[perm[d]] and dst[perm[d]] = src[d], d < n.
void launch_gather(const int* perm, const double* src, double* dst, long long n, cudaStream_t s);
void launch_scatter(const int* perm, const double* src, double* dst, long long n, cudaStream_t s);

// Backward: dA, dB.
void launch_grad_a(const DevCsr& A, const DevCsr& B, const int* C_rp, const int* C_col, const double* W, double* dA,
                   Counters* ctr, cudaStream_t s);
void launch_grad_b(const DevCsr& A, const DevCsr& B, const void* tws, const int* C_rp, const int* C_col,
                   const double* W, double* dB, Counters* ctr, cudaStream_t s);

int num_sms();

// Resident blocks per SM of kern with `threads` threads and `smem` bytes of dynamic shared memory,
// on the current device.  The first call for a (kernel, size) raises the kernel's dynamic
// shared-memory limit to the size and asks the occupancy calculator; later calls reuse the answer
// (a small product would otherwise spend more host time on these driver calls than on its kernels).
int blocks_per_sm(const void* kern, int threads, size_t smem);

// Largest B.cols the merge classes accept (their sort keys hold column << 6).
int merge_max_cols();

// Pattern reuse (replay.cu): a position map for the products of the sort-class rows.
size_t replay_map_bytes(int rows, int max_u);
void launch_replay_record(const DevCsr& A, const DevCsr& B, const uint8_t* cls, const int* C_rp, const int* C_col,
                          void* map, unsigned long long* scan_state, Counters* ctr, cudaStream_t s);
void launch_replay(int wide, const DevCsr& A, const DevCsr& B, const uint8_t* cls, const int* C_rp, const void* map,
                   double* C_val, cudaStream_t s);

}  // namespace spg
