// Device-side types and warp helpers shared by the SpGEMM kernels.
#pragma once
#include <cstdint>
#include <climits>
#include <algorithm>
#include <cuda_runtime.h>

namespace spg {

constexpr unsigned FULL = 0xffffffffu;
constexpr int KEY_NONE = INT_MAX;       // merge sentinel / empty hash key (valid columns are < INT_MAX)

// Row classes chosen by the binning pass (Section IV-B "Combined": a cheap per-row
// choice of the storing strategy, here of the accumulator).
enum RowClass : uint8_t {
  CLS_M1 = 0,   // <= 8 A entries, <= 32 products: register sort, one lane per row, 32-row tiles
  CLS_M2 = 1,   // <= 8 A entries, <= 64 products: register sort, two lanes per row, 16-row tiles
  CLS_W = 2,    // warp per row: bit vector, register sort or hash table in shared memory
  CLS_B = 3,    // block-per-row shared-memory hash
  CLS_G = 4,    // dense accumulator in global memory over [min, max] (MinMax)
  NUM_CLS = 5,
  CLS_NONE = 255   // a row with an invalid entry: no class kernel reads it (the status says INVALID)
};

// Status bits (sticky, read by the host after a synchronising call).
enum StatusBits : unsigned {
  ST_INVALID = 1u,     // index out of range / negative row length
  ST_OVERFLOW = 2u,    // a count does not fit int32
  ST_TABLE_FULL = 4u,  // a hash table ran out of probes
  ST_TIMEOUT = 8u,     // a bounded device wait gave up
  ST_MISMATCH = 16u,   // numeric produced a different count than symbolic (pattern changed)
  ST_UNSORTED = 32u,   // a row of B is not sorted by column (merge classes need sorted runs)
};

struct DevCsr {
  int rows, cols;
  long long nnz;
  const int* rp;
  const int* col;
  const double* val;
};

// One workspace-resident block of counters; zeroed by the plan.
struct Counters {
  unsigned long long F;      // total products (intermediate products) of the product
  long long nnzC;            // total of C, written by the scan
  unsigned status;           // StatusBits
  unsigned ticket;           // scan tile ticket
  int count[NUM_CLS];        // rows per class
  int max_u;                 // largest row product count
  int max_u_merge;           // largest product count among merge-class rows
  int max_u_w;               // largest product count among class-W rows
  int max_u_b;               // largest product count among class-B rows
  int pad[3];
};

struct Limits {
  int merge_k;     // max A entries per row for the merge classes
  int m1_u;        // max products, class M1
  int m2_u;        // max products, class M2
  int warp_u;      // max products, class W
  int block_u;     // max products, class B
};

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m; asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m)); return m;
}
__device__ __forceinline__ unsigned lanemask_le() {
  unsigned m; asm("mov.u32 %0, %%lanemask_le;" : "=r"(m)); return m;
}

// Asynchronous global -> shared copies (LDGSTS), 4 and 8 bytes; the source must be aligned to the size.
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Exclusive warp scan of an int; *total receives the warp sum.
__device__ __forceinline__ int warp_excl_scan(int v, int* total) {
  const int lane = threadIdx.x & 31;
  int x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int y = __shfl_up_sync(FULL, x, d);
    if (lane >= d) x += y;
  }
  *total = __shfl_sync(FULL, x, 31);
  return x - v;
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(FULL, v, d);
  return v;
}

__device__ __forceinline__ int warp_sum(int v) { return __reduce_add_sync(FULL, v); }

// Fibonacci hashing of a column into a power-of-two table.
__device__ __forceinline__ unsigned hash_slot(int key, unsigned log2t) {
  return ((unsigned)key * 0x9E3779B1u) >> (32 - log2t);
}

}  // namespace spg
