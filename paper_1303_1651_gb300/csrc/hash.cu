// a2 symbolic and a4 numeric for rows too long for the merge classes.
//
// Classes W (a warp per row, 1024-slot table) and B (a 512-thread block per
// row, 8192-slot table) replace the dense temporary vector of the row-major
// algorithm (Section IV-A) with an open-addressing hash table in shared memory
// (linear probing, bounded to the table size).  The numeric pass then orders
// the touched columns -- the "Sort" store of Section IV-B -- with a bitonic
// sort of the compacted table, and appends the row to C.
//
// Class G (rows beyond the block table) uses the dense temporary vector itself,
// one per CTA in global memory, scanned over [min, max] of the touched columns
// in ascending order: the "MinMax" store of Section IV-B.  Flags mark touched
// positions, so entries that cancel to 0.0 are kept.
#include "internal.h"

namespace spg {

template <int GROUP>
__device__ __forceinline__ void group_sync() {
  if constexpr (GROUP == 32) __syncwarp(); else __syncthreads();
}

// Insert key; returns slot, sets *fresh when this call created the entry.  -1 when the table is full.
__device__ __forceinline__ int hash_insert(int* keys, int x, unsigned log2t, bool* fresh) {
  const unsigned mask = (1u << log2t) - 1u;
  unsigned h = hash_slot(x, log2t);
  volatile int* vk = keys;
  for (unsigned probe = 0; probe <= mask; ++probe) {
    const int k = vk[h];
    if (k == x) { *fresh = false; return (int)h; }
    if (k == KEY_NONE) {
      const int old = atomicCAS(&keys[h], KEY_NONE, x);
      if (old == KEY_NONE) { *fresh = true; return (int)h; }
      if (old == x) { *fresh = false; return (int)h; }
    }
    h = (h + 1u) & mask;
  }
  *fresh = false;
  return -1;
}

template <int GROUP>
__device__ __forceinline__ int group_sum(int v, int* s_red) {
  if constexpr (GROUP == 32) {
    return __reduce_add_sync(FULL, v);
  } else {
    v = __reduce_add_sync(FULL, v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) s_red[w] = v;
    __syncthreads();
    int t = 0;
    for (int i = 0; i < GROUP / 32; ++i) t += s_red[i];
    __syncthreads();
    return t;
  }
}

template <int GROUP, int LOG2T, int GPB>
struct HashSmem {
  static constexpr int T = 1 << LOG2T;
  static constexpr size_t sym_per_group = 4 * T;
  // numeric: vals[T] + cvals[T/2] (doubles), keys[T] + ckeys[T/2] (ints), counter
  static constexpr size_t num_per_group = 8 * T + 8 * (T / 2) + 4 * T + 4 * (T / 2) + 16;
  static constexpr size_t sym_bytes = GPB * sym_per_group + 4 * 32;
  static constexpr size_t num_bytes = GPB * num_per_group + 4 * 32;
};

template <int GROUP, int LOG2T, int GPB>
__global__ void __launch_bounds__(GROUP * GPB)
k_hash_sym(DevCsr A, DevCsr B, const int* __restrict__ list, int count, int* __restrict__ counts,
           Counters* __restrict__ ctr) {
  using L = HashSmem<GROUP, LOG2T, GPB>;
  constexpr int T = L::T;
  extern __shared__ __align__(16) unsigned char smem[];
  const int g = threadIdx.x / GROUP, gt = threadIdx.x % GROUP;
  int* keys = reinterpret_cast<int*>(smem + g * L::sym_per_group);
  int* s_red = reinterpret_cast<int*>(smem + GPB * L::sym_per_group);
  for (int idx = blockIdx.x * GPB + g; idx < count; idx += gridDim.x * GPB) {
    for (int i = gt; i < T; i += GROUP) keys[i] = KEY_NONE;
    group_sync<GROUP>();
    const int r = list[idx];
    const int a0 = A.rp[r], a1 = A.rp[r + 1];
    int cnt = 0;
    bool full = false;
    for (int p = a0; p < a1; ++p) {
      const int j = __ldg(A.col + p);
      const int bs = __ldg(B.rp + j), be = __ldg(B.rp + j + 1);
      for (int q = bs + gt; q < be; q += GROUP) {
        bool fresh;
        const int slot = hash_insert(keys, __ldg(B.col + q), LOG2T, &fresh);
        if (slot < 0) full = true;
        cnt += fresh;
      }
    }
    if (full) atomicOr(&ctr->status, ST_TABLE_FULL);
    const int total = group_sum<GROUP>(cnt, s_red);
    if (gt == 0) counts[r] = total;
    group_sync<GROUP>();
  }
}

template <int GROUP, int LOG2T, int GPB>
__global__ void __launch_bounds__(GROUP * GPB)
k_hash_num(DevCsr A, DevCsr B, const int* __restrict__ list, int count, const int* __restrict__ rp,
           int* __restrict__ C_col, double* __restrict__ C_val, Counters* __restrict__ ctr) {
  using L = HashSmem<GROUP, LOG2T, GPB>;
  constexpr int T = L::T;
  extern __shared__ __align__(16) unsigned char smem[];
  const int g = threadIdx.x / GROUP, gt = threadIdx.x % GROUP;
  unsigned char* gb = smem + g * L::num_per_group;
  double* vals = reinterpret_cast<double*>(gb);
  double* cvals = vals + T;
  int* keys = reinterpret_cast<int*>(cvals + T / 2);
  int* ckeys = keys + T;
  int* s_n = ckeys + T / 2;
  for (int idx = blockIdx.x * GPB + g; idx < count; idx += gridDim.x * GPB) {
    for (int i = gt; i < T; i += GROUP) { keys[i] = KEY_NONE; vals[i] = 0.0; }
    if (gt == 0) *s_n = 0;
    group_sync<GROUP>();
    const int r = list[idx];
    const int a0 = A.rp[r], a1 = A.rp[r + 1];
    bool full = false;
    for (int p = a0; p < a1; ++p) {
      const int j = __ldg(A.col + p);
      const double a = __ldg(A.val + p);
      const int bs = __ldg(B.rp + j), be = __ldg(B.rp + j + 1);
      for (int q = bs + gt; q < be; q += GROUP) {
        bool fresh;
        const int slot = hash_insert(keys, __ldg(B.col + q), LOG2T, &fresh);
        if (slot < 0) { full = true; continue; }
        atomicAdd(&vals[slot], __dmul_rn(a, __ldg(B.val + q)));
      }
    }
    if (full) atomicOr(&ctr->status, ST_TABLE_FULL);
    group_sync<GROUP>();
    // compact the touched slots (any order), then sort them by column
    for (int i = gt; i < T; i += GROUP) {
      const int k = keys[i];
      if (k != KEY_NONE) {
        const int pos = atomicAdd(s_n, 1);
        if (pos < T / 2) { ckeys[pos] = k; cvals[pos] = vals[i]; }
      }
    }
    group_sync<GROUP>();
    const int n = min(*s_n, T / 2);
    int n2 = 1;
    while (n2 < n) n2 <<= 1;
    for (int i = n + gt; i < n2; i += GROUP) { ckeys[i] = KEY_NONE; cvals[i] = 0.0; }
    group_sync<GROUP>();
    for (int kk = 2; kk <= n2; kk <<= 1) {
      for (int jj = kk >> 1; jj > 0; jj >>= 1) {
        for (int i = gt; i < n2; i += GROUP) {
          const int ixj = i ^ jj;
          if (ixj > i) {
            const int ki = ckeys[i], kj = ckeys[ixj];
            const bool up = (i & kk) == 0;
            if ((ki > kj) == up) {
              ckeys[i] = kj; ckeys[ixj] = ki;
              const double t = cvals[i]; cvals[i] = cvals[ixj]; cvals[ixj] = t;
            }
          }
        }
        group_sync<GROUP>();
      }
    }
    const int g0 = rp[r], g1 = rp[r + 1];
    if (gt == 0 && g1 - g0 != n) atomicOr(&ctr->status, ST_MISMATCH);
    for (int i = gt; i < n && g0 + i < g1; i += GROUP) {
      C_col[g0 + i] = ckeys[i];
      C_val[g0 + i] = cvals[i];
    }
    group_sync<GROUP>();
  }
}

template <int GROUP, int LOG2T, int GPB, bool NUM>
static void launch_hash(const DevCsr& A, const DevCsr& B, const int* list, int count, int* counts, const int* rp,
                        int* C_col, double* C_val, Counters* ctr, cudaStream_t s) {
  if (count <= 0) return;
  using L = HashSmem<GROUP, LOG2T, GPB>;
  const size_t bytes = NUM ? L::num_bytes : L::sym_bytes;
  int per_sm = 0;
  if (NUM) {
    auto kern = k_hash_num<GROUP, LOG2T, GPB>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, GROUP * GPB, bytes);
    const int blocks = std::max(1, std::min((count + GPB - 1) / GPB, num_sms() * std::max(per_sm, 1)));
    kern<<<blocks, GROUP * GPB, bytes, s>>>(A, B, list, count, rp, C_col, C_val, ctr);
  } else {
    auto kern = k_hash_sym<GROUP, LOG2T, GPB>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, GROUP * GPB, bytes);
    const int blocks = std::max(1, std::min((count + GPB - 1) / GPB, num_sms() * std::max(per_sm, 1)));
    kern<<<blocks, GROUP * GPB, bytes, s>>>(A, B, list, count, counts, ctr);
  }
}

void launch_hash_symbolic(int cls, const DevCsr& A, const DevCsr& B, const int* list, int count, int* counts,
                          Counters* ctr, cudaStream_t s) {
  if (cls == CLS_W) launch_hash<32, 10, 8, false>(A, B, list, count, counts, nullptr, nullptr, nullptr, ctr, s);
  else launch_hash<512, 13, 1, false>(A, B, list, count, counts, nullptr, nullptr, nullptr, ctr, s);
}

void launch_hash_numeric(int cls, const DevCsr& A, const DevCsr& B, const int* list, int count, const int* rp,
                         int* C_col, double* C_val, Counters* ctr, cudaStream_t s) {
  if (cls == CLS_W) launch_hash<32, 10, 4, true>(A, B, list, count, nullptr, rp, C_col, C_val, ctr, s);
  else launch_hash<512, 13, 1, true>(A, B, list, count, nullptr, rp, C_col, C_val, ctr, s);
}

// ---------------------------------------------------------------------------
// Class G: dense accumulator per CTA.  Slab layout: double acc[ncols], int flag[ncols].
// Invariant between rows: the slab is all zero (each row clears what it touched).
// ---------------------------------------------------------------------------
constexpr int G_THREADS = 1024;

size_t dense_slab_bytes(int ncols) {
  const size_t n = (size_t)std::max(ncols, 1);
  return ((n * 12 + 255) / 256) * 256;
}

__device__ __forceinline__ void block_minmax_count(int& mn, int& mx, int& cnt, int* s_a, int* s_b, int* s_c) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  mn = __reduce_min_sync(FULL, mn);
  mx = __reduce_max_sync(FULL, mx);
  cnt = __reduce_add_sync(FULL, cnt);
  if (lane == 0) { s_a[w] = mn; s_b[w] = mx; s_c[w] = cnt; }
  __syncthreads();
  mn = INT_MAX; mx = -1; cnt = 0;
  for (int i = 0; i < G_THREADS / 32; ++i) { mn = min(mn, s_a[i]); mx = max(mx, s_b[i]); cnt += s_c[i]; }
  __syncthreads();
}

template <bool NUM>
__global__ void __launch_bounds__(G_THREADS)
k_dense(DevCsr A, DevCsr B, const int* __restrict__ list, int count, unsigned char* slabs, size_t slab_bytes,
        int* __restrict__ counts, const int* __restrict__ rp, int* __restrict__ C_col, double* __restrict__ C_val,
        Counters* __restrict__ ctr) {
  __shared__ int s_a[32], s_b[32], s_c[32];
  __shared__ int s_scan[32];
  const int n = B.cols;
  double* acc = reinterpret_cast<double*>(slabs + blockIdx.x * slab_bytes);
  int* flag = reinterpret_cast<int*>(acc + n);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int idx = blockIdx.x; idx < count; idx += gridDim.x) {
    const int r = list[idx];
    const int a0 = A.rp[r], a1 = A.rp[r + 1];
    int mn = INT_MAX, mx = -1, cnt = 0;
    bool bad = false;
    for (int p = a0; p < a1; ++p) {
      const int j = __ldg(A.col + p);
      const double a = NUM ? __ldg(A.val + p) : 0.0;
      const int bs = __ldg(B.rp + j), be = __ldg(B.rp + j + 1);
      for (int q = bs + threadIdx.x; q < be; q += G_THREADS) {
        const int x = __ldg(B.col + q);
        if ((unsigned)x >= (unsigned)n) { bad = true; continue; }
        if (atomicExch(&flag[x], 1) == 0) { ++cnt; mn = min(mn, x); mx = max(mx, x); }
        if (NUM) atomicAdd(&acc[x], __dmul_rn(a, __ldg(B.val + q)));
      }
    }
    if (bad) atomicOr(&ctr->status, ST_INVALID);
    block_minmax_count(mn, mx, cnt, s_a, s_b, s_c);   // includes __syncthreads
    if (!NUM) {
      if (threadIdx.x == 0) counts[r] = cnt;
      for (long long x = (long long)mn + threadIdx.x; x <= mx; x += G_THREADS) flag[x] = 0;
    } else {
      // ordered output: block-wide exclusive scan of flags over [mn, mx], chunk by chunk
      const int g0 = rp[r], g1 = rp[r + 1];
      int pos = 0;
      for (long long chunk = mn; chunk <= mx; chunk += G_THREADS) {
        const long long xl = chunk + threadIdx.x;
        const int x = (int)xl;
        // flags and sums were updated by atomics at L2: read around L1
        const int f = (xl <= mx) ? __ldcg(flag + x) : 0;
        const unsigned bal = __ballot_sync(FULL, f);
        const int before = __popc(bal & lanemask_lt());
        if (lane == 0) s_scan[w] = __popc(bal);
        __syncthreads();
        int woff = 0, tot = 0;
        for (int i = 0; i < G_THREADS / 32; ++i) { if (i < w) woff += s_scan[i]; tot += s_scan[i]; }
        if (f) {
          const int dstp = g0 + pos + woff + before;
          if (dstp < g1) { C_col[dstp] = x; C_val[dstp] = __ldcg(acc + x); }
          acc[x] = 0.0;
          flag[x] = 0;
        }
        pos += tot;
        __syncthreads();
      }
      if (threadIdx.x == 0 && pos != g1 - g0) atomicOr(&ctr->status, ST_MISMATCH);
    }
    __syncthreads();
  }
}

void launch_dense_symbolic(const DevCsr& A, const DevCsr& B, const int* list, int count, void* slabs, int nslabs,
                           int* counts, Counters* ctr, cudaStream_t s) {
  if (count <= 0 || nslabs <= 0) return;
  const int blocks = std::min(count, nslabs);
  k_dense<false><<<blocks, G_THREADS, 0, s>>>(A, B, list, count, (unsigned char*)slabs, dense_slab_bytes(B.cols),
                                              counts, nullptr, nullptr, nullptr, ctr);
}

void launch_dense_numeric(const DevCsr& A, const DevCsr& B, const int* list, int count, void* slabs, int nslabs,
                          const int* rp, int* C_col, double* C_val, Counters* ctr, cudaStream_t s) {
  if (count <= 0 || nslabs <= 0) return;
  const int blocks = std::min(count, nslabs);
  k_dense<true><<<blocks, G_THREADS, 0, s>>>(A, B, list, count, (unsigned char*)slabs, dense_slab_bytes(B.cols),
                                             nullptr, rp, C_col, C_val, ctr);
}

}  // namespace spg
