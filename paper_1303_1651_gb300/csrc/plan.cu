// a1 row binning and a3 exclusive scan.
#include "internal.h"

namespace spg {

int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// ---------------------------------------------------------------------------
// a1: u_r = sum over j in row r of A of nnz(B_j) -- the number of multiplications
// of row r (Section III); summed over rows it is the never-underestimating nnz
// estimate of Section IV-B.  Each row gets the class of accumulator it will use.
// ---------------------------------------------------------------------------
constexpr int BIN_THREADS = 1024;

__global__ void __launch_bounds__(BIN_THREADS)
k_bin(DevCsr A, DevCsr B, Limits lim, uint8_t* __restrict__ cls, int* l0, int* l1, int* l2, int* l3, int* l4,
      Counters* __restrict__ ctr) {
  int* lists[NUM_CLS] = {l0, l1, l2, l3, l4};
  const int r = blockIdx.x * BIN_THREADS + threadIdx.x;
  const int lane = threadIdx.x & 31;
  long long u = 0;
  int c = -1;
  bool bad = false;
  if (r < A.rows) {
    const int a0 = A.rp[r], a1 = A.rp[r + 1];
    const int k = a1 - a0;
    if (k < 0) bad = true;
    // eight entries per round, all loads of a round in flight together
    for (int p0 = a0; p0 < a1; p0 += 8) {
      int j[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) j[i] = (p0 + i < a1) ? __ldg(A.col + p0 + i) : -1;
      int lo[8], hi[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        lo[i] = hi[i] = 0;
        if (j[i] >= 0) {
          if ((unsigned)j[i] >= (unsigned)B.rows) { bad = true; continue; }
          lo[i] = __ldg(B.rp + j[i]);
          hi[i] = __ldg(B.rp + j[i] + 1);
        } else if (p0 + i < a1) {
          bad = true;   // negative column index
        }
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int len = hi[i] - lo[i];
        if (len < 0) bad = true; else u += len;
      }
    }
    if (k <= lim.merge_k && u <= lim.m1_u) c = CLS_M1;
    else if (k <= lim.merge_k && u <= lim.m2_u) c = CLS_M2;
    else if (u <= lim.warp_u) c = CLS_W;
    else if (u <= lim.block_u) c = CLS_B;
    else c = CLS_G;
    cls[r] = (uint8_t)c;
  }
  // warp-aggregated appends to the class lists (rare classes), block-aggregated counts
  __shared__ int s_cnt[NUM_CLS];
  __shared__ long long s_sum[BIN_THREADS / 32];
  __shared__ long long s_max[BIN_THREADS / 32];
  if (threadIdx.x < NUM_CLS) s_cnt[threadIdx.x] = 0;
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NUM_CLS; ++q) {
    const unsigned mask = __ballot_sync(FULL, c == q);
    if (mask) {
      if (lists[q]) {
        const int leader = __ffs(mask) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(&ctr->count[q], __popc(mask));
        base = __shfl_sync(FULL, base, leader);
        if (c == q) lists[q][base + __popc(mask & lanemask_lt())] = r;
      } else if (lane == 0) {
        atomicAdd(&s_cnt[q], __popc(mask));
      }
    }
  }
  // block totals: F, the largest row, the largest merge-class row
  long long ws = warp_sum_ll(u);
  long long wm = u;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) wm = max(wm, __shfl_xor_sync(FULL, wm, d));
  const int um = __reduce_max_sync(FULL, (c == CLS_M1 || c == CLS_M2) ? (int)u : 0);
  if (lane == 0 && um > 0) atomicMax(&ctr->max_u_merge, um);
  const bool anybad = __any_sync(FULL, bad);
  if (lane == 0) {
    s_sum[threadIdx.x >> 5] = ws;
    s_max[threadIdx.x >> 5] = wm;
    if (anybad) atomicOr(&ctr->status, ST_INVALID);
  }
  __syncthreads();
  if (threadIdx.x < NUM_CLS && s_cnt[threadIdx.x]) atomicAdd(&ctr->count[threadIdx.x], s_cnt[threadIdx.x]);
  if (threadIdx.x == 0) {
    long long t = 0, mx = 0;
    for (int w = 0; w < BIN_THREADS / 32; ++w) { t += s_sum[w]; mx = max(mx, s_max[w]); }
    if (t) atomicAdd(&ctr->F, (unsigned long long)t);
    if (mx > INT_MAX) { atomicOr(&ctr->status, ST_OVERFLOW); mx = INT_MAX; }
    atomicMax(&ctr->max_u, (int)mx);
  }
}

void launch_bin(const DevCsr& A, const DevCsr& B, const Limits& lim_in, uint8_t* cls, int* const lists[NUM_CLS],
                Counters* ctr, cudaStream_t s) {
  if (A.rows <= 0) return;
  Limits lim = lim_in;
  if (B.cols > merge_max_cols()) { lim.m1_u = -1; lim.m2_u = -1; }   // sort keys hold column << log2(N)
  const int grid = (A.rows + BIN_THREADS - 1) / BIN_THREADS;
  k_bin<<<grid, BIN_THREADS, 0, s>>>(A, B, lim, cls, lists[0], lists[1], lists[2], lists[3], lists[4], ctr);
}

// ---------------------------------------------------------------------------
// a3: single-pass exclusive scan with decoupled look-back.  Tiles take a ticket
// in launch order, so every predecessor of a tile has started; the look-back
// wait is still bounded (ST_TIMEOUT) rather than trusted.  Sums are 64-bit so
// nnz(C) > INT32_MAX is detected (ST_OVERFLOW) instead of wrapping.
// Tile state word: value << 2 | flag, flag 1 = tile aggregate, 2 = inclusive prefix.
// ---------------------------------------------------------------------------
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;
constexpr long long LOOKBACK_SPIN_LIMIT = 1LL << 24;

size_t scan_tile_state_bytes(long long n) {
  return (size_t)((n + SCAN_TILE - 1) / SCAN_TILE) * sizeof(unsigned long long);
}

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.volatile.global.u64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}

__global__ void __launch_bounds__(SCAN_THREADS)
k_scan(int* __restrict__ rp, long long n, unsigned long long* __restrict__ ts, Counters* __restrict__ ctr,
       long long* __restrict__ total_out) {
  __shared__ int s_tile;
  __shared__ long long s_warp[SCAN_THREADS / 32];
  __shared__ long long s_prefix;
  if (threadIdx.x == 0) s_tile = (int)atomicAdd(&ctr->ticket, 1u);
  __syncthreads();
  const int tile = s_tile;
  const long long base = (long long)tile * SCAN_TILE + (long long)threadIdx.x * SCAN_ITEMS;
  // element n-1 (row_ptr[rows]) carries no count: it receives the total
  long long v[SCAN_ITEMS];
  long long run = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    const long long idx = base + i;
    const long long x = (idx < n - 1) ? (long long)rp[idx] : 0;
    v[i] = run;          // thread-local exclusive
    run += x;
  }
  // block exclusive scan of per-thread totals
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long incl = run;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    long long y = __shfl_up_sync(FULL, incl, d);
    if (lane >= d) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  long long warp_off = 0, tile_total = 0;
  for (int w = 0; w < SCAN_THREADS / 32; ++w) {
    if (w < warp) warp_off += s_warp[w];
    tile_total += s_warp[w];
  }
  const long long thread_off = warp_off + incl - run;
  if (threadIdx.x == 0) {
    long long prefix = 0;
    if (tile == 0) {
      __threadfence();
      atomicExch(&ts[0], ((unsigned long long)tile_total << 2) | 2ull);
    } else {
      atomicExch(&ts[tile], ((unsigned long long)tile_total << 2) | 1ull);
      int pred = tile - 1;
      long long spins = 0;
      while (pred >= 0) {
        const unsigned long long w = ld_volatile_u64(&ts[pred]);
        const unsigned flag = (unsigned)(w & 3ull);
        if (flag == 0) {
          if (++spins > LOOKBACK_SPIN_LIMIT) { atomicOr(&ctr->status, ST_TIMEOUT); break; }
          __nanosleep(20);
          continue;
        }
        prefix += (long long)(w >> 2);
        if (flag == 2) break;
        --pred;
      }
      __threadfence();
      atomicExch(&ts[tile], ((unsigned long long)(prefix + tile_total) << 2) | 2ull);
    }
    s_prefix = prefix;
  }
  __syncthreads();
  const long long off = s_prefix + thread_off;
  bool ovf = false;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    const long long idx = base + i;
    if (idx < n) {
      const long long e = off + v[i];
      if (e > INT_MAX) ovf = true;
      rp[idx] = (int)e;
      if (idx == n - 1 && total_out) *total_out = e;
    }
  }
  if (__any_sync(FULL, ovf) && lane == 0) atomicOr(&ctr->status, ST_OVERFLOW);
}

void launch_scan(int* rp, long long n, unsigned long long* tile_state, Counters* ctr, long long* total_out,
                 cudaStream_t s) {
  const long long tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  k_scan<<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(rp, n, tile_state, ctr, total_out);
}

}  // namespace spg
