// a1 row binning and a3 exclusive scan.
#include <map>
#include <mutex>
#include <tuple>

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

int blocks_per_sm(const void* kern, int threads, size_t smem) {
  static std::mutex mu;
  static std::map<std::tuple<int, const void*, int, size_t>, int> cache;
  static std::map<std::pair<int, const void*>, size_t> limit;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_tuple(dev, kern, threads, smem);
  const auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  size_t& lim = limit[std::make_pair(dev, kern)];
  if (smem > lim) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    lim = smem;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (per_sm < 1) per_sm = 1;
  cache[key] = per_sm;
  return per_sm;
}

// ---------------------------------------------------------------------------
// a1: u_r = sum over j in row r of A of nnz(B_j) -- the number of multiplications
// of row r (Section III); summed over rows it is the never-underestimating nnz
// estimate of Section IV-B.  Each row gets the class of accumulator it will use.
// ---------------------------------------------------------------------------
constexpr int BIN_THREADS = 256;
constexpr int BIN_ROWS = 2;   // rows per thread and step, their loads in flight together
constexpr int BIN_EPR = 8;    // entries of A per row loaded in the first round

// Products of entries [p0, a1) of A (the rare rows longer than BIN_EPR); -1 for an invalid entry
__device__ __noinline__ long long bin_tail(const DevCsr A, const DevCsr B, int p0, int a1) {
  long long u = 0;
  for (int p = p0; p < a1; ++p) {
    const int j = __ldg(A.col + p);
    if ((unsigned)j >= (unsigned)B.rows) return -1;
    const int len = __ldg(B.rp + j + 1) - __ldg(B.rp + j);
    if (len < 0) return -1;
    u += len;
  }
  return u;
}

// Grid-stride: each thread takes BIN_ROWS rows per step (rows r and r + G, G = threads in the
// grid, so every load instruction of a warp stays coalesced), keeps its counters in registers
// and adds them to the global counters once per block at the end.
__global__ void __launch_bounds__(BIN_THREADS)
k_bin(DevCsr A, DevCsr B, Limits lim, uint8_t* __restrict__ cls, int* l0, int* l1, int* l2, int* l3, int* l4,
      Counters* __restrict__ ctr, unsigned long long* __restrict__ zero, long long nzero) {
  int* lists[NUM_CLS] = {l0, l1, l2, l3, l4};
  const int lane = threadIdx.x & 31;
  const long long G = (long long)gridDim.x * BIN_THREADS;
  if (zero) {   // the single-pass product's tile states, and its ticket (a conversion's scan used it)
    for (long long i = (long long)blockIdx.x * BIN_THREADS + threadIdx.x; i < nzero; i += G) zero[i] = 0ull;
    if (blockIdx.x == 0 && threadIdx.x == 0) ctr->ticket = 0u;
  }
  long long F = 0, umax = 0;
  int umax_merge = 0, umax_w = 0, umax_b = 0, cnt[NUM_CLS] = {0, 0, 0, 0, 0};
  bool bad = false;
  // the loop bound is warp-uniform (the warp's first row) so the ballots below see every lane
  for (long long wb = (long long)blockIdx.x * BIN_THREADS + (threadIdx.x & ~31); wb < A.rows; wb += G * BIN_ROWS) {
    int r[BIN_ROWS], a0[BIN_ROWS], a1[BIN_ROWS];
#pragma unroll
    for (int q = 0; q < BIN_ROWS; ++q) {
      const long long rl = wb + lane + q * G;
      r[q] = rl < A.rows ? (int)rl : -1;
      a0[q] = a1[q] = 0;
      if (r[q] >= 0) { a0[q] = __ldg(A.rp + r[q]); a1[q] = __ldg(A.rp + r[q] + 1); }
    }
    int j[BIN_ROWS][BIN_EPR];
#pragma unroll
    for (int q = 0; q < BIN_ROWS; ++q)
#pragma unroll
      for (int i = 0; i < BIN_EPR; ++i) j[q][i] = (a0[q] + i < a1[q]) ? __ldg(A.col + a0[q] + i) : -1;
    int len[BIN_ROWS][BIN_EPR];
#pragma unroll
    for (int q = 0; q < BIN_ROWS; ++q)
#pragma unroll
      for (int i = 0; i < BIN_EPR; ++i) {
        len[q][i] = 0;
        if (a0[q] + i < a1[q]) {
          if ((unsigned)j[q][i] >= (unsigned)B.rows) len[q][i] = -1;   // also a negative column
          else len[q][i] = __ldg(B.rp + j[q][i] + 1) - __ldg(B.rp + j[q][i]);
        }
      }
#pragma unroll
    for (int q = 0; q < BIN_ROWS; ++q) {
      long long u = 0;
      bool rowbad = false;   // an entry of A outside B's rows, or a decreasing row pointer
#pragma unroll
      for (int i = 0; i < BIN_EPR; ++i) {
        if (len[q][i] < 0) rowbad = true; else u += len[q][i];
      }
      if (a1[q] - a0[q] > BIN_EPR) {
        const long long t = bin_tail(A, B, a0[q] + BIN_EPR, a1[q]);
        if (t < 0) rowbad = true; else u += t;
      }
      int c = -1;
      if (r[q] >= 0 && (rowbad || a1[q] < a0[q])) {
        // no class: the class kernels would address B's row pointer with the invalid entry
        bad = true;
        cls[r[q]] = (uint8_t)CLS_NONE;
      } else if (r[q] >= 0) {
        const int k = a1[q] - a0[q];
        if (k <= lim.merge_k && u <= lim.m1_u) c = CLS_M1;
        else if (k <= lim.merge_k && u <= lim.m2_u) c = CLS_M2;
        else if (u <= lim.warp_u) c = CLS_W;
        else if (u <= lim.block_u) c = CLS_B;
        else c = CLS_G;
        cls[r[q]] = (uint8_t)c;
        F += u;
        umax = max(umax, u);
        if (c == CLS_M1 || c == CLS_M2) umax_merge = max(umax_merge, (int)u);
        if (c == CLS_W) umax_w = max(umax_w, (int)u);
        if (c == CLS_B) umax_b = max(umax_b, (int)u);
      }
      // listed classes (the rare long rows): warp-aggregated appends; the others are only counted
#pragma unroll
      for (int cc = 0; cc < NUM_CLS; ++cc) {
        if (lists[cc]) {
          const unsigned mask = __ballot_sync(FULL, c == cc);
          if (mask) {
            const int leader = __ffs(mask) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(&ctr->count[cc], __popc(mask));
            base = __shfl_sync(FULL, base, leader);
            if (c == cc) lists[cc][base + __popc(mask & lanemask_lt())] = r[q];
          }
        } else {
          cnt[cc] += (c == cc);
        }
      }
    }
  }
  // block totals, then one global atomic of each per block
  __shared__ long long s_F[BIN_THREADS / 32], s_umax[BIN_THREADS / 32];
  __shared__ int s_um[BIN_THREADS / 32], s_uw[BIN_THREADS / 32], s_ub[BIN_THREADS / 32], s_cnt[BIN_THREADS / 32][NUM_CLS];
  const int w = threadIdx.x >> 5;
  const long long wF = warp_sum_ll(F);
  long long wm = umax;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) wm = max(wm, __shfl_xor_sync(FULL, wm, d));
  const int wum = __reduce_max_sync(FULL, umax_merge);
  const int wuw = __reduce_max_sync(FULL, umax_w);
  const int wub = __reduce_max_sync(FULL, umax_b);
  int wc[NUM_CLS];
#pragma unroll
  for (int cc = 0; cc < NUM_CLS; ++cc) wc[cc] = __reduce_add_sync(FULL, cnt[cc]);
  if (__any_sync(FULL, bad) && lane == 0) atomicOr(&ctr->status, ST_INVALID);
  if (lane == 0) {
    s_F[w] = wF; s_umax[w] = wm; s_um[w] = wum; s_uw[w] = wuw; s_ub[w] = wub;
#pragma unroll
    for (int cc = 0; cc < NUM_CLS; ++cc) s_cnt[w][cc] = wc[cc];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0, mx = 0;
    int mm = 0, mw = 0, mb = 0;
    for (int i = 0; i < BIN_THREADS / 32; ++i) {
      t += s_F[i]; mx = max(mx, s_umax[i]); mm = max(mm, s_um[i]); mw = max(mw, s_uw[i]); mb = max(mb, s_ub[i]);
    }
    if (t) atomicAdd(&ctr->F, (unsigned long long)t);
    if (mm > 0) atomicMax(&ctr->max_u_merge, mm);
    if (mw > 0) atomicMax(&ctr->max_u_w, mw);
    if (mb > 0) atomicMax(&ctr->max_u_b, mb);
    if (mx > INT_MAX) { atomicOr(&ctr->status, ST_OVERFLOW); mx = INT_MAX; }
    if (mx > 0) atomicMax(&ctr->max_u, (int)mx);
  }
  if (threadIdx.x < NUM_CLS && !lists[threadIdx.x]) {
    int t = 0;
    for (int i = 0; i < BIN_THREADS / 32; ++i) t += s_cnt[i][threadIdx.x];
    if (t) atomicAdd(&ctr->count[threadIdx.x], t);
  }
}

void launch_bin(const DevCsr& A, const DevCsr& B, const Limits& lim_in, uint8_t* cls, int* const lists[NUM_CLS],
                Counters* ctr, cudaStream_t s, unsigned long long* zero, long long nzero) {
  if (A.rows <= 0) return;
  Limits lim = lim_in;
  if (B.cols > merge_max_cols()) { lim.m1_u = -1; lim.m2_u = -1; }   // sort keys hold column << log2(N)
  const int per_sm = blocks_per_sm((const void*)k_bin, BIN_THREADS, 0);
  const long long need = ((long long)A.rows + (long long)BIN_THREADS * BIN_ROWS - 1) / ((long long)BIN_THREADS * BIN_ROWS);
  const int grid = (int)std::max(1LL, std::min(need, (long long)num_sms() * per_sm));
  k_bin<<<grid, BIN_THREADS, 0, s>>>(A, B, lim, cls, lists[0], lists[1], lists[2], lists[3], lists[4], ctr, zero,
                                     zero ? nzero : 0);
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
      rp[idx] = (int)(e > INT_MAX ? (long long)INT_MAX : e);   // clamped when it does not fit
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
