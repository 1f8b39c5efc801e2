// a2 symbolic and a4 numeric for rows too long for the merge classes.
//
// Class W (a warp per row, up to 1024 products) stages the row's products in
// shared memory and orders them per row by the cheapest of three ways: a bit
// vector over the row's column range, a register sort across the warp, or a
// hash table (details at k_warp_row).  Class B (a 512-thread block per row,
// 8192-slot table) replaces the dense temporary vector of the row-major
// algorithm (Section IV-A) with an open-addressing hash table in shared memory
// (linear probing, bounded to the table size); its numeric pass orders the
// touched columns -- the "Sort" store of Section IV-B -- with a bitonic sort of
// the compacted table, and appends the row to C.
//
// Class G (rows beyond the block table) uses the dense temporary vector itself,
// one per CTA in global memory, scanned over [min, max] of the touched columns
// in ascending order: the "MinMax" store of Section IV-B.  Flags mark touched
// positions, so entries that cancel to 0.0 are kept.
#include "internal.h"

namespace spg {

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

// ---------------------------------------------------------------------------
// Class W: one warp per row, up to WR_UMAX products.  The row's products are staged in shared
// memory (a_rj * b_jx computed there, lane-parallel); then, when the row's columns span at most
// WR_RANGE values, a bit vector over [min, max] orders them -- the "Brute Force"-bool lookup
// vector of Section IV-B restricted to the MinMax range: per-word prefix popcounts give every
// column its rank, values are summed at their rank, and the columns come out ascending by
// scanning the bits.  Wider rows use a hash table sized to the row, compacted in place and sorted
// by a bitonic network over the distinct columns only.
// ---------------------------------------------------------------------------
constexpr int WR_UMAX = 1024;   // the largest bound U of the W kernels
constexpr int WR_RANGE = 65536;
constexpr int WR_WARPS = 2;

// Bitonic sort of 32*E keys held E per lane: after it, lane l holds sorted positions l*E .. l*E+E-1.
// Stages with stride < E stay inside a lane (static register indices); wider ones exchange with
// lane ^ (stride / E) by shuffles.
template <int E>
__device__ __forceinline__ void warp_bitonic(unsigned (&k)[E]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int size = 2; size <= 32 * E; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      if (stride >= E) {
        const int lm = stride / E;
        const bool lower = (lane & lm) == 0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const unsigned other = __shfl_xor_sync(FULL, k[e], lm);
          const bool up = ((lane * E + e) & size) == 0;
          k[e] = (up == lower) ? min(k[e], other) : max(k[e], other);
        }
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          if ((e & stride) == 0) {
            const int f = e | stride;
            const bool up = ((lane * E + e) & size) == 0;
            const unsigned a = k[e], b = k[f];
            const unsigned lo = min(a, b), hi = max(a, b);
            k[e] = up ? lo : hi;
            k[f] = up ? hi : lo;
          }
        }
      }
    }
  }
}

// Product-index bits of a register-sort key over 32 * E products, and so the widest column range
// whose keys fit 32 bits below the pad: range < 2^(32 - bits).
__host__ __device__ constexpr int regsort_index_bits(int E) { return E <= 4 ? 7 : E <= 8 ? 8 : E <= 16 ? 9 : 10; }

// Register-sort mode of class W: keys (column - mn) << IB | product index (IB bits for the 32 * E
// products), sorted across the warp; each product's rank among the distinct columns comes from
// group-start flags; values are added at their rank.  Returns the number of distinct columns;
// writes the columns (ascending) to outc and their sums to sums (numeric).
template <int E, bool NUM>
__device__ __forceinline__ int warp_sort_rank(const int* s_col, const double* s_val, int u, int mn, int* outc,
                                              double* sums) {
  static_assert(E == 4 || E == 8 || E == 16 || E == 32, "32 * E products per warp");
  constexpr int IB = regsort_index_bits(E);
  constexpr unsigned IMASK = (1u << IB) - 1u;
  const int lane = threadIdx.x & 31;
  constexpr unsigned PAD = 0xffffffffu;
  unsigned k[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int g = e * 32 + lane;   // initial placement is free: read lane-contiguous (no bank conflicts)
    k[e] = g < u ? ((unsigned)(s_col[g] - mn) << IB) | (unsigned)g : PAD;
  }
  warp_bitonic<E>(k);
  // group starts: position p starts a new column if its column differs from position p-1's
  const unsigned prev_last = __shfl_up_sync(FULL, k[E - 1], 1);
  int starts = 0;
  bool st[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const unsigned pk = (e == 0) ? (lane == 0 ? PAD : prev_last) : k[e - 1];
    st[e] = k[e] != PAD && (lane * E + e == 0 || (k[e] >> IB) != (pk >> IB));
    starts += st[e];
  }
  int total;
  int rank = warp_excl_scan(starts, &total) - 1;
  if (NUM) {
    for (int q = lane; q < total; q += 32) sums[q] = 0.0;
    __syncwarp();
  }
#pragma unroll
  for (int e = 0; e < E; ++e) {
    if (k[e] != PAD) {
      rank += st[e];
      if (NUM) {
        if (st[e]) outc[rank] = mn + (int)(k[e] >> IB);
        atomicAdd(&sums[rank], s_val[k[e] & IMASK]);
      }
    }
  }
  __syncwarp();
  return total;
}

// Shared memory of one warp of the W kernel for rows of at most U products.  Every piece scales
// with U, so the rows of a matrix get the smallest footprint that holds its longest W row (and
// with it the most warps per SM).  Region, per mode (NUM / symbolic):
//   bit vector: bits uint[RW] @0, rank ushort[RW], sums double[U] (NUM)  -- RW = min(4U, WR_RANGE/32)
//   register sort: columns int[U] @0, sums double[U] (NUM only)
//   hash: vals double[2U] @0, keys int[2U] (NUM); keys int[2U] @0 (symbolic)
template <bool NUM, int U>
struct WarpRowSmem {
  static constexpr int RW = (4 * U < WR_RANGE / 32) ? 4 * U : WR_RANGE / 32;
  static constexpr int TMAX = 2 * U;
  static constexpr size_t s_val = 0;                                  // double [U] products
  static constexpr size_t s_col = s_val + (NUM ? 8 * U : 0);          // int    [U] columns
  static constexpr size_t region = s_col + 4 * U;
  static constexpr size_t bv_rank = 4 * RW;
  static constexpr size_t bv_sums = (6 * RW + 7) / 8 * 8;
  static constexpr size_t rs_sums = 4 * U;
  static constexpr size_t h_keys = NUM ? 8 * TMAX : 0;
  static constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
  static constexpr size_t region_bytes =
      NUM ? cmax(cmax(bv_sums + 8 * U, rs_sums + 8 * U), h_keys + 4 * TMAX) : cmax(4 * RW, 4 * TMAX);
  static constexpr size_t bytes = (region + region_bytes + 15) / 16 * 16;
};

__device__ __forceinline__ int warp_min_i(int v) { return __reduce_min_sync(FULL, v); }
__device__ __forceinline__ int warp_max_i(int v) { return __reduce_max_sync(FULL, v); }

template <bool NUM, int U>
__global__ void __launch_bounds__(WR_WARPS * 32, 1)
k_warp_row(DevCsr A, DevCsr B, const int* __restrict__ list, int count, int* __restrict__ rp,
           int* __restrict__ C_col, double* __restrict__ C_val, Counters* __restrict__ ctr, WarpOrder wo,
           const int* __restrict__ count_dev) {
  if (count_dev) count = *count_dev;   // the row count as the binning pass left it on the device
  using L = WarpRowSmem<NUM, U>;
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* wb = smem + (size_t)warp * L::bytes;
  double* s_val = reinterpret_cast<double*>(wb + L::s_val);
  int* s_col = reinterpret_cast<int*>(wb + L::s_col);
  unsigned char* reg = wb + L::region;
  for (int idx = blockIdx.x * WR_WARPS + warp; idx < count; idx += gridDim.x * WR_WARPS) {
    const int r = list[idx];
    const int a0 = __ldg(A.rp + r), a1 = __ldg(A.rp + r + 1);
    // 1. stage the products, 32 runs (entries of A) at a time
    int u = 0, mn = INT_MAX, mx = -1;
    bool over = false;
    for (int c0 = a0; c0 < a1; c0 += 32) {
      const int e = c0 + lane;
      int bs = 0, len = 0;
      double a = 0.0;
      if (e < a1) {
        const int j = __ldg(A.col + e);
        bs = __ldg(B.rp + j);
        len = __ldg(B.rp + j + 1) - bs;
        if (NUM) a = __ldg(A.val + e);
      }
      int tot;
      const int off = warp_excl_scan(len, &tot);
      if (u + tot > U) { over = true; break; }   // the launch picks U >= every W row: unreachable
      // WB chunks of 32 products at a time: their runs first, then all their loads in flight
      constexpr int WB = 4;
      for (int cb = 0; cb < tot; cb += 32 * WB) {
        int sp[WB];
        double at[WB];
#pragma unroll
        for (int v = 0; v < WB; ++v) {
          const int q = cb + 32 * v + lane;
          int t = 0;   // last run whose offset is <= q (empty runs share the next run's offset)
#pragma unroll
          for (int step = 16; step > 0; step >>= 1) {
            const int cnd = t + step;
            if (__shfl_sync(FULL, off, cnd) <= q) t = cnd;
          }
          sp[v] = __shfl_sync(FULL, bs, t) + (q - __shfl_sync(FULL, off, t));
          at[v] = NUM ? __shfl_sync(FULL, a, t) : 0.0;
        }
        int x[WB];
        double b[WB];
#pragma unroll
        for (int v = 0; v < WB; ++v) {
          const int q = cb + 32 * v + lane;
          x[v] = q < tot ? __ldg(B.col + sp[v]) : 0;
          b[v] = (NUM && q < tot) ? __ldg(B.val + sp[v]) : 0.0;
        }
#pragma unroll
        for (int v = 0; v < WB; ++v) {
          const int q = cb + 32 * v + lane;
          if (q < tot) {
            s_col[u + q] = x[v];
            if (NUM) s_val[u + q] = __dmul_rn(at[v], b[v]);
            mn = min(mn, x[v]);
            mx = max(mx, x[v]);
          }
        }
      }
      u += tot;
    }
    if (over) {
      if (lane == 0) atomicOr(&ctr->status, ST_TABLE_FULL);
      continue;
    }
    mn = warp_min_i(mn);
    mx = warp_max_i(mx);
    __syncwarp();
    int cnt = 0;
    int g0 = 0, g1 = 0;
    if (NUM) { g0 = __ldg(rp + r); g1 = __ldg(rp + r + 1); }
    const long long range = (long long)mx - (long long)mn + 1;
    // Choice of ordering (the "Combined" idea of Section IV-B): the bit vector when the column
    // range is small next to the row (at most wo.bitvec_ratio columns per product, at most 128,
    // which is 4u words), a register sort when the keys fit 32 bits, a hash table otherwise.  The
    // sort's index takes 7 to 10 bits (by the sort size that holds u), so its keys fit ranges
    // below 2^25 to 2^22; in the automatic choice, past 2^22 it is taken only for rows of more
    // than 32 products: a row of at most 32 products inserts into the hash table in one step,
    // cheaper there than a sort of 128 keys (measured on random rows of 16 products over 10^7
    // columns: 21.0 ms by hash, 25.0 ms by sort).  wo.order forces one of the three where it fits.
    const bool bv_fits = range <= WR_RANGE && ((range + 31) >> 5) <= 4 * (long long)u;   // words <= 4u <= RW
    const int ib = regsort_index_bits(u <= 128 ? 4 : u <= 256 ? 8 : u <= 512 ? 16 : 32);
    const bool rs_fits = range < (1LL << (32 - ib));
    bool bitvec, regsort;
    if (wo.order == 1) {
      bitvec = bv_fits;
      regsort = !bitvec && rs_fits;
    } else if (wo.order == 2) {
      regsort = rs_fits;
      bitvec = !regsort && bv_fits;
    } else if (wo.order == 3) {
      bitvec = regsort = false;
    } else {
      bitvec = bv_fits && range <= (long long)wo.bitvec_ratio * u;
      regsort = !bitvec && (range < (1 << 22) || (u > 32 && rs_fits));
    }
    if (u > 0 && regsort) {
      int* outc = reinterpret_cast<int*>(reg);
      double* sums = reinterpret_cast<double*>(reg + L::rs_sums);
      if (u <= 128) cnt = warp_sort_rank<4, NUM>(s_col, s_val, u, mn, outc, sums);
      else if constexpr (U >= 256) {
        if (u <= 256) cnt = warp_sort_rank<8, NUM>(s_col, s_val, u, mn, outc, sums);
        else if constexpr (U >= 512) {
          if (u <= 512) cnt = warp_sort_rank<16, NUM>(s_col, s_val, u, mn, outc, sums);
          else cnt = warp_sort_rank<32, NUM>(s_col, s_val, u, mn, outc, sums);
        }
      }
      if (NUM) {
        if (lane == 0 && g1 - g0 != cnt) atomicOr(&ctr->status, ST_MISMATCH);
        for (int q = lane; q < cnt && g0 + q < g1; q += 32) {
          C_col[g0 + q] = outc[q];
          C_val[g0 + q] = sums[q];
        }
      }
    } else if (u > 0 && bitvec) {
      // 2a. bit vector over [mn, mx]
      unsigned* bits = reinterpret_cast<unsigned*>(reg);
      unsigned short* rank = reinterpret_cast<unsigned short*>(reg + L::bv_rank);
      const int W = (int)((range + 31) >> 5);
      for (int w = lane; w < W; w += 32) bits[w] = 0u;
      __syncwarp();
      for (int q = lane; q < u; q += 32) {
        const int d = s_col[q] - mn;
        atomicOr(&bits[d >> 5], 1u << (d & 31));
      }
      __syncwarp();
      int base = 0;
      for (int w0 = 0; w0 < W; w0 += 32) {
        const int w = w0 + lane;
        const unsigned b = w < W ? bits[w] : 0u;
        int t2;
        const int ex = warp_excl_scan(__popc(b), &t2);
        if (NUM && w < W) rank[w] = (unsigned short)(base + ex);
        base += t2;
      }
      cnt = base;
      if (NUM) {
        double* sums = reinterpret_cast<double*>(reg + L::bv_sums);
        for (int q = lane; q < cnt; q += 32) sums[q] = 0.0;
        __syncwarp();
        for (int q = lane; q < u; q += 32) {
          const int d = s_col[q] - mn;
          const int w = d >> 5;
          const int k = rank[w] + __popc(bits[w] & ((1u << (d & 31)) - 1u));
          atomicAdd(&sums[k], s_val[q]);
        }
        __syncwarp();
        if (lane == 0 && g1 - g0 != cnt) atomicOr(&ctr->status, ST_MISMATCH);
        for (int w0 = 0; w0 < W; w0 += 32) {
          const int w = w0 + lane;
          unsigned b = w < W ? bits[w] : 0u;
          int k = w < W ? (int)rank[w] : 0;
          while (b) {
            const int bit = __ffs(b) - 1;
            b &= b - 1;
            if (k < g1 - g0) {
              C_col[g0 + k] = mn + (w << 5) + bit;
              C_val[g0 + k] = sums[k];
            }
            ++k;
          }
        }
      }
    } else if (u > 0) {
      // 2b. hash table of T = pow2 >= 2u slots
      int logT = 6;
      while ((1 << logT) < 2 * u) ++logT;
      const int T = 1 << logT;
      int* keys = reinterpret_cast<int*>(reg + L::h_keys);
      double* vals = reinterpret_cast<double*>(reg);
      for (int i = lane; i < T; i += 32) { keys[i] = KEY_NONE; if (NUM) vals[i] = 0.0; }
      __syncwarp();
      int mine = 0;
      bool full = false;
      for (int q = lane; q < u; q += 32) {
        bool fresh;
        const int slot = hash_insert(keys, s_col[q], (unsigned)logT, &fresh);
        if (slot < 0) { full = true; continue; }
        mine += fresh;
        if (NUM) atomicAdd(&vals[slot], s_val[q]);
      }
      if (__any_sync(FULL, full) && lane == 0) atomicOr(&ctr->status, ST_TABLE_FULL);
      cnt = __reduce_add_sync(FULL, mine);
      __syncwarp();
      if (NUM) {
        // compact in slot order (in place: every entry moves down), then sort the distinct columns
        int wr = 0;
        for (int i0 = 0; i0 < T; i0 += 32) {
          const int i = i0 + lane;
          const int k = keys[i];
          const double v = vals[i];
          const bool valid = k != KEY_NONE;
          const unsigned m = __ballot_sync(FULL, valid);
          const int pos = wr + __popc(m & lanemask_lt());
          __syncwarp();
          if (valid) { keys[pos] = k; vals[pos] = v; }
          wr += __popc(m);
          __syncwarp();
        }
        int n2 = 1;
        while (n2 < cnt) n2 <<= 1;
        for (int i = cnt + lane; i < n2; i += 32) { keys[i] = KEY_NONE; vals[i] = 0.0; }
        __syncwarp();
        for (int kk = 2; kk <= n2; kk <<= 1) {
          for (int jj = kk >> 1; jj > 0; jj >>= 1) {
            for (int i = lane; i < n2; i += 32) {
              const int ixj = i ^ jj;
              if (ixj > i) {
                const int ki = keys[i], kj = keys[ixj];
                if ((ki > kj) == ((i & kk) == 0)) {
                  keys[i] = kj; keys[ixj] = ki;
                  const double t = vals[i]; vals[i] = vals[ixj]; vals[ixj] = t;
                }
              }
            }
            __syncwarp();
          }
        }
        if (lane == 0 && g1 - g0 != cnt) atomicOr(&ctr->status, ST_MISMATCH);
        for (int i = lane; i < cnt && g0 + i < g1; i += 32) {
          C_col[g0 + i] = keys[i];
          C_val[g0 + i] = vals[i];
        }
      }
    } else if (NUM && lane == 0 && g1 != g0) {
      atomicOr(&ctr->status, ST_MISMATCH);
    }
    if (!NUM && lane == 0) rp[r] = cnt;
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Class B: one block of 512 threads per row, its columns ordered by a bit vector -- the MinMax
// store of Section IV-B with the flags as bits, kept in shared memory; no hash table, no sort.
// The bit vector covers a window of columns above the row's smallest column not yet done: all of B
// when B has at most BB_WINDOW columns, else BB_WIDE_WINDOW columns (a block then holds little
// shared memory and many blocks fit an SM); a row whose columns span more is done window by window,
// each window starting at the smallest column past the last.  Per window:
//   1. mark  -- each product in the window sets its column's bit (a warp per entry of A, lanes
//               along the row of B); the window's largest column and the next window's first
//               column come out of the same pass;
//   2. rank  -- the words up to the largest are ranked by a block prefix of their popcounts,
//               512 words per round;
//   3. sum   -- numeric: every product a_rj * b_jx in the window is added to sums[rank of its
//               column] (products rounded on their own, added in no fixed order);
//   4. write -- the set bits, walked in order, give the window's entries of C, columns ascending,
//               after the entries of the windows before it.
// Sums hold up to BB_MAX_U entries per window; class B rows have at most that many products.  When
// B has at most BB_WINDOW columns the window starts at column 0 and the first pass (the row's
// smallest column) is skipped.
// ---------------------------------------------------------------------------
constexpr int BB_WINDOW = 1 << 18;        // B up to this many columns: one window over all of B
constexpr int BB_WIDE_WINDOW = 1 << 16;   // wider B: windows of this many columns
constexpr int BB_MAX_WARPS = 16;     // the largest block: 512 threads

// words of the bit vector: all of B's columns when they are at most BB_WINDOW, else BB_WIDE_WINDOW
__host__ __device__ inline int bb_words(int ncols) {
  const int n = ncols < 1 ? 1 : ncols;
  return ((n <= (1 << 18) ? n : (1 << 16)) + 31) / 32;
}

size_t block_bitvec_smem(int ncols, int sums, bool num) {
  const size_t words = (size_t)bb_words(ncols);
  return (num ? 8 * (size_t)sums : 0) + 4 * words + (2 * words + 15) / 16 * 16 + 4 * 4 * BB_MAX_WARPS;
}

// Block minimum and maximum (reduction slots red[0 .. 2 * BB_WARPS)).
template <int BB_WARPS>
__device__ __forceinline__ void bb_minmax(int& mn, int& mx, int* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  mn = __reduce_min_sync(FULL, mn);
  mx = __reduce_max_sync(FULL, mx);
  if (lane == 0) { red[warp] = mn; red[BB_WARPS + warp] = mx; }
  __syncthreads();
  mn = INT_MAX; mx = INT_MIN;
#pragma unroll
  for (int i = 0; i < BB_WARPS; ++i) { mn = min(mn, red[i]); mx = max(mx, red[BB_WARPS + i]); }
  __syncthreads();   // red is reused
}

template <bool NUM, int BB_THREADS>
__global__ void __launch_bounds__(BB_THREADS)
k_block_bitvec(DevCsr A, DevCsr B, const int* __restrict__ list, int count, int sums_cap, int* __restrict__ rp,
               int* __restrict__ C_col, double* __restrict__ C_val, Counters* __restrict__ ctr,
               const int* __restrict__ count_dev) {
  if (count_dev) count = *count_dev;   // the row count as the binning pass left it on the device
  if ((int)blockIdx.x >= count) return;   // no row for this block (uniform)
  constexpr int BB_WARPS = BB_THREADS / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  const int W = bb_words(B.cols);
  double* sums = reinterpret_cast<double*>(smem);                                          // [sums_cap] (NUM)
  unsigned* bits = reinterpret_cast<unsigned*>(smem + (NUM ? 8 * (size_t)sums_cap : 0));   // [W]
  unsigned short* rank = reinterpret_cast<unsigned short*>(bits + W);                      // [W]
  int* red = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(rank) + ((size_t)2 * W + 15) / 16 * 16);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool one_window = B.cols <= BB_WINDOW;
  const int win = one_window ? 32 * W : BB_WIDE_WINDOW;   // columns per window
  for (int w = tid; w < W; w += BB_THREADS) bits[w] = 0u;
  __syncthreads();
  for (int idx = blockIdx.x; idx < count; idx += gridDim.x) {
    const int r = list[idx];
    const int a0 = __ldg(A.rp + r), a1 = __ldg(A.rp + r + 1);
    int g0 = 0, g1 = 0;
    if (NUM) { g0 = __ldg(rp + r); g1 = __ldg(rp + r + 1); }
    // the first window's start: column 0, or the row's smallest column
    int lo = 0;
    bool bad = false;
    if (!one_window) {
      int mn = INT_MAX, mx = INT_MIN;
      for (int e = a0 + warp; e < a1; e += BB_WARPS) {
        const int j = __ldg(A.col + e);
        const int bs = __ldg(B.rp + j), be = __ldg(B.rp + j + 1);
        for (int q = bs + lane; q < be; q += 32) mn = min(mn, __ldg(B.col + q));
      }
      bb_minmax<BB_WARPS>(mn, mx, red);
      lo = mn;
    }
    int done = 0;   // entries of the row in the windows before this one
    while (lo != INT_MAX) {   // block-uniform
      const long long hi = (long long)lo + win;   // window [lo, hi)
      // 1. mark
      int wmax = INT_MIN, next = INT_MAX;
      for (int e = a0 + warp; e < a1; e += BB_WARPS) {
        const int j = __ldg(A.col + e);
        const int bs = __ldg(B.rp + j), be = __ldg(B.rp + j + 1);
        for (int q = bs + lane; q < be; q += 32) {
          const int c = __ldg(B.col + q);
          if ((unsigned)c >= (unsigned)B.cols) { bad = true; continue; }
          if (c < lo) continue;
          if (c >= hi) { next = min(next, c); continue; }
          const int d = c - lo;
          atomicOr(&bits[d >> 5], 1u << (d & 31));
          wmax = max(wmax, d);
        }
      }
      {
        int nmin = next, wmx = wmax;
        bb_minmax<BB_WARPS>(nmin, wmx, red);   // red[0..]: next window (min), this window's largest (max)
        next = nmin;
        wmax = wmx;
      }
      const int whi = wmax >= 0 ? wmax >> 5 : -1;
      // 2. rank the words 0 .. whi
      int total = 0;
      for (int wb = 0; wb <= whi; wb += BB_THREADS) {
        const int w = wb + tid;
        const int pc = w <= whi ? __popc(bits[w]) : 0;
        int incl = pc;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const int y = __shfl_up_sync(FULL, incl, d);
          if (lane >= d) incl += y;
        }
        if (lane == 31) red[2 * BB_WARPS + warp] = incl;
        __syncthreads();
        int woff = 0, round = 0;
#pragma unroll
        for (int i = 0; i < BB_WARPS; ++i) {
          const int t = red[2 * BB_WARPS + i];
          woff += i < warp ? t : 0;
          round += t;
        }
        if (NUM && w <= whi) rank[w] = (unsigned short)(total + woff + incl - pc);
        total += round;
        __syncthreads();   // red is rewritten by the next round
      }
      if (NUM) {
        if (total > sums_cap) {
          if (tid == 0) atomicOr(&ctr->status, ST_TABLE_FULL);   // the launch sizes sums for every row
        } else {
          // 3. sums
          for (int i = tid; i < total; i += BB_THREADS) sums[i] = 0.0;
          __syncthreads();
          for (int e = a0 + warp; e < a1; e += BB_WARPS) {
            const int j = __ldg(A.col + e);
            const double a = __ldg(A.val + e);
            const int bs = __ldg(B.rp + j), be = __ldg(B.rp + j + 1);
            for (int q = bs + lane; q < be; q += 32) {
              const int c = __ldg(B.col + q);
              if ((unsigned)c >= (unsigned)B.cols || c < lo || c >= hi) continue;
              const int d = c - lo;
              const int w = d >> 5;
              const int k = rank[w] + __popc(bits[w] & ((1u << (d & 31)) - 1u));
              atomicAdd(&sums[k], __dmul_rn(a, __ldg(B.val + q)));
            }
          }
          __syncthreads();
          // 4. write, consecutive threads on consecutive words
          for (int w = tid; w <= whi; w += BB_THREADS) {
            unsigned b = bits[w];
            int k = rank[w];
            while (b) {
              const int bit = __ffs(b) - 1;
              b &= b - 1;
              const int o = done + k;
              if (o < g1 - g0) {
                C_col[g0 + o] = lo + (w << 5) + bit;
                C_val[g0 + o] = sums[k];
              }
              ++k;
            }
          }
        }
      }
      done += total;
      __syncthreads();
      for (int w = tid; w <= whi; w += BB_THREADS) bits[w] = 0u;
      __syncthreads();
      lo = next;
    }
    if (bad) atomicOr(&ctr->status, ST_INVALID);
    if (tid == 0) {
      if (!NUM) rp[r] = done;
      else if (g1 - g0 != done) atomicOr(&ctr->status, ST_MISMATCH);
    }
  }
}

// ---------------------------------------------------------------------------
// Class B, rows of up to BB_STAGE_U products: the same windowed bit vector, with the row's products
// staged in shared memory first.  The block reads the row's entries of A and the ranges of the rows
// of B they select once (a thread per entry), then copies every product's column (and, numeric, its
// product a_rj * b_jx) with a thread per product, all loads of the block in flight together; the
// mark and sum passes then read shared memory instead of repeating the dependent loads.  Ranks come
// from one block scan over runs of consecutive words, one run per thread (the runs have an odd
// length, so the 32 lanes of a warp read 32 different banks).  The sum pass also records each
// entry's column by its rank, so C is written (and the vector cleared) entry by entry, consecutive
// threads on consecutive entries of C, without walking the vector's words again.
// ---------------------------------------------------------------------------
constexpr int BB_STAGE_U = 2048;

// Shared memory of k_block_staged, in bytes: sums, products and the entries' columns (numeric),
// the products' columns, bits, reduction slots, ranks (numeric).  The entry tables of the staging
// step (a of the chunk's entries, starts, sources) are only needed before the windows: in the
// numeric kernel they share the space of the sums and of the entries' columns (36 KB for rows of
// up to 1024 products and windows of 2^16 columns, six blocks per SM), in the symbolic one they
// follow the bits.
struct StagedSmem {
  size_t sums, prod, ocol, sa, scol, bits, start, src, red, rank, bytes;
  __host__ __device__ StagedSmem(int words, int ucap, bool num, int threads) {
    const size_t u = (size_t)ucap, t = (size_t)threads;
    sums = 0;
    prod = sums + (num ? (8 * u > 8 * t ? 8 * u : 8 * t) : 0);
    ocol = prod + (num ? 8 * u : 0);
    scol = ocol + (num ? (4 * u > 8 * t ? 4 * u : 8 * t) : 0);
    scol = (scol + 7) / 8 * 8;
    bits = scol + 4 * u;
    red = bits + 4 * (size_t)words + (num ? 0 : 8 * t);
    rank = red + 4 * 4 * (t / 32);
    bytes = rank + (num ? 2 * (size_t)words : 0);
    sa = sums;                                       // numeric only
    start = num ? ocol : bits + 4 * (size_t)words;
    src = start + 4 * t;
  }
};

// Exclusive prefix of v over the block; *total gets the block's sum.  red: BB_WARPS ints.
template <int BB_WARPS>
__device__ __forceinline__ int bb_excl_scan(int v, int* red, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(FULL, incl, d);
    if (lane >= d) incl += y;
  }
  if (lane == 31) red[warp] = incl;
  __syncthreads();
  int woff = 0, sum = 0;
#pragma unroll
  for (int i = 0; i < BB_WARPS; ++i) {
    const int t = red[i];
    woff += i < warp ? t : 0;
    sum += t;
  }
  __syncthreads();   // red is reused
  *total = sum;
  return woff + incl - v;
}

template <bool NUM, int BB_THREADS>
__global__ void __launch_bounds__(BB_THREADS)
k_block_staged(DevCsr A, DevCsr B, const int* __restrict__ list, int count, int ucap, int* __restrict__ rp,
               int* __restrict__ C_col, double* __restrict__ C_val, Counters* __restrict__ ctr,
               const int* __restrict__ count_dev) {
  if (count_dev) count = *count_dev;   // the row count as the binning pass left it on the device
  if ((int)blockIdx.x >= count) return;   // no row for this block (uniform)
  constexpr int BB_WARPS = BB_THREADS / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  const int W = bb_words(B.cols);
  const StagedSmem L(W, ucap, NUM, BB_THREADS);
  double* sums = reinterpret_cast<double*>(smem + L.sums);      // [ucap]
  double* prod = reinterpret_cast<double*>(smem + L.prod);      // [ucap]
  int* ocol = reinterpret_cast<int*>(smem + L.ocol);            // [ucap] window column of entry k
  double* s_a = reinterpret_cast<double*>(smem + L.sa);         // [BB_THREADS]
  int* scol = reinterpret_cast<int*>(smem + L.scol);            // [ucap]
  unsigned* bits = reinterpret_cast<unsigned*>(smem + L.bits);  // [W]
  int* s_start = reinterpret_cast<int*>(smem + L.start);        // [BB_THREADS] an entry's first product
  int* s_src = reinterpret_cast<int*>(smem + L.src);            // [BB_THREADS] B index of product p, less p
  int* red = reinterpret_cast<int*>(smem + L.red);
  unsigned short* rank = reinterpret_cast<unsigned short*>(smem + L.rank);   // [W]
  const int tid = threadIdx.x;
  const bool one_window = B.cols <= BB_WINDOW;
  const int win = one_window ? 32 * W : BB_WIDE_WINDOW;
  for (int w = tid; w < W; w += BB_THREADS) bits[w] = 0u;
  __syncthreads();
  for (int idx = blockIdx.x; idx < count; idx += gridDim.x) {
    const int r = list[idx];
    const int a0 = __ldg(A.rp + r), a1 = __ldg(A.rp + r + 1);
    int g0 = 0, g1 = 0;
    if (NUM) { g0 = __ldg(rp + r); g1 = __ldg(rp + r + 1); }
    // 1. stage the products, BB_THREADS entries of A at a time
    int u = 0, mn = INT_MAX, mx = INT_MIN;
    bool bad = false, full = false;
    for (int e0 = a0; e0 < a1; e0 += BB_THREADS) {   // block-uniform
      const int e = e0 + tid;
      int len = 0, src = 0;
      if (e < a1) {
        const int j = __ldg(A.col + e);
        src = __ldg(B.rp + j);
        len = __ldg(B.rp + j + 1) - src;
        if (NUM) s_a[tid] = __ldg(A.val + e);
      }
      int chunk;
      const int off = bb_excl_scan<BB_WARPS>(len, red, &chunk);
      if (u + chunk > ucap) { full = true; break; }   // block-uniform; not within the class limit
      s_start[tid] = off;   // entries past the row start at `chunk`, above every product
      s_src[tid] = src - off;
      __syncthreads();
#pragma unroll 4
      for (int p = tid; p < chunk; p += BB_THREADS) {
        int i = 0;   // the last entry that starts at or before p
#pragma unroll
        for (int step = BB_THREADS / 2; step > 0; step >>= 1)
          if (s_start[i + step] <= p) i += step;
        const int q = s_src[i] + p;
        const int c = __ldg(B.col + q);
        scol[u + p] = c;
        if (NUM) prod[u + p] = __dmul_rn(s_a[i], __ldg(B.val + q));
        if ((unsigned)c >= (unsigned)B.cols) bad = true;
        else { mn = min(mn, c); mx = max(mx, c); }
      }
      u += chunk;
      __syncthreads();   // the entry tables are rewritten by the next chunk
    }
    if (full && tid == 0) atomicOr(&ctr->status, ST_TABLE_FULL);
    bb_minmax<BB_WARPS>(mn, mx, red);
    int lo = (mn == INT_MAX || full) ? INT_MAX : (one_window ? 0 : mn);
    int done = 0;   // entries of the row in the windows before this one
    while (lo != INT_MAX) {   // block-uniform
      const long long hi = (long long)lo + win;   // window [lo, hi)
      // 2. mark
      int wmax = INT_MIN, next = INT_MAX;
      for (int p = tid; p < u; p += BB_THREADS) {
        const int c = scol[p];
        if ((unsigned)c >= (unsigned)B.cols || c < lo) continue;
        if (c >= hi) { next = min(next, c); continue; }
        const int d = c - lo;
        atomicOr(&bits[d >> 5], 1u << (d & 31));
        wmax = max(wmax, d);
      }
      bb_minmax<BB_WARPS>(next, wmax, red);
      const int nw = wmax >= 0 ? (wmax >> 5) + 1 : 0;   // words holding the window's columns
      // 3. rank: thread t owns the cw words from t * cw (cw odd: the lanes of a warp on 32 banks)
      const int cw = ((nw + BB_THREADS - 1) / BB_THREADS) | 1;
      const int w0 = min(nw, tid * cw), w1 = min(nw, w0 + cw);
      int pc = 0;
      for (int w = w0; w < w1; ++w) pc += __popc(bits[w]);
      int total;
      int run = bb_excl_scan<BB_WARPS>(pc, red, &total);
      if (NUM) {
        for (int w = w0; w < w1; ++w) {
          rank[w] = (unsigned short)run;
          run += __popc(bits[w]);
        }
        for (int i = tid; i < total; i += BB_THREADS) sums[i] = 0.0;
        __syncthreads();
        // 4. sums (products rounded on their own, added in no fixed order); every product of an
        //    entry records the entry's window column
        for (int p = tid; p < u; p += BB_THREADS) {
          const int c = scol[p];
          if ((unsigned)c >= (unsigned)B.cols || c < lo || c >= hi) continue;
          const int d = c - lo;
          const int w = d >> 5;
          const int k = rank[w] + __popc(bits[w] & ((1u << (d & 31)) - 1u));
          ocol[k] = d;
          atomicAdd(&sums[k], prod[p]);
        }
        __syncthreads();
        // 5. write entry by entry, consecutive threads on consecutive entries; clear the words
        for (int k = tid; k < total; k += BB_THREADS) {
          const int d = ocol[k];
          const int o = done + k;
          if (o < g1 - g0) {
            C_col[g0 + o] = lo + d;
            C_val[g0 + o] = sums[k];
          }
          bits[d >> 5] = 0u;
        }
      } else {
        for (int w = w0; w < w1; ++w) bits[w] = 0u;   // after the scan: every popcount is taken
      }
      done += total;
      __syncthreads();
      lo = next;
    }
    if (bad) atomicOr(&ctr->status, ST_INVALID);
    if (tid == 0 && !full) {
      if (!NUM) rp[r] = done;
      else if (g1 - g0 != done) atomicOr(&ctr->status, ST_MISMATCH);
    }
  }
}

template <bool NUM, int THREADS>
static void launch_block_staged_t(const DevCsr& A, const DevCsr& B, const int* list, int count, int ucap, int* rp,
                                  int* C_col, double* C_val, Counters* ctr, cudaStream_t s, const int* count_dev) {
  const size_t bytes = StagedSmem(bb_words(B.cols), ucap, NUM, THREADS).bytes;
  auto kern = k_block_staged<NUM, THREADS>;
  const int per_sm = blocks_per_sm((const void*)kern, THREADS, bytes);
  const int blocks = std::max(1, std::min(count, num_sms() * std::max(per_sm, 1)));
  kern<<<blocks, THREADS, bytes, s>>>(A, B, list, count, ucap, rp, C_col, C_val, ctr, count_dev);
}

template <bool NUM, int THREADS>
static void launch_block_bitvec_t(const DevCsr& A, const DevCsr& B, const int* list, int count, int sums_cap, int* rp,
                                  int* C_col, double* C_val, Counters* ctr, cudaStream_t s, const int* count_dev) {
  const size_t bytes = block_bitvec_smem(B.cols, sums_cap, NUM);
  auto kern = k_block_bitvec<NUM, THREADS>;
  const int per_sm = blocks_per_sm((const void*)kern, THREADS, bytes);
  const int blocks = std::max(1, std::min(count, num_sms() * per_sm));
  kern<<<blocks, THREADS, bytes, s>>>(A, B, list, count, sums_cap, rp, C_col, C_val, ctr, count_dev);
}

// The block takes about eight products per thread: 128 threads for rows of up to 1024 products,
// 256 up to 2048 (both staged), 512 beyond (umax: the longest row of the launch).  The structure
// pass of rows of up to 1024 products runs 64 threads a row (about sixteen products each): 24.3 against
// 25.2 ms for the batched workload, where 32 threads, 256, or 64 for the value pass too were slower.
template <bool NUM>
static void launch_block_bitvec(const DevCsr& A, const DevCsr& B, const int* list, int count, int umax, int* rp,
                                int* C_col, double* C_val, Counters* ctr, cudaStream_t s, const int* count_dev) {
  if (count <= 0) return;
  const int sums_cap = std::max(1, std::min(umax, BB_MAX_U));
  if (umax <= 1024 && !NUM) launch_block_staged_t<NUM, 64>(A, B, list, count, sums_cap, rp, C_col, C_val, ctr, s, count_dev);
  else if (umax <= 1024) launch_block_staged_t<NUM, 128>(A, B, list, count, sums_cap, rp, C_col, C_val, ctr, s, count_dev);
  else if (umax <= BB_STAGE_U) launch_block_staged_t<NUM, 256>(A, B, list, count, sums_cap, rp, C_col, C_val, ctr, s, count_dev);
  else launch_block_bitvec_t<NUM, 512>(A, B, list, count, sums_cap, rp, C_col, C_val, ctr, s, count_dev);
}

template <bool NUM, int U>
static void launch_warp_row_u(const DevCsr& A, const DevCsr& B, const int* list, int count, int* rp, int* C_col,
                              double* C_val, Counters* ctr, cudaStream_t s, WarpOrder wo, const int* count_dev) {
  constexpr size_t bytes = (size_t)WR_WARPS * WarpRowSmem<NUM, U>::bytes;
  auto kern = k_warp_row<NUM, U>;
  const int per_sm = blocks_per_sm((const void*)kern, WR_WARPS * 32, bytes);
  const int blocks = std::max(1, std::min((count + WR_WARPS - 1) / WR_WARPS, num_sms() * per_sm));
  kern<<<blocks, WR_WARPS * 32, bytes, s>>>(A, B, list, count, rp, C_col, C_val, ctr, wo, count_dev);
}

// umax: the longest W row (products); the smallest bound U >= umax is launched
template <bool NUM>
static void launch_warp_row(const DevCsr& A, const DevCsr& B, const int* list, int count, int umax, int* rp,
                            int* C_col, double* C_val, Counters* ctr, cudaStream_t s, WarpOrder wo,
                            const int* count_dev) {
  if (count <= 0) return;
  wo.bitvec_ratio = std::max(1, std::min(wo.bitvec_ratio, 128));
  if (umax <= 128) launch_warp_row_u<NUM, 128>(A, B, list, count, rp, C_col, C_val, ctr, s, wo, count_dev);
  else if (umax <= 256) launch_warp_row_u<NUM, 256>(A, B, list, count, rp, C_col, C_val, ctr, s, wo, count_dev);
  else launch_warp_row_u<NUM, WR_UMAX>(A, B, list, count, rp, C_col, C_val, ctr, s, wo, count_dev);
}

void launch_hash_symbolic(int cls, const DevCsr& A, const DevCsr& B, const int* list, int count, int* counts,
                          Counters* ctr, cudaStream_t s, int umax, WarpOrder wo, const int* count_dev) {
  if (cls == CLS_W) launch_warp_row<false>(A, B, list, count, umax, counts, nullptr, nullptr, ctr, s, wo, count_dev);
  else launch_block_bitvec<false>(A, B, list, count, umax, counts, nullptr, nullptr, ctr, s, count_dev);
}

void launch_hash_numeric(int cls, const DevCsr& A, const DevCsr& B, const int* list, int count, const int* rp,
                         int* C_col, double* C_val, Counters* ctr, cudaStream_t s, int umax, WarpOrder wo,
                         const int* count_dev) {
  if (cls == CLS_W)
    launch_warp_row<true>(A, B, list, count, umax, const_cast<int*>(rp), C_col, C_val, ctr, s, wo, count_dev);
  else launch_block_bitvec<true>(A, B, list, count, umax, const_cast<int*>(rp), C_col, C_val, ctr, s, count_dev);
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
        Counters* __restrict__ ctr, const int* __restrict__ count_dev, bool zero_slab) {
  __shared__ int s_a[32], s_b[32], s_c[32];
  __shared__ int s_scan[32];
  if (count_dev) count = *count_dev;   // the row count as the binning pass left it on the device
  const int n = B.cols;
  double* acc = reinterpret_cast<double*>(slabs + blockIdx.x * slab_bytes);
  int* flag = reinterpret_cast<int*>(acc + n);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (zero_slab && (int)blockIdx.x < count) {   // a slab not known to be clear: clear it before its first row
    for (int x = threadIdx.x; x < n; x += G_THREADS) { acc[x] = 0.0; flag[x] = 0; }
    __syncthreads();
  }
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
                           int* counts, Counters* ctr, cudaStream_t s, const int* count_dev, bool zero_slabs) {
  if (count <= 0 || nslabs <= 0) return;
  const int blocks = std::min(count, nslabs);
  k_dense<false><<<blocks, G_THREADS, 0, s>>>(A, B, list, count, (unsigned char*)slabs, dense_slab_bytes(B.cols),
                                              counts, nullptr, nullptr, nullptr, ctr, count_dev, zero_slabs);
}

void launch_dense_numeric(const DevCsr& A, const DevCsr& B, const int* list, int count, void* slabs, int nslabs,
                          const int* rp, int* C_col, double* C_val, Counters* ctr, cudaStream_t s,
                          const int* count_dev) {
  if (count <= 0 || nslabs <= 0) return;
  const int blocks = std::min(count, nslabs);
  k_dense<true><<<blocks, G_THREADS, 0, s>>>(A, B, list, count, (unsigned char*)slabs, dense_slab_bytes(B.cols),
                                             nullptr, rp, C_col, C_val, ctr, count_dev, false);
}

}  // namespace spg
