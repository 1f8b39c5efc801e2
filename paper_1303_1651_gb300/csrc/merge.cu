// a2 symbolic and a4 numeric for rows with few, short contributions (classes M1, M2).
//
// The row-major algorithm of Section IV-A builds row r of C from the rows B_j
// (j in row r of A) scaled by a_rj.  With every B_j sorted by column, row r of
// C is the merge of those k sorted runs, and merging produces the columns in
// ascending order directly -- the "Sort" store of Section IV-B without a sort,
// and the paper's future-work item of a cheaper ordering for short lists.
//
// One warp owns a tile of 32 consecutive rows; lane t owns row tile*32+t.
//   1. run table   -- lane t gathers its <= 8 runs (A entry -> B row range).
//   2. expand      -- the warp copies every run element into shared memory with
//                     lane-parallel, coalesced loads (lanes walk the products of
//                     the tile; a redux.or of run-start bits gives each lane its
//                     run).  The numeric pass multiplies a_rj * b_jx here, once
//                     per product, with every lane busy.
//   3. merge       -- lane t merges its runs from shared memory.  Equal columns
//                     are combined in run order, and within a run in storage
//                     order, i.e. in exactly the order of the dense-accumulator
//                     loop, starting from the first product (no add to zero).
//   4. write       -- (numeric) outputs go through a small per-lane buffer of 8
//                     entries that the warp flushes cooperatively, so stores to
//                     C are coalesced per row segment.
#include "internal.h"

namespace spg {

constexpr int MERGE_K = 8;                 // max runs per row (A entries)
constexpr int MAXR = 32 * MERGE_K;         // run table entries per tile
constexpr int FSTRIDE = 9;                 // flush buffer row stride (odd: no bank conflicts)
constexpr int FDEPTH = 8;                  // outputs buffered per lane before a flush

template <bool NUM, int PCAP>
struct MergeSmem {
  // doubles first (8-byte alignment), then ints
  static constexpr size_t s_val = 0;
  static constexpr size_t r_a = s_val + (NUM ? 8 * PCAP : 0);
  static constexpr size_t f_val = r_a + (NUM ? 8 * MAXR : 0);
  static constexpr size_t s_col = f_val + (NUM ? 8 * 32 * FSTRIDE : 0);
  static constexpr size_t r_src = s_col + 4 * PCAP;
  static constexpr size_t r_dst = r_src + 4 * MAXR;
  static constexpr size_t f_col = r_dst + 4 * MAXR;
  static constexpr size_t bytes = f_col + (NUM ? 4 * 32 * FSTRIDE : 0) + 16;
};

template <bool NUM, int PCAP, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_merge(DevCsr A, DevCsr B, const uint8_t* __restrict__ rowcls, int cls, const int* __restrict__ rp,
        int* __restrict__ counts, int* __restrict__ C_col, double* __restrict__ C_val, Counters* __restrict__ ctr) {
  using L = MergeSmem<NUM, PCAP>;
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* wb = smem + (size_t)warp * L::bytes;
  double* s_val = reinterpret_cast<double*>(wb + L::s_val);
  double* r_a = reinterpret_cast<double*>(wb + L::r_a);
  double* f_val = reinterpret_cast<double*>(wb + L::f_val);
  int* s_col = reinterpret_cast<int*>(wb + L::s_col);
  int* r_src = reinterpret_cast<int*>(wb + L::r_src);
  int* r_dst = reinterpret_cast<int*>(wb + L::r_dst);
  int* f_col = reinterpret_cast<int*>(wb + L::f_col);

  const int ntiles = (A.rows + 31) >> 5;
  for (int tile = blockIdx.x * WARPS + warp; tile < ntiles; tile += gridDim.x * WARPS) {
    const int r = tile * 32 + lane;
    const bool mine = r < A.rows && rowcls[r] == cls;
    if (!__any_sync(FULL, mine)) continue;

    // 1. run table
    int a0 = 0, k = 0;
    if (mine) { a0 = A.rp[r]; k = A.rp[r + 1] - a0; }
    int src[MERGE_K], len[MERGE_K];
    double av[MERGE_K];
    int u = 0, nz = 0;
#pragma unroll
    for (int i = 0; i < MERGE_K; ++i) {
      len[i] = 0; src[i] = 0; av[i] = 0.0;
      if (i < k) {
        const int j = __ldg(A.col + a0 + i);
        const int bs = __ldg(B.rp + j);
        len[i] = __ldg(B.rp + j + 1) - bs;
        src[i] = bs;
        if (NUM) av[i] = __ldg(A.val + a0 + i);
        u += len[i];
        nz += len[i] > 0;
      }
    }
    int P, R;
    const int pofs = warp_excl_scan(u, &P);   // P <= PCAP: class limits bound every row
    const int rofs = warp_excl_scan(nz, &R);
    int dst[MERGE_K];
    {
      int d = pofs, q = rofs;
#pragma unroll
      for (int i = 0; i < MERGE_K; ++i) {
        dst[i] = d;
        if (len[i] > 0) {
          r_src[q] = src[i];
          r_dst[q] = d;
          if (NUM) r_a[q] = av[i];
          ++q;
          d += len[i];
        }
      }
    }
    __syncwarp();

    // 2. expand: position p of the tile's product space belongs to the last run starting at or before p
    int e_cur = 0;
    for (int base = 0; base < P; base += 32) {
      const int cand = e_cur + 1 + lane;
      const int s = cand < R ? r_dst[cand] : KEY_NONE;
      const unsigned off = (unsigned)(s - base);
      const unsigned bit = off < 32u ? (1u << off) : 0u;
      const unsigned M = __reduce_or_sync(FULL, bit);
      const int e = e_cur + __popc(M & lanemask_le());
      const int p = base + lane;
      if (p < P) {
        const int sp = r_src[e] + (p - r_dst[e]);
        s_col[p] = __ldg(B.col + sp);
        if (NUM) s_val[p] = __dmul_rn(r_a[e], __ldg(B.val + sp));
      }
      e_cur = __shfl_sync(FULL, e, 31);
    }
    __syncwarp();

    // 3. merge the runs of this lane's row
    int h[MERGE_K], cur[MERGE_K], end[MERGE_K];
#pragma unroll
    for (int i = 0; i < MERGE_K; ++i) {
      cur[i] = dst[i];
      end[i] = dst[i] + len[i];
      h[i] = len[i] > 0 ? s_col[cur[i]] : KEY_NONE;
    }
    bool unsorted = false;
    if (!NUM) {
      int cnt = 0, last = -1;
      while (true) {
        int m = h[0];
#pragma unroll
        for (int i = 1; i < MERGE_K; ++i) m = min(m, h[i]);
        if (m == KEY_NONE) break;
        cnt += (m != last);
        last = m;
#pragma unroll
        for (int i = 0; i < MERGE_K; ++i) {
          if (h[i] == m) {
            ++cur[i];
            h[i] = cur[i] < end[i] ? s_col[cur[i]] : KEY_NONE;
            unsorted |= h[i] < m;
          }
        }
      }
      if (mine) counts[r] = cnt;
    } else {
      int g = 0, gend = 0;
      if (mine) { g = rp[r]; gend = rp[r + 1]; }
      int cnt = 0;
      auto flush = [&]() {
        __syncwarp();
#pragma unroll
        for (int jj = 0; jj < FDEPTH; ++jj) {
          const int t = (lane >> 3) + 4 * jj, s = lane & 7;
          const int ct = __shfl_sync(FULL, cnt, t);
          const int gt = __shfl_sync(FULL, g, t);
          const int et = __shfl_sync(FULL, gend, t);
          if (s < ct && gt + s < et) {
            C_col[gt + s] = f_col[t * FSTRIDE + s];
            C_val[gt + s] = f_val[t * FSTRIDE + s];
          }
        }
        g += cnt;
        cnt = 0;
        __syncwarp();
      };
      while (true) {
        int m = h[0];
#pragma unroll
        for (int i = 1; i < MERGE_K; ++i) m = min(m, h[i]);
        const bool act = m != KEY_NONE;
        if (!__any_sync(FULL, act)) break;
        if (act) {
          double v = 0.0;
          bool first = true;
#pragma unroll
          for (int i = 0; i < MERGE_K; ++i) {
            while (h[i] == m) {
              const double x = s_val[cur[i]];
              if (first) v = x; else v = __dadd_rn(v, x);
              first = false;
              ++cur[i];
              h[i] = cur[i] < end[i] ? s_col[cur[i]] : KEY_NONE;
            }
            unsorted |= h[i] < m;
          }
          f_col[lane * FSTRIDE + cnt] = m;
          f_val[lane * FSTRIDE + cnt] = v;
          ++cnt;
        }
        if (__any_sync(FULL, cnt == FDEPTH)) flush();
      }
      if (__any_sync(FULL, cnt > 0)) flush();
      if (mine && g != gend) atomicOr(&ctr->status, ST_MISMATCH);
    }
    if (unsorted) atomicOr(&ctr->status, ST_UNSORTED);
    __syncwarp();
  }
}

template <bool NUM, int PCAP, int WARPS>
static void launch_merge(const DevCsr& A, const DevCsr& B, const uint8_t* rowcls, int cls, const int* rp,
                         int* counts, int* C_col, double* C_val, Counters* ctr, cudaStream_t s) {
  constexpr size_t bytes = (size_t)WARPS * MergeSmem<NUM, PCAP>::bytes;
  auto kern = k_merge<NUM, PCAP, WARPS>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  const int ntiles = (A.rows + 31) / 32;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WARPS * 32, bytes);
  if (per_sm < 1) per_sm = 1;
  const int blocks = std::min((ntiles + WARPS - 1) / WARPS, num_sms() * per_sm * 8);
  kern<<<blocks, WARPS * 32, bytes, s>>>(A, B, rowcls, cls, rp, counts, C_col, C_val, ctr);
}

void launch_merge_symbolic(int cls, const DevCsr& A, const DevCsr& B, const uint8_t* rowcls, int* counts,
                           Counters* ctr, cudaStream_t s) {
  if (cls == CLS_M1) launch_merge<false, 1024, 8>(A, B, rowcls, cls, nullptr, counts, nullptr, nullptr, ctr, s);
  else launch_merge<false, 2048, 8>(A, B, rowcls, cls, nullptr, counts, nullptr, nullptr, ctr, s);
}

void launch_merge_numeric(int cls, const DevCsr& A, const DevCsr& B, const uint8_t* rowcls, const int* rp,
                          int* C_col, double* C_val, Counters* ctr, cudaStream_t s) {
  if (cls == CLS_M1) launch_merge<true, 1024, 4>(A, B, rowcls, cls, rp, nullptr, C_col, C_val, ctr, s);
  else launch_merge<true, 2048, 4>(A, B, rowcls, cls, rp, nullptr, C_col, C_val, ctr, s);
}

}  // namespace spg
