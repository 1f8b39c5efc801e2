// a2 symbolic, a4 numeric, and the fused single pass, for rows with few, short
// contributions (classes M1 and M2: at most 8 entries of A, at most 64 products).
//
// The row-major algorithm of Section IV-A builds row r of C from the rows B_j
// (j in row r of A) scaled by a_rj.  Its dense temporary vector is replaced here
// by the products of the row themselves, held in registers and put in column
// order by a sorting network -- the "Sort" store of Section IV-B, with the
// short-list sort the paper's conclusion asks for.
//
// One warp owns a tile of 32 consecutive rows; lane t owns row tile*32 + t,
// whose u_t <= N products (N = 32 or 64, chosen per matrix from the longest
// merge-class row) come from at most 8 entries of A.
//   1. run table   -- lane t gathers its runs (A entry -> B row range) and, from
//                     them, the start mask of its runs and the B offset of each run.
//   2. expand      -- the warp copies every product's column (and, in the staged
//                     form, b_jx) into shared memory with lane-parallel, coalesced
//                     cp.async copies, the whole tile in flight at once.  Lanes walk
//                     the tile's product space 32 products at a time; a redux.or of
//                     run-start bits names each lane's run.  Row t's products are
//                     contiguous, one slot of skew per row.
//   3. sort        -- lane t loads keys (column | product index) into registers and
//                     runs Batcher's odd-even merge network.  Products are numbered
//                     run by run, so equal columns end up adjacent, in run order and
//                     then B order: the order of the dense-accumulator loop.  A
//                     product's run is the number of run starts at or below its index.
//   4. count       -- distinct columns of the row (symbolic result).
//   5. reduce      -- acc = fma(a_rj, b_jx, acc) along each group of equal columns
//                     in that order, the first product against +0.0.
//   6. place       -- numeric: C's row pointer is known.  Fused: the tile publishes
//                     its entry count and finds its offset in C by a decoupled
//                     look-back over the preceding tiles (the streaming append of
//                     Section IV-B: one allocation sized by the multiplication
//                     count, rows appended in order), then writes C's row pointers.
//   7. write       -- consecutive lanes store consecutive entries of C.
// Two forms of steps 5-7: the staged form keeps b_jx in shared memory, writes each
// group's sum back there and stores C in a coalesced pass; the direct form reads
// b_jx from B in the reduce (four positions' loads in flight at a time) and stores
// each finished entry of C from there; it also reads the columns straight from B when it
// builds the keys (no expand), so it needs only the run tables in shared memory.
// Rows of B need not be sorted: the network orders everything.  Keys hold the
// column above 5 or 6 index bits, so B may have at most 2^26 - 2 columns; wider
// matrices use the hash classes.
//
// Rows of up to 64 products are split over lanes: two lanes per row in the symbolic
// and numeric passes (k_merge_pair), four in the fused pass (k_merge_quad below);
// both give the same sums as one lane per row.  The fused pass places its tiles in
// groups of four warps (one CTA), one look-back per group.
#include "internal.h"

namespace spg {

constexpr int MERGE_K = 8;            // max runs (A entries) per row
constexpr int MAXR = 32 * MERGE_K;    // run-table entries per tile
constexpr long long FUSED_SPIN_LIMIT = 1LL << 24;

enum MergeMode { MODE_SYM = 0, MODE_NUM = 1, MODE_FUSED = 2 };

template <int MODE, int N, bool DIRECT = false>
struct SortSmem {
  // Staging: row t's products are contiguous, at pofs_t + t (one slot of skew per row keeps
  // lanes that read the same position of their rows on different banks).  The direct form
  // stages nothing: it reads the columns from B when it builds the keys and the values in the
  // reduce, and writes C from the reduce; it keeps only the run tables here.
  static constexpr int SLOTS = 32 * N + 32;
  static constexpr bool V = MODE != MODE_SYM;
  static constexpr bool SV = V && !DIRECT;                          // values staged
  static constexpr size_t s_val = 0;                               // double [SLOTS]  b_jx, later group sums
  static constexpr size_t s_col = s_val + (SV ? 8 * SLOTS : 0);    // uint   [SLOTS]  columns, later output keys
  static constexpr size_t r_run = s_col + (DIRECT ? 0 : 4 * SLOTS);  // int2   [MAXR]   (first B entry, start << 8 | lane);
                                                                     // the direct form stages no columns
  static constexpr size_t s_bofs = r_run + 8 * MAXR;               // int    [8][32]  (DIRECT) B offset of a run rank
  static constexpr size_t s_cfr = s_bofs + (DIRECT ? 4 * 8 * 32 : 0);  // int [N]  (N = 64) run holding product 32c
  static constexpr size_t bytes = s_cfr + (N == 64 ? 4 * N : 0);   // s_a (double [8][32], a_rj by run rank
                                                                   // and lane) reuses r_run: after the expand,
                                                                   // or from the run table on (direct form)
  static_assert(8 * 8 * 32 <= 8 * MAXR, "a table must fit in the run table");
};

// Batcher's odd-even merge sort in registers (static indices): 191 compare-exchanges for 32 keys
// and 543 for 64, against 240 and 672 for the bitonic network.
template <int N>
__device__ __forceinline__ void oddeven_sort(unsigned (&k)[N]) {
#pragma unroll
  for (int p = 1; p < N; p <<= 1) {
#pragma unroll
    for (int s = p; s >= 1; s >>= 1) {
#pragma unroll
      for (int t = 0; t < N; ++t) {
        // t = i + j with j = s % p + 2s*m and 0 <= i < s: the lower end of a compare-exchange
        const int r = s % p;
        if (t >= r && (t - r) % (2 * s) < s && t + s < N && t / (2 * p) == (t + s) / (2 * p)) {
          const unsigned a = k[t], b = k[t + s];
          k[t] = min(a, b);
          k[t + s] = max(a, b);
        }
      }
    }
  }
}

// Rank of the nonempty run holding product idx of a row: bit x of `starts` marks a run that
// starts at product x (x > 0), so the rank is the number of marks at or below idx.
__device__ __forceinline__ int run_rank(unsigned long long starts, int idx) {
  return __popcll(starts & ((2ull << idx) - 1ull));
}

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.volatile.global.u64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}

// Decoupled look-back over tiles.  State word: value << 2 | flag, flag 1 = the tile's own total,
// 2 = inclusive prefix.  A tile publishes its total as soon as it is known (tile_publish), does
// other work, then (tile_lookback) reads 32 predecessors per step, adds totals back to the
// nearest inclusive prefix and publishes its own.  Every wait is bounded (ST_TIMEOUT).
__device__ __forceinline__ void tile_publish(unsigned long long* ts, int tile, long long total) {
  if ((threadIdx.x & 31) == 0) atomicExch(&ts[tile], ((unsigned long long)total << 2) | (tile == 0 ? 2ull : 1ull));
}

// Row pointer entry of a row the fused pass places at pos.  Entries past the capacity of C (or
// past INT_MAX; rp_cap is the smaller of the two) are stored clamped to it: the hash and dense
// kernels write row r into [rp[r], rp[r+1]) afterwards, so a product that does not fit leaves
// them inside C_col / C_val (their rows past the end come out empty) while the status reports
// the overflow.
__device__ __forceinline__ int placed_rp(long long pos, int rp_cap) {
  return (int)min(pos, (long long)rp_cap);
}

// Lane l reads the states of tiles pred - l - 32q, q < LOOKBACK_Q, all in flight together, so a
// step covers 32 * LOOKBACK_Q predecessors.  Only the states from pred down to the nearest
// inclusive prefix are needed: those that have published nothing yet are re-read (alone) until
// they have, the others are not waited for.  The spin bound counts the warp's rounds of re-reads;
// past it, unresolved states count as an inclusive prefix of 0 and the status reports the timeout.
// One word per lane measured fastest: 2 and 4 words per lane (64 and 128 predecessors per step)
// cost more registers and instructions than the round trips they save.
constexpr int LOOKBACK_Q = 1;

__device__ long long tile_lookback(unsigned long long* ts, int tile, long long total, Counters* ctr,
                                   long long spin_limit, bool publish) {
  const int lane = threadIdx.x & 31;
  if (tile == 0) return 0;
  long long prefix = 0;
  int pred = tile - 1;
  long long spins = 0;
  bool timed_out = false;
  while (true) {
    unsigned long long w[LOOKBACK_Q];
#pragma unroll
    for (int q = 0; q < LOOKBACK_Q; ++q) {
      const int p = pred - 32 * q - lane;
      w[q] = p >= 0 ? ld_volatile_u64(&ts[p]) : 2ull;   // before tile 0: an inclusive prefix of 0
    }
    unsigned need[LOOKBACK_Q];
    bool found;
    while (true) {
      found = false;
      unsigned wait[LOOKBACK_Q], any = 0u;
#pragma unroll
      for (int q = 0; q < LOOKBACK_Q; ++q) {
        const unsigned incl = __ballot_sync(FULL, (w[q] & 3ull) == 2ull);
        need[q] = found ? 0u : (incl ? (0xffffffffu >> (32 - __ffs(incl))) : FULL);
        found = found || incl != 0u;
        wait[q] = __ballot_sync(FULL, (w[q] & 3ull) == 0ull) & need[q];
        any |= wait[q];
      }
      if (!any) break;
      const bool give_up = ++spins > spin_limit;
      timed_out = timed_out || give_up;
      if (!give_up) __nanosleep(32);
#pragma unroll
      for (int q = 0; q < LOOKBACK_Q; ++q)
        if ((wait[q] >> lane) & 1u) w[q] = give_up ? 2ull : ld_volatile_u64(&ts[pred - 32 * q - lane]);
    }
    long long part = 0;
#pragma unroll
    for (int q = 0; q < LOOKBACK_Q; ++q) part += ((need[q] >> lane) & 1u) ? (long long)(w[q] >> 2) : 0LL;
    prefix += warp_sum_ll(part);
    if (found) break;
    pred -= 32 * LOOKBACK_Q;
  }
  if (timed_out && lane == 0) atomicOr(&ctr->status, ST_TIMEOUT);
  if (publish && lane == 0) atomicExch(&ts[tile], ((unsigned long long)(prefix + total) << 2) | 2ull);
  return prefix;
}

struct MergeArgs {
  DevCsr A, B;
  const uint8_t* rowcls;
  int* rp;                       // SYM: counts out; NUM: C row pointer in; FUSED: counts of other classes in, row pointer out
  int* C_col;
  double* C_val;
  long long capacity;            // FUSED: entries available in C_col / C_val
  unsigned long long* tile_state;
  Counters* ctr;
  int rp_cap;                    // FUSED: min(capacity, INT_MAX), the largest row pointer entry stored
  long long spin_limit;          // FUSED: rounds of re-reads before a look-back gives up
  int drop_tile;                 // FUSED, testing: a tile that publishes nothing (-1: none)
  const int* max_u_dev;          // FUSED: when not NULL, the largest sort-class row on the device; the
  int want_wide;                 //   launch runs only if (*max_u_dev > 32) == want_wide
};

// Grouped placement (the fused direct form): the CTA's warps place their tiles as one group, so the
// look-backs run over four times fewer, larger units.  Each warp leaves its tile's entry count in
// shared memory; warp 0 publishes the group's total, looks back over the groups before it and hands
// each warp its offset in C.  Every warp of the CTA calls this once per group.
template <int WARPS>
__device__ __forceinline__ long long group_place(const MergeArgs& g, int grp, int total) {
  __shared__ int s_tot[WARPS];
  __shared__ long long s_off[WARPS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) s_tot[warp] = total;
  __syncthreads();
  if (warp == 0) {
    int sum;
    const int ex = warp_excl_scan(lane < WARPS ? s_tot[lane] : 0, &sum);
    const bool publish = grp != g.drop_tile;
    if (publish) tile_publish(g.tile_state, grp, sum);
    const long long off = tile_lookback(g.tile_state, grp, sum, g.ctr, g.spin_limit, publish);
    if (lane < WARPS) s_off[lane] = off + ex;
  }
  __syncthreads();
  return s_off[warp];
}

// A fused launch made before the host knows the tile form: it runs only if its form is the one
// the binning pass chose (one of the two launched forms returns at once; uniform across the grid).
__device__ __forceinline__ bool fused_form_selected(const MergeArgs& g) {
  return !g.max_u_dev || ((*g.max_u_dev > 32) == (g.want_wide != 0));
}

template <int MODE, int N, int WARPS, bool DIRECT, bool RK>
__device__ __forceinline__ void merge_tile(const MergeArgs& g, int tile, unsigned char* wb) {
  using L = SortSmem<MODE, N, DIRECT>;
  constexpr bool V = L::V;
  constexpr int IB = (N == 32) ? 5 : 6;     // product-index bits of a key
  constexpr int KB = RK ? IB + 3 : IB;      // key = col << KB | (RK: run rank << IB) | index
  constexpr unsigned PAD = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  double* s_val = reinterpret_cast<double*>(wb + L::s_val);
  unsigned* s_col = reinterpret_cast<unsigned*>(wb + L::s_col);
  int2* r_run = reinterpret_cast<int2*>(wb + L::r_run);
  double* s_a = reinterpret_cast<double*>(wb + L::r_run);
  int* s_bofs = reinterpret_cast<int*>(wb + L::s_bofs);
  int* s_cfr = reinterpret_cast<int*>(wb + L::s_cfr);
  const DevCsr& A = g.A;
  const DevCsr& B = g.B;

  const int r = tile * 32 + lane;
  const bool inrange = r < A.rows;
  const int c = inrange ? (int)g.rowcls[r] : -1;
  const bool mine = c == CLS_M1 || c == CLS_M2;
  constexpr bool GROUPED = MODE == MODE_FUSED && DIRECT && WARPS > 1;   // tiles placed by CTA groups
  if (MODE != MODE_FUSED && !__any_sync(FULL, mine)) return;

  // 1. run table
  int a0 = 0, k = 0;
  if (mine) { a0 = __ldg(A.rp + r); k = __ldg(A.rp + r + 1) - a0; }
  int other = 0;    // FUSED: entry count of a row of another class (from its symbolic pass)
  if (MODE == MODE_FUSED && inrange && !mine && c != CLS_NONE) other = g.rp[r];   // a row without class stays empty
  int gbeg = 0, gend = 0;   // NUM: C's row range
  if (MODE == MODE_NUM && mine) { gbeg = __ldg(g.rp + r); gend = __ldg(g.rp + r + 1); }
  int jcol[MERGE_K];
  double av[MERGE_K];
#pragma unroll
  for (int i = 0; i < MERGE_K; ++i) {
    jcol[i] = -1;
    av[i] = 0.0;
    if (i < k) {
      jcol[i] = __ldg(A.col + a0 + i);
      if (V) av[i] = __ldg(A.val + a0 + i);
    }
  }
  int src[MERGE_K], len[MERGE_K];
#pragma unroll
  for (int i = 0; i < MERGE_K; ++i) {
    src[i] = 0; len[i] = 0;
    if (jcol[i] >= 0) {
      src[i] = __ldg(B.rp + jcol[i]);
      len[i] = __ldg(B.rp + jcol[i] + 1) - src[i];
    }
  }
  int u = 0, nz = 0;
#pragma unroll
  for (int i = 0; i < MERGE_K; ++i) { u += len[i]; nz += len[i] > 0; }
  int P, R;
  const int pofs = warp_excl_scan(u, &P);
  const int rofs = warp_excl_scan(nz, &R);
  const int base = pofs + lane;            // this row's first staging slot
  unsigned long long starts = 0;
  unsigned nem = 0;
  {
    int d = 0, q = rofs, qq = 0;
#pragma unroll
    for (int i = 0; i < MERGE_K; ++i) {
      if (len[i] > 0) {
        if (!DIRECT) {
          r_run[q] = make_int2(src[i], ((pofs + d) << 8) | lane);
          if (N == 64)   // chunks of 32 products whose first product lies in this run
            for (int c = (pofs + d + 31) >> 5; (c << 5) < pofs + d + len[i]; ++c) s_cfr[c] = q;
        } else if (V) {
          s_a[qq * 32 + lane] = av[i];
        }
        if (d > 0) starts |= 1ull << d;                    // bit x: a nonempty run starts at product x
        if (DIRECT) s_bofs[qq * 32 + lane] = src[i] - d;   // b of product index x of this run: B.val[bofs + x]
        nem |= 1u << i;                                    // entry i of A has a nonempty run
        ++q; ++qq;
        d += len[i];
      }
    }
  }
  __syncwarp();

  // 2. expand: asynchronous global -> shared copies of the tile's columns and values, all in flight
  if constexpr (!DIRECT) {   // the direct form reads the columns from B when it builds the keys
    int e_cur = 0;
#pragma unroll 2
    for (int cb = 0; cb < P; cb += 32) {
      if (N == 64) e_cur = s_cfr[cb >> 5];   // independent of the previous chunk: chunks overlap
      const int cand = e_cur + 1 + lane;
      const int st = cand < R ? (r_run[cand].y >> 8) : KEY_NONE;
      const unsigned off = (unsigned)(st - cb);
      const unsigned bit = off < 32u ? (1u << off) : 0u;
      const unsigned M = __reduce_or_sync(FULL, bit);
      const int e = e_cur + __popc(M & lanemask_le());
      const int p = cb + lane;
      if (p < P) {
        const int2 rr = r_run[e];
        const int sp = rr.x + (p - (rr.y >> 8));
        const int d = p + (rr.y & 31);      // product p of row t lives at slot p + t
        cp_async4(s_col + d, B.col + sp);
        if (L::SV) cp_async8(s_val + d, B.val + sp);
      }
      if (N != 64) e_cur = __shfl_sync(FULL, e, 31);
    }
    cp_async_wait_all();
  }
  __syncwarp();   // all copies landed; the run table is free

  // 3. sort this lane's products by (column, run, index).  The run field is the rank of the
  //    product's nonempty run: bits of `starts` mark where each nonempty run after the first begins.
  unsigned key[N];
  {
    int q = 0;
#pragma unroll
    for (int i = 0; i < MERGE_K; ++i) {
      if ((nem >> i) & 1u) {
        if (V && !DIRECT) s_a[q * 32 + lane] = av[i];
        ++q;
      }
    }
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const unsigned rj = (unsigned)__popcll(starts & ((2ull << j) - 1ull));
      const unsigned rk = RK ? (rj << IB) : 0u;
      if constexpr (DIRECT)   // column straight from B: all N loads of the lane in flight together
        key[j] = (j < u) ? (((unsigned)__ldg(B.col + s_bofs[rj * 32 + lane] + j) << KB) | rk | (unsigned)j) : PAD;
      else
        key[j] = (j < u) ? ((s_col[base + j] << KB) | rk | (unsigned)j) : PAD;
    }
  }
  __syncwarp();   // every lane has its keys: s_col may now be overwritten
  oddeven_sort<N>(key);

  // 4. distinct columns
  unsigned samemask_lo = 0, samemask_hi = 0;   // bit j: position j continues a group
#pragma unroll
  for (int j = 1; j < N; ++j) {
    const bool same = (key[j] != PAD) && ((key[j] >> KB) == (key[j - 1] >> KB));
    if (j < 32) samemask_lo |= same ? (1u << j) : 0u; else samemask_hi |= same ? (1u << (j - 32)) : 0u;
  }
  const int cnt = u - __popc(samemask_lo) - __popc(samemask_hi);
  if (MODE == MODE_SYM) {
    if (mine) g.rp[r] = cnt;
    return;
  }
  // fused: the tile's entry count is known now; publish it before the reduce so the tiles
  // after this one rarely wait for it
  const int mycount = mine ? cnt : other;
  int TA = 0;
  const int oa = (MODE == MODE_FUSED) ? warp_excl_scan(mycount, &TA) : 0;
  if (MODE == MODE_FUSED && !GROUPED && tile != g.drop_tile) tile_publish(g.tile_state, tile, TA);

  if constexpr (DIRECT) {
    // 5'. place first (the offset in C is needed to store from the reduce), then reduce: values
    //     straight from B, each finished entry straight to C.
    long long gstart = 0;
    int lim = INT_MAX;
    if (MODE == MODE_NUM) {
      gstart = gbeg;
      lim = gend - gbeg;
      if (mine && lim != cnt) atomicOr(&g.ctr->status, ST_MISMATCH);
    } else {
      const int mycount = mine ? cnt : other;
      int TA;
      const int oa = warp_excl_scan(mycount, &TA);
      const long long off = GROUPED ? group_place<WARPS>(g, tile / WARPS, TA)
                                    : tile_lookback(g.tile_state, tile, TA, g.ctr, g.spin_limit, tile != g.drop_tile);
      gstart = off + oa;
      if (inrange) {
        if (gstart + mycount > g.rp_cap) atomicOr(&g.ctr->status, ST_OVERFLOW);
        g.rp[r] = placed_rp(gstart, g.rp_cap);
        if (r == A.rows - 1) {
          g.rp[r + 1] = placed_rp(gstart + mycount, g.rp_cap);
          g.ctr->nnzC = gstart + mycount;
        }
      }
      if (off + TA > g.capacity) {
        if (lane == 0) atomicOr(&g.ctr->status, ST_OVERFLOW);
        return;
      }
    }
    const int umax = __reduce_max_sync(FULL, u);
    int o = 0;
    double acc = 0.0;
    // b_jx and a_rj of CH positions are loaded together, so that CH loads from B are in flight at
    // once (the loads cannot move past the stores to C on their own).  Larger CH costs registers
    // and with them warps.
    constexpr int CH = 4 < N ? 4 : N;
    double bb[CH], aa[CH];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      if ((j % CH) == 0 && j < umax) {
#pragma unroll
        for (int q = 0; q < CH; ++q) {
          const unsigned kq = key[j + q];
          bb[q] = 0.0; aa[q] = 0.0;
          if (j + q < umax && kq != PAD) {
            const int idx = (int)(kq & (unsigned)(N - 1));
            const int run = RK ? (int)((kq >> IB) & 7u) : run_rank(starts, idx);
            bb[q] = __ldg(B.val + s_bofs[run * 32 + lane] + idx);
            aa[q] = s_a[run * 32 + lane];
          }
        }
      }
      if (j < umax) {
        const unsigned kj = key[j];
        const bool valid = kj != PAD;
        const double a = aa[j % CH], b = bb[j % CH];
        const bool same = (j < 32) ? ((samemask_lo >> j) & 1u) : ((samemask_hi >> (j - 32)) & 1u);
        acc = __fma_rn(a, b, same ? acc : 0.0);
        bool next_same = false;
        if (j + 1 < N) next_same = ((j + 1) < 32) ? ((samemask_lo >> (j + 1)) & 1u) : ((samemask_hi >> (j + 1 - 32)) & 1u);
        if (valid && !next_same) {
          if (o < lim) {
            g.C_col[gstart + o] = (int)(kj >> KB);
            g.C_val[gstart + o] = acc;
          }
          ++o;
        }
      }
    }
    return;
  }

  // 5. reduce: acc = fma(a_rj, b_jx, acc) along each group in product order, the first product
  //    added to +0.0 (the dense accumulator's start).  One FP64 instruction per sorted position,
  //    issued only up to the longest row of the tile (the FP64 pipe costs a full warp slot even
  //    for partial warps).  The group's sum goes to the slot of its last product (already read);
  //    its key to output slot o of this lane's row.
  const int umax = __reduce_max_sync(FULL, u);
  {
    int o = 0;
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      if (j < umax) {
        const unsigned kj = key[j];
        const bool valid = kj != PAD;
        const int idx = (int)(kj & (unsigned)(N - 1));
        const int run = RK ? (int)((kj >> IB) & 7u) : run_rank(starts, idx);
        double a = 0.0, b = 0.0;
        if (valid) {
          b = s_val[base + idx];
          a = s_a[run * 32 + lane];
        }
        const bool same = (j < 32) ? ((samemask_lo >> j) & 1u) : ((samemask_hi >> (j - 32)) & 1u);
        acc = __fma_rn(a, b, same ? acc : 0.0);
        bool next_same = false;
        if (j + 1 < N) next_same = ((j + 1) < 32) ? ((samemask_lo >> (j + 1)) & 1u) : ((samemask_hi >> (j + 1 - 32)) & 1u);
        if (valid && !next_same) {
          s_col[base + o] = kj;
          s_val[base + idx] = acc;
          ++o;
        }
      }
    }
  }

  // 6. place the tile in C
  int TM;
  const int om = warp_excl_scan(mine ? cnt : 0, &TM);   // this row's position in the tile's output list
  long long gstart = 0;   // this row's first entry in C
  int lim = INT_MAX;      // entries this row may write
  if (MODE == MODE_NUM) {
    gstart = gbeg;
    lim = gend - gbeg;
    if (mine && lim != cnt) atomicOr(&g.ctr->status, ST_MISMATCH);
  } else {
    const long long off = tile_lookback(g.tile_state, tile, TA, g.ctr, g.spin_limit, tile != g.drop_tile);
    gstart = off + oa;
    if (inrange) {
      if (gstart + mycount > g.rp_cap) atomicOr(&g.ctr->status, ST_OVERFLOW);
      g.rp[r] = placed_rp(gstart, g.rp_cap);
      if (r == A.rows - 1) {
        g.rp[r + 1] = placed_rp(gstart + mycount, g.rp_cap);
        g.ctr->nnzC = gstart + mycount;
      }
    }
    if (off + TA > g.capacity) {
      if (lane == 0) atomicOr(&g.ctr->status, ST_OVERFLOW);
      return;
    }
  }
  __syncwarp();

  // 7. write the tile's entries: consecutive lanes on consecutive entries of C.
  if (TM >= 24 * __popc(__ballot_sync(FULL, mine && cnt > 0))) {
    // long rows: one row at a time
    const int ctl = min(cnt, lim);
    for (unsigned rows = __ballot_sync(FULL, mine && cnt > 0); rows;) {
      const int t0 = __ffs(rows) - 1;
      rows &= rows - 1;
      const int t1 = rows ? __ffs(rows) - 1 : t0;
      const bool two = rows != 0;
      rows &= rows - 1;
      const int ct0 = __shfl_sync(FULL, ctl, t0), ct1 = two ? __shfl_sync(FULL, ctl, t1) : 0;
      const int bt0 = __shfl_sync(FULL, base, t0), bt1 = __shfl_sync(FULL, base, t1);
      const long long gt0 = __shfl_sync(FULL, gstart, t0), gt1 = __shfl_sync(FULL, gstart, t1);
      unsigned k0[N / 32], k1[N / 32];
      double v0[N / 32], v1[N / 32];
#pragma unroll
      for (int h = 0; h < N / 32; ++h) {
        const int o = lane + 32 * h;
        k0[h] = o < ct0 ? s_col[bt0 + o] : 0u;
        k1[h] = o < ct1 ? s_col[bt1 + o] : 0u;
      }
#pragma unroll
      for (int h = 0; h < N / 32; ++h) {
        const int o = lane + 32 * h;
        if (o < ct0) v0[h] = s_val[bt0 + (int)(k0[h] & (unsigned)(N - 1))];
        if (o < ct1) v1[h] = s_val[bt1 + (int)(k1[h] & (unsigned)(N - 1))];
      }
#pragma unroll
      for (int h = 0; h < N / 32; ++h) {
        const int o = lane + 32 * h;
        if (o < ct0) { g.C_col[gt0 + o] = (int)(k0[h] >> KB); g.C_val[gt0 + o] = v0[h]; }
        if (o < ct1) { g.C_col[gt1 + o] = (int)(k1[h] >> KB); g.C_val[gt1 + o] = v1[h]; }
      }
    }
  } else {
    // short rows: entry f of the tile's list belongs to the last row t with om_t <= f (rows
    // without entries share the start of the next row, so they are never chosen)
    for (int cb = 0; cb < TM; cb += 32) {
      const int f = cb + lane;
      int t = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int cnd = t + step;
        if (__shfl_sync(FULL, om, cnd) <= f) t = cnd;
      }
      const int o = f - __shfl_sync(FULL, om, t);
      const int bt = __shfl_sync(FULL, base, t);
      const long long gt = __shfl_sync(FULL, gstart, t);
      const int lt = __shfl_sync(FULL, lim, t);
      if (f < TM && o < lt) {
        const unsigned kf = s_col[bt + o];
        const double vf = s_val[bt + (int)(kf & (unsigned)(N - 1))];
        g.C_col[gt + o] = (int)(kf >> KB);
        g.C_val[gt + o] = vf;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Rows of up to 64 products, two lanes per row (staged form).  A warp owns 16 consecutive
// rows; lane 2t+h holds half h of row t's products.  Each lane sorts its 32 keys, the pair
// merges them (lane 1 reversed, one compare-exchange across the pair, then a bitonic merge in
// each lane), so lane 2t holds the row's sorted positions 0..31 and lane 2t+1 positions
// 32..63.  Each lane reduces its positions; a group of equal columns that crosses from lane 2t
// into lane 2t+1 is finished by lane 2t+1 from lane 2t's partial sum, in the same order as a
// single chain.  Per warp this needs half the shared memory of the one-lane-per-row form, so
// twice as many warps fit on an SM.
// ---------------------------------------------------------------------------
template <int MODE>
struct PairSmem {
  static constexpr int ROWS = 16;
  static constexpr int N = 64;
  static constexpr int SLOTS = ROWS * N + ROWS;                    // one slot of skew per row
  static constexpr bool V = MODE != MODE_SYM;
  static constexpr size_t s_val = 0;                               // double [SLOTS]  b_jx, later group sums
  static constexpr size_t s_col = s_val + (V ? 8 * SLOTS : 0);     // uint   [SLOTS]  columns, later output keys
  static constexpr size_t r_run = s_col + 4 * SLOTS;               // int2   [ROWS * 8]; s_a later: a_rj of row t,
                                                                   // run q at [t * 9 + q] (an odd stride puts the
                                                                   // two lanes of a row on different banks)
  static constexpr size_t s_cfr = r_run + 8 * ROWS * (MERGE_K + 1);   // int  [32]  run holding product 32c
  static constexpr size_t bytes = s_cfr + 4 * 32;
};

template <int N>
__device__ __forceinline__ void bitonic_merge(unsigned (&k)[N]) {
#pragma unroll
  for (int stride = N >> 1; stride > 0; stride >>= 1) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int j = i ^ stride;
      if (j > i) {
        const unsigned a = k[i], b = k[j];
        k[i] = min(a, b);
        k[j] = max(a, b);
      }
    }
  }
}

template <int MODE>
__device__ __forceinline__ void merge_tile_pair(const MergeArgs& g, int tile, unsigned char* wb) {
  using L = PairSmem<MODE>;
  constexpr bool V = L::V;
  constexpr int H = 32;                     // sorted positions per lane
  constexpr int IB = 6;                     // product-index bits of a key
  constexpr int KB = IB;                    // key = col << KB | index
  constexpr unsigned PAD = 0xffffffffu;
  const int lane = threadIdx.x & 31, t = lane >> 1, h = lane & 1;
  double* s_val = reinterpret_cast<double*>(wb + L::s_val);
  unsigned* s_col = reinterpret_cast<unsigned*>(wb + L::s_col);
  int2* r_run = reinterpret_cast<int2*>(wb + L::r_run);
  double* s_a = reinterpret_cast<double*>(wb + L::r_run);
  int* s_cfr = reinterpret_cast<int*>(wb + L::s_cfr);
  const DevCsr& A = g.A;
  const DevCsr& B = g.B;

  const int r = tile * L::ROWS + t;
  const bool inrange = r < A.rows;
  const int c = inrange ? (int)g.rowcls[r] : -1;
  const bool mine = c == CLS_M1 || c == CLS_M2;
  if (MODE != MODE_FUSED && !__any_sync(FULL, mine)) return;

  // 1. run table: both lanes of a row read the same entries; lane h = 0 writes the tables
  int a0 = 0, k = 0;
  if (mine) { a0 = __ldg(A.rp + r); k = __ldg(A.rp + r + 1) - a0; }
  int other = 0;
  if (MODE == MODE_FUSED && inrange && !mine && c != CLS_NONE && h == 0) other = g.rp[r];
  int gbeg = 0, gend = 0;
  if (MODE == MODE_NUM && mine) { gbeg = __ldg(g.rp + r); gend = __ldg(g.rp + r + 1); }
  int jcol[MERGE_K];
  double av[MERGE_K];
#pragma unroll
  for (int i = 0; i < MERGE_K; ++i) {
    jcol[i] = -1;
    av[i] = 0.0;
    if (i < k) {
      jcol[i] = __ldg(A.col + a0 + i);
      if (V) av[i] = __ldg(A.val + a0 + i);
    }
  }
  int src[MERGE_K], len[MERGE_K];
#pragma unroll
  for (int i = 0; i < MERGE_K; ++i) {
    src[i] = 0; len[i] = 0;
    if (jcol[i] >= 0) {
      src[i] = __ldg(B.rp + jcol[i]);
      len[i] = __ldg(B.rp + jcol[i] + 1) - src[i];
    }
  }
  int u = 0, nz = 0;
#pragma unroll
  for (int i = 0; i < MERGE_K; ++i) { u += len[i]; nz += len[i] > 0; }
  int P, R;
  const int pofs = __shfl_sync(FULL, warp_excl_scan(h == 0 ? u : 0, &P), lane & ~1);   // the row's, in both lanes
  const int rofs = warp_excl_scan(h == 0 ? nz : 0, &R);   // used by lane 2t only
  const int base = pofs + t;               // this row's first staging slot
  unsigned long long starts = 0;           // bit x: a nonempty run starts at product x (x > 0)
  unsigned nem = 0;                        // bit i: entry i of A has a nonempty run
  {
    int d = 0, q = rofs;
#pragma unroll
    for (int i = 0; i < MERGE_K; ++i) {
      if (len[i] > 0) {
        if (h == 0) {
          r_run[q] = make_int2(src[i], ((pofs + d) << 8) | t);
          for (int cc = (pofs + d + 31) >> 5; (cc << 5) < pofs + d + len[i]; ++cc) s_cfr[cc] = q;
        }
        if (d > 0) starts |= 1ull << d;
        nem |= 1u << i;
        ++q;
        d += len[i];
      }
    }
  }
  __syncwarp();

  // 2. expand: the tile's columns (and values) into shared memory, all copies in flight
#pragma unroll 2
  for (int cb = 0; cb < P; cb += 32) {
    const int e_cur = s_cfr[cb >> 5];
    const int cand = e_cur + 1 + lane;
    const int st = cand < R ? (r_run[cand].y >> 8) : KEY_NONE;
    const unsigned off = (unsigned)(st - cb);
    const unsigned bit = off < 32u ? (1u << off) : 0u;
    const unsigned M = __reduce_or_sync(FULL, bit);
    const int e = e_cur + __popc(M & lanemask_le());
    const int p = cb + lane;
    if (p < P) {
      const int2 rr = r_run[e];
      const int sp = rr.x + (p - (rr.y >> 8));
      const int d = p + (rr.y & 31);      // product p of row t lives at slot p + t
      cp_async4(s_col + d, B.col + sp);
      if (V) cp_async8(s_val + d, B.val + sp);
    }
  }
  cp_async_wait_all();
  __syncwarp();   // all copies landed; the run table is free

  // 3. keys of this lane's half (products 32h .. 32h + 31), sort, then merge across the pair
  unsigned key[H];
  {
    if (V && h == 0) {
      int q = 0;
#pragma unroll
      for (int i = 0; i < MERGE_K; ++i) {
        if ((nem >> i) & 1u) {
          s_a[t * (MERGE_K + 1) + q] = av[i];
          ++q;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < H; ++j) {
      const int x = H * h + ((j + 16 * h) & (H - 1));   // lane 2t+1 rotated by 16: the pair reads different banks
      key[j] = (x < u) ? ((s_col[base + x] << KB) | (unsigned)x) : PAD;
    }
  }
  __syncwarp();   // every lane has its keys: s_col may now be overwritten
  oddeven_sort<H>(key);
#pragma unroll
  for (int i = 0; i < H / 2; ++i) {   // lane 2t+1: descending, so the pair forms one bitonic sequence
    const unsigned x = key[i], y = key[H - 1 - i];
    key[i] = h ? y : x;
    key[H - 1 - i] = h ? x : y;
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {
    const unsigned o = __shfl_xor_sync(FULL, key[i], 1);
    key[i] = h ? max(key[i], o) : min(key[i], o);
  }
  bitonic_merge<H>(key);

  // 4. distinct columns; bit 0 of lane 2t+1's mask: its first group continues lane 2t's last
  unsigned samemask = 0;
#pragma unroll
  for (int j = 1; j < H; ++j) {
    const bool same = (key[j] != PAD) && ((key[j] >> KB) == (key[j - 1] >> KB));
    samemask |= same ? (1u << j) : 0u;
  }
  const unsigned prev_last = __shfl_xor_sync(FULL, key[H - 1], 1);
  const bool cont0 = h == 1 && key[0] != PAD && (key[0] >> KB) == (prev_last >> KB);
  samemask |= cont0 ? 1u : 0u;
  const int nvalid = h == 0 ? min(u, H) : max(u - H, 0);
  const int cnt_lane = nvalid - __popc(samemask);
  const int cnt = cnt_lane + __shfl_xor_sync(FULL, cnt_lane, 1);   // the row's distinct columns
  if (MODE == MODE_SYM) {
    if (mine && h == 0) g.rp[r] = cnt;
    return;
  }
  const int mycount = h == 0 ? (mine ? cnt : other) : 0;
  int TA = 0;
  const int oa = (MODE == MODE_FUSED) ? warp_excl_scan(mycount, &TA) : 0;
  if (MODE == MODE_FUSED && tile != g.drop_tile) tile_publish(g.tile_state, tile, TA);

  // 5. reduce, pass 1: each lane's chains; a continued first group (cont0) is left for pass 2
  const bool next_cont = __shfl_xor_sync(FULL, cont0 ? 1 : 0, 1) != 0 && h == 0;   // lane 2t: last group goes on
  // lane 2t's entries come first; lane 2t+1 starts after them (and after the continued group)
  const unsigned endmask = ~((samemask >> 1) | (next_cont ? 0x80000000u : 0u));   // bit j: position j ends a group
  const unsigned validmask = nvalid >= 32 ? 0xffffffffu : ((1u << nvalid) - 1u);
  const int ends_lane = __popc(endmask & validmask);
  const int ends_lo = __shfl_sync(FULL, ends_lane, lane & ~1);
  int o = h == 0 ? 0 : ends_lo + (cont0 ? 1 : 0);
  const int umax = __reduce_max_sync(FULL, nvalid);
  double acc = 0.0;
  {
    bool first_open = cont0;   // lane 2t+1 inside the continued group
#pragma unroll
    for (int j = 0; j < H; ++j) {
      if (j < umax) {
        const unsigned kj = key[j];
        const bool valid = kj != PAD;
        const int idx = (int)(kj & 63u);
        const int run = run_rank(starts, idx);
        double a = 0.0, b = 0.0;
        if (valid) {
          b = s_val[base + idx];
          a = s_a[t * (MERGE_K + 1) + run];
        }
        const bool same = j > 0 && ((samemask >> j) & 1u);
        acc = __fma_rn(a, b, same ? acc : 0.0);
        if (valid && ((endmask >> j) & 1u)) {
          if (!first_open) {
            s_col[base + o] = kj;
            s_val[base + idx] = acc;
            ++o;
          }
          first_open = false;
        }
      }
    }
  }
  // pass 2: lane 2t+1 finishes the continued group from lane 2t's partial sum (acc after its
  // last position, which is valid whenever the group continues)
  const double carry = __shfl_xor_sync(FULL, acc, 1);
  const int glen = cont0 ? ((~samemask == 0u) ? H : (__ffs(~samemask) - 1)) : 0;   // positions 0 .. glen-1
  const int gmax = __reduce_max_sync(FULL, glen);
  if (gmax > 0) {
    double acc2 = carry;
#pragma unroll
    for (int j = 0; j < H; ++j) {
      if (j < gmax) {
        if (j < glen) {
          const unsigned kj = key[j];
          const int idx = (int)(kj & 63u);
          const int run = run_rank(starts, idx);
          acc2 = __fma_rn(s_a[t * (MERGE_K + 1) + run], s_val[base + idx], acc2);
          if (j == glen - 1) {
            s_col[base + ends_lo] = kj;
            s_val[base + idx] = acc2;
          }
        }
      }
    }
  }

  // 6. place the tile in C
  const int oa_row = __shfl_sync(FULL, oa, lane & ~1);
  long long gstart = 0;
  int lim = INT_MAX;
  if (MODE == MODE_NUM) {
    gstart = gbeg;
    lim = gend - gbeg;
    if (mine && h == 0 && lim != cnt) atomicOr(&g.ctr->status, ST_MISMATCH);
  } else {
    const long long off = tile_lookback(g.tile_state, tile, TA, g.ctr, g.spin_limit, tile != g.drop_tile);
    gstart = off + oa_row;
    if (inrange && h == 0) {
      const int rowcount = mine ? cnt : other;
      if (gstart + rowcount > g.rp_cap) atomicOr(&g.ctr->status, ST_OVERFLOW);
      g.rp[r] = placed_rp(gstart, g.rp_cap);
      if (r == A.rows - 1) {
        g.rp[r + 1] = placed_rp(gstart + rowcount, g.rp_cap);
        g.ctr->nnzC = gstart + rowcount;
      }
    }
    if (off + TA > g.capacity) {
      if (lane == 0) atomicOr(&g.ctr->status, ST_OVERFLOW);
      return;
    }
  }
  __syncwarp();

  // 7. write: rows in lane order (h = 0 lanes), two rows per step, consecutive lanes on
  //    consecutive entries of C
  const int ctl = min(cnt, lim);
  for (unsigned rows = __ballot_sync(FULL, h == 0 && mine && cnt > 0); rows;) {
    const int t0 = __ffs(rows) - 1;
    rows &= rows - 1;
    const int t1 = rows ? __ffs(rows) - 1 : t0;
    const bool two = rows != 0;
    rows &= rows - 1;
    const int ct0 = __shfl_sync(FULL, ctl, t0), ct1 = two ? __shfl_sync(FULL, ctl, t1) : 0;
    const int bt0 = __shfl_sync(FULL, base, t0), bt1 = __shfl_sync(FULL, base, t1);
    const long long gt0 = __shfl_sync(FULL, gstart, t0), gt1 = __shfl_sync(FULL, gstart, t1);
    unsigned k0[2], k1[2];
    double v0[2], v1[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int oo = lane + 32 * q;
      k0[q] = oo < ct0 ? s_col[bt0 + oo] : 0u;
      k1[q] = oo < ct1 ? s_col[bt1 + oo] : 0u;
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int oo = lane + 32 * q;
      if (oo < ct0) v0[q] = s_val[bt0 + (int)(k0[q] & 63u)];
      if (oo < ct1) v1[q] = s_val[bt1 + (int)(k1[q] & 63u)];
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int oo = lane + 32 * q;
      if (oo < ct0) { g.C_col[gt0 + oo] = (int)(k0[q] >> KB); g.C_val[gt0 + oo] = v0[q]; }
      if (oo < ct1) { g.C_col[gt1 + oo] = (int)(k1[q] >> KB); g.C_val[gt1 + oo] = v1[q]; }
    }
  }
}

// 16 warps of at most 128 registers: shared memory allows 17 per SM
template <int MODE>
__global__ void __launch_bounds__(32, 16)
k_merge_pair(MergeArgs g) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int ntiles = (g.A.rows + PairSmem<MODE>::ROWS - 1) / PairSmem<MODE>::ROWS;
  if (MODE == MODE_FUSED && !fused_form_selected(g)) return;
  if (MODE != MODE_FUSED) {
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      merge_tile_pair<MODE>(g, tile, smem);
      __syncwarp();
    }
  } else {
    while (true) {
      int tile = 0;
      if (lane == 0) tile = (int)atomicAdd(&g.ctr->ticket, 1u);
      tile = __shfl_sync(FULL, tile, 0);
      if (tile >= ntiles) break;
      merge_tile_pair<MODE>(g, tile, smem);
      __syncwarp();
    }
  }
}

template <int MODE>
static void launch_merge_pair(const MergeArgs& g, cudaStream_t s) {
  constexpr size_t bytes = PairSmem<MODE>::bytes;
  auto kern = k_merge_pair<MODE>;
  const int ntiles = (g.A.rows + PairSmem<MODE>::ROWS - 1) / PairSmem<MODE>::ROWS;
  const int per_sm = blocks_per_sm((const void*)kern, 32, bytes);
  const int blocks = std::max(1, std::min(ntiles, num_sms() * per_sm * (MODE == MODE_FUSED ? 1 : 4)));
  kern<<<blocks, 32, bytes, s>>>(g);
}

// ---------------------------------------------------------------------------
// Rows of up to 64 products, four lanes per row (the fused pass).  A warp owns 8 consecutive rows;
// lane 4t+q holds sorted positions 16q .. 16q+15 of row t.  Each lane sorts its 16 keys; the lane
// pairs (q, q^1) merge them into 32 (the odd lane reversed, one compare-exchange across the pair, a
// bitonic merge in each lane); then the two pairs merge into 64 (the second pair reversed, compare-
// exchanges across lanes at distances of 32 and 16 positions, a bitonic merge in each lane).  A
// group of equal columns may run across lanes: the lanes finish such a group one after another,
// each from the partial sum of the lane before, in the order of a single chain, so the sums are
// bit-identical to the one-lane form.  Per warp this needs half the shared memory of the two-lanes-
// per-row form, so about twice as many warps fit on an SM.
// ---------------------------------------------------------------------------
struct QuadSmem {
  static constexpr int ROWS = 8;
  static constexpr int N = 64;
  static constexpr int SLOTS = ROWS * N + ROWS;                    // one slot of skew per row
  static constexpr size_t s_val = 0;                               // double [SLOTS]  b_jx, later group sums
  static constexpr size_t s_col = s_val + 8 * SLOTS;               // uint   [SLOTS]  columns, later output keys
  static constexpr size_t r_run = s_col + 4 * SLOTS;               // int2   [ROWS * 8]; s_a later: a_rj of row t,
                                                                   // run q at [t * 9 + q]
  static constexpr size_t s_cfr = r_run + 8 * ROWS * (MERGE_K + 1);   // int  [16]  run holding product 32c
  static constexpr size_t bytes = s_cfr + 4 * 16;
};

template <int WARPS>
__device__ __forceinline__ void merge_tile_quad(const MergeArgs& g, int tile, unsigned char* wb) {
  using L = QuadSmem;
  constexpr int H = 16;                     // sorted positions per lane
  constexpr int KB = 6;                     // key = col << KB | index
  constexpr unsigned PAD = 0xffffffffu;
  __shared__ int s_gtot[WARPS];
  __shared__ long long s_goff[WARPS];
  const int warp = threadIdx.x >> 5;
  int gsum = 0;
  const int lane = threadIdx.x & 31, t = lane >> 2, q4 = lane & 3, lead = lane & ~3;
  double* s_val = reinterpret_cast<double*>(wb + L::s_val);
  unsigned* s_col = reinterpret_cast<unsigned*>(wb + L::s_col);
  int2* r_run = reinterpret_cast<int2*>(wb + L::r_run);
  double* s_a = reinterpret_cast<double*>(wb + L::r_run);
  int* s_cfr = reinterpret_cast<int*>(wb + L::s_cfr);
  const DevCsr& A = g.A;
  const DevCsr& B = g.B;

  const int r = tile * L::ROWS + t;
  const bool inrange = r < A.rows;
  const int c = inrange ? (int)g.rowcls[r] : -1;
  const bool mine = c == CLS_M1 || c == CLS_M2;

  // 1. run table: the four lanes of a row read the same entries; lane 4t writes the tables
  int a0 = 0, k = 0;
  if (mine) { a0 = __ldg(A.rp + r); k = __ldg(A.rp + r + 1) - a0; }
  int other = 0;
  if (inrange && !mine && c != CLS_NONE && q4 == 0) other = g.rp[r];
  int jcol[MERGE_K];
  double av[MERGE_K];
#pragma unroll
  for (int i = 0; i < MERGE_K; ++i) {
    jcol[i] = -1;
    av[i] = 0.0;
    if (i < k) {
      jcol[i] = __ldg(A.col + a0 + i);
      av[i] = __ldg(A.val + a0 + i);
    }
  }
  int src[MERGE_K], len[MERGE_K];
#pragma unroll
  for (int i = 0; i < MERGE_K; ++i) {
    src[i] = 0; len[i] = 0;
    if (jcol[i] >= 0) {
      src[i] = __ldg(B.rp + jcol[i]);
      len[i] = __ldg(B.rp + jcol[i] + 1) - src[i];
    }
  }
  int u = 0, nz = 0;
#pragma unroll
  for (int i = 0; i < MERGE_K; ++i) { u += len[i]; nz += len[i] > 0; }
  int P, R;
  const int pofs = __shfl_sync(FULL, warp_excl_scan(q4 == 0 ? u : 0, &P), lead);   // the row's, in its four lanes
  const int rofs = warp_excl_scan(q4 == 0 ? nz : 0, &R);   // used by lane 4t only
  const int base = pofs + t;               // this row's first staging slot
  unsigned long long starts = 0;           // bit x: a nonempty run starts at product x (x > 0)
  unsigned nem = 0;                        // bit i: entry i of A has a nonempty run
  {
    int d = 0, q = rofs;
#pragma unroll
    for (int i = 0; i < MERGE_K; ++i) {
      if (len[i] > 0) {
        if (q4 == 0) {
          r_run[q] = make_int2(src[i], ((pofs + d) << 8) | t);
          for (int cc = (pofs + d + 31) >> 5; (cc << 5) < pofs + d + len[i]; ++cc) s_cfr[cc] = q;
        }
        if (d > 0) starts |= 1ull << d;
        nem |= 1u << i;
        ++q;
        d += len[i];
      }
    }
  }
  __syncwarp();

  // 2. expand: the tile's columns and values into shared memory, all copies in flight
#pragma unroll 2
  for (int cb = 0; cb < P; cb += 32) {
    const int e_cur = s_cfr[cb >> 5];
    const int cand = e_cur + 1 + lane;
    const int st = cand < R ? (r_run[cand].y >> 8) : KEY_NONE;
    const unsigned off = (unsigned)(st - cb);
    const unsigned bit = off < 32u ? (1u << off) : 0u;
    const unsigned M = __reduce_or_sync(FULL, bit);
    const int e = e_cur + __popc(M & lanemask_le());
    const int p = cb + lane;
    if (p < P) {
      const int2 rr = r_run[e];
      const int sp = rr.x + (p - (rr.y >> 8));
      const int d = p + (rr.y & 31);      // product p of row t lives at slot p + t
      cp_async4(s_col + d, B.col + sp);
      cp_async8(s_val + d, B.val + sp);
    }
  }
  cp_async_wait_all();
  __syncwarp();   // all copies landed; the run table is free

  // 3. keys of this lane's quarter (products 16q .. 16q + 15), sort, then merge across the lanes
  unsigned key[H];
  {
    if (q4 == 0) {
      int q = 0;
#pragma unroll
      for (int i = 0; i < MERGE_K; ++i) {
        if ((nem >> i) & 1u) {
          s_a[t * (MERGE_K + 1) + q] = av[i];
          ++q;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < H; ++j) {
      const int x = H * q4 + ((j + 8 * (q4 >> 1)) & (H - 1));   // lanes 4t+2, 4t+3 rotated by 8: 32 banks
      key[j] = (x < u) ? ((s_col[base + x] << KB) | (unsigned)x) : PAD;
    }
  }
  __syncwarp();   // every lane has its keys: s_col may now be overwritten
  oddeven_sort<H>(key);
  const bool odd = (q4 & 1) != 0, upper = (q4 & 2) != 0;
#pragma unroll
  for (int i = 0; i < H / 2; ++i) {   // odd lane descending: each pair forms a bitonic sequence
    const unsigned x = key[i], y = key[H - 1 - i];
    key[i] = odd ? y : x;
    key[H - 1 - i] = odd ? x : y;
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {
    const unsigned o = __shfl_xor_sync(FULL, key[i], 1);
    key[i] = odd ? max(key[i], o) : min(key[i], o);
  }
  bitonic_merge<H>(key);
#pragma unroll
  for (int i = 0; i < H / 2; ++i) {   // the upper pair reversed: lane 4t+2 takes 4t+3's keys backwards and so on
    const unsigned x = __shfl_xor_sync(FULL, key[H - 1 - i], 1), y = __shfl_xor_sync(FULL, key[i], 1);
    if (upper) { key[i] = x; key[H - 1 - i] = y; }
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {   // distance 32 positions: lane q against q + 2
    const unsigned o = __shfl_xor_sync(FULL, key[i], 2);
    key[i] = upper ? max(key[i], o) : min(key[i], o);
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {   // distance 16 positions: lane q against q + 1
    const unsigned o = __shfl_xor_sync(FULL, key[i], 1);
    key[i] = odd ? max(key[i], o) : min(key[i], o);
  }
  bitonic_merge<H>(key);

  // 4. distinct columns; bit 0 of the mask: this lane's first group continues the lane before
  unsigned samemask = 0;
#pragma unroll
  for (int j = 1; j < H; ++j) {
    const bool same = (key[j] != PAD) && ((key[j] >> KB) == (key[j - 1] >> KB));
    samemask |= same ? (1u << j) : 0u;
  }
  const unsigned prev_last = __shfl_up_sync(FULL, key[H - 1], 1);
  const bool cont0 = q4 > 0 && key[0] != PAD && (key[0] >> KB) == (prev_last >> KB);
  samemask |= cont0 ? 1u : 0u;
  const int nvalid = min(max(u - H * q4, 0), H);
  const int cnt_lane = nvalid - __popc(samemask);
  int cnt = cnt_lane + __shfl_xor_sync(FULL, cnt_lane, 1);
  cnt += __shfl_xor_sync(FULL, cnt, 2);   // the row's distinct columns
  const int mycount = q4 == 0 ? (mine ? cnt : other) : 0;
  int TA = 0;
  const int oa = warp_excl_scan(mycount, &TA);
  if (lane == 0) s_gtot[warp] = TA;
  __syncthreads();
  if (warp == 0) {
    const int ex = warp_excl_scan(lane < WARPS ? s_gtot[lane] : 0, &gsum);
    if (lane < WARPS) s_goff[lane] = ex;
    if (tile / WARPS != g.drop_tile) tile_publish(g.tile_state, tile / WARPS, gsum);
  }

  // 5. reduce, pass 1: each lane's chains; a continued first group (cont0) is left for pass 2
  const int cont_next = __shfl_down_sync(FULL, cont0 ? 1 : 0, 1);   // every lane takes part in the shuffle
  const bool next_cont = q4 < 3 && cont_next != 0;                  // my last group goes on
  const unsigned endmask = ~((samemask >> 1) | (next_cont ? (1u << (H - 1)) : 0u));   // bit j: position j ends a group
  const unsigned validmask = (1u << nvalid) - 1u;
  const int ends_lane = __popc(endmask & validmask);
  int ends_incl = ends_lane;   // groups that end in this lane or the lanes of the row before it
  {
    int y = __shfl_up_sync(FULL, ends_incl, 1);
    if (q4 >= 1) ends_incl += y;
    y = __shfl_up_sync(FULL, ends_incl, 2);
    if (q4 >= 2) ends_incl += y;
  }
  const int ends_before = ends_incl - ends_lane;   // output slot of a continued group that ends here
  int o = ends_before + (cont0 ? 1 : 0);
  const int umax = __reduce_max_sync(FULL, nvalid);
  double acc = 0.0;
  {
    bool first_open = cont0;   // inside the continued group
#pragma unroll
    for (int j = 0; j < H; ++j) {
      if (j < umax) {
        const unsigned kj = key[j];
        const bool valid = kj != PAD;
        const int idx = (int)(kj & 63u);
        const int run = run_rank(starts, idx);
        double a = 0.0, b = 0.0;
        if (valid) {
          b = s_val[base + idx];
          a = s_a[t * (MERGE_K + 1) + run];
        }
        const bool same = j > 0 && ((samemask >> j) & 1u);
        acc = __fma_rn(a, b, same ? acc : 0.0);
        if (valid && ((endmask >> j) & 1u)) {
          if (!first_open) {
            s_col[base + o] = kj;
            s_val[base + idx] = acc;
            ++o;
          }
          first_open = false;
        }
      }
    }
  }
  // pass 2: the continued groups, lane after lane, each from the partial sum the lane before left
  // at its last position (valid whenever the next lane continues its group)
  const int glen = cont0 ? (__ffs(~samemask) - 1) : 0;   // positions 0 .. glen-1
  const bool gends = glen < nvalid || !next_cont;        // the continued group ends in this lane
  const int gmax = __reduce_max_sync(FULL, glen);
  if (gmax > 0) {
    double accf = acc;   // the partial sum handed to the next lane
#pragma unroll 1
    for (int step = 1; step < 4; ++step) {
      const double carry = __shfl_up_sync(FULL, accf, 1);
      const bool act = q4 == step && glen > 0;
      double acc2 = carry;
#pragma unroll
      for (int j = 0; j < H; ++j) {
        if (j < gmax && act && j < glen) {
          const unsigned kj = key[j];
          const int idx = (int)(kj & 63u);
          const int run = run_rank(starts, idx);
          acc2 = __fma_rn(s_a[t * (MERGE_K + 1) + run], s_val[base + idx], acc2);
          if (j == glen - 1 && gends) {
            s_col[base + ends_before] = kj;
            s_val[base + idx] = acc2;
          }
        }
      }
      if (act && !gends) accf = acc2;   // the whole lane belongs to the group: carry it on
    }
  }

  // 6. place the tile in C
  const int oa_row = __shfl_sync(FULL, oa, lead);
  long long off;
  {
    const int grp = tile / WARPS;
    if (warp == 0) {
      const long long go = tile_lookback(g.tile_state, grp, gsum, g.ctr, g.spin_limit, grp != g.drop_tile);
      if (lane < WARPS) s_goff[lane] += go;
    }
    __syncthreads();
    off = s_goff[warp];
  }
  const long long gstart = off + oa_row;
  if (inrange && q4 == 0) {
    const int rowcount = mine ? cnt : other;
    if (gstart + rowcount > g.rp_cap) atomicOr(&g.ctr->status, ST_OVERFLOW);
    g.rp[r] = placed_rp(gstart, g.rp_cap);
    if (r == A.rows - 1) {
      g.rp[r + 1] = placed_rp(gstart + rowcount, g.rp_cap);
      g.ctr->nnzC = gstart + rowcount;
    }
  }
  if (off + TA > g.capacity) {
    if (lane == 0) atomicOr(&g.ctr->status, ST_OVERFLOW);
    return;
  }
  __syncwarp();

  // 7. write: rows in order (lanes 4t), two rows per step, consecutive lanes on consecutive entries
  for (unsigned rows = __ballot_sync(FULL, q4 == 0 && mine && cnt > 0); rows;) {
    const int t0 = __ffs(rows) - 1;
    rows &= rows - 1;
    const int t1 = rows ? __ffs(rows) - 1 : t0;
    const bool two = rows != 0;
    rows &= rows - 1;
    const int ct0 = __shfl_sync(FULL, cnt, t0), ct1 = two ? __shfl_sync(FULL, cnt, t1) : 0;
    const int bt0 = __shfl_sync(FULL, base, t0), bt1 = __shfl_sync(FULL, base, t1);
    const long long gt0 = __shfl_sync(FULL, gstart, t0), gt1 = __shfl_sync(FULL, gstart, t1);
    unsigned k0[2], k1[2];
    double v0[2], v1[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int oo = lane + 32 * q;
      k0[q] = oo < ct0 ? s_col[bt0 + oo] : 0u;
      k1[q] = oo < ct1 ? s_col[bt1 + oo] : 0u;
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int oo = lane + 32 * q;
      if (oo < ct0) v0[q] = s_val[bt0 + (int)(k0[q] & 63u)];
      if (oo < ct1) v1[q] = s_val[bt1 + (int)(k1[q] & 63u)];
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int oo = lane + 32 * q;
      if (oo < ct0) { g.C_col[gt0 + oo] = (int)(k0[q] >> KB); g.C_val[gt0 + oo] = v0[q]; }
      if (oo < ct1) { g.C_col[gt1 + oo] = (int)(k1[q] >> KB); g.C_val[gt1 + oo] = v1[q]; }
    }
  }
}

// The fused pass of 64-product rows: CTAs of four warps (32 rows placed as one group), seven CTAs
// per SM (28 warps of at most 72 registers, no spills).  Against the two-lanes-per-row form (16
// warps per SM, groups of 64 rows): 0.56 against 0.72 ms for the random 1M x 8 product, with C
// bit-identical; six CTAs per SM measured 0.58 ms.
template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 7)
k_merge_quad(MergeArgs g) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5;
  const int ntiles = (g.A.rows + QuadSmem::ROWS - 1) / QuadSmem::ROWS;
  if (!fused_form_selected(g)) return;
  unsigned char* wb = smem + (size_t)warp * QuadSmem::bytes;
  __shared__ int s_ticket;
  const int ngroups = (ntiles + WARPS - 1) / WARPS;
  while (true) {
    if (threadIdx.x == 0) s_ticket = (int)atomicAdd(&g.ctr->ticket, 1u);
    __syncthreads();
    const int grp = s_ticket;
    if (grp >= ngroups) break;
    merge_tile_quad<WARPS>(g, grp * WARPS + warp, wb);
  }
}

template <int WARPS>
static void launch_merge_quad(const MergeArgs& g, cudaStream_t s) {
  constexpr size_t bytes = WARPS * QuadSmem::bytes;
  auto kern = k_merge_quad<WARPS>;
  const int ntiles = (g.A.rows + QuadSmem::ROWS - 1) / QuadSmem::ROWS;
  const int groups = (ntiles + WARPS - 1) / WARPS;
  const int per_sm = blocks_per_sm((const void*)kern, WARPS * 32, bytes);
  const int blocks = std::max(1, std::min(groups, num_sms() * per_sm));
  kern<<<blocks, WARPS * 32, bytes, s>>>(g);
}

// The fused direct form with 32-product tiles runs in CTAs of four warps (a group of 128 rows placed
// together), five CTAs per SM: at most 102 registers a thread, no spills.  Measured against 28
// one-warp CTAs of at most 72 registers (a few spills) and one look-back per 32 rows: 0.66 against
// 0.79 ms for the Laplacian^2 2048^2.  The other forms keep their natural register counts.
template <int MODE, int N, int WARPS, bool DIRECT, bool RK>
__global__ void __launch_bounds__(WARPS * 32, (N == 32 && DIRECT && MODE == MODE_FUSED && WARPS == 4) ? 5 : 1)
k_merge(MergeArgs g) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* wb = smem + (size_t)warp * SortSmem<MODE, N, DIRECT>::bytes;
  const int ntiles = (g.A.rows + 31) >> 5;
  if (MODE == MODE_FUSED && !fused_form_selected(g)) return;
  if (MODE != MODE_FUSED) {
    for (int tile = blockIdx.x * WARPS + warp; tile < ntiles; tile += gridDim.x * WARPS) {
      merge_tile<MODE, N, WARPS, DIRECT, RK>(g, tile, wb);
      __syncwarp();
    }
  } else if constexpr (DIRECT && WARPS > 1) {
    // The CTA takes its next group of WARPS tiles from a ticket, so the groups in flight are
    // consecutive and every group a look-back waits on is held by a CTA that is already running.
    // Thread 0 writes the next ticket only after both barriers of group_place, which every warp
    // reaches after it has read the current one.
    __shared__ int s_ticket;
    const int ngroups = (ntiles + WARPS - 1) / WARPS;
    while (true) {
      if (threadIdx.x == 0) s_ticket = (int)atomicAdd(&g.ctr->ticket, 1u);
      __syncthreads();
      const int grp = s_ticket;
      if (grp >= ngroups) break;
      merge_tile<MODE, N, WARPS, DIRECT, RK>(g, grp * WARPS + warp, wb);
    }
  } else {
    // Each warp takes its next tile from a ticket, so the tiles in flight are consecutive and
    // every tile a look-back waits on is held by a warp that is already running.
    while (true) {
      int tile = 0;
      if (lane == 0) tile = (int)atomicAdd(&g.ctr->ticket, 1u);
      tile = __shfl_sync(FULL, tile, 0);
      if (tile >= ntiles) break;
      merge_tile<MODE, N, WARPS, DIRECT, RK>(g, tile, wb);
      __syncwarp();
    }
  }
}

template <int MODE, int N, int WARPS, bool DIRECT = false>
static void launch_merge(const MergeArgs& g, cudaStream_t s) {
  constexpr size_t bytes = (size_t)WARPS * SortSmem<MODE, N, DIRECT>::bytes;
  // The 32-product direct form also keeps the run rank in its keys (one shift instead of a
  // popcount per position of the reduce) while the column fits above 8 bits: B.cols <= 2^24 - 2.
  constexpr bool RK_FORM = N == 32 && DIRECT;
  auto kern = (RK_FORM && g.B.cols <= (1 << 24) - 2) ? k_merge<MODE, N, WARPS, DIRECT, RK_FORM>
                                                      : k_merge<MODE, N, WARPS, DIRECT, false>;
  const int ntiles = (g.A.rows + 31) / 32;
  const int per_sm = blocks_per_sm((const void*)kern, WARPS * 32, bytes);
  int blocks;
  if (MODE == MODE_FUSED) {
    blocks = std::max(1, std::min((ntiles + WARPS - 1) / WARPS, num_sms() * per_sm));
  } else {
    blocks = std::max(1, std::min((ntiles + WARPS - 1) / WARPS, num_sms() * per_sm * 4));
  }
  kern<<<blocks, WARPS * 32, bytes, s>>>(g);
}

int merge_max_cols() { return (1 << 26) - 2; }

// one state per placement unit: groups of 128 rows (direct form) or 32 rows (four lanes per row),
// tiles of 32 rows (staged form); sized for one per 16 rows
size_t fused_tile_state_bytes(int rows) { return (size_t)((rows + 15) / 16) * sizeof(unsigned long long); }

void launch_merge_symbolic(int wide, const DevCsr& A, const DevCsr& B, const uint8_t* rowcls, int* counts,
                           Counters* ctr, cudaStream_t s) {
  MergeArgs g{A, B, rowcls, counts, nullptr, nullptr, 0, nullptr, ctr, 0, 0, -1, nullptr, 0};
  if (!wide) launch_merge<MODE_SYM, 32, 4>(g, s);
  else launch_merge<MODE_SYM, 64, 4>(g, s);
}

void launch_merge_numeric(int wide, int values_mode, const DevCsr& A, const DevCsr& B, const uint8_t* rowcls,
                          const int* rp, int* C_col, double* C_val, Counters* ctr, cudaStream_t s) {
  MergeArgs g{A, B, rowcls, const_cast<int*>(rp), C_col, C_val, 0, nullptr, ctr, 0, 0, -1, nullptr, 0};
  const bool direct = values_mode == 1 || (values_mode == 0 && !wide);
  if (direct) {
    if (!wide) launch_merge<MODE_NUM, 32, 1, true>(g, s);
    else launch_merge<MODE_NUM, 64, 1, true>(g, s);
  } else {
    if (!wide) launch_merge<MODE_NUM, 32, 1>(g, s);
    else launch_merge_pair<MODE_NUM>(g, s);
  }
}

void launch_merge_fused(int wide, int values_mode, const DevCsr& A, const DevCsr& B, const uint8_t* rowcls, int* rp,
                        int* C_col, double* C_val, long long capacity, unsigned long long* tile_state, Counters* ctr,
                        cudaStream_t s, int spin_limit, int drop_tile, const int* max_u_dev) {
  MergeArgs g{A, B, rowcls, rp, C_col, C_val, capacity, tile_state, ctr,
              (int)std::min(capacity, (long long)INT_MAX), spin_limit > 0 ? (long long)spin_limit : FUSED_SPIN_LIMIT,
              drop_tile, max_u_dev, wide};
  const bool direct = values_mode == 1 || (values_mode == 0 && !wide);
  if (direct) {
    if (!wide) launch_merge<MODE_FUSED, 32, 4, true>(g, s);   // grouped placement
    else launch_merge<MODE_FUSED, 64, 1, true>(g, s);
  } else {
    if (!wide) launch_merge<MODE_FUSED, 32, 1>(g, s);
    else launch_merge_quad<4>(g, s);   // four lanes per row, grouped placement
  }
}

}  // namespace spg
