// Pattern reuse: C's values again after the values of A and B change, C's structure kept.
//
// The row-major loop of Section IV-A visits the products of row r in a fixed order (the entries
// a_rj of row r in storage order, and for each the entries of B_j in storage order), and the
// store of Section IV-B gives every column of row r a fixed position in C.  Recording, once,
// the position each product lands on turns every later numeric pass into a plain accumulation
// c[pos] = fma(a_rj, b_jx, c[pos]) in that same loop order -- no sort, no hash -- which is exactly
// the order, and so gives exactly the bits, of the sort classes' numeric pass.
//
// The map covers the rows of the sort classes (at most 8 entries of A and 64 products, so a
// position fits one byte).  Layout: int32 tile offsets (one per tile of 32 rows, then the
// total), 256-byte aligned, then per tile 32 * umax bytes (umax = the tile's longest row),
// position-major: byte x * 32 + t is the position of product x of row tile*32 + t, so the 32
// lanes of a warp read one product each from 32 consecutive bytes.  Longer rows are recomputed
// by the hash and dense kernels.
#include "internal.h"

namespace spg {

constexpr int RP_MERGE_K = 8;

size_t replay_map_bytes(int rows, int max_u) {
  const size_t ntiles = (size_t)(rows + 31) / 32;
  return (4 * (ntiles + 1) + 255) / 256 * 256 + 32 * ntiles * (size_t)std::max(std::min(max_u, 64), 1);
}

// Entries and products of row r (a sort-class row): the run table of the merge kernels.
struct RowRuns {
  int a0, k, u;
  int src[RP_MERGE_K], len[RP_MERGE_K];
};

__device__ __forceinline__ void row_runs(const DevCsr& A, const DevCsr& B, int r, bool mine, RowRuns& rr) {
  rr.a0 = 0; rr.k = 0; rr.u = 0;
  if (mine) { rr.a0 = __ldg(A.rp + r); rr.k = min(__ldg(A.rp + r + 1) - rr.a0, RP_MERGE_K); }
  int j[RP_MERGE_K];
#pragma unroll
  for (int i = 0; i < RP_MERGE_K; ++i) j[i] = i < rr.k ? __ldg(A.col + rr.a0 + i) : -1;
#pragma unroll
  for (int i = 0; i < RP_MERGE_K; ++i) {
    rr.src[i] = 0; rr.len[i] = 0;
    if (j[i] >= 0) { rr.src[i] = __ldg(B.rp + j[i]); rr.len[i] = __ldg(B.rp + j[i] + 1) - rr.src[i]; }
    rr.u += rr.len[i];
  }
}

__device__ __forceinline__ bool sort_class(const uint8_t* cls, int r, int rows) {
  if (r >= rows) return false;
  const int c = cls[r];
  return c == CLS_M1 || c == CLS_M2;
}

// Map bytes of each tile of 32 rows: 32 * its longest sort-class row (the scan turns them into offsets).
__global__ void k_replay_count(DevCsr A, DevCsr B, const uint8_t* __restrict__ cls, int* __restrict__ tile_off) {
  const int warps = blockDim.x >> 5;
  const int lane = threadIdx.x & 31;
  const int ntiles = (A.rows + 31) >> 5;
  for (int tile = blockIdx.x * warps + (threadIdx.x >> 5); tile < ntiles; tile += gridDim.x * warps) {
    const int r = tile * 32 + lane;
    RowRuns rr;
    row_runs(A, B, r, sort_class(cls, r, A.rows), rr);
    const int umax = __reduce_max_sync(FULL, rr.u);
    if (lane == 0) tile_off[tile] = 32 * umax;
  }
}

// Position of every product within its row of C: binary search of the product's column among
// the row's sorted columns.  A column that is not there means C is not this product's result.
__global__ void k_replay_record(DevCsr A, DevCsr B, const uint8_t* __restrict__ cls, const int* __restrict__ C_rp,
                                const int* __restrict__ C_col, const int* __restrict__ tile_off,
                                uint8_t* __restrict__ map, Counters* __restrict__ ctr) {
  const int warps = blockDim.x >> 5;
  const int lane = threadIdx.x & 31;
  const int ntiles = (A.rows + 31) >> 5;
  bool miss = false;
  for (int tile = blockIdx.x * warps + (threadIdx.x >> 5); tile < ntiles; tile += gridDim.x * warps) {
    const int r = tile * 32 + lane;
    const bool mine = sort_class(cls, r, A.rows);
    RowRuns rr;
    row_runs(A, B, r, mine, rr);
    uint8_t* m_row = map + tile_off[tile] + lane;   // product x of this row at m_row[32 * x]
    if (mine) {
      const int c0 = __ldg(C_rp + r), c1 = __ldg(C_rp + r + 1);
      int x = 0;
      for (int i = 0; i < rr.k; ++i) {
        for (int q = rr.src[i]; q < rr.src[i] + rr.len[i]; ++q, ++x) {
          const int col = __ldg(B.col + q);
          int lo = c0, hi = c1;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(C_col + mid) < col) lo = mid + 1; else hi = mid;
          }
          const bool found = lo < c1 && __ldg(C_col + lo) == col && lo - c0 < 256;
          if (!found) miss = true;
          m_row[32 * x] = (uint8_t)(found ? lo - c0 : 0);
        }
      }
    }
  }
  if (__any_sync(FULL, miss) && lane == 0) atomicOr(&ctr->status, ST_MISMATCH);
}

// Replay: lane t owns row tile*32 + t.  The warp zeroes its accumulator (the rows' entries of C,
// from +0.0); then all lanes walk their products x = 0, 1, ... together, in loop order, so that
// every FP64 instruction has the warp's lanes busy (this GB300 charges an FP64 instruction the
// full warp slot, whatever its active lanes), and the 32 map bytes of step x are one coalesced
// load.  Product x of a row belongs to the nonempty run counted by the run-start mask; its value
// of B is B.val[bofs(run) + x].  Values of CH steps are loaded together, then accumulated in
// order, and the warp stores the tile's values.
template <int N>
__global__ void __launch_bounds__(32)
k_replay(DevCsr A, DevCsr B, const uint8_t* __restrict__ cls, const int* __restrict__ C_rp,
         const int* __restrict__ tile_off, const uint8_t* __restrict__ map, double* __restrict__ C_val) {
  constexpr int CH = 8;
  __shared__ double acc[32 * N];
  __shared__ double s_a[RP_MERGE_K * 32];   // a_rj of the q-th nonempty run of lane t at [q * 32 + t]
  __shared__ int s_bofs[RP_MERGE_K * 32];   // B offset of that run: b of product x is B.val[bofs + x]
  const int lane = threadIdx.x & 31;
  const int ntiles = (A.rows + 31) >> 5;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int r = tile * 32 + lane;
    const bool mine = sort_class(cls, r, A.rows);
    RowRuns rr;
    row_runs(A, B, r, mine, rr);
    unsigned long long starts = 0;
    {
      int d = 0, q = 0;
#pragma unroll
      for (int i = 0; i < RP_MERGE_K; ++i) {
        if (rr.len[i] > 0) {
          if (d > 0) starts |= 1ull << d;
          s_a[q * 32 + lane] = __ldg(A.val + rr.a0 + i);
          s_bofs[q * 32 + lane] = rr.src[i] - d;
          ++q;
          d += rr.len[i];
        }
      }
    }
    int c0 = 0, cnt = 0;
    if (mine) { c0 = __ldg(C_rp + r); cnt = __ldg(C_rp + r + 1) - c0; }
    int TM;
    const int aoff = warp_excl_scan(cnt, &TM);    // this row's slice of the accumulator
    const uint8_t* m_row = map + tile_off[tile] + lane;
    for (int f = lane; f < TM; f += 32) acc[f] = 0.0;
    __syncwarp();
    double* a_row = acc + aoff;
    const int umax = __reduce_max_sync(FULL, rr.u);
    for (int x0 = 0; x0 < umax; x0 += CH) {
      double a[CH], b[CH];
      int pos[CH];
#pragma unroll
      for (int v = 0; v < CH; ++v) {
        const int x = x0 + v;
        a[v] = 0.0; b[v] = 0.0; pos[v] = N;
        if (x < rr.u) {
          const int run = __popcll(starts & ((2ull << x) - 1ull));
          b[v] = __ldg(B.val + s_bofs[run * 32 + lane] + x);
          a[v] = s_a[run * 32 + lane];
          pos[v] = __ldg(m_row + 32 * x);
        }
      }
#pragma unroll
      for (int v = 0; v < CH; ++v) {
        if (x0 + v < umax && pos[v] < cnt)   // pos >= cnt only for a mismatch, reported by the record
          a_row[pos[v]] = __fma_rn(a[v], b[v], a_row[pos[v]]);
      }
    }
    __syncwarp();
    // all rows of the tile in the sort classes and contiguous in C: one flat coalesced store
    const unsigned rows_mine = __ballot_sync(FULL, mine);
    const unsigned rows_in = __ballot_sync(FULL, r < A.rows);
    if (rows_mine == rows_in) {
      const int cbeg = __shfl_sync(FULL, c0, 0);
      for (int f = lane; f < TM; f += 32) C_val[cbeg + f] = acc[f];
    } else {
      for (unsigned rows = __ballot_sync(FULL, mine && cnt > 0); rows; rows &= rows - 1) {
        const int t = __ffs(rows) - 1;
        const int ct = __shfl_sync(FULL, cnt, t), ot = __shfl_sync(FULL, aoff, t), gt = __shfl_sync(FULL, c0, t);
        for (int o = lane; o < ct; o += 32) C_val[gt + o] = acc[ot + o];
      }
    }
    __syncwarp();
  }
}

void launch_replay_record(const DevCsr& A, const DevCsr& B, const uint8_t* cls, const int* C_rp, const int* C_col,
                          void* map, unsigned long long* scan_state, Counters* ctr, cudaStream_t s) {
  const int ntiles = (A.rows + 31) / 32;
  int* tile_off = (int*)map;
  uint8_t* bytes = (uint8_t*)map + (4 * ((size_t)ntiles + 1) + 255) / 256 * 256;
  const int grid = std::max(1, std::min((ntiles + 7) / 8, num_sms() * 8));
  cudaMemsetAsync(tile_off + ntiles, 0, sizeof(int), s);
  k_replay_count<<<grid, 256, 0, s>>>(A, B, cls, tile_off);
  cudaMemsetAsync(&ctr->ticket, 0, sizeof(unsigned), s);
  cudaMemsetAsync(scan_state, 0, scan_tile_state_bytes((long long)ntiles + 1), s);
  launch_scan(tile_off, (long long)ntiles + 1, scan_state, ctr, nullptr, s);
  k_replay_record<<<grid, 256, 0, s>>>(A, B, cls, C_rp, C_col, tile_off, bytes, ctr);
}

void launch_replay(int wide, const DevCsr& A, const DevCsr& B, const uint8_t* cls, const int* C_rp, const void* map,
                   double* C_val, cudaStream_t s) {
  const int ntiles = (A.rows + 31) / 32;
  const int* tile_off = (const int*)map;
  const uint8_t* bytes = (const uint8_t*)map + (4 * ((size_t)ntiles + 1) + 255) / 256 * 256;
  if (!wide) {
    const int per_sm = blocks_per_sm((const void*)k_replay<32>, 32, 0);
    const int grid = std::max(1, std::min(ntiles, num_sms() * per_sm));
    k_replay<32><<<grid, 32, 0, s>>>(A, B, cls, C_rp, tile_off, bytes, C_val);
  } else {
    const int per_sm = blocks_per_sm((const void*)k_replay<64>, 32, 0);
    const int grid = std::max(1, std::min(ntiles, num_sms() * per_sm));
    k_replay<64><<<grid, 32, 0, s>>>(A, B, cls, C_rp, tile_off, bytes, C_val);
  }
}

}  // namespace spg
