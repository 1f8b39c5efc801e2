/*
 * The paper's "Combined" row-major kernel (Section IV-B) for C = A * B on CSR matrices, on the
 * host cores: an optimised CPU baseline timed beside the GPU path.  It is neither the oracle nor
 * part of the GPU library: the benchmark times it and the tests check it against the oracle.
 *
 * Row r of C is accumulated into a dense temporary vector (the row-major loop of Section IV-A:
 * for every entry a_rj of row r of A, a_rj * b_jx is added at position x for every entry of row
 * j of B).  While the row is built, the touched columns go into an index list (a char flag per
 * column marks them), and their minimum and maximum are kept.  The row is then appended to C by
 * one of two storing strategies, chosen per row by a test meant to be cheap rather than exact:
 *   MinMax -- walk the temporary vector from the minimum to the maximum column, when that range
 *             is shorter than twice the number of the row's entries;
 *   Sort   -- otherwise sort the index list (std::sort) and visit only its columns.
 * Entries are kept by structure: the MinMax walk tests the flags, not the values, so an entry
 * whose products cancel to 0.0 is still stored (the paper's MinMax tests the double values and
 * would drop it).  With the products rounded on their own (no FMA contraction) and added in the
 * loop order, every value equals the oracle's bit for bit.
 *
 * C is one allocation of F entries (F = the number of multiplications, the estimate of Section
 * IV-B that never falls below nnz(C)), rows appended in order.  With several threads, the rows
 * are cut into chunks; each chunk is computed by one thread into the scratch arrays at its upper
 * bound offset (the multiplications of the rows before it), and a second pass packs the chunks
 * into C.  One thread writes C directly.
 *
 * Build: c++ -O3 -ffp-contract=off -fPIC -shared [-fopenmp].
 */
#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr int64_t CHUNK_ROWS = 1024;

struct RowBuffers {
  std::vector<double> acc;      // the dense temporary vector, all 0.0 between rows
  std::vector<char> flag;       // touched columns of the current row
  std::vector<int32_t> idx;     // the index list of the current row
  explicit RowBuffers(int64_t n, int64_t umax) : acc((size_t)n, 0.0), flag((size_t)n, 0), idx((size_t)std::max<int64_t>(umax, 1)) {}
};

// Rows [r0, r1) appended at out_col/out_val; row lengths to len[r - r0].  Returns the entries
// written, and counts the rows stored by each strategy.
int64_t rows_combined(int64_t r0, int64_t r1, const int32_t* A_rp, const int32_t* A_col, const double* A_val,
                      const int32_t* B_rp, const int32_t* B_col, const double* B_val, RowBuffers& rb,
                      int32_t* out_col, double* out_val, int64_t* len, int64_t* n_minmax, int64_t* n_sort) {
  double* acc = rb.acc.data();
  char* flag = rb.flag.data();
  int32_t* idx = rb.idx.data();
  int64_t pos = 0;
  for (int64_t r = r0; r < r1; ++r) {
    int32_t cnt = 0, mn = INT32_MAX, mx = -1;
    for (int32_t p = A_rp[r]; p < A_rp[r + 1]; ++p) {
      const int32_t j = A_col[p];
      const double a = A_val[p];
      for (int32_t q = B_rp[j]; q < B_rp[j + 1]; ++q) {
        const int32_t x = B_col[q];
        const double prod = a * B_val[q];
        acc[x] += prod;
        if (!flag[x]) {
          flag[x] = 1;
          idx[cnt++] = x;
          mn = std::min(mn, x);
          mx = std::max(mx, x);
        }
      }
    }
    const int64_t start = pos;
    if (cnt > 0) {
      if ((int64_t)mx - mn + 1 < 2 * (int64_t)cnt) {
        for (int32_t x = mn; x <= mx; ++x) {
          if (flag[x]) {
            out_col[pos] = x;
            out_val[pos] = acc[x];
            ++pos;
            flag[x] = 0;
            acc[x] = 0.0;
          }
        }
        ++*n_minmax;
      } else {
        std::sort(idx, idx + cnt);
        for (int32_t t = 0; t < cnt; ++t) {
          const int32_t x = idx[t];
          out_col[pos] = x;
          out_val[pos] = acc[x];
          ++pos;
          flag[x] = 0;
          acc[x] = 0.0;
        }
        ++*n_sort;
      }
    }
    len[r - r0] = pos - start;
  }
  return pos;
}

}  // namespace

extern "C" {

// Threads the library was built to use (1 without OpenMP).
int combined_max_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// F, the number of multiplications (the sum over A's entries of the length of the row of B they
// select), after checking every column index.  Returns -1 for an index out of range.  u[m]
// receives each row's count.
int64_t combined_products(int64_t m, int64_t k, const int32_t* A_rp, const int32_t* A_col, const int32_t* B_rp,
                          int64_t* u) {
  int64_t F = 0;
  bool bad = false;
  for (int64_t r = 0; r < m; ++r) {
    int64_t s = 0;
    for (int32_t p = A_rp[r]; p < A_rp[r + 1]; ++p) {
      const int32_t j = A_col[p];
      if (j < 0 || j >= k) { bad = true; continue; }
      s += B_rp[j + 1] - B_rp[j];
    }
    u[r] = s;
    F += s;
  }
  return bad ? -1 : F;
}

// C = A * B by the Combined kernel.  A is m x k and B is k x n, int32 indices, double values.
//   u        -- the per-row multiplication counts of combined_products; F their sum.
//   C_rp     -- m + 1 entries; C_col / C_val: F entries each.
//   S_col / S_val -- F entries each of scratch (used with more than one thread; may alias nothing).
//   stats    -- receives the rows stored by MinMax and by Sort.
// Returns nnz(C), or -1 if a column of B is out of range, -2 on allocation failure, -3 if the
// counts u do not sum to F.
int64_t combined_spgemm(int64_t m, int64_t k, int64_t n, const int32_t* A_rp, const int32_t* A_col,
                        const double* A_val, const int32_t* B_rp, const int32_t* B_col, const double* B_val,
                        const int64_t* u, int64_t F, int threads, int64_t* C_rp, int32_t* C_col, double* C_val,
                        int32_t* S_col, double* S_val, int64_t* stats) {
  stats[0] = stats[1] = 0;
  C_rp[0] = 0;
  if (m == 0) return 0;
  for (int64_t q = 0; q < B_rp[k]; ++q)
    if (B_col[q] < 0 || B_col[q] >= n) return -1;
  int64_t umax = 0, total = 0;
  for (int64_t r = 0; r < m; ++r) {
    umax = std::max(umax, u[r]);
    total += u[r];
  }
  if (total != F) return -3;
#ifndef _OPENMP
  threads = 1;
#endif
  if (threads <= 1) {
    try {
      RowBuffers rb(n, umax);
      std::vector<int64_t> len((size_t)m);
      const int64_t nnz = rows_combined(0, m, A_rp, A_col, A_val, B_rp, B_col, B_val, rb, C_col, C_val, len.data(),
                                        &stats[0], &stats[1]);
      for (int64_t r = 0; r < m; ++r) C_rp[r + 1] = C_rp[r] + len[(size_t)r];
      return nnz;
    } catch (...) {
      return -2;
    }
  }
  const int64_t nchunks = (m + CHUNK_ROWS - 1) / CHUNK_ROWS;
  std::vector<int64_t> ub((size_t)nchunks + 1, 0), got((size_t)nchunks, 0), off((size_t)nchunks + 1, 0);
  for (int64_t c = 0; c < nchunks; ++c) {
    int64_t s = 0;
    for (int64_t r = c * CHUNK_ROWS; r < std::min(m, (c + 1) * CHUNK_ROWS); ++r) s += u[r];
    ub[(size_t)c + 1] = ub[(size_t)c] + s;
  }
  int64_t minmax = 0, sorted = 0;
  bool failed = false;
#ifdef _OPENMP
#pragma omp parallel num_threads(threads) reduction(+ : minmax, sorted)
#endif
  {
    RowBuffers* rb = nullptr;
    try {
      rb = new RowBuffers(n, umax);
    } catch (...) {
      rb = nullptr;
    }
    if (!rb) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
      failed = true;
    }
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
    for (int64_t c = 0; c < nchunks; ++c) {
      if (!rb) continue;
      const int64_t r0 = c * CHUNK_ROWS, r1 = std::min(m, r0 + CHUNK_ROWS);
      got[(size_t)c] = rows_combined(r0, r1, A_rp, A_col, A_val, B_rp, B_col, B_val, *rb, S_col + ub[(size_t)c],
                                     S_val + ub[(size_t)c], C_rp + r0 + 1, &minmax, &sorted);
    }
    delete rb;
  }
  if (failed) return -2;
  for (int64_t c = 0; c < nchunks; ++c) off[(size_t)c + 1] = off[(size_t)c] + got[(size_t)c];
#ifdef _OPENMP
#pragma omp parallel for num_threads(threads) schedule(dynamic, 4)
#endif
  for (int64_t c = 0; c < nchunks; ++c) {
    const int64_t r0 = c * CHUNK_ROWS, r1 = std::min(m, r0 + CHUNK_ROWS);
    std::memcpy(C_col + off[(size_t)c], S_col + ub[(size_t)c], (size_t)got[(size_t)c] * sizeof(int32_t));
    std::memcpy(C_val + off[(size_t)c], S_val + ub[(size_t)c], (size_t)got[(size_t)c] * sizeof(double));
    int64_t p = off[(size_t)c];
    for (int64_t r = r0; r < r1; ++r) {   // lengths -> row pointer
      p += C_rp[r + 1];
      C_rp[r + 1] = p;
    }
  }
  stats[0] = minmax;
  stats[1] = sorted;
  return off[(size_t)nchunks];
}

}  // extern "C"
