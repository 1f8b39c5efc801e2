/*
 * spgemm_gb300.h -- C ABI of the GB300 sparse x sparse product C = A * B.
 *
 * The operation is the sparse matrix-matrix multiplication (spMMM) analysed in
 * Scharpff, Iglberger, Hager, Ruede, "Model-guided Performance Analysis of the
 * Sparse Matrix-Matrix Multiplication" (arXiv:1303.1651):
 *   - Section IV-A: the row-major (Gustavson) algorithm on three CSR matrices --
 *     row r of C is the sum over the entries a_rj of row r of A of a_rj times
 *     row j of B;
 *   - Section IV-B: the result is stored row by row, columns ascending within a
 *     row, into one contiguous block sized once from a never-underestimating nnz
 *     estimate (the number of multiplications);
 *   - Section III: the multiplication count sum_k nnz(A(:,k)) * nnz(B(k,:)) and
 *     the flop convention of two flops per multiplication.
 *
 * Matrices are CSR with int32 row pointers and column indices and float64
 * values (the paper stores 64-bit indices; this library uses 32-bit ones and
 * reports SPGEMM_ERR_OVERFLOW where a count does not fit).
 *
 * Semantics:
 *   - The structure of C is the union of the structures of the scaled rows of
 *     B: an entry whose products cancel to 0.0, or that comes from an explicit
 *     zero in A or B, is stored.
 *   - Rows of C come out sorted by column, without duplicates.
 *   - Rows of A and of B may be in any order and may repeat a column (repeated
 *     entries each contribute their products).
 *   - Each value of C is the FP64 sum of its products a_rj * b_jx, rounded to
 *     nearest.  Short rows (the sort classes) add them in storage order with
 *     fused multiply-adds, the first against +0.0.  Longer rows (the hash and
 *     dense classes) add separately rounded products in no fixed order.  An
 *     entry made of one product is exactly the rounded product in every class.
 *
 * Memory and ownership:
 *   - All matrix arrays and the workspace are DEVICE pointers owned by the
 *     caller, who must keep them alive and unchanged until the last call that
 *     uses them has completed on its stream.
 *   - The library allocates no device memory.  spgemm_plan allocates the small
 *     host-side plan object, which spgemm_free releases.  Once per process, on the
 *     first spgemm_plan, it also allocates an 18 KB pinned host buffer: each live plan
 *     reads its counters back through one slot of it.  Plans beyond its 256 slots
 *     use their own pageable copy.
 *   - A plan is not thread-safe.  Use it from one host thread and on one stream
 *     at a time.
 *
 * Streams: every call enqueues its work on `stream` (a cudaStream_t; NULL is the
 * legacy default stream).  spgemm_plan and spgemm_symbolic synchronise `stream`
 * before they return, to read back the row classes and nnz(C); spgemm_numeric
 * does not.
 *
 * Errors: every function returns an spgemm_status_t.  Device-side errors
 * (table overflow, a changed pattern, a bounded wait that gave up) are sticky
 * in the plan and are reported by the next synchronising call, or by
 * spgemm_status.  Each structure pass (spgemm_symbolic, spgemm_compute,
 * spgemm_compute_async) starts from a clear status, so a product can be retried
 * on the same plan, e.g. with a larger C after SPGEMM_ERR_OVERFLOW.  No kernel
 * traps or waits without a bound.
 */
#ifndef SPGEMM_GB300_H
#define SPGEMM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SPGEMM_OK = 0,
  SPGEMM_ERR_INVALID = 1,     /* bad argument: NULL pointer, negative size, A.cols != B.rows,
                                 a column index out of range, a decreasing row pointer */
  SPGEMM_ERR_ALLOC = 2,       /* the workspace passed is smaller than spgemm_workspace_size */
  SPGEMM_ERR_OVERFLOW = 3,    /* nnz(C) exceeds INT32_MAX (or the capacity given to spgemm_compute),
                                 or the products of one row exceed INT32_MAX */
  SPGEMM_ERR_TABLE_FULL = 4,  /* a hash table ran out of slots (cannot happen within the class limits) */
  SPGEMM_ERR_CUDA = 5,        /* a CUDA runtime call or launch failed */
  SPGEMM_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up */
  SPGEMM_ERR_STATE = 7,       /* calls made out of order (numeric before symbolic, ...) */
  SPGEMM_ERR_UNSORTED = 8,    /* reserved (inputs need not be sorted; not returned by this version) */
  SPGEMM_ERR_MISMATCH = 9,    /* numeric found a different structure than symbolic (inputs changed) */
  SPGEMM_ERR_SCRATCH_LIMIT = 10 /* a size exceeds the fixed scratch of spgemm_scan_counts_noalloc */
} spgemm_status_t;

/* A CSR matrix in device memory.  row_ptr has rows+1 entries with row_ptr[0] = 0 and
 * row_ptr[rows] = nnz; col_idx and val have nnz entries.  val may be NULL where only the
 * structure is read (spgemm_plan, spgemm_symbolic). */
typedef struct {
  int32_t rows;
  int32_t cols;
  int64_t nnz;
  const int32_t* row_ptr;
  const int32_t* col_idx;
  const double* val;
} spgemm_csr_t;

/* Tuning knobs.  A zero field takes the default.  Limits larger than what a class's kernel
 * can hold are clamped to it.  Row classes are chosen per row from k_r (the number of
 * entries of row r of A) and u_r (its multiplications), in the spirit of the per-row
 * strategy switch of the "Combined" kernel (Section IV-B). */
typedef struct {
  int32_t merge_max_k;    /* rows with k_r <= this (max 8) may use the merge classes (default 8).
                             The merge classes need B.cols <= 2^26 - 2 (their 32-bit sort keys hold
                             the column above 5 or 6 bits of product index); for wider B every row
                             goes to the classes below */
  int32_t m1_max_u;       /* class M1 (register sort of <= 32 products, one lane per row):
                             u_r <= this (max 32, default 32) */
  int32_t m2_max_u;       /* class M2 (register sort of <= 64 products; with the staged values,
                             two lanes per row): u_r <= this (max 64, default 64) */
  int32_t warp_max_u;     /* warp-per-row class W (bit vector over the row's column range; a
                             register sort across the warp when the range fits its 32-bit keys:
                             below 2^25 for u_r <= 128 down to 2^22 for u_r > 512, and for u_r <= 32
                             below 2^22 only; else a hash table): u_r <= this (max 1024, default
                             256; longer rows run faster in class B) */
  int32_t block_max_u;    /* block-per-row class B (the row's columns ordered by a bit vector over
                             windows of 2^18 columns, one window after another): u_r <= this (max
                             8192, default 8192); longer rows use a dense accumulator in global
                             memory (class G) */
  int32_t dense_slabs;    /* CTAs (each owning one dense accumulator of B.cols doubles and flags, 12
                             bytes per column) for class G; default: as many as fit in 128 MB, at
                             least 2 and at most one per SM of the current device */
  int32_t validate;       /* nonzero: also check row_ptr monotonicity and every column index of A and
                             B before planning (one extra pass over both matrices) */
  int32_t merge_values;   /* classes M1/M2: 0 automatic (default: the direct form for 32-product
                             tiles, the staged form for 64-product tiles), 1 direct: columns and
                             values read from B, C written from the reduce (little shared memory,
                             more warps; best when neighbouring rows of A reach neighbouring rows of
                             B), 2 staged: columns and values copied into shared memory with the
                             tile, C written by a coalesced pass */
  int32_t a_storage;      /* 0: A is in compressed rows (CSR).  1: A is in compressed columns (CSC): its
                             descriptor keeps A's own rows and cols, but row_ptr holds cols + 1 column
                             pointers and col_idx the row index of every entry, and A's values are
                             passed in that column-major order (Section IV-A, mixed storage orders).
                             The plan converts the structure once, into the workspace, with the
                             counting-sort transpose; every call that takes A's values gathers them
                             into row order first, and spgemm_backward returns dA in column order.
                             Within a row the converted entries are ordered by column, then by
                             position in the given arrays */
  int32_t b_storage;      /* the same for B */
  int32_t warp_bitvec_ratio;  /* class W: a row is ordered by a bit vector over its column range when
                             that range holds at most this many columns per product of the row
                             (1 .. 128, default 128, i.e. 4 bit-vector words per product).  2 is the
                             switch of the paper's "Combined" kernel (Section IV-B: MinMax when the
                             range is below twice the row's entries), with the row's products
                             standing in for its entries, which are not known before the ordering */
  int32_t warp_order;     /* class W: 0 automatic (the bit vector as above, else the register sort
                             when its keys fit, else the hash table), 1 the bit vector whenever the
                             range fits it (at most 4 words per product and 65536 columns), 2 the
                             register sort whenever its keys fit, 3 always the hash table */
  int32_t debug_spin_limit;   /* testing: rounds of re-reads after which a look-back of the single-pass
                             product gives up (0: 2^24).  With a small limit and debug_drop_tile, a
                             test can make the wait run out (SPGEMM_ERR_TIMEOUT) */
  int32_t debug_drop_tile;    /* testing: 0 none; t > 0: placement unit t - 1 of the single-pass product
                             (groups of 128 rows, or of 32 where some sort-class row has more than 32
                             products; tiles of 32 rows with merge_values = 2) publishes neither its
                             entry count nor its prefix, so the look-backs
                             that reach it give up after debug_spin_limit rounds.  C is then wrong
                             and spgemm_compute returns SPGEMM_ERR_TIMEOUT; nothing is written
                             outside the caller's buffers */
  int32_t reserved[2];
} spgemm_options_t;

/* Counters of a plan, valid after spgemm_plan (and nnz_c after spgemm_symbolic). */
typedef struct {
  int64_t products;       /* F = sum_r u_r: multiplications (Section III); flops = 2 F */
  int64_t nnz_c;          /* nnz(C), -1 before spgemm_symbolic */
  int32_t max_row_products;
  int32_t rows_per_class[5];   /* M1, M2, W, B, G */
} spgemm_info_t;

typedef struct spgemm_plan_s* spgemm_plan_t;

/* Bytes of device workspace that spgemm_plan needs for this A (rows) and B (cols).  It depends
 * only on the shapes and the options, not on the device data.  Returns SPGEMM_ERR_INVALID for
 * negative sizes or mismatched inner dimensions. */
spgemm_status_t spgemm_workspace_size(const spgemm_csr_t* A, const spgemm_csr_t* B, const spgemm_options_t* opt,
                                      size_t* bytes);

/* Plan C = A * B: a1 of the pipeline -- per-row multiplication counts u_r, the row classes
 * and per-class row lists, and F (Section III count; the Section IV-B nnz estimate).
 *   out        -- receives the new plan (host object; release it with spgemm_free).
 *   A, B       -- device CSR descriptors; only the structure is read here.  The descriptors are
 *                 copied; the arrays they point to must stay valid for the plan's lifetime.
 *   opt        -- may be NULL (defaults).
 *   workspace  -- device memory of at least workspace_bytes >= spgemm_workspace_size(...),
 *                 256-byte aligned, owned by the caller, used exclusively by this plan.
 * Enqueues on stream and synchronises it.  Errors: INVALID, ALLOC, OVERFLOW, CUDA. */
spgemm_status_t spgemm_plan(spgemm_plan_t* out, const spgemm_csr_t* A, const spgemm_csr_t* B,
                            const spgemm_options_t* opt, void* workspace, size_t workspace_bytes,
                            void* stream);

/* a2 + a3: count the distinct columns of every row of C and build C's row pointer.
 *   C_row_ptr -- device, A.rows + 1 int32, written with the exclusive prefix sums
 *                (C_row_ptr[0] = 0, C_row_ptr[rows] = nnz(C)).
 *   nnz_c     -- host, receives nnz(C) (size C_col/C_val with it).
 * Enqueues on stream and synchronises it.  Errors: STATE, OVERFLOW (nnz(C) > INT32_MAX),
 * TABLE_FULL, TIMEOUT, CUDA; after an error the plan holds no structure and spgemm_numeric
 * returns STATE.  May be called again (re-runs the symbolic pass). */
spgemm_status_t spgemm_symbolic(spgemm_plan_t plan, int32_t* C_row_ptr, int64_t* nnz_c, void* stream);

/* a4: compute C's column indices and values.
 *   A_val, B_val -- device values aligned with A's and B's entries (may differ between calls;
 *                   the structure must be the one planned).
 *   C_col, C_val -- device, nnz(C) entries each.  The C_row_ptr given to spgemm_symbolic must
 *                   still hold its result.
 * Enqueues on stream and returns without synchronising; repeatable.  Errors: STATE, INVALID
 * (NULL value pointers), CUDA.  A structure that changed since spgemm_symbolic is reported
 * as SPGEMM_ERR_MISMATCH by spgemm_status. */
spgemm_status_t spgemm_numeric(spgemm_plan_t plan, const double* A_val, const double* B_val, int32_t* C_col,
                               double* C_val, void* stream);

/* a2 + a3 + a4 in one pass: the whole product C = A * B after spgemm_plan, without the separate
 * symbolic pass.  As in Section IV-B, C is allocated once from the never-underestimating estimate
 * (the multiplication count F of spgemm_plan_info) and rows are appended in order: every tile
 * of 32 rows finds its offset in C from the tiles before it (decoupled look-back).
 *   A_val, B_val -- device values aligned with A's and B's entries.
 *   C_row_ptr    -- device, A.rows + 1 int32, written with C's row pointer.
 *   C_col, C_val -- device, `capacity` entries each; capacity >= F always suffices.
 *   nnz_c        -- host, receives nnz(C).
 * Enqueues on stream and synchronises it.  Errors: STATE, INVALID, OVERFLOW (nnz(C) > capacity or
 * > INT32_MAX; C's contents are then incomplete, but nothing is written past `capacity` entries
 * and C_row_ptr's entries are clamped to min(capacity, INT32_MAX)), TABLE_FULL, TIMEOUT, CUDA.  After it
 * succeeds, the plan is in the same state as after spgemm_symbolic: spgemm_numeric can recompute
 * values in place; after an error spgemm_numeric returns STATE. */
spgemm_status_t spgemm_compute(spgemm_plan_t plan, const double* A_val, const double* B_val, int32_t* C_row_ptr,
                               int32_t* C_col, double* C_val, int64_t capacity, int64_t* nnz_c, void* stream);

/* spgemm_compute without the host synchronisation, for CUDA-graph capture and for batches: the
 * work is only enqueued on stream.  nnz(C) lands in C_row_ptr[A.rows] and, if nnz_c_device is not
 * NULL, as an int64 in device memory at nnz_c_device.  Device errors are read by spgemm_status.
 * Capture it after spgemm_plan (which synchronises) and replay the graph as long as A's and B's
 * structures and the buffers stay the same; values may change between replays.  A batch of
 * independent products runs as one call on the block-diagonal matrices diag(A_1..A_P) and
 * diag(B_1..B_P): each problem's rows only reach its own block of B.
 * Errors: STATE, INVALID, CUDA. */
spgemm_status_t spgemm_compute_async(spgemm_plan_t plan, const double* A_val, const double* B_val,
                                     int32_t* C_row_ptr, int32_t* C_col, double* C_val, int64_t capacity,
                                     int64_t* nnz_c_device, void* stream);

/* The whole product in one call with one host synchronisation: spgemm_plan + spgemm_compute without
 * the read-back between them, for small products, where that read-back and the launches cost more
 * than the kernels.  As in Section IV-B, C is stored row by row into one block sized by the caller;
 * the call returns the multiplication count F (Section III), which always suffices as capacity.
 *   A, B         -- device descriptors WITH values (and the storage options of spgemm_plan).
 *   opt          -- may be NULL.
 *   workspace    -- as for spgemm_plan (spgemm_workspace_size bytes, 256-byte aligned).
 *   C_row_ptr    -- device, A.rows + 1 int32.
 *   C_col, C_val -- device, `capacity` entries each.
 *   nnz_c        -- host, receives nnz(C) (also on OVERFLOW).
 *   products     -- host, receives F (also on OVERFLOW): retry with capacity >= F.
 * No plan is kept.  The class kernels are launched before the row classes are known (each reads
 * its row count on the device), so a product whose rows all fall in one class still pays a few
 * empty launches.  Enqueues on stream and synchronises it once.  Errors: INVALID, ALLOC, OVERFLOW
 * (nnz(C) > capacity or > INT32_MAX; nothing is written past `capacity` entries), TABLE_FULL,
 * TIMEOUT, CUDA. */
spgemm_status_t spgemm_multiply(const spgemm_csr_t* A, const spgemm_csr_t* B, const spgemm_options_t* opt,
                                void* workspace, size_t workspace_bytes, int32_t* C_row_ptr, int32_t* C_col,
                                double* C_val, int64_t capacity, int64_t* nnz_c, int64_t* products, void* stream);

/* spgemm_multiply without the host synchronisation: the work is only enqueued on stream, and
 * nnz(C), F and the status stay in the workspace's counters, where spgemm_multiply_result reads
 * them.  Nothing the call enqueues depends on the data on the host side (every class kernel reads
 * its row count on the device), so the call can be captured into a CUDA graph once (after one
 * eager call, which sets the kernels' attributes) and the graph replayed for new contents of the
 * same arrays: a product of the same shapes per replay, with one read-back.  The class kernels
 * that do not depend on one another run on two internal streams, forked from and joined back to
 * stream by events within the call (a captured graph holds them side by side); the streams and
 * events are created on the calling thread's first call on a device and kept until it ends.  Errors: INVALID,
 * ALLOC, CUDA (host checks and launches; device errors are reported by spgemm_multiply_result). */
spgemm_status_t spgemm_multiply_async(const spgemm_csr_t* A, const spgemm_csr_t* B, const spgemm_options_t* opt,
                                      void* workspace, size_t workspace_bytes, int32_t* C_row_ptr, int32_t* C_col,
                                      double* C_val, int64_t capacity, void* stream);

/* Synchronise stream and read the counters that the last spgemm_multiply_async on `workspace` left
 * there: nnz(C) and F (host, always written), and the status (OK, OVERFLOW when nnz(C) passed the
 * capacity or INT32_MAX, TABLE_FULL, TIMEOUT, INVALID).  Errors: INVALID (NULL or misaligned
 * workspace), CUDA. */
spgemm_status_t spgemm_multiply_result(const void* workspace, int64_t* nnz_c, int64_t* products, void* stream);

/* Pattern reuse: new values of A and B, the same structures, C's structure kept.
 *
 * The row-major loop of Section IV-A visits the products of a row in a fixed order (A's entries
 * in storage order, each followed by its row of B in storage order), and the store of Section
 * IV-B gives each column of the row a fixed position in C.  spgemm_replay_record stores, once,
 * the position each product of the short rows lands on (the rows of the sort classes: at most
 * 8 entries of A and 64 products, so one byte per product).  spgemm_replay then recomputes C's
 * values as c[pos] = fma(a_rj, b_jx, c[pos]) in that loop order, without sorting or hashing.
 * On these rows its results equal spgemm_numeric's bit for bit.  Longer rows run
 * spgemm_numeric's own kernels, whose atomic sums have no fixed order (same tolerance).
 *
 * spgemm_replay_size: bytes of the position map, a device buffer the caller owns: 4 bytes per
 * tile of 32 rows, rounded up to 256, then 32 * U bytes per tile, U the longest short row (at
 * most 64 products; for the Laplacian^2 about F bytes in all).  Host only.
 * Errors: STATE (no plan), INVALID. */
spgemm_status_t spgemm_replay_size(spgemm_plan_t plan, size_t* bytes);

/* Record the position map for C's current structure.  Needs the plan after spgemm_symbolic +
 * spgemm_numeric, or after spgemm_compute.  C_col holds C's column indices (device).  map is
 * device memory, 256-byte aligned, of at least spgemm_replay_size bytes, and is kept by the
 * plan for spgemm_replay.  Enqueues on stream and synchronises it.  Errors: STATE, INVALID,
 * ALLOC, OVERFLOW (the map would pass INT32_MAX bytes), MISMATCH (a product's column is
 * not in its row of C: C_col is not this product's structure), CUDA. */
spgemm_status_t spgemm_replay_record(spgemm_plan_t plan, const int32_t* C_col, void* map, size_t map_bytes,
                                     void* stream);

/* Recompute C's values from new values of A and B with the map recorded for this plan.  C_val
 * (device, nnz(C)) is written; C_col (device) is rewritten, with the same indices, for the rows
 * outside the sort classes.  Enqueues on stream; no synchronisation; repeatable.  Errors: STATE
 * (no map recorded for this plan, or another map passed), INVALID, CUDA. */
spgemm_status_t spgemm_replay(spgemm_plan_t plan, const double* A_val, const double* B_val, const void* map,
                              int32_t* C_col, double* C_val, void* stream);

/* Bytes of device workspace spgemm_backward needs to form dB: the transpose of A's structure (the
 * CSR -> CSC conversion of Section IV-A).  Errors: INVALID. */
spgemm_status_t spgemm_backward_workspace_size(const spgemm_csr_t* A, const spgemm_csr_t* B, size_t* bytes);

/* Gradients of a loss L through C = A * B, given dC = dL/dC on C's structure (aligned with C_col):
 *   dA_ij = sum_x B_jx dC_ix  for every entry (i, j) of A   (aligned with A's entries),
 *   dB_jx = sum_i A_ij dC_ix  for every entry (j, x) of B   (aligned with B's entries).
 * Needs the plan after spgemm_compute / spgemm_numeric (C's structure).  dA_val or dB_val may be
 * NULL to skip it; B_val is read for dA and A_val for dB.  workspace (device, 256-byte aligned, at
 * least spgemm_backward_workspace_size bytes) is needed only for dB; the transpose built in it is
 * kept and reused while the same workspace is passed.  Each entry accumulates its terms in
 * storage order with fused multiply-adds.  Enqueues on stream; no synchronisation.
 * Errors: STATE, INVALID, ALLOC, CUDA; a term missing from C's structure sets SPGEMM_ERR_MISMATCH
 * (read by spgemm_status). */
spgemm_status_t spgemm_backward(spgemm_plan_t plan, const double* A_val, const double* B_val, const double* dC_val,
                                double* dA_val, double* dB_val, void* workspace, size_t workspace_bytes,
                                void* stream);

/* Synchronise stream and report the plan's sticky device status (OK or the first error). */
spgemm_status_t spgemm_status(spgemm_plan_t plan, void* stream);

/* Copy the plan's counters (host-side copies; no synchronisation). */
spgemm_status_t spgemm_plan_info(spgemm_plan_t plan, spgemm_info_t* info);

/* Optional timing hook: two cudaEvent_t created by the caller (or both NULL to clear).  From now on
 * spgemm_numeric and spgemm_compute record start_event on their stream right before their first
 * compute kernel and stop_event right after their last one, so a caller can time the kernels
 * without the host synchronisation that spgemm_compute performs.  Errors: INVALID. */
spgemm_status_t spgemm_plan_set_events(spgemm_plan_t plan, void* start_event, void* stop_event);

/* Release the plan object.  The workspace stays the caller's.  NULL is accepted. */
spgemm_status_t spgemm_free(spgemm_plan_t plan);

/* Row pointers from per-row counts, without a workspace and without allocating.
 *
 * The paper has no counterpart to this entry point; it exists for callers that can neither
 * allocate device memory nor lend a workspace when they call, for instance code running where
 * another framework's pooling allocator has reserved the device memory, or a service that keeps
 * a fixed memory footprint after start-up.  For them an allocation at call time could fail, or
 * would change a footprint they must hold constant.
 *
 * It performs the step that spgemm_symbolic uses to turn the per-row entry counts of C into C's
 * row pointers: an exclusive prefix sum of the per-row counts into row pointers, by the same
 * single-pass scan kernel.  Instead of a workspace, the scan's scratch
 * (one state word per 2048 rows plus a 256-byte header) lives in a fixed device array of
 * SPGEMM_NOALLOC_SCRATCH_BYTES bytes, which every device that runs this call keeps until the
 * process exits.  That array bounds the size: at most SPGEMM_NOALLOC_MAX_ROWS rows.
 *
 *   row_ptr  DEVICE, rows + 1 int32, caller-owned, updated in place.  On entry row_ptr[r] is the
 *            count of row r (>= 0) for r < rows; row_ptr[rows] is ignored.  On return row_ptr[r]
 *            is the sum of the counts of rows 0 .. r-1, so row_ptr[0] = 0 and row_ptr[rows] is
 *            the total.
 *   rows     number of rows, 0 <= rows <= SPGEMM_NOALLOC_MAX_ROWS.
 *   total    HOST, may be NULL: receives the total as a 64-bit count (also on OVERFLOW).
 *   stream   cudaStream_t of the current device.  The call synchronises it before it returns.
 *
 * Errors: INVALID (row_ptr NULL, rows < 0); SCRATCH_LIMIT (rows > SPGEMM_NOALLOC_MAX_ROWS:
 * rejected before any CUDA call, row_ptr untouched); OVERFLOW (a prefix sum exceeds INT32_MAX,
 * entries past it are stored as INT32_MAX); TIMEOUT; CUDA.
 *
 * Set-up: every call looks up the device address of the scratch array in the current context
 * (the lookup allocates nothing), so a device reset or another context between calls is safe.
 *
 * Capture: the call copies its counters to the host and synchronises `stream`, so it must not be
 * called while `stream` (or, in the global capture mode, any stream) is being captured into a
 * CUDA graph.
 *
 * Concurrency: all calls on one device share the one scratch array.  Calls that overlap in time,
 * from several host threads or on several streams, race on it and give wrong results: serialise
 * them. */
#define SPGEMM_NOALLOC_MAX_ROWS 67108863          /* 2^26 - 1 */
#define SPGEMM_NOALLOC_SCRATCH_BYTES 262400       /* 256 + 8 * 2^26 / 2048 */
spgemm_status_t spgemm_scan_counts_noalloc(int32_t* row_ptr, int64_t rows, int64_t* total, void* stream);

/* Static string naming a status code. */
const char* spgemm_error_string(int code);

/* Library version as major * 10000 + minor * 100 + patch. */
int32_t spgemm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SPGEMM_GB300_H */
