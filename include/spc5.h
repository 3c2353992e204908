/*
 * spc5.h -- C ABI of the GB300 SPC5 library.
 *
 * SPC5 (Regnault & Bramas, "SPC5: an efficient SpMV framework vectorized
 * using ARM SVE and x86 AVX-512") stores a sparse matrix in the beta(r,c)
 * block format (Section 2.4): rows are grouped into panels of r rows; each
 * block of a panel holds one start column and r masks of c bits (bit k of
 * row q set <=> the entry at column start + k of that row exists); only the
 * nonzeros are stored, packed in the order in which Algorithm 1 visits them
 * (block by block, row by row, ascending bit).  y = A x over that format is
 * Algorithm 1.
 *
 * Conventions for every entry point:
 *   - Sizes and indices are 64-bit in the signatures; the stored matrix uses
 *     32-bit indices, so nrows, ncols, nnz and the number of blocks must stay
 *     below 2^31 (else SPC5_EOVERFLOW).
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Work is enqueued on it.
 *   - Array arguments may live in device memory or in host memory; the
 *     library asks the CUDA runtime which one (cudaPointerGetAttributes).
 *     Host arguments are copied through device buffers (spc5_spmv writes a
 *     pinned host y in place through its device mapping) and make the call
 *     blocking.
 *   - No call throws, aborts or uses a device fault to report an error: every
 *     failure is a returned spc5_status, and spc5_last_error() gives a
 *     one-line description of the last failure on the calling thread.
 *   - Layouts are C order; all arrays are borrowed (never freed or kept)
 *     unless stated otherwise.
 */
#ifndef SPC5_H
#define SPC5_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque handle of a matrix converted to beta(r,c); owns its device arrays. */
typedef struct spc5_matrix spc5_matrix;

/* Opaque handle of a batch of products (see spc5_batch_create). */
typedef struct spc5_batch spc5_batch;

/* Element types.  Input values are FP64; the converted values are stored
 * in FP64, FP32 or BF16 (rounded to nearest, ties to even).  An FP64 matrix
 * multiplies FP64 vectors with FP64 accumulation; FP32 and BF16 matrices
 * multiply FP32 vectors with FP32 accumulation. */
typedef enum { SPC5_F64 = 0, SPC5_F32 = 1, SPC5_BF16 = 2 } spc5_dtype;

typedef enum {
  SPC5_OK = 0,
  SPC5_EINVAL = 1,          /* null handle or pointer, negative size, bad alpha/beta use */
  SPC5_EUNSORTED = 2,       /* a row's column indices are not strictly ascending */
  SPC5_EUNSUPPORTED_RC = 3, /* (r, c) is not a supported block shape */
  SPC5_EOVERFLOW = 4,       /* a size does not fit 32-bit indexing */
  SPC5_ECUDA = 5,           /* a CUDA runtime call failed */
  SPC5_ENOMEM = 6,          /* a device or pinned-host allocation failed */
  SPC5_EDEVICE = 7,         /* a kernel reported an internal inconsistency */
  SPC5_ERANGE = 8,          /* a column index lies outside [0, ncols) */
  SPC5_EROWPTR = 9,         /* rowptr[0] != 0, rowptr decreasing, or rowptr[nrows] != nnz */
  SPC5_EUNSUPPORTED = 10    /* a requested option or dtype is not implemented */
} spc5_status;

/* Description of a converted matrix. */
typedef struct {
  int64_t nrows, ncols, nnz;
  int32_t r, c;            /* block shape beta(r,c) */
  int64_t npanels;         /* ceil(nrows / r) */
  int64_t nblocks;         /* number of blocks */
  double filling;          /* nnz / (nblocks * r * c): Table 1's block filling */
  spc5_dtype value_dtype;  /* storage type of the values */
  int32_t mask_bytes;      /* bytes of one block's packed mask word: r * c / 8 */
  int64_t device_bytes;    /* device memory held by the handle */
  int32_t device;          /* CUDA device ordinal the matrix lives on */
  int32_t lanes_per_row;   /* lanes sharing one row in the SpMV's row groups (1, 2, 4, ...) */
  int32_t launches_per_spmv; /* kernel launches one spc5_spmv call makes (1, or 2 with pieces) */
  int64_t ntiles;          /* work tiles of the plan the SpMV uses */
  int64_t long_panels;     /* panels split into pieces whose partial sums are added in order */
  int32_t stages;          /* shared-memory pipeline stages per SM */
  int32_t consumers;       /* consumer warps per SM */
  uint32_t device_error;   /* nonzero if a kernel gave up a bounded wait (reading it syncs) */
  double tuned_us;         /* SpMV time of the plan chosen by spc5_tune, 0 if untuned */
  int32_t flat;            /* work mapping of the SpMV: 0 lanes own rows (row-group plan);
                              1 blocks dealt to lanes evenly (block-balanced plan);
                              2 each tile's values split evenly over the lanes (expanded);
                              3 block-balanced tiles, each round's values split evenly over
                              the lanes (value-balanced) */
  double group_efficiency; /* busy share of the row-group plan's block slots; below 0.7 the
                              converter picks plan 3 for r >= 4 and plan 1 for r <= 2 */
  int32_t hybrid;          /* 1 for a matrix from spc5_convert_hybrid */
  int64_t nscalars;        /* hybrid: single-value blocks stored as scalars (nnz counts them;
                              nblocks and filling describe the remaining blocks) */
  double tuned_rows_us;    /* SpMV time of the fastest row-group plan spc5_tune tried (the
                              plan of the batched, transposed and gradient kernels), 0 if
                              untuned */
  int64_t pieces;          /* pieces the SpMV's plan cuts long panels into (r partial sums
                              each) */
  int64_t scalar_pieces;   /* hybrid: pieces of long scalar rows (one partial sum each) */
  int32_t body;            /* row-group plan's loop: 0 per-block set-bit loop, 1 predicated
                              loop over the c bits, 2 row stream, 3 queued row stream,
                              4 four-block rounds, 5 row stream passing empty blocks,
                              6 row stream at 64 warps per SM, 7 pipelined row stream
                              passing empty blocks */
  int32_t dynamic;         /* 1 if row-group tiles are taken from a counter, 0 grid-stride */
  int32_t transposed;      /* 1 if spc5_build_transpose attached a transposed copy */
  int32_t halves;          /* 1 if the row-group plan cut the groups of the last round of
                              tiles into two half tiles (tried by spc5_tune, kept when
                              faster; it applies when that round fills at most half the
                              resident warps) */
} spc5_info;

/*
 * spc5_convert_csr -- build beta(r,c) from CSR (Section 2.4).
 *
 * Block rule: within each panel of r consecutive rows (the last panel may be
 * shorter), the smallest column of the rows' union that no block covers yet
 * opens a block covering columns [start, start + c) in all r rows; blocks
 * are ordered by ascending start.  For r = 1 this is the paper's rule that a
 * block starts at a nonzero and takes the next nonzeros up to start + c - 1.
 *
 * nrows, ncols, nnz  matrix shape and number of stored entries
 * rowptr[nrows+1]    CSR row pointers, rowptr[0] = 0, rowptr[nrows] = nnz
 * colidx[nnz]        column of every entry, strictly ascending in each row
 * vals[nnz]          values of type vals_dtype (must be SPC5_F64)
 * store_dtype        storage type of the converted values: SPC5_F64, or
 *                    SPC5_F32 / SPC5_BF16 (round to nearest even from FP64)
 * r, c               block shape; (1,8) (2,4) (2,8) (4,4) (4,8) (8,4) are
 *                    supported, others give SPC5_EUNSUPPORTED_RC
 * stream             stream the conversion runs on; the call returns after
 *                    the conversion has finished (it reads back the block
 *                    count to size the arrays)
 * out                receives the new handle (unchanged on failure)
 *
 * Validation (sorted unique columns, column range, row pointers) runs on
 * the device before any index is trusted.  Explicitly stored zeros are kept.
 *
 * Memory: besides the handle's arrays, a conversion takes temporary scratch
 * (about 12 bytes per entry, more for very long rows) from a private
 * stream-ordered memory pool of the device.  The pool keeps up to 8 GiB of
 * it mapped between calls, so that later conversions skip the mapping; the
 * process holds that memory until it exits, and anything above 8 GiB is
 * returned at the next synchronisation.
 */
spc5_status spc5_convert_csr(int64_t nrows, int64_t ncols, int64_t nnz, const int32_t *rowptr,
                             const int32_t *colidx, const void *vals, spc5_dtype vals_dtype,
                             spc5_dtype store_dtype, int r, int c, void *stream,
                             spc5_matrix **out);

/*
 * spc5_convert_hybrid -- the hybrid form the paper proposes for low-filling
 * matrices (closing remarks: SPC5 is slower than CSR below about two values
 * per block, so mix the block format with a scalar one).  Converts like
 * spc5_convert_csr, then moves every block whose r masks hold exactly one
 * set bit to a CSR of scalars (row, column, value; each row's columns
 * ascending); the other blocks stay a beta(r,c) matrix with values in
 * Algorithm 1's order.  A single-value block's bit is its block's first
 * column, so a scalar's column is its block's start column.
 *
 * spc5_spmv, spc5_spmv_noalloc, spc5_tune, spc5_ircg, spc5_matrix_info,
 * spc5_export (the block part) and spc5_export_hybrid (the scalars) take the
 * handle; the transposed product, the value gradient, spc5_set_values and
 * the batched product give SPC5_EUNSUPPORTED.  Same arguments, ownership
 * and errors as spc5_convert_csr.
 */
spc5_status spc5_convert_hybrid(int64_t nrows, int64_t ncols, int64_t nnz, const int32_t *rowptr,
                                const int32_t *colidx, const void *vals, spc5_dtype vals_dtype,
                                spc5_dtype store_dtype, int r, int c, void *stream,
                                spc5_matrix **out);

/*
 * spc5_export_hybrid -- device pointers to a hybrid matrix's scalars, owned
 * by the handle: s_rowptr[nrows + 1] (int32), s_colidx[nscalars] (int32),
 * s_vals[nscalars] in the storage type.  SPC5_EINVAL if A is not hybrid.
 * Any output pointer may be NULL.
 */
spc5_status spc5_export_hybrid(const spc5_matrix *A, const int32_t **s_rowptr,
                               const int32_t **s_colidx, const void **s_vals);

/* Fill *info with the matrix description (host-only, no device work). */
spc5_status spc5_matrix_info(const spc5_matrix *A, spc5_info *info);

/*
 * spc5_export -- device pointers to the converted arrays (owned by A, valid
 * until spc5_destroy).  Any output pointer may be NULL.
 *   block_rowptr[npanels+1] int32  first block of each panel (Algorithm 1's
 *                                  mat.block_rowptr)
 *   panel_vptr[npanels+1]   int32  offset of each panel's first value (equal
 *                                  to the CSR row pointer of the panel's first
 *                                  row); lets a panel be processed without
 *                                  summing the popcounts of all earlier blocks
 *   block_colidx[nblocks]   int32  start column of each block (idxCol)
 *   block_masks[nblocks]           one little-endian word of r*c bits per
 *                                  block (uint8 for r*c = 8, uint16 for 16,
 *                                  uint32 for 32), row q at bits [q*c, (q+1)*c):
 *                                  for c = 8 the bytes equal the paper's
 *                                  block_masks[idxBlock * r + idxRowBlock]
 *   values[nnz]                    packed values in Algorithm 1's idxVal order
 */
spc5_status spc5_export(const spc5_matrix *A, const int32_t **block_rowptr,
                        const int32_t **panel_vptr, const int32_t **block_colidx,
                        const void **block_masks, const void **values);

/*
 * spc5_spmv -- y = alpha * A x + beta * y (Algorithm 1 computes y = A x).
 *
 * x[ncols], y[nrows] are vectors in device or host memory: FP64 for an
 * FP64 matrix, FP32 for FP32 and BF16 matrices (accumulation in the vector
 * type).  With beta == 0, y is not read (no NaN or Inf from a previous y
 * propagates).
 * Device vectors: asynchronous on `stream`.  Host vectors: x (and a pageable
 * y) are copied through device buffers owned by A; a pinned (page-locked)
 * host y is written in place by the kernels through its device mapping, so
 * the result crosses to the host while the product runs; the call returns
 * when y is on the host.  x and y
 * must not overlap; device memory of another GPU than the matrix's gives
 * SPC5_EINVAL.  Products on the same handle whose kernels could overlap
 * on the GPU (different streams) must be serialised by the caller: they
 * share the handle's buffer of partial sums and its tile counter.
 *
 * Work mapping (chosen at conversion, see spc5_info.flat): lanes own rows
 * of groups of panels (row-group plan); or, for matrices whose rows have
 * very different lengths, the blocks of runs of panels are dealt to the
 * lanes evenly and row sums are assembled by a segmented warp scan
 * (block-balanced plan), or a warp lays the values of a run of panels out
 * row by row in shared memory and splits them evenly over its lanes
 * (expanded plan).  All give y within the same error bound; the summation
 * order differs.
 */
spc5_status spc5_spmv(const spc5_matrix *A, const void *x, void *y, double alpha, double beta,
                      void *stream);

/*
 * spc5_spmv_t -- dx = alpha * A^T g + beta * dx, the product with the
 * transposed matrix (the input gradient of y = A x: dx = A^T dy).  With a
 * transposed copy (spc5_build_transpose) it is spc5_spmv over that copy:
 * deterministic.  Without one it walks the stored blocks of Algorithm 1's
 * layout and scatters values[idxVal] * g[row] into dx[idxCol + k] with
 * atomic additions, so the summation order (and the last bits of the
 * result) may differ from run to run.  g[nrows] and dx[ncols] are device
 * vectors typed as for spc5_spmv.  With beta == 0, dx is not read.
 * Asynchronous on `stream`.
 */
spc5_status spc5_spmv_t(const spc5_matrix *A, const void *g, void *dx, double alpha, double beta,
                        void *stream);

/*
 * spc5_build_transpose -- attach to A its transpose A^T, converted to
 * beta(r,c) with A's block shape and storage type (Section 2.4's rule
 * applied to the columns of A), so that spc5_spmv_t becomes an ordinary
 * product over A^T (Algorithm 1): deterministic, and as fast as a forward
 * product.  The paper transposes nothing; this is the backward product of
 * the differentiation extension.  Built on the device from A's stored blocks
 * (the CSR A came from is not needed); the copy belongs to A (released by
 * spc5_destroy(A)), spc5_set_values(A, vals) updates it too, and calling
 * again rebuilds it.  A must be a plain (not hybrid) matrix on the current
 * device.  Errors: SPC5_EUNSUPPORTED for a hybrid matrix or when a column
 * of A holds more than 65536 entries (spc5_spmv_t then keeps its atomic
 * scatter), SPC5_EDEVICE, SPC5_ECUDA / SPC5_ENOMEM from the conversion.
 * Synchronises `stream`; allocates about 5 times A's value bytes of
 * temporaries while it runs and a second matrix of A's size.
 */
spc5_status spc5_build_transpose(spc5_matrix *A, void *stream);

/*
 * spc5_values_grad -- dvals[e] = alpha * g[row(e)] * x[col(e)] for every
 * stored entry e (the gradient of <g, A x> with respect to the matrix
 * values), computed over the stored mask bits and written in CSR order
 * (dvals[e] belongs to the e-th entry of the CSR given to spc5_convert_csr).
 * g[nrows], x[ncols], dvals[nnz]: device arrays, FP64 for an FP64 matrix,
 * FP32 otherwise.  Asynchronous on `stream`.
 */
spc5_status spc5_values_grad(const spc5_matrix *A, const void *g, const void *x, void *dvals,
                             double alpha, void *stream);

/*
 * spc5_set_values -- replace the stored values with vals[nnz] (FP64, device
 * memory, CSR order of the conversion), keeping the pattern, the blocks and
 * the work plan; values are rounded to the matrix's storage type.  For
 * matrices whose values change while the pattern does not (training,
 * Newton iterations).  Asynchronous on `stream`.
 */
spc5_status spc5_set_values(spc5_matrix *A, const double *vals, void *stream);

/*
 * spc5_tune -- autotune the SpMV mapping of a converted matrix: time the
 * candidate plans (lanes sharing one row: 1, 2, 4, 8, those that fit 32 / r,
 * with the one-lane-per-row bodies; the two block-balanced plans; the
 * expanded plan) over `iters` products with the caller's vectors x and y
 * (device memory, typed as for spc5_spmv; y is overwritten) and keep the
 * fastest, with the fastest row-group plan kept for the transposed,
 * gradient and batched kernels (spc5_info.tuned_us, tuned_rows_us).  The
 * paper observes that the best blocking depends on the machine and the
 * matrix (Section 4.3); the tuner measures instead of modelling.
 * Synchronises `stream`; rebuilds the plan (reallocates its buffers).
 */
spc5_status spc5_tune(spc5_matrix *A, const void *x, void *y, int iters, void *stream);

/*
 * spc5_convert_tuned -- spc5_convert_csr into each block shape of
 * `shapes` (nshapes (r, c) pairs; NULL = all six supported shapes), each
 * tuned by spc5_tune on a zero vector, keeping the matrix with the fastest
 * product.  Same arguments and ownership as spc5_convert_csr otherwise.
 */
spc5_status spc5_convert_tuned(int64_t nrows, int64_t ncols, int64_t nnz, const int32_t *rowptr,
                               const int32_t *colidx, const void *vals, spc5_dtype vals_dtype,
                               spc5_dtype store_dtype, const int *shapes, int nshapes, int iters,
                               void *stream, spc5_matrix **out);

/*
 * spc5_convert_tuned_ex -- spc5_convert_tuned with the ranking chosen by
 * `rows_plan`: 0 ranks the shapes by their fastest SpMV plan (as
 * spc5_convert_tuned); nonzero ranks them by their fastest row-group plan,
 * the plan that spc5_spmv_batched, spc5_spmv_t and spc5_values_grad run
 * (spc5_info.tuned_rows_us).  The matrix returned is tuned as by spc5_tune.
 */
spc5_status spc5_convert_tuned_ex(int64_t nrows, int64_t ncols, int64_t nnz,
                                  const int32_t *rowptr, const int32_t *colidx, const void *vals,
                                  spc5_dtype vals_dtype, spc5_dtype store_dtype, const int *shapes,
                                  int nshapes, int iters, int rows_plan, void *stream,
                                  spc5_matrix **out);

/*
 * spc5_spmv_batched -- Y[m] = A[m] X[m] for m < nmat in one launch, with k
 * right-hand sides per matrix (k in {1, 2, 4, 8, 16}).  X[m] is row-major
 * [ncols_m][k] and Y[m] row-major [nrows_m][k], device memory, FP64 for FP64
 * matrices and FP32 otherwise; all matrices share one value dtype and one
 * device and may have different sizes and block shapes.  Creates a batch,
 * runs it once and destroys it; synchronises `stream`.  Algorithm 1 applied
 * to many matrices and vectors at once (the paper's kernel handles one).
 */
spc5_status spc5_spmv_batched(int nmat, const spc5_matrix *const *A, const void *const *X,
                              void *const *Y, int k, void *stream);

/*
 * spc5_batch_create -- prepare the batch above for repeated runs: builds, in
 * device memory owned by the batch, a table of the matrices' arrays and the
 * vectors' addresses, a map from global work tile to matrix and a buffer for
 * the partial sums of split panels (k per row).  The matrices and vectors
 * must outlive the batch; their addresses are fixed at creation.
 * Synchronises `stream`.
 */
spc5_status spc5_batch_create(int nmat, const spc5_matrix *const *A, const void *const *X,
                              void *const *Y, int k, void *stream, spc5_batch **out);

/*
 * spc5_batch_run -- Y[m] = alpha * A[m] X[m] + beta * Y[m] for the whole
 * batch: one persistent kernel over all matrices' tiles plus one fixup
 * kernel when some panel was split.  Asynchronous; allocates nothing and
 * copies nothing from the host, so it can be captured in a CUDA graph.
 */
spc5_status spc5_batch_run(const spc5_batch *B, double alpha, double beta, void *stream);

/* Release a batch (synchronising). */
spc5_status spc5_batch_destroy(spc5_batch *B);

/* Outcome of spc5_ircg. */
typedef struct {
  int32_t outer_iters; /* refinement steps taken (FP64 residuals computed = outer_iters + 1) */
  int32_t inner_iters; /* inner CG iterations, summed over the refinement steps */
  double relres;       /* ||b - A64 x|| / ||b|| at the last FP64 residual */
} spc5_cg_report;

/*
 * spc5_ircg -- solve A x = b for a symmetric positive definite A by
 * mixed-precision iterative refinement: FP64 outer residual r = b - A64 x
 * (spc5_spmv on the FP64 matrix), FP64 norms and updates x += ||r|| d, and
 * an inner conjugate-gradient solve of Alo d = r / ||r|| with FP32 vectors
 * (FP64 dot-product accumulation) on Alo, the same matrix stored in FP32
 * or BF16 (or FP64: then the inner solve runs in FP64).  The iterative
 * solvers that motivate a fast SpMV (Section 1) are the use case; the
 * solver itself is not part of the paper.
 *   A64, Alo   the matrix in FP64 and in the inner precision (same pattern
 *              and size, square); b[n], x[n] FP64 device vectors, x holds
 *              the initial guess on entry and the solution on return
 *   tol        stop when ||b - A64 x|| <= tol ||b||
 *   max_outer  maximum refinement steps
 *   inner_tol  relative residual at which an inner solve stops (0 < . < 1)
 *   max_inner  maximum CG iterations per inner solve
 * One inner iteration is captured once as a CUDA graph and replayed; the
 * host reads the inner r.r every 8 iterations and ||r|| once per step.
 * Synchronises `stream`; allocates work vectors (5 n) for the call.
 */
spc5_status spc5_ircg(const spc5_matrix *A64, const spc5_matrix *Alo, const double *b, double *x,
                      double tol, int max_outer, double inner_tol, int max_inner, void *stream,
                      spc5_cg_report *report);

/*
 * spc5_spmv_noalloc -- the same product as spc5_spmv for callers that must
 * not allocate device memory during the call: a real-time loop that must
 * never reach the allocator (or the device-wide synchronisation a cudaFree
 * implies), a library that may use only the memory its host application
 * hands it, or code under a device-memory budget fixed at start-up.  The
 * paper has no counterpart: this is a deployment variant of Algorithm 1's
 * product, not part of the method.
 *
 * x[ncols], y[nrows] must be in device (or managed) memory, typed as for
 * spc5_spmv (FP64 for an FP64 matrix, FP32 otherwise);
 * host vectors give SPC5_EINVAL, since copying them needs staging buffers.
 * The partial sums of panels that the work plan splits into pieces go to a
 * fixed array inside the library (1 MiB = 131072 doubles, kept on every
 * GPU that loads the library until the process exits) instead of the
 * handle's own buffer; a matrix needing more than 131072 partial sums
 * (spc5_info.pieces * r + spc5_info.scalar_pieces) is rejected with
 * SPC5_EOVERFLOW before any work is queued.  x and y must be memory of the
 * matrix's device (or managed memory), else SPC5_EINVAL.
 * The call makes no cudaMalloc, cudaFree or other allocating call.
 *
 * The tile counter of the block-balanced and expanded plans is likewise a
 * fixed pair of 32-bit words inside the library; every launch leaves it at
 * zero.
 *
 * The array and the counter are shared by every call on a device:
 * concurrent calls whose kernels overlap on the GPU (different streams, or
 * different handles at once) race on them and must be serialised by the
 * caller.  No state carries over between calls (each call writes every
 * partial sum it reads).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.
 */
spc5_status spc5_spmv_noalloc(const spc5_matrix *A, const void *x, void *y, double alpha,
                              double beta, void *stream);

/*
 * spc5_measure_fma_peak -- measured FMA throughput of the current device in
 * TFLOP/s (2 flop per FMA), for dtype SPC5_F64 or SPC5_F32: a kernel of
 * eight independent FMA chains per thread on every SM, the best of five
 * timed launches (CUDA events on `stream`).  Not part of the paper: the
 * arithmetic ceiling that SpMV throughput is reported against (GB300 runs
 * FP64 FMAs at 1/64 of the FP32 rate, so FP64 SpMV can be bound by it
 * rather than by memory).  Synchronises `stream`; allocates and frees a
 * small result buffer.  SPC5_EUNSUPPORTED for other dtypes, SPC5_EINVAL if
 * tflops is NULL.
 */
spc5_status spc5_measure_fma_peak(spc5_dtype dtype, void *stream, double *tflops);

/* Release the handle and every device array it owns (synchronising). */
spc5_status spc5_destroy(spc5_matrix *A);

/* Static name of a status code. */
const char *spc5_status_str(spc5_status s);

/* One-line description of the last failure on the calling thread ("" if none). */
const char *spc5_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SPC5_H */
