/*
 * CPU oracle for the SPC5 beta(r,c) sparse matrix-vector product.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this file's library.  The CUDA
 * product path never calls it, links it, or shares code with it.
 *
 * Plain, slow, obviously correct FP64 code written from the paper
 * (Regnault & Bramas, "SPC5: an efficient SpMV framework vectorized using
 * ARM SVE and x86 AVX-512"):
 *
 *   oracle_csr_spmv     y = A x from CSR (Section 2.3), the parity reference
 *   oracle_spc5_convert CSR -> beta(r,c) blocks (Section 2.4)
 *   oracle_spc5_spmv    Algorithm 1, scalar path, over beta(r,c)
 *   oracle_spc5_to_csr  beta(r,c) -> CSR (inverse of the conversion)
 *   oracle_pack_masks   the r per-row c-bit masks of a block as one word
 *   oracle_quantize     FP64 values -> FP32 or BF16 storage, round to
 *                       nearest even (the reduced-precision value forms)
 *   oracle_csr_transpose  A^T in CSR (for dx = A^T g, the input gradient)
 *   oracle_values_grad  dvals[e] = g[row(e)] * x[col(e)] (value gradient)
 *   oracle_hybrid_split beta(r,c) -> blocks of two or more values plus the
 *                       single-value blocks as scalar (CSR) entries
 *
 * Readings of the paper taken here (each one is also listed in the design
 * notes):
 *   - Block formation for r > 1 (Section 2.4 describes one row; a block
 *     "is mapped to several rows"): within a panel of r consecutive rows,
 *     take the sorted union U of the rows' column indices; a block starts
 *     at the smallest column s of U not yet covered and covers columns
 *     [s, s+c) in all r rows.  For r = 1 this is the paper's rule verbatim.
 *   - Bit k of a row mask (least significant bit = 0) means that column
 *     idxCol + k is stored (Algorithm 1 tests (1 << k) AND mask and reads
 *     x[idxCol + k]; Fig. 3's caption: mask 1101 selects three elements).
 *   - Values are packed block by block, within a block row by row, within a
 *     row in ascending bit order: the order in which Algorithm 1 advances
 *     idxVal.  For r = 1 this is exactly CSR order (Section 5).
 *   - Loop bounds "0 to r", "0 to c" of Algorithm 1 are half-open.
 *   - The last panel of an n not divisible by r has fewer rows; the missing
 *     rows hold no entries.
 *   - Explicitly stored zeros are entries like any other.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum {
  ORACLE_OK = 0,
  ORACLE_EINVAL = 1,   /* bad sizes, r or c out of range */
  ORACLE_EUNSORTED = 2, /* a row's columns are not strictly ascending */
  ORACLE_ERANGE = 3,   /* a column index outside [0, ncols) */
  ORACLE_EROWPTR = 4,  /* row pointers not monotone or not starting at 0 */
};

/* Check that (rowptr, colidx) is a CSR pattern with strictly ascending
 * columns in [0, ncols) in every row. */
int oracle_check_csr(int64_t nrows, int64_t ncols, const int32_t *rowptr, const int32_t *colidx) {
  if (nrows < 0 || ncols < 0) return ORACLE_EINVAL;
  if (rowptr[0] != 0) return ORACLE_EROWPTR;
  for (int64_t i = 0; i < nrows; ++i) {
    if (rowptr[i + 1] < rowptr[i]) return ORACLE_EROWPTR;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      if (colidx[e] < 0 || colidx[e] >= ncols) return ORACLE_ERANGE;
      if (e > rowptr[i] && colidx[e] <= colidx[e - 1]) return ORACLE_EUNSORTED;
    }
  }
  return ORACLE_OK;
}

/*
 * CSR SpMV, Section 2.3: y_i = sum over the stored entries (i, j) of
 * a_ij * x_j, visiting a row's entries in ascending column order.
 *
 * The sum is compensated (Neumaier's variant of Kahan summation) so that
 * the reference itself stays accurate to about one rounding of y_i even on
 * rows with millions of entries; the products a_ij * x_j are rounded once.
 * scale_i = sum |a_ij * x_j| is the per-row magnitude that the tolerances
 * of the parity tests are stated against.  `scale` may be NULL.
 */
int oracle_csr_spmv(int64_t nrows, const int32_t *rowptr, const int32_t *colidx,
                    const double *vals, const double *x, double *y, double *scale) {
#pragma omp parallel for schedule(static, 1024)
  for (int64_t i = 0; i < nrows; ++i) {
    double s = 0.0, comp = 0.0, mag = 0.0;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      double term = vals[e] * x[colidx[e]];
      double t = s + term;
      if (fabs(s) >= fabs(term))
        comp += (s - t) + term;
      else
        comp += (term - t) + s;
      s = t;
      mag += fabs(term);
    }
    y[i] = s + comp;
    if (scale) scale[i] = mag;
  }
  return ORACLE_OK;
}

/* Plain sequential CSR SpMV, no compensation: the textbook loop.  Used to
 * time the CPU baseline and as an extra consistency check. */
int oracle_csr_spmv_plain(int64_t nrows, const int32_t *rowptr, const int32_t *colidx,
                          const double *vals, const double *x, double *y) {
#pragma omp parallel for schedule(static, 1024)
  for (int64_t i = 0; i < nrows; ++i) {
    double s = 0.0;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) s += vals[e] * x[colidx[e]];
    y[i] = s;
  }
  return ORACLE_OK;
}

/*
 * Host threads of the two CSR products above.  Rows are independent and each
 * row is summed by one thread in the order stated above, so the results do
 * not depend on the thread count.  The library built without OpenMP (the
 * one the tests use) ignores the request and returns 1; the build with
 * OpenMP (used only to time the CPU baseline) returns the count set.
 */
int oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/*
 * CSR -> beta(r,c), Section 2.4.
 *
 * For every panel of r rows (the last panel may be shorter), walk the rows'
 * sorted column lists together.  The smallest column s not yet consumed in
 * any row opens a block; the block takes, row by row, every entry whose
 * column lies in [s, s + c), setting bit (column - s) of that row's mask and
 * appending the value.  Blocks therefore come out in ascending s and never
 * overlap.
 *
 * Two uses:
 *   - count: block_colidx == NULL.  Writes block_rowptr[0..npanels] (first
 *     block of each panel, as in Algorithm 1's block_rowptr) and returns the
 *     number of blocks through *nblocks.
 *   - fill: block_rowptr already holds the counts' prefix sums; writes
 *     block_colidx[nblocks], block_masks[nblocks * r] (mask of row q of
 *     block b at index b * r + q, bit k <-> column block_colidx[b] + k) and
 *     values[nnz].
 */
int oracle_spc5_convert(int64_t nrows, int64_t ncols, const int32_t *rowptr,
                        const int32_t *colidx, const double *vals, int r, int c,
                        int64_t *block_rowptr, int64_t *nblocks, int32_t *block_colidx,
                        uint64_t *block_masks, double *values) {
  if (r < 1 || r > 64 || c < 1 || c > 64 || nrows < 0) return ORACLE_EINVAL;
  int rc = oracle_check_csr(nrows, ncols, rowptr, colidx);
  if (rc) return rc;
  int fill = block_colidx != NULL;
  int64_t npanels = (nrows + r - 1) / r;
  int64_t *ptr = (int64_t *)malloc(sizeof(int64_t) * (size_t)r);
  int64_t *end = (int64_t *)malloc(sizeof(int64_t) * (size_t)r);
  if (!ptr || !end) {
    free(ptr);
    free(end);
    return ORACLE_EINVAL;
  }
  int64_t b = 0, v = 0;
  if (!fill) block_rowptr[0] = 0;
  for (int64_t p = 0; p < npanels; ++p) {
    if (fill) b = block_rowptr[p];
    for (int q = 0; q < r; ++q) {
      int64_t row = p * r + q;
      ptr[q] = row < nrows ? rowptr[row] : 0;
      end[q] = row < nrows ? rowptr[row + 1] : 0;
    }
    for (;;) {
      /* the smallest column not yet consumed in any row of the panel */
      int64_t s = -1;
      for (int q = 0; q < r; ++q)
        if (ptr[q] < end[q] && (s < 0 || colidx[ptr[q]] < s)) s = colidx[ptr[q]];
      if (s < 0) break;
      if (fill) block_colidx[b] = (int32_t)s;
      for (int q = 0; q < r; ++q) {
        uint64_t mask = 0;
        while (ptr[q] < end[q] && colidx[ptr[q]] < s + c) {
          mask |= 1ULL << (colidx[ptr[q]] - s);
          if (fill) values[v] = vals[ptr[q]];
          ++v;
          ++ptr[q];
        }
        if (fill) block_masks[b * r + q] = mask;
      }
      ++b;
    }
    if (!fill) block_rowptr[p + 1] = b;
  }
  if (nblocks) *nblocks = b;
  free(ptr);
  free(end);
  return ORACLE_OK;
}

/*
 * Algorithm 1, scalar path: for each panel, zero r partial sums; for each
 * of the panel's blocks read idxCol; for each row of the block read its
 * mask and, for every set bit k, add x[idxCol + k] * values[idxVal] to the
 * row's sum and advance idxVal; finally store the r sums into y.  Here y is
 * overwritten (y = A x) instead of accumulated into; rows past nrows in a
 * short last panel are not written.
 */
int oracle_spc5_spmv(int64_t nrows, int r, int c, const int64_t *block_rowptr,
                     const int32_t *block_colidx, const uint64_t *block_masks,
                     const double *values, const double *x, double *y) {
  if (r < 1 || r > 64 || c < 1 || c > 64) return ORACLE_EINVAL;
  double *sum = (double *)malloc(sizeof(double) * (size_t)r);
  if (!sum) return ORACLE_EINVAL;
  int64_t idxVal = 0;
  for (int64_t idxRow = 0; idxRow < nrows; idxRow += r) {
    for (int q = 0; q < r; ++q) sum[q] = 0.0;
    for (int64_t idxBlock = block_rowptr[idxRow / r]; idxBlock < block_rowptr[idxRow / r + 1];
         ++idxBlock) {
      int64_t idxCol = block_colidx[idxBlock];
      for (int idxRowBlock = 0; idxRowBlock < r; ++idxRowBlock) {
        uint64_t valMask = block_masks[idxBlock * r + idxRowBlock];
        for (int k = 0; k < c; ++k) {
          if ((1ULL << k) & valMask) {
            sum[idxRowBlock] += x[idxCol + k] * values[idxVal];
            idxVal += 1;
          }
        }
      }
    }
    for (int q = 0; q < r && idxRow + q < nrows; ++q) y[idxRow + q] = sum[q];
  }
  free(sum);
  return ORACLE_OK;
}

/*
 * beta(r,c) -> CSR.  Walk the blocks in storage order exactly as
 * Algorithm 1 does (running idxVal) and hand every value to its row, at
 * column idxCol + k.  Within a panel the blocks are ascending and disjoint,
 * so each row's entries arrive in ascending column order.
 * rowptr_out[nrows + 1]; colidx_out and vals_out hold nnz entries.
 */
int oracle_spc5_to_csr(int64_t nrows, int r, int c, const int64_t *block_rowptr,
                       const int32_t *block_colidx, const uint64_t *block_masks,
                       const double *values, int32_t *rowptr_out, int32_t *colidx_out,
                       double *vals_out) {
  if (r < 1 || r > 64 || c < 1 || c > 64) return ORACLE_EINVAL;
  int64_t npanels = (nrows + r - 1) / r;
  /* row lengths = number of set bits of the row's masks */
  for (int64_t i = 0; i <= nrows; ++i) rowptr_out[i] = 0;
  for (int64_t p = 0; p < npanels; ++p)
    for (int64_t b = block_rowptr[p]; b < block_rowptr[p + 1]; ++b)
      for (int q = 0; q < r; ++q) {
        uint64_t m = block_masks[b * r + q];
        int64_t row = p * r + q;
        for (int k = 0; k < c; ++k)
          if ((1ULL << k) & m) {
            if (row >= nrows) return ORACLE_EINVAL; /* bits in a missing row */
            rowptr_out[row + 1]++;
          }
      }
  for (int64_t i = 0; i < nrows; ++i) rowptr_out[i + 1] += rowptr_out[i];
  int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nrows > 0 ? nrows : 1));
  if (!next) return ORACLE_EINVAL;
  for (int64_t i = 0; i < nrows; ++i) next[i] = rowptr_out[i];
  int64_t idxVal = 0;
  for (int64_t p = 0; p < npanels; ++p)
    for (int64_t b = block_rowptr[p]; b < block_rowptr[p + 1]; ++b)
      for (int q = 0; q < r; ++q) {
        uint64_t m = block_masks[b * r + q];
        int64_t row = p * r + q;
        for (int k = 0; k < c; ++k)
          if ((1ULL << k) & m) {
            colidx_out[next[row]] = (int32_t)(block_colidx[b] + k);
            vals_out[next[row]] = values[idxVal];
            ++next[row];
            ++idxVal;
          }
      }
  free(next);
  return ORACLE_OK;
}

/*
 * Physical mask layout: the r masks of block b, each c bits, are stored as
 * one little-endian word of r*c bits (ceil(r*c/8) bytes), row q occupying
 * bits [q*c, (q+1)*c).  For c = 8 this is byte-for-byte the paper's
 * block_masks array indexed by idxBlock * r + idxRowBlock.
 */
int oracle_pack_masks(int64_t nblocks, int r, int c, const uint64_t *block_masks,
                      uint8_t *packed) {
  if (r < 1 || c < 1 || r * c > 64) return ORACLE_EINVAL;
  int nbytes = (r * c + 7) / 8;
  for (int64_t b = 0; b < nblocks; ++b) {
    uint64_t word = 0;
    for (int q = 0; q < r; ++q) word |= (block_masks[b * r + q] & ((c == 64) ? ~0ULL : ((1ULL << c) - 1))) << (q * c);
    for (int t = 0; t < nbytes; ++t) packed[b * nbytes + t] = (uint8_t)(word >> (8 * t));
  }
  return ORACLE_OK;
}

/*
 * Reduced-precision storage of the values: FP64 -> FP32 or BF16, round to
 * nearest, ties to even.
 *
 * FP32: the C conversion (float)d rounds to nearest even in the default
 * rounding mode.
 *
 * BF16 (1 sign, 8 exponent, 7 fraction bits; the upper half of an FP32):
 * rounding twice (FP64 -> FP32 -> BF16, both to nearest) can differ from
 * one correct rounding when the first rounding lands exactly on a BF16
 * midpoint.  Rounding the first step to odd instead (Boldo and Melquiond,
 * "Emulation of FMA and correctly rounded sums: proved algorithms using
 * rounding to odd", IEEE TC 2008) makes the second rounding correct, since
 * FP32 keeps at least two more significand bits than BF16:
 *   1. f = d truncated toward zero to FP32; if f != d, force f's last bit to 1;
 *   2. round f to the nearest BF16, ties to even, on its bit pattern.
 * Finite inputs whose magnitude stays inside the FP32 normal range.
 */
static float round_to_odd_f32(double d) {
  float f = (float)d;
  /* move toward zero if the nearest rounding went away from zero */
  if (fabs((double)f) > fabs(d)) f = nextafterf(f, 0.0f);
  if ((double)f != d) {
    uint32_t b;
    memcpy(&b, &f, 4);
    b |= 1u;
    memcpy(&f, &b, 4);
  }
  return f;
}

static uint16_t bf16_from_f32_rne(float f) {
  uint32_t b;
  memcpy(&b, &f, 4);
  uint32_t lsb = (b >> 16) & 1u;
  b += 0x7FFFu + lsb;
  return (uint16_t)(b >> 16);
}

/* dtype 1: out is float[n]; dtype 2: out is uint16_t[n] (BF16 bit patterns). */
int oracle_quantize(int64_t n, const double *in, int dtype, void *out) {
  if (dtype == 1) {
    float *o = (float *)out;
    for (int64_t i = 0; i < n; ++i) o[i] = (float)in[i];
    return ORACLE_OK;
  }
  if (dtype == 2) {
    uint16_t *o = (uint16_t *)out;
    for (int64_t i = 0; i < n; ++i) o[i] = bf16_from_f32_rne(round_to_odd_f32(in[i]));
    return ORACLE_OK;
  }
  return ORACLE_EINVAL;
}

/*
 * Transpose of a CSR matrix (nrows x ncols -> ncols x nrows): entries are
 * counted per column, the counts prefix-summed, and the entries dealt out
 * row by row, so every row of the transpose lists its columns (the
 * original rows) in ascending order.  dx = A^T g is then oracle_csr_spmv on
 * the transpose.  rowptr_t[ncols+1], colidx_t[nnz], vals_t[nnz].
 */
int oracle_csr_transpose(int64_t nrows, int64_t ncols, const int32_t *rowptr,
                         const int32_t *colidx, const double *vals, int32_t *rowptr_t,
                         int32_t *colidx_t, double *vals_t) {
  for (int64_t j = 0; j <= ncols; ++j) rowptr_t[j] = 0;
  for (int64_t e = 0; e < rowptr[nrows]; ++e) rowptr_t[colidx[e] + 1]++;
  for (int64_t j = 0; j < ncols; ++j) rowptr_t[j + 1] += rowptr_t[j];
  int32_t *next = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ncols > 0 ? ncols : 1));
  if (!next) return ORACLE_EINVAL;
  for (int64_t j = 0; j < ncols; ++j) next[j] = rowptr_t[j];
  for (int64_t i = 0; i < nrows; ++i)
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      int32_t t = next[colidx[e]]++;
      colidx_t[t] = (int32_t)i;
      vals_t[t] = vals[e];
    }
  free(next);
  return ORACLE_OK;
}

/* Gradient of <g, A x> with respect to the stored values: one product per
 * entry, in CSR order. */
int oracle_values_grad(int64_t nrows, const int32_t *rowptr, const int32_t *colidx,
                       const double *g, const double *x, double *dvals) {
  for (int64_t i = 0; i < nrows; ++i)
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) dvals[e] = g[i] * x[colidx[e]];
  return ORACLE_OK;
}

/*
 * Hybrid form (the paper's closing remarks: a block holding a single value
 * costs SPC5 a block's metadata and a mask test for one product, and the
 * paper measures SPC5 slower than CSR below about two values per block; it
 * proposes mixing the block format with a scalar one).  Reading taken here:
 * a block whose r masks hold exactly one set bit becomes a scalar entry
 * (its row, column idxCol + k, its value); every other block stays a block.
 *
 * Outputs:
 *   block part  brp_b[npanels+1], bcol_b[*nb_b], masks_b[*nb_b * r],
 *               vals_b[nnz - *ns]: the kept blocks in storage order, their
 *               values in Algorithm 1's order (a beta(r,c) matrix of its own);
 *   scalars     s_rowptr[nrows+1], s_colidx[*ns], s_vals[*ns]: CSR by row,
 *               each row's scalars in ascending column order (blocks of a
 *               panel are ascending and disjoint).
 * Arrays must be sized for the worst case (nblocks blocks, nnz values).
 */
int oracle_hybrid_split(int64_t nrows, int r, int c, const int64_t *block_rowptr,
                        const int32_t *block_colidx, const uint64_t *block_masks,
                        const double *values, int64_t *brp_b, int32_t *bcol_b,
                        uint64_t *masks_b, double *vals_b, int64_t *nb_b, int32_t *s_rowptr,
                        int32_t *s_colidx, double *s_vals, int64_t *ns) {
  if (r < 1 || r > 64 || c < 1 || c > 64) return ORACLE_EINVAL;
  int64_t npanels = (nrows + r - 1) / r;
  /* pass 1: scalars per row */
  for (int64_t i = 0; i <= nrows; ++i) s_rowptr[i] = 0;
  for (int64_t p = 0; p < npanels; ++p)
    for (int64_t b = block_rowptr[p]; b < block_rowptr[p + 1]; ++b) {
      int bits = 0, qs = 0;
      for (int q = 0; q < r; ++q) {
        uint64_t m = block_masks[b * r + q];
        for (int k = 0; k < c; ++k)
          if ((1ULL << k) & m) {
            ++bits;
            qs = q;
          }
      }
      if (bits == 1) {
        if (p * r + qs >= nrows) return ORACLE_EINVAL;
        s_rowptr[p * r + qs + 1]++;
      }
    }
  for (int64_t i = 0; i < nrows; ++i) s_rowptr[i + 1] += s_rowptr[i];
  int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nrows > 0 ? nrows : 1));
  if (!next) return ORACLE_EINVAL;
  for (int64_t i = 0; i < nrows; ++i) next[i] = s_rowptr[i];
  /* pass 2: walk the blocks with Algorithm 1's running idxVal */
  int64_t idxVal = 0, kept = 0, keptVal = 0;
  for (int64_t p = 0; p < npanels; ++p) {
    brp_b[p] = kept;
    for (int64_t b = block_rowptr[p]; b < block_rowptr[p + 1]; ++b) {
      int bits = 0;
      for (int q = 0; q < r; ++q) {
        uint64_t m = block_masks[b * r + q];
        for (int k = 0; k < c; ++k)
          if ((1ULL << k) & m) ++bits;
      }
      if (bits == 1) {
        for (int q = 0; q < r; ++q) {
          uint64_t m = block_masks[b * r + q];
          for (int k = 0; k < c; ++k)
            if ((1ULL << k) & m) {
              int64_t row = p * r + q;
              s_colidx[next[row]] = (int32_t)(block_colidx[b] + k);
              s_vals[next[row]] = values[idxVal];
              ++next[row];
            }
        }
        idxVal += 1;
      } else {
        bcol_b[kept] = block_colidx[b];
        for (int q = 0; q < r; ++q) masks_b[kept * r + q] = block_masks[b * r + q];
        for (int i = 0; i < bits; ++i) vals_b[keptVal++] = values[idxVal++];
        ++kept;
      }
    }
  }
  brp_b[npanels] = kept;
  *nb_b = kept;
  *ns = nrows > 0 ? s_rowptr[nrows] : 0;
  free(next);
  return ORACLE_OK;
}
