// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "spc5.h"

namespace spc5 {

// One unit of SpMV work, produced by the planner at conversion time.
//   group tile:   whole panels [p0, p1), lanes-per-row 2^(mode & 15); the
//                 kernel stages the tile's block_rowptr and panel_vptr slices;
//                 with mode & kSkip, bit j of `slot` marks panel p0 + j as
//                 handled by tiles of its own (a heavy panel), so the group
//                 tile leaves its rows alone
//   segment tile: blocks [b0, b1) of the single panel p0 (mode & kSegment),
//                 32/r lanes per row; with mode & kPartial the r row sums go
//                 to partial[slot * r + q] and a fixup adds the pieces.
//   flat tile:    (mode & kFlat) whole panels [p0, p1) whose blocks
//                 [b0, b1) are dealt to the lanes in rounds (four blocks
//                 per lane, or each round's values split evenly); with
//                 mode & kPartial the blocks [b0, b1) of the single long
//                 panel p0, whose r row sums go to partial[slot * r + q].
//   expanded tile: (mode & kExpand) whole panels [p0, p1) whose values are
//                 laid out row by row in shared memory and split evenly
//                 over the lanes; with mode & kPartial the blocks [b0, b1)
//                 of the single long panel p0, whose r row sums go to
//                 partial[slot * r + q].
// [b0, b1) and [v0, v1) are the tile's block and value ranges.
struct Tile {
  int32_t p0, p1, b0, b1, v0, v1, slot, mode;
};
constexpr int32_t kSegment = 16;
constexpr int32_t kPartial = 32;
constexpr int32_t kFlat = 64;
constexpr int32_t kExpand = 128;
constexpr int32_t kSkip = 256;

// Expanded tiles: at most kExpandCap values and kExpandRows rows (shared
// memory of the expanded SpMV kernel); panels are packed by windows of
// kExpandWindow values.
constexpr int32_t kExpandCap = 1024;
constexpr int32_t kExpandWindow = 512;
constexpr int32_t kExpandRows = 128;

// Packed mask word of one block: r * c bits, row q at bits [q * c, (q + 1) * c)
// (uint8 for r * c = 8, uint16 for 16, uint32 for 32).
template <int R, int C>
struct MaskType {
  using T = uint32_t;
};
template <>
struct MaskType<1, 8> {
  using T = uint8_t;
};
template <>
struct MaskType<2, 4> {
  using T = uint8_t;
};
template <>
struct MaskType<2, 8> {
  using T = uint16_t;
};
template <>
struct MaskType<4, 4> {
  using T = uint16_t;
};

// log2 of a block height r in {1, 2, 4, 8}.
template <int R>
struct Log2 {
  static constexpr int v = R == 1 ? 0 : R == 2 ? 1 : R == 4 ? 2 : 3;
};

#ifdef __CUDACC__
// Stored value -> accumulation type.  FP64 and FP32 are used as they are;
// a BF16 bit pattern is the upper half of an FP32, so widening is exact.
__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ float widen(float v) { return v; }
__device__ __forceinline__ float widen(uint16_t v) { return __uint_as_float((uint32_t)v << 16); }
#endif

}  // namespace spc5

// A converted matrix.  Every array is device memory owned by the handle.
struct spc5_matrix {
  int64_t nrows = 0, ncols = 0, nnz = 0;
  int r = 0, c = 0;
  int64_t npanels = 0, nblocks = 0;
  int device = 0;
  spc5_dtype value_dtype = SPC5_F64;
  int32_t *block_rowptr = nullptr;  // npanels + 1 (+16 bytes of padding)
  int32_t *panel_vptr = nullptr;    // npanels + 1 (+16 bytes of padding)
  int32_t *block_colidx = nullptr;  // nblocks (+16 bytes of padding)
  void *masks = nullptr;            // nblocks * r * c / 8 bytes (+16 bytes of padding)
  void *values = nullptr;           // nnz values (+16 bytes of padding)
  int32_t *value_src = nullptr;     // CSR index of every stored value (nnz)
  int32_t *csr_rowptr = nullptr;    // the conversion's CSR row pointer (nrows + 1): the
                                    // values gradient writes a row's entries from it
  int64_t device_bytes = 0;

  // SpMV plan (built by the converter)
  spc5::Tile *tiles = nullptr;
  int64_t ntiles = 0;
  int32_t *long_panels = nullptr;   // panels split into pieces
  int32_t *long_slots = nullptr;    // [2 * nlong]: first and end piece slot of each
  int64_t nlong = 0, npieces = 0;
  double *partial = nullptr;        // npieces * r partial row sums (FP64 or FP32 slots)
  int log2_group_lanes = 0;         // lanes per row in group tiles
  int vcap = 0, bcap = 0;           // stage capacity (values, blocks)
  int group_panels = 0;             // panels per group tile
  int stages = 0, consumers = 0, stage_bytes = 0;
  int body = 0;                     // consumer body: bit 0 = predicated loop over the c
                                    // bits (else set-bit loop), bit 1 = x staged in smem
  int kernel = 0;                   // 0: direct tile kernel, 1: staged tile kernel
  int dynamic = 0;                  // row-group kernel: tiles from a counter (else grid-stride)
  int halves = 0;                   // row-group plan: the last round's groups cut in halves
  double tuned_us = 0.0;            // SpMV time of the plan chosen by spc5_tune (0 = untuned)
  double tuned_rows_us = 0.0;       // SpMV time of the best row-group plan it found
  uint32_t *dev_error = nullptr;    // set by kernels on a timed-out wait

  // Block-balanced (flat = 1) or expanded (flat = 2) plan, used by the SpMV
  // instead of the row groups above when `flat` is set; the transposed
  // product, the gradient and the batched kernel always use the row-group
  // plan.
  int flat = 0;
  double group_efficiency = 0.0;    // busy share of the row-group plan's block slots
  spc5::Tile *ftiles = nullptr;
  int64_t fntiles = 0;
  int32_t *flong_panels = nullptr;
  int32_t *flong_slots = nullptr;
  int64_t fnlong = 0, fnpieces = 0;
  double *fpartial = nullptr;       // fnpieces * r partial row sums
  uint16_t *frowoff = nullptr;      // expanded plan: (npanels + fnpieces) * r row starts

  // Hybrid form (hybrid != 0): the single-value blocks were moved to a CSR of
  // scalars; the arrays above then hold the blocks of two or more values
  // (nblocks of them, nnz values) and the scalars come on top.
  int hybrid = 0;
  int64_t nscalars = 0;
  int32_t *s_rowptr = nullptr;      // nrows + 1
  int32_t *s_colidx = nullptr;      // nscalars (+16 bytes of padding)
  void *s_vals = nullptr;           // nscalars values in the storage type (+16 bytes)
  spc5::Tile *stiles = nullptr;     // expanded tiles over the scalars' rows
  int64_t sntiles = 0;
  int32_t *slong_rows = nullptr, *slong_slots = nullptr;
  int64_t snlong = 0, snpieces = 0;
  double *spartial = nullptr;       // snpieces partial sums
  uint32_t *fsched = nullptr;       // [2]: next tile, finished warps (reset by the kernel)

  // staging for host vectors in spc5_spmv
  void *x_stage = nullptr;
  void *y_stage = nullptr;

  // A^T in beta(r,c), built by spc5_build_transpose (owned; its value_src
  // holds CSR indices of this matrix's conversion, so that
  // spc5_set_values refreshes both)
  spc5_matrix *transpose = nullptr;
};

namespace spc5 {

// Thread-local last error text.
void set_error(const std::string &msg);

// Status of the last CUDA call; records a message on failure.
spc5_status cuda_check(cudaError_t e, const char *what);

// Supported block shapes.
bool supported_rc(int r, int c);

// Multiprocessor count of the current device (looked up once per device).
int device_sm_count();

// Stream-ordered scratch of the builders (conversion, tile planning,
// transposition, hybrid split, CSR staging), freed with cudaFreeAsync: it
// comes from a private memory pool of the current device that keeps up to
// kScratchKeep bytes mapped between calls, so that a conversion does not map
// and unmap gigabytes of scratch every time (mapping is most of the host
// time of a large conversion).  Memory above that is returned to the device
// at the next synchronisation, as with the default pool.
constexpr uint64_t kScratchKeep = 8ull << 30;
cudaError_t scratch_alloc(void **p, size_t bytes, cudaStream_t s);

// Largest device ordinal the library's per-device tables hold, plus one.
constexpr int kMaxDevices = 64;

// Conversion: fills A (sizes set by the caller) from a device CSR.
spc5_status convert_device(spc5_matrix *A, const int32_t *d_rowptr, const int32_t *d_colidx,
                           const double *d_vals, cudaStream_t stream);

// Planner options; -1 = default (environment variable, else heuristic).
struct PlanOptions {
  int kernel = -1;  // 0 direct, 1 staged
  int log2g = -1;   // lanes per row in group tiles = 2^log2g
  int vcap = -1;    // tile capacity in values
  int bcap = -1;    // tile capacity in blocks
  int body = -1;    // consumer body
  int flat = -1;    // 0: row groups, 1: block-balanced plan, 2: expanded plan
  int dynamic = -1; // row groups: 1 = tiles taken from a counter, 0 = dealt grid-stride
  int halves = -1;  // row groups: 1 = the groups of the last round of tiles as two half tiles
};

// Work plan of the SpMV kernels; called by the converter while the
// per-block popcounts (mask32) and value offsets (boff) are still alive.
spc5_status plan_tiles(spc5_matrix *A, const uint32_t *mask32, const int32_t *boff,
                       cudaStream_t stream, const PlanOptions &opt = PlanOptions());

// Rebuild the plan of a converted matrix with other options (recomputes the
// per-block popcounts and value offsets from the stored masks).
spc5_status replan(spc5_matrix *A, cudaStream_t stream, const PlanOptions &opt);

// SpMV launch on device vectors.
// x, y: FP64 for an FP64 matrix, FP32 for FP32 and BF16 matrices.
spc5_status spmv_device(const spc5_matrix *A, const void *x, void *y, double alpha, double beta,
                        cudaStream_t stream);

// The same with the partial sums of split panels written to `partial`
// (spmv_pieces(A) * r doubles) instead of the handle's own buffer, and the
// expanded plan's two tile-scheduling counters at `sched` (zero before the
// first call; every launch leaves them zero again) instead of the handle's.
spc5_status spmv_device_scratch(const spc5_matrix *A, const void *x, void *y, double alpha,
                                double beta, cudaStream_t stream, void *partial,
                                uint32_t *sched);

// Pieces of split panels in the plan the SpMV uses.
int64_t spmv_pieces(const spc5_matrix *A);

// Expanded tiles over panels of `r` rows whose blocks hold the values
// [vptr[p], vptr[p+1]) (boff[b] = value offset of block b): tiles of whole
// panels (at most kExpandCap values and kExpandRows rows) and pieces of
// longer panels.  Allocates tiles, long_panels and long_slots.
struct ExpandedPlan {
  Tile *tiles = nullptr;
  int32_t *long_panels = nullptr, *long_slots = nullptr;
  int64_t ntiles = 0, nlong = 0, npieces = 0;
};
spc5_status build_expanded(int64_t npanels, int64_t nblocks, int64_t nvalues, int r,
                           const int32_t *brp, const int32_t *vptr, const int32_t *boff,
                           cudaStream_t stream, ExpandedPlan *out);

// Row starts of the expanded plan's tiles (A->frowoff, allocated), computed
// on the GPU once the tiles are written.
spc5_status expand_row_starts(spc5_matrix *A, cudaStream_t stream);

// Number of kernel launches one spmv_device call makes.
int spmv_launches(const spc5_matrix *A);

// Hybrid form: move the single-value blocks of a converted matrix to a CSR
// of scalars, rebuild the block part's plan and build the scalars' plan.
spc5_status hybrid_split(spc5_matrix *A, cudaStream_t stream);

// y += alpha * S x for the scalars of a hybrid matrix (after the block part
// wrote y), partial sums of split rows at `partial` (snpieces values), tile
// counters at `sched`.
spc5_status spmv_scalars(const spc5_matrix *A, const void *x, void *y, double alpha,
                         cudaStream_t stream, void *partial, uint32_t *sched);

}  // namespace spc5
