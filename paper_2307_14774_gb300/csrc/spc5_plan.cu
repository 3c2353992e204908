// Work plan of the staged SpMV kernel, built on the GPU at conversion time.
//
// The SpMV streams the matrix through shared memory one tile at a time, so a
// tile's values, block columns and masks must fit one pipeline stage
// (vcap values, bcap blocks).  Tiles:
//   - group tiles: panels in fixed groups of group_panels = 32 / (r * G)
//     consecutive panels, G lanes per row (G = 2^log2_group_lanes);
//   - a group that does not fit a stage is "fat": each of its panels becomes
//     its own segment tile (32 / r lanes per row) when it fits, otherwise a
//     long panel, cut at block boundaries into pieces that fit; a piece's
//     row sums go to a partial buffer and a fixup kernel adds the pieces of
//     each long panel in order (deterministic, no atomics);
//   - direct kernel: only the group's heavy panels (more than eight times
//     the mean panel's values or blocks, and every panel that fits no tile)
//     leave it, as segment tiles or long panels; the group tile keeps the
//     other panels and skips the heavy ones (mode & kSkip, a mask in
//     `slot`), so one long row of a skewed matrix neither holds up the 31
//     rows around it nor turns them into 31 tiles of one panel each.
// Piece boundaries are where the block's value offset or block index enters
// a new window of (vcap - 32) values or bcap blocks; a block holds at most
// 32 values, so every piece fits a stage.
// All steps are flat passes plus prefix sums; nothing walks a panel serially.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include <algorithm>
#include <climits>

#include "spc5_internal.h"
#include "spc5_scan.cuh"

namespace spc5 {
namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(int64_t n) {
  int64_t blocks = (n + kThreads - 1) / kThreads;
  if (blocks < 1) blocks = 1;
  if (blocks > 1048576) blocks = 1048576;
  return (unsigned)blocks;
}

#define GRID_STRIDE(i, n) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); \
       i += (int64_t)gridDim.x * blockDim.x)

struct PlanParams {
  int64_t npanels, nblocks;
  int32_t gp;       // panels per group
  int32_t vcap, bcap, vwin;
  int32_t log2g_group, log2g_segment;
  const int32_t *brp, *vptr;
  int32_t skip;     // direct kernel: heavy panels leave their group tile
  int32_t hv, hb;   // a panel is heavy above hv values or hb blocks
  int64_t half_from;  // groups from this one on (without heavy panels) are
                      // two tiles of gp / 2 panels, twice the lanes per row
};

__device__ __forceinline__ bool group_fat(const PlanParams &P, int64_t g) {
  int64_t a = g * P.gp, b = (a + P.gp < P.npanels) ? a + P.gp : P.npanels;
  return (P.vptr[b] - P.vptr[a]) > P.vcap || (P.brp[b] - P.brp[a]) > P.bcap;
}

__device__ __forceinline__ bool panel_heavy(const PlanParams &P, int64_t p) {
  return (P.vptr[p + 1] - P.vptr[p]) > P.hv || (P.brp[p + 1] - P.brp[p]) > P.hb;
}

// Panels with tiles of their own: with skip, the heavy panels; otherwise
// every panel of a fat group.
__device__ __forceinline__ bool panel_own(const PlanParams &P, int64_t p) {
  return P.skip ? panel_heavy(P, p) : group_fat(P, p / P.gp);
}

// A panel cut into pieces (it fits no stage or tile).  hv <= vcap and
// hb <= bcap, so a long panel is always heavy (skip) and its group fat.
__device__ __forceinline__ bool panel_long(const PlanParams &P, int64_t p) {
  return panel_own(P, p) &&
         ((P.vptr[p + 1] - P.vptr[p]) > P.vcap || (P.brp[p + 1] - P.brp[p]) > P.bcap);
}

// Heavy panels of group g (bit j = panel g * gp + j).
__device__ __forceinline__ uint32_t group_heavy(const PlanParams &P, int64_t g) {
  const int64_t a = g * P.gp, b = (a + P.gp < P.npanels) ? a + P.gp : P.npanels;
  uint32_t h = 0;
  for (int64_t p = a; p < b; ++p)
    if (panel_heavy(P, p)) h |= 1u << (p - a);
  return h;
}

// Whether the group of panel p (p % gp == 0) has a group tile: always
// without skip (unless its panels have their own tiles, see panel_own);
// with skip, unless every panel of the group is heavy.
__device__ __forceinline__ bool has_group_tile(const PlanParams &P, int64_t p) {
  const int64_t n = (p + P.gp < P.npanels) ? P.gp : P.npanels - p;
  const uint32_t all = n >= 32 ? 0xffffffffu : ((1u << n) - 1u);
  return group_heavy(P, p / P.gp) != all;
}

// Group of panel p cut into two tiles of half the panels (the last round of
// the tile dealing, see plan_tiles).
__device__ __forceinline__ bool group_halved(const PlanParams &P, int64_t p) {
  const int64_t g = p / P.gp;
  return P.skip && P.gp >= 2 && g >= P.half_from && group_heavy(P, g) == 0u;
}

// Index of a panel's first own tile: with skip, the first panel of a group
// comes after the group tile.
__device__ __forceinline__ int32_t own_base(const PlanParams &P, const int32_t *tbase,
                                            int64_t p) {
  return tbase[p] + ((P.skip && p % P.gp == 0 && has_group_tile(P, p)) ? 1 : 0);
}

// mark[b] counts the panels p >= 1 whose first block is b; an inclusive scan
// gives the panel of every block.
__global__ void k_mark_panels(PlanParams P, int32_t *mark) {
  GRID_STRIDE(p, P.npanels - 1) {
    int32_t b = P.brp[p + 1];
    if (b < P.nblocks) atomicAdd(&mark[b], 1);
  }
}

// *flag = 1 if some panel is cut into pieces (set to 0 beforehand).
__global__ void k_any_long(PlanParams P, int32_t *flag) {
  GRID_STRIDE(p, P.npanels) {
    if (panel_long(P, p)) *flag = 1;
  }
}

// Piece starts inside long panels.
__global__ void k_piece_flags(PlanParams P, const int32_t *bpanel, const int32_t *boff,
                              int32_t *pf) {
  GRID_STRIDE(b, P.nblocks) {
    int32_t p = bpanel[b];
    int32_t f = 0;
    if (panel_long(P, p)) {
      int32_t first = P.brp[p];
      if (b == first) {
        f = 1;
      } else {
        int32_t v0 = P.vptr[p];
        bool newv = (boff[b] - v0) / P.vwin != (boff[b - 1] - v0) / P.vwin;
        bool newb = (b - first) / P.bcap != (b - 1 - first) / P.bcap;
        f = (newv || newb) ? 1 : 0;
      }
    }
    pf[b] = f;
  }
}

// Tiles contributed by each panel, and the long-panel flags.
__global__ void k_tile_counts(PlanParams P, const int32_t *pscan, int32_t *tc, int32_t *lf) {
  GRID_STRIDE(p, P.npanels) {
    int32_t t = 0, l = 0;
    if (P.skip && group_halved(P, p)) {
      t = (p % (P.gp / 2) == 0) ? 1 : 0;
    } else if (P.skip) {  // the group tile, then the panel's own tiles
      t = (p % P.gp == 0 && has_group_tile(P, p)) ? 1 : 0;
      if (panel_long(P, p)) {
        t += pscan[P.brp[p + 1]] - pscan[P.brp[p]];
        l = 1;
      } else if (panel_heavy(P, p)) {
        t += 1;
      }
    } else if (!group_fat(P, p / P.gp)) {
      t = (p % P.gp == 0) ? 1 : 0;
    } else if (panel_long(P, p)) {
      t = pscan[P.brp[p + 1]] - pscan[P.brp[p]];
      l = 1;
    } else {
      t = 1;
    }
    tc[p] = t;
    lf[p] = l;
  }
}

__global__ void k_write_panel_tiles(PlanParams P, const int32_t *tbase, const int32_t *lbase,
                                    const int32_t *pscan, Tile *tiles, int32_t *long_panels,
                                    int32_t *long_slots) {
  GRID_STRIDE(p, P.npanels) {
    if (group_halved(P, p)) {  // one of the group's two half tiles
      const int32_t h = P.gp / 2;
      if (p % h == 0) {
        const int64_t p1 = (p + h < P.npanels) ? p + h : P.npanels;
        tiles[tbase[p]] = Tile{(int32_t)p, (int32_t)p1, P.brp[p], P.brp[p1], P.vptr[p],
                               P.vptr[p1], -1, P.log2g_group + 1};
      }
      continue;
    }
    const bool own = panel_own(P, p);
    if (p % P.gp == 0 && (P.skip ? has_group_tile(P, p) : !own)) {  // the group tile
      int64_t p1 = (p + P.gp < P.npanels) ? p + P.gp : P.npanels;
      const uint32_t heavy = P.skip ? group_heavy(P, p / P.gp) : 0u;
      tiles[tbase[p]] = Tile{(int32_t)p, (int32_t)p1, P.brp[p], P.brp[p1], P.vptr[p],
                             P.vptr[p1], heavy ? (int32_t)heavy : -1,
                             P.log2g_group | (heavy ? kSkip : 0)};
    }
    if (!own) {
    } else if (!panel_long(P, p)) {
      tiles[own_base(P, tbase, p)] =
          Tile{(int32_t)p, (int32_t)p + 1, P.brp[p], P.brp[p + 1], P.vptr[p], P.vptr[p + 1], -1,
               P.log2g_segment | kSegment};
    } else {
      int32_t l = lbase[p];
      long_panels[l] = (int32_t)p;
      long_slots[2 * l] = pscan[P.brp[p]];
      long_slots[2 * l + 1] = pscan[P.brp[p + 1]];
    }
  }
}

__global__ void k_write_piece_tiles(PlanParams P, const int32_t *bpanel, const int32_t *pf,
                                    const int32_t *pscan, const int32_t *tbase,
                                    const int32_t *boff, const uint32_t *mask32, Tile *tiles) {
  GRID_STRIDE(b, P.nblocks) {
    int32_t p = bpanel[b];
    if (!panel_long(P, p)) continue;
    int32_t first = P.brp[p];
    int32_t piece = pscan[b] + pf[b] - 1;  // global index of the piece holding b
    Tile *t = &tiles[own_base(P, tbase, p) + piece - pscan[first]];
    if (pf[b]) {
      t->p0 = p;
      t->p1 = p + 1;
      t->b0 = (int32_t)b;
      t->v0 = boff[b];
      t->slot = piece;
      t->mode = P.log2g_segment | kSegment | kPartial;
    }
    bool last = (b + 1 == P.brp[p + 1]) || pf[b + 1];
    if (last) {
      t->b1 = (int32_t)b + 1;
      t->v1 = boff[b] + __popc(mask32[b]);
    }
  }
}

// ------------------------------------------------- block-balanced plan ----
// Block-balanced plan: consecutive whole panels are packed into tiles of
// about `fbcap` blocks (a panel joins the tile of the window of fbcap blocks
// holding its first block), and panels of more than fbcap blocks are cut
// into pieces of fbcap blocks whose row sums go to the partial buffer.

struct FlatParams {
  int64_t npanels, nblocks, nnz;
  int32_t fbcap;
  const int32_t *brp, *vptr;
};

__device__ __forceinline__ bool flat_long(const FlatParams &F, int64_t p) {
  return F.brp[p + 1] - F.brp[p] > F.fbcap;
}

__device__ __forceinline__ bool flat_start(const FlatParams &F, int64_t p) {
  if (flat_long(F, p)) return false;
  if (p == 0 || flat_long(F, p - 1)) return true;
  return F.brp[p] / F.fbcap != F.brp[p - 1] / F.fbcap;
}

__device__ __forceinline__ int32_t flat_pieces(const FlatParams &F, int64_t p) {
  const int32_t nbp = F.brp[p + 1] - F.brp[p];
  return nbp > F.fbcap ? (nbp + F.fbcap - 1) / F.fbcap : 0;
}

// tiles per panel, long-panel flags and pieces per panel
__global__ void k_flat_counts(FlatParams F, int32_t *tc, int32_t *lf, int32_t *pc) {
  GRID_STRIDE(p, F.npanels) {
    const int32_t np_ = flat_pieces(F, p);
    tc[p] = np_ > 0 ? np_ : (flat_start(F, p) ? 1 : 0);
    lf[p] = np_ > 0 ? 1 : 0;
    pc[p] = np_;
  }
}

__global__ void k_flat_write(FlatParams F, const int32_t *tbase, const int32_t *lbase,
                             const int32_t *sbase, const int32_t *boff, Tile *tiles,
                             int32_t *long_panels, int32_t *long_slots) {
  GRID_STRIDE(p, F.npanels) {
    const int32_t np_ = flat_pieces(F, p);
    if (np_ > 0) {
      const int32_t l = lbase[p];
      long_panels[l] = (int32_t)p;
      long_slots[2 * l] = sbase[p];
      long_slots[2 * l + 1] = sbase[p] + np_;
      const int32_t first = F.brp[p], end = F.brp[p + 1];
      for (int32_t k = 0; k < np_; ++k) {
        const int32_t b0 = first + k * F.fbcap;
        const int32_t b1 = (b0 + F.fbcap < end) ? b0 + F.fbcap : end;
        const int32_t v1 = (b1 < F.nblocks) ? boff[b1] : (int32_t)F.nnz;
        tiles[tbase[p] + k] = Tile{(int32_t)p, (int32_t)p + 1, b0, b1, boff[b0], v1, sbase[p] + k,
                                   kFlat | kPartial};
      }
      continue;
    }
    const bool start = flat_start(F, p);
    const int32_t idx = start ? tbase[p] : tbase[p] - 1;
    if (start) {
      tiles[idx].p0 = (int32_t)p;
      tiles[idx].b0 = F.brp[p];
      tiles[idx].v0 = F.vptr[p];
      tiles[idx].slot = -1;
      tiles[idx].mode = kFlat;
    }
    const bool last = (p + 1 == F.npanels) || flat_long(F, p + 1) || flat_start(F, p + 1);
    if (last) {
      tiles[idx].p1 = (int32_t)p + 1;
      tiles[idx].b1 = F.brp[p + 1];
      tiles[idx].v1 = F.vptr[p + 1];
    }
  }
}

// ------------------------------------------------------ expanded plan ----
// Tiles of the expanded SpMV kernel, which lays a tile's values out row by
// row in shared memory (at most kExpandCap values and kExpandRows rows per
// tile):
//   - a panel of more than kExpandCap values is long: it is cut at block
//     boundaries into pieces whose value offsets lie in one window of
//     kExpandCap - 32 values (a block holds at most 32 values), and the
//     pieces' row sums go to the partial buffer;
//   - a panel of more than kExpandCap - kExpandWindow values is a tile of
//     its own;
//   - the other panels are packed into tiles of consecutive panels whose
//     first values lie in the same window of kExpandWindow values and whose
//     indices lie in the same run of kExpandRows / r panels, so a tile holds
//     at most kExpandWindow + (kExpandCap - kExpandWindow) values.

struct ExpandParams {
  int64_t npanels, nblocks, nnz;
  int32_t pp;  // panels per row window: kExpandRows / r
  const int32_t *brp, *vptr;
};

__device__ __forceinline__ int32_t panel_values(const ExpandParams &E, int64_t p) {
  return E.vptr[p + 1] - E.vptr[p];
}

__device__ __forceinline__ bool ex_long(const ExpandParams &E, int64_t p) {
  return panel_values(E, p) > kExpandCap;
}

__device__ __forceinline__ bool ex_single(const ExpandParams &E, int64_t p) {
  const int32_t nv = panel_values(E, p);
  return nv > kExpandCap - kExpandWindow && nv <= kExpandCap;
}

__device__ __forceinline__ bool ex_start(const ExpandParams &E, int64_t p) {
  if (ex_long(E, p)) return false;
  if (p == 0 || ex_long(E, p - 1) || ex_single(E, p) || ex_single(E, p - 1)) return true;
  return E.vptr[p] / kExpandWindow != E.vptr[p - 1] / kExpandWindow ||
         p / E.pp != (p - 1) / E.pp;
}

// Piece starts inside long panels (block b starts a piece).
__global__ void k_ex_piece_flags(ExpandParams E, const int32_t *bpanel, const int32_t *boff,
                                 int32_t *pf) {
  GRID_STRIDE(b, E.nblocks) {
    const int32_t p = bpanel[b];
    int32_t f = 0;
    if (ex_long(E, p)) {
      const int32_t first = E.brp[p], v0 = E.vptr[p];
      constexpr int32_t win = kExpandCap - 32;
      f = (b == first || (boff[b] - v0) / win != (boff[b - 1] - v0) / win) ? 1 : 0;
    }
    pf[b] = f;
  }
}

// tiles per panel and long-panel flags
__global__ void k_ex_counts(ExpandParams E, const int32_t *pscan, int32_t *tc, int32_t *lf) {
  GRID_STRIDE(p, E.npanels) {
    const bool lg = ex_long(E, p);
    tc[p] = lg ? pscan[E.brp[p + 1]] - pscan[E.brp[p]] : (ex_start(E, p) ? 1 : 0);
    lf[p] = lg ? 1 : 0;
  }
}

__global__ void k_ex_write_panels(ExpandParams E, const int32_t *tbase, const int32_t *lbase,
                                  const int32_t *pscan, Tile *tiles, int32_t *long_panels,
                                  int32_t *long_slots) {
  GRID_STRIDE(p, E.npanels) {
    if (ex_long(E, p)) {
      const int32_t l = lbase[p];
      long_panels[l] = (int32_t)p;
      long_slots[2 * l] = pscan[E.brp[p]];
      long_slots[2 * l + 1] = pscan[E.brp[p + 1]];
      continue;
    }
    const bool start = ex_start(E, p);
    const int32_t idx = start ? tbase[p] : tbase[p] - 1;
    if (start) {
      tiles[idx].p0 = (int32_t)p;
      tiles[idx].b0 = E.brp[p];
      tiles[idx].v0 = E.vptr[p];
      tiles[idx].slot = -1;
      tiles[idx].mode = kExpand;
    }
    const bool last = (p + 1 == E.npanels) || ex_long(E, p + 1) || ex_start(E, p + 1);
    if (last) {
      tiles[idx].p1 = (int32_t)p + 1;
      tiles[idx].b1 = E.brp[p + 1];
      tiles[idx].v1 = E.vptr[p + 1];
    }
  }
}

__global__ void k_ex_write_pieces(ExpandParams E, const int32_t *bpanel, const int32_t *pf,
                                  const int32_t *pscan, const int32_t *tbase,
                                  const int32_t *boff, Tile *tiles) {
  GRID_STRIDE(b, E.nblocks) {
    const int32_t p = bpanel[b];
    if (!ex_long(E, p)) continue;
    const int32_t first = E.brp[p];
    const int32_t piece = pscan[b] + pf[b] - 1;  // global index of the piece holding b
    Tile *t = &tiles[tbase[p] + piece - pscan[first]];
    if (pf[b]) {
      t->p0 = p;
      t->p1 = p + 1;
      t->b0 = (int32_t)b;
      t->v0 = boff[b];
      t->slot = piece;
      t->mode = kExpand | kPartial;
    }
    const bool last = (b + 1 == E.brp[p + 1]) || pf[b + 1];
    if (last) {
      t->b1 = (int32_t)b + 1;
      t->v1 = (b + 1 < E.nblocks) ? boff[b + 1] : (int32_t)E.nnz;
    }
  }
}

// Busy share of the row-group plan's block slots: a group tile keeps its
// panels * G = 32 / r slots busy for as many rounds as its longest panel
// needs (per_round = 32 / r).
__global__ void k_group_efficiency(const Tile *tiles, int64_t ntiles, const int32_t *brp,
                                   int per_round, unsigned long long *acc) {
  unsigned long long used = 0, slots = 0;
  GRID_STRIDE(t, ntiles) {
    const Tile T = tiles[t];
    const int64_t G = 1ll << (T.mode & 15);
    if (T.mode & kSegment) {
      const int64_t nbt = T.b1 - T.b0;
      used += nbt;
      slots += G * ((nbt + G - 1) / G);
    } else {
      int64_t mx = 0;
      for (int32_t p = T.p0; p < T.p1; ++p) {
        if ((T.mode & kSkip) && ((T.slot >> (p - T.p0)) & 1)) continue;
        const int64_t nbp = brp[p + 1] - brp[p];
        used += nbp;
        mx = nbp > mx ? nbp : mx;
      }
      slots += (int64_t)per_round * ((mx + G - 1) / G);
    }
  }
  // one atomic per warp: same-address atomics from every thread were most
  // of this kernel's time
  for (int o = 16; o > 0; o >>= 1) {
    used += __shfl_xor_sync(0xffffffffu, used, o);
    slots += __shfl_xor_sync(0xffffffffu, slots, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&acc[0], used);
    atomicAdd(&acc[1], slots);
  }
}

template <typename T>
struct Tmp {
  T *p = nullptr;
  cudaStream_t s;
  explicit Tmp(cudaStream_t st) : s(st) {}
  cudaError_t alloc(int64_t n) {
    return scratch_alloc((void **)&p, (size_t)std::max<int64_t>(n, 1) * sizeof(T), s);
  }
  ~Tmp() {
    if (p) cudaFreeAsync(p, s);
  }
};

struct ReadI32 {
  const int32_t *m;
  __device__ int32_t operator()(int64_t i) const { return m[i]; }
};
struct ReadI32Pad {  // m[i] for i < n, 0 at i == n (so an exclusive scan of n+1 gives the total)
  const int32_t *m;
  int64_t n;
  __device__ int32_t operator()(int64_t i) const { return i < n ? m[i] : 0; }
};
struct WriteI32 {
  int32_t *o;
  __device__ void operator()(int64_t i, int32_t v) const { o[i] = v; }
};

int env_int(const char *name, int dflt) {
  const char *e = getenv(name);
  return (e && *e) ? atoi(e) : dflt;
}

int round_up(int v, int m) { return (v + m - 1) / m * m; }

}  // namespace

#define CK(call, what)                            \
  do {                                            \
    spc5_status _st = cuda_check((call), (what)); \
    if (_st != SPC5_OK) return _st;               \
  } while (0)

spc5_status build_expanded(int64_t np, int64_t nb, int64_t nvalues, int r, const int32_t *brp,
                           const int32_t *vptr, const int32_t *boff, cudaStream_t s,
                           ExpandedPlan *out) {
  *out = ExpandedPlan{};
  int32_t counts[3] = {0, 0, 0};
  Tmp<int32_t> bpanel(s), pf(s), pscan(s), tc(s), lf(s), tbase(s), lbase(s), tmp(s);
  ExpandParams E{np, nb, nvalues, kExpandRows / r, brp, vptr};
  PlanParams P{};
  P.npanels = np;
  P.nblocks = nb;
  P.brp = brp;
  if (np > 0) {
    CK(bpanel.alloc(nb), "alloc");
    CK(pf.alloc(nb), "alloc");
    CK(pscan.alloc(nb + 1), "alloc");
    CK(tc.alloc(np), "alloc");
    CK(lf.alloc(np), "alloc");
    CK(tbase.alloc(np + 1), "alloc");
    CK(lbase.alloc(np + 1), "alloc");
    CK(tmp.alloc(scan_tmp_elems(std::max<int64_t>(nb, np) + 1)), "alloc");
    if (nb > 0) {
      CK(cudaMemsetAsync(bpanel.p, 0, (size_t)nb * sizeof(int32_t), s), "memset");
      if (np > 1) k_mark_panels<<<grid_for(np), kThreads, 0, s>>>(P, bpanel.p);
      CK(device_scan<int32_t>(nb, ReadI32{bpanel.p}, WriteI32{bpanel.p}, AddI32{}, 0, true,
                              tmp.p, s),
         "scan panels");
      k_ex_piece_flags<<<grid_for(nb), kThreads, 0, s>>>(E, bpanel.p, boff, pf.p);
    }
    CK(device_scan<int32_t>(nb + 1, ReadI32Pad{pf.p, nb}, WriteI32{pscan.p}, AddI32{}, 0, false,
                            tmp.p, s),
       "scan pieces");
    k_ex_counts<<<grid_for(np), kThreads, 0, s>>>(E, pscan.p, tc.p, lf.p);
    CK(device_scan<int32_t>(np + 1, ReadI32Pad{tc.p, np}, WriteI32{tbase.p}, AddI32{}, 0, false,
                            tmp.p, s),
       "scan expanded tiles");
    CK(device_scan<int32_t>(np + 1, ReadI32Pad{lf.p, np}, WriteI32{lbase.p}, AddI32{}, 0, false,
                            tmp.p, s),
       "scan expanded long panels");
    CK(cudaMemcpyAsync(&counts[0], tbase.p + np, 4, cudaMemcpyDeviceToHost, s), "rd");
    CK(cudaMemcpyAsync(&counts[1], lbase.p + np, 4, cudaMemcpyDeviceToHost, s), "rd");
    CK(cudaMemcpyAsync(&counts[2], pscan.p + nb, 4, cudaMemcpyDeviceToHost, s), "rd");
  }
  CK(cudaStreamSynchronize(s), "sync expanded plan counts");
  out->ntiles = counts[0];
  out->nlong = counts[1];
  out->npieces = counts[2];
  CK(cudaMalloc((void **)&out->tiles, (size_t)std::max<int64_t>(out->ntiles, 1) * sizeof(Tile)),
     "alloc expanded tiles");
  CK(cudaMalloc((void **)&out->long_panels, (size_t)std::max<int64_t>(out->nlong, 1) * 4),
     "alloc");
  CK(cudaMalloc((void **)&out->long_slots, (size_t)std::max<int64_t>(out->nlong, 1) * 8),
     "alloc");
  if (np > 0) {
    k_ex_write_panels<<<grid_for(np), kThreads, 0, s>>>(E, tbase.p, lbase.p, pscan.p, out->tiles,
                                                        out->long_panels, out->long_slots);
    if (nb > 0 && out->nlong > 0)
      k_ex_write_pieces<<<grid_for(nb), kThreads, 0, s>>>(E, bpanel.p, pf.p, pscan.p, tbase.p,
                                                          boff, out->tiles);
  }
  CK(cudaGetLastError(), "expanded plan kernels");
  return SPC5_OK;
}

namespace {

// Device arrays of the block-balanced or expanded plan (fntiles, fnlong and
// fnpieces set).
cudaError_t alloc_flat_arrays(spc5_matrix *A) {
  cudaError_t e = cudaMalloc((void **)&A->ftiles,
                             (size_t)std::max<int64_t>(A->fntiles, 1) * sizeof(Tile));
  if (e == cudaSuccess)
    e = cudaMalloc((void **)&A->flong_panels, (size_t)std::max<int64_t>(A->fnlong, 1) * 4);
  if (e == cudaSuccess)
    e = cudaMalloc((void **)&A->flong_slots, (size_t)std::max<int64_t>(A->fnlong, 1) * 8);
  if (e == cudaSuccess)
    e = cudaMalloc((void **)&A->fpartial,
                   (size_t)std::max<int64_t>(A->fnpieces, 1) * A->r * sizeof(double));
  if (e == cudaSuccess)
    A->device_bytes += A->fntiles * (int64_t)sizeof(Tile) + A->fnlong * 12 +
                       A->fnpieces * A->r * (int64_t)sizeof(double);
  return e;
}

// Builds the block-balanced or the expanded plan, deciding first which plan
// the SpMV uses.
spc5_status plan_flat(spc5_matrix *A, const int32_t *boff, cudaStream_t s,
                      const PlanOptions &opt) {
  const int64_t np = A->npanels, nb = A->nblocks;
  A->fntiles = A->fnlong = A->fnpieces = 0;
  CK(cudaMalloc((void **)&A->fsched, 2 * sizeof(uint32_t)), "alloc tile counters");
  CK(cudaMemsetAsync(A->fsched, 0, 2 * sizeof(uint32_t), s), "zero tile counters");
  A->device_bytes += 8;

  // busy share of the row-group plan
  Tmp<unsigned long long> acc(s);
  CK(acc.alloc(2), "alloc");
  CK(cudaMemsetAsync(acc.p, 0, 2 * sizeof(unsigned long long), s), "memset");
  if (A->ntiles > 0)
    k_group_efficiency<<<std::min<unsigned>(grid_for(A->ntiles), 1024u), kThreads, 0, s>>>(
        A->tiles, A->ntiles, A->block_rowptr, 32 / A->r, acc.p);
  unsigned long long hacc[2] = {0, 0};
  CK(cudaMemcpyAsync(hacc, acc.p, sizeof(hacc), cudaMemcpyDeviceToHost, s), "rd");

  CK(cudaStreamSynchronize(s), "sync group efficiency");
  A->group_efficiency = hacc[1] > 0 ? (double)hacc[0] / (double)hacc[1] : 1.0;
  // Which plan the SpMV uses.  The staged kernel reads its tiles as
  // contiguous panel ranges, so the other plans are for the direct kernels.
  // Default: row groups unless they would keep less than 70% of their block
  // slots busy; then the block-balanced plan, with values split evenly over
  // the lanes for r >= 4 (plan 3: the cross-lane scan of r sums is paid per
  // 256 blocks) and four blocks per lane for r <= 2 (plan 1, cheaper per
  // value there).  The expanded plan measured slower on every block shape;
  // spc5_tune still tries it.
  const int dflt = A->group_efficiency < 0.7 ? (A->r >= 4 ? 3 : 1) : 0;
  int flat = opt.flat >= 0 ? opt.flat : env_int("SPC5_FLAT", dflt);
  if (flat < 0 || flat > 3) flat = dflt;
  A->flat = A->kernel == 0 ? flat : 0;
  const bool expanded = A->flat == 2;

  if (A->flat == 0) return SPC5_OK;  // row groups or staged: no second tile set

  int32_t counts[3] = {0, 0, 0};
  Tmp<int32_t> bpanel(s), pf(s), pscan(s), tc(s), lf(s), tbase(s), lbase(s), tmp(s);
  if (!expanded) {  // block-balanced tiles
    int dev = 0, sms = 1;
    CK(cudaGetDevice(&dev), "cudaGetDevice");
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "sm count");
    // about eight tiles for every resident warp (48 per SM)
    const int64_t want = (int64_t)8 * sms * 48;
    int64_t fb = (nb + want - 1) / want;
    fb = (fb + 31) / 32 * 32;
    const int fbcap = (int)std::min<int64_t>(std::max<int64_t>(fb, 64), 2048);
    FlatParams F{np, nb, A->nnz, fbcap, A->block_rowptr, A->panel_vptr};
    if (np > 0) {
      CK(tc.alloc(np), "alloc");
      CK(lf.alloc(np), "alloc");
      CK(pf.alloc(np), "alloc");
      CK(tbase.alloc(np + 1), "alloc");
      CK(lbase.alloc(np + 1), "alloc");
      CK(pscan.alloc(np + 1), "alloc");
      CK(tmp.alloc(scan_tmp_elems(np + 1)), "alloc");
      k_flat_counts<<<grid_for(np), kThreads, 0, s>>>(F, tc.p, lf.p, pf.p);
      CK(device_scan<int32_t>(np + 1, ReadI32Pad{tc.p, np}, WriteI32{tbase.p}, AddI32{}, 0,
                              false, tmp.p, s),
         "scan flat tiles");
      CK(device_scan<int32_t>(np + 1, ReadI32Pad{lf.p, np}, WriteI32{lbase.p}, AddI32{}, 0,
                              false, tmp.p, s),
         "scan flat long panels");
      CK(device_scan<int32_t>(np + 1, ReadI32Pad{pf.p, np}, WriteI32{pscan.p}, AddI32{}, 0,
                              false, tmp.p, s),
         "scan flat pieces");
      CK(cudaMemcpyAsync(&counts[0], tbase.p + np, 4, cudaMemcpyDeviceToHost, s), "rd");
      CK(cudaMemcpyAsync(&counts[1], lbase.p + np, 4, cudaMemcpyDeviceToHost, s), "rd");
      CK(cudaMemcpyAsync(&counts[2], pscan.p + np, 4, cudaMemcpyDeviceToHost, s), "rd");
    }
    CK(cudaStreamSynchronize(s), "sync flat plan counts");
    A->fntiles = counts[0];
    A->fnlong = counts[1];
    A->fnpieces = counts[2];
    CK(alloc_flat_arrays(A), "alloc flat plan");
    if (np > 0)
      k_flat_write<<<grid_for(np), kThreads, 0, s>>>(F, tbase.p, lbase.p, pscan.p, boff,
                                                     A->ftiles, A->flong_panels, A->flong_slots);
    CK(cudaGetLastError(), "flat plan kernels");
    return SPC5_OK;
  }

  ExpandedPlan ep;
  {
    spc5_status st = build_expanded(np, nb, A->nnz, A->r, A->block_rowptr, A->panel_vptr, boff, s,
                                    &ep);
    if (st != SPC5_OK) return st;
  }
  A->ftiles = ep.tiles;
  A->flong_panels = ep.long_panels;
  A->flong_slots = ep.long_slots;
  A->fntiles = ep.ntiles;
  A->fnlong = ep.nlong;
  A->fnpieces = ep.npieces;
  CK(cudaMalloc((void **)&A->fpartial,
                (size_t)std::max<int64_t>(A->fnpieces, 1) * A->r * sizeof(double)),
     "alloc expanded partial");
  A->device_bytes += A->fntiles * (int64_t)sizeof(Tile) + A->fnlong * 12 +
                     A->fnpieces * A->r * (int64_t)sizeof(double);
  const int64_t nro = (np + A->fnpieces) * A->r;
  CK(cudaMalloc((void **)&A->frowoff, (size_t)std::max<int64_t>(nro, 1) * sizeof(uint16_t)),
     "alloc expanded row starts");
  A->device_bytes += nro * (int64_t)sizeof(uint16_t);
  return expand_row_starts(A, s);
}

void free_flat(spc5_matrix *A) {
  cudaFree(A->ftiles);
  cudaFree(A->flong_panels);
  cudaFree(A->flong_slots);
  cudaFree(A->fpartial);
  cudaFree(A->fsched);
  A->device_bytes -= A->fntiles * (int64_t)sizeof(Tile) + A->fnlong * 12 +
                     A->fnpieces * A->r * (int64_t)sizeof(double) + 8;
  if (A->frowoff) {
    cudaFree(A->frowoff);
    A->device_bytes -= (A->npanels + A->fnpieces) * A->r * (int64_t)sizeof(uint16_t);
    A->frowoff = nullptr;
  }
  A->ftiles = nullptr;
  A->flong_panels = nullptr;
  A->flong_slots = nullptr;
  A->fpartial = nullptr;
  A->fsched = nullptr;
  A->fntiles = A->fnlong = A->fnpieces = 0;
}

}  // namespace

spc5_status plan_tiles(spc5_matrix *A, const uint32_t *mask32, const int32_t *boff,
                       cudaStream_t s, const PlanOptions &opt) {
  const int r = A->r;
  const int64_t np = A->npanels, nb = A->nblocks;
  int log2r = 0;
  while ((1 << log2r) < r) ++log2r;
  const int log2g_segment = 5 - log2r;

  // the staged kernel is built for FP64 values only
  const int want_kernel = opt.kernel >= 0 ? opt.kernel : env_int("SPC5_KERNEL", 0);
  A->kernel = (A->value_dtype == SPC5_F64 && want_kernel) ? 1 : 0;
  const bool staged = A->kernel == 1;
  // lanes per row in group tiles: a few block rounds per tile
  double avg_b = np > 0 ? (double)nb / (double)np : 0.0;
  double avg_v = np > 0 ? (double)A->nnz / (double)np : 0.0;
  int log2g = 0;
  const double rounds = staged ? 12.0 : 8.0;
  const int max_log2g = staged ? log2g_segment : std::min(2, log2g_segment);
  while (log2g < max_log2g && avg_b / (double)(1 << log2g) > rounds) ++log2g;
  log2g = opt.log2g >= 0 ? opt.log2g : env_int("SPC5_LOG2G_GROUP", log2g);
  log2g = std::min(std::max(log2g, 0), log2g_segment);
  const int gp = 32 >> (log2r + log2g);

  // Tile capacity.  Staged kernel: one shared-memory stage.  Direct kernel:
  // only bounds the work of one warp (long panels are cut into pieces).
  int vcap, bcap;
  if (staged) {
    vcap = std::min(std::max(round_up((int)(1.5 * gp * avg_v) + 64, 64), 512), 4096);
    bcap = std::min(std::max(round_up((int)(1.5 * gp * avg_b) + 32, 32), 128), 1024);
  } else {
    vcap = std::min(std::max(round_up((int)(2.0 * gp * avg_v) + 64, 64), 2048), 8192);
    bcap = std::min(std::max(round_up((int)(2.0 * gp * avg_b) + 32, 32), 256), 2048);
    // A small matrix with long rows (the dense 2048 x 2048 has 64 groups of
    // eight 4-row panels, 65536 values each) gives far fewer tiles than the
    // GPU holds warps: lower the caps until its long panels are cut into
    // about one piece per two resident warps (measured on the dense matrix:
    // finer pieces cost more in partial sums than they gain in balance).
    // Small matrices with short rows keep their groups: they are cheap, and
    // batches supply the parallelism.
    const int64_t warps = (int64_t)device_sm_count() * 48;
    if ((np + gp - 1) / gp < 2 * warps && gp * avg_v >= 4096.0) {
      const int64_t vper = 2 * A->nnz / warps, bper = 2 * nb / warps;
      vcap = (int)std::min<int64_t>(vcap, std::max<int64_t>(round_up((int)vper, 64), 256));
      bcap = (int)std::min<int64_t>(bcap, std::max<int64_t>(round_up((int)bper, 32), 32));
    }
  }
  vcap = opt.vcap > 0 ? opt.vcap : env_int("SPC5_VCAP", vcap);
  bcap = opt.bcap > 0 ? opt.bcap : env_int("SPC5_BCAP", bcap);
  if (vcap < 64 || bcap < 1) {
    set_error("invalid stage capacity");
    return SPC5_EINVAL;
  }
  const int mb = A->r * A->c / 8;
  auto r16 = [](int v) { return (v + 15) / 16 * 16; };
  int stage = 64 + r16(vcap * 8 + 16) + r16(bcap * 4 + 16) + r16(bcap * mb + 16) +
              2 * r16((gp + 1) * 4 + 16);
  double filling = nb > 0 ? (double)A->nnz / ((double)nb * A->r * A->c) : 0.0;
  int body = opt.body >= 0 ? opt.body : env_int("SPC5_BODY", filling >= 0.3 ? 3 : 2);
  body = std::min(std::max(body, 0), 3);
  int dev = 0, optin = 0;
  CK(cudaGetDevice(&dev), "cudaGetDevice");
  CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), "smem attr");
  int budget = optin - 2048;
  int consumers;
  int stages;
  const int xs_bytes = (1024 + 32) * 8;  // per consumer, bodies 2 and 3
  if (body >= 2) {
    consumers = std::min(std::max(env_int("SPC5_CONSUMERS", 8), 1), 16);
    stages = std::min(32, (budget - consumers * xs_bytes) / stage);
  } else {
    stages = std::min(32, budget / stage);
    consumers = std::min(16, std::max(2, stages / 2 + 1));
    consumers = std::min(std::max(env_int("SPC5_CONSUMERS", consumers), 1), 16);
  }
  stages = std::min(stages, env_int("SPC5_STAGES", stages));
  if (staged && stages < 2) {
    set_error("pipeline stage does not fit shared memory");
    return SPC5_EINVAL;
  }
  A->log2_group_lanes = log2g;
  A->group_panels = gp;
  A->vcap = vcap;
  A->bcap = bcap;
  A->stages = stages;
  A->consumers = consumers;
  A->stage_bytes = stage;
  // direct kernel bodies: 0 per-block set-bit loop, 1 per-block predicated
  // loop over the c bits, 2 row stream across blocks, 3 queued row stream,
  // 4 four-block rounds, 5 row stream passing empty blocks, 6 row stream at
  // 64 warps per SM, 7 pipelined row stream passing empty blocks (2 to 7 on
  // row-group tiles with one lane per row; other tiles use body 0)
  A->body = staged ? body
                   : std::min(std::max(opt.body >= 0 ? opt.body : env_int("SPC5_BODY", 0), 0), 7);
  A->dynamic = (opt.dynamic >= 0 ? opt.dynamic : env_int("SPC5_DYNAMIC", 0)) != 0 ? 1 : 0;

  A->halves = 0;
  if (np == 0) return SPC5_OK;
  PlanParams P{np, nb, gp, vcap, bcap, vcap - 32, log2g, log2g_segment,
               A->block_rowptr, A->panel_vptr, staged ? 0 : 1,
               (int32_t)std::min<double>(std::max(8.0 * avg_v, 64.0), (double)vcap),
               (int32_t)std::min<double>(std::max(8.0 * avg_b, 8.0), (double)bcap),
               INT64_MAX};

  Tmp<int32_t> bpanel(s), pf(s), pscan(s), tc(s), tbase(s), lf(s), lbase(s), tmp(s);
  CK(bpanel.alloc(nb), "alloc");
  CK(pf.alloc(nb), "alloc");
  CK(pscan.alloc(nb + 1), "alloc");
  CK(tc.alloc(np), "alloc");
  CK(lf.alloc(np), "alloc");
  CK(tbase.alloc(np + 1), "alloc");
  CK(lbase.alloc(np + 1), "alloc");
  CK(tmp.alloc(scan_tmp_elems(std::max<int64_t>(nb, np) + 1)), "alloc");
  // The block-level passes (each block's panel, piece starts and their
  // prefix sum) only serve panels cut into pieces: without any (stencils,
  // FEM meshes, uniform rows) the piece prefix is all zeros.
  int32_t any_long = 0;
  if (nb > 0 && np > 0) {
    CK(cudaMemsetAsync(tc.p, 0, sizeof(int32_t), s), "memset");
    k_any_long<<<grid_for(np), kThreads, 0, s>>>(P, tc.p);
    CK(cudaMemcpyAsync(&any_long, tc.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "rd");
    CK(cudaStreamSynchronize(s), "sync long panels");
  }
  if (any_long) {
    CK(cudaMemsetAsync(bpanel.p, 0, (size_t)nb * sizeof(int32_t), s), "memset");
    if (np > 1) k_mark_panels<<<grid_for(np), kThreads, 0, s>>>(P, bpanel.p);
    CK(device_scan<int32_t>(nb, ReadI32{bpanel.p}, WriteI32{bpanel.p}, AddI32{}, 0, true, tmp.p,
                            s),
       "scan panels");
    k_piece_flags<<<grid_for(nb), kThreads, 0, s>>>(P, bpanel.p, boff, pf.p);
    CK(device_scan<int32_t>(nb + 1, ReadI32Pad{pf.p, nb}, WriteI32{pscan.p}, AddI32{}, 0, false,
                            tmp.p, s),
       "scan pieces");
  } else {
    CK(cudaMemsetAsync(pscan.p, 0, (size_t)(nb + 1) * sizeof(int32_t), s), "zero pieces");
  }
  k_tile_counts<<<grid_for(np), kThreads, 0, s>>>(P, pscan.p, tc.p, lf.p);
  CK(device_scan<int32_t>(np + 1, ReadI32Pad{tc.p, np}, WriteI32{tbase.p}, AddI32{}, 0, false,
                          tmp.p, s),
     "scan tiles");
  CK(device_scan<int32_t>(np + 1, ReadI32Pad{lf.p, np}, WriteI32{lbase.p}, AddI32{}, 0, false,
                          tmp.p, s),
     "scan long panels");
  int32_t counts[3] = {0, 0, 0};
  CK(cudaMemcpyAsync(&counts[0], tbase.p + np, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "rd");
  CK(cudaMemcpyAsync(&counts[1], lbase.p + np, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "rd");
  CK(cudaMemcpyAsync(&counts[2], pscan.p + nb, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "rd");
  CK(cudaStreamSynchronize(s), "sync plan counts");
  {
    // The direct kernel deals tiles grid-stride over its resident warps W,
    // so T tiles take ceil(T / W) rounds and the last one, T mod W tiles,
    // keeps part of the GPU busy for a whole tile's time (27-point 100^3,
    // beta(4,8): 31250 tiles over 7296 warps, a fifth round for 2066 of
    // them).  When that round fills at most half the warps, its groups are
    // cut into two tiles of half the panels with twice the lanes per row:
    // each half tile takes about half a tile's time, but runs the general
    // loop instead of a one-lane-per-row body (measured -7 % to +7 %), so
    // spc5_tune tries it on the winning row-group plan.
    const int per_sm = A->body == 4 ? 40 : (A->body == 6 ? 64 : 48);
    const int64_t W = (int64_t)device_sm_count() * per_sm;
    const int64_t T = counts[0], rem = W > 0 ? T % W : 0;
    const int64_t ngroups = (np + gp - 1) / gp;
    const bool want = (opt.halves >= 0 ? opt.halves : env_int("SPC5_HALVES", 0)) != 0;
    A->halves = 0;
    if (!staged && want && gp >= 2 && log2g < log2g_segment && T > W && rem > 0 &&
        2 * rem <= W && rem <= ngroups) {
      A->halves = 1;
      P.half_from = ngroups - rem;
      k_tile_counts<<<grid_for(np), kThreads, 0, s>>>(P, pscan.p, tc.p, lf.p);
      CK(device_scan<int32_t>(np + 1, ReadI32Pad{tc.p, np}, WriteI32{tbase.p}, AddI32{}, 0,
                              false, tmp.p, s),
         "scan tiles");
      CK(cudaMemcpyAsync(&counts[0], tbase.p + np, sizeof(int32_t), cudaMemcpyDeviceToHost, s),
         "rd");
      CK(cudaStreamSynchronize(s), "sync plan counts");
    }
  }
  A->ntiles = counts[0];
  A->nlong = counts[1];
  A->npieces = counts[2];
  CK(cudaMalloc((void **)&A->tiles, (size_t)std::max<int64_t>(A->ntiles, 1) * sizeof(Tile)),
     "alloc tiles");
  CK(cudaMalloc((void **)&A->long_panels, (size_t)std::max<int64_t>(A->nlong, 1) * 4), "alloc");
  CK(cudaMalloc((void **)&A->long_slots, (size_t)std::max<int64_t>(A->nlong, 1) * 8), "alloc");
  CK(cudaMalloc((void **)&A->partial,
                (size_t)std::max<int64_t>(A->npieces, 1) * A->r * sizeof(double)),
     "alloc partial");
  A->device_bytes += A->ntiles * (int64_t)sizeof(Tile) + A->nlong * 12 +
                     A->npieces * A->r * (int64_t)sizeof(double);
  k_write_panel_tiles<<<grid_for(np), kThreads, 0, s>>>(P, tbase.p, lbase.p, pscan.p, A->tiles,
                                                       A->long_panels, A->long_slots);
  if (nb > 0 && A->nlong > 0)
    k_write_piece_tiles<<<grid_for(nb), kThreads, 0, s>>>(P, bpanel.p, pf.p, pscan.p, tbase.p,
                                                         boff, mask32, A->tiles);
  CK(cudaGetLastError(), "plan kernels");
  return plan_flat(A, boff, s, opt);
}

namespace {
template <typename MaskT>
__global__ void k_mask32(int64_t nb, const MaskT *masks, uint32_t *mask32) {
  GRID_STRIDE(b, nb) { mask32[b] = (uint32_t)masks[b]; }
}
struct PopcRead {
  const uint32_t *m;
  __device__ int32_t operator()(int64_t i) const { return __popc(m[i]); }
};
}  // namespace

spc5_status replan(spc5_matrix *A, cudaStream_t s, const PlanOptions &opt) {
  CK(cudaStreamSynchronize(s), "sync before replan");
  cudaFree(A->tiles);
  cudaFree(A->long_panels);
  cudaFree(A->long_slots);
  cudaFree(A->partial);
  A->device_bytes -= A->ntiles * (int64_t)sizeof(Tile) + A->nlong * 12 +
                     A->npieces * A->r * (int64_t)sizeof(double);
  A->tiles = nullptr;
  A->long_panels = nullptr;
  A->long_slots = nullptr;
  A->partial = nullptr;
  A->ntiles = A->nlong = A->npieces = 0;
  free_flat(A);
  const int64_t nb = A->nblocks;
  Tmp<uint32_t> mask32(s);
  Tmp<int32_t> boff(s), tmp(s);
  CK(mask32.alloc(nb), "alloc");
  CK(boff.alloc(nb), "alloc");
  CK(tmp.alloc(scan_tmp_elems(nb)), "alloc");
  if (nb > 0) {
    const int mb = A->r * A->c / 8;
    if (mb == 1)
      k_mask32<uint8_t><<<grid_for(nb), kThreads, 0, s>>>(nb, (const uint8_t *)A->masks, mask32.p);
    else if (mb == 2)
      k_mask32<uint16_t><<<grid_for(nb), kThreads, 0, s>>>(nb, (const uint16_t *)A->masks,
                                                           mask32.p);
    else
      k_mask32<uint32_t><<<grid_for(nb), kThreads, 0, s>>>(nb, (const uint32_t *)A->masks,
                                                           mask32.p);
    CK(device_scan<int32_t>(nb, PopcRead{mask32.p}, WriteI32{boff.p}, AddI32{}, 0, false, tmp.p,
                            s),
       "scan popcounts");
  }
  spc5_status st = plan_tiles(A, mask32.p, boff.p, s, opt);
  if (st != SPC5_OK) return st;
  CK(cudaStreamSynchronize(s), "sync replan");
  return SPC5_OK;
}

}  // namespace spc5
