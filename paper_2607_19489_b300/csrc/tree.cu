// tree.cu -- BuildTree for all levels (Sec. 3.1, Alg. 2) and the neighbour
// index that the merged-tree searches of Sec. 3.2 reduce to.
//
// Per level l, from lmax down to lmin, the cells of level l are the input
// leaves plus the parents of the level l+1 octs.  They are radix sorted by
// Morton key (x in the lowest bit of each triple); consecutive runs of the
// same key>>3 are the octs of level l, so after sorting cell id = 8*oct +
// (key & 7), the order the paper's oct tree (RAMSES) and the oracle use.
// Levels below lmin are complete grids.
//
// The 27-neighbour index is then built top-down without hashing: the
// neighbour (dx,dy,dz) of oct o's parent cell lies in the parent oct's own
// neighbour table, and its child oct (or its leaf status) is read from that
// level's cell_child array -- the fully threaded tree idea of RAMSES.
//
// Oct counts follow from the leaf counts alone (n_oct[l] = (leaves[l] +
// n_oct[l+1]) / 8), so the host sizes everything up front and the whole build
// runs without synchronising; duplicates, incomplete octs, out-of-box
// indices, non-finite masses and graded-rule violations are latched as error
// bits, every kernel bounds-checks the indices it follows, and one
// synchronisation at the end reads the error word and the list lengths.
#include <cub/cub.cuh>

#include <chrono>

#include "fmm_internal.cuh"

namespace fmm {
namespace {

__device__ __forceinline__ uint64_t spread3(uint32_t v) {
  uint64_t x = v & 0x1FFFFF;
  x = (x | (x << 32)) & 0x1F00000000FFFFull;
  x = (x | (x << 16)) & 0x1F0000FF0000FFull;
  x = (x | (x << 8)) & 0x100F00F00F00F00Full;
  x = (x | (x << 4)) & 0x10C30C30C30C30C3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

__global__ void k_leaf_keys(int64_t n, const int32_t* __restrict__ ijk, const double* __restrict__ mass,
                            int level, uint64_t* keys, int32_t* vals, unsigned* err) {
  pdl_wait();
  pdl_trigger();
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int x = ijk[3 * i], y = ijk[3 * i + 1], z = ijk[3 * i + 2];
  int lim = 1 << level;
  if (x < 0 || y < 0 || z < 0 || x >= lim || y >= lim || z >= lim) {
    atomicOr(err, kErrOutOfBox);
    x = y = z = 0;
  }
  if (!isfinite(mass[i])) atomicOr(err, kErrNonFinite);
  keys[i] = spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
  vals[i] = (int32_t)(-1 - i);
}

__global__ void k_refined_keys(int64_t n, const uint64_t* __restrict__ octkey_next, uint64_t* keys,
                               int32_t* vals) {
  pdl_wait();
  pdl_trigger();
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  keys[i] = octkey_next[i];
  vals[i] = (int32_t)i;
}

__global__ void k_oct_flags(int64_t n, const uint64_t* __restrict__ k, int32_t* flags, unsigned* err) {
  pdl_wait();
  pdl_trigger();
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int f = 1;
  if (i > 0) {
    if (k[i] == k[i - 1]) atomicOr(err, kErrDuplicate);
    f = (k[i] >> 3) != (k[i - 1] >> 3);
  }
  flags[i] = f;
}

// Cell id = sorted position.  A level is consistent only if every run of
// siblings is a complete oct, i.e. position == 8 * oct + (key & 7) everywhere
// and the number of octs equals the count derived from the leaf counts.
// check_keys: a partial update re-sorts this level but must not change its
// octs; their keys are compared with the stored ones instead of written.
__global__ void k_scatter_level(int64_t n, int64_t n_oct, const uint64_t* __restrict__ k,
                                const int32_t* __restrict__ v, const int32_t* __restrict__ scan, uint64_t* oct_key,
                                int32_t* cell_child, int32_t* leaf_cell, int32_t* oct_parent_next,
                                int64_t n_oct_next, int64_t n_leaf, int check_keys, unsigned* err) {
  pdl_wait();
  pdl_trigger();
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t oct = scan[i] - 1;
  uint64_t key = k[i];
  if (i == n - 1 && oct + 1 != n_oct) atomicOr(err, kErrIncomplete);
  if (oct >= n_oct || i != 8 * oct + (int64_t)(key & 7)) {
    atomicOr(err, kErrIncomplete);
    return;
  }
  if (i == 0 || (k[i - 1] >> 3) != (key >> 3)) {
    if (!check_keys)
      oct_key[oct] = key >> 3;
    else if (oct_key[oct] != key >> 3)
      atomicOr(err, kErrStructure);
  }
  int32_t val = v[i];
  cell_child[i] = val;
  if (val >= 0) {
    if (val < n_oct_next) oct_parent_next[val] = (int32_t)i;
  } else {
    int64_t li = -1 - (int64_t)val;
    if (li < n_leaf) leaf_cell[li] = (int32_t)i;
  }
}

// The base level lmin covers the box, so in Morton order its cells are exactly
// 0 .. 8^lmin - 1: a cell's sorted position is its key, and the leaves and the
// parents of the level lmin+1 octs are placed there directly (no sort).  A
// position taken twice is a duplicate; with the counts checked on the host,
// no duplicate means no gap.  cell_child starts filled with kUnsetCell.
constexpr int32_t kUnsetCell = (int32_t)0x80808080;  // byte 0x80 memset; never a valid entry

__global__ void k_place_complete(int level, int64_t n_leaf, int64_t n_ref, int64_t n_cells,
                                 const int32_t* __restrict__ ijk, const double* __restrict__ mass,
                                 const uint64_t* __restrict__ octkey_next, int32_t* __restrict__ cell_child,
                                 int32_t* __restrict__ leaf_cell, int32_t* __restrict__ oct_parent_next,
                                 unsigned* err) {
  pdl_wait();
  pdl_trigger();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n_leaf + n_ref) return;
  uint64_t key;
  int32_t val;
  if (i < n_leaf) {
    const int x = ijk[3 * i], y = ijk[3 * i + 1], z = ijk[3 * i + 2];
    const int lim = 1 << level;
    if (x < 0 || y < 0 || z < 0 || x >= lim || y >= lim || z >= lim) {
      atomicOr(err, kErrOutOfBox);
      return;
    }
    if (!isfinite(mass[i])) atomicOr(err, kErrNonFinite);
    key = spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
    val = (int32_t)(-1 - i);
    leaf_cell[i] = (int32_t)key;
  } else {
    const int64_t j = i - n_leaf;
    key = octkey_next[j];
    if (key >= (uint64_t)n_cells) {  // only after an invalid finer level (already flagged)
      atomicOr(err, kErrIncomplete);
      return;
    }
    val = (int32_t)j;
    oct_parent_next[j] = (int32_t)key;
  }
  if (atomicExch(cell_child + key, val) != kUnsetCell) atomicOr(err, kErrDuplicate);
}

// The level above a complete base level, without a sort: its octs are the
// refined base cells in Morton order, so marking the parent of every entry
// (leaf or refined cell) in a dense array over the 8^lmin base cells and
// scanning it gives each oct its index; a cell then sits at 8 oct + (key & 7).
// The result is the sorted pass's (same octs, cells, keys and maps).  Entries
// are the level's leaves (i < n_leaf) and its refined cells (the octs of the
// next level, whose keys are their parents' keys).
__device__ __forceinline__ bool dense_key(int64_t i, int level, int64_t n_leaf, const int32_t* __restrict__ ijk,
                                          const uint64_t* __restrict__ octkey_next, uint64_t& key) {
  if (i < n_leaf) {
    const int x = ijk[3 * i], y = ijk[3 * i + 1], z = ijk[3 * i + 2];
    const int lim = 1 << level;
    if (x < 0 || y < 0 || z < 0 || x >= lim || y >= lim || z >= lim) return false;
    key = spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
  } else {
    key = octkey_next[i - n_leaf];
  }
  return true;
}

__global__ void k_dense_mark(int level, int64_t n_leaf, int64_t n_ref, int64_t n_base,
                             const int32_t* __restrict__ ijk, const double* __restrict__ mass,
                             const uint64_t* __restrict__ octkey_next, int32_t* __restrict__ flags, unsigned* err) {
  pdl_wait();
  pdl_trigger();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n_leaf + n_ref) return;
  uint64_t key;
  if (!dense_key(i, level, n_leaf, ijk, octkey_next, key)) {
    atomicOr(err, kErrOutOfBox);
    return;
  }
  if (i < n_leaf && !isfinite(mass[i])) atomicOr(err, kErrNonFinite);
  if ((key >> 3) >= (uint64_t)n_base) {  // only after an invalid finer level
    atomicOr(err, kErrIncomplete);
    return;
  }
  flags[key >> 3] = 1;
}

__global__ void k_dense_place(int level, int64_t n_leaf, int64_t n_ref, int64_t n_base, int64_t n_oct,
                              const int32_t* __restrict__ ijk, const uint64_t* __restrict__ octkey_next,
                              const int32_t* __restrict__ scan, uint64_t* __restrict__ oct_key,
                              int32_t* __restrict__ cell_child, int32_t* __restrict__ leaf_cell,
                              int32_t* __restrict__ oct_parent_next, unsigned* err) {
  pdl_wait();
  pdl_trigger();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i == 0 && scan[n_base - 1] != n_oct) atomicOr(err, kErrIncomplete);  // refined base cells != octs
  if (i >= n_leaf + n_ref) return;
  uint64_t key;
  if (!dense_key(i, level, n_leaf, ijk, octkey_next, key) || (key >> 3) >= (uint64_t)n_base) return;  // flagged
  const int64_t oct = (int64_t)scan[key >> 3] - 1;
  if (oct < 0 || oct >= n_oct) {
    atomicOr(err, kErrIncomplete);
    return;
  }
  const int64_t cell = 8 * oct + (int64_t)(key & 7);
  oct_key[oct] = key >> 3;  // every cell of the oct writes the same key
  const int32_t val = i < n_leaf ? (int32_t)(-1 - i) : (int32_t)(i - n_leaf);
  if (atomicExch(cell_child + cell, val) != kUnsetCell) atomicOr(err, kErrDuplicate);
  if (i < n_leaf)
    leaf_cell[i] = (int32_t)cell;
  else
    oct_parent_next[i - n_leaf] = (int32_t)cell;
}

// Levels 1..lmin (complete grids): oct o of level l sits under cell o of level
// l-1, whose 27 neighbours are found by decoding o's Morton index; levels below
// lmin are fully refined (the child oct of cell c is c).  One thread per oct of
// all these levels; level lmin's cells come from k_place_complete.
struct CompleteLevels {
  int lmin;
  int periodic;  // neighbours wrap around the box
  int64_t oct0[kMaxLevel + 2];  // first oct of level l in the thread index space
  uint64_t* oct_key[kMaxLevel + 1];
  int32_t* oct_parent[kMaxLevel + 1];
  int32_t* cell_child[kMaxLevel + 1];
  int32_t* nbr[kMaxLevel + 1];
};

__device__ __forceinline__ uint32_t compact3(uint64_t x) {  // inverse of spread3
  x &= 0x1249249249249249ull;
  x = (x ^ (x >> 2)) & 0x10C30C30C30C30C3ull;
  x = (x ^ (x >> 4)) & 0x100F00F00F00F00Full;
  x = (x ^ (x >> 8)) & 0x1F0000FF0000FFull;
  x = (x ^ (x >> 16)) & 0x1F00000000FFFFull;
  x = (x ^ (x >> 32)) & 0x1FFFFFull;
  return (uint32_t)x;
}

__global__ void k_complete_levels(const __grid_constant__ CompleteLevels P) {
  pdl_wait();
  pdl_trigger();
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= P.oct0[P.lmin + 1]) return;
  int l = 1;
  while (t >= P.oct0[l + 1]) ++l;
  const int64_t o = t - P.oct0[l];
  const int pl = l - 1;  // level of the parent cell o
  const int px = (int)compact3((uint64_t)o), py = (int)compact3((uint64_t)o >> 1), pz = (int)compact3((uint64_t)o >> 2);
  const int lim = 1 << pl;
  int32_t* nb = P.nbr[l] + o * 27;
  for (int q = 0; q < 27; ++q) {
    int x = px + q % 3 - 1, y = py + (q / 3) % 3 - 1, z = pz + q / 9 - 1;
    if (P.periodic) {  // the image's box (lim is a power of two)
      x &= lim - 1;
      y &= lim - 1;
      z &= lim - 1;
    }
    nb[q] = (x < 0 || y < 0 || z < 0 || x >= lim || y >= lim || z >= lim)
                ? -1
                : (int32_t)(spread3(x) | (spread3(y) << 1) | (spread3(z) << 2));
  }
  P.oct_parent[l][o] = (int32_t)o;
  P.oct_key[l][o] = (uint64_t)o;
  if (l < P.lmin)
    for (int c = 0; c < 8; ++c) P.cell_child[l][o * 8 + c] = (int32_t)(o * 8 + c);
}

// nbr[l][o][q] from the level l-1 tables.  One thread per (oct, q).
__global__ void k_nbr(int level, int64_t n_oct, int64_t n_oct_up, const int32_t* __restrict__ oct_parent,
                      const int32_t* __restrict__ nbr_up, const int32_t* __restrict__ cell_child_up,
                      const int32_t* __restrict__ cell_child_here, int32_t* nbr, unsigned* err) {
  pdl_wait();
  pdl_trigger();
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n_oct * 27) return;
  int64_t o = t / 27;
  int q = (int)(t - o * 27);
  int d[3] = {q % 3 - 1, (q / 3) % 3 - 1, q / 9 - 1};
  int32_t res = -1;
  if (level == 1) {
    res = (q == 13) ? 0 : -1;
  } else {
    int32_t pc = oct_parent[o];
    if (pc < 0 || pc >= 8 * n_oct_up) {  // only after an inconsistent level (already flagged)
      atomicOr(err, kErrIncomplete);
      nbr[t] = -1;
      return;
    }
    int32_t op = pc >> 3;
    int cp = pc & 7;
    int e = 0, newc = 0, mul = 1;
    for (int i = 0; i < 3; ++i) {
      int ex = ((cp >> i) & 1) + d[i];  // -1..2
      int ei = (ex < 0) ? -1 : (ex >> 1);
      e += (ei + 1) * mul;
      mul *= 3;
      newc |= (ex & 1) << i;
    }
    int32_t nb = nbr_up[(int64_t)op * 27 + e];
    if (nb == -1) {
      res = -1;  // outside the unit box
    } else if (nb < -1 || nb >= n_oct_up) {
      // the parent's neighbour at level l-1 does not exist although the parent is
      // refined: its father has an unrefined neighbour (Sec. 3.2)
      atomicOr(err, kErrNotGraded);
      res = -1;
    } else {
      int32_t ncell = nb * 8 + newc;
      int32_t ch = cell_child_up[ncell];
      res = (ch >= 0) ? ch : (-2 - ncell);
    }
  }
  nbr[t] = res;
  // graded rule: a refined cell of this oct needs all in-box neighbours of its father refined
  if (res < -1) {
    bool any_ref = false;
    for (int c = 0; c < 8; ++c) any_ref |= cell_child_here[o * 8 + c] >= 0;
    if (any_ref) atomicOr(err, kErrNotGraded);
  }
}

// ---- row lists of all levels in three launches -------------------------------
// For every oct of every level four flags, all in gather form:
//   rows  (bit 0): the oct holds a refined cell (its M2M output / M2P row);
//   tgt   (bit 1): the oct holds a leaf (a target oct);
//   rowsL (bit 2): a cell of the oct has grandchildren (it needs a local
//                  expansion), levels 1..lmax-2; in bottom mode 1 (M2L + L2P)
//                  a cell of the oct is refined (its children evaluate its local
//                  expansion), levels 1..lmax-1;
//   irows (bit 3): the oct holds a leaf and one of its 3^3 neighbour octs holds
//                  a refined cell (near-field M2P / nearest field), levels
//                  lmin..lmax.
// Blocks of kListBlock octs never straddle levels; k_lists_count counts per
// block, k_lists_scan turns the counts into per-level block offsets and list
// lengths, k_lists_write compacts in ascending oct order.
constexpr int kListBlock = 256;

struct ListLevel {
  int64_t n_oct, n_oct_next;
  int64_t blk0;  // first block of this level
  const int32_t* cell_child;
  const int32_t* cell_child_next;  // level + 1, or null
  const int32_t* nbr;
  int32_t* out[4];  // rows, tgt, rowsL, irows
  uint8_t* leafmask;
  const uint8_t* leafmask_next;  // level + 1 (or null)
  int32_t* slotL;    // [n_oct]: position in rowsL or -1
  // local-expansion rows (k_lslots): lslot[o] = 8 slotL_far[G >> 3] + (G & 7), G the
  // oct's ancestor cell at level l - dl (dl = 2, bottom mode 1: 1), or -1
  const int32_t* oct_parent;     // level l
  const int32_t* oct_parent_up;  // level l - 1 (dl = 2)
  const int32_t* slotL_far;      // slotL of level l - dl, or null (no local expansion)
  int32_t* lslot;
  int64_t n_oct_up, n_oct_far;   // octs of levels l - 1 and l - dl
  int want_rowsL, want_irows;
  int rowsL_refined;  // bottom mode 1: rowsL holds the octs with a refined cell
};

struct ListParams {
  int nlev, level0, stride;
  int64_t n_blocks;
  ListLevel lev[kMaxLevel];
};

__device__ __forceinline__ int list_level(const ListParams& P, int64_t blk) {
  int k = 0;
  while (k + 1 < P.nlev && blk >= P.lev[k + 1].blk0) ++k;
  return k;
}

// Leaf masks of every oct of every level (bit c: cell c is a leaf); an oct
// holds a refined cell iff its mask is not 0xFF.  Read by the list flags below.
__global__ void __launch_bounds__(kListBlock) k_leafmasks(const __grid_constant__ ListParams P) {
  pdl_wait();
  pdl_trigger();
  const int64_t blk = blockIdx.x;
  const ListLevel& L = P.lev[list_level(P, blk)];
  const int64_t o = (blk - L.blk0) * kListBlock + threadIdx.x;
  if (o >= L.n_oct) return;
  int mask = 0;
  for (int c = 0; c < 8; ++c) mask |= (L.cell_child[o * 8 + c] < 0) << c;
  L.leafmask[o] = (uint8_t)mask;
}

// The loops below have no early exit, so each one's loads are issued together
// (one round of child links or neighbour indices, one round of leaf masks).
__device__ __forceinline__ unsigned oct_list_flags(const ListLevel& L, int64_t o) {
  const unsigned mask = L.leafmask[o];
  const int leaf = mask != 0, refined = mask != 0xFFu;
  int grand = 0;
  if (L.want_rowsL && refined && L.rowsL_refined) grand = 1;
  if (L.want_rowsL && refined && !L.rowsL_refined) {
    int32_t ch[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) ch[c] = L.cell_child[o * 8 + c];
#pragma unroll
    for (int c = 0; c < 8; ++c)
      if (ch[c] >= 0 && ch[c] < L.n_oct_next) grand |= L.leafmask_next[ch[c]] != 0xFFu;
  }
  int near_ref = 0;
  if (L.want_irows && leaf) {
    int32_t nb[27];
#pragma unroll
    for (int q = 0; q < 27; ++q) nb[q] = L.nbr[o * 27 + q];
#pragma unroll
    for (int q = 0; q < 27; ++q)
      if (nb[q] >= 0 && nb[q] < L.n_oct) near_ref |= L.leafmask[nb[q]] != 0xFFu;
  }
  return (unsigned)refined | ((unsigned)leaf << 1) | ((unsigned)grand << 2) | ((unsigned)(leaf && near_ref) << 3);
}

__global__ void __launch_bounds__(kListBlock) k_lists_count(const __grid_constant__ ListParams P, uint8_t* __restrict__ flags,
                                                            int32_t* __restrict__ blk_counts) {
  pdl_wait();
  pdl_trigger();
  const int64_t blk = blockIdx.x;
  const ListLevel& L = P.lev[list_level(P, blk)];
  const int64_t o = (blk - L.blk0) * kListBlock + threadIdx.x;
  unsigned f = 0;
  if (o < L.n_oct) {
    f = oct_list_flags(L, o);
    L.slotL[o] = -1;
  }
  flags[blk * kListBlock + threadIdx.x] = (uint8_t)f;
  for (int k = 0; k < 4; ++k) {
    const int n = __syncthreads_count((f >> k) & 1);
    if (threadIdx.x == 0) blk_counts[blk * 4 + k] = n;
  }
}

// One block per (level, list): an exclusive scan of the level's block counts.
__global__ void __launch_bounds__(1024) k_lists_scan(const __grid_constant__ ListParams P,
                                                     const int32_t* __restrict__ blk_counts,
                                                     int32_t* __restrict__ blk_off, int32_t* __restrict__ counts) {
  pdl_wait();
  pdl_trigger();
  __shared__ int32_t warp_sum[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int li = blockIdx.x >> 2, k = blockIdx.x & 3;
  const ListLevel& L = P.lev[li];
  const int64_t nb = (L.n_oct + kListBlock - 1) / kListBlock;
  int32_t carry = 0;
  for (int64_t base = 0; base < nb; base += 1024) {
    const int64_t b = base + threadIdx.x;
    const int32_t v = b < nb ? blk_counts[(L.blk0 + b) * 4 + k] : 0;
    int32_t x = v;  // inclusive warp scan
    for (int d = 1; d < 32; d <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= d) x += y;
    }
    if (lane == 31) warp_sum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int32_t w = warp_sum[lane];
      for (int d = 1; d < 32; d <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, w, d);
        if (lane >= d) w += y;
      }
      warp_sum[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    const int32_t excl = x - v + (warp > 0 ? warp_sum[warp - 1] : 0);
    if (b < nb) blk_off[(L.blk0 + b) * 4 + k] = carry + excl;
    carry += warp_sum[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) counts[k * P.stride + P.level0 + li] = carry;
}

__global__ void __launch_bounds__(kListBlock) k_lists_write(const __grid_constant__ ListParams P, const uint8_t* __restrict__ flags,
                                                            const int32_t* __restrict__ blk_off) {
  pdl_wait();
  pdl_trigger();
  __shared__ int32_t warp_cnt[kListBlock / 32][4];
  const int64_t blk = blockIdx.x;
  const ListLevel& L = P.lev[list_level(P, blk)];
  const int64_t o = (blk - L.blk0) * kListBlock + threadIdx.x;
  const unsigned f = flags[blk * kListBlock + threadIdx.x];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned ball[4];
  for (int k = 0; k < 4; ++k) {
    ball[k] = __ballot_sync(0xffffffffu, (f >> k) & 1);
    if (lane == 0) warp_cnt[warp][k] = __popc(ball[k]);
  }
  __syncthreads();
  if (o >= L.n_oct) return;
  for (int k = 0; k < 4; ++k) {
    if (!((f >> k) & 1)) continue;
    int32_t pos = blk_off[blk * 4 + k] + __popc(ball[k] & ((1u << lane) - 1));
    for (int w = 0; w < warp; ++w) pos += warp_cnt[w][k];
    L.out[k][pos] = (int32_t)o;
    if (k == 2) L.slotL[o] = pos;
  }
}

// The local-expansion row of every oct (the near-field kernel's far field),
// read once per target oct instead of through the parent chain in its loop.
// Runs before the build's errors are read: every link is checked against the
// size of the level it points into, as in the list flags above (an invalid
// hierarchy leaves -1 and is rejected afterwards).
__global__ void __launch_bounds__(kListBlock) k_lslots(const __grid_constant__ ListParams P, int dl) {
  pdl_wait();
  pdl_trigger();
  const int64_t blk = blockIdx.x;
  const ListLevel& L = P.lev[list_level(P, blk)];
  const int64_t o = (blk - L.blk0) * kListBlock + threadIdx.x;
  if (o >= L.n_oct) return;
  int32_t r = -1;
  if (L.slotL_far) {
    const int32_t par = L.oct_parent[o];
    int32_t g = -1;
    if (par >= 0 && par < 8 * L.n_oct_up) g = dl == 1 ? par : L.oct_parent_up[par >> 3];
    if (g >= 0 && g < 8 * L.n_oct_far) {
      const int32_t s = L.slotL_far[g >> 3];
      r = s < 0 ? -1 : 8 * s + (g & 7);
    }
  }
  L.lslot[o] = r;
}

// Ancestor lists of level d: the octs of each level b < d with a descendant
// oct at level d.  Every level-d oct walks up its parent chain; the first
// walker to reach an oct sets its visited flag, appends it to its level's
// list and goes on, later walkers stop there.  Work is proportional to the
// ancestors, not to the octs of the coarser levels.
struct AncParams {
  int d;
  int64_t n_oct[kMaxLevel + 1];
  int64_t flag_off[kMaxLevel + 1];  // byte offset of level b's flags (multiple of 4)
  const int32_t* oct_parent[kMaxLevel + 1];
  int32_t* anc[kMaxLevel + 1];
  uint8_t* flags;
  int32_t* counts;  // [b]: length of level b's list
};

__global__ void k_anc_walk(const __grid_constant__ AncParams A, int64_t n_oct_d) {
  pdl_wait();
  pdl_trigger();
  const int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (o >= n_oct_d) return;
  int32_t cur = (int32_t)o;
  for (int l = A.d; l >= 2; --l) {
    const int32_t up = A.oct_parent[l][cur] >> 3;
    if (up < 0 || up >= A.n_oct[l - 1]) return;
    unsigned int* word = (unsigned int*)(A.flags + A.flag_off[l - 1] + (up & ~3));
    const unsigned int bit = 1u << (8 * (up & 3));
    if (atomicOr(word, bit) & bit) return;
    A.anc[l - 1][atomicAdd(A.counts + (l - 1), 1)] = up;
    cur = up;
  }
}

inline unsigned nblk(int64_t n, int b = 256) { return (unsigned)((n + b - 1) / b); }

#define CK(x)                                                                  \
  do {                                                                         \
    cudaError_t e_ = (x);                                                      \
    if (e_ != cudaSuccess) {                                                   \
      c->last_error = std::string("tree: " #x ": ") + cudaGetErrorString(e_);  \
      return e_ == cudaErrorMemoryAllocation ? FMM_ERR_OOM : FMM_ERR_CUDA;     \
    }                                                                          \
  } while (0)

fmm_status err_to_status(unsigned e) {
  if (e & kErrOutOfBox) return FMM_ERR_OUT_OF_BOX;
  if (e & kErrNonFinite) return FMM_ERR_NONFINITE;
  if (e & kErrDuplicate) return FMM_ERR_DUPLICATE;
  if (e & kErrIncomplete) return FMM_ERR_INCOMPLETE;
  if (e & kErrNotGraded) return FMM_ERR_NOT_GRADED;
  if (e & kErrStructure) return FMM_ERR_STATE;
  if (e & kErrTimeout) return FMM_ERR_TIMEOUT;
  return FMM_OK;
}

}  // namespace

fmm_status tree_prepare(Ctx* c) {
  const int lmin = c->lmin, lmax = c->lmax;
  const int lo = c->tree_lo;  // lmin: full build; above: levels lo..lmax only
  // ---- oct counts from the leaf counts ----------------------------------------
  // An inconsistent count is latched, not returned at once: the device checks
  // below may name the cause (a duplicate, an out-of-box index) more precisely.
  unsigned* host_err = c->tree_host_err;
  for (int l = 0; l <= kMaxLevel; ++l) host_err[l] = 0;
  bool any_host = false;
  const int64_t old_lo_octs = c->lev[lo].n_oct;
  for (int l = lmax; l >= lo; --l) {
    const int64_t n = c->lev[l].n_leaf + ((l < lmax) ? c->lev[l + 1].n_oct : 0);
    if (n == 0 || n > (int64_t)INT32_MAX / 2) {
      c->last_error = "tree: level " + std::to_string(l) + " has no cells or too many";
      return n == 0 ? FMM_ERR_INCOMPLETE : FMM_ERR_ARG;
    }
    if (n % 8) {
      host_err[l] |= kErrIncomplete;
      any_host = true;
    }
    c->lev[l].n_oct = (n + 7) / 8;
  }
  if (lo > lmin) {
    if (c->lev[lo].n_oct != old_lo_octs || any_host) {
      c->last_error = "tree: a partial update (lo = " + std::to_string(lo) +
                      ") must keep the cells of level lo; update from lo - 1 instead";
      c->lev[lo].n_oct = old_lo_octs;
      return FMM_ERR_STATE;
    }
  } else {
    if (c->lev[lmin].n_oct != (int64_t)1 << (3 * (lmin - 1))) host_err[lmin] |= kErrIncomplete;
    for (int l = 1; l < lmin; ++l) {
      c->lev[l].n_oct = (int64_t)1 << (3 * (l - 1));
      c->lev[l].n_leaf = 0;
    }
    c->lev[0].n_oct = 0;
  }
  // ---- size everything ----------------------------------------------------------
  int64_t nmax = 0;
  for (int l = 1; l <= lmax; ++l) {
    LevelTree& T = c->lev[l];
    nmax = std::max<int64_t>(nmax, 8 * T.n_oct);
    CK(buf_ensure(c, T.oct_key, T.n_oct * 8));
    CK(buf_ensure(c, T.oct_parent, T.n_oct * 4));
    CK(buf_ensure(c, T.cell_child, T.n_oct * 32));
    CK(buf_ensure(c, T.leaf_cell, std::max<int64_t>(T.n_leaf, 1) * 4));
    CK(buf_ensure(c, T.nbr, T.n_oct * 27 * 4));
    CK(buf_ensure(c, T.rows, T.n_oct * 4));
    CK(buf_ensure(c, T.tgt, T.n_oct * 4));
    CK(buf_ensure(c, T.rowsL, T.n_oct * 4));
    CK(buf_ensure(c, T.irows, T.n_oct * 4));
    CK(buf_ensure(c, T.leafmask, T.n_oct));
    CK(buf_ensure(c, T.slotL, T.n_oct * 4));
    CK(buf_ensure(c, T.lslot, T.n_oct * 4));
    CK(buf_ensure(c, T.anc, T.n_oct * 4));
  }
  {
    int64_t nf = 4;
    for (int b = 1; b < c->anc_req && b <= lmax; ++b) nf += (c->lev[b].n_oct + 3) & ~(int64_t)3;
    CK(buf_ensure(c, c->anc_flags, nf));
  }
  CK(buf_ensure(c, c->lev[0].cell_child, 32));
  CK(buf_ensure(c, c->keys_a, nmax * 8));
  CK(buf_ensure(c, c->keys_b, nmax * 8));
  CK(buf_ensure(c, c->vals_a, nmax * 4));
  CK(buf_ensure(c, c->vals_b, nmax * 4));
  int64_t list_blocks = 0;
  for (int l = 1; l <= lmax; ++l) list_blocks += (c->lev[l].n_oct + kListBlock - 1) / kListBlock;
  CK(buf_ensure(c, c->flags, std::max<int64_t>(nmax * 8, list_blocks * kListBlock)));
  CK(buf_ensure(c, c->scan, std::max<int64_t>(nmax * 4, list_blocks * 32)));
  CK(buf_ensure(c, c->counter, 5 * 4 * (lmax + 2)));
  // CUB temporary storage for the largest sort and scan of this build.  The size
  // queries are host work repeated on every call, so their answer is kept for
  // as long as the sorted levels and their sizes stay the same.
  std::vector<int64_t> sig = {lo, lmax};
  for (int l = lo; l <= lmax; ++l) sig.push_back(c->lev[l].n_oct);
  if (sig != c->cub_sig) {
    size_t tmp_max = 0;
    for (int l = lo; l <= lmax; ++l) {
      const int n = (int)(8 * c->lev[l].n_oct);
      size_t t = 0;
      CK(cub::DeviceRadixSort::SortPairs(nullptr, t, (uint64_t*)nullptr, (uint64_t*)nullptr, (int32_t*)nullptr,
                                         (int32_t*)nullptr, n, 0, 3 * l));
      tmp_max = std::max(tmp_max, t);
      t = 0;
      CK(cub::DeviceScan::InclusiveSum(nullptr, t, (int32_t*)nullptr, (int32_t*)nullptr, n));
      tmp_max = std::max(tmp_max, t);
    }
    c->cub_sig = sig;
    c->cub_tmp = tmp_max;
  }
  CK(buf_ensure(c, c->sort_tmp, c->cub_tmp));
  return FMM_OK;
}

// All device work of the tree build: stream-ordered, no allocation and no
// synchronisation, so it can be captured in a CUDA graph.
fmm_status tree_enqueue(Ctx* c, cudaStream_t st) {
  const int lmin = c->lmin, lmax = c->lmax;
  const int lo = c->tree_lo;
  const bool partial = lo > lmin;
  unsigned* err0 = c->d_err + 1;  // err0[l]: errors found by the sorted pass of level l
  int32_t* d_counts = (int32_t*)c->counter.ptr;  // [5][lmax+2]: rows, tgt, rowsL, irows, anc
  CK(cudaMemsetAsync(err0, 0, (kErrWords - 1) * sizeof(unsigned), st));
  CK(cudaMemsetAsync(d_counts, 0, 5 * 4 * (lmax + 2), st));
  // ---- bottom-up sorted passes, levels lmax..lo -----------------------------
  // (a full build places the complete base level directly instead of sorting it)
  const bool place_base = !partial && c->lev[lmin].n_oct == (int64_t)1 << (3 * (lmin - 1)) &&
                          (c->lev[lmin].n_leaf + (lmin < lmax ? c->lev[lmin + 1].n_oct : 0)) % 8 == 0;
  for (int l = lmax; l >= lo; --l) {
    LevelTree& T = c->lev[l];
    unsigned* err = err0 + l;
    const int64_t n_ref = (l < lmax) ? c->lev[l + 1].n_oct : 0;
    const int64_t n = T.n_leaf + n_ref;
    int32_t* par_next = (l < lmax) ? (int32_t*)c->lev[l + 1].oct_parent.ptr : nullptr;
    if (l == lmin && place_base) {
      CK(cudaMemsetAsync(T.cell_child.ptr, 0x80, T.n_oct * 32, st));
      ++c->n_launch;
      CK(launch_pdl(k_place_complete, nblk(n), 256, 0, st, l, T.n_leaf, n_ref, 8 * T.n_oct, (const int32_t*)T.ijk.ptr,
                                                (const double*)T.mass.ptr,
                                                n_ref ? (const uint64_t*)c->lev[l + 1].oct_key.ptr : nullptr,
                                                (int32_t*)T.cell_child.ptr, (int32_t*)T.leaf_cell.ptr, par_next, err));
      continue;
    }
    if (l == lmin + 1 && place_base) {  // the octs above the complete base level, unsorted
      const int64_t nbase = 8 * c->lev[lmin].n_oct;
      int32_t* flags = (int32_t*)c->flags.ptr;  // [8^lmin] refined base cells
      int32_t* scan = (int32_t*)c->scan.ptr;
      CK(cudaMemsetAsync(flags, 0, nbase * 4, st));
      CK(cudaMemsetAsync(T.cell_child.ptr, 0x80, T.n_oct * 32, st));
      const uint64_t* okn = n_ref ? (const uint64_t*)c->lev[l + 1].oct_key.ptr : nullptr;
      c->n_launch += 2;
      CK(launch_pdl(k_dense_mark, nblk(n), 256, 0, st, l, T.n_leaf, n_ref, nbase, (const int32_t*)T.ijk.ptr,
                    (const double*)T.mass.ptr, okn, flags, err));
      size_t tmp = c->sort_tmp.bytes;
      ++c->n_cub;
      CK(cub::DeviceScan::InclusiveSum(c->sort_tmp.ptr, tmp, flags, scan, (int)nbase, st));
      CK(launch_pdl(k_dense_place, nblk(n), 256, 0, st, l, T.n_leaf, n_ref, nbase, T.n_oct,
                    (const int32_t*)T.ijk.ptr, okn, (const int32_t*)scan, (uint64_t*)T.oct_key.ptr,
                    (int32_t*)T.cell_child.ptr, (int32_t*)T.leaf_cell.ptr, par_next, err));
      continue;
    }
    uint64_t* ka = (uint64_t*)c->keys_a.ptr;
    uint64_t* kb = (uint64_t*)c->keys_b.ptr;
    int32_t* va = (int32_t*)c->vals_a.ptr;
    int32_t* vb = (int32_t*)c->vals_b.ptr;
    if (T.n_leaf) {
      ++c->n_launch;
      CK(launch_pdl(k_leaf_keys, nblk(T.n_leaf), 256, 0, st, T.n_leaf, (const int32_t*)T.ijk.ptr,
                                                  (const double*)T.mass.ptr, l, ka, va, err));
    }
    if (n_ref) {
      ++c->n_launch;
      CK(launch_pdl(k_refined_keys, nblk(n_ref), 256, 0, st, n_ref, (const uint64_t*)c->lev[l + 1].oct_key.ptr,
                                                  ka + T.n_leaf, va + T.n_leaf));
    }
    size_t tmp = c->sort_tmp.bytes;
    ++c->n_cub;
    CK(cub::DeviceRadixSort::SortPairs(c->sort_tmp.ptr, tmp, ka, kb, va, vb, (int)n, 0, 3 * l, st));
    int32_t* flags = (int32_t*)c->flags.ptr;
    int32_t* scan = (int32_t*)c->scan.ptr;
    ++c->n_launch;
    CK(launch_pdl(k_oct_flags, nblk(n), 256, 0, st, n, kb, flags, err));
    tmp = c->sort_tmp.bytes;
    ++c->n_cub;
    CK(cub::DeviceScan::InclusiveSum(c->sort_tmp.ptr, tmp, flags, scan, (int)n, st));
    ++c->n_launch;
    CK(launch_pdl(k_scatter_level, nblk(n), 256, 0, st, n, T.n_oct, kb, vb, scan, (uint64_t*)T.oct_key.ptr,
                                             (int32_t*)T.cell_child.ptr, (int32_t*)T.leaf_cell.ptr, par_next,
                                             n_ref, T.n_leaf, partial && l == lo, err));
  }
  // ---- complete grids: levels 1..lmin-1, and the parents and neighbours of the
  // level-lmin octs (one launch); the root cell ------------------------------------
  if (!partial) {
    CompleteLevels P{};
    P.lmin = lmin;
    P.periodic = c->cfg.periodic;
    int64_t tot = 0;
    for (int l = 1; l <= lmin; ++l) {
      LevelTree& T = c->lev[l];
      P.oct0[l] = tot;
      tot += T.n_oct;
      P.oct_key[l] = (uint64_t*)T.oct_key.ptr;
      P.oct_parent[l] = (int32_t*)T.oct_parent.ptr;
      P.cell_child[l] = (int32_t*)T.cell_child.ptr;
      P.nbr[l] = (int32_t*)T.nbr.ptr;
    }
    P.oct0[lmin + 1] = tot;
    ++c->n_launch;
    CK(launch_pdl(k_complete_levels, nblk(tot), 256, 0, st, P));
    CK(cudaMemsetAsync(c->lev[0].cell_child.ptr, 0, 4, st));
  }
  // ---- neighbour tables above the complete levels, top-down (levels below lo
  // are unchanged in a partial build) -----------------------------------------------
  for (int l = partial ? lo : lmin + 1; l <= lmax; ++l) {
    LevelTree& T = c->lev[l];
    const int32_t* nbr_up = (const int32_t*)c->lev[l - 1].nbr.ptr;
    const int32_t* cc_up = (const int32_t*)c->lev[l - 1].cell_child.ptr;
    const int64_t n_up = c->lev[l - 1].n_oct;
    ++c->n_launch;
    CK(launch_pdl(k_nbr, nblk(T.n_oct * 27), 256, 0, st, l, T.n_oct, n_up, (const int32_t*)T.oct_parent.ptr, nbr_up, cc_up,
                                              (const int32_t*)T.cell_child.ptr, (int32_t*)T.nbr.ptr,
                                              c->d_err + kErrNbr0 + l));
  }
  // ---- row lists (a partial build changes the lists of levels lo-1..lmax only) ----
  const int list0 = partial ? lo - 1 : 1;
  const int m1 = c->cfg.bottom_mode == FMM_BOTTOM_M2L_L2P;  // local expansions down to level lmax-1
  {
    const int stride = lmax + 2;
    ListParams P{};
    P.nlev = lmax - list0 + 1;
    P.level0 = list0;
    P.stride = stride;
    int64_t nb = 0;
    for (int l = list0; l <= lmax; ++l) {
      LevelTree& T = c->lev[l];
      ListLevel& L = P.lev[l - list0];
      L.n_oct = T.n_oct;
      L.n_oct_next = l < lmax ? c->lev[l + 1].n_oct : 0;
      L.blk0 = nb;
      L.cell_child = (const int32_t*)T.cell_child.ptr;
      L.cell_child_next = l < lmax ? (const int32_t*)c->lev[l + 1].cell_child.ptr : nullptr;
      L.nbr = (const int32_t*)T.nbr.ptr;
      L.out[0] = (int32_t*)T.rows.ptr;
      L.out[1] = (int32_t*)T.tgt.ptr;
      L.out[2] = (int32_t*)T.rowsL.ptr;
      L.out[3] = (int32_t*)T.irows.ptr;
      L.leafmask = (uint8_t*)T.leafmask.ptr;
      L.leafmask_next = l < lmax ? (const uint8_t*)c->lev[l + 1].leafmask.ptr : nullptr;
      L.slotL = (int32_t*)T.slotL.ptr;
      L.want_rowsL = l + 2 - m1 <= lmax;
      L.rowsL_refined = m1;
      L.want_irows = l >= lmin;
      L.oct_parent = (const int32_t*)T.oct_parent.ptr;
      L.oct_parent_up = l >= 2 ? (const int32_t*)c->lev[l - 1].oct_parent.ptr : nullptr;
      L.slotL_far = l - (2 - m1) >= first_local_level(c) ? (const int32_t*)c->lev[l - (2 - m1)].slotL.ptr : nullptr;
      L.lslot = (int32_t*)T.lslot.ptr;
      L.n_oct_up = l >= 2 ? c->lev[l - 1].n_oct : 0;
      L.n_oct_far = l - (2 - m1) >= 1 ? c->lev[l - (2 - m1)].n_oct : 0;
      nb += (T.n_oct + kListBlock - 1) / kListBlock;
    }
    P.n_blocks = nb;
    uint8_t* fl = (uint8_t*)c->flags.ptr;            // nb * kListBlock bytes
    int32_t* blk_counts = (int32_t*)c->scan.ptr;     // nb * 4
    int32_t* blk_off = blk_counts + nb * 4;          // nb * 4
    c->n_launch += 5;
    CK(launch_pdl(k_leafmasks, (unsigned)nb, kListBlock, 0, st, P));
    CK(launch_pdl(k_lists_count, (unsigned)nb, kListBlock, 0, st, P, fl, blk_counts));
    CK(launch_pdl(k_lists_scan, (unsigned)(4 * P.nlev), 1024, 0, st, P, blk_counts, blk_off, d_counts));
    CK(launch_pdl(k_lists_write, (unsigned)nb, kListBlock, 0, st, P, fl, blk_off));
    CK(launch_pdl(k_lslots, (unsigned)nb, kListBlock, 0, st, P, 2 - m1));
  }
  // ---- ancestor lists of level anc_req (incremental solves) ------------------------
  const int d = c->anc_req;
  if (d > lmin && d <= lmax) {
    AncParams A{};
    A.d = d;
    int64_t off = 0;
    for (int b = 1; b < d; ++b) {
      LevelTree& B = c->lev[b];
      A.flag_off[b] = off;
      A.n_oct[b] = B.n_oct;
      off += (B.n_oct + 3) & ~(int64_t)3;  // 4-byte aligned: the walk sets flags with word atomics
      A.oct_parent[b + 1] = (const int32_t*)c->lev[b + 1].oct_parent.ptr;
      A.anc[b] = (int32_t*)B.anc.ptr;
    }
    A.flags = (uint8_t*)c->anc_flags.ptr;
    A.counts = d_counts + 4 * (lmax + 2);
    CK(cudaMemsetAsync(A.flags, 0, off, st));
    ++c->n_launch;
    CK(launch_pdl(k_anc_walk, nblk(c->lev[d].n_oct), 256, 0, st, A, c->lev[d].n_oct));
  }
  return FMM_OK;
}

// The one synchronisation of a tree build: error words and list lengths.  An
// invalid level also corrupts the levels above it (their keys come from its
// octs), so the finest level with an error names the cause; errors of the
// sorted passes come before those of the neighbour stage, which reads their
// output.
fmm_status tree_finish(Ctx* c, cudaStream_t st) {
  const int lmin = c->lmin, lmax = c->lmax;
  const int stride = lmax + 2;
  int32_t* d_counts = (int32_t*)c->counter.ptr;
  // both into the context's pinned buffer: asynchronous copies, one synchronisation
  int32_t* counts = (int32_t*)c->h_rb;
  const unsigned* ev = (const unsigned*)(c->h_rb + (size_t)5 * 4 * (kMaxLevel + 2));
  CK(cudaMemcpyAsync(counts, d_counts, 5 * 4 * stride, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync((void*)ev, c->d_err, kErrWords * 4, cudaMemcpyDeviceToHost, st));
  // The calling thread polls instead of blocking: a thread that sleeps in the
  // wait can take far longer to wake than the build takes (a descheduled
  // virtual CPU), and the device idles meanwhile.  Long waits fall back to a
  // blocking wait after 20 ms.
  CK(cudaEventRecord(c->ev_sync, st));
  {
    const auto t0 = std::chrono::steady_clock::now();
    cudaError_t q;
    while ((q = cudaEventQuery(c->ev_sync)) == cudaErrorNotReady) {
      if (std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(20)) {
        q = cudaEventSynchronize(c->ev_sync);
        break;
      }
    }
    CK(q);
  }
  for (int group = 0; group < 2; ++group) {
    for (int l = lmax; l >= 1; --l) {
      const unsigned e = group == 0 ? ev[1 + l] | c->tree_host_err[l] : ev[kErrNbr0 + l];
      const fmm_status s = err_to_status(e);
      if (s != FMM_OK) {
        c->last_error = (e & kErrStructure)
                            ? "tree: a partial update changed the cells of its lowest level; update from one level coarser"
                            : "tree: invalid hierarchy at level " + std::to_string(l) + " (error bits " +
                                  std::to_string(e) + ")";
        return s;
      }
    }
  }
  const int list0 = c->tree_lo > lmin ? c->tree_lo - 1 : 1;  // the levels whose lists were rebuilt
  const int m1 = c->cfg.bottom_mode == FMM_BOTTOM_M2L_L2P;
  for (int l = 1; l <= lmax; ++l) {
    LevelTree& T = c->lev[l];
    if (l >= list0) {
      T.n_rows = counts[0 * stride + l];
      T.n_tgt = counts[1 * stride + l];
      T.n_rowsL = (l + 2 - m1 <= lmax) ? counts[2 * stride + l] : 0;
      T.n_irows = (l >= lmin) ? counts[3 * stride + l] : 0;
    }
    T.n_anc = (l < c->anc_req) ? counts[4 * stride + l] : 0;
  }
  return FMM_OK;
}

}  // namespace fmm
