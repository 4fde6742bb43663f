// static_solve.cu -- a complete solve of a small unigrid that allocates no
// device memory.
//
// Some callers cannot call cudaMalloc while they run: host codes whose
// device memory is owned by another allocator (for example one that reserves
// the whole GPU at start-up) or loops that must not allocate after their
// initialisation.  fmm_solve_unigrid_static serves them for unigrids of up to
// 16^3 cells: every per-hierarchy array the solve needs (tree index,
// multipoles, local expansions, M2P sums) is carved out of one file-scope
// static device array of kStaticBytes, and the kernels are the library's own,
// launched on a view of that array.  Only the translation tables come from
// the context, which allocated them when it was created.
//
// The array's name is a host-side stand-in in host code; its device address
// is looked up once per device with cudaGetSymbolAddress, by the first call
// on that device (make that first call before any stream capture).  Every
// call shares the array and it keeps the last call's contents; the tree view
// is rewritten and the sums that accumulate are cleared on every call, and
// calls that overlap on the GPU race with each other.
#include <cstring>

#include "fmm_internal.cuh"

namespace fmm {
namespace {

constexpr size_t kStaticBytes = (size_t)2 << 20;  // 2 MiB, held by every device that loads the library
constexpr int kStaticMaxLevel = 4;                // 16^3 cells
constexpr int kStaticMaxP = 6;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

void* g_scratch_dev[64] = {};  // device address of g_static_scratch per device ordinal

__device__ __forceinline__ uint32_t morton3(uint32_t x, uint32_t y, uint32_t z, int bits) {
  uint32_t k = 0;
  for (int b = 0; b < bits; ++b)
    k |= (((x >> b) & 1u) << (3 * b)) | (((y >> b) & 1u) << (3 * b + 1)) | (((z >> b) & 1u) << (3 * b + 2));
  return k;
}

struct UnigridView {
  int32_t* cell_child[kStaticMaxLevel + 1];
  int32_t* oct_parent[kStaticMaxLevel + 1];
  int32_t* nbr[kStaticMaxLevel + 1];
  int32_t* iota;
  uint8_t* leafmask;  // finest level: every cell a leaf
  int32_t* lslot;     // finest level: local-expansion row of each oct's level L-2 grandparent cell
  unsigned* status;
  int level;
};

// The tree index of a complete grid is analytic: cells and octs sorted by
// Morton key have ids equal to their keys, every cell above the finest level
// is refined, and neighbours are found from coordinates.
__global__ void k_unigrid_tree(UnigridView V) {
  const int L = V.level;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i == 0) *V.status = 0u;
  for (int k = 0; k <= L; ++k) {
    const int64_t ncell = (int64_t)1 << (3 * k);
    const int64_t noct = k ? ((int64_t)1 << (3 * (k - 1))) : 0;
    if (i < ncell) V.cell_child[k][i] = (k < L) ? (int32_t)i : INT32_MIN;  // finest level: filled by the leaves
    if (k >= 1 && i < noct) {
      V.oct_parent[k][i] = (int32_t)i;
      uint32_t x = 0, y = 0, z = 0;  // coordinates of the parent cell (level k-1)
      for (int b = 0; b < k - 1; ++b) {
        x |= ((uint32_t)(i >> (3 * b)) & 1u) << b;
        y |= ((uint32_t)(i >> (3 * b + 1)) & 1u) << b;
        z |= ((uint32_t)(i >> (3 * b + 2)) & 1u) << b;
      }
      const int n = 1 << (k - 1);
      for (int q = 0; q < 27; ++q) {
        const int nx = (int)x + q % 3 - 1, ny = (int)y + (q / 3) % 3 - 1, nz = (int)z + q / 9 - 1;
        const bool in = nx >= 0 && ny >= 0 && nz >= 0 && nx < n && ny < n && nz < n;
        V.nbr[k][i * 27 + q] = in ? (int32_t)morton3(nx, ny, nz, k - 1) : -1;
      }
    }
  }
  if (i < ((int64_t)1 << (3 * (L - 1)))) {
    V.iota[i] = (int32_t)i;
    V.leafmask[i] = 0xFFu;
    // oct i's parent cell is cell i of level L-1, whose parent is cell i >> 3 of
    // level L-2; with one slot per oct (slotL = iota) that cell's row is i >> 3
    V.lslot[i] = L - 2 >= 2 ? (int32_t)(i >> 3) : -1;
  }
}

// Each input cell claims its slot of the finest level; a slot claimed twice or
// a cell outside the box is reported through the status word.
__global__ void k_unigrid_leaves(UnigridView V, int64_t n, const int32_t* __restrict__ ijk,
                                 const double* __restrict__ mass) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int L = V.level, lim = 1 << L;
  const int x = ijk[3 * i], y = ijk[3 * i + 1], z = ijk[3 * i + 2];
  if (x < 0 || y < 0 || z < 0 || x >= lim || y >= lim || z >= lim) {
    atomicOr(V.status, kErrOutOfBox);
    return;
  }
  if (!isfinite(mass[i])) atomicOr(V.status, kErrNonFinite);
  const uint32_t key = morton3(x, y, z, L);
  if (atomicCAS(&V.cell_child[L][key], INT32_MIN, (int32_t)(-1 - i)) != INT32_MIN) atomicOr(V.status, kErrDuplicate);
}

// Bump allocator over the static array (256-byte aligned pieces).
struct Carve {
  unsigned char* base;
  size_t off = 0;
  void* take(size_t bytes) {
    void* p = base + off;
    off += (bytes + 255) / 256 * 256;
    return p;
  }
};

void set_buf(DevBuf& b, void* p, size_t bytes) {
  b.ptr = p;
  b.bytes = bytes;
}

}  // namespace
}  // namespace fmm

using namespace fmm;

extern "C" fmm_status fmm_solve_unigrid_static(fmm_ctx* cx, int level, int64_t n, const int32_t* ijk,
                                               const double* mass, void* phi, void* accel, void* stream) {
  Ctx* c = reinterpret_cast<Ctx*>(cx);
  if (!c) return FMM_ERR_ARG;
  if (!ijk || !mass || !phi || !accel) {
    c->last_error = "fmm_solve_unigrid_static: a NULL pointer";
    return FMM_ERR_ARG;
  }
  if (level < 2 || level > kStaticMaxLevel) {
    c->last_error = "fmm_solve_unigrid_static: level must be 2..4 (at most 16^3 cells)";
    return FMM_ERR_ARG;
  }
  if (n != ((int64_t)1 << (3 * level))) {
    c->last_error = "fmm_solve_unigrid_static: n must be 8^level (every cell of the grid once)";
    return FMM_ERR_ARG;
  }
  if (c->cfg.bottom_mode != FMM_BOTTOM_M2P || c->cfg.precision == FMM_MIXED_TF32 || c->cfg.delta_l == 2 ||
      c->cfg.periodic) {
    c->last_error = "fmm_solve_unigrid_static: needs the bottom M2P mode, delta_l = 1 and FP64 or split-BF16 precision";
    return FMM_ERR_ARG;
  }
  if (c->cfg.p > kStaticMaxP) {
    c->last_error = "fmm_solve_unigrid_static: expansion order above 6 needs more than the static scratch";
    return FMM_ERR_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    c->last_error = "fmm_solve_unigrid_static: no current CUDA device";
    return FMM_ERR_CUDA;
  }
  if (dev != c->device) {  // the context's tables live on its own device
    c->last_error = "fmm_solve_unigrid_static: the current device is not the context's device";
    return FMM_ERR_ARG;
  }
  // the kernels read and write these directly: a host pointer would be an illegal access
  if (!is_device_ptr(ijk) || !is_device_ptr(mass) || !is_device_ptr(phi) || !is_device_ptr(accel)) {
    c->last_error = "fmm_solve_unigrid_static: ijk, mass, phi and accel must be device pointers";
    return FMM_ERR_ARG;
  }
  if (!g_scratch_dev[dev]) {  // once per device, with that device current
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      c->last_error = std::string("fmm_solve_unigrid_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      cudaGetLastError();
      return FMM_ERR_CUDA;
    }
    g_scratch_dev[dev] = p;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int L = level, nc = c->tab.nc;
  const bool f64 = c->cfg.precision == FMM_FP64;

  // ---- carve the view; levels 0..L of a complete grid ----
  Carve cv{(unsigned char*)g_scratch_dev[dev]};
  UnigridView V;
  std::memset(&V, 0, sizeof(V));
  V.level = L;
  LevelTree view[kStaticMaxLevel + 1];
  for (int k = 0; k <= L; ++k) {
    LevelTree& T = view[k];
    T = LevelTree();
    const int64_t ncell = (int64_t)1 << (3 * k);
    const int64_t noct = k ? ncell / 8 : 0;
    T.n_oct = noct;
    T.n_leaf = (k == L) ? n : 0;
    T.n_rows = (k >= 1 && k < L) ? noct : 0;
    T.n_tgt = (k == L) ? noct : 0;
    T.n_rowsL = (k >= 1 && k + 2 <= L) ? noct : 0;
    T.m_is_f64 = true;  // levels <= 4: FP64 multipoles in both precisions
    V.cell_child[k] = (int32_t*)cv.take(ncell * 4);
    set_buf(T.cell_child, V.cell_child[k], ncell * 4);
    if (k >= 1) {
      V.oct_parent[k] = (int32_t*)cv.take(noct * 4);
      V.nbr[k] = (int32_t*)cv.take(noct * 27 * 4);
      set_buf(T.oct_parent, V.oct_parent[k], noct * 4);
      set_buf(T.nbr, V.nbr[k], noct * 27 * 4);
      set_buf(T.mono, cv.take(ncell * 8), ncell * 8);
    }
    if (k >= 1 && k < L) {
      set_buf(T.M, cv.take(ncell * nc * 8), ncell * nc * 8);
      if (!f64) {
        set_buf(T.Mhi, cv.take(ncell * nc * 2), ncell * nc * 2);
        set_buf(T.Mlo, cv.take(ncell * nc * 2), ncell * nc * 2);
      }
    }
    if (k >= 2 && k + 2 <= L) {
      set_buf(T.L, cv.take(ncell * nc * 8), ncell * nc * 8);
      if (!f64) {
        set_buf(T.Lm, cv.take(ncell * nc * 4), ncell * nc * 4);
        set_buf(T.Lf, cv.take(ncell * nc * 4), ncell * nc * 4);  // FP32 copy for the near field
      }
    }
    if (k == L) {
      set_buf(T.acc, cv.take(ncell * 4 * (f64 ? 8 : 4)), ncell * 4 * (f64 ? 8 : 4));
      set_buf(T.mass, (void*)mass, n * 8);
    }
  }
  V.iota = (int32_t*)cv.take(((int64_t)1 << (3 * (L - 1))) * 4);
  V.leafmask = (uint8_t*)cv.take((int64_t)1 << (3 * (L - 1)));
  V.lslot = (int32_t*)cv.take(((int64_t)1 << (3 * (L - 1))) * 4);
  V.status = (unsigned*)cv.take(256);
  if (cv.off > kStaticBytes) {
    c->last_error = "fmm_solve_unigrid_static: static scratch too small for this order";
    return FMM_ERR_ARG;
  }
  for (int k = 1; k <= L; ++k) {
    LevelTree& T = view[k];
    set_buf(T.rows, V.iota, T.n_oct * 4);
    set_buf(T.rowsL, V.iota, T.n_oct * 4);
    set_buf(T.slotL, V.iota, T.n_oct * 4);  // every oct of a complete grid has its own slot
    set_buf(T.tgt, V.iota, T.n_oct * 4);
  }
  // the near-field kernel reads these two tables of the target level
  set_buf(view[L].leafmask, V.leafmask, view[L].n_oct);
  set_buf(view[L].lslot, V.lslot, view[L].n_oct * 4);

  // ---- tree index and leaves ----
  const int64_t nmax = (int64_t)1 << (3 * L);
  k_unigrid_tree<<<(unsigned)((nmax + 255) / 256), 256, 0, st>>>(V);
  k_unigrid_leaves<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(V, n, ijk, mass);
  c->n_launch += 2;
  unsigned status = 0;
  cudaError_t e = cudaMemcpyAsync(&status, V.status, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    c->last_error = std::string("fmm_solve_unigrid_static: ") + cudaGetErrorString(e);
    return FMM_ERR_CUDA;
  }
  if (status & kErrOutOfBox) {
    c->last_error = "fmm_solve_unigrid_static: a cell index outside [0, 2^level)";
    return FMM_ERR_OUT_OF_BOX;
  }
  if (status & kErrNonFinite) {
    c->last_error = "fmm_solve_unigrid_static: a mass is NaN or infinite";
    return FMM_ERR_NONFINITE;
  }
  if (status & kErrDuplicate) {
    c->last_error = "fmm_solve_unigrid_static: a cell given twice";
    return FMM_ERR_DUPLICATE;
  }

  // ---- the solve, on the view (the context's own hierarchy is put back after) ----
  LevelTree saved[kStaticMaxLevel + 1];
  for (int k = 0; k <= L; ++k) saved[k] = c->lev[k];
  const int s_lmin = c->lmin, s_lmax = c->lmax;
  for (int k = 0; k <= L; ++k) c->lev[k] = view[k];
  c->lmin = c->lmax = L;
  launch_mono_leaves(c, L, st);
  for (int b = L - 1; b >= 1; --b) launch_upward(c, b, st);
  if (L - 2 >= 2) {
    if (f64) {
      launch_l2l_add(c, 2, st);
      launch_gemm_f64(c, c->op_m2l, kModeM2L, 2, st);
    } else {
      cudaMemsetAsync(c->lev[2].Lm.ptr, 0, c->lev[2].Lm.bytes, st);
      const int lv = 2;
      launch_gemm_tc(c, c->op_m2l, kModeM2L, &lv, 1, st);
      launch_l2l_add(c, 2, st);
    }
  }
  cudaMemsetAsync(c->lev[L].acc.ptr, 0, c->lev[L].acc.bytes, st);
  if (f64) {
    launch_gemm_f64(c, c->op_m2p, kModeM2P, L - 1, st);
  } else {
    const int lv = L - 1;
    launch_gemm_tc(c, c->op_m2p, kModeM2P, &lv, 1, st);
  }
  void* pp[1] = {phi};
  void* pa[1] = {accel};
  launch_near(c, L, pp, pa, c->cfg.out_fp32, st);
  for (int k = 0; k <= L; ++k) c->lev[k] = saved[k];
  c->lmin = s_lmin;
  c->lmax = s_lmax;
  c->last_stream = st;
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    c->last_error = std::string("fmm_solve_unigrid_static: ") + cudaGetErrorString(e);
    return FMM_ERR_CUDA;
  }
  return FMM_OK;
}
