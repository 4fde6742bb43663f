// fmm_internal.cuh -- shared declarations of the CUDA library.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/fmm.h"
#include "tables.h"

namespace fmm {

constexpr int kMaxLevel = 20;

// Error bits latched by kernels (atomicOr into DeviceState::err).
enum : unsigned {
  kErrOutOfBox = 1u,
  kErrDuplicate = 2u,
  kErrNotGraded = 4u,
  kErrIncomplete = 8u,
  kErrNonFinite = 16u,
  kErrTimeout = 32u,
  kErrStructure = 64u,  // a partial update changed the cells of its lowest level
};
// Device error words: [0] solves (timeouts), [1 + l] the sorted pass of level l,
// [kErrNbr0 + l] the neighbour tables of level l.  The sorted passes see the
// input itself; the neighbour stage reads the links the passes wrote, so its
// words name the cause only when every pass was clean.  Within each group the
// finest level with an error names the cause (errors propagate upwards).
constexpr int kErrNbr0 = kMaxLevel + 2;
constexpr int kErrWords = kErrNbr0 + kMaxLevel + 1;

// Programmatic dependent launch: kernels launched with launch_pdl may start
// while the previous kernel on the stream drains; each one waits for it
// (griddepcontrol.wait) before touching memory it produced, and lets its own
// successor start early.  Both instructions are no-ops in a normal launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Sign of prod_{i: e_i = 1} s_i for child c, s_i = +1 if bit i of c is set
// (child in the upper half along axis i) else -1.
__host__ __device__ inline int child_sign(int c, int e) {
  return (__builtin_popcount(e & ~c & 7) & 1) ? -1 : 1;
}

// One coefficient of a contraction operand row: split-BF16 (hi + lo) for the
// kind::f16 contraction, or, when lo is null (TF32 precision), the value
// rounded to nearest TF32 (10 mantissa bits) and stored as FP32 in hi's
// buffer, which then holds 4 bytes per coefficient.
// Index of coefficient k of a cell in the contraction operand rows.  An oct's
// eight cells form one row of 8 nc values, ordered (alpha, cell): the
// coefficients of degree <= q then come first, 8 ncoef(q) of them, so an
// output column that only reads those (M2L keeps |alpha| + |beta| <= p, Eq. 3)
// needs a prefix of every row.
__host__ __device__ __forceinline__ int64_t op_index(int64_t cell, int k, int nc) {
  return (cell >> 3) * 8 * nc + (int64_t)k * 8 + (cell & 7);
}

template <typename T>
__device__ __forceinline__ void put_operand(T v, __nv_bfloat16* hi, __nv_bfloat16* lo, int64_t i) {
  const float f = (float)v;
  if (lo) {
    const __nv_bfloat16 h = __float2bfloat16_rn(f);
    hi[i] = h;
    lo[i] = __float2bfloat16_rn(f - __bfloat162float(h));
  } else {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(f));
    reinterpret_cast<float*>(hi)[i] = __uint_as_float(r);
  }
}

// A grow-only device allocation.
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

struct Ctx;
cudaError_t buf_ensure(Ctx* c, DevBuf& b, size_t bytes);
// true for device (or managed) memory; cudaPointerGetAttributes allocates nothing
bool is_device_ptr(const void* p);

// Device-resident tree of one level.
struct LevelTree {
  int64_t n_oct = 0;     // octs of this level (level 0: 0; its single cell is the root)
  int64_t n_leaf = 0;    // input leaves of this level
  int64_t n_rows = 0;    // octs holding at least one refined cell
  int64_t n_tgt = 0;     // octs holding at least one leaf cell
  int64_t n_rowsL = 0;   // octs holding a cell with grandchildren (need a local expansion)
  int64_t n_irows = 0;   // target octs with a refined cell among their 3^3 neighbour octs
  DevBuf oct_key;        // uint64 [n_oct]
  DevBuf oct_parent;     // int32 [n_oct] cell id at level-1
  DevBuf cell_child;     // int32 [8 n_oct]: >=0 child oct at level+1, else -1-leaf index
  DevBuf nbr;            // int32 [n_oct][27]
  DevBuf leaf_cell;      // int32 [n_leaf]
  DevBuf rows;           // int32 [n_rows]
  DevBuf tgt;            // int32 [n_tgt]
  DevBuf rowsL;          // int32 [n_rowsL]
  DevBuf irows;          // int32 [n_irows]
  DevBuf leafmask;       // uint8 [n_oct]: bit c set when cell c of the oct is a leaf
  DevBuf slotL;          // int32 [n_oct]: position of the oct in rowsL (its local-expansion
                         // slot), -1 if it has none
  DevBuf lslot;          // int32 [n_oct]: row of the local expansion the oct's cells evaluate
                         // (8 slotL + cell of their level l-2 grandparent cell; bottom mode 1:
                         // of their parent cell, level l-1), -1 where that level is below 2
  // adjoint (FP64): mass cotangents and the octs read by the contractions
  DevBuf gmass;          // double [n_leaf]
  DevBuf srcP, srcL;     // int32: octs read by M2P rows / by M2L rows of this level
  int64_t n_srcP = 0, n_srcL = 0;
  // incremental solves: octs with a descendant at level Ctx::anc_d (ancestor lists)
  DevBuf anc;           // int32 [n_anc]
  int64_t n_anc = 0;
  // inputs kept for adaptive time stepping (replaced by set_levels)
  DevBuf ijk;            // int32 [n_leaf][3]
  DevBuf mass;           // double [n_leaf]
  DevBuf vel;            // double [n_leaf][3] velocities (multipole drifting), input order
  bool vel_valid = false;
  // multipole drifting scratch: one stale tree's multipoles and (mass, momentum)
  // per cell of this level, FP64 box units
  DevBuf dS, dQ;
  // expansions (box units)
  DevBuf M;              // [8 n_oct][nc] double (FP64 path / top levels) or float; rows of
                         // refined cells and of the leaves in interface octs (irows)
  DevBuf Mhi, Mlo;       // bf16 [8 n_oct][nc] (mixed path GEMM operands)
  DevBuf mono;           // [8 n_oct] total mass per cell (double or float)
  DevBuf L;              // double [8 n_rowsL][nc] local expansions (levels 2..lmax-2, or
                         // 2..lmax-1 in bottom mode 1), by slot
  DevBuf Lf;             // float [8 n_rowsL][nc] FP32 copy of L read by the mixed near field
  DevBuf Lm;             // float [8 n_rowsL][nc] this level's M2L sum (mixed path), by slot;
                         // zero between solves (the L2L step clears what it consumes)
  DevBuf Chi, Clo;       // Delta l = 2, level lmax-1: the 8 child masses of each cell as
                         // contraction operand rows (bf16 hi/lo by op_index with nc = 8;
                         // TF32: FP32 in Chi; FP64: double [cell][8] in Chi)
  DevBuf acc;            // [8 n_oct][4] M2P result (double or float), targets of this level;
                         // mixed path: zero between solves (the near field clears what it reads)
  bool m_is_f64 = true;
};

constexpr int kTopLevelFP64 = 3;  // mixed precisions with fp64_top: box levels <= 3 use FP64 M2M
constexpr int kTcBK = 32;  // K slice of the tensor-core contraction (elements per operand row per stage)

struct GemmOperand {  // one operator for the GEMM kernels
  int N = 0, K = 0;     // logical sizes
  int Npad = 0, Kpad = 0, BN = 0, ntile = 0;
  DevBuf f64;           // FP64 [K][N] (N fastest) for the DFMA kernel
  DevBuf hi, lo;        // bf16 [Npad][Kpad] (K fastest) for tcgen05
  alignas(64) unsigned char tmap_hi[128];
  alignas(64) unsigned char tmap_lo[128];
  DevBuf klimit;        // int32 [N]: K entries per 26-offset segment to visit (FP64 kernel)
  int kseg = 0;         // entries per offset segment (8*nc)
  // tensor-core layout: K ordered (q, alpha, s), each offset segment padded to
  // kqp (a multiple of kTcBK); columns of N tile y read only the first
  // tile_slices[y] slices of every segment (the coefficients they keep)
  int kqp = 0;
  std::vector<int> tile_slices;
  DevBuf colmap;        // M2L, int32 [8 nc]: column (position in a slot's M2L sums) of (cell s, beta) at s nc + beta
};

struct Ctx {
  fmm_config cfg{};
  Tables tab;
  int lmin = -1, lmax = -1;  // lmax: the finest level that holds cells
  int lmax_user = -1;        // the caller's lmax (levels above lmax are empty)
  bool have_levels = false;
  LevelTree lev[kMaxLevel + 1];
  // device tables
  DevBuf d_m2m_off, d_m2m_g, d_m2m_e, d_m2m_c, d_m2m_c32;
  DevBuf d_m2m_w0, d_m2m_w0_32, d_m2m_e0;  // per alpha: the gamma = 0 pair (leaf-only octs)
  DevBuf d_l2l_off, d_l2l_off8, d_l2l_g, d_l2l_e, d_l2l_c, d_l2l_c32;
  DevBuf d_near64, d_near32, d_l2p64, d_l2p32;
  GemmOperand op_m2p, op_m2l;
  GemmOperand op_m2p2, op_p2pr;  // Delta l = 2: M2P from level l-2, P2P ring from level l-1
  DevBuf d_lat64, d_lat32;       // periodic: the level-1 lattice operator [8 nc][8 nc]
  // scratch
  DevBuf sort_tmp, keys_a, keys_b, vals_a, vals_b, flags, scan, err_word, counter;
  DevBuf anc_flags;     // uint8: one visited flag per oct of levels 1..anc_req-1 (ancestor walks)
  std::vector<int64_t> cub_sig;  // sorted levels and their sizes of the last CUB size query
  size_t cub_tmp = 0;            // and its answer (bytes of sort_tmp needed)
  DevBuf out_stage;     // device staging for host outputs
  DevBuf in_stage;      // device staging for host inputs
  DevBuf mass_stage;    // FP32 masses (config.mass_fp32) on their way to the FP64 copies
  DevBuf err_buf;       // the device error words (d_err points into it)
  // pinned host copy of the tree build's list lengths and error words (one
  // synchronisation per build reads them back)
  static constexpr size_t kReadbackBytes = (size_t)5 * 4 * (kMaxLevel + 2) + (size_t)4 * kErrWords;
  unsigned char* h_rb = nullptr;
  unsigned* d_err = nullptr;
  // the caller's allocator (null: cudaMalloc / cudaFree)
  fmm_alloc_fn alloc = nullptr;
  void* alloc_user = nullptr;
  double wait_s = 2.0;  // limit of every bounded device-side wait (fmm_set_wait_limit)
  // multipole drifting: dt per level lmin.. (empty: off), the multi-index
  // components of each coefficient on the device
  std::vector<double> drift_dt;
  DevBuf d_alpha;
  size_t bytes_in_use = 0;
  std::string last_error;
  cudaStream_t last_stream = nullptr;
  int device = 0;
  int num_sms = 148;
  bool timing = false;
  cudaEvent_t ev[6] = {};
  double stage_ms[5] = {0, 0, 0, 0, 0};  // upward, downward, m2p, near-field M2P, near field
  bool tables_on_device = false;
  int64_t n_launch = 0, n_cub = 0, n_solve = 0, n_set = 0;
  // CUDA graphs of fmm_solve's device work, keyed by (layout generation, lo,
  // output pointers).  The generation changes whenever a buffer is reallocated
  // or the tree's list lengths change, so a cached graph never sees stale
  // pointers or grid sizes.
  struct SolveGraph {
    std::vector<uintptr_t> key;
    cudaGraphExec_t exec = nullptr;
    int64_t launches = 0;   // kernels of this library in the graph
    int64_t cub_calls = 0;  // CUB primitives in the graph
  };
  std::vector<SolveGraph> graphs;
  std::vector<SolveGraph> tree_graphs;
  // adjoint: transposed pair lists and operators (built on first use), and the
  // layout generation the source lists were built for
  DevBuf d_m2mT_off, d_m2mT_a, d_m2mT_c, d_l2lT_off, d_l2lT_b, d_l2lT_e, d_l2lT_c, d_m2pT, d_m2lT;
  bool adj_tables = false;
  uint64_t adj_gen = 0;  // tree build + clearing, keyed by layout and leaf counts
  unsigned tree_host_err[kMaxLevel + 1] = {};
  // Incremental updates (adaptive time stepping).  tree_lo: lowest level the
  // current tree build re-sorts (lmin: all).  dirty_lo: lowest level whose
  // masses or cells changed since the last upward pass (kClean: none).  anc_d:
  // the level whose ancestor lists exist (0: none); anc_req: requested of the
  // tree build in progress.
  static constexpr int kClean = 1 << 20;
  int tree_lo = 0;
  int dirty_lo = kClean;
  int anc_d = 0, anc_req = 0;
  uint64_t layout_gen = 1;
  std::vector<int64_t> count_sig;
  cudaStream_t cap_stream = nullptr;
  // second branch of a solve: the bottom M2P needs only the multipoles, so it
  // runs beside the downward pass (fork after the upward pass, join before
  // the near field)
  cudaStream_t aux_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_sync = nullptr;  // the tree build's one synchronisation (polled, see tree_finish)
  bool use_graphs = true;
  // launch shapes picked by fmm_autotune (0: built-in choice)
  int tune_split[2] = {0, 0};  // split-K of the tcgen05 contraction, [kModeM2P], [kModeM2L]
  int tune_lo = -1;            // solves from this level use tune_split (-1: every level)
  int cur_lo = 0;              // lo of the solve being enqueued
  int tune_opb = 0;            // target octs per block of the near-field kernel
  // translation tables shared with other contexts of the same device, p and precision
  bool tables_shared = false;
  int64_t n_graph_launch = 0, n_graph_build = 0;
};

// ---- launchers (stream-ordered, no synchronisation) -----------------------
// tree.cu
fmm_status tree_prepare(Ctx* c);                 // oct counts, allocation (host)
fmm_status tree_enqueue(Ctx* c, cudaStream_t st);  // device work, capturable
fmm_status tree_finish(Ctx* c, cudaStream_t st);   // the one synchronisation
// upward.cu
fmm_status upward_init(Ctx* c);
void launch_mono_leaves(Ctx* c, int level, cudaStream_t st);
// octs / rows: optional lists restricting the pass (null: the full level)
void launch_upward(Ctx* c, int level, cudaStream_t st, const int32_t* octs = nullptr, int64_t n_octs = 0);
void launch_l2l_add(Ctx* c, int level, cudaStream_t st, const int32_t* rows = nullptr, int64_t nrows = 0);
// partial upward passes: the ancestor M2M of levels b_top..2 in one block (short lists only)
int m2m_chain_warps(const Ctx* c);
void launch_m2m_chain(Ctx* c, int b_top, cudaStream_t st);
// mixed paths: the whole L2L chain for the levels the near field of targets >= lo reads
void launch_l2l_path(Ctx* c, int lo, cudaStream_t st);
// mixed paths: clears the M2L sums of the rows the next M2L writes (levels[i],
// rows[i] / nrows[i]; null rows: the level's full list)
void launch_zero_lm(Ctx* c, const std::vector<int>& levels, const std::vector<const int32_t*>& rows,
                    const std::vector<int64_t>& nrows, cudaStream_t st);
// gemm_f64.cu
void launch_gemm_f64(Ctx* c, const GemmOperand& op, int mode, int level_rows, cudaStream_t st,
                     const int32_t* rows = nullptr, int64_t nrows = 0);
// gemm_tc.cu
fmm_status make_tensor_maps(Ctx* c, GemmOperand& op);
// rows[i] / nrows[i]: optional per-level row lists (null: the level's full list);
// sm_budget: SMs the split-K factor may fill (0: all; fewer leave room for
// kernels running beside it)
void launch_gemm_tc(Ctx* c, const GemmOperand& op, int mode, const int* row_levels, int nlev, cudaStream_t st,
                    const int32_t* const* rows = nullptr, const int64_t* nrows = nullptr, int sm_budget = 0);
// near.cu
fmm_status near_init(Ctx* c);
void launch_near_m2p(Ctx* c, int lo, cudaStream_t st);
void launch_near(Ctx* c, int lo, void* const* phi, void* const* accel, int out_fp32, cudaStream_t st);
int near_opb(const Ctx* c);

// drift.cu: true when a solve from lo drifts some stale tree; the device work
bool drift_active(const Ctx* c, int lo);
fmm_status drift_prepare(Ctx* c);  // scratch and tables (host, allocates)
void launch_drift(Ctx* c, int lo, cudaStream_t st);

// adjoint.cu
void launch_adj_mark(Ctx* c, const int32_t* rows, int64_t nrows, const int32_t* nbr, int32_t* flags,
                     cudaStream_t st);
void launch_adjoint(Ctx* c, int lo, const void* const* g_phi, const void* const* g_accel, int in_fp32,
                    cudaStream_t st);

// contraction modes: the bottom M2P (rows of level l-1, targets their
// grandchildren), M2L, the Delta l = 2 M2P (rows of level l-2, targets three
// levels down) and the Delta l = 2 near-field ring (P2P from child masses,
// rows and targets as kModeM2P)
enum { kModeM2P = 0, kModeM2L = 1, kModeM2P2 = 2, kModeP2PR = 3 };
// operator kinds of build_operator
enum { kOpM2P = 0, kOpM2L = 1, kOpP2P = 2 };

// Delta l = 2: the 8 child masses of every cell of level lmax-1 as operand rows
void launch_child_masses(Ctx* c, cudaStream_t st);
// periodic boundaries: the level-1 local expansions from the lattice (adds into
// Lm of level 1, or L in FP64)
void launch_lattice(Ctx* c, cudaStream_t st);

// Highest box level holding local expansions: lmax-2 (the paper's bottom
// M2P), lmax-1 with bottom mode 1 (M2L into the parent box, then L2P).
// With Delta l = 2 the level lmax-2 expansions are the L2L of lmax-3's (the
// near field reads them there) and M2L stops one level higher.
inline int top_local_level(const Ctx* c) {
  return c->lmax - 2 + (c->cfg.bottom_mode == FMM_BOTTOM_M2L_L2P ? 1 : 0);
}
inline int top_m2l_level(const Ctx* c) { return top_local_level(c) - (c->cfg.delta_l == 2 ? 1 : 0); }
// First box level with an interaction list (and a local expansion): 2, or 1
// with periodic boundaries (the images of the root around level 1).
inline int first_local_level(const Ctx* c) { return c->cfg.periodic ? 1 : 2; }

}  // namespace fmm
