// upward.cu -- Upward pass (P2M, Eq. 1; M2M, Eq. 2; Alg. 2) and the L2L step
// of the downward pass (Eq. 4, Alg. 3).
//
// Expansions are kept in box units (tables.h).  A leaf cell's multipole is its
// mass as a monopole (P2M of one point mass at the cell centre) with all other
// coefficients zero.  It is kept as that one value ("mono"); a full coefficient
// row is written only for the leaves that a contraction reads (those in the
// interface octs, next to refined cells).  A refined cell's multipole is the M2M sum of its
// eight children, read from their masses where they are leaves.  Because the child offsets are (+-1/4)^3 of the parent box,
// M2M factors into a sign transform over the children,
//     S_e[gamma] = sum_c sign(c, e) Mt_c[gamma],  e in {0,1}^3,
// (a 3-stage butterfly, one stage per axis) followed by one short sum per
// output coefficient alpha over gamma <= alpha with the sign pattern
// e = (alpha - gamma) mod 2.  L2L runs the same factorisation backwards: per
// output beta one sum per pattern e, then the butterfly over the children.
//
// The multipole of a box is the sum over the paper's per-level trees T_j of
// their multipoles (each tree holds the mass of one AMR level and M2M is
// linear): the sources M2L and M2P need (the merged tree of Sec. 3.1 plus the
// tree of the target level).
//
// Cell masses ("mono") are stored in the precision of the near-field kernel
// that reads them: FP32 in the mixed path, FP64 in the FP64 path.
#include "fmm_internal.cuh"

namespace fmm {
namespace {

constexpr int kNcMax = 168;  // ncoef(8) = 165



// x[c] -> S[e] = sum_c sign(c, e) x[c]: per axis, (a, b) -> (a + b, b - a).
template <typename T>
__device__ __forceinline__ void sign_transform(T x[8]) {
#pragma unroll
  for (int axis = 0; axis < 3; ++axis) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (c & (1 << axis)) continue;
      const T a = x[c], b = x[c | (1 << axis)];
      x[c] = a + b;
      x[c | (1 << axis)] = b - a;
    }
  }
}

// S[e] -> y[c] = sum_e sign(c, e) S[e]: per axis, (s0, s1) -> (s0 - s1, s0 + s1).
template <typename T>
__device__ __forceinline__ void sign_transform_back(T x[8]) {
#pragma unroll
  for (int axis = 0; axis < 3; ++axis) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (c & (1 << axis)) continue;
      const T s0 = x[c], s1 = x[c | (1 << axis)];
      x[c] = s0 - s1;
      x[c | (1 << axis)] = s0 + s1;
    }
  }
}

// Leaf cells of one level: monopole = mass.
// Block-wide copies of translation tables into shared memory with every load
// of a batch in flight before the first store: these small kernels are bound
// by memory latency, and a plain strided loop pays one round trip per stride.
template <int U, typename T, typename F>
__device__ __forceinline__ void stage_block(int n, F&& load, T* dst) {
  for (int base = 0; base < n; base += U * (int)blockDim.x) {
    T r[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = base + u * (int)blockDim.x + (int)threadIdx.x;
      if (j < n) r[u] = load(j);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = base + u * (int)blockDim.x + (int)threadIdx.x;
      if (j < n) dst[j] = r[u];
    }
  }
}

template <typename TMono>
__global__ void k_leaf_mono(int64_t ncell, const int32_t* __restrict__ cell_child, const double* __restrict__ mass,
                            TMono* __restrict__ mono) {
  pdl_wait();
  pdl_trigger();
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= ncell) return;
  int32_t ch = cell_child[i];
  if (ch >= 0) return;
  mono[i] = (TMono)mass[-1 - (int64_t)ch];
}

// Delta l = 2: the masses of the 8 children of every cell of level lmax-1, as
// the operand rows of the near-field ring contraction (one thread per child;
// consecutive threads write consecutive entries of an oct's row).
template <typename TMono>
__global__ void k_child_masses(int64_t n, const int32_t* __restrict__ cell_child, const TMono* __restrict__ mono,
                               __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                               double* __restrict__ f64) {
  pdl_wait();
  pdl_trigger();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t cell = (i >> 6) * 8 + (i & 7);  // i = 64 oct + 8 child + cell in oct
  const int k = (int)((i >> 3) & 7);
  const int32_t ch = cell_child[cell];
  const TMono v = ch >= 0 ? mono[(int64_t)ch * 8 + k] : (TMono)0;
  if (f64)
    f64[cell * 8 + k] = (double)v;
  else
    put_operand(v, hi, lo, op_index(cell, k, 8));
}

// Coefficient rows of the leaf cells that a contraction can read: a leaf is a
// source of M2L or M2P only when its oct lies in the 3^3 neighbourhood of an
// oct with a refined cell, i.e. only in the interface octs (irows).  Those
// rows get the monopole and explicit zeros; other leaf rows are never read and
// never written.  One warp per interface oct.
template <typename Tout>
__global__ void __launch_bounds__(256) k_leaf_rows(int64_t n, int nc, const int32_t* __restrict__ irows,
                                                   const int32_t* __restrict__ cell_child,
                                                   const double* __restrict__ mass, Tout* __restrict__ M,
                                                   __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  pdl_wait();
  pdl_trigger();
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n) return;  // warp-uniform
  const int64_t o = irows[w];
  // lanes 0..7 fetch the eight cells' links and masses together
  const int32_t chl = lane < 8 ? cell_child[o * 8 + lane] : 0;
  const double ml = (lane < 8 && chl < 0) ? mass[-1 - (int64_t)chl] : 0.0;
  for (int c = 0; c < 8; ++c) {
    const int32_t ch = __shfl_sync(0xffffffffu, chl, c);
    const Tout m = (Tout)__shfl_sync(0xffffffffu, ml, c);
    if (ch >= 0) continue;  // warp-uniform
    const int64_t row = (o * 8 + c) * nc;
    const int64_t obase = op_index(o * 8 + c, 0, nc);
    for (int k = lane; k < nc; k += 32) {
      const Tout v = k == 0 ? m : (Tout)0;
      M[row + k] = v;
      if (hi) put_operand(v, hi, lo, obase + 8 * k);
    }
  }
}

// M2M in FP32 (box levels above the FP64 top of the tree): one warp per oct
// of level b+1, i.e. per refined cell of level b, eight warps per block.  An
// oct whose eight cells are all leaves (the bulk of a refined region's parent
// level) has point-mass children only: after the sign transform over the
// children only gamma = 0 survives, so each output is one product
// w0[alpha] * S[e0[alpha]] with S held in lanes 0..7.  Other octs stage the
// children's coefficients in the warp's slice of shared memory, transform them
// in place and run the per-alpha sums over pair tables that the block stages
// once (only when one of its warps needs them).  Dynamic shared memory:
// m2m_smem.
constexpr int kM2MWarps = 8;

inline size_t m2m_smem(int nc, int npairs) {
  return (size_t)npairs * 8 + (size_t)(nc + 1) * 4 + kM2MWarps * 8 * 4 + (size_t)kM2MWarps * 8 * nc * 4;
}

__global__ void __launch_bounds__(32 * kM2MWarps) k_m2m(
    int64_t n_oct_next, const int32_t* __restrict__ octs, int nc, int npairs,
    const int32_t* __restrict__ oct_parent_next, const int32_t* __restrict__ cell_child_next,
    const float* __restrict__ Mnext, const double* __restrict__ mass_next, float* __restrict__ Mout,
    __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, float* __restrict__ mono,
    const int* __restrict__ poff, const int* __restrict__ pg, const int* __restrict__ pe,
    const float* __restrict__ pc, const float* __restrict__ w0, const int* __restrict__ e0) {
  extern __shared__ __align__(16) unsigned char dsm[];
  float* cf = (float*)dsm;                   // [npairs] coefficients
  int* gx = (int*)(cf + npairs);             // [npairs] gamma + nc * e
  int* off = gx + npairs;                    // [nc + 1]
  int* ccs = off + nc + 1;                   // [warps][8] children of each warp's oct
  float* Sall = (float*)(ccs + 8 * kM2MWarps);  // [warps][8 * nc]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // Before the wait on the previous kernel (the level below, whose rows this
  // one reads): the tree links and leaf masses (set by the tree build and the
  // input staging, kernels that completed before that one started) and the
  // pair tables, so that their latency overlaps the previous level's tail.
  const int64_t i = (int64_t)blockIdx.x * kM2MWarps + warp;
  const bool valid = i < n_oct_next;
  const int64_t o = valid ? (octs ? octs[i] : i) : 0;
  const int64_t cell = valid ? oct_parent_next[o] : 0;
  const int64_t c0 = o * 8;
  const int32_t cc = (valid && lane < 8) ? cell_child_next[c0 + lane] : -1;
  const unsigned full = 0xffffffffu;
  const bool leaf_only = __all_sync(full, cc < 0);
  if (__syncthreads_or(valid && !leaf_only)) {  // block-uniform: stage the pair tables
    stage_block<4>(npairs, [&](int j) { return pc[j]; }, cf);
    stage_block<4>(npairs, [&](int j) { return pg[j] + nc * pe[j]; }, gx);
    stage_block<1>(nc + 1, [&](int j) { return poff[j]; }, off);
    __syncthreads();
  }
  pdl_wait();
  pdl_trigger();
  if (!valid) return;  // warp-uniform; no block-wide barrier below
  if (leaf_only) {
    // table entries first (independent of the masses), all loads in flight together
    int ek[4];
    float wk[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int k = 32 * u + lane;
      ek[u] = k < nc ? e0[k] : 0;
      wk[u] = k < nc ? w0[k] : 0.0f;
    }
    float m = lane < 8 ? (float)mass_next[-1 - (int64_t)cc] : 0.0f;
#pragma unroll
    for (int axis = 0; axis < 3; ++axis) {  // S_e over lanes 0..7, as sign_transform
      const float other = __shfl_xor_sync(full, m, 1 << axis);
      m = (lane & (1 << axis)) ? m - other : m + other;
    }
    for (int kb = 0; kb < nc; kb += 32) {
      const int k = kb + lane;
      const int u = kb >> 5;
      const int e = u < 4 ? ek[u] : (k < nc ? e0[k] : 0);
      const float sv = __shfl_sync(full, m, e);
      if (k < nc) {
        const float v = (u < 4 ? wk[u] : w0[k]) * sv;
        Mout[cell * nc + k] = v;
        if (hi) put_operand(v, hi, lo, op_index(cell, k, nc));
        if (k == 0) mono[cell] = v;
      }
    }
    return;
  }
  int* wcc = ccs + 8 * warp;
  float* S = Sall + (size_t)warp * 8 * nc;
  if (lane < 8) wcc[lane] = cc;
  __syncwarp();
  // the children's rows: every load of a batch in flight before the first store
  for (int base = 0; base < 8 * nc; base += 32 * 12) {
    float r[12];
#pragma unroll
    for (int u = 0; u < 12; ++u) {
      const int idx = base + 32 * u + lane;
      if (idx < 8 * nc) {
        const int c = idx / nc, g = idx - c * nc;
        const int32_t ch = wcc[c];
        r[u] = ch < 0 ? (g == 0 ? (float)mass_next[-1 - (int64_t)ch] : 0.0f) : Mnext[(c0 + c) * nc + g];
      }
    }
#pragma unroll
    for (int u = 0; u < 12; ++u) {
      const int idx = base + 32 * u + lane;
      if (idx < 8 * nc) S[idx] = r[u];
    }
  }
  __syncwarp();
  for (int g = lane; g < nc; g += 32) {
    float x[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = S[c * nc + g];
    sign_transform(x);
#pragma unroll
    for (int e = 0; e < 8; ++e) S[e * nc + g] = x[e];
  }
  __syncwarp();
  for (int k = lane; k < nc; k += 32) {
    float out = 0;
    for (int j = off[k]; j < off[k + 1]; ++j) out += cf[j] * S[gx[j]];
    Mout[cell * nc + k] = out;
    if (hi) put_operand(out, hi, lo, op_index(cell, k, nc));
    if (k == 0) mono[cell] = out;
  }
}

// M2M with FP64 accumulation (the top of the tree and the FP64 path): one
// block per oct of level b+1.  These levels are small, so the kernel is
// latency-bound: the block stages the pair tables and the eight children's
// rows in shared memory and spreads the transform and the per-alpha sums over
// all its threads.  Dynamic shared memory: see m2m_block_smem.
template <typename Tin, typename Tout, typename TMono>
__global__ void __launch_bounds__(128) k_m2m_block(
    const int32_t* __restrict__ octs, int nc, int npairs, const int32_t* __restrict__ oct_parent_next, const int32_t* __restrict__ cell_child_next,
    const Tin* __restrict__ Mnext, const double* __restrict__ mass_next, Tout* __restrict__ Mout,
    __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, TMono* __restrict__ mono,
    const int* __restrict__ poff, const int* __restrict__ pg, const int* __restrict__ pe,
    const double* __restrict__ pc) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char dsm[];
  double* S = (double*)dsm;                   // [8][nc]
  double* cf = S + 8 * nc;                    // [npairs]
  int* gx = (int*)(cf + npairs);              // [npairs]: gamma + nc * e
  int* off = gx + npairs;                     // [nc + 1]
  const int64_t o = octs ? octs[blockIdx.x] : blockIdx.x;
  const int64_t cell = oct_parent_next[o];
  const int64_t c0 = o * 8;
  __shared__ int32_t ccs[8];
  if (threadIdx.x < 8) ccs[threadIdx.x] = cell_child_next[c0 + threadIdx.x];
  stage_block<8>(npairs, [&](int j) { return pc[j]; }, cf);
  stage_block<8>(npairs, [&](int j) { return pg[j] + nc * pe[j]; }, gx);
  stage_block<1>(nc + 1, [&](int j) { return poff[j]; }, off);
  __syncthreads();
  stage_block<6>(8 * nc, [&](int idx) {
    const int c = idx / nc, g = idx - c * nc;
    const int32_t cc = ccs[c];
    return cc < 0 ? (g == 0 ? mass_next[-1 - (int64_t)cc] : 0.0) : (double)Mnext[(c0 + c) * nc + g];
  }, S);
  __syncthreads();
  for (int g = threadIdx.x; g < nc; g += blockDim.x) {
    double x[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = S[c * nc + g];
    sign_transform(x);
#pragma unroll
    for (int e = 0; e < 8; ++e) S[e * nc + g] = x[e];
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nc; k += blockDim.x) {
    double v = 0;
    for (int j = off[k]; j < off[k + 1]; ++j) v += cf[j] * S[gx[j]];
    const Tout w = (Tout)v;
    Mout[cell * nc + k] = w;
    if (hi) put_operand(w, hi, lo, op_index(cell, k, nc));
    if (k == 0) mono[cell] = (TMono)w;
  }
}

inline size_t m2m_block_smem(int nc, int npairs) { return (size_t)8 * nc * 8 + (size_t)npairs * 12 + (nc + 1) * 4; }

// The M2M chain of a partial upward pass (the ancestor octs of an updated
// level), when every level's list is short: one block runs all those levels
// in order, a barrier between levels, instead of one latency-bound launch per
// level.  One warp per oct, as k_m2m's general path, with S in FP64 where the
// output level keeps FP64 multipoles (the top of the tree) and FP32 below; the
// pair tables are staged once.  A level's inputs that this block wrote one
// level earlier are read at L2 (.cg) after the barrier.
struct ChainLevel {            // M2M from the listed octs of level b+1 into their parents (level b)
  const int32_t* octs;         // level b+1 octs (an ancestor list)
  const int32_t* oct_parent;   // level b+1
  const int32_t* cell_child;   // level b+1
  const double* mass;          // level b+1 leaf masses
  const void* Min;             // level b+1 rows (float, or double if in_f64)
  void* Mout;                  // level b rows (float, or double if out_f64)
  __nv_bfloat16* hi;           // level b operand rows, or null
  __nv_bfloat16* lo;           // null for TF32
  void* mono;                  // level b monopoles
  int n, in_f64, out_f64;
};
struct ChainParams {
  ChainLevel lev[kMaxLevel];
  int nlev, nc, npairs;
  const int* poff;
  const int* pg;
  const int* pe;
  const double* pc;
  const float* pc32;
};

inline size_t chain_smem(int nc, int npairs, int warps) {
  return (size_t)npairs * 16 + (size_t)(nc + 1) * 4 + 16 + (size_t)warps * 8 * nc * 8;
}
constexpr size_t kChainSmemMax = 200 * 1024;

template <typename TS>
__device__ __forceinline__ TS chain_child(const ChainLevel& U, int nc, int64_t c0, const int32_t* wcc,
                                          const double* wml, int idx) {
  const int c = idx / nc, g = idx - c * nc;
  const int64_t i = (c0 + c) * nc + g;
  if (wcc[c] < 0) return g == 0 ? (TS)wml[c] : (TS)0;
  return U.in_f64 ? (TS)__ldcg((const double*)U.Min + i) : (TS)__ldcg((const float*)U.Min + i);
}

// One general M2M of oct o (level b+1) into its parent by one warp; S: the
// warp's [8][nc] staging area, in the output's precision.
template <typename TS, typename TMono>
__device__ __forceinline__ void chain_m2m(const ChainLevel& U, int nc, int64_t o, int lane, TS* S, int32_t* wcc,
                                          double* wml, const int* off, const int* gx, const TS* cf) {
  const int64_t cell = U.oct_parent[o];
  const int64_t c0 = o * 8;
  if (lane < 8) {
    const int32_t ch = U.cell_child[c0 + lane];
    wcc[lane] = ch;
    wml[lane] = ch < 0 ? U.mass[-1 - (int64_t)ch] : 0.0;
  }
  __syncwarp();
  for (int base = 0; base < 8 * nc; base += 32 * 8) {
    TS r[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + 32 * u + lane;
      if (idx < 8 * nc) r[u] = chain_child<TS>(U, nc, c0, wcc, wml, idx);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + 32 * u + lane;
      if (idx < 8 * nc) S[idx] = r[u];
    }
  }
  __syncwarp();
  for (int g = lane; g < nc; g += 32) {
    TS x[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = S[c * nc + g];
    sign_transform(x);
#pragma unroll
    for (int e = 0; e < 8; ++e) S[e * nc + g] = x[e];
  }
  __syncwarp();
  for (int k = lane; k < nc; k += 32) {
    TS out = 0;
    for (int j = off[k]; j < off[k + 1]; ++j) out += cf[j] * S[gx[j]];
    if (U.out_f64)
      ((double*)U.Mout)[cell * nc + k] = (double)out;
    else
      ((float*)U.Mout)[cell * nc + k] = (float)out;
    if (U.hi) put_operand(out, U.hi, U.lo, op_index(cell, k, nc));
    if (k == 0) ((TMono*)U.mono)[cell] = (TMono)out;
  }
  __syncwarp();  // S and wcc are reused by the warp's next oct
}

template <typename TMono>
__global__ void __launch_bounds__(1024) k_m2m_chain(const __grid_constant__ ChainParams P) {
  extern __shared__ __align__(16) unsigned char dsm[];
  const int nc = P.nc, np = P.npairs, warps = blockDim.x >> 5;
  double* cf64 = (double*)dsm;            // [np]
  float* cf32 = (float*)(cf64 + np);      // [np]
  int* gx = (int*)(cf32 + np);            // [np]: gamma + nc * e
  int* off = gx + np;                     // [nc + 1]
  double* Sall = (double*)(((uintptr_t)(off + nc + 1) + 15) & ~(uintptr_t)15);  // [warps][8 nc]
  __shared__ int32_t s_cc[32][8];
  __shared__ double s_ml[32][8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  stage_block<4>(np, [&](int j) { return P.pc[j]; }, cf64);
  stage_block<4>(np, [&](int j) { return (float)P.pc[j]; }, cf32);
  stage_block<4>(np, [&](int j) { return P.pg[j] + nc * P.pe[j]; }, gx);
  stage_block<1>(nc + 1, [&](int j) { return P.poff[j]; }, off);
  pdl_wait();
  pdl_trigger();
  __syncthreads();
  for (int k = 0; k < P.nlev; ++k) {
    const ChainLevel& U = P.lev[k];
    for (int i = warp; i < U.n; i += warps) {
      const int64_t o = U.octs[i];
      if (U.out_f64)
        chain_m2m<double, TMono>(U, nc, o, lane, Sall + (size_t)warp * 8 * nc, s_cc[warp], s_ml[warp], off, gx, cf64);
      else
        chain_m2m<float, TMono>(U, nc, o, lane, (float*)(Sall + (size_t)warp * 8 * nc), s_cc[warp], s_ml[warp], off,
                                gx, cf32);
    }
    __threadfence_block();
    __syncthreads();  // the next level reads these rows
  }
}

// Downward step for the row octs of level b: L = L2L(parent's L) + this level's
// M2L sum (accumulated by the contraction in FP32, added here in FP64).  A
// slot's M2L sums are in the contraction's column order: (cell c, beta) sits at
// lmcol[c nc + beta].
// One thread per output coefficient beta, all 8 children at once; the pair
// tables and the parent's expansion are staged in shared memory (dynamic:
// l2l_smem), since these small levels are latency-bound.
__global__ void __launch_bounds__(128) k_l2l_add(int nc, int npairs, const int32_t* __restrict__ rows,
                                                 const int32_t* __restrict__ oct_parent,
                                                 const int32_t* __restrict__ slot, const int32_t* __restrict__ slot_up,
                                                 const double* __restrict__ Lup, float* __restrict__ Lm,
                                                 double* __restrict__ L, float* __restrict__ Lf,
                                                 const int* __restrict__ lmcol, const int* __restrict__ poff8,
                                                 const int* __restrict__ pg, const double* __restrict__ pc) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char dsm[];
  double* Lp = (double*)dsm;            // [nc]
  double* cf = Lp + nc;                 // [npairs]
  int* gg = (int*)(cf + npairs);        // [npairs]
  int* off = gg + npairs;               // [8 nc + 1]
  const int32_t o = rows[blockIdx.x];
  const int64_t so = slot[o];
  if (Lup) {
    const int32_t par = oct_parent[o];
    const int64_t sp = (int64_t)slot_up[par >> 3] * 8 + (par & 7);
    stage_block<2>(nc, [&](int k) { return Lup[sp * nc + k]; }, Lp);
    stage_block<8>(npairs, [&](int j) { return pc[j]; }, cf);
    stage_block<8>(npairs, [&](int j) { return pg[j]; }, gg);
    stage_block<6>(8 * nc + 1, [&](int k) { return poff8[k]; }, off);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nc; b += blockDim.x) {
    double acc[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      double s = 0.0;
      if (Lup)
        for (int j = off[b * 8 + e]; j < off[b * 8 + e + 1]; ++j) s += cf[j] * Lp[gg[j]];
      acc[e] = s;
    }
    sign_transform_back(acc);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int64_t idx = (so * 8 + c) * nc + b;
      if (Lm) {
        const int64_t im = so * 8 * nc + lmcol[c * nc + b];
        const double v = acc[c] + (double)Lm[im];
        L[idx] = v;
        Lf[idx] = (float)v;  // converted once here rather than by every target of the near field
        Lm[im] = 0.0f;       // the M2L contraction adds into a cleared slot next time
      } else {
        L[idx] = acc[c];
      }
    }
  }
}

inline size_t l2l_smem(int nc, int npairs) { return (size_t)nc * 8 + (size_t)npairs * 12 + (8 * nc + 1) * 4; }

// Downward pass of the mixed paths in one launch.  Only the levels whose local
// expansions the near field evaluates (target level minus 2; bottom mode 1:
// minus 1) get blocks, one per row oct.  A block walks the path from its level-2
// ancestor cell down to its own oct, L(cell_k) = L2L(L(cell_{k-1})) + M2L sum,
// one cell per level, then all eight cells of its own oct.  L2L is exact, so
// the result is the level-by-level chain's; the ancestors' expansions are
// recomputed by every block that needs them instead of being handed down
// between launches, which leaves one launch and no waits between blocks.  The
// eight S_e sums of a step serve all children alike (see k_l2l_add); a path
// step keeps one child, y = sum_e sign(c, e) S_e with
// sign(c, e) = (-1)^popc(e & ~c) (the back transform of one output).  The M2L
// sums are read, not cleared: k_zero_rows clears them before the next M2L.
// TA is the accumulation type: FP32 by default, FP64 with config.fp64_top (the
// FP32 M2L sums are then added to the FP64 shifted parent).  Each (beta, e) sum
// has a thread of its own: ~11 dependent pairs at p = 6 instead of the up to 84
// a thread per beta chains (FP64 runs about two DFMA per clock per SM on B300).
// Output: the FP32 expansion the near field reads.
struct L2LPathSeg {
  const int32_t* rows;  // row octs of this level
  int64_t n;
  int blk0, level;
};
struct L2LPathParams {
  L2LPathSeg seg[kMaxLevel];
  int nseg, nc, npairs, max_level;
  int l0;  // first level of every path (2; 1 with periodic boundaries)
  const int32_t* oct_parent[kMaxLevel + 1];
  const int32_t* slotL[kMaxLevel + 1];
  const float* Lm[kMaxLevel + 1];  // M2L sums, per slot in the contraction's column order (lmcol)
  float* Lf[kMaxLevel + 1];
  const int* lmcol;
  const int* poff8;
  const int* pg;
  const void* pc;  // coefficients in TA
};

constexpr int kPathThreads = 256;

// S[e][beta] of the expansion Lp for every (beta, e), one pair sum per thread
template <typename TA>
__device__ __forceinline__ void l2l_pattern_sums(int nc, const TA* Lp, const TA* cf, const int* gg,
                                                 const int* off, TA* S) {
  for (int i = threadIdx.x; i < 8 * nc; i += kPathThreads) {  // i = beta * 8 + e
    TA v = 0;
    const int j1 = off[i + 1];
    for (int j = off[i]; j < j1; ++j) v = fma(cf[j], Lp[gg[j]], v);
    S[(i & 7) * nc + (i >> 3)] = v;
  }
}

template <typename TA>
__global__ void __launch_bounds__(kPathThreads) k_l2l_path(const __grid_constant__ L2LPathParams P) {
  extern __shared__ __align__(16) unsigned char dsm[];
  const int nc = P.nc, np = P.npairs;
  TA* cf = (TA*)dsm;                          // [np]
  TA* Lp = cf + np;                           // [nc] expansion of the current path cell
  TA* S = Lp + nc;                            // [8][nc] pattern sums
  int* gg = (int*)(S + 8 * nc);               // [np]
  int* off = gg + np;                         // [8 nc + 1]
  float* Lmp = (float*)(off + 8 * nc + 1);    // [max_level - l0][nc] M2L sums of the path cells
  __shared__ int32_t s_row[kMaxLevel + 1];    // row (8 slot + cell) of the path cell at level k
  __shared__ int s_pos[kMaxLevel + 1];        // its position in its oct
  int si = 0;
  while (si + 1 < P.nseg && (int)blockIdx.x >= P.seg[si + 1].blk0) ++si;
  const L2LPathSeg& Sg = P.seg[si];
  const int b = Sg.level, l0 = P.l0;
  // tree data and tables (written before this solve): read before the wait
  const int32_t o = Sg.rows[blockIdx.x - Sg.blk0];
  const int64_t so = P.slotL[b][o];
  if (threadIdx.x == 0) {
    int32_t cell = b > l0 ? P.oct_parent[b][o] : 0;
    for (int k = b - 1; k >= l0; --k) {
      const int32_t oc = cell >> 3;
      s_row[k] = P.slotL[k][oc] * 8 + (cell & 7);
      s_pos[k] = cell & 7;
      if (k > l0) cell = P.oct_parent[k][oc];
    }
  }
  if (b > l0) {
    stage_block<8>(np, [&](int j) { return ((const TA*)P.pc)[j]; }, cf);
    stage_block<8>(np, [&](int j) { return P.pg[j]; }, gg);
    stage_block<4>(8 * nc + 1, [&](int k) { return P.poff8[k]; }, off);
  }
  pdl_wait();
  pdl_trigger();
  __syncthreads();
  // the M2L sums: the path's (levels l0..b-1) to shared memory, the own oct's to registers
  for (int k = l0; k < b; ++k)
    for (int j = threadIdx.x; j < nc; j += kPathThreads)
      Lmp[(k - l0) * nc + j] = P.Lm[k][(int64_t)(s_row[k] >> 3) * 8 * nc + __ldg(P.lmcol + (s_row[k] & 7) * nc + j)];
  const int beta = threadIdx.x;  // nc <= 165 < kPathThreads
  float own[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) own[c] = beta < nc ? P.Lm[b][so * 8 * nc + __ldg(P.lmcol + c * nc + beta)] : 0.f;
  __syncthreads();
  if (b > l0 && beta < nc) Lp[beta] = (TA)Lmp[beta];  // level l0: the M2L sum alone
  __syncthreads();
  for (int k = l0 + 1; k < b; ++k) {
    l2l_pattern_sums(nc, Lp, cf, gg, off, S);
    __syncthreads();
    if (beta < nc) {
      const unsigned nc_pos = ~(unsigned)s_pos[k] & 7u;
      TA y = (TA)Lmp[(k - l0) * nc + beta];
#pragma unroll
      for (int e = 0; e < 8; ++e) y += (__popc((unsigned)e & nc_pos) & 1) ? -S[e * nc + beta] : S[e * nc + beta];
      Lp[beta] = y;  // every thread has read Lp (barrier above) before it changes
    }
    __syncthreads();
  }
  // the own oct: all eight cells
  TA acc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = 0;
  if (b > l0) {
    l2l_pattern_sums(nc, Lp, cf, gg, off, S);
    __syncthreads();
    if (beta < nc) {
#pragma unroll
      for (int e = 0; e < 8; ++e) acc[e] = S[e * nc + beta];
      sign_transform_back(acc);
    }
  }
  if (beta >= nc) return;
#pragma unroll
  for (int c = 0; c < 8; ++c) P.Lf[b][(so * 8 + c) * nc + beta] = (float)(acc[c] + (TA)own[c]);
}

template <typename TA>
inline size_t l2l_path_smem(int nc, int npairs, int max_level, int l0 = 2) {
  return (size_t)npairs * (sizeof(TA) + 4) + (size_t)nc * sizeof(TA) * 9 + (size_t)(8 * nc + 1) * 4 +
         (size_t)std::max(max_level - l0, 0) * nc * 4;
}

// Periodic boundaries: the level-1 local expansions gain the images of the root
// beyond its 3^3 and the background, L(1) += A M(1), A the dense 8 nc x 8 nc
// host-built map (M2M to the root, the lattice M2L, L2L back).  One warp per
// output row; M(1) is the one level-1 oct's 8 cells (oct 0), its expansion slot
// slot1[0].  The mixed paths add into the M2L sums (column order lmcol), FP64
// into L.
template <typename TM, typename TA>
__global__ void __launch_bounds__(256) k_lattice(int nc, const TA* __restrict__ A, const TM* __restrict__ M1,
                                                 const int32_t* __restrict__ slot1, float* __restrict__ Lm,
                                                 const int* __restrict__ lmcol, double* __restrict__ L64) {
  pdl_wait();
  pdl_trigger();
  const int K = 8 * nc;
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= K) return;
  double s = 0.0;
  for (int k = lane; k < K; k += 32) s += (double)A[(int64_t)row * K + k] * (double)M1[k];
#pragma unroll
  for (int d = 16; d; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
  if (lane) return;
  const int64_t so = slot1[0];
  const int c = row / nc, beta = row - c * nc;
  if (L64)
    atomicAdd(L64 + (so * 8 + c) * nc + beta, s);
  else
    atomicAdd(Lm + so * 8 * nc + lmcol[c * nc + beta], (float)s);
}

// Clears the M2L sums of the row octs the next M2L writes (their slots: 8 nc
// floats each, 2 nc float4), all levels in one launch.
struct ZeroRowsSeg {
  const int32_t* rows;  // row octs of the level (the M2L's list)
  const int32_t* slot;  // local-expansion slot of each oct of the level
  float4* Lm;
  int64_t end;          // cumulative float4 count up to and including this level
};
struct ZeroRows {
  ZeroRowsSeg seg[kMaxLevel + 1];
  int n, nc;
};
__global__ void k_zero_rows(const __grid_constant__ ZeroRows Z) {
  pdl_wait();
  pdl_trigger();
  const int64_t total = Z.seg[Z.n - 1].end;
  const int per = 2 * Z.nc;  // float4 per slot
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    int k = 0;
    while (i >= Z.seg[k].end) ++k;
    const int64_t u = i - (k ? Z.seg[k - 1].end : 0);
    const int64_t r = u / per;
    Z.seg[k].Lm[(int64_t)Z.seg[k].slot[Z.seg[k].rows[r]] * per + (u - r * per)] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

}  // namespace

// Kernel attributes set once per context creation (not inside a stream capture):
// the FP32 M2M needs more than 48 KB of dynamic shared memory at p = 8.
fmm_status upward_init(Ctx* c) {
  cudaError_t e = cudaFuncSetAttribute(k_m2m, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)m2m_smem(165, 3003));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_l2l_path<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)l2l_path_smem<double>(165, 3003, kMaxLevel, 1));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_l2l_path<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)l2l_path_smem<float>(165, 3003, kMaxLevel, 1));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_m2m_chain<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kChainSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_m2m_chain<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kChainSmemMax);

  if (e != cudaSuccess) {
    c->last_error = std::string("upward_init: ") + cudaGetErrorString(e);
    return FMM_ERR_CUDA;
  }
  return FMM_OK;
}

void launch_child_masses(Ctx* c, cudaStream_t st) {
  const int l1 = c->lmax - 1;
  LevelTree& T = c->lev[l1];
  const int64_t n = 64 * T.n_oct;
  if (l1 < 1 || !n) return;
  const int32_t* cc = (const int32_t*)T.cell_child.ptr;
  const unsigned g = (unsigned)((n + 255) / 256);
  ++c->n_launch;
  if (c->cfg.precision == FMM_FP64) {
    launch_pdl(k_child_masses<double>, g, 256, 0, st, n, cc, (const double*)c->lev[c->lmax].mono.ptr,
               (__nv_bfloat16*)nullptr, (__nv_bfloat16*)nullptr, (double*)T.Chi.ptr);
  } else {
    __nv_bfloat16* lo = c->cfg.precision == FMM_MIXED_TF32 ? nullptr : (__nv_bfloat16*)T.Clo.ptr;
    launch_pdl(k_child_masses<float>, g, 256, 0, st, n, cc, (const float*)c->lev[c->lmax].mono.ptr,
               (__nv_bfloat16*)T.Chi.ptr, lo, (double*)nullptr);
  }
}

void launch_mono_leaves(Ctx* c, int l, cudaStream_t st) {
  LevelTree& T = c->lev[l];
  int64_t n = 8 * T.n_oct;
  if (!n || !T.n_leaf) return;
  unsigned g = (unsigned)((n + 255) / 256);
  const int32_t* cc = (const int32_t*)T.cell_child.ptr;
  const double* mass = (const double*)T.mass.ptr;
  const bool f64 = c->cfg.precision == FMM_FP64;
  ++c->n_launch;
  if (f64)
    launch_pdl(k_leaf_mono<double>, g, 256, 0, st, n, cc, mass, (double*)T.mono.ptr);
  else
    launch_pdl(k_leaf_mono<float>, g, 256, 0, st, n, cc, mass, (float*)T.mono.ptr);
  if (l == c->lmax || !T.n_irows) return;  // no coefficient rows at the finest level
  const unsigned gr = (unsigned)((T.n_irows * 32 + 255) / 256);
  const int32_t* ir = (const int32_t*)T.irows.ptr;
  __nv_bfloat16* hi = (__nv_bfloat16*)T.Mhi.ptr;
  // TF32 precision: one FP32 (TF32-rounded) operand per coefficient in Mhi, no lo half
  __nv_bfloat16* lo = c->cfg.precision == FMM_MIXED_TF32 ? nullptr : (__nv_bfloat16*)T.Mlo.ptr;
  ++c->n_launch;
  if (T.m_is_f64)
    launch_pdl(k_leaf_rows<double>, gr, 256, 0, st, T.n_irows, c->tab.nc, ir, cc, mass, (double*)T.M.ptr,
                                            f64 ? nullptr : hi, f64 ? nullptr : lo);
  else
    launch_pdl(k_leaf_rows<float>, gr, 256, 0, st, T.n_irows, c->tab.nc, ir, cc, mass, (float*)T.M.ptr, hi, lo);
}

void launch_upward(Ctx* c, int b, cudaStream_t st, const int32_t* octs, int64_t n_octs) {
  LevelTree& T = c->lev[b];
  LevelTree& N = c->lev[b + 1];
  if (!N.n_oct) return;
  const int nc = c->tab.nc;
  const bool f64 = c->cfg.precision == FMM_FP64;
  const int* poff = (const int*)c->d_m2m_off.ptr;
  const int* pg = (const int*)c->d_m2m_g.ptr;
  const int* pe = (const int*)c->d_m2m_e.ptr;
  const double* pc = (const double*)c->d_m2m_c.ptr;
  const int* e0 = (const int*)c->d_m2m_e0.ptr;
  const int64_t n = octs ? n_octs : N.n_oct;  // child octs of level b+1 to process
  if (!n) return;
  const int32_t* par = (const int32_t*)N.oct_parent.ptr;
  const int32_t* ccn = (const int32_t*)N.cell_child.ptr;
  const double* mn = (const double*)N.mass.ptr;
  __nv_bfloat16* hi = (__nv_bfloat16*)T.Mhi.ptr;
  __nv_bfloat16* lo = c->cfg.precision == FMM_MIXED_TF32 ? nullptr : (__nv_bfloat16*)T.Mlo.ptr;
  const unsigned g32 = (unsigned)((n + kM2MWarps - 1) / kM2MWarps);
  ++c->n_launch;
  const int np = (int)c->tab.m2m_g.size();
  const size_t smb = m2m_block_smem(nc, np);
  if (f64) {
    launch_pdl(k_m2m_block<double, double, double>, (unsigned)n, 128, smb, st, octs, nc, np, par, ccn, (const double*)N.M.ptr, mn,
                                                                     (double*)T.M.ptr, hi, lo, (double*)T.mono.ptr,
                                                                     poff, pg, pe, pc);
  } else if (T.m_is_f64) {  // mixed path, top of the tree: FP64 shifts
    if (N.m_is_f64)
      launch_pdl(k_m2m_block<double, double, float>, (unsigned)n, 128, smb, st, octs, nc, np, par, ccn, (const double*)N.M.ptr, mn,
                                                                      (double*)T.M.ptr, hi, lo, (float*)T.mono.ptr,
                                                                      poff, pg, pe, pc);
    else
      launch_pdl(k_m2m_block<float, double, float>, (unsigned)n, 128, smb, st, octs, nc, np, par, ccn, (const float*)N.M.ptr, mn,
                                                                     (double*)T.M.ptr, hi, lo, (float*)T.mono.ptr,
                                                                     poff, pg, pe, pc);
  } else {
    const size_t sm32 = m2m_smem(nc, np);
    launch_pdl(k_m2m, g32, 32 * kM2MWarps, sm32, st, n, octs, nc, np, par, ccn, (const float*)N.M.ptr, mn,
               (float*)T.M.ptr, hi, lo, (float*)T.mono.ptr, poff, pg, pe, (const float*)c->d_m2m_c32.ptr,
               (const float*)c->d_m2m_w0_32.ptr, e0);
  }
}

void launch_l2l_path(Ctx* c, int lo, cudaStream_t st) {
  const int m1 = c->cfg.bottom_mode == FMM_BOTTOM_M2L_L2P;
  const int top = top_local_level(c);
  L2LPathParams P{};
  int blocks = 0;
  const int l0 = first_local_level(c);
  P.l0 = l0;
  for (int b = std::max(l0, lo - (2 - m1)); b <= top; ++b) {
    LevelTree& T = c->lev[b];
    if (!T.n_rowsL) continue;
    L2LPathSeg& S = P.seg[P.nseg++];
    S.rows = (const int32_t*)T.rowsL.ptr;
    S.n = T.n_rowsL;
    S.blk0 = blocks;
    S.level = b;
    blocks += (int)T.n_rowsL;
    P.max_level = b;
  }
  if (!blocks) return;
  for (int k = l0; k <= P.max_level; ++k) {
    LevelTree& T = c->lev[k];
    P.oct_parent[k] = (const int32_t*)T.oct_parent.ptr;
    P.slotL[k] = (const int32_t*)T.slotL.ptr;
    P.Lm[k] = (const float*)T.Lm.ptr;
    P.Lf[k] = (float*)T.Lf.ptr;
  }
  P.nc = c->tab.nc;
  P.npairs = (int)c->tab.l2l_g.size();
  P.lmcol = (const int*)c->op_m2l.colmap.ptr;
  P.poff8 = (const int*)c->d_l2l_off8.ptr;
  P.pg = (const int*)c->d_l2l_g.ptr;
  ++c->n_launch;
  if (c->cfg.fp64_top) {
    P.pc = c->d_l2l_c.ptr;
    launch_pdl(k_l2l_path<double>, (unsigned)blocks, kPathThreads,
               l2l_path_smem<double>(P.nc, P.npairs, P.max_level, l0), st, P);
  } else {
    P.pc = c->d_l2l_c32.ptr;
    launch_pdl(k_l2l_path<float>, (unsigned)blocks, kPathThreads,
               l2l_path_smem<float>(P.nc, P.npairs, P.max_level, l0), st, P);
  }
}

void launch_zero_lm(Ctx* c, const std::vector<int>& levels, const std::vector<const int32_t*>& rows,
                    const std::vector<int64_t>& nrows, cudaStream_t st) {
  ZeroRows Z{};
  Z.nc = c->tab.nc;
  int64_t tot = 0;
  for (size_t i = 0; i < levels.size(); ++i) {
    LevelTree& T = c->lev[levels[i]];
    const int32_t* r = rows[i] ? rows[i] : (const int32_t*)T.rowsL.ptr;
    const int64_t n = rows[i] ? nrows[i] : T.n_rowsL;
    if (!n || !T.Lm.ptr) continue;
    tot += n * 2 * Z.nc;
    ZeroRowsSeg& S = Z.seg[Z.n++];
    S.rows = r;
    S.slot = (const int32_t*)T.slotL.ptr;
    S.Lm = (float4*)T.Lm.ptr;
    S.end = tot;
  }
  if (!tot) return;
  ++c->n_launch;
  const unsigned g = (unsigned)std::min<int64_t>((tot + 255) / 256, 4 * c->num_sms);
  launch_pdl(k_zero_rows, g, 256, 0, st, Z);
}

int m2m_chain_warps(const Ctx* c) {
  const int nc = c->tab.nc, np = (int)c->tab.m2m_g.size();
  const size_t fixed = chain_smem(nc, np, 0);
  const int w = fixed >= kChainSmemMax ? 0 : (int)((kChainSmemMax - fixed) / ((size_t)64 * nc));
  return std::min(32, w);
}

void launch_m2m_chain(Ctx* c, int b_top, cudaStream_t st) {
  const int nc = c->tab.nc;
  const bool f64 = c->cfg.precision == FMM_FP64;
  const bool tf32 = c->cfg.precision == FMM_MIXED_TF32;
  ChainParams P{};
  for (int b = b_top; b >= 2; --b) {
    LevelTree& T = c->lev[b];
    LevelTree& N = c->lev[b + 1];
    if (!N.n_anc) continue;
    ChainLevel& U = P.lev[P.nlev++];
    U.octs = (const int32_t*)N.anc.ptr;
    U.n = (int)N.n_anc;
    U.oct_parent = (const int32_t*)N.oct_parent.ptr;
    U.cell_child = (const int32_t*)N.cell_child.ptr;
    U.mass = (const double*)N.mass.ptr;
    U.Min = N.M.ptr;
    U.in_f64 = N.m_is_f64 ? 1 : 0;
    U.Mout = T.M.ptr;
    U.out_f64 = T.m_is_f64 ? 1 : 0;
    U.hi = f64 ? nullptr : (__nv_bfloat16*)T.Mhi.ptr;
    U.lo = (f64 || tf32) ? nullptr : (__nv_bfloat16*)T.Mlo.ptr;
    U.mono = T.mono.ptr;
  }
  if (!P.nlev) return;
  P.nc = nc;
  P.npairs = (int)c->tab.m2m_g.size();
  P.poff = (const int*)c->d_m2m_off.ptr;
  P.pg = (const int*)c->d_m2m_g.ptr;
  P.pe = (const int*)c->d_m2m_e.ptr;
  P.pc = (const double*)c->d_m2m_c.ptr;
  const int w = m2m_chain_warps(c);
  ++c->n_launch;
  if (f64)
    launch_pdl(k_m2m_chain<double>, 1u, 32u * w, chain_smem(nc, P.npairs, w), st, P);
  else
    launch_pdl(k_m2m_chain<float>, 1u, 32u * w, chain_smem(nc, P.npairs, w), st, P);
}

void launch_lattice(Ctx* c, cudaStream_t st) {
  LevelTree& T = c->lev[1];
  if (!T.n_rowsL) return;
  const int nc = c->tab.nc;
  const unsigned g = (unsigned)((8 * nc + 7) / 8);
  const int32_t* slot1 = (const int32_t*)T.slotL.ptr;
  ++c->n_launch;
  if (c->cfg.precision == FMM_FP64) {
    launch_pdl(k_lattice<double, double>, g, 256, 0, st, nc, (const double*)c->d_lat64.ptr, (const double*)T.M.ptr,
               slot1, (float*)nullptr, (const int*)nullptr, (double*)T.L.ptr);
  } else if (T.m_is_f64) {
    launch_pdl(k_lattice<double, float>, g, 256, 0, st, nc, (const float*)c->d_lat32.ptr, (const double*)T.M.ptr,
               slot1, (float*)T.Lm.ptr, (const int*)c->op_m2l.colmap.ptr, (double*)nullptr);
  } else {
    launch_pdl(k_lattice<float, float>, g, 256, 0, st, nc, (const float*)c->d_lat32.ptr, (const float*)T.M.ptr,
               slot1, (float*)T.Lm.ptr, (const int*)c->op_m2l.colmap.ptr, (double*)nullptr);
  }
}

void launch_l2l_add(Ctx* c, int b, cudaStream_t st, const int32_t* rows, int64_t nrows) {
  LevelTree& T = c->lev[b];
  if (!rows) {
    rows = (const int32_t*)T.rowsL.ptr;
    nrows = T.n_rowsL;
  }
  if (!nrows) return;
  ++c->n_launch;
  const int np = (int)c->tab.l2l_g.size();
  launch_pdl(k_l2l_add, (unsigned)nrows, 128, l2l_smem(c->tab.nc, np), st,
      c->tab.nc, np, rows, (const int32_t*)T.oct_parent.ptr, (const int32_t*)T.slotL.ptr,
      b > first_local_level(c) ? (const int32_t*)c->lev[b - 1].slotL.ptr : nullptr,
      b > first_local_level(c) ? (const double*)c->lev[b - 1].L.ptr : nullptr,
      c->cfg.precision == FMM_FP64 ? nullptr : (float*)T.Lm.ptr, (double*)T.L.ptr, (float*)T.Lf.ptr,
      (const int*)c->op_m2l.colmap.ptr, (const int*)c->d_l2l_off8.ptr, (const int*)c->d_l2l_g.ptr, (const double*)c->d_l2l_c.ptr);
}

}  // namespace fmm
