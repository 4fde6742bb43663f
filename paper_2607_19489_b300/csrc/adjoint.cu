// adjoint.cu -- the adjoint (exact transpose) of the FP64 solve.
//
// The map from cell masses m to (phi, accel) computed by fmm_solve is linear:
// P2M / M2M (Eqs. 1-2), M2L and L2L (Eqs. 3-4, Alg. 3), M2P, L2P and P2P
// (Fig. 2, Alg. 4) are each a fixed linear operator applied to the masses.
// Given cotangents (g_phi, g_accel) of the outputs, the gradient of
// <g_phi, phi> + <g_accel, accel> with respect to every mass is therefore the
// transposed chain applied in reverse order:
//
//   scatter^T / P2P^T  near-field pairs, scattered onto the source masses
//   L2P^T              onto the local expansion of each level l-2 box
//   near M2P^T         onto the multipoles of the refined level-l cells
//   M2P^T, M2L^T       gather-form transposed contractions: the row is a
//                      source oct, its inputs are the cotangents of the octs
//                      at the opposite offsets, the operator is transposed
//   L2L^T              bottom-up, onto the parent's local expansion
//   M2M^T              top-down, onto the children's multipoles; a leaf child
//                      (a point mass: monopole only) takes the monopole part
//
// No forward expansion is needed (the map is linear), so the cotangents reuse
// the FP64 expansion buffers: acc holds the cotangent of the M2P accumulator,
// L of the local expansions, M of the multipoles.
#include "fmm_internal.cuh"

namespace fmm {
namespace {

constexpr int kNcMax = 168;
constexpr int kMaxAdjSeg = 8;
constexpr int kAdjOPB = 8;  // target octs per block of the near-field transpose

__constant__ int c_adj_nbr26[26] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12,
                                    14, 15, 16, 17, 18, 19, 20, 21, 22, 23, 24, 25, 26};

// ---- near field and scatter ------------------------------------------------
struct AdjNearSeg {
  const int32_t* tgt;
  const int32_t* nbr;
  const int32_t* cc_l;   // cell_child of the target level l
  const int32_t* cc_up;  // level l-1
  const int32_t* cc_dn;  // level l+1 (or null)
  const void* g_phi;     // cotangents in the caller's order, [n_leaf] and [n_leaf][3]
  const void* g_accel;
  double* gacc;          // [cells of level l][4]: cotangent of the M2P accumulator
  double* gm_l;          // mass cotangents of the leaves of levels l, l-1, l+1
  double* gm_up;
  double* gm_dn;
  double s1, s2;
  int64_t n_tgt;
  int blk0;
};
struct AdjNearParams {
  AdjNearSeg seg[kMaxAdjSeg];
  int nseg, in_fp32;
};

// Cotangent of one P2P pair for the source: d(u_phi phi + u_a . a)/dm with
// phi = -m/r, a = m d/r^3, d = source - target.
__device__ __forceinline__ double p2p_adj(double dx, double dy, double dz, double uphi, double ux, double uy,
                                          double uz) {
  const double r2 = dx * dx + dy * dy + dz * dz;
  const double ir = 1.0 / sqrt(r2);
  return -uphi * ir + (ux * dx + uy * dy + uz * dz) * (ir * ir * ir);
}

// 8 threads per target oct (one per cell).  For every source the eight
// targets' terms are summed with shuffles and added to the source's mass
// cotangent with one atomic.
__global__ void __launch_bounds__(8 * kAdjOPB) k_adj_near(const __grid_constant__ AdjNearParams P) {
  __shared__ int32_t s_nb[kAdjOPB][28];
  int si = 0;
  while (si + 1 < P.nseg && (int)blockIdx.x >= P.seg[si + 1].blk0) ++si;
  const AdjNearSeg& S = P.seg[si];
  const int g = threadIdx.x >> 3, tp = threadIdx.x & 7;
  const int64_t gi = (int64_t)(blockIdx.x - S.blk0) * kAdjOPB + g;
  const bool oct_ok = gi < S.n_tgt;
  const int32_t o = oct_ok ? S.tgt[gi] : 0;
  if (oct_ok)
    for (int q = tp; q < 27; q += 8) s_nb[g][q] = S.nbr[(int64_t)o * 27 + q];
  __syncthreads();
  if (!oct_ok) return;  // the 8 threads of an oct leave together
  const unsigned gmask = 0xFFu << (threadIdx.x & 24);
  const int64_t cell = (int64_t)o * 8 + tp;
  const int32_t self = S.cc_l[cell];
  double uphi = 0, ux = 0, uy = 0, uz = 0;
  if (self < 0) {
    const int64_t li = -1 - (int64_t)self;
    double gp, gx, gy, gz;
    if (P.in_fp32) {
      gp = ((const float*)S.g_phi)[li];
      const float* ga = (const float*)S.g_accel + 3 * li;
      gx = ga[0];
      gy = ga[1];
      gz = ga[2];
    } else {
      gp = ((const double*)S.g_phi)[li];
      const double* ga = (const double*)S.g_accel + 3 * li;
      gx = ga[0];
      gy = ga[1];
      gz = ga[2];
    }
    uphi = S.s1 * gp;
    ux = S.s2 * gx;
    uy = S.s2 * gy;
    uz = S.s2 * gz;
    // phi = s1 (... + pm / 2 + ...), accel = s2 (... + am / 4 + ...)
    S.gacc[cell * 4 + 0] = 0.5 * uphi;
    S.gacc[cell * 4 + 1] = 0.25 * ux;
    S.gacc[cell * 4 + 2] = 0.25 * uy;
    S.gacc[cell * 4 + 3] = 0.25 * uz;
  }
  const int tbx = tp & 1, tby = (tp >> 1) & 1, tbz = (tp >> 2) & 1;
  auto group_sum = [&](double v) {
    v += __shfl_xor_sync(gmask, v, 1, 8);
    v += __shfl_xor_sync(gmask, v, 2, 8);
    v += __shfl_xor_sync(gmask, v, 4, 8);
    return v;
  };
  for (int q = 0; q < 27; ++q) {
    const int32_t nb = s_nb[g][q];
    const int dqx = q % 3 - 1, dqy = (q / 3) % 3 - 1, dqz = q / 9 - 1;
    if (nb <= -2) {  // a level l-1 leaf covering this slot: one source at its centre
      const int64_t C = -2 - (int64_t)nb;
      double v = 0;
      if (self < 0)
        v = p2p_adj(2 * dqx + 0.5 - tbx, 2 * dqy + 0.5 - tby, 2 * dqz + 0.5 - tbz, uphi, ux, uy, uz);
      v = group_sum(v);
      if (tp == 0) atomicAdd(S.gm_up - 1 - S.cc_up[C], v);
      continue;
    }
    if (nb < 0) continue;  // outside the box
    for (int c = 0; c < 8; ++c) {
      const int64_t pc = (int64_t)nb * 8 + c;
      const int32_t ch = S.cc_l[pc];
      // source lower corner 2 dq + bits(c); target at bits(tp): centre offsets
      const int rx = 2 * dqx + (c & 1) - tbx, ry = 2 * dqy + ((c >> 1) & 1) - tby,
                rz = 2 * dqz + ((c >> 2) & 1) - tbz;
      if (ch < 0) {  // a leaf of level l
        double v = 0;
        if (self < 0 && !(q == 13 && c == tp)) v = p2p_adj(rx, ry, rz, uphi, ux, uy, uz);
        v = group_sum(v);
        if (tp == 0) atomicAdd(S.gm_l - 1 - ch, v);
      } else if (S.cc_dn) {  // refined: nearest field for the targets it touches
        const bool touch = self < 0 && abs(rx) <= 1 && abs(ry) <= 1 && abs(rz) <= 1;
        for (int kk = 0; kk < 8; ++kk) {
          double v = 0;
          if (touch)
            v = p2p_adj(rx + ((kk & 1) * 2 - 1) * 0.25, ry + (((kk >> 1) & 1) * 2 - 1) * 0.25,
                        rz + (((kk >> 2) & 1) * 2 - 1) * 0.25, uphi, ux, uy, uz);
          v = group_sum(v);
          if (tp == 0 && v != 0.0) {
            const int32_t lc = S.cc_dn[(int64_t)ch * 8 + kk];
            if (lc < 0) atomicAdd(S.gm_dn - 1 - lc, v);
          }
        }
      }
    }
  }
}

// ---- near-field M2P ---------------------------------------------------------
struct AdjM2PSeg {
  const int32_t* irows;
  const int32_t* nbr;
  const int32_t* cc_l;
  const double* gacc;  // level l
  double* gM;          // multipole cotangents of level l
  int64_t n;
  int blk0;
};
struct AdjM2PParams {
  AdjM2PSeg seg[kMaxAdjSeg];
  int nseg, nc;
  const double* nearop;  // [343][nc][4]
};

// One block per interface oct; warp w takes every 8th refined neighbour cell,
// lanes the coefficients.
__global__ void __launch_bounds__(256) k_adj_near_m2p(const __grid_constant__ AdjM2PParams P) {
  __shared__ int16_t s_list[216];
  __shared__ int s_cnt;
  __shared__ int32_t s_nb[27];
  __shared__ double s_g[8][4];
  int si = 0;
  while (si + 1 < P.nseg && (int)blockIdx.x >= P.seg[si + 1].blk0) ++si;
  const AdjM2PSeg& S = P.seg[si];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t gi = (int64_t)(blockIdx.x - S.blk0);
  if (gi >= S.n) return;
  const int32_t o = S.irows[gi];
  if (threadIdx.x < 27) s_nb[threadIdx.x] = S.nbr[(int64_t)o * 27 + threadIdx.x];
  if (threadIdx.x >= 32 && threadIdx.x < 64) {
    const int t = (threadIdx.x - 32) >> 2, comp = threadIdx.x & 3;
    const int64_t cell = (int64_t)o * 8 + t;
    s_g[t][comp] = S.cc_l[cell] < 0 ? S.gacc[cell * 4 + comp] * (comp == 0 ? 2.0 : 4.0) : 0.0;
  }
  __syncthreads();
  if (w == 0) {
    int cnt = 0;
    for (int s0 = 0; s0 < 216; s0 += 32) {
      const int s = s0 + lane;
      const int32_t nb = (s < 216) ? s_nb[s >> 3] : -1;
      const bool ref = nb >= 0 && S.cc_l[(int64_t)nb * 8 + (s & 7)] >= 0;
      const unsigned m = __ballot_sync(0xffffffffu, ref);
      if (ref) s_list[cnt + __popc(m & ((1u << lane) - 1))] = (int16_t)s;
      cnt += __popc(m);
    }
    if (lane == 0) s_cnt = cnt;
  }
  __syncthreads();
  const int cnt = s_cnt, nc = P.nc;
  for (int k = w; k < cnt; k += 8) {
    const int s = s_list[k];
    const int q = s >> 3, cc = s & 7;
    const int64_t pc = (int64_t)s_nb[q] * 8 + cc;
    for (int a = lane; a < nc; a += 32) {
      double v = 0;
      for (int t = 0; t < 8; ++t) {
        const int rx = (t & 1) - (2 * (q % 3 - 1) + (cc & 1));
        const int ry = ((t >> 1) & 1) - (2 * ((q / 3) % 3 - 1) + ((cc >> 1) & 1));
        const int rz = ((t >> 2) & 1) - (2 * (q / 9 - 1) + ((cc >> 2) & 1));
        if (abs(rx) <= 1 && abs(ry) <= 1 && abs(rz) <= 1) continue;  // nearest field, not M2P
        const int ridx = ((rz + 3) * 7 + (ry + 3)) * 7 + (rx + 3);
        const double* op = P.nearop + ((int64_t)ridx * nc + a) * 4;
        v += op[0] * s_g[t][0] + op[1] * s_g[t][1] + op[2] * s_g[t][2] + op[3] * s_g[t][3];
      }
      if (v != 0.0) atomicAdd(S.gM + pc * nc + a, v);
    }
  }
}

// ---- L2P^T ------------------------------------------------------------------
// One block per oct O of level b = l-2 that needs a local expansion; thread
// (c, beta) gathers the 64 grandchild targets of cell c.
__global__ void __launch_bounds__(256) k_adj_l2p(int nc, const int32_t* __restrict__ rowsL,
                                                 const int32_t* __restrict__ cc_b,
                                                 const int32_t* __restrict__ cc_b1, const double* __restrict__ gacc,
                                                 const double* __restrict__ l2p, double* __restrict__ gL) {
  const int32_t O = rowsL[blockIdx.x];
  for (int idx = threadIdx.x; idx < 8 * nc; idx += blockDim.x) {
    const int c = idx / nc, beta = idx - c * nc;
    const int32_t ch1 = cc_b[(int64_t)O * 8 + c];
    if (ch1 < 0) continue;
    double v = 0;
    for (int f = 0; f < 8; ++f) {
      const int32_t ch2 = cc_b1[(int64_t)ch1 * 8 + f];
      if (ch2 < 0) continue;
      for (int t = 0; t < 8; ++t) {
        const double* g = gacc + ((int64_t)ch2 * 8 + t) * 4;
        const double* T = l2p + ((int64_t)(f * 8 + t) * nc + beta) * 4;
        // phi takes L2P / 4, accel L2P / 16 (level l-2 units): with gacc = (u_phi / 2, u_a / 4)
        v += 0.5 * g[0] * T[0] + 0.25 * (g[1] * T[1] + g[2] * T[2] + g[3] * T[3]);
      }
    }
    gL[((int64_t)blockIdx.x * 8 + c) * nc + beta] += v;  // rowsL position = slot
  }
}

// ---- M2P^T and M2L^T: gather-form transposed contractions -------------------
constexpr int ATM = 8;   // source octs per block
constexpr int AKC = 32;  // input chunk staged in shared memory

struct AdjGemmParams {
  const int32_t* rows;   // source octs S of level b
  int64_t nrows;
  const int32_t* nbr;    // level b
  const double* BT;      // [26][N][KQ]: the forward operator, transposed per offset
  int N, KQ, nc, mode;
  const int32_t* cc_b;   // M2P: cell_child of level b (the forward row's refined cells)
  const double* gacc;    // M2P: cotangent of the accumulator, level b+1 cells [cells][4]
  const double* gL;      // M2L: cotangent of the local expansions of level b, by slot
  const int32_t* slot;   // M2L: local-expansion slot of each oct (-1: none)
  double* gM;            // out: multipole cotangents of level b
};

__global__ void __launch_bounds__(256) k_adj_gemm(const __grid_constant__ AdjGemmParams P) {
  __shared__ double As[ATM][AKC];
  __shared__ int32_t s_R[ATM][26];
  const int k = blockIdx.y * 256 + threadIdx.x;
  const bool k_ok = k < P.KQ;
  const int64_t r0 = (int64_t)blockIdx.x * ATM;
  for (int i = threadIdx.x; i < ATM * 26; i += 256) {
    const int r = i / 26, qi = i - r * 26;
    const int64_t ri = r0 + r;
    // the forward row R that read source S in its slot qi: S's neighbour at the opposite offset
    s_R[r][qi] = (ri < P.nrows) ? P.nbr[(int64_t)P.rows[ri] * 27 + (26 - c_adj_nbr26[qi])] : -1;
  }
  double acc[ATM];
#pragma unroll
  for (int r = 0; r < ATM; ++r) acc[r] = 0.0;
  for (int qi = 0; qi < 26; ++qi) {
    for (int n0 = 0; n0 < P.N; n0 += AKC) {
      __syncthreads();
      for (int i = threadIdx.x; i < ATM * AKC; i += 256) {
        const int r = i / AKC, nn = i - r * AKC, n = n0 + nn;
        const int32_t R = s_R[r][qi];
        double v = 0.0;
        if (R >= 0 && n < P.N) {
          if (P.mode == kModeM2P) {
            const int32_t ch = P.cc_b[(int64_t)R * 8 + (n >> 5)];  // n = (f*8 + t)*4 + comp
            if (ch >= 0) v = P.gacc[((int64_t)ch * 8 + ((n >> 2) & 7)) * 4 + (n & 3)];
          } else {
            const int32_t sl = P.slot[R];
            if (sl >= 0) v = P.gL[(int64_t)sl * 8 * P.nc + n];
          }
        }
        As[r][nn] = v;
      }
      __syncthreads();
      if (!k_ok) continue;
      const int nend = min(AKC, P.N - n0);
      const double* Bp = P.BT + ((int64_t)qi * P.N + n0) * P.KQ + k;
      for (int nn = 0; nn < nend; ++nn) {
        const double b = Bp[(int64_t)nn * P.KQ];
#pragma unroll
        for (int r = 0; r < ATM; ++r) acc[r] = fma(As[r][nn], b, acc[r]);
      }
    }
  }
  if (!k_ok) return;
  for (int r = 0; r < ATM; ++r) {
    const int64_t ri = r0 + r;
    if (ri >= P.nrows) break;
    P.gM[(int64_t)P.rows[ri] * P.KQ + k] += acc[r];  // k = s * nc + alpha
  }
}

// ---- L2L^T ------------------------------------------------------------------
// Per oct o of level b >= 3 with a local expansion: sign transform over the
// children's cotangents, then the transposed pair lists (grouped by the input
// coefficient gamma) onto the parent cell's cotangent.
__global__ void __launch_bounds__(128) k_adj_l2l(int nc, const int32_t* __restrict__ rowsL,
                                                 const int32_t* __restrict__ oct_parent,
                                                 const int32_t* __restrict__ slot_up,
                                                 const double* __restrict__ gL, double* __restrict__ gLup,
                                                 const int* __restrict__ toff, const int* __restrict__ tb,
                                                 const int* __restrict__ te, const double* __restrict__ tc) {
  __shared__ double Sb[8][kNcMax];
  const int32_t o = rowsL[blockIdx.x];
  const int64_t so = blockIdx.x;  // rowsL position = slot
  for (int b = threadIdx.x; b < nc; b += blockDim.x) {
    double x[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = gL[(so * 8 + c) * nc + b];
#pragma unroll
    for (int axis = 0; axis < 3; ++axis)  // S_e = sum_c sign(c, e) x_c
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        if (c & (1 << axis)) continue;
        const double a = x[c], bb = x[c | (1 << axis)];
        x[c] = a + bb;
        x[c | (1 << axis)] = bb - a;
      }
#pragma unroll
    for (int e = 0; e < 8; ++e) Sb[e][b] = x[e];
  }
  __syncthreads();
  const int32_t par = oct_parent[o];
  const int64_t sp = (int64_t)slot_up[par >> 3] * 8 + (par & 7);
  for (int g = threadIdx.x; g < nc; g += blockDim.x) {
    double v = 0;
    for (int j = toff[g]; j < toff[g + 1]; ++j) v += tc[j] * Sb[te[j]][tb[j]];
    gLup[sp * nc + g] += v;
  }
}

// ---- M2M^T ------------------------------------------------------------------
// One warp per oct of level b+1 (the children of one refined cell of level b):
// the transposed pair lists (grouped by (gamma, e)) and the inverse sign
// transform give each child's cotangent; refined children add it to their
// multipole cotangent, leaf children (point masses) take its monopole.
__global__ void __launch_bounds__(128) k_adj_m2m(int64_t n_oct_next, int nc, const int32_t* __restrict__ oct_parent_next,
                                                 const int32_t* __restrict__ cc_next, const double* __restrict__ gM,
                                                 double* __restrict__ gMnext, double* __restrict__ gm_next,
                                                 const int* __restrict__ toff, const int* __restrict__ ta,
                                                 const double* __restrict__ tc) {
  __shared__ double s_row[4][kNcMax];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t o = (int64_t)blockIdx.x * 4 + warp;
  if (o >= n_oct_next) return;
  const int64_t cell = oct_parent_next[o];
  for (int a = lane; a < nc; a += 32) s_row[warp][a] = gM[cell * nc + a];
  __syncwarp();
  for (int g = lane; g < nc; g += 32) {
    double x[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      double v = 0;
      for (int j = toff[g * 8 + e]; j < toff[g * 8 + e + 1]; ++j) v += tc[j] * s_row[warp][ta[j]];
      x[e] = v;
    }
#pragma unroll
    for (int axis = 0; axis < 3; ++axis)  // y_c = sum_e sign(c, e) S_e
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        if (c & (1 << axis)) continue;
        const double s0 = x[c], s1 = x[c | (1 << axis)];
        x[c] = s0 - s1;
        x[c | (1 << axis)] = s0 + s1;
      }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int32_t ch = cc_next[o * 8 + c];
      if (ch >= 0) {
        if (gMnext) gMnext[(o * 8 + c) * nc + g] += x[c];
      } else if (g == 0) {
        gm_next[-1 - (int64_t)ch] += x[c];
      }
    }
  }
}

// ---- leaf rows --------------------------------------------------------------
// The interface leaves whose coefficient rows the contractions read: their
// mass is the row's monopole.
__global__ void k_adj_leaf_rows(int64_t n, int nc, const int32_t* __restrict__ irows,
                                const int32_t* __restrict__ cc, const double* __restrict__ gM,
                                double* __restrict__ gm) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n * 8) return;
  const int64_t cell = (int64_t)irows[i >> 3] * 8 + (i & 7);
  const int32_t ch = cc[cell];
  if (ch < 0) gm[-1 - (int64_t)ch] += gM[cell * nc];
}

// ---- source lists -----------------------------------------------------------
// Octs read by some forward contraction row: the 26 neighbours of each row.
__global__ void k_adj_mark(int64_t nrows, const int32_t* __restrict__ rows, const int32_t* __restrict__ nbr,
                           int32_t* __restrict__ flags) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nrows * 26) return;
  const int64_t r = i / 26;
  const int32_t nb = nbr[(int64_t)rows[r] * 27 + c_adj_nbr26[i - r * 26]];
  if (nb >= 0) flags[nb] = 1;
}

inline unsigned nblk(int64_t n, int b = 256) { return (unsigned)((n + b - 1) / b); }

}  // namespace

// Lists of the octs whose multipoles a contraction reads (M2P rows of level b
// and local-expansion rows of level b): flags written here, compacted by the
// caller.
void launch_adj_mark(Ctx* c, const int32_t* rows, int64_t nrows, const int32_t* nbr, int32_t* flags,
                     cudaStream_t st) {
  if (!nrows) return;
  ++c->n_launch;
  k_adj_mark<<<nblk(nrows * 26), 256, 0, st>>>(nrows, rows, nbr, flags);
}

void launch_adjoint(Ctx* c, int lo, const void* const* g_phi, const void* const* g_accel, int in_fp32,
                    cudaStream_t st) {
  const int lmin = c->lmin, lmax = c->lmax, nc = c->tab.nc;
  // 1. near field, scatter and the cotangent of the M2P accumulator
  {
    AdjNearParams P{};
    P.in_fp32 = in_fp32;
    int blocks = 0;
    for (int l = lo; l <= lmax; ++l) {
      LevelTree& T = c->lev[l];
      if (!T.n_tgt || !T.n_leaf) continue;
      if (P.nseg == kMaxAdjSeg) {
        ++c->n_launch;
        k_adj_near<<<(unsigned)blocks, 8 * kAdjOPB, 0, st>>>(P);
        P.nseg = 0;
        blocks = 0;
      }
      AdjNearSeg& S = P.seg[P.nseg++];
      S.tgt = (const int32_t*)T.tgt.ptr;
      S.nbr = (const int32_t*)T.nbr.ptr;
      S.cc_l = (const int32_t*)T.cell_child.ptr;
      S.cc_up = (const int32_t*)c->lev[l - 1].cell_child.ptr;
      S.cc_dn = l < lmax ? (const int32_t*)c->lev[l + 1].cell_child.ptr : nullptr;
      S.g_phi = g_phi[l - lo];
      S.g_accel = g_accel[l - lo];
      S.gacc = (double*)T.acc.ptr;
      S.gm_l = (double*)T.gmass.ptr;
      S.gm_up = (double*)c->lev[l - 1].gmass.ptr;
      S.gm_dn = l < lmax ? (double*)c->lev[l + 1].gmass.ptr : nullptr;
      S.s1 = c->cfg.G * std::ldexp(1.0, l);
      S.s2 = c->cfg.G * std::ldexp(1.0, 2 * l);
      S.n_tgt = T.n_tgt;
      S.blk0 = blocks;
      blocks += (int)((T.n_tgt + kAdjOPB - 1) / kAdjOPB);
    }
    if (blocks) {
      ++c->n_launch;
      k_adj_near<<<(unsigned)blocks, 8 * kAdjOPB, 0, st>>>(P);
    }
  }
  // 2. near-field M2P of the interface octs
  {
    AdjM2PParams P{};
    P.nc = nc;
    P.nearop = (const double*)c->d_near64.ptr;
    int blocks = 0;
    for (int l = lo; l <= lmax; ++l) {
      LevelTree& T = c->lev[l];
      if (!T.n_irows || !T.n_leaf || l == lmax) continue;  // refined neighbours exist below lmax only
      if (P.nseg == kMaxAdjSeg) {
        ++c->n_launch;
        k_adj_near_m2p<<<(unsigned)blocks, 256, 0, st>>>(P);
        P.nseg = 0;
        blocks = 0;
      }
      AdjM2PSeg& S = P.seg[P.nseg++];
      S.irows = (const int32_t*)T.irows.ptr;
      S.nbr = (const int32_t*)T.nbr.ptr;
      S.cc_l = (const int32_t*)T.cell_child.ptr;
      S.gacc = (const double*)T.acc.ptr;
      S.gM = (double*)T.M.ptr;
      S.n = T.n_irows;
      S.blk0 = blocks;
      blocks += (int)T.n_irows;
    }
    if (blocks) {
      ++c->n_launch;
      k_adj_near_m2p<<<(unsigned)blocks, 256, 0, st>>>(P);
    }
  }
  // 3. L2P^T onto the level l-2 boxes
  for (int l = std::max(lo, 4); l <= lmax; ++l) {
    const int b = l - 2;
    LevelTree& B = c->lev[b];
    if (!B.n_rowsL || !c->lev[l].n_leaf) continue;
    ++c->n_launch;
    k_adj_l2p<<<(unsigned)B.n_rowsL, 256, 0, st>>>(nc, (const int32_t*)B.rowsL.ptr, (const int32_t*)B.cell_child.ptr,
                                                    (const int32_t*)c->lev[b + 1].cell_child.ptr,
                                                    (const double*)c->lev[l].acc.ptr, (const double*)c->d_l2p64.ptr,
                                                    (double*)B.L.ptr);
  }
  // 4. M2P^T onto the level l-1 multipoles
  for (int l = lo; l <= lmax; ++l) {
    const int b = l - 1;
    LevelTree& B = c->lev[b];
    if (!B.n_srcP || !c->lev[l].n_leaf) continue;
    AdjGemmParams P{};
    P.rows = (const int32_t*)B.srcP.ptr;
    P.nrows = B.n_srcP;
    P.nbr = (const int32_t*)B.nbr.ptr;
    P.BT = (const double*)c->d_m2pT.ptr;
    P.N = 256;
    P.KQ = 8 * nc;
    P.nc = nc;
    P.mode = kModeM2P;
    P.cc_b = (const int32_t*)B.cell_child.ptr;
    P.gacc = (const double*)c->lev[l].acc.ptr;
    P.gM = (double*)B.M.ptr;
    ++c->n_launch;
    k_adj_gemm<<<dim3((unsigned)((B.n_srcP + ATM - 1) / ATM), (unsigned)((P.KQ + 255) / 256)), 256, 0, st>>>(P);
  }
  // 5. downward pass reversed: M2L^T at level b, then L2L^T onto level b-1
  for (int b = lmax - 2; b >= 2; --b) {
    LevelTree& B = c->lev[b];
    if (B.n_srcL) {
      AdjGemmParams P{};
      P.rows = (const int32_t*)B.srcL.ptr;
      P.nrows = B.n_srcL;
      P.nbr = (const int32_t*)B.nbr.ptr;
      P.BT = (const double*)c->d_m2lT.ptr;
      P.N = 8 * nc;
      P.KQ = 8 * nc;
      P.nc = nc;
      P.mode = kModeM2L;
      P.gL = (const double*)B.L.ptr;
      P.slot = (const int32_t*)B.slotL.ptr;
      P.gM = (double*)B.M.ptr;
      ++c->n_launch;
      k_adj_gemm<<<dim3((unsigned)((B.n_srcL + ATM - 1) / ATM), (unsigned)((P.KQ + 255) / 256)), 256, 0, st>>>(P);
    }
    if (b >= 3 && B.n_rowsL) {
      ++c->n_launch;
      k_adj_l2l<<<(unsigned)B.n_rowsL, 128, 0, st>>>(nc, (const int32_t*)B.rowsL.ptr, (const int32_t*)B.oct_parent.ptr,
                                                     (const int32_t*)c->lev[b - 1].slotL.ptr,
                                                     (const double*)B.L.ptr, (double*)c->lev[b - 1].L.ptr,
                                                     (const int*)c->d_l2lT_off.ptr, (const int*)c->d_l2lT_b.ptr,
                                                     (const int*)c->d_l2lT_e.ptr, (const double*)c->d_l2lT_c.ptr);
    }
  }
  // 6. upward pass reversed (top-down): M2M^T
  for (int b = 1; b <= lmax - 1; ++b) {
    LevelTree& N = c->lev[b + 1];
    if (!N.n_oct) continue;
    ++c->n_launch;
    k_adj_m2m<<<(unsigned)((N.n_oct + 3) / 4), 128, 0, st>>>(
        N.n_oct, nc, (const int32_t*)N.oct_parent.ptr, (const int32_t*)N.cell_child.ptr,
        (const double*)c->lev[b].M.ptr, b + 1 < lmax ? (double*)N.M.ptr : nullptr, (double*)N.gmass.ptr,
        (const int*)c->d_m2mT_off.ptr, (const int*)c->d_m2mT_a.ptr, (const double*)c->d_m2mT_c.ptr);
  }
  // 7. the interface leaves read as coefficient rows
  for (int l = lmin; l < lmax; ++l) {
    LevelTree& T = c->lev[l];
    if (!T.n_irows || !T.n_leaf) continue;
    ++c->n_launch;
    k_adj_leaf_rows<<<nblk(T.n_irows * 8), 256, 0, st>>>(T.n_irows, nc, (const int32_t*)T.irows.ptr,
                                                         (const int32_t*)T.cell_child.ptr, (const double*)T.M.ptr,
                                                         (double*)T.gmass.ptr);
  }
}

}  // namespace fmm
