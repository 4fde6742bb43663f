// gemm_f64.cu -- M2L (Eq. 3) and bottom M2P (Fig. 2, Alg. 4) in FP64 as
// gathered contractions on the CUDA cores.
//
// A row is an oct of the source/target grid.  For each of the 26 neighbour
// offsets q of the oct's parent, the 8 cells of the neighbour oct supply their
// multipoles (the sources of the interaction list, Sec. 2); the operator maps
// them to the 8 target cells (M2L: 8 local expansions) or to the 64 grandchild
// cells (M2P: phi and accel).  The operator table is stored [K][N] with K
// ordered (q, alpha, s) so that an output column with |beta| = d only visits
// the prefix |alpha| <= p - d of each offset segment (the Eq. 3 truncation),
// which skips the zeros of M2L entirely.  Small levels split the 26 offsets
// over grid.z (partial sums added with FP64 atomics) so that every SM has work;
// M2P adds only into leaf targets, whose accumulators are zero between solves
// (the near-field kernel clears what it reads).  The Delta l = 2 variant
// (footnote of Sec. 2) adds M2P from the level l-2 grid (2048 columns, the 512
// level-l cells under a row oct) and the near-field ring (the sources are the
// 8 child masses of each level l-1 cell: P2P as a contraction).
#include "fmm_internal.cuh"

namespace fmm {
namespace {

constexpr int TM = 16;   // rows per block
constexpr int KC = 64;   // K chunk staged in shared memory
__constant__ int c_nbr26[26] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12,
                                14, 15, 16, 17, 18, 19, 20, 21, 22, 23, 24, 25, 26};

struct F64Params {
  const double* M;          // sources [cells][nc] of the row level
  const int32_t* rows;
  int64_t nrows;
  const int32_t* nbr;       // [oct][27] of the row level
  const double* B;          // [26*KQ][N]
  const int32_t* klimit;    // [N]
  int KQ, N, nc;
  int mode;
  double* acc;              // M2P: [cells of level l][4]
  const int32_t* cell_child_rows;
  const int32_t* cell_child_mid;  // M2P2: cell_child of the level between rows and targets
  const int32_t* cell_child_tgt;  // M2P: cell_child of the target level (refined targets get nothing)
  int q_per_split;          // neighbour offsets per grid.z slice
  double* L;                // M2L: [slot*8 + cell][nc]
  const int32_t* slot;      // M2L: local-expansion slot of each oct
};

__global__ void __launch_bounds__(256) k_gemm_f64(F64Params P) {
  pdl_wait();  // no early trigger: a long kernel sharing the SMs with the other branch
  __shared__ double As[TM][KC];
  __shared__ int32_t src[TM][26];
  const int n = blockIdx.y * 256 + threadIdx.x;
  const bool col_ok = n < P.N;
  const int64_t r0 = (int64_t)blockIdx.x * TM;
  for (int i = threadIdx.x; i < TM * 26; i += 256) {
    int r = i / 26, q = i - r * 26;
    int64_t ri = r0 + r;
    src[r][q] = (ri < P.nrows) ? P.nbr[(int64_t)P.rows[ri] * 27 + c_nbr26[q]] : -1;
  }
  // block-wide K extent of a segment: max klimit over this block's columns
  __shared__ int kmax_s;
  if (threadIdx.x == 0) kmax_s = 0;
  __syncthreads();
  const int mylim = col_ok ? P.klimit[n] : 0;
  atomicMax(&kmax_s, mylim);
  __syncthreads();
  const int kmax = kmax_s;
  double acc[TM];
#pragma unroll
  for (int r = 0; r < TM; ++r) acc[r] = 0.0;
  const int q_end = min(26, ((int)blockIdx.z + 1) * P.q_per_split);
  for (int q = (int)blockIdx.z * P.q_per_split; q < q_end; ++q) {
    for (int k0 = 0; k0 < kmax; k0 += KC) {
      __syncthreads();
      for (int i = threadIdx.x; i < TM * KC; i += 256) {
        int r = i / KC, kk = i - r * KC;
        int k = k0 + kk;  // k = alpha*8 + s inside the segment
        double v = 0.0;
        int32_t so = src[r][q];
        if (so >= 0 && k < P.KQ) {
          int alpha = k >> 3, s = k & 7;
          v = P.M[((int64_t)so * 8 + s) * P.nc + alpha];
        }
        As[r][kk] = v;
      }
      __syncthreads();
      int kend = min(KC, mylim - k0);
      const double* Bp = P.B + ((int64_t)q * P.KQ + k0) * P.N + n;
      for (int kk = 0; kk < kend; ++kk) {
        double b = Bp[(int64_t)kk * P.N];
#pragma unroll
        for (int r = 0; r < TM; ++r) acc[r] = fma(As[r][kk], b, acc[r]);
      }
    }
  }
  if (!col_ok) return;
  for (int r = 0; r < TM; ++r) {
    int64_t ri = r0 + r;
    if (ri >= P.nrows) break;
    int32_t o = P.rows[ri];
    if (P.mode == kModeM2P2) {
      const int g = n >> 8, f = (n >> 5) & 7, t = (n >> 2) & 7, comp = n & 3;
      const int32_t mid = P.cell_child_rows[(int64_t)o * 8 + g];
      const int32_t ch = mid >= 0 ? P.cell_child_mid[(int64_t)mid * 8 + f] : -1;
      if (ch >= 0 && P.cell_child_tgt[(int64_t)ch * 8 + t] < 0)
        atomicAdd(&P.acc[((int64_t)ch * 8 + t) * 4 + comp], acc[r]);
    } else if (P.mode != kModeM2L) {
      int f = n >> 5, t = (n >> 2) & 7, comp = n & 3;
      int32_t ch = P.cell_child_rows[(int64_t)o * 8 + f];
      if (ch >= 0 && P.cell_child_tgt[(int64_t)ch * 8 + t] < 0)
        atomicAdd(&P.acc[((int64_t)ch * 8 + t) * 4 + comp], acc[r]);
    } else {
      int b = n / P.nc, beta = n - b * P.nc;
      atomicAdd(&P.L[((int64_t)P.slot[o] * 8 + b) * P.nc + beta], acc[r]);
    }
  }
}

}  // namespace

void launch_gemm_f64(Ctx* c, const GemmOperand& op, int mode, int lr, cudaStream_t st, const int32_t* rows,
                     int64_t nrows) {
  LevelTree& R = c->lev[lr];
  // M2P (and the Delta l = 2 modes): octs with a refined cell; M2L: octs with a
  // cell that has grandchildren
  const bool m2l = mode == kModeM2L;
  const int lt = lr + (mode == kModeM2P2 ? 2 : 1);  // target level of the bottom modes
  const int64_t nr = rows ? nrows : (m2l ? R.n_rowsL : R.n_rows);
  if (!nr) return;
  F64Params P;
  P.M = (const double*)(mode == kModeP2PR ? R.Chi.ptr : R.M.ptr);
  P.rows = rows ? rows : (const int32_t*)(m2l ? R.rowsL.ptr : R.rows.ptr);
  P.slot = (const int32_t*)R.slotL.ptr;
  P.nrows = nr;
  P.nbr = (const int32_t*)R.nbr.ptr;
  P.B = (const double*)op.f64.ptr;
  P.klimit = (const int32_t*)op.klimit.ptr;
  P.KQ = op.kseg;
  P.N = op.N;
  P.nc = mode == kModeP2PR ? 8 : c->tab.nc;
  P.mode = mode;
  P.acc = m2l ? nullptr : (double*)c->lev[lt].acc.ptr;
  P.cell_child_rows = (const int32_t*)R.cell_child.ptr;
  P.cell_child_mid = mode == kModeM2P2 ? (const int32_t*)c->lev[lr + 1].cell_child.ptr : nullptr;
  P.cell_child_tgt = m2l ? nullptr : (const int32_t*)c->lev[lt].cell_child.ptr;
  P.L = m2l ? (double*)R.L.ptr : nullptr;
  // split the 26 offsets until about two blocks per SM are in flight
  const int64_t blocks2 = ((nr + TM - 1) / TM) * ((op.N + 255) / 256);
  int split = (int)std::min<int64_t>(26, std::max<int64_t>(1, (2 * c->num_sms + blocks2 - 1) / blocks2));
  P.q_per_split = (26 + split - 1) / split;
  split = (26 + P.q_per_split - 1) / P.q_per_split;
  dim3 grid((unsigned)((nr + TM - 1) / TM), (unsigned)((op.N + 255) / 256), (unsigned)split);
  ++c->n_launch;
  // a normal launch: this long kernel shares the SMs with the other branch of the
  // solve, and early-launched waiting blocks of a successor would take its slots
  k_gemm_f64<<<grid, 256, 0, st>>>(P);
}

}  // namespace fmm
