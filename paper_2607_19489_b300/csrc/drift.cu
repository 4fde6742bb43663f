// drift.cu -- multipole drifting of the stale trees of a subcycle solve.
//
// The paper rebuilds the trees of the active levels at every subcycle and uses
// the inactive (stale) trees as they were last built; Sec. 4 names drifting
// those multipoles with the centre-of-mass velocity (as SWIFT does) as future
// work.  Here, in a solve from level lo, every box of a stale tree T_j (j < lo)
// at box level b >= 2 (the levels M2L reads) is moved by d = v * dt_j, v the
// centre-of-mass velocity of T_j's cells inside it and dt_j the time since
// level j was last set: its moments about the box centre c become those of the
// moved mass, i.e. its moments about c - d,
//     M'_alpha = sum_{gamma <= alpha} C(alpha, gamma) d^(alpha - gamma) M_gamma
// (the shift of Eq. 2).  Cells used as point masses (P2P, P2L) stay put.
//
// The library stores total multipoles (the sum of all trees), so the drift is
// added as a correction: per stale tree, its own multipoles are rebuilt in FP64
// from its leaves (P2M, then M2M up to box level 2), with the mass and momentum
// of each box, and M' - M is added to the totals (and the tensor-core operand
// rows are rewritten).  The upward pass before it recomputes every total, so
// corrections never stack.  Box units as everywhere (tables.h): Mt = M / h^|alpha|.
#include "fmm_internal.cuh"

namespace fmm {
namespace {

constexpr int kNcMax = 168;

// P2M of tree j: for each oct o of level j, the moments of its leaf cells about
// the centre of the parent cell (level j-1), and their mass and momentum.  A
// child at +-1/4 of the parent box contributes m (+-1/4)^alpha:
// 4^-|alpha| m sign(c, alpha mod 2).  One warp per oct.
__global__ void __launch_bounds__(256) k_drift_leaf(int64_t n_oct, int nc, const int32_t* __restrict__ oct_parent,
                                                   const int32_t* __restrict__ cell_child,
                                                   const double* __restrict__ mass, const double* __restrict__ vel,
                                                   const int32_t* __restrict__ alpha, double* __restrict__ S_up,
                                                   double* __restrict__ Q_up) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n_oct) return;
  const int64_t P = oct_parent[w];  // cell id at level j-1
  double m[8];
  double q = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int32_t ch = cell_child[w * 8 + c];
    m[c] = ch < 0 ? mass[-1 - (int64_t)ch] : 0.0;  // refined children belong to finer trees
    q += m[c];
  }
  if (lane < 4) {
    double v = q;
    if (lane > 0) {
      v = 0.0;
      for (int c = 0; c < 8; ++c) {
        const int32_t ch = cell_child[w * 8 + c];
        if (ch < 0) v += m[c] * vel[3 * (-1 - (int64_t)ch) + lane - 1];
      }
    }
    Q_up[P * 4 + lane] = v;
  }
  for (int k = lane; k < nc; k += 32) {
    const int a = alpha[3 * k], b = alpha[3 * k + 1], cz = alpha[3 * k + 2];
    const int e = (a & 1) | ((b & 1) << 1) | ((cz & 1) << 2);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += child_sign(c, e) * m[c];
    S_up[P * nc + k] = ldexp(s, -2 * (a + b + cz));
  }
}

// M2M of tree j from level b+1 to level b (Eq. 2 in box units, the library's
// pair tables) and the sums of mass and momentum.  One block per oct of level
// b+1, one thread per output coefficient.
__global__ void __launch_bounds__(128) k_drift_m2m(int nc, const int32_t* __restrict__ oct_parent_next,
                                                  const double* __restrict__ S_next, const double* __restrict__ Q_next,
                                                  const int* __restrict__ poff, const int* __restrict__ pg,
                                                  const int* __restrict__ pe, const double* __restrict__ pc,
                                                  double* __restrict__ S, double* __restrict__ Q) {
  __shared__ double s_child[8][kNcMax];
  const int64_t o = blockIdx.x;
  for (int i = threadIdx.x; i < 8 * nc; i += blockDim.x) s_child[i / nc][i % nc] = S_next[o * 8 * nc + i];
  __syncthreads();
  const int64_t P = oct_parent_next[o];
  for (int k = threadIdx.x; k < nc; k += blockDim.x) {
    double acc = 0.0;
    for (int j = poff[k]; j < poff[k + 1]; ++j) {
      const int g = pg[j], e = pe[j];
      double s = 0.0;
#pragma unroll
      for (int c = 0; c < 8; ++c) s += child_sign(c, e) * s_child[c][g];
      acc += pc[j] * s;
    }
    S[P * nc + k] = acc;
  }
  if (threadIdx.x < 4) {
    double v = 0.0;
    for (int c = 0; c < 8; ++c) v += Q_next[(o * 8 + c) * 4 + threadIdx.x];
    Q[P * 4 + threadIdx.x] = v;
  }
}

// The correction of one level: for every cell with tree-j mass, D = (p / m) dt / h
// (box units) and M' - M = sum_{gamma < alpha} C(alpha, gamma) D^(alpha-gamma)
// M_gamma, added to the total multipole; the operand row is rewritten from it.
template <typename TM>
__global__ void __launch_bounds__(128) k_drift_apply(int64_t ncell, int nc, double dt_over_h,
                                                    const int32_t* __restrict__ alpha,
                                                    const double* __restrict__ S, const double* __restrict__ Q,
                                                    TM* __restrict__ M, __nv_bfloat16* __restrict__ hi,
                                                    __nv_bfloat16* __restrict__ lo) {
  __shared__ double s_m[kNcMax];
  __shared__ double s_pow[3][9];  // D_i^n / n! for n <= 8
  const int64_t cell = blockIdx.x;
  if (cell >= ncell) return;
  const double m = Q[cell * 4];
  if (m == 0.0) return;  // no mass of this tree here (uniform across the block)
  for (int k = threadIdx.x; k < nc; k += blockDim.x) s_m[k] = S[cell * nc + k];
  if (threadIdx.x < 3) {
    const double D = Q[cell * 4 + 1 + threadIdx.x] / m * dt_over_h;
    double v = 1.0;
    for (int n = 0; n <= 8; ++n) {
      s_pow[threadIdx.x][n] = v;  // D^n / n!
      v *= D / (n + 1);
    }
  }
  __syncthreads();
  // C(alpha, gamma) D^(alpha-gamma) = alpha! prod_i D_i^(a_i-g_i)/(a_i-g_i)! / gamma!
  for (int k = threadIdx.x; k < nc; k += blockDim.x) {
    const int a0 = alpha[3 * k], a1 = alpha[3 * k + 1], a2 = alpha[3 * k + 2];
    double fa = 1.0;  // alpha!
    for (int i = 2; i <= a0; ++i) fa *= i;
    for (int i = 2; i <= a1; ++i) fa *= i;
    for (int i = 2; i <= a2; ++i) fa *= i;
    double d = 0.0;
    double f0 = 1.0;  // gamma_0!
    for (int g0 = 0; g0 <= a0; ++g0) {
      if (g0) f0 *= g0;
      double f1 = 1.0;
      for (int g1 = 0; g1 <= a1; ++g1) {
        if (g1) f1 *= g1;
        double f2 = 1.0;
        for (int g2 = 0; g2 <= a2; ++g2) {
          if (g2) f2 *= g2;
          if (g0 == a0 && g1 == a1 && g2 == a2) continue;  // the unmoved term
          const int n = g0 + g1 + g2, y = g1 + g2;         // graded index of gamma
          const int gi = n * (n + 1) * (n + 2) / 6 + y * (y + 1) / 2 + g2;
          d += s_pow[0][a0 - g0] * s_pow[1][a1 - g1] * s_pow[2][a2 - g2] / (f0 * f1 * f2) * s_m[gi];
        }
      }
    }
    const TM v = (TM)((double)M[cell * nc + k] + fa * d);
    M[cell * nc + k] = v;
    if (hi) put_operand(v, hi, lo, op_index(cell, k, nc));
  }
}

}  // namespace

bool drift_active(const Ctx* c, int lo) {
  if (c->drift_dt.empty() || lo <= c->lmin) return false;
  for (int j = c->lmin; j < lo && j <= c->lmax; ++j)
    if (j >= 3 && c->drift_dt[j - c->lmin] != 0.0) return true;
  return false;
}

fmm_status drift_prepare(Ctx* c) {
  const int nc = c->tab.nc;
  if (!c->d_alpha.ptr) {
    std::vector<int32_t> a(3 * nc);
    for (int k = 0; k < nc; ++k)
      for (int i = 0; i < 3; ++i) a[3 * k + i] = c->tab.mi.list[k][i];
    if (buf_ensure(c, c->d_alpha, a.size() * 4) != cudaSuccess ||
        cudaMemcpy(c->d_alpha.ptr, a.data(), a.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
      c->last_error = "drift: cannot upload the multi-index table";
      return FMM_ERR_OOM;
    }
  }
  if (!c->have_levels && c->lmax < 0) return FMM_OK;
  for (int b = 2; b < c->lmax; ++b) {
    LevelTree& T = c->lev[b];
    const int64_t ncell = std::max<int64_t>(8 * T.n_oct, 1);
    cudaError_t e = buf_ensure(c, T.dS, ncell * nc * 8);
    if (e == cudaSuccess) e = buf_ensure(c, T.dQ, ncell * 4 * 8);
    if (e != cudaSuccess) {
      c->last_error = "drift: scratch allocation failed";
      return e == cudaErrorMemoryAllocation ? FMM_ERR_OOM : FMM_ERR_CUDA;
    }
  }
  return FMM_OK;
}

// After the (full) upward pass of a solve from lo: the correction of every
// stale tree j in lmin..lo-1 with a time step, one tree after the other.
void launch_drift(Ctx* c, int lo, cudaStream_t st) {
  const int nc = c->tab.nc;
  const bool f64 = c->cfg.precision == FMM_FP64;
  const bool tf32 = c->cfg.precision == FMM_MIXED_TF32;
  const int32_t* alpha = (const int32_t*)c->d_alpha.ptr;
  for (int j = c->lmin; j < lo && j <= c->lmax; ++j) {
    const double dt = c->drift_dt[j - c->lmin];
    if (dt == 0.0 || j < 3 || !c->lev[j].n_leaf) continue;
    for (int b = 2; b <= j - 1; ++b) {  // scratch of the levels this tree reaches
      LevelTree& T = c->lev[b];
      cudaMemsetAsync(T.dS.ptr, 0, 8 * T.n_oct * nc * 8, st);
      cudaMemsetAsync(T.dQ.ptr, 0, 8 * T.n_oct * 4 * 8, st);
    }
    {
      LevelTree& J = c->lev[j];
      LevelTree& U = c->lev[j - 1];
      ++c->n_launch;
      k_drift_leaf<<<(unsigned)((J.n_oct * 32 + 255) / 256), 256, 0, st>>>(
          J.n_oct, nc, (const int32_t*)J.oct_parent.ptr, (const int32_t*)J.cell_child.ptr, (const double*)J.mass.ptr,
          (const double*)J.vel.ptr, alpha, (double*)U.dS.ptr, (double*)U.dQ.ptr);
    }
    for (int b = j - 2; b >= 2; --b) {
      LevelTree& N = c->lev[b + 1];
      LevelTree& T = c->lev[b];
      if (!N.n_oct) continue;
      ++c->n_launch;
      k_drift_m2m<<<(unsigned)N.n_oct, 128, 0, st>>>(
          nc, (const int32_t*)N.oct_parent.ptr, (const double*)N.dS.ptr, (const double*)N.dQ.ptr,
          (const int*)c->d_m2m_off.ptr, (const int*)c->d_m2m_g.ptr, (const int*)c->d_m2m_e.ptr,
          (const double*)c->d_m2m_c.ptr, (double*)T.dS.ptr, (double*)T.dQ.ptr);
    }
    for (int b = 2; b <= j - 1; ++b) {
      LevelTree& T = c->lev[b];
      const int64_t ncell = 8 * T.n_oct;
      if (!ncell) continue;
      const double dt_over_h = dt * std::ldexp(1.0, b);
      __nv_bfloat16* hi = f64 ? nullptr : (__nv_bfloat16*)T.Mhi.ptr;
      __nv_bfloat16* lo_ = (f64 || tf32) ? nullptr : (__nv_bfloat16*)T.Mlo.ptr;
      ++c->n_launch;
      if (T.m_is_f64)
        k_drift_apply<double><<<(unsigned)ncell, 128, 0, st>>>(ncell, nc, dt_over_h, alpha, (const double*)T.dS.ptr,
                                                              (const double*)T.dQ.ptr, (double*)T.M.ptr, hi, lo_);
      else
        k_drift_apply<float><<<(unsigned)ncell, 128, 0, st>>>(ncell, nc, dt_over_h, alpha, (const double*)T.dS.ptr,
                                                             (const double*)T.dQ.ptr, (float*)T.M.ptr, hi, lo_);
    }
  }
}

}  // namespace fmm
