// upward.cu -- Upward pass (P2M, Eq. 1; M2M, Eq. 2; Alg. 2) and L2L (Eq. 4).
//
// Expansions are kept in box units (tables.h).  A leaf cell's multipole is its
// mass as a monopole; a refined cell's multipole is the M2M sum of its eight
// children.  Because the eight child offsets are (+-1/4)^3 of the parent box,
// M2M factors into a sign transform over the children,
//     S_e[gamma] = sum_c sign(c, e) Mt_c[gamma],  e in {0,1}^3,
// followed by one short sum per output coefficient alpha over gamma <= alpha
// with the sign pattern e = (alpha - gamma) mod 2.  L2L uses the same sign
// rule on the parent's local expansion.
//
// The multipole of a box equals the sum over all trees T_j of the paper's
// per-level multipoles (each tree holds the mass of one AMR level, and M2M is
// linear), which is the form the M2L and M2P sources need (the merged tree of
// Sec. 3.1 plus the tree of the target level).
#include "fmm_internal.cuh"

namespace fmm {
namespace {

constexpr int kNcMax = 168;  // ncoef(8) = 165

template <typename T>
__device__ __forceinline__ float to_f(T v) { return (float)v; }

template <typename Tin, typename Tacc, typename Tout>
__global__ void __launch_bounds__(192) k_upward(
    int nc, const int32_t* __restrict__ cell_child, const int32_t* __restrict__ cell_child_next,
    const Tin* __restrict__ Mnext, const double* __restrict__ mass_here,
    const double* __restrict__ mass_next, Tout* __restrict__ Mout, __nv_bfloat16* __restrict__ hi,
    __nv_bfloat16* __restrict__ lo, double* __restrict__ mono, const int* __restrict__ poff,
    const int* __restrict__ pg, const int* __restrict__ pe, const double* __restrict__ pc) {
  __shared__ Tacc Mc[8 * kNcMax];
  __shared__ Tacc S[8 * kNcMax];
  const int64_t cell = blockIdx.x;
  const int a = threadIdx.x;
  const int32_t ch = cell_child[cell];
  if (ch < 0) {  // leaf: monopole = mass (P2M of a single point mass at the cell centre)
    Tout m = (Tout)mass_here[-1 - (int64_t)ch];
    for (int k = a; k < nc; k += blockDim.x) {
      Tout v = (k == 0) ? m : (Tout)0;
      Mout[cell * nc + k] = v;
      if (hi) {
        float f = to_f(v);
        __nv_bfloat16 h = __float2bfloat16_rn(f);
        hi[cell * nc + k] = h;
        lo[cell * nc + k] = __float2bfloat16_rn(f - __bfloat162float(h));
      }
    }
    if (a == 0) mono[cell] = (double)m;
    return;
  }
  const int64_t c0 = (int64_t)ch * 8;
  for (int idx = a; idx < 8 * nc; idx += blockDim.x) {
    int c = idx / nc, g = idx - c * nc;
    int32_t cc = cell_child_next[c0 + c];
    Tacc v;
    if (cc < 0)
      v = (g == 0) ? (Tacc)mass_next[-1 - (int64_t)cc] : (Tacc)0;
    else
      v = (Tacc)Mnext[(c0 + c) * nc + g];
    Mc[c * nc + g] = v;
  }
  __syncthreads();
  for (int g = a; g < nc; g += blockDim.x) {
    Tacc x[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = Mc[c * nc + g];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      Tacc s = 0;
#pragma unroll
      for (int c = 0; c < 8; ++c) s += (child_sign(c, e) > 0) ? x[c] : -x[c];
      S[e * nc + g] = s;
    }
  }
  __syncthreads();
  for (int k = a; k < nc; k += blockDim.x) {
    Tacc out = 0;
    for (int j = poff[k]; j < poff[k + 1]; ++j) out += (Tacc)pc[j] * S[pe[j] * nc + pg[j]];
    Tout v = (Tout)out;
    Mout[cell * nc + k] = v;
    if (hi) {
      float f = to_f(v);
      __nv_bfloat16 h = __float2bfloat16_rn(f);
      hi[cell * nc + k] = h;
      lo[cell * nc + k] = __float2bfloat16_rn(f - __bfloat162float(h));
    }
    if (k == 0) mono[cell] = (double)v;
  }
}

__global__ void k_mono_leaves(int64_t ncell, const int32_t* __restrict__ cell_child,
                              const double* __restrict__ mass, double* __restrict__ mono) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= ncell) return;
  int32_t ch = cell_child[i];
  mono[i] = (ch < 0) ? mass[-1 - (int64_t)ch] : 0.0;
}

// L2L into the 8 cells of each row oct of level b from its parent cell (b-1).
__global__ void __launch_bounds__(256) k_l2l(int nc, int64_t n_rows, const int32_t* __restrict__ rows,
                                             const int32_t* __restrict__ oct_parent,
                                             const double* __restrict__ Lup, double* __restrict__ L,
                                             const int* __restrict__ poff, const int* __restrict__ pg,
                                             const int* __restrict__ pe, const double* __restrict__ pc) {
  __shared__ double Lp[kNcMax];
  int64_t r = blockIdx.x;
  if (r >= n_rows) return;
  int32_t o = rows[r];
  int32_t par = oct_parent[o];
  for (int k = threadIdx.x; k < nc; k += blockDim.x) Lp[k] = Lup[(int64_t)par * nc + k];
  __syncthreads();
  for (int idx = threadIdx.x; idx < 8 * nc; idx += blockDim.x) {
    int c = idx / nc, b = idx - c * nc;
    double s = 0.0;
    for (int j = poff[b]; j < poff[b + 1]; ++j) s += pc[j] * (double)child_sign(c, pe[j]) * Lp[pg[j]];
    L[((int64_t)o * 8 + c) * nc + b] = s;
  }
}

}  // namespace

void launch_mono_leaves(Ctx* c, int l, cudaStream_t st) {
  LevelTree& T = c->lev[l];
  int64_t n = 8 * T.n_oct;
  if (!n) return;
  unsigned g = (unsigned)((n + 255) / 256);
  ++c->n_launch;
  k_mono_leaves<<<g, 256, 0, st>>>(n, (const int32_t*)T.cell_child.ptr, (const double*)T.mass.ptr,
                                   (double*)T.mono.ptr);
}

void launch_upward(Ctx* c, int b, cudaStream_t st) {
  LevelTree& T = c->lev[b];
  LevelTree& N = c->lev[b + 1];
  int64_t ncell = (b == 0) ? 1 : 8 * T.n_oct;
  if (!ncell) return;
  const int nc = c->tab.nc;
  const int* poff = (const int*)c->d_m2m_off.ptr;
  const int* pg = (const int*)c->d_m2m_g.ptr;
  const int* pe = (const int*)c->d_m2m_e.ptr;
  const double* pc = (const double*)c->d_m2m_c.ptr;
  int threads = ((nc + 31) / 32) * 32;
  if (threads > 192) threads = 192;
  dim3 grid((unsigned)ncell);
  const int32_t* cc = (const int32_t*)T.cell_child.ptr;
  const int32_t* ccn = (const int32_t*)N.cell_child.ptr;
  const double* mh = (const double*)T.mass.ptr;
  const double* mn = (const double*)N.mass.ptr;
  __nv_bfloat16* hi = (__nv_bfloat16*)T.Mhi.ptr;
  __nv_bfloat16* lo = (__nv_bfloat16*)T.Mlo.ptr;
  if (T.m_is_f64) {
    if (N.m_is_f64)
      ++c->n_launch;
      k_upward<double, double, double><<<grid, threads, 0, st>>>(nc, cc, ccn, (const double*)N.M.ptr, mh, mn,
                                                                 (double*)T.M.ptr, hi, lo, (double*)T.mono.ptr,
                                                                 poff, pg, pe, pc);
    else
      ++c->n_launch;
      k_upward<float, double, double><<<grid, threads, 0, st>>>(nc, cc, ccn, (const float*)N.M.ptr, mh, mn,
                                                                (double*)T.M.ptr, hi, lo, (double*)T.mono.ptr,
                                                                poff, pg, pe, pc);
  } else {
    ++c->n_launch;
    k_upward<float, float, float><<<grid, threads, 0, st>>>(nc, cc, ccn, (const float*)N.M.ptr, mh, mn,
                                                            (float*)T.M.ptr, hi, lo, (double*)T.mono.ptr, poff,
                                                            pg, pe, pc);
  }
}

void launch_l2l(Ctx* c, int b, cudaStream_t st) {
  LevelTree& T = c->lev[b];
  if (!T.n_rows) return;
  ++c->n_launch;
  k_l2l<<<(unsigned)T.n_rows, 256, 0, st>>>(c->tab.nc, T.n_rows, (const int32_t*)T.rows.ptr,
                                            (const int32_t*)T.oct_parent.ptr, (const double*)c->lev[b - 1].L.ptr,
                                            (double*)T.L.ptr, (const int*)c->d_l2l_off.ptr,
                                            (const int*)c->d_l2l_g.ptr, (const int*)c->d_l2l_e.ptr,
                                            (const double*)c->d_l2l_c.ptr);
}

}  // namespace fmm
