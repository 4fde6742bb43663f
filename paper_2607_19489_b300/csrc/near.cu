// near.cu -- PotentialEvaluation (Alg. 4) for the leaf cells of one level:
// near and nearest fields (Sec. 3.2, Fig. 2), the far field by L2P from the
// level l-2 local expansion, plus the bottom intermediate field computed
// beforehand by the M2P contraction; scattered to the caller's order.
//
// For a target t at level l with parent F (level l-1), the sources are the
// 3^3 neighbours N of F:
//   * N a leaf of level l-1  -> P2P with N's mass at its centre, once;
//   * N refined: each child P (level l) of N
//       - leaf P != t          -> P2P;
//       - refined, touching t  -> P2P with P's 8 children (nearest field; the
//                                 graded rule makes them leaves);
//       - refined, not touching-> M2P from P's multipole (the merged tree
//                                 at FMM level l).
// Offsets are exact in level-l units (integers, halves and quarters).
#include "fmm_internal.cuh"

namespace fmm {
namespace {

template <typename T>
__device__ __forceinline__ T rsqrt_t(T x);
template <>
__device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ double rsqrt_t<double>(double x) { return 1.0 / sqrt(x); }

template <typename T>
__device__ __forceinline__ void p2p(T m, T dx, T dy, T dz, T& phi, T& ax, T& ay, T& az) {
  // d = source - target; phi += -m/|d|, accel += m d / |d|^3
  T r2 = dx * dx + dy * dy + dz * dz;
  T ir = rsqrt_t<T>(r2);
  T mir = m * ir;
  T mir3 = mir * ir * ir;
  phi -= mir;
  ax += mir3 * dx;
  ay += mir3 * dy;
  az += mir3 * dz;
}

struct NearParams {
  int level, nc;
  int64_t n_tgt;
  const int32_t* tgt;         // target octs (level l)
  const int32_t* nbr;         // [oct][27] level l
  const int32_t* cc_l;        // cell_child level l
  const int32_t* cc_up;       // cell_child level l-1 (unused)
  const int32_t* par_l;       // oct_parent level l
  const int32_t* par_up;      // oct_parent level l-1
  const double* mono_up;      // masses of level l-1 cells
  const double* mono_l;       // level l
  const double* mono_dn;      // level l+1
  const void* M_l;            // multipoles of level l cells
  int M_l_f64;
  const double* L2;           // local expansions of level l-2 (or null)
  const void* acc;            // M2P results for level l cells [cells][4]
  const void* nearop;         // [343][nc][4]
  const void* l2pop;          // [64][nc][4]
  double G, h;                // gravitational constant, cell size of level l
  void* phi;
  void* accel;
  int out_fp32;
};

template <typename T>
__global__ void __launch_bounds__(128) k_near(NearParams P) {
  const int64_t gi = (int64_t)blockIdx.x * 16 + (threadIdx.x >> 3);
  if (gi >= P.n_tgt) return;
  const int tp = threadIdx.x & 7;
  const int32_t o = P.tgt[gi];
  const int64_t cell = (int64_t)o * 8 + tp;
  const int32_t self = P.cc_l[cell];
  if (self >= 0) return;  // refined: not a target of this level
  const int tb[3] = {tp & 1, (tp >> 1) & 1, (tp >> 2) & 1};
  const T* nearop = (const T*)P.nearop;
  T phi = 0, ax = 0, ay = 0, az = 0;
  const int32_t* nb27 = P.nbr + (int64_t)o * 27;
  for (int q = 0; q < 27; ++q) {
    const int32_t nb = nb27[q];
    if (nb == -1) continue;
    const int dq[3] = {q % 3 - 1, (q / 3) % 3 - 1, q / 9 - 1};
    if (nb <= -2) {  // coarse leaf of level l-1: centre at 2 dq + 1 in level-l units
      const T m = (T)P.mono_up[-2 - (int64_t)nb];
      p2p<T>(m, (T)(2 * dq[0] - tb[0]) + (T)0.5, (T)(2 * dq[1] - tb[1]) + (T)0.5,
             (T)(2 * dq[2] - tb[2]) + (T)0.5, phi, ax, ay, az);
      continue;
    }
    for (int c = 0; c < 8; ++c) {
      const int rx = 2 * dq[0] + (c & 1) - tb[0];
      const int ry = 2 * dq[1] + ((c >> 1) & 1) - tb[1];
      const int rz = 2 * dq[2] + ((c >> 2) & 1) - tb[2];
      if ((rx | ry | rz) == 0) continue;
      const int64_t pc = (int64_t)nb * 8 + c;
      const int32_t ch = P.cc_l[pc];
      if (ch < 0) {
        p2p<T>((T)P.mono_l[pc], (T)rx, (T)ry, (T)rz, phi, ax, ay, az);
      } else if (abs(rx) <= 1 && abs(ry) <= 1 && abs(rz) <= 1) {
        // nearest field: the 8 children of the touching refined cell
        for (int k = 0; k < 8; ++k) {
          const T m = (T)P.mono_dn[(int64_t)ch * 8 + k];
          p2p<T>(m, (T)rx + (T)(((k & 1) * 2 - 1)) * (T)0.25, (T)ry + (T)((((k >> 1) & 1) * 2 - 1)) * (T)0.25,
                 (T)rz + (T)((((k >> 2) & 1) * 2 - 1)) * (T)0.25, phi, ax, ay, az);
        }
      } else {
        // near-field refined cell: M2P at integer offset R = t - P
        const int ridx = ((-rz + 3) * 7 + (-ry + 3)) * 7 + (-rx + 3);
        const T* op = nearop + (int64_t)ridx * P.nc * 4;
        if (P.M_l_f64) {
          const double* M = (const double*)P.M_l + pc * P.nc;
          for (int a = 0; a < P.nc; ++a) {
            T mv = (T)M[a];
            phi += op[4 * a] * mv;
            ax += op[4 * a + 1] * mv;
            ay += op[4 * a + 2] * mv;
            az += op[4 * a + 3] * mv;
          }
        } else {
          const float* M = (const float*)P.M_l + pc * P.nc;
          for (int a = 0; a < P.nc; ++a) {
            T mv = (T)M[a];
            phi += op[4 * a] * mv;
            ax += op[4 * a + 1] * mv;
            ay += op[4 * a + 2] * mv;
            az += op[4 * a + 3] * mv;
          }
        }
      }
    }
  }
  // bottom intermediate field (M2P, level l-1 units) and far field (L2P, level l-2 units)
  const T* acc = (const T*)P.acc;
  T pm = acc[cell * 4], xm = acc[cell * 4 + 1], ym = acc[cell * 4 + 2], zm = acc[cell * 4 + 3];
  T pl = 0, xl = 0, yl = 0, zl = 0;
  if (P.L2) {
    const int32_t F = P.par_l[o];
    const int32_t G2 = P.par_up[F >> 3];
    const int pos = (F & 7) * 8 + tp;
    const double* L = P.L2 + (int64_t)G2 * P.nc;
    const T* op = (const T*)P.l2pop + (int64_t)pos * P.nc * 4;
    for (int b = 0; b < P.nc; ++b) {
      T lb = (T)L[b];
      pl += op[4 * b] * lb;
      xl += op[4 * b + 1] * lb;
      yl += op[4 * b + 2] * lb;
      zl += op[4 * b + 3] * lb;
    }
  }
  const double s1 = P.G / P.h, s2 = P.G / (P.h * P.h);
  const double ph = s1 * ((double)phi + 0.5 * (double)pm + 0.25 * (double)pl);
  const double gx = s2 * ((double)ax + 0.25 * (double)xm + 0.0625 * (double)xl);
  const double gy = s2 * ((double)ay + 0.25 * (double)ym + 0.0625 * (double)yl);
  const double gz = s2 * ((double)az + 0.25 * (double)zm + 0.0625 * (double)zl);
  const int64_t li = -1 - (int64_t)self;
  if (P.out_fp32) {
    ((float*)P.phi)[li] = (float)ph;
    float* a = (float*)P.accel + 3 * li;
    a[0] = (float)gx;
    a[1] = (float)gy;
    a[2] = (float)gz;
  } else {
    ((double*)P.phi)[li] = ph;
    double* a = (double*)P.accel + 3 * li;
    a[0] = gx;
    a[1] = gy;
    a[2] = gz;
  }
}

}  // namespace

void launch_near(Ctx* c, int l, void* phi, void* accel, int out_fp32, cudaStream_t st) {
  LevelTree& T = c->lev[l];
  if (!T.n_tgt) return;
  const bool f64 = c->cfg.precision == FMM_FP64;
  NearParams P;
  P.level = l;
  P.nc = c->tab.nc;
  P.n_tgt = T.n_tgt;
  P.tgt = (const int32_t*)T.tgt.ptr;
  P.nbr = (const int32_t*)T.nbr.ptr;
  P.cc_l = (const int32_t*)T.cell_child.ptr;
  P.cc_up = (const int32_t*)c->lev[l - 1].cell_child.ptr;
  P.par_l = (const int32_t*)T.oct_parent.ptr;
  P.par_up = (const int32_t*)c->lev[l - 1].oct_parent.ptr;
  P.mono_up = (const double*)c->lev[l - 1].mono.ptr;
  P.mono_l = (const double*)T.mono.ptr;
  P.mono_dn = (l < c->lmax) ? (const double*)c->lev[l + 1].mono.ptr : nullptr;
  P.M_l = T.M.ptr;
  P.M_l_f64 = T.m_is_f64 ? 1 : 0;
  P.L2 = (l - 2 >= 2) ? (const double*)c->lev[l - 2].L.ptr : nullptr;
  P.acc = T.acc.ptr;
  P.nearop = f64 ? c->d_near64.ptr : c->d_near32.ptr;
  P.l2pop = f64 ? c->d_l2p64.ptr : c->d_l2p32.ptr;
  P.G = c->cfg.G;
  P.h = std::ldexp(1.0, -l);
  P.phi = phi;
  P.accel = accel;
  P.out_fp32 = out_fp32;
  unsigned grid = (unsigned)((T.n_tgt + 15) / 16);
  if (f64)
    ++c->n_launch;
    k_near<double><<<grid, 128, 0, st>>>(P);
  else
    ++c->n_launch;
    k_near<float><<<grid, 128, 0, st>>>(P);
}

}  // namespace fmm
