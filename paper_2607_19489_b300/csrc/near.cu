// near.cu -- PotentialEvaluation (Alg. 4) for the leaf cells of the target
// levels: near and nearest fields (Sec. 3.2, Fig. 2), the far field by L2P from
// the level l-2 local expansion, plus the bottom intermediate field computed
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
//
// Layout: 8 threads per target oct (one per cell), OPB octs per block, all
// target levels in one launch (a segment per level).  The 216 source cells of
// an oct are staged once in shared memory: their masses (zero for anything
// that is not a level-l leaf) and a short list of the coarse-leaf and refined
// entries, which only occur next to coarse-fine interfaces.  The kernel is
// bound by the latency of its loads, so they are issued in as few dependent
// rounds as possible: the tree data (target oct, its 27 neighbours, their leaf
// masks, the row of its local expansion) before the wait on the previous
// kernel, then every mass, the M2P accumulator and the local expansion at
// once, each neighbour oct's eight masses with two 16-byte loads.  The P2P
// loop is then branch-free.  The local expansion of the oct's level l-2 box
// (bottom mode 1: of its parent box, level l-1) is evaluated directly,
// phi = sum_beta L_beta rho^beta / beta!.
#include <utility>

#include "fmm_internal.cuh"

namespace fmm {
namespace {

constexpr int kNcMax = 168;  // ncoef(8) = 165
constexpr int kMaxNearSeg = 8;  // levels per launch (keeps the parameter block ~1 KB)

// Source positions relative to the target oct's origin, level-l units:
// cell c of neighbour slot q sits at 2 dq + bits(c) (its lower corner; the
// target uses the same convention, so differences are centre differences).
__constant__ float c_src_pos[216][3];
// index of the multi-index (a,b,c) in the graded order, a,b,c <= 8
__constant__ int16_t c_lut[9][9][9];
// 1/(k+1) in each precision (an FP32 table would limit the FP64 path to 1e-8)
__constant__ float c_inv_f[9] = {1.f, 1.f / 2, 1.f / 3, 1.f / 4, 1.f / 5, 1.f / 6, 1.f / 7, 1.f / 8, 1.f / 9};
__constant__ double c_inv_d[9] = {1.0, 1.0 / 2, 1.0 / 3, 1.0 / 4, 1.0 / 5, 1.0 / 6, 1.0 / 7, 1.0 / 8, 1.0 / 9};
template <typename T>
__device__ __forceinline__ T inv_k(int k);
template <>
__device__ __forceinline__ float inv_k<float>(int k) { return c_inv_f[k]; }
template <>
__device__ __forceinline__ double inv_k<double>(int k) { return c_inv_d[k]; }

template <typename T>
__device__ __forceinline__ T rsqrt_t(T x);
template <>
__device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ double rsqrt_t<double>(double x) { return 1.0 / sqrt(x); }

// float -> double by the IEEE-754 encodings (sign, exponent rebiased by
// 1023 - 127, mantissa shifted by 52 - 23), exact for every normal value, zero,
// inf and NaN; FP32 subnormals are flushed anyway (--ftz).  B300 runs the
// hardware conversion on the FP64 pipe, which is what this avoids.
__device__ __forceinline__ double widen(float x) {
  const uint32_t u = __float_as_uint(x);
  const uint32_t e = (u >> 23) & 0xFFu;
  const uint64_t sign = (uint64_t)(u >> 31) << 63;
  const uint64_t ex = e == 0 ? 0ull : (e == 0xFFu ? 0x7FFull : (uint64_t)(e + 896u));
  const uint64_t man = e == 0 ? 0ull : (uint64_t)(u & 0x7FFFFFu) << 29;
  return __longlong_as_double((long long)(sign | (ex << 52) | man));
}
__device__ __forceinline__ double widen(double x) { return x; }

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

struct NearSeg {
  const int32_t* tgt;         // target octs (level l)
  const int32_t* nbr;         // [oct][27] level l
  const int32_t* cc_l;        // cell_child level l
  const int32_t* par_l;       // oct_parent level l
  const void* mono_up;        // masses of level l-1 cells (in the kernel's precision)
  const void* mono_l;         // level l
  const void* mono_dn;        // level l+1
  const void* M_l;            // multipoles of level l cells
  const void* L2;             // local expansions of level l-2 (bottom mode 1: l-1), or null,
                              // by slot, in T
  const int32_t* lslot;       // [oct of level l]: row of L2 its cells evaluate, or -1
  const uint8_t* leafmask;    // level l: bit c set when cell c of the oct is a leaf
  void* acc;                  // M2P results for level l cells [cells][4]; cleared after reading
  void* phi;
  void* accel;
  double s1, s2;              // G / h and G / h^2, h the cell size of level l
  float s1f, s2f;             // the same in FP32
  int64_t n_tgt;
  int blk0;                   // first block of this segment
  int M_l_f64;
};

struct NearParams {
  NearSeg seg[kMaxNearSeg];
  int nseg, nc, p, out_fp32;
  int bottom1;                // bottom mode 1: far field from the parent box (level l-1)
  const void* nearop;         // [343][nc][4]
  double G;
};

// Index of the multi-index (a,b,c) in the graded order (degree, a descending,
// b descending), for compile-time evaluation.
__host__ __device__ constexpr int gidx(int a, int b, int c) {
  return (a + b + c) * (a + b + c + 1) * (a + b + c + 2) / 6 + (b + c) * (b + c + 1) / 2 + c;
}

// ---- FP32 lattice pairs with compile-time coefficients -------------------------
// The 216 lattice sources of a target at position t of its oct sit at offsets
// i - 2 - t (level-l cells, i = 0..5 per axis).  Mirroring an axis on which t's
// bit is set maps the offset (i - 2) - 1 to -((5 - i) - 2): every position's
// pair geometry is position 0's, read at mirrored source slots, with the
// mirrored force components negated at the end.  One unrolled pair loop then
// serves every position with position 0's coefficients (-1/r and d/r^3) as
// compile-time constants: a pair costs an address add, one shared-memory load
// and four FFMAs, and no reciprocal square root.
__host__ __device__ constexpr double lat_sqrt(double n) {  // Newton's iteration for sqrt, n >= 1
  double x = n;
  for (int i = 0; i < 64; ++i) x = 0.5 * (x + n / x);
  return x;
}

template <int S>  // lattice source S = ix + 6 iy + 36 iz, seen from position 0
struct LatPair {
  static constexpr int ix = S % 6, iy = (S / 6) % 6, iz = S / 36;
  static constexpr int dx = ix - 2, dy = iy - 2, dz = iz - 2;
  static constexpr int r2 = dx * dx + dy * dy + dz * dz;
  static constexpr double ir = r2 ? 1.0 / lat_sqrt((double)r2) : 0.0;
  static constexpr double ir3 = ir * ir * ir;
  static constexpr float kp = (float)(-ir);
  static constexpr float kx = (float)(dx * ir3), ky = (float)(dy * ir3), kz = (float)(dz * ir3);
};

// The pairs of one target, seen from position 0 through the mirrors of its own
// position: load(slot) returns the mass at a lattice slot of the target's oct.
// The x mirror MX is the same for a whole warp (the threads are laid out so),
// which makes the x part of every slot a compile-time offset from the row base
// (iy, iz): one add per six pairs, the loads take immediate offsets.
template <int MX, int S, typename Load>
__device__ __forceinline__ void lat_pair(const Load& load, const int (&AY)[6], const int (&AZ)[6],
                                         float (&a)[2][4]) {
  using Q = LatPair<S>;
  if constexpr (Q::r2 != 0) {  // the target itself is not a source
    constexpr int jx = MX ? 5 - Q::ix : Q::ix;
    constexpr int ox = 8 * (jx >> 1) + (jx & 1);
    const float m = load((AY[Q::iy] + AZ[Q::iz]) + ox);
    float* r = a[S & 1];  // two accumulator sets: shorter FFMA dependency chains
    r[0] = fmaf(m, Q::kp, r[0]);
    r[1] = fmaf(m, Q::kx, r[1]);
    r[2] = fmaf(m, Q::ky, r[2]);
    r[3] = fmaf(m, Q::kz, r[3]);
  }
}

template <int MX, typename Load, int... S>
__device__ __forceinline__ void lat_all(std::integer_sequence<int, S...>, const Load& load, const int (&AY)[6],
                                        const int (&AZ)[6], float (&a)[2][4]) {
  (lat_pair<MX, S>(load, AY, AZ, a), ...);
}


// PC > 0: expansion order known at compile time (the L2P loops unroll); 0: runtime P.p.
// Eight consecutive values (one oct's cells) with 16-byte loads; p is 32-byte
// aligned (an oct's row in a 256-byte aligned buffer).
__device__ __forceinline__ void load8(const float* p, float (&m)[8]) {
  const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
  m[0] = a.x; m[1] = a.y; m[2] = a.z; m[3] = a.w; m[4] = b.x; m[5] = b.y; m[6] = b.z; m[7] = b.w;
}
__device__ __forceinline__ void load8(const double* p, double (&m)[8]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double2 a = reinterpret_cast<const double2*>(p)[k];
    m[2 * k] = a.x;
    m[2 * k + 1] = a.y;
  }
}
__device__ __forceinline__ void load4(const float* p, float& a, float& b, float& c, float& d) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  a = v.x; b = v.y; c = v.z; d = v.w;
}
__device__ __forceinline__ void load4(const double* p, double& a, double& b, double& c, double& d) {
  const double2 u = reinterpret_cast<const double2*>(p)[0], v = reinterpret_cast<const double2*>(p)[1];
  a = u.x; b = u.y; c = v.x; d = v.y;
}

// Thread layout: a pair of warps serves 8 target octs, warp 2k + x holding the
// targets at x-position x of octs 8k..8k+7, lane 4 m + 2 y + z the target at
// (x, y, z) of oct 8k + m.  The x mirror of the pair loop is then uniform per
// warp.  For staging, thread ts = 4 x + (lane & 3) of an oct (0..7) owns the
// neighbour slots q = ts + 8 j; each half (x = 0, 1) keeps its own list of
// coarse-leaf / refined entries.  OPB (octs per block) is 8 or 16.
// FP32: 896 threads per SM.
template <typename T, int OPB, int PC>
__global__ void __launch_bounds__(8 * OPB, sizeof(T) == 4 ? 112 / OPB : 1) k_near(const __grid_constant__ NearParams P) {
  static_assert(OPB % 8 == 0, "a warp pair serves eight octs");
  __shared__ __align__(16) T s_m[OPB][216];
  // local expansion of the oct's level l-2 box (rows of ncoef(PC) when the order is fixed)
  constexpr int kNcL = PC > 0 ? (PC + 1) * (PC + 2) * (PC + 3) / 6 : kNcMax;
  __shared__ __align__(16) T s_L[OPB][kNcL];
  __shared__ int32_t s_nb[OPB][28];        // the 27 neighbour slots of the oct
  constexpr int kSpecHalf = 15 * 8;        // a half owns at most 15 slots
  __shared__ uint8_t s_spec[OPB][2][kSpecHalf];  // source slots that are coarse leaves or refined cells
  __shared__ int s_nspec[OPB][2];
  int si = 0;
  while (si + 1 < P.nseg && (int)blockIdx.x >= P.seg[si + 1].blk0) ++si;
  const NearSeg& S = P.seg[si];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tbx = warp & 1, tby = (lane >> 1) & 1, tbz = lane & 1;
  const int g = (warp >> 1) * 8 + (lane >> 2);  // oct in the block
  const int tp = tbx + 2 * tby + 4 * tbz;       // target position in the oct
  const int ts = 4 * tbx + (lane & 3);          // staging index in the oct
  const int64_t gi = (int64_t)(blockIdx.x - S.blk0) * OPB + g;
  const bool oct_ok = gi < S.n_tgt;
  // ---- tree data (written by the tree build, before this solve): read before
  // the wait on the previous kernel, all in three dependent rounds ----
  const int32_t o = oct_ok ? S.tgt[gi] : 0;
  const int64_t cell = (int64_t)o * 8 + tp;
  // thread ts owns neighbour slots q = ts + 8 j (j < 4, q < 27)
  int32_t nbq[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int q = ts + 8 * j;
    nbq[j] = (oct_ok && q < 27) ? S.nbr[(int64_t)o * 27 + q] : -1;
  }
  const int32_t self = oct_ok ? S.cc_l[cell] : 0;
  const int32_t lrow = (oct_ok && S.L2) ? S.lslot[o] : -1;
  const int fpos = (oct_ok && S.L2 && !P.bottom1) ? (S.par_l[o] & 7) : 0;
  unsigned lm[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) lm[j] = nbq[j] >= 0 ? (unsigned)S.leafmask[nbq[j]] : 0xFFu;
  // entries of the coarse-leaf / refined lists: refined cells of each level-l
  // neighbour oct, one per level l-1 leaf; placed by an exclusive scan over
  // the half's four lanes (a fixed order)
  int cnt = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) cnt += nbq[j] >= 0 ? 8 - __popc(lm[j]) : (nbq[j] <= -2 ? 1 : 0);
  int incl = cnt;
#pragma unroll
  for (int d = 1; d < 4; d <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, d, 4);
    if ((lane & 3) >= d) incl += y;
  }
  int pos = incl - cnt;
  if ((lane & 3) == 3) s_nspec[g][tbx] = incl;
  pdl_wait();
  pdl_trigger();
  // ---- masses, the M2P accumulator and the local expansion (this solve) ----
  const T* mono_l = (const T*)S.mono_l;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int q = ts + 8 * j;
    if (q >= 27) break;
    const int32_t nb = nbq[j];
    T m[8];
    if (nb >= 0) {
      load8(mono_l + (int64_t)nb * 8, m);
#pragma unroll
      for (int cc = 0; cc < 8; ++cc) {
        if ((lm[j] >> cc) & 1) continue;
        m[cc] = (T)0;  // a refined cell: nearest field or near-field M2P
        s_spec[g][tbx][pos++] = (uint8_t)(q * 8 + cc);
      }
    } else {
#pragma unroll
      for (int cc = 0; cc < 8; ++cc) m[cc] = (T)0;
      if (nb <= -2) s_spec[g][tbx][pos++] = (uint8_t)(q * 8);  // a level l-1 leaf, once
    }
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) s_m[g][q * 8 + cc] = m[cc];
    s_nb[g][q] = nb;
  }
  T pm = 0, xm = 0, ym = 0, zm = 0;
  if (oct_ok && self < 0) load4((const T*)S.acc + cell * 4, pm, xm, ym, zm);
  if (lrow >= 0)
    for (int b = ts; b < P.nc; b += 8) s_L[g][b] = ((const T*)S.L2)[(int64_t)lrow * P.nc + b];
  __syncthreads();
  if (!oct_ok) return;
  if (self >= 0) return;  // refined: not a target of this level
  const T tx = (T)tbx, ty = (T)tby, tz = (T)tbz;
  T phi = 0, ax = 0, ay = 0, az = 0;
  // ---- P2P with the level-l leaves of the 3^3 neighbour octs ----
  // Source cell c of slot q has its lower corner at 2 dq + bits(c); relative to
  // the target that is i - 2 - t along each axis, i = 2 (dq+1) + bit in 0..5.
  // With both loops unrolled the six offsets per axis live in registers.
  if constexpr (sizeof(T) == 4) {
    // FP32: position 0's pairs at this position's mirrored slots, compile-time
    // coefficients (see LatPair); slot of lattice index j = 2 q + bit per axis:
    // 8 (9 qz + 3 qy + qx) + 4 bz + 2 by + bx
    int AY[6], AZ[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const int jy = tby ? 5 - i : i, jz = tbz ? 5 - i : i;
      AY[i] = 24 * (jy >> 1) + 2 * (jy & 1);
      AZ[i] = 72 * (jz >> 1) + 4 * (jz & 1);
    }
    float a[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    auto load = [&](int slot) { return (float)s_m[g][slot]; };  // indexed directly: shared-memory loads
    if (tbx)  // warp-uniform
      lat_all<1>(std::make_integer_sequence<int, 216>{}, load, AY, AZ, a);
    else
      lat_all<0>(std::make_integer_sequence<int, 216>{}, load, AY, AZ, a);
    phi = (T)(a[0][0] + a[1][0]);
    ax = (T)(tbx ? -(a[0][1] + a[1][1]) : a[0][1] + a[1][1]);
    ay = (T)(tby ? -(a[0][2] + a[1][2]) : a[0][2] + a[1][2]);
    az = (T)(tbz ? -(a[0][3] + a[1][3]) : a[0][3] + a[1][3]);
  } else {
  T X[6], Y[6], Z[6], X2[6], Y2[6], Z2[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    X[i] = (T)(i - 2) - tx;
    Y[i] = (T)(i - 2) - ty;
    Z[i] = (T)(i - 2) - tz;
    X2[i] = X[i] * X[i];
    Y2[i] = Y[i] * Y[i];
    Z2[i] = Z[i] * Z[i];
  }
#pragma unroll
  for (int q = 0; q < 27; ++q) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int ix = 2 * (q % 3) + (c & 1), iy = 2 * ((q / 3) % 3) + ((c >> 1) & 1),
                iz = 2 * (q / 9) + ((c >> 2) & 1);
      T m = s_m[g][q * 8 + c];  // indexed directly so the compiler emits shared-memory loads
      T r2 = X2[ix] + Y2[iy] + Z2[iz];
      if (q == 13) {  // the target's own oct: skip the self term
        const bool me = (c == tp);
        m = me ? (T)0 : m;
        r2 = me ? (T)1 : r2;
      }
      const T ir = rsqrt_t<T>(r2);
      const T mir = m * ir;
      const T mir3 = mir * (ir * ir);
      phi -= mir;
      ax += mir3 * X[ix];
      ay += mir3 * Y[iy];
      az += mir3 * Z[iz];
    }
  }
  }
  // ---- coarse leaves and refined cells (coarse-fine interfaces only) ----
  const int nspec0 = s_nspec[g][0], nspec = nspec0 + s_nspec[g][1];
  for (int k = 0; k < nspec; ++k) {
    const int s = k < nspec0 ? s_spec[g][0][k] : s_spec[g][1][k - nspec0];
    const int32_t nb = s_nb[g][s >> 3];
    if (nb <= -2) {  // coarse leaf of level l-1: centre at 2 dq + 1
      const T m = ((const T*)S.mono_up)[-2 - (int64_t)nb];
      p2p<T>(m, (T)c_src_pos[s][0] + (T)0.5 - tx, (T)c_src_pos[s][1] + (T)0.5 - ty,
             (T)c_src_pos[s][2] + (T)0.5 - tz, phi, ax, ay, az);
      continue;
    }
    const int64_t pc = (int64_t)nb * 8 + (s & 7);
    const int rx = (int)c_src_pos[s][0] - tbx;
    const int ry = (int)c_src_pos[s][1] - tby;
    const int rz = (int)c_src_pos[s][2] - tbz;
    if (abs(rx) <= 1 && abs(ry) <= 1 && abs(rz) <= 1) {
      // nearest field: the 8 children of the touching refined cell
      const int32_t ch = S.cc_l[pc];
      for (int kk = 0; kk < 8; ++kk) {
        const T m = ((const T*)S.mono_dn)[(int64_t)ch * 8 + kk];
        p2p<T>(m, (T)rx + (T)((kk & 1) * 2 - 1) * (T)0.25, (T)ry + (T)(((kk >> 1) & 1) * 2 - 1) * (T)0.25,
               (T)rz + (T)(((kk >> 2) & 1) * 2 - 1) * (T)0.25, phi, ax, ay, az);
      }
    }
    // refined cells not touching t: M2P, done beforehand by k_near_m2p into acc
  }
  // ---- bottom intermediate field (M2P, level l-1 units) and far field (L2P, level l-2 units)
  T* acc = (T*)S.acc;
  // the accumulator (read above) is zero between solves: the contractions add into it next time
  acc[cell * 4] = (T)0;
  acc[cell * 4 + 1] = (T)0;
  acc[cell * 4 + 2] = (T)0;
  acc[cell * 4 + 3] = (T)0;
  T pl = 0, xl = 0, yl = 0, zl = 0;
  if (lrow >= 0) {
    // phi = sum_beta L_beta rho^beta / beta!, grad_i = sum_gamma L_{gamma+e_i} rho^gamma / gamma!,
    // rho = target - box centre in units of the level l-2 box (mode 1: of the
    // level l-1 box, where the target sits at +-1/4)
    const T q = P.bottom1 ? (T)0.5 : (T)0.25, q0 = P.bottom1 ? (T)0.25 : (T)0.375;
    const T rx = (T)(2 * (fpos & 1) + tbx) * q - q0;
    const T ry = (T)(2 * ((fpos >> 1) & 1) + tby) * q - q0;
    const T rz = (T)(2 * ((fpos >> 2) & 1) + tbz) * q - q0;
    // s_L indexed directly (a plain pointer into it compiles to generic loads)
    if constexpr (PC > 0) {
      T xa = 1;
#pragma unroll
      for (int a = 0; a <= PC; ++a) {
        T xy = xa;
#pragma unroll
        for (int b = 0; a + b <= PC; ++b) {
          T m = xy;
#pragma unroll
          for (int cz = 0; a + b + cz <= PC; ++cz) {
            pl += s_L[g][gidx(a, b, cz)] * m;
            if (a + b + cz < PC) {
              xl -= s_L[g][gidx(a + 1, b, cz)] * m;
              yl -= s_L[g][gidx(a, b + 1, cz)] * m;
              zl -= s_L[g][gidx(a, b, cz + 1)] * m;
            }
            m *= rz * (T)(1.0 / (cz + 1));
          }
          xy *= ry * (T)(1.0 / (b + 1));
        }
        xa *= rx * (T)(1.0 / (a + 1));
      }
    } else {
    const int p = P.p;
    T xa = 1;
    for (int a = 0; a <= p; ++a) {
      T xy = xa;
      for (int b = 0; a + b <= p; ++b) {
        T m = xy;
        for (int cz = 0; a + b + cz <= p; ++cz) {
          pl += s_L[g][c_lut[a][b][cz]] * m;
          if (a + b + cz < p) {
            xl -= s_L[g][c_lut[a + 1][b][cz]] * m;
            yl -= s_L[g][c_lut[a][b + 1][cz]] * m;
            zl -= s_L[g][c_lut[a][b][cz + 1]] * m;
          }
          m *= rz * inv_k<T>(cz);
        }
        xy *= ry * inv_k<T>(b);
      }
      xa *= rx * inv_k<T>(a);
    }
    }
  }
  // level-l units: the M2P sum is in level l-1 units, the local expansion in level l-2
  // units (mode 1: l-1)
  const T fl1 = P.bottom1 ? (T)0.5 : (T)0.25, fl2 = P.bottom1 ? (T)0.25 : (T)0.0625;
  T s1, s2;
  if constexpr (sizeof(T) == 4) {
    s1 = S.s1f;
    s2 = S.s2f;
  } else {
    s1 = S.s1;
    s2 = S.s2;
  }
  const T ph = s1 * (phi + (T)0.5 * pm + fl1 * pl);
  const T gx = s2 * (ax + (T)0.25 * xm + fl2 * xl);
  const T gy = s2 * (ay + (T)0.25 * ym + fl2 * yl);
  const T gz = s2 * (az + (T)0.25 * zm + fl2 * zl);
  const int64_t li = -1 - (int64_t)self;
  if (P.out_fp32) {
    ((float*)S.phi)[li] = (float)ph;
    float* a = (float*)S.accel + 3 * li;
    a[0] = (float)gx;
    a[1] = (float)gy;
    a[2] = (float)gz;
  } else {
    ((double*)S.phi)[li] = widen(ph);
    double* a = (double*)S.accel + 3 * li;
    a[0] = widen(gx);
    a[1] = widen(gy);
    a[2] = widen(gz);
  }
}



// Near-field M2P (Fig. 2: "M2P from the merged tree at FMM level l") for the
// target octs that have refined cells among their 3^3 neighbour octs: one warp
// per oct.  The refined cells are listed with a ballot, each one's multipole is
// staged in shared memory, and lane 4t + j sums phi and accel of target t over
// the coefficients alpha = j, j+4, ... with float4 loads of the [R][alpha][4]
// operator.  Cells touching t are left to the nearest field.  The result is
// added to the M2P accumulator of the target (level l-1 units: x2, x4).
struct NearM2PSeg {
  const int32_t* irows;
  const int32_t* nbr;
  const int32_t* cc_l;
  const void* M_l;
  void* acc;
  int64_t n;
  int blk0, M_l_f64;
};
struct NearM2PParams {
  NearM2PSeg seg[kMaxNearSeg];
  int nseg, nc;
  const void* nearop;
};

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
  using type = float4;
};
template <>
struct Vec4<double> {
  using type = double4;
};

// One block of 8 warps per interface oct: warp 0 lists the refined cells, the
// warps take every 8th cell, and the partial sums of the 8 targets are reduced
// through shared memory at the end.
template <typename T>
__global__ void __launch_bounds__(256) k_near_m2p(const __grid_constant__ NearM2PParams P) {
  pdl_wait();
  pdl_trigger();
  __shared__ int16_t s_list[216];
  __shared__ int s_cnt;
  __shared__ int32_t s_nb[27];
  __shared__ T s_M[8][kNcMax];
  __shared__ T s_part[8][32][4];
  int si = 0;
  while (si + 1 < P.nseg && (int)blockIdx.x >= P.seg[si + 1].blk0) ++si;
  const NearM2PSeg& S = P.seg[si];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t gi = (int64_t)(blockIdx.x - S.blk0);
  if (gi >= S.n) return;  // whole block
  const int32_t o = S.irows[gi];
  if (threadIdx.x < 27) s_nb[threadIdx.x] = S.nbr[(int64_t)o * 27 + threadIdx.x];
  __syncthreads();
  if (w == 0) {  // list the refined cells of the 27 neighbour octs
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
  const int cnt = s_cnt;
  const int t = lane >> 2, j = lane & 3;
  const int tbx = t & 1, tby = (t >> 1) & 1, tbz = (t >> 2) & 1;
  const int nc = P.nc;
  using V4 = typename Vec4<T>::type;
  T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  for (int k = w; k < cnt; k += 8) {
    const int s = s_list[k];
    const int q = s >> 3, cc = s & 7;
    const int64_t pc = (int64_t)s_nb[q] * 8 + cc;
    if (S.M_l_f64)
      for (int a = lane; a < nc; a += 32) s_M[w][a] = (T)((const double*)S.M_l)[pc * nc + a];
    else
      for (int a = lane; a < nc; a += 32) s_M[w][a] = (T)((const float*)S.M_l)[pc * nc + a];
    __syncwarp();
    // R = t - P in level-l units (lower corners: P at 2 dq + bits(cc))
    const int rx = tbx - (2 * (q % 3 - 1) + (cc & 1));
    const int ry = tby - (2 * ((q / 3) % 3 - 1) + ((cc >> 1) & 1));
    const int rz = tbz - (2 * (q / 9 - 1) + ((cc >> 2) & 1));
    if (abs(rx) > 1 || abs(ry) > 1 || abs(rz) > 1) {
      const int ridx = ((rz + 3) * 7 + (ry + 3)) * 7 + (rx + 3);
      const V4* op = (const V4*)((const T*)P.nearop + (int64_t)ridx * nc * 4);
#pragma unroll 4
      for (int a = j; a < nc; a += 4) {
        const T mv = s_M[w][a];
        const V4 o4 = op[a];
        a0 += o4.x * mv;
        a1 += o4.y * mv;
        a2 += o4.z * mv;
        a3 += o4.w * mv;
      }
    }
    __syncwarp();
  }
  // sum the four coefficient phases of each target, then the eight warps
#pragma unroll
  for (int d = 1; d < 4; d <<= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, d);
    a1 += __shfl_xor_sync(0xffffffffu, a1, d);
    a2 += __shfl_xor_sync(0xffffffffu, a2, d);
    a3 += __shfl_xor_sync(0xffffffffu, a3, d);
  }
  s_part[w][lane][0] = a0;
  s_part[w][lane][1] = a1;
  s_part[w][lane][2] = a2;
  s_part[w][lane][3] = a3;
  __syncthreads();
  if (threadIdx.x < 32) {  // thread 4t + comp
    const int tt = threadIdx.x >> 2, comp = threadIdx.x & 3;
    T v = 0;
    for (int ww = 0; ww < 8; ++ww) v += s_part[ww][tt * 4][comp];
    const int64_t cell = (int64_t)o * 8 + tt;
    // atomic: in the mixed path the bottom M2P may be adding into the same cells concurrently
    if (S.cc_l[cell] < 0) atomicAdd((T*)S.acc + cell * 4 + comp, (comp == 0 ? (T)2 : (T)4) * v);
  }
}

}  // namespace

fmm_status near_init(Ctx* c) {
  int16_t lut[9][9][9];
  {
    int k = 0;
    for (int n = 0; n <= 24; ++n)
      for (int a = n; a >= 0; --a)
        for (int b = n - a; b >= 0; --b) {
          int cc = n - a - b;
          if (a <= 8 && b <= 8 && cc <= 8) lut[a][b][cc] = (int16_t)(n <= 8 ? k : -1);
          ++k;
        }
  }
  cudaError_t el = cudaMemcpyToSymbol(c_lut, lut, sizeof(lut));
  if (el != cudaSuccess) {
    c->last_error = std::string("near_init: ") + cudaGetErrorString(el);
    return FMM_ERR_CUDA;
  }
  float pos[216][3];
  for (int s = 0; s < 216; ++s) {
    int q = s >> 3, cc = s & 7;
    int dq[3] = {q % 3 - 1, (q / 3) % 3 - 1, q / 9 - 1};
    for (int i = 0; i < 3; ++i) pos[s][i] = (float)(2 * dq[i] + ((cc >> i) & 1));
  }
  cudaError_t e = cudaMemcpyToSymbol(c_src_pos, pos, sizeof(pos));
  if (e != cudaSuccess) {
    c->last_error = std::string("near_init: ") + cudaGetErrorString(e);
    return FMM_ERR_CUDA;
  }
  return FMM_OK;
}

namespace {

template <typename T, int OPB>
void near_dispatch(int p, unsigned blocks, cudaStream_t st, const NearParams& P) {
  if (p == 4)
    launch_pdl(k_near<T, OPB, 4>, blocks, 8 * OPB, 0, st, P);
  else if (p == 6)
    launch_pdl(k_near<T, OPB, 6>, blocks, 8 * OPB, 0, st, P);
  else
    launch_pdl(k_near<T, OPB, 0>, blocks, 8 * OPB, 0, st, P);
}

}  // namespace

int near_opb(const Ctx* c) {  // a pair of warps serves eight octs: 8 or 16 per block
  const bool f64 = c->cfg.precision == FMM_FP64;
  const int o = c->tune_opb;
  if (f64) return 8;
  return (o == 8 || o == 16) ? o : 16;
}

void launch_near(Ctx* c, int lo, void* const* phi, void* const* accel, int out_fp32, cudaStream_t st) {
  const bool f64 = c->cfg.precision == FMM_FP64;
  const int opb = near_opb(c);
  int l = lo;
  while (l <= c->lmax) {  // up to kMaxNearSeg target levels per launch
    NearParams P;
    P.nseg = 0;
    P.nc = c->tab.nc;
    P.p = c->cfg.p;
    P.out_fp32 = out_fp32;
    P.nearop = f64 ? c->d_near64.ptr : c->d_near32.ptr;
    P.G = c->cfg.G;
    P.bottom1 = c->cfg.bottom_mode == FMM_BOTTOM_M2L_L2P;
    const int dl = P.bottom1 ? 1 : 2;  // level difference to the box of the far field
    int blocks = 0;
    for (; l <= c->lmax && P.nseg < kMaxNearSeg; ++l) {
      LevelTree& T = c->lev[l];
      if (!T.n_tgt || !T.n_leaf) continue;
      NearSeg& S = P.seg[P.nseg++];
      S.tgt = (const int32_t*)T.tgt.ptr;
      S.nbr = (const int32_t*)T.nbr.ptr;
      S.cc_l = (const int32_t*)T.cell_child.ptr;
      S.par_l = (const int32_t*)T.oct_parent.ptr;
      S.mono_up = c->lev[l - 1].mono.ptr;
      S.mono_l = T.mono.ptr;
      S.mono_dn = (l < c->lmax) ? c->lev[l + 1].mono.ptr : nullptr;
      S.M_l = T.M.ptr;
      S.M_l_f64 = T.m_is_f64 ? 1 : 0;
      S.L2 = (l - dl >= first_local_level(c)) ? (f64 ? c->lev[l - dl].L.ptr : c->lev[l - dl].Lf.ptr) : nullptr;
      S.lslot = (const int32_t*)T.lslot.ptr;
      S.leafmask = (const uint8_t*)T.leafmask.ptr;
      S.acc = T.acc.ptr;
      S.phi = phi[l - lo];
      S.accel = accel[l - lo];
      S.s1 = c->cfg.G * std::ldexp(1.0, l);
      S.s2 = c->cfg.G * std::ldexp(1.0, 2 * l);
      S.s1f = (float)S.s1;
      S.s2f = (float)S.s2;
      S.n_tgt = T.n_tgt;
      S.blk0 = blocks;
      blocks += (int)((T.n_tgt + opb - 1) / opb);
    }
    if (!blocks) continue;
    ++c->n_launch;
    const int p = c->cfg.p;
    if (f64) {
      near_dispatch<double, 8>(p, (unsigned)blocks, st, P);
    } else {
      if (opb == 8)
        near_dispatch<float, 8>(p, (unsigned)blocks, st, P);
      else
        near_dispatch<float, 16>(p, (unsigned)blocks, st, P);
    }
  }
}

void launch_near_m2p(Ctx* c, int lo, cudaStream_t st) {
  const bool f64 = c->cfg.precision == FMM_FP64;
  int l = lo;
  while (l <= c->lmax) {
    NearM2PParams P;
    P.nseg = 0;
    P.nc = c->tab.nc;
    P.nearop = f64 ? c->d_near64.ptr : c->d_near32.ptr;
    int blocks = 0;
    for (; l <= c->lmax && P.nseg < kMaxNearSeg; ++l) {
      LevelTree& T = c->lev[l];
      if (!T.n_irows || !T.n_leaf) continue;
      NearM2PSeg& S = P.seg[P.nseg++];
      S.irows = (const int32_t*)T.irows.ptr;
      S.nbr = (const int32_t*)T.nbr.ptr;
      S.cc_l = (const int32_t*)T.cell_child.ptr;
      S.M_l = T.M.ptr;
      S.M_l_f64 = T.m_is_f64 ? 1 : 0;
      S.acc = T.acc.ptr;
      S.n = T.n_irows;
      S.blk0 = blocks;
      blocks += (int)T.n_irows;
    }
    if (!blocks) continue;
    ++c->n_launch;
    if (f64)
      launch_pdl(k_near_m2p<double>, (unsigned)blocks, 256, 0, st, P);
    else
      launch_pdl(k_near_m2p<float>, (unsigned)blocks, 256, 0, st, P);
  }
}

}  // namespace fmm
