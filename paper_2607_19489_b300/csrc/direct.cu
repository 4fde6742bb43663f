// direct.cu -- the direct sum the FMM approximates: phi and accel of selected
// leaf cells of one level from every leaf cell of the current hierarchy, in
// FP64, O(targets x cells).  It is the reference of the method's accuracy
// (Sec. 4 compares FMM solutions against exact ones), not part of the solve.
//
// Each thread owns one target; the block streams every level's leaves through
// shared memory in tiles of kTile cells (centre and mass, FP64), so each source
// is read from HBM once per block.  g(R) = -1/|R|; the self term is skipped by
// comparing centres exactly, as a point mass has no self-potential.
#include "fmm_internal.cuh"

namespace fmm {
namespace {

constexpr int kThreads = 128;
constexpr int kTile = 256;

struct DirectLevel {
  const int32_t* ijk;  // [n][3]
  const double* mass;  // [n]
  int64_t n;
  double h;            // cell size 2^-l
};

struct DirectParams {
  DirectLevel lev[kMaxLevel + 1];
  int nlev;
  const int32_t* t_ijk;  // target level's cells
  int64_t t_n;           // their number
  double t_h;
  const int64_t* sel;    // [n_sel] indices into the target level
  int64_t n_sel;
  double G;
  double* phi;           // [n_sel]
  double* accel;         // [n_sel][3]
};

__global__ void __launch_bounds__(kThreads) k_direct(const __grid_constant__ DirectParams P) {
  __shared__ double4 s_src[kTile];
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const bool in = i < P.n_sel;
  const int64_t t = in ? P.sel[i] : 0;
  const bool ok = in && t >= 0 && t < P.t_n;  // an index outside the level gives NaN outputs
  double x = 0, y = 0, z = 0;
  if (ok) {
    x = ((double)P.t_ijk[3 * t] + 0.5) * P.t_h;
    y = ((double)P.t_ijk[3 * t + 1] + 0.5) * P.t_h;
    z = ((double)P.t_ijk[3 * t + 2] + 0.5) * P.t_h;
  }
  double phi = 0, ax = 0, ay = 0, az = 0;
  for (int k = 0; k < P.nlev; ++k) {
    const DirectLevel& L = P.lev[k];
    for (int64_t base = 0; base < L.n; base += kTile) {
      __syncthreads();
      for (int j = threadIdx.x; j < kTile; j += kThreads) {
        const int64_t s = base + j;
        double4 v = make_double4(0.0, 0.0, 0.0, 0.0);
        if (s < L.n)
          v = make_double4(((double)L.ijk[3 * s] + 0.5) * L.h, ((double)L.ijk[3 * s + 1] + 0.5) * L.h,
                           ((double)L.ijk[3 * s + 2] + 0.5) * L.h, L.mass[s]);
        s_src[j] = v;
      }
      __syncthreads();
      const int m = (L.n - base < kTile) ? (int)(L.n - base) : kTile;
      for (int j = 0; j < m; ++j) {
        const double4 v = s_src[j];
        const double dx = v.x - x, dy = v.y - y, dz = v.z - z;
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 == 0.0) continue;  // the target itself
        const double ir = 1.0 / sqrt(r2);
        const double mir = v.w * ir;
        phi -= mir;
        const double mir3 = mir * ir * ir;  // accel = -grad phi = sum m (y - x) / r^3
        ax += mir3 * dx;
        ay += mir3 * dy;
        az += mir3 * dz;
      }
    }
  }
  if (!in) return;
  if (!ok) phi = ax = ay = az = __longlong_as_double(0x7FF8000000000000ll);
  P.phi[i] = P.G * phi;
  P.accel[3 * i] = P.G * ax;
  P.accel[3 * i + 1] = P.G * ay;
  P.accel[3 * i + 2] = P.G * az;
}

}  // namespace
}  // namespace fmm

using namespace fmm;

extern "C" fmm_status fmm_direct_sum(fmm_ctx* cx, int level, int64_t n_sel, const int64_t* sel, double* phi,
                                     double* accel, void* stream) {
  Ctx* c = reinterpret_cast<Ctx*>(cx);
  if (!c) return FMM_ERR_ARG;
  if (!c->have_levels) {
    c->last_error = "fmm_direct_sum before fmm_set_levels";
    return FMM_ERR_STATE;
  }
  if (level < c->lmin || level > c->lmax_user || n_sel < 0) {
    c->last_error = "fmm_direct_sum: level outside lmin..lmax or a negative count";
    return FMM_ERR_ARG;
  }
  if (c->cfg.periodic) {
    c->last_error = "fmm_direct_sum: the isolated sum; a periodic context has no plain pair sum";
    return FMM_ERR_ARG;
  }
  if (n_sel == 0 || level > c->lmax) return FMM_OK;
  if (!is_device_ptr(sel) || !is_device_ptr(phi) || !is_device_ptr(accel)) {
    c->last_error = "fmm_direct_sum: sel, phi and accel must be device pointers";
    return FMM_ERR_ARG;
  }
  DirectParams P{};
  P.nlev = 0;
  for (int l = c->lmin; l <= c->lmax; ++l) {
    const LevelTree& T = c->lev[l];
    if (!T.n_leaf) continue;
    DirectLevel& L = P.lev[P.nlev++];
    L.ijk = (const int32_t*)T.ijk.ptr;
    L.mass = (const double*)T.mass.ptr;
    L.n = T.n_leaf;
    L.h = std::ldexp(1.0, -l);
  }
  P.t_ijk = (const int32_t*)c->lev[level].ijk.ptr;
  P.t_n = c->lev[level].n_leaf;
  P.t_h = std::ldexp(1.0, -level);
  P.sel = sel;
  P.n_sel = n_sel;
  P.G = c->cfg.G;
  P.phi = phi;
  P.accel = accel;
  cudaStream_t st = (cudaStream_t)stream;
  c->last_stream = st;
  ++c->n_launch;
  k_direct<<<(unsigned)((n_sel + kThreads - 1) / kThreads), kThreads, 0, st>>>(P);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    c->last_error = std::string("fmm_direct_sum: ") + cudaGetErrorString(e);
    return FMM_ERR_CUDA;
  }
  return FMM_OK;
}
