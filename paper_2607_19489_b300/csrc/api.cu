// api.cu -- the C ABI (include/fmm.h): context, hierarchy, and the solve
// schedule of Alg. 1 for the target levels lo..lmax.
//
// Schedule of fmm_solve (all on one stream, no host synchronisation):
//   1. Upward (Alg. 2): P2M/M2M from the finest level to level 1, giving
//      every cell the multipole of all mass inside it (the sum of the paper's
//      per-level trees; stale levels keep the masses they were last given).
//   2. MultipoleToLocal (Alg. 3): for box levels 2..lmax-2, L2L from the
//      parent then M2L over the interaction list (gathered contraction).
//      The far field of a box does not depend on the target level, so one
//      downward pass serves all target levels.
//   3. PotentialEvaluation (Alg. 4) per target level: the bottom intermediate
//      field as an M2P contraction, then near/nearest fields, L2P and the
//      scatter to the caller's order.
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include <cub/cub.cuh>
#include <thrust/iterator/counting_iterator.h>

#include "fmm_internal.cuh"

namespace fmm {

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {  // allocates nothing
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device memory comes from the caller's allocator when one was given to
// fmm_create, else from cudaMalloc.  Memory handed back to a caller's allocator
// may be reused at once in the order of the call's stream; all of the library's
// work is ordered on that stream (its second stream joins it before a solve
// ends), so nothing still reads a released buffer out of order.
static void dev_release(Ctx* c, void* p, size_t bytes) {
  if (!p) return;
  if (c->alloc)
    c->alloc(c->alloc_user, p, bytes, (void*)c->last_stream);
  else
    cudaFree(p);
}

static cudaError_t dev_acquire(Ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  if (!c->alloc) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
      *p = nullptr;
      cudaGetLastError();
    }
    return e;
  }
  void* q = c->alloc(c->alloc_user, nullptr, bytes, (void*)c->last_stream);
  if (!q) return cudaErrorMemoryAllocation;
  if ((uintptr_t)q % 256) {  // tensor maps and vector loads rely on 256-byte alignment
    c->alloc(c->alloc_user, q, bytes, (void*)c->last_stream);
    return cudaErrorMisalignedAddress;
  }
  *p = q;
  return cudaSuccess;
}

cudaError_t buf_ensure(Ctx* c, DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return cudaSuccess;
  if (b.ptr) {
    dev_release(c, b.ptr, b.bytes);
    c->bytes_in_use -= b.bytes;
    b.ptr = nullptr;
    b.bytes = 0;
  }
  ++c->layout_gen;  // cached solve graphs hold the old pointers
  if (c->cfg.mem_budget && c->bytes_in_use + bytes > c->cfg.mem_budget) return cudaErrorMemoryAllocation;
  cudaError_t e = dev_acquire(c, &b.ptr, bytes);
  if (e != cudaSuccess) return e;
  b.bytes = bytes;
  c->bytes_in_use += bytes;
  return cudaSuccess;
}

static void buf_free(Ctx* c, DevBuf& b) {
  if (b.ptr) {
    dev_release(c, b.ptr, b.bytes);
    c->bytes_in_use -= b.bytes;
  }
  b.ptr = nullptr;
  b.bytes = 0;
}

namespace {
// masses given as float (config.mass_fp32): widened exactly to the FP64 copy
__global__ void k_widen_mass(int64_t n, const float* __restrict__ in, double* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (double)in[i];
}
}  // namespace

namespace {
// The inputs of every level given by device pointers in one launch: cell
// indices (ijk may be null: masses only) and masses, float masses widened.
struct StageLevel {
  const int32_t* ijk;
  const void* mass;
  int32_t* dijk;
  double* dmass;
  int64_t end;  // cumulative cell count up to and including this level
};
struct StageParams {
  StageLevel lev[kMaxLevel + 1];
  int nlev, mass_f32;
};
__global__ void k_stage_inputs(const __grid_constant__ StageParams P) {
  const int64_t total = P.lev[P.nlev - 1].end;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    int k = 0;
    while (i >= P.lev[k].end) ++k;
    const StageLevel& L = P.lev[k];
    const int64_t j = i - (k ? P.lev[k - 1].end : 0);
    if (L.ijk) {
      L.dijk[3 * j] = L.ijk[3 * j];
      L.dijk[3 * j + 1] = L.ijk[3 * j + 1];
      L.dijk[3 * j + 2] = L.ijk[3 * j + 2];
    }
    L.dmass[j] = P.mass_f32 ? (double)((const float*)L.mass)[j] : ((const double*)L.mass)[j];
  }
}
}  // namespace

// Copies the inputs of levels lo..lo+nlev-1 into the context (ijk null: masses
// only) with one kernel when every source is device memory; false when a source
// is host memory (the caller then copies level by level).
static bool stage_device_inputs(Ctx* c, int lo, int nlev, const int32_t* const* ijk, const void* const* mass,
                                cudaStream_t st) {
  StageParams P{};
  P.mass_f32 = c->cfg.mass_fp32;
  int64_t tot = 0;
  for (int k = 0; k < nlev; ++k) {
    LevelTree& T = c->lev[lo + k];
    if (!T.n_leaf) continue;
    if ((ijk && !is_device_ptr(ijk[k])) || !is_device_ptr(mass[k])) return false;
    StageLevel& L = P.lev[P.nlev++];
    L.ijk = ijk ? ijk[k] : nullptr;
    L.mass = mass[k];
    L.dijk = (int32_t*)T.ijk.ptr;
    L.dmass = (double*)T.mass.ptr;
    tot += T.n_leaf;
    L.end = tot;
  }
  if (!tot) return true;
  ++c->n_launch;
  const unsigned g = (unsigned)std::min<int64_t>((tot + 255) / 256, 8 * c->num_sms);
  k_stage_inputs<<<g, 256, 0, st>>>(P);
  return cudaGetLastError() == cudaSuccess;
}

// Copies the masses of one level into its FP64 array: double input directly,
// float input through the staging buffer and a widening kernel.
static fmm_status copy_masses(Ctx* c, LevelTree& T, const void* mass, int64_t nl, cudaStream_t st) {
  if (!nl) return FMM_OK;
  if (!c->cfg.mass_fp32) {
    cudaError_t e = cudaMemcpyAsync(T.mass.ptr, mass, nl * 8, cudaMemcpyDefault, st);
    if (e != cudaSuccess) {
      c->last_error = std::string("mass copy: ") + cudaGetErrorString(e);
      return FMM_ERR_CUDA;
    }
    return FMM_OK;
  }
  cudaError_t e = cudaMemcpyAsync(c->mass_stage.ptr, mass, nl * 4, cudaMemcpyDefault, st);
  if (e == cudaSuccess) {
    k_widen_mass<<<(unsigned)((nl + 255) / 256), 256, 0, st>>>(nl, (const float*)c->mass_stage.ptr,
                                                               (double*)T.mass.ptr);
    ++c->n_launch;
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    c->last_error = std::string("mass copy: ") + cudaGetErrorString(e);
    return FMM_ERR_CUDA;
  }
  return FMM_OK;
}

namespace {

#define CKS(x)                                                             \
  do {                                                                     \
    cudaError_t e_ = (x);                                                  \
    if (e_ != cudaSuccess) {                                               \
      c->last_error = std::string(#x) + ": " + cudaGetErrorString(e_);     \
      return e_ == cudaErrorMemoryAllocation ? FMM_ERR_OOM : FMM_ERR_CUDA; \
    }                                                                      \
  } while (0)

template <typename T>
fmm_status upload(Ctx* c, DevBuf& b, const std::vector<T>& v) {
  CKS(buf_ensure(c, b, v.size() * sizeof(T)));
  CKS(cudaMemcpy(b.ptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return FMM_OK;
}

#define TRY(x)                     \
  do {                             \
    fmm_status s_ = (x);           \
    if (s_ != FMM_OK) return s_;   \
  } while (0)

inline uint16_t bf16_bits(float f) {  // round to nearest even
  uint32_t u;
  std::memcpy(&u, &f, 4);
  uint32_t r = u + 0x7FFF + ((u >> 16) & 1);
  return (uint16_t)(r >> 16);
}
inline float bf16_val(uint16_t b) {
  uint32_t u = (uint32_t)b << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}
// FP32 rounded to TF32 (10 explicit mantissa bits) to nearest, ties away from
// zero: add half of the last kept unit to the magnitude, then drop the 13 bits
inline float tf32_round(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7F800000u) != 0x7F800000u) u = (u + 0x1000u) & 0xFFFFE000u;
  std::memcpy(&f, &u, 4);
  return f;
}

// Build the device copies of one contraction operator.  `src` is [N][K] with
// K ordered (q, s, alpha).
//
// Tensor-core layout.  K is reordered (q, alpha, s) to match the operand rows
// (op_index), each offset segment padded to a whole number of kTcBK slices.
// M2L keeps |alpha| + |beta| <= p (and |alpha| <= p_m; Eq. 3), so its columns
// are ordered by |beta| descending, cell by cell within a degree: an N tile
// whose lowest column degree is d needs only alpha of degree <= min(p - d,
// p_m), a prefix of every segment, and the tiles of high degree (most of the
// columns) read a few slices instead of all of them.  The M2L sums of a slot
// are kept in this column order (colmap); M2P columns read every alpha <= p_m.
fmm_status build_operator(Ctx* c, GemmOperand& op, const std::vector<double>& src, int N, int kind) {
  // kind: kOpM2P / kOpM2L (nc coefficients per source cell) or kOpP2P (the 8
  // child masses of each source cell, all read)
  const bool m2l = kind == kOpM2L;
  const int nc = c->tab.nc, nsrc = kind == kOpP2P ? 8 : nc, KQ = 8 * nsrc, K = 26 * KQ;
  op.N = N;
  op.K = K;
  op.kseg = KQ;
  // K entries of a segment that column n reads: alpha of degree <= min(p - |beta|,
  // p_m) (M2L), <= p_m (M2P), every child (P2P)
  auto keep_len = [&](int d) { return kind == kOpP2P ? KQ : 8 * ncoef(std::min(c->tab.p - d, c->tab.pm)); };
  if (c->cfg.precision == FMM_FP64) {
    // [K'][N] with K' ordered (q, alpha, s) and per-column segment limits
    std::vector<double> f((size_t)K * N);
    std::vector<int32_t> lim(N);
    for (int n = 0; n < N; ++n) lim[n] = keep_len(m2l ? c->tab.degree[n % nc] : 0);
    for (int q = 0; q < 26; ++q)
      for (int s = 0; s < 8; ++s)
        for (int a = 0; a < nsrc; ++a) {
          size_t kin = (size_t)(q * 8 + s) * nsrc + a;
          size_t kout = (size_t)q * KQ + a * 8 + s;
          for (int n = 0; n < N; ++n) f[kout * N + n] = src[(size_t)n * K + kin];
        }
    TRY(upload(c, op.f64, f));
    TRY(upload(c, op.klimit, lim));
    op.BN = 256;
    op.ntile = (N + 255) / 256;
    return FMM_OK;
  }
  const int p = c->tab.p;
  // columns: order (new column -> source column) and the K entries of a segment each reads
  std::vector<int> order(N);
  std::vector<int> keep(N);
  if (m2l) {
    int n = 0;
    for (int d = p; d >= 0; --d)
      for (int b = 0; b < nc; ++b)
        if (c->tab.degree[b] == d)
          for (int s = 0; s < 8; ++s) {
            order[n] = s * nc + b;
            keep[n] = keep_len(d);
            ++n;
          }
    std::vector<int32_t> colmap(N);
    for (int j = 0; j < N; ++j) colmap[order[j]] = j;
    TRY(upload(c, op.colmap, colmap));
    op.BN = 96;  // finer tiles track the degree prefixes more closely
  } else {
    for (int n = 0; n < N; ++n) {
      order[n] = n;
      keep[n] = keep_len(0);
    }
    op.BN = ((N + 255) / 256 == 1) ? (N + 31) / 32 * 32 : 256;
  }
  op.ntile = (N + op.BN - 1) / op.BN;
  op.Npad = op.ntile * op.BN;
  op.kqp = (KQ + kTcBK - 1) / kTcBK * kTcBK;
  op.Kpad = 26 * op.kqp;
  op.tile_slices.assign(op.ntile, 0);
  for (int y = 0; y < op.ntile; ++y) {
    int q = 0;
    for (int n = y * op.BN; n < std::min(N, (y + 1) * op.BN); ++n) q = std::max(q, keep[n]);
    op.tile_slices[y] = (q + kTcBK - 1) / kTcBK;
  }
  // element (new column j, source K index (q, s, alpha)) -> (j, q kqp + alpha 8 + s)
  auto each = [&](auto&& put) {
    for (int j = 0; j < N; ++j)
      for (int q = 0; q < 26; ++q)
        for (int s = 0; s < 8; ++s)
          for (int a = 0; a < nsrc; ++a)
            put((size_t)j * op.Kpad + (size_t)q * op.kqp + a * 8 + s,
                src[(size_t)order[j] * K + (size_t)(q * 8 + s) * nsrc + a]);
  };
  if (c->cfg.precision == FMM_MIXED_TF32) {  // one FP32 operand, rounded to TF32
    std::vector<float> f((size_t)op.Npad * op.Kpad, 0.0f);
    each([&](size_t i, double v) { f[i] = tf32_round((float)v); });
    TRY(upload(c, op.hi, f));
    return make_tensor_maps(c, op);
  }
  std::vector<uint16_t> hi((size_t)op.Npad * op.Kpad, 0), lo((size_t)op.Npad * op.Kpad, 0);
  each([&](size_t i, double v) {
    const uint16_t h = bf16_bits((float)v);
    hi[i] = h;
    lo[i] = bf16_bits((float)(v - (double)bf16_val(h)));
  });
  TRY(upload(c, op.hi, hi));
  TRY(upload(c, op.lo, lo));
  return make_tensor_maps(c, op);
}

fmm_status init_tables(Ctx* c) {
  Tables& t = c->tab;
  t.build(c->cfg.p, c->cfg.p_m);
  TRY(upload(c, c->d_m2m_off, t.m2m_off));
  TRY(upload(c, c->d_m2m_g, t.m2m_g));
  TRY(upload(c, c->d_m2m_e, t.m2m_e));
  TRY(upload(c, c->d_m2m_c, t.m2m_c));
  TRY(upload(c, c->d_m2m_c32, std::vector<float>(t.m2m_c.begin(), t.m2m_c.end())));
  {  // the gamma = 0 term of each alpha: all an oct of point masses needs
    std::vector<double> w0(t.nc, 0.0);
    std::vector<int> e0(t.nc, 0);
    for (int k = 0; k < t.nc; ++k)
      for (int j = t.m2m_off[k]; j < t.m2m_off[k + 1]; ++j)
        if (t.m2m_g[j] == 0) {
          w0[k] = t.m2m_c[j];
          e0[k] = t.m2m_e[j];
        }
    TRY(upload(c, c->d_m2m_w0, w0));
    TRY(upload(c, c->d_m2m_w0_32, std::vector<float>(w0.begin(), w0.end())));
    TRY(upload(c, c->d_m2m_e0, e0));
  }
  TRY(upload(c, c->d_l2l_off, t.l2l_off));
  TRY(upload(c, c->d_l2l_off8, t.l2l_off8));
  TRY(upload(c, c->d_l2l_g, t.l2l_g));
  TRY(upload(c, c->d_l2l_e, t.l2l_e));
  TRY(upload(c, c->d_l2l_c, t.l2l_c));
  TRY(upload(c, c->d_l2l_c32, std::vector<float>(t.l2l_c.begin(), t.l2l_c.end())));
  if (c->cfg.precision == FMM_FP64) {
    TRY(upload(c, c->d_near64, t.nearop));
    TRY(upload(c, c->d_l2p64, t.l2p));
  } else {
    std::vector<float> nf(t.nearop.begin(), t.nearop.end()), lf(t.l2p.begin(), t.l2p.end());
    TRY(upload(c, c->d_near32, nf));
    TRY(upload(c, c->d_l2p32, lf));
  }
  TRY(build_operator(c, c->op_m2p, t.m2p, 256, kOpM2P));
  TRY(build_operator(c, c->op_m2l, t.m2l, 8 * t.nc, kOpM2L));
  if (c->cfg.periodic) {
    t.build_lattice();
    if (c->cfg.precision == FMM_FP64)
      TRY(upload(c, c->d_lat64, t.lattice));
    else
      TRY(upload(c, c->d_lat32, std::vector<float>(t.lattice.begin(), t.lattice.end())));
    std::vector<double>().swap(t.lattice);
  }
  if (c->cfg.delta_l == 2) {
    t.build_dl2();
    TRY(build_operator(c, c->op_m2p2, t.m2p2, 2048, kOpM2P));
    TRY(build_operator(c, c->op_p2pr, t.p2pr, 256, kOpP2P));
  }
  // the tables are only needed on the device from here on
  std::vector<double>().swap(t.m2p);
  std::vector<double>().swap(t.m2l);
  std::vector<double>().swap(t.m2p2);
  std::vector<double>().swap(t.p2pr);
  c->tables_on_device = true;
  return FMM_OK;
}

// Sizes every per-level array so that fmm_solve allocates nothing.  The local
// expansions are stored per slot (octs that need one, known after the tree
// build: size_locals); the buffers that are zero between solves (Lm, and acc
// in the mixed path) are cleared when they are (re)allocated.
fmm_status size_expansions(Ctx* c, cudaStream_t st) {
  const int nc = c->tab.nc;
  const bool f64 = c->cfg.precision == FMM_FP64;
  for (int l = 1; l <= c->lmax; ++l) {
    LevelTree& T = c->lev[l];
    const int64_t ncell = 8 * T.n_oct;
    T.m_is_f64 = f64 || (c->cfg.fp64_top && l <= kTopLevelFP64);
    CKS(buf_ensure(c, T.mono, ncell * 8));
    if (l < c->lmax) {
      CKS(buf_ensure(c, T.M, ncell * nc * (T.m_is_f64 ? 8 : 4)));
      if (c->cfg.precision == FMM_MIXED_TF32) {
        CKS(buf_ensure(c, T.Mhi, ncell * nc * 4));  // FP32 operand rows (TF32-rounded)
      } else if (!f64) {
        CKS(buf_ensure(c, T.Mhi, ncell * nc * 2));
        CKS(buf_ensure(c, T.Mlo, ncell * nc * 2));
      }
    }
    if (c->cfg.delta_l == 2 && l == c->lmax - 1) {  // the 8 child masses of each cell
      if (f64) {
        CKS(buf_ensure(c, T.Chi, ncell * 8 * 8));
      } else if (c->cfg.precision == FMM_MIXED_TF32) {
        CKS(buf_ensure(c, T.Chi, ncell * 8 * 4));
      } else {
        CKS(buf_ensure(c, T.Chi, ncell * 8 * 2));
        CKS(buf_ensure(c, T.Clo, ncell * 8 * 2));
      }
    }
    if (l >= c->lmin) {
      // a grown buffer may come back at the same address (a caching allocator
      // reuses the block it was just given): compare sizes as well as pointers
      void* old = T.acc.ptr;
      const size_t old_bytes = T.acc.bytes;
      CKS(buf_ensure(c, T.acc, ncell * 4 * (f64 ? 8 : 4)));
      if (T.acc.ptr != old || T.acc.bytes != old_bytes) CKS(cudaMemsetAsync(T.acc.ptr, 0, T.acc.bytes, st));
    }
  }
  return FMM_OK;
}

fmm_status size_locals(Ctx* c, cudaStream_t st) {
  const int nc = c->tab.nc;
  const bool f64 = c->cfg.precision == FMM_FP64;
  for (int l = first_local_level(c); l <= top_local_level(c); ++l) {
    LevelTree& T = c->lev[l];
    const int64_t nrow = 8 * std::max<int64_t>(T.n_rowsL, 1);
    if (f64) CKS(buf_ensure(c, T.L, nrow * nc * 8));  // the mixed paths keep the FP32 expansions only
    if (!f64) {
      void* old = T.Lm.ptr;
      const size_t old_bytes = T.Lm.bytes;
      CKS(buf_ensure(c, T.Lm, nrow * nc * 4));
      if (T.Lm.ptr != old || T.Lm.bytes != old_bytes) CKS(cudaMemsetAsync(T.Lm.ptr, 0, T.Lm.bytes, st));
      CKS(buf_ensure(c, T.Lf, nrow * nc * 4));
    }
  }
  return FMM_OK;
}

void stage_event(Ctx* c, int i, cudaStream_t st) {
  if (c->timing) cudaEventRecord(c->ev[i], st);
}

// ---- adjoint preparation ------------------------------------------------------
// Transposed pair lists of M2M (grouped by input gamma and sign pattern e) and
// L2L (grouped by input gamma), and the contraction operators transposed per
// neighbour offset: BT[qi][n][s*nc + alpha] = B[n][(qi*8 + s)*nc + alpha].
fmm_status adjoint_tables(Ctx* c) {
  if (c->adj_tables) return FMM_OK;
  const Tables& t = c->tab;
  const int nc = t.nc;
  {
    std::vector<std::vector<std::pair<int, double>>> by(nc * 8);
    for (int a = 0; a < nc; ++a)
      for (int j = t.m2m_off[a]; j < t.m2m_off[a + 1]; ++j) by[t.m2m_g[j] * 8 + t.m2m_e[j]].push_back({a, t.m2m_c[j]});
    std::vector<int> off(1, 0), ia;
    std::vector<double> cf;
    for (auto& v : by) {
      for (auto& pr : v) {
        ia.push_back(pr.first);
        cf.push_back(pr.second);
      }
      off.push_back((int)ia.size());
    }
    TRY(upload(c, c->d_m2mT_off, off));
    TRY(upload(c, c->d_m2mT_a, ia));
    TRY(upload(c, c->d_m2mT_c, cf));
  }
  {
    struct E {
      int b, e;
      double c;
    };
    std::vector<std::vector<E>> by(nc);
    for (int b = 0; b < nc; ++b)
      for (int e = 0; e < 8; ++e)
        for (int j = t.l2l_off8[b * 8 + e]; j < t.l2l_off8[b * 8 + e + 1]; ++j) by[t.l2l_g[j]].push_back({b, e, t.l2l_c[j]});
    std::vector<int> off(1, 0), ib, ie;
    std::vector<double> cf;
    for (auto& v : by) {
      for (auto& x : v) {
        ib.push_back(x.b);
        ie.push_back(x.e);
        cf.push_back(x.c);
      }
      off.push_back((int)ib.size());
    }
    TRY(upload(c, c->d_l2lT_off, off));
    TRY(upload(c, c->d_l2lT_b, ib));
    TRY(upload(c, c->d_l2lT_e, ie));
    TRY(upload(c, c->d_l2lT_c, cf));
  }
  const int KQ = 8 * nc, K = 26 * KQ;
  Tables full;  // the context keeps no host copy of the contraction operators
  full.build(c->cfg.p, c->cfg.p_m);
  for (int w = 0; w < 2; ++w) {
    const std::vector<double>& src = w == 0 ? full.m2p : full.m2l;
    if (src.size() != (size_t)(w == 0 ? 256 : 8 * nc) * K) {
      c->last_error = "adjoint: operator table has an unexpected size";
      return FMM_ERR_ARG;
    }
    const int N = w == 0 ? 256 : 8 * nc;
    std::vector<double> bt((size_t)26 * N * KQ);
    for (int qi = 0; qi < 26; ++qi)
      for (int n = 0; n < N; ++n)
        std::memcpy(&bt[((size_t)qi * N + n) * KQ], &src[(size_t)n * K + (size_t)qi * KQ], KQ * sizeof(double));
    TRY(upload(c, w == 0 ? c->d_m2pT : c->d_m2lT, bt));
  }
  c->adj_tables = true;
  return FMM_OK;
}

// Per level the octs whose multipoles an M2P row (srcP) or an M2L row (srcL)
// reads: the 26 neighbours of each row, compacted.  Built once per tree layout.
fmm_status adjoint_lists(Ctx* c, cudaStream_t st) {
  if (c->adj_gen == c->layout_gen) return FMM_OK;
  const int lmax = c->lmax;
  int64_t nmax = 1;
  for (int l = 1; l <= lmax; ++l) nmax = std::max(nmax, c->lev[l].n_oct);
  CKS(buf_ensure(c, c->flags, nmax * 4));
  CKS(buf_ensure(c, c->counter, 8 * (lmax + 1)));
  int32_t* flags = (int32_t*)c->flags.ptr;
  int32_t* d_cnt = (int32_t*)c->counter.ptr;  // [lmax+1][2]
  CKS(cudaMemsetAsync(d_cnt, 0, 8 * (lmax + 1), st));
  thrust::counting_iterator<int32_t> it(0);
  size_t tmp = 0;
  CKS(cub::DeviceSelect::Flagged(nullptr, tmp, it, flags, (int32_t*)nullptr, d_cnt, (int)nmax, st));
  CKS(buf_ensure(c, c->sort_tmp, tmp));
  for (int b = 1; b <= lmax; ++b) {
    LevelTree& B = c->lev[b];
    CKS(buf_ensure(c, B.srcP, B.n_oct * 4));
    CKS(buf_ensure(c, B.srcL, B.n_oct * 4));
    for (int w = 0; w < 2; ++w) {
      const bool m2p = w == 0;
      const int64_t nr = m2p ? B.n_rows : B.n_rowsL;
      if (!nr || (m2p ? b > lmax - 1 : (b < 2 || b > lmax - 2))) continue;
      CKS(cudaMemsetAsync(flags, 0, B.n_oct * 4, st));
      launch_adj_mark(c, (const int32_t*)(m2p ? B.rows.ptr : B.rowsL.ptr), nr, (const int32_t*)B.nbr.ptr, flags, st);
      size_t tb = c->sort_tmp.bytes;
      CKS(cub::DeviceSelect::Flagged(c->sort_tmp.ptr, tb, it, flags, (int32_t*)(m2p ? B.srcP.ptr : B.srcL.ptr),
                                     d_cnt + 2 * b + w, (int)B.n_oct, st));
    }
  }
  std::vector<int32_t> cnt(2 * (lmax + 1));
  CKS(cudaMemcpyAsync(cnt.data(), d_cnt, 8 * (lmax + 1), cudaMemcpyDeviceToHost, st));
  CKS(cudaStreamSynchronize(st));
  for (int b = 1; b <= lmax; ++b) {
    c->lev[b].n_srcP = cnt[2 * b];
    c->lev[b].n_srcL = cnt[2 * b + 1];
  }
  c->adj_gen = c->layout_gen;
  return FMM_OK;
}

// ---- translation tables shared between contexts ---------------------------------
// The tables depend only on (device, p, precision) and are read-only once
// built, so every context of the same kind uses one device copy (a batch of 64
// hierarchies would otherwise hold 64 copies of the ~65 MB contraction
// operators).  Reference-counted; the last context frees them.
DevBuf Ctx::*const kTableBufs[] = {
    &Ctx::d_m2m_off, &Ctx::d_m2m_g,   &Ctx::d_m2m_e,    &Ctx::d_m2m_c,  &Ctx::d_m2m_c32, &Ctx::d_m2m_w0,
    &Ctx::d_m2m_w0_32, &Ctx::d_m2m_e0, &Ctx::d_l2l_off, &Ctx::d_l2l_off8, &Ctx::d_l2l_g, &Ctx::d_l2l_e,
    &Ctx::d_l2l_c,   &Ctx::d_l2l_c32, &Ctx::d_near64,  &Ctx::d_near32,   &Ctx::d_l2p64,  &Ctx::d_l2p32,
    &Ctx::d_lat64,   &Ctx::d_lat32};
constexpr int kNumTableBufs = sizeof(kTableBufs) / sizeof(kTableBufs[0]);

struct TableSet {
  int refs = 0;
  Tables tab;
  DevBuf bufs[kNumTableBufs];
  GemmOperand op_m2p, op_m2l, op_m2p2, op_p2pr;
};
// (device, p, precision, p_m, Delta l, periodic, allocator, allocator's user
// pointer): contexts of another allocator get their own copy, released through
// that allocator
using TableKey = std::tuple<int, int, int, int, int, int, uintptr_t, uintptr_t>;
std::mutex g_tables_mu;
std::map<TableKey, TableSet*> g_tables;

TableKey table_key(const Ctx* c) {
  return TableKey(c->device, c->cfg.p, c->cfg.precision, c->cfg.p_m, c->cfg.delta_l, c->cfg.periodic,
                  (uintptr_t)c->alloc, (uintptr_t)c->alloc_user);
}

fmm_status acquire_tables(Ctx* c) {
  std::lock_guard<std::mutex> lock(g_tables_mu);
  auto it = g_tables.find(table_key(c));
  if (it != g_tables.end()) {
    TableSet* ts = it->second;
    ++ts->refs;
    c->tab = ts->tab;
    for (int i = 0; i < kNumTableBufs; ++i) c->*kTableBufs[i] = ts->bufs[i];
    c->op_m2p = ts->op_m2p;
    c->op_m2l = ts->op_m2l;
    c->op_m2p2 = ts->op_m2p2;
    c->op_p2pr = ts->op_p2pr;
    c->tables_on_device = true;
    c->tables_shared = true;
    return FMM_OK;
  }
  TRY(init_tables(c));
  TableSet* ts = new TableSet();
  ts->refs = 1;
  ts->tab = c->tab;
  for (int i = 0; i < kNumTableBufs; ++i) ts->bufs[i] = c->*kTableBufs[i];
  ts->op_m2p = c->op_m2p;
  ts->op_m2l = c->op_m2l;
  ts->op_m2p2 = c->op_m2p2;
  ts->op_p2pr = c->op_p2pr;
  g_tables[table_key(c)] = ts;
  c->tables_shared = true;
  return FMM_OK;
}

// Drops this context's reference; when others remain, clears its copies of
// the shared buffers so that destroying it leaves them alone.
void release_tables(Ctx* c) {
  if (!c->tables_shared) return;
  std::lock_guard<std::mutex> lock(g_tables_mu);
  auto it = g_tables.find(table_key(c));
  if (it == g_tables.end()) return;
  TableSet* ts = it->second;
  if (--ts->refs > 0) {
    for (int i = 0; i < kNumTableBufs; ++i) c->*kTableBufs[i] = DevBuf();
    for (GemmOperand* op : {&c->op_m2p, &c->op_m2l, &c->op_m2p2, &c->op_p2pr})
      op->f64 = op->hi = op->lo = op->klimit = op->colmap = DevBuf();
  } else {
    g_tables.erase(it);
    delete ts;  // this context frees the buffers
  }
  c->tables_shared = false;
}

// ---- batched solves -------------------------------------------------------------
// One CUDA graph for the solves of many contexts: each context's work is a
// branch of its own (forked from the capture stream, spread over a few
// streams), so small hierarchies run side by side.  Cached by the contexts,
// their layout generations, lo and the output pointers.
struct BatchGraph {
  std::vector<uintptr_t> key;
  std::vector<Ctx*> ctxs;
  std::vector<int64_t> launches;
  cudaGraphExec_t exec = nullptr;
};
std::mutex g_batch_mu;
std::vector<BatchGraph> g_batch;
constexpr int kBatchBranches = 8;
cudaStream_t g_batch_streams[kBatchBranches + 1] = {};
int g_batch_dev = -1;

void drop_batch_graphs_of(Ctx* c) {
  std::lock_guard<std::mutex> lock(g_batch_mu);
  for (size_t i = 0; i < g_batch.size();) {
    bool has = false;
    for (Ctx* x : g_batch[i].ctxs) has |= x == c;
    if (has) {
      cudaGraphExecDestroy(g_batch[i].exec);
      g_batch.erase(g_batch.begin() + i);
    } else {
      ++i;
    }
  }
}

}  // namespace
}  // namespace fmm

using namespace fmm;

struct fmm_ctx : public fmm::Ctx {};

extern "C" {

fmm_status fmm_create(const fmm_config* cfg, fmm_alloc_fn alloc, void* alloc_user, fmm_ctx** out) {
  if (!cfg || !out) return FMM_ERR_ARG;
  *out = nullptr;
  if (cfg->p < 1 || cfg->p > 8) return FMM_ERR_ARG;
  if (cfg->p_m < 0 || cfg->p_m > cfg->p) return FMM_ERR_ARG;
  if (cfg->precision != FMM_FP64 && cfg->precision != FMM_MIXED_BF16X3 && cfg->precision != FMM_MIXED_TF32)
    return FMM_ERR_ARG;
  if (cfg->bottom_mode != FMM_BOTTOM_M2P && cfg->bottom_mode != FMM_BOTTOM_M2L_L2P) return FMM_ERR_ARG;
  if (cfg->mass_fp32 != 0 && cfg->mass_fp32 != 1) return FMM_ERR_ARG;
  if (cfg->fp64_top != 0 && cfg->fp64_top != 1) return FMM_ERR_ARG;
  if (cfg->delta_l < 0 || cfg->delta_l > 2) return FMM_ERR_ARG;
  if (cfg->delta_l == 2 && cfg->bottom_mode != FMM_BOTTOM_M2P) return FMM_ERR_ARG;
  if (cfg->periodic != 0 && cfg->periodic != 1) return FMM_ERR_ARG;
  if (cfg->periodic && (cfg->bottom_mode != FMM_BOTTOM_M2P || cfg->delta_l == 2)) return FMM_ERR_ARG;
  if (!std::isfinite(cfg->G)) return FMM_ERR_ARG;
  fmm_ctx* c = new fmm_ctx();
  c->cfg = *cfg;
  if (c->cfg.p_m == c->cfg.p) c->cfg.p_m = 0;  // one key for the full order
  if (c->cfg.delta_l == 0) c->cfg.delta_l = 1;
  c->alloc = alloc;
  c->alloc_user = alloc_user;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return FMM_ERR_CUDA;
  }
  c->device = dev;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = buf_ensure(c, c->err_buf, kErrWords * 4);
  if (e != cudaSuccess) {
    delete c;
    return e == cudaErrorMemoryAllocation ? FMM_ERR_OOM : FMM_ERR_CUDA;
  }
  c->d_err = (unsigned*)c->err_buf.ptr;
  cudaMemset(c->d_err, 0, kErrWords * 4);
  if (cudaMallocHost((void**)&c->h_rb, Ctx::kReadbackBytes) != cudaSuccess) {
    cudaGetLastError();
    buf_free(c, c->err_buf);
    delete c;
    return FMM_ERR_OOM;
  }
  for (auto& ev : c->ev) cudaEventCreate(&ev);
  if (cudaStreamCreateWithFlags(&c->aux_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_sync, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    c->aux_stream = nullptr;  // one stream then: the solve stays correct, only serial
  }
  fmm_status s = near_init(c);
  if (s == FMM_OK) s = upward_init(c);
  if (s == FMM_OK) s = acquire_tables(c);
  if (s != FMM_OK) {
    fmm_destroy(c);
    return s;
  }
  *out = c;
  return FMM_OK;
}

// The tree build's device work as a
// CUDA graph, captured once per (layout generation, levels, leaf counts).
static fmm_status launch_tree_graph(Ctx* c, cudaStream_t st) {
  std::vector<uintptr_t> key = {(uintptr_t)c->layout_gen, (uintptr_t)c->lmin, (uintptr_t)c->lmax,
                                (uintptr_t)c->tree_lo, (uintptr_t)c->anc_req};
  for (int l = c->lmin; l <= c->lmax; ++l) key.push_back((uintptr_t)c->lev[l].n_leaf);
  Ctx::SolveGraph* g = nullptr;
  for (auto& e : c->tree_graphs)
    if (e.key == key) g = &e;
  if (!g) {
    for (size_t i = 0; i < c->tree_graphs.size();)
      if (c->tree_graphs[i].key[0] != (uintptr_t)c->layout_gen || c->tree_graphs.size() >= 4) {
        cudaGraphExecDestroy(c->tree_graphs[i].exec);
        c->tree_graphs.erase(c->tree_graphs.begin() + i);
      } else {
        ++i;
      }
    if (!c->cap_stream) CKS(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    const int64_t n0 = c->n_launch, k0 = c->n_cub;
    CKS(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    fmm_status s = tree_enqueue(c, c->cap_stream);
    cudaGraph_t graph = nullptr;
    cudaError_t ee = cudaStreamEndCapture(c->cap_stream, &graph);
    if (s != FMM_OK) {
      if (graph) cudaGraphDestroy(graph);
      return s;
    }
    CKS(ee);
    cudaGraphExec_t exec = nullptr;
    cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    CKS(ei);
    c->tree_graphs.push_back({key, exec, c->n_launch - n0, c->n_cub - k0});
    c->n_launch = n0;
    c->n_cub = k0;
    ++c->n_graph_build;
    g = &c->tree_graphs.back();
  }
  CKS(cudaGraphLaunch(g->exec, st));
  c->n_launch += g->launches;
  c->n_cub += g->cub_calls;
  ++c->n_graph_launch;
  return FMM_OK;
}

static fmm_status set_levels_impl(fmm_ctx* c, int lmin, int lmax, int lo, const int64_t* n,
                                  const int32_t* const* ijk, const void* const* mass, void* stream);

// A hierarchy that does not fit (FMM_ERR_OOM) leaves no half-grown workspace
// behind: every per-hierarchy buffer is released (the shared tables stay), so a
// smaller hierarchy fits the budget again.  The context then has no hierarchy.
static void release_workspace(Ctx* c) {
  if (c->last_stream) cudaStreamSynchronize(c->last_stream);
  for (auto& T : c->lev)
    for (DevBuf* b : {&T.oct_key, &T.oct_parent, &T.cell_child, &T.nbr, &T.leaf_cell, &T.rows, &T.rowsL, &T.irows,
                      &T.leafmask, &T.gmass, &T.srcP, &T.srcL, &T.slotL, &T.lslot, &T.anc, &T.tgt, &T.ijk, &T.mass, &T.M,
                      &T.Mhi, &T.Mlo, &T.mono, &T.L, &T.Lf, &T.Lm, &T.acc, &T.vel, &T.dS, &T.dQ})
      buf_free(c, *b);
  for (DevBuf* b : {&c->sort_tmp, &c->keys_a, &c->keys_b, &c->vals_a, &c->vals_b, &c->flags, &c->scan, &c->counter,
                    &c->anc_flags, &c->out_stage, &c->in_stage, &c->mass_stage})
    buf_free(c, *b);
  for (auto& T : c->lev) T.n_oct = T.n_leaf = T.n_rows = T.n_tgt = T.n_rowsL = T.n_irows = T.n_anc = 0;
  c->cub_sig.clear();
  c->count_sig.clear();
  c->adj_gen = 0;
  ++c->layout_gen;
  c->have_levels = false;
}

fmm_status fmm_set_levels(fmm_ctx* c, int lmin, int lmax, int lo, const int64_t* n, const int32_t* const* ijk,
                          const void* const* mass, void* stream) {
  fmm_status s = set_levels_impl(c, lmin, lmax, lo, n, ijk, mass, stream);
  if (s == FMM_ERR_OOM && c) {
    const std::string msg = c->last_error;
    release_workspace(c);
    c->last_error = msg + " (the hierarchy's workspace was released)";
  }
  return s;
}

static fmm_status set_levels_impl(fmm_ctx* c, int lmin, int lmax, int lo, const int64_t* n,
                                  const int32_t* const* ijk, const void* const* mass, void* stream) {
  if (!c || !n || !ijk || !mass) return FMM_ERR_ARG;
  if (lmin < 2 || lmax < lmin || lmax > kMaxLevel || lo < lmin || lo > lmax) return FMM_ERR_ARG;
  if (!c->have_levels) {
    if (lo != lmin) {
      c->last_error = "first fmm_set_levels must give the whole hierarchy (lo == lmin)";
      return FMM_ERR_STATE;
    }
  } else if (lo > lmin && (lmin != c->lmin || lmax != c->lmax_user)) {
    c->last_error = "fmm_set_levels: lmin/lmax differ from the hierarchy being updated";
    return FMM_ERR_STATE;
  }
  for (int k = 0; k <= lmax - lo; ++k)
    if (n[k] < 0 || (n[k] > 0 && (!ijk[k] || !mass[k]))) return FMM_ERR_ARG;
  if (c->cfg.delta_l == 2 && (lmin != lmax || lmin < 3)) {
    c->last_error = "delta_l = 2 takes one complete level (lmin == lmax >= 3)";
    return FMM_ERR_ARG;
  }
  if (c->cfg.periodic && lmin < 3) {
    c->last_error = "periodic boundaries need lmin >= 3";
    return FMM_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  c->last_stream = st;
  ++c->n_set;
  c->lmin = lmin;
  c->lmax = lmax;
  c->have_levels = false;
  if (c->cfg.mass_fp32) {
    int64_t nmax = 1;
    for (int k = 0; k <= lmax - lo; ++k) nmax = std::max(nmax, n[k]);
    CKS(buf_ensure(c, c->mass_stage, nmax * 4));
  }
  for (int l = lo; l <= lmax; ++l) {
    LevelTree& T = c->lev[l];
    int64_t nl = n[l - lo];
    T.n_leaf = nl;
    T.vel_valid = false;  // the cells may have changed: fmm_set_velocities again
    CKS(buf_ensure(c, T.ijk, nl * 12));
    CKS(buf_ensure(c, T.mass, nl * 8));
  }
  if (!stage_device_inputs(c, lo, lmax - lo + 1, ijk, mass, st)) {
    cudaGetLastError();
    for (int l = lo; l <= lmax; ++l) {
      LevelTree& T = c->lev[l];
      const int64_t nl = T.n_leaf;
      if (nl) {
        CKS(cudaMemcpyAsync(T.ijk.ptr, ijk[l - lo], nl * 12, cudaMemcpyDefault, st));
        TRY(copy_masses(c, T, mass[l - lo], nl, st));
      }
    }
  }
  // trailing empty levels: the tree ends at the finest level that holds leaves
  int eff = lmax;
  while (eff > lmin && c->lev[eff].n_leaf == 0) --eff;
  c->lmax = eff;
  c->lmax_user = lmax;
  // lo == lmin: a full build; lo > lmin: levels lo..lmax are re-sorted and the
  // next solve recomputes only what depends on them (adaptive time stepping)
  const bool full = lo == lmin;
  c->tree_lo = full ? lmin : lo;
  c->dirty_lo = full ? lmin : std::min(c->dirty_lo, lo);
  c->anc_req = (c->dirty_lo > lmin && c->dirty_lo <= eff) ? c->dirty_lo : 0;
  c->anc_d = 0;
  for (int l = eff + 1; l <= lmax; ++l) {
    LevelTree& T = c->lev[l];
    T.n_oct = T.n_rows = T.n_tgt = T.n_rowsL = T.n_irows = T.n_srcP = T.n_srcL = 0;
  }
  TRY(tree_prepare(c));
  TRY(size_expansions(c, st));
  if (c->use_graphs) {
    TRY(launch_tree_graph(c, st));
  } else {
    TRY(tree_enqueue(c, st));
  }
  {
    fmm_status fs = tree_finish(c, st);
    if (fs != FMM_OK) {
      c->dirty_lo = lmin;
      return fs;
    }
  }
  c->anc_d = c->anc_req;
  TRY(size_locals(c, st));
  if (!c->drift_dt.empty()) TRY(drift_prepare(c));
  {  // list lengths decide grid sizes: a change retires the cached solve graphs
    std::vector<int64_t> sig = {c->lmin, c->lmax};
    for (int l = 0; l <= c->lmax; ++l) {
      const LevelTree& T = c->lev[l];
      sig.insert(sig.end(), {T.n_oct, T.n_leaf, T.n_rows, T.n_tgt, T.n_rowsL, T.n_irows});
    }
    if (sig != c->count_sig) {
      c->count_sig = std::move(sig);
      ++c->layout_gen;
    }
  }
  c->have_levels = true;
  return FMM_OK;
}

// SMs left to the L2L chain and the near-field M2P while the bottom M2P runs
#ifndef FMM_M2P_SIDE_SMS
#define FMM_M2P_SIDE_SMS 40
#endif
constexpr int kM2PSideSMs = FMM_M2P_SIDE_SMS;

// The device work of one solve (no host synchronisation, no allocation).
static fmm_status enqueue_solve(Ctx* c, int lo, void* const* dphi, void* const* dacc, cudaStream_t st) {
  if (lo > c->lmax) return FMM_OK;  // only empty levels
  const bool f64 = c->cfg.precision == FMM_FP64;
  const int lmin = c->lmin, lmax = c->lmax;
  const int d = c->dirty_lo;  // lowest level changed since the last upward pass
  c->cur_lo = lo;
  stage_event(c, 0, st);
  // 1. upward: leaf monopoles, then M2M from the finest level up.  After an
  // update of levels d..lmax only the cells with descendants at level d change
  // (multipoles are totals over the finer levels): M2M runs on all octs of
  // levels >= d and on the ancestor octs above; with no change it is skipped.
  // Nothing reads the multipoles of level 1: its cells are never leaves (lmin
  // >= 2), and M2L (box levels >= 2) and M2P (the 26 neighbour octs of the one
  // level-1 oct lie outside the box) have no level-1 sources.
  // A drifting solve recomputes every total from the masses, then adds the
  // drift of each stale tree (corrections must not stack from solve to solve).
  const bool drift = drift_active(c, lo);
  // Rows of the downward pass over box levels 2..top (top = lmax-2, or lmax-1
  // in bottom mode 1): L = L2L(parent) + M2L.  For targets at levels >= lo >
  // lmin, the levels b <= lo-3 (lo-2 in mode 1) only feed the L2L chain of the
  // ancestors of level lo: their ancestor lists replace the full row lists.
  const int m1 = c->cfg.bottom_mode == FMM_BOTTOM_M2L_L2P;
  const bool dl2 = c->cfg.delta_l == 2;  // one level: lo == lmin, no stale trees
  const int top = top_local_level(c);
  const int top_m2l = top_m2l_level(c);
  const int l0 = first_local_level(c);  // 1 with periodic boundaries
  const bool periodic = c->cfg.periodic;
  const bool restrict_dn = lo > lmin && c->anc_d == lo;
  std::vector<const int32_t*> drows(lmax + 1, nullptr);
  std::vector<int64_t> dn(lmax + 1, 0);
  for (int b = l0; b <= top; ++b)
    if (restrict_dn && b <= lo - 3 + m1) {
      drows[b] = (const int32_t*)c->lev[b].anc.ptr;
      dn[b] = c->lev[b].n_anc;
    }
  std::vector<int> dl;  // box levels with M2L rows
  std::vector<const int32_t*> dr;
  std::vector<int64_t> dnr;
  for (int b = l0; b <= top_m2l; ++b) {
    if (drows[b] && !dn[b]) continue;
    dl.push_back(b);
    dr.push_back(drows[b]);
    dnr.push_back(dn[b]);
  }
  if (!f64) launch_zero_lm(c, dl, dr, dnr, st);  // the M2L contraction adds into these sums
  if (d <= lmin || (d <= lmax && c->anc_d != d) || drift) {
    for (int l = 1; l <= lmax; ++l) launch_mono_leaves(c, l, st);
    if (dl2) launch_child_masses(c, st);
    for (int b = lmax - 1; b >= l0; --b) launch_upward(c, b, st);
    if (drift) launch_drift(c, lo, st);
  } else if (d <= lmax) {
    for (int l = d; l <= lmax; ++l) launch_mono_leaves(c, l, st);
    for (int b = lmax - 1; b >= d - 1; --b) launch_upward(c, b, st);
    // ancestors: one launch per level while the lists are long, then the rest
    // of the chain in one block (each list at most two rounds of its warps;
    // lists only shrink towards the root)
    const int w = m2m_chain_warps(c);
    int b = d - 2;
    for (; b >= 2 && (w == 0 || c->lev[b + 1].n_anc > 2 * w); --b)
      launch_upward(c, b, st, (const int32_t*)c->lev[b + 1].anc.ptr, c->lev[b + 1].n_anc);
    if (b >= 2) launch_m2m_chain(c, b, st);
    if (periodic) launch_upward(c, 1, st);  // the level-1 multipoles feed level-1 M2L and the lattice
  }
  // periodic: the images of the root beyond its 3^3 (and the background), and
  // level 1's M2L from the 26 nearest, into the level-1 M2L sums (FP64: in the
  // L2L chain, after level 1's expansion is set)
  if (periodic && !f64) launch_lattice(c, st);
  stage_event(c, 1, st);
  // 2. downward (below): the M2L rows of each box level
  // M2L of all box levels: one tcgen05 launch (mixed), or per level (FP64)
  // (periodic: level 1's M2L is part of the lattice product, launch_lattice)
  const size_t tc0 = (!dl.empty() && dl[0] == 1) ? 1 : 0;
  auto m2l_tc = [&](cudaStream_t s2) {
    if (dl.size() > tc0)
      launch_gemm_tc(c, c->op_m2l, kModeM2L, dl.data() + tc0, (int)(dl.size() - tc0), s2, dr.data() + tc0,
                     dnr.data() + tc0);
  };
  // Delta l = 2: the level lmax-2 expansions (read by the near field) are the
  // L2L of lmax-3's, zero when lmax-3 < 2
  auto l2l_chain = [&](cudaStream_t s2) {
    if (!f64) {  // one launch: each block recomputes its ancestors' expansions
      if (!dl.empty() || (dl2 && top >= 2)) launch_l2l_path(c, lo, s2);
      return;
    }
    for (size_t i = 0; i < dl.size(); ++i) {
      launch_l2l_add(c, dl[i], s2, dr[i], dnr[i]);
      if (dl[i] == 1)  // periodic: the lattice and level 1's own M2L in one product
        launch_lattice(c, s2);
      else
        launch_gemm_f64(c, c->op_m2l, kModeM2L, dl[i], s2, dr[i], dnr[i]);
    }
    if (dl2 && top >= 2) launch_l2l_add(c, top, s2);
  };
  // 3a. bottom intermediate field: M2P from level l-1 cells (bottom mode 1: in
  // the local expansions already)
  auto m2p = [&](cudaStream_t s2, int sm_budget) {
    if (m1) return;
    if (dl2) {  // M2P from the level l-2 interaction list, P2P from the ring of level-l cells
      const int l2 = lmax - 2, l1 = lmax - 1;
      if (f64) {
        launch_gemm_f64(c, c->op_m2p2, kModeM2P2, l2, s2);
        launch_gemm_f64(c, c->op_p2pr, kModeP2PR, l1, s2);
      } else {
        launch_gemm_tc(c, c->op_m2p2, kModeM2P2, &l2, 1, s2, nullptr, nullptr, sm_budget);
        launch_gemm_tc(c, c->op_p2pr, kModeP2PR, &l1, 1, s2, nullptr, nullptr, sm_budget);
      }
      return;
    }
    std::vector<int> lv;
    for (int l = lo; l <= lmax; ++l) {
      if (!c->lev[l].n_leaf) continue;
      if (f64)
        launch_gemm_f64(c, c->op_m2p, kModeM2P, l - 1, s2);
      else
        lv.push_back(l - 1);
    }
    if (!f64 && !lv.empty())
      launch_gemm_tc(c, c->op_m2p, kModeM2P, lv.data(), (int)lv.size(), s2, nullptr, nullptr, sm_budget);
  };
  // The bottom field needs only the multipoles, so it runs on a second branch
  // beside the downward pass.  Mixed: a tcgen05 CTA fills an SM's shared
  // memory, so M2L goes first; then M2P, split over all but kM2PSideSMs SMs,
  // overlaps the latency-bound L2L chain and the near-field M2P on the rest
  // (both add atomically into the zeroed accumulator).  FP64: the DFMA
  // contractions share SMs, so the fork comes right after the upward pass, and
  // the near-field M2P follows the FP64 M2P on the same branch (both add into
  // the accumulator, zero between solves).  With stage timing on, everything
  // stays in order.
  if (!c->timing && c->aux_stream) {
    if (!f64) m2l_tc(st);
    CKS(cudaEventRecord(c->ev_fork, st));
    CKS(cudaStreamWaitEvent(c->aux_stream, c->ev_fork, 0));
    m2p(c->aux_stream, dl.empty() ? 0 : std::max(1, c->num_sms - kM2PSideSMs));
    if (f64) launch_near_m2p(c, lo, c->aux_stream);
    CKS(cudaEventRecord(c->ev_join, c->aux_stream));
    l2l_chain(st);
    if (!f64) launch_near_m2p(c, lo, st);
    CKS(cudaStreamWaitEvent(st, c->ev_join, 0));
  } else {
    if (!f64) m2l_tc(st);
    l2l_chain(st);
    stage_event(c, 2, st);
    m2p(st, 0);
    stage_event(c, 3, st);
    launch_near_m2p(c, lo, st);
    stage_event(c, 4, st);
  }
  // 3b. near / nearest / far fields and the scatter, all target levels in one launch
  launch_near(c, lo, dphi + lo, dacc + lo, c->cfg.out_fp32, st);
  stage_event(c, 5, st);
  return FMM_OK;
}

// Replays the solve as a CUDA graph: captured once per (layout generation, lo,
// output pointers) on the library's own stream, then launched on the caller's.
static fmm_status launch_solve_graph(Ctx* c, int lo, void* const* dphi, void* const* dacc, cudaStream_t st) {
  // the ancestor lists differ per updated level: their lengths are part of the key
  std::vector<uintptr_t> key = {(uintptr_t)c->layout_gen, (uintptr_t)lo, (uintptr_t)c->dirty_lo, (uintptr_t)c->anc_d};
  for (int l = 1; l < c->anc_d; ++l) key.push_back((uintptr_t)c->lev[l].n_anc);
  for (int l = lo; l <= c->lmax; ++l) {
    key.push_back((uintptr_t)dphi[l]);
    key.push_back((uintptr_t)dacc[l]);
  }
  if (drift_active(c, lo))  // the time steps are launch parameters of the drift kernels
    for (double t : c->drift_dt) {
      uint64_t bits;
      std::memcpy(&bits, &t, 8);
      key.push_back((uintptr_t)bits);
    }
  Ctx::SolveGraph* g = nullptr;
  for (auto& e : c->graphs)
    if (e.key == key) g = &e;
  if (!g) {
    // drop graphs of older layouts, and the oldest if the cache is full
    for (size_t i = 0; i < c->graphs.size();)
      if (c->graphs[i].key[0] != (uintptr_t)c->layout_gen || c->graphs.size() >= 8) {
        cudaGraphExecDestroy(c->graphs[i].exec);
        c->graphs.erase(c->graphs.begin() + i);
      } else {
        ++i;
      }
    if (!c->cap_stream) CKS(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    const int64_t n0 = c->n_launch;
    CKS(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    fmm_status s = enqueue_solve(c, lo, dphi, dacc, c->cap_stream);
    cudaGraph_t graph = nullptr;
    cudaError_t ee = cudaStreamEndCapture(c->cap_stream, &graph);
    if (s != FMM_OK) {
      if (graph) cudaGraphDestroy(graph);
      return s;
    }
    CKS(ee);
    cudaGraphExec_t exec = nullptr;
    cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    CKS(ei);
    c->graphs.push_back({key, exec, c->n_launch - n0});
    c->n_launch = n0;  // counted when launched
    ++c->n_graph_build;
    g = &c->graphs.back();
  }
  CKS(cudaGraphLaunch(g->exec, st));
  c->n_launch += g->launches;
  ++c->n_graph_launch;
  return FMM_OK;
}

fmm_status fmm_solve(fmm_ctx* c, int lo, void* const* phi, void* const* accel, void* stream) {
  if (!c || !phi || !accel) return FMM_ERR_ARG;
  if (!c->have_levels) {
    c->last_error = "fmm_solve before fmm_set_levels";
    return FMM_ERR_STATE;
  }
  if (lo < c->lmin || lo > c->lmax_user) return FMM_ERR_ARG;
  const bool drift = drift_active(c, lo);
  if (drift)
    for (int j = c->lmin; j < lo && j <= c->lmax; ++j)
      if (c->drift_dt[j - c->lmin] != 0.0 && c->lev[j].n_leaf && !c->lev[j].vel_valid) {
        c->last_error = "fmm_solve: drifting level " + std::to_string(j) + " needs its velocities (fmm_set_velocities)";
        return FMM_ERR_STATE;
      }
  cudaStream_t st = (cudaStream_t)stream;
  c->last_stream = st;
  ++c->n_solve;
  if (lo > c->lmax) return FMM_OK;  // only empty levels
  const int ob = c->cfg.out_fp32 ? 4 : 8;
  // outputs: device pointers are written directly, host pointers go through staging
  std::vector<void*> dphi(c->lmax + 1, nullptr), dacc(c->lmax + 1, nullptr);
  std::vector<char> host_out(c->lmax + 1, 0);
  size_t stage_bytes = 0;
  for (int l = lo; l <= c->lmax; ++l) {
    int64_t nl = c->lev[l].n_leaf;
    if (!nl) continue;
    if (!phi[l - lo] || !accel[l - lo]) return FMM_ERR_ARG;
    host_out[l] = !(is_device_ptr(phi[l - lo]) && is_device_ptr(accel[l - lo]));
    if (host_out[l]) stage_bytes += nl * 4 * ob + 256;
  }
  if (stage_bytes) {
    if (c->out_stage.bytes < stage_bytes) {
      // only host outputs ever allocate here; device outputs never do
      CKS(buf_ensure(c, c->out_stage, stage_bytes));
    }
    size_t off = 0;
    for (int l = lo; l <= c->lmax; ++l)
      if (host_out[l]) {
        int64_t nl = c->lev[l].n_leaf;
        dphi[l] = (char*)c->out_stage.ptr + off;
        off += (nl * ob + 255) / 256 * 256;
        dacc[l] = (char*)c->out_stage.ptr + off;
        off += (nl * 3 * ob + 255) / 256 * 256;
      }
  }
  for (int l = lo; l <= c->lmax; ++l)
    if (!host_out[l]) {
      dphi[l] = phi[l - lo];
      dacc[l] = accel[l - lo];
    }

  if (c->timing || !c->use_graphs) {
    TRY(enqueue_solve(c, lo, dphi.data(), dacc.data(), st));
  } else {
    TRY(launch_solve_graph(c, lo, dphi.data(), dacc.data(), st));
  }
  // every multipole now matches the current masses, unless drift corrections
  // were added to them
  c->dirty_lo = drift ? c->lmin : Ctx::kClean;
  CKS(cudaGetLastError());
  for (int l = lo; l <= c->lmax; ++l)
    if (host_out[l]) {
      int64_t nl = c->lev[l].n_leaf;
      CKS(cudaMemcpyAsync(phi[l - lo], dphi[l], nl * ob, cudaMemcpyDeviceToHost, st));
      CKS(cudaMemcpyAsync(accel[l - lo], dacc[l], nl * 3 * ob, cudaMemcpyDeviceToHost, st));
    }
  return FMM_OK;
}

fmm_status fmm_batch_solve(fmm_ctx* const* ctxs, int nctx, const int* lo, void* const* const* phi,
                           void* const* const* accel, void* stream) {
  if (!ctxs || nctx < 0 || (nctx && (!lo || !phi || !accel))) return FMM_ERR_ARG;
  if (!nctx) return FMM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = -1;
  std::vector<uintptr_t> key = {(uintptr_t)nctx};
  std::vector<std::vector<void*>> dphi(nctx), dacc(nctx);
  for (int i = 0; i < nctx; ++i) {
    Ctx* c = ctxs[i];
    if (!c || !phi[i] || !accel[i]) return FMM_ERR_ARG;
    if (!c->have_levels) {
      c->last_error = "fmm_batch_solve before fmm_set_levels";
      return FMM_ERR_STATE;
    }
    if (lo[i] < c->lmin || lo[i] > c->lmax_user) return FMM_ERR_ARG;
    if (dev < 0) dev = c->device;
    if (c->device != dev) {
      c->last_error = "fmm_batch_solve: contexts on different devices";
      return FMM_ERR_ARG;
    }
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == c) {
        c->last_error = "fmm_batch_solve: a context appears twice";
        return FMM_ERR_ARG;
      }
    dphi[i].assign(std::max(c->lmax, lo[i]) + 1, nullptr);
    dacc[i].assign(std::max(c->lmax, lo[i]) + 1, nullptr);
    key.insert(key.end(), {(uintptr_t)c, (uintptr_t)c->layout_gen, (uintptr_t)lo[i], (uintptr_t)c->dirty_lo,
                           (uintptr_t)c->anc_d});
    for (int l = 1; l < c->anc_d; ++l) key.push_back((uintptr_t)c->lev[l].n_anc);
    for (int l = lo[i]; l <= c->lmax; ++l) {
      if (!c->lev[l].n_leaf) continue;
      void* pp = phi[i][l - lo[i]];
      void* pa = accel[i][l - lo[i]];
      if (!is_device_ptr(pp) || !is_device_ptr(pa)) {
        c->last_error = "fmm_batch_solve takes device outputs only";
        return FMM_ERR_ARG;
      }
      dphi[i][l] = pp;
      dacc[i][l] = pa;
      key.push_back((uintptr_t)pp);
      key.push_back((uintptr_t)pa);
    }
  }
  std::lock_guard<std::mutex> lock(g_batch_mu);
  BatchGraph* g = nullptr;
  for (auto& b : g_batch)
    if (b.key == key) g = &b;
  if (!g) {
    Ctx* c0 = ctxs[0];
    Ctx* c = c0;  // error text goes to the first context
    if (g_batch_dev != dev) {
      for (auto& x : g_batch_streams)
        if (!x) CKS(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
      g_batch_dev = dev;
    }
    while (g_batch.size() >= 4) {
      cudaGraphExecDestroy(g_batch.front().exec);
      g_batch.erase(g_batch.begin());
    }
    cudaStream_t cap = g_batch_streams[0];
    std::vector<cudaEvent_t> evs(kBatchBranches + 1, nullptr);
    for (auto& e : evs) CKS(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    BatchGraph b;
    b.key = key;
    fmm_status s = FMM_OK;
    cudaError_t ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) ce = cudaEventRecord(evs[0], cap);
    const int nbr = std::min(nctx, kBatchBranches);
    for (int j = 0; j < nbr && ce == cudaSuccess; ++j) ce = cudaStreamWaitEvent(g_batch_streams[1 + j], evs[0], 0);
    for (int i = 0; i < nctx && ce == cudaSuccess && s == FMM_OK; ++i) {
      Ctx* c = ctxs[i];
      const bool timing = c->timing;
      c->timing = false;
      const int64_t n0 = c->n_launch;
      s = enqueue_solve(c, lo[i], dphi[i].data(), dacc[i].data(), g_batch_streams[1 + i % kBatchBranches]);
      b.ctxs.push_back(c);
      b.launches.push_back(c->n_launch - n0);
      c->n_launch = n0;
      c->timing = timing;
    }
    for (int j = 0; j < nbr && ce == cudaSuccess; ++j) {
      ce = cudaEventRecord(evs[1 + j], g_batch_streams[1 + j]);
      if (ce == cudaSuccess) ce = cudaStreamWaitEvent(cap, evs[1 + j], 0);
    }
    cudaGraph_t graph = nullptr;
    cudaError_t ee = cudaStreamEndCapture(cap, &graph);
    for (auto& e : evs) cudaEventDestroy(e);
    if (s != FMM_OK || ce != cudaSuccess || ee != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      if (s == FMM_OK) {
        c0->last_error = std::string("fmm_batch_solve capture: ") +
                         cudaGetErrorString(ce != cudaSuccess ? ce : ee);
        s = FMM_ERR_CUDA;
      }
      return s;
    }
    cudaError_t ei = cudaGraphInstantiate(&b.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      c0->last_error = std::string("fmm_batch_solve instantiate: ") + cudaGetErrorString(ei);
      return FMM_ERR_CUDA;
    }
    g_batch.push_back(std::move(b));
    g = &g_batch.back();
  }
  cudaError_t e = cudaGraphLaunch(g->exec, st);
  if (e != cudaSuccess) {
    ctxs[0]->last_error = std::string("fmm_batch_solve launch: ") + cudaGetErrorString(e);
    return FMM_ERR_CUDA;
  }
  for (size_t i = 0; i < g->ctxs.size(); ++i) {
    g->ctxs[i]->n_launch += g->launches[i];
    ++g->ctxs[i]->n_solve;
    g->ctxs[i]->last_stream = st;
    g->ctxs[i]->dirty_lo = drift_active(g->ctxs[i], lo[i]) ? g->ctxs[i]->lmin : Ctx::kClean;
  }
  return FMM_OK;
}

// Times the candidate launch shapes on the context's own hierarchy (direct
// launches, CUDA events, best of 3 after a warm-up) and keeps the fastest:
// split-K of the two tcgen05 contractions (mixed precision), then the
// near-field octs per block.
fmm_status fmm_autotune(fmm_ctx* c, int lo, void* stream) {
  if (!c) return FMM_ERR_ARG;
  if (!c->have_levels) {
    c->last_error = "fmm_autotune before fmm_set_levels";
    return FMM_ERR_STATE;
  }
  if (lo < c->lmin || lo > c->lmax_user) return FMM_ERR_ARG;
  if (lo > c->lmax) return FMM_OK;  // nothing to time
  cudaStream_t st = (cudaStream_t)stream;
  c->last_stream = st;
  const int ob = c->cfg.out_fp32 ? 4 : 8;
  size_t bytes = 0;
  for (int l = lo; l <= c->lmax; ++l) bytes += (c->lev[l].n_leaf * 4 * ob + 255) / 256 * 256 + 256;
  CKS(buf_ensure(c, c->out_stage, bytes));
  std::vector<void*> dphi(c->lmax + 1, nullptr), dacc(c->lmax + 1, nullptr);
  size_t off = 0;
  for (int l = lo; l <= c->lmax; ++l) {
    const int64_t nl = c->lev[l].n_leaf;
    dphi[l] = (char*)c->out_stage.ptr + off;
    off += (nl * ob + 255) / 256 * 256;
    dacc[l] = (char*)c->out_stage.ptr + off;
    off += (nl * 3 * ob + 255) / 256 * 256;
  }
  const bool timing = c->timing;
  c->timing = false;
  const int anc_d = c->anc_d;
  c->anc_d = 0;  // time the full passes
  c->tune_lo = lo;  // the split factors tuned here serve solves from lo
  cudaEvent_t e0, e1;
  CKS(cudaEventCreate(&e0));
  CKS(cudaEventCreate(&e1));
  auto measure = [&](float& best) -> fmm_status {
    best = 1e30f;
    for (int r = 0; r < 4; ++r) {
      c->dirty_lo = c->lmin;
      CKS(cudaEventRecord(e0, st));
      TRY(enqueue_solve(c, lo, dphi.data(), dacc.data(), st));
      CKS(cudaEventRecord(e1, st));
      CKS(cudaEventSynchronize(e1));
      float ms = 0;
      CKS(cudaEventElapsedTime(&ms, e0, e1));
      if (r > 0) best = std::min(best, ms);  // the first run warms up
    }
    return FMM_OK;
  };
  const int64_t n0 = c->n_launch;
  fmm_status s = FMM_OK;
  auto tune = [&](int* knob, const std::vector<int>& cands) {
    int best_v = *knob;
    float best_t = 1e30f;
    for (int v : cands) {
      if (s != FMM_OK) return;
      *knob = v;
      float t;
      s = measure(t);
      if (s == FMM_OK && t < best_t * 0.98f) {  // keep the earlier (simpler) choice within 2%
        best_t = t;
        best_v = v;
      }
    }
    *knob = best_v;
  };
  if (c->cfg.precision != FMM_FP64) {
    const std::vector<int> splits = {0, 1, 2, 3, 4, 6, 8, 12, 16, 24};
    if (c->cfg.bottom_mode == FMM_BOTTOM_M2P) tune(&c->tune_split[0], splits);  // mode 1 runs no M2P
    tune(&c->tune_split[1], splits);
    tune(&c->tune_opb, {16, 8});
  }
  c->n_launch = n0;  // tuning runs are not the caller's solves
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->timing = timing;
  c->anc_d = anc_d;
  c->dirty_lo = s == FMM_OK ? Ctx::kClean : c->lmin;
  ++c->layout_gen;  // cached graphs carry the old launch shapes
  if (s == FMM_OK) s = fmm_sync(c);
  return s;
}

fmm_status fmm_set_tuning(fmm_ctx* c, const int* in3) {
  if (!c || !in3 || in3[0] < 0 || in3[1] < 0 || in3[2] < 0) return FMM_ERR_ARG;
  c->tune_split[0] = in3[0];
  c->tune_split[1] = in3[1];
  c->tune_opb = in3[2];
  c->tune_lo = -1;
  ++c->layout_gen;
  return FMM_OK;
}

fmm_status fmm_get_tuning(const fmm_ctx* c, int* out3) {
  if (!c || !out3) return FMM_ERR_ARG;
  out3[0] = c->tune_split[0];
  out3[1] = c->tune_split[1];
  out3[2] = near_opb(c);
  return FMM_OK;
}


fmm_status fmm_solve_adjoint(fmm_ctx* c, int lo, const void* const* g_phi, const void* const* g_accel,
                             double* const* g_mass, void* stream) {
  if (!c || !g_phi || !g_accel || !g_mass) return FMM_ERR_ARG;
  if (!c->have_levels) {
    c->last_error = "fmm_solve_adjoint before fmm_set_levels";
    return FMM_ERR_STATE;
  }
  if (c->cfg.precision != FMM_FP64) {
    c->last_error = "fmm_solve_adjoint needs an FMM_FP64 context";
    return FMM_ERR_ARG;
  }
  if (c->cfg.delta_l == 2 || c->cfg.periodic) {
    c->last_error = "fmm_solve_adjoint: isolated boundaries and delta_l = 1 only";
    return FMM_ERR_ARG;
  }
  if (c->cfg.bottom_mode != FMM_BOTTOM_M2P) {
    c->last_error = "fmm_solve_adjoint: the transposed chain follows the paper's bottom M2P only";
    return FMM_ERR_ARG;
  }
  if (lo < c->lmin || lo > c->lmax_user) return FMM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  c->last_stream = st;
  const int lmin = c->lmin, lmax = c->lmax;
  const int ib = c->cfg.out_fp32 ? 4 : 8;
  for (int l = lo; l <= lmax; ++l)
    if (c->lev[l].n_leaf && (!g_phi[l - lo] || !g_accel[l - lo])) return FMM_ERR_ARG;
  for (int l = lmin; l <= lmax; ++l)
    if (c->lev[l].n_leaf && !g_mass[l - lmin]) return FMM_ERR_ARG;
  for (int l = 1; l <= lmax; ++l)  // before the lists: an allocation here changes the layout generation
    CKS(buf_ensure(c, c->lev[l].gmass, std::max<int64_t>(c->lev[l].n_leaf, 1) * 8));
  TRY(adjoint_tables(c));
  TRY(adjoint_lists(c, st));
  // cotangent inputs: host arrays are staged on the device
  std::vector<const void*> dphi(lmax + 1, nullptr), dacc(lmax + 1, nullptr);
  size_t in_bytes = 0;
  for (int l = lo; l <= lmax; ++l)
    if (c->lev[l].n_leaf && !(is_device_ptr(g_phi[l - lo]) && is_device_ptr(g_accel[l - lo])))
      in_bytes += (c->lev[l].n_leaf * 4 * ib + 255) / 256 * 256 + 256;
  if (in_bytes) CKS(buf_ensure(c, c->in_stage, in_bytes));
  size_t off = 0;
  for (int l = lo; l <= lmax; ++l) {
    const int64_t nl = c->lev[l].n_leaf;
    if (!nl) continue;
    if (is_device_ptr(g_phi[l - lo]) && is_device_ptr(g_accel[l - lo])) {
      dphi[l] = g_phi[l - lo];
      dacc[l] = g_accel[l - lo];
      continue;
    }
    char* p = (char*)c->in_stage.ptr + off;
    CKS(cudaMemcpyAsync(p, g_phi[l - lo], nl * ib, cudaMemcpyDefault, st));
    dphi[l] = p;
    off += (nl * ib + 255) / 256 * 256;
    p = (char*)c->in_stage.ptr + off;
    CKS(cudaMemcpyAsync(p, g_accel[l - lo], nl * 3 * ib, cudaMemcpyDefault, st));
    dacc[l] = p;
    off += (nl * 3 * ib + 255) / 256 * 256;
  }
  // cotangent buffers: the FP64 expansion arrays and one mass array per level
  for (int l = 1; l <= lmax; ++l) {
    LevelTree& T = c->lev[l];
    if (T.n_leaf) CKS(cudaMemsetAsync(T.gmass.ptr, 0, T.n_leaf * 8, st));
    if (l < lmax) CKS(cudaMemsetAsync(T.M.ptr, 0, 8 * T.n_oct * c->tab.nc * 8, st));
    if (l >= 2 && l <= lmax - 2)
      CKS(cudaMemsetAsync(T.L.ptr, 0, 8 * std::max<int64_t>(T.n_rowsL, 1) * c->tab.nc * 8, st));
    if (l >= lmin) CKS(cudaMemsetAsync(T.acc.ptr, 0, 8 * T.n_oct * 4 * 8, st));
  }
  launch_adjoint(c, lo, dphi.data() + lo, dacc.data() + lo, c->cfg.out_fp32, st);
  c->dirty_lo = lmin;  // the expansion arrays now hold cotangents
  // the M2P accumulators are zero between forward solves (the contractions add into them)
  for (int l = lmin; l <= lmax; ++l)
    if (c->lev[l].acc.ptr) CKS(cudaMemsetAsync(c->lev[l].acc.ptr, 0, c->lev[l].acc.bytes, st));
  CKS(cudaGetLastError());
  for (int l = lmin; l <= lmax; ++l) {
    const int64_t nl = c->lev[l].n_leaf;
    if (nl) CKS(cudaMemcpyAsync(g_mass[l - lmin], c->lev[l].gmass.ptr, nl * 8, cudaMemcpyDefault, st));
  }
  return FMM_OK;
}

fmm_status fmm_update_masses(fmm_ctx* c, int lo, const void* const* mass, void* stream) {
  if (!c || !mass) return FMM_ERR_ARG;
  if (!c->have_levels) {
    c->last_error = "fmm_update_masses before fmm_set_levels";
    return FMM_ERR_STATE;
  }
  if (lo < c->lmin || lo > c->lmax_user) return FMM_ERR_ARG;
  for (int l = lo; l <= c->lmax; ++l)
    if (c->lev[l].n_leaf && !mass[l - lo]) return FMM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  c->last_stream = st;
  if (c->cfg.mass_fp32) {
    int64_t nmax = 1;
    for (int l = lo; l <= c->lmax; ++l) nmax = std::max(nmax, c->lev[l].n_leaf);
    CKS(buf_ensure(c, c->mass_stage, nmax * 4));
  }
  if (!stage_device_inputs(c, lo, c->lmax - lo + 1, nullptr, mass, st)) {
    cudaGetLastError();
    for (int l = lo; l <= c->lmax; ++l) TRY(copy_masses(c, c->lev[l], mass[l - lo], c->lev[l].n_leaf, st));
  }
  c->dirty_lo = std::min(c->dirty_lo, lo);
  return FMM_OK;
}

fmm_status fmm_set_velocities(fmm_ctx* c, int lo, const double* const* vel, void* stream) {
  if (!c || !vel) return FMM_ERR_ARG;
  if (!c->have_levels) {
    c->last_error = "fmm_set_velocities before fmm_set_levels";
    return FMM_ERR_STATE;
  }
  if (lo < c->lmin || lo > c->lmax_user) return FMM_ERR_ARG;
  for (int l = lo; l <= c->lmax; ++l)
    if (c->lev[l].n_leaf && !vel[l - lo]) return FMM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  c->last_stream = st;
  for (int l = lo; l <= c->lmax; ++l) {
    LevelTree& T = c->lev[l];
    const int64_t nl = T.n_leaf;
    CKS(buf_ensure(c, T.vel, std::max<int64_t>(nl, 1) * 24));
    if (nl) CKS(cudaMemcpyAsync(T.vel.ptr, vel[l - lo], nl * 24, cudaMemcpyDefault, st));
    T.vel_valid = true;
  }
  return FMM_OK;
}

fmm_status fmm_set_drift(fmm_ctx* c, const double* dt, int n) {
  if (!c) return FMM_ERR_ARG;
  if (!dt) {
    c->drift_dt.clear();
    return FMM_OK;
  }
  if (c->cfg.periodic) {  // the level-1 multipoles (level-1 M2L, the lattice) are not drifted
    c->last_error = "fmm_set_drift: isolated boundaries only";
    return FMM_ERR_ARG;
  }
  if (!c->have_levels) {
    c->last_error = "fmm_set_drift before fmm_set_levels";
    return FMM_ERR_STATE;
  }
  if (n != c->lmax_user - c->lmin + 1) {
    c->last_error = "fmm_set_drift: n must be lmax - lmin + 1";
    return FMM_ERR_ARG;
  }
  for (int k = 0; k < n; ++k)
    if (!std::isfinite(dt[k])) return FMM_ERR_ARG;
  c->drift_dt.assign(dt, dt + n);
  return drift_prepare(c);
}

fmm_status fmm_set_wait_limit(fmm_ctx* c, double seconds) {
  if (!c || !std::isfinite(seconds) || seconds < 0.0 || seconds > 3600.0) return FMM_ERR_ARG;
  c->wait_s = seconds;
  ++c->layout_gen;  // cached graphs carry the old limit in their launch parameters
  return FMM_OK;
}

fmm_status fmm_sync(fmm_ctx* c) {
  if (!c) return FMM_ERR_ARG;
  CKS(cudaStreamSynchronize(c->last_stream));
  unsigned e = 0;
  CKS(cudaMemcpy(&e, c->d_err, 4, cudaMemcpyDeviceToHost));
  if (c->timing) {
    for (int i = 0; i < 5; ++i) {
      float ms = 0;
      cudaEventElapsedTime(&ms, c->ev[i], c->ev[i + 1]);
      c->stage_ms[i] = ms;
    }
  }
  if (e & kErrTimeout) {
    c->last_error = "a bounded device-side wait timed out";
    cudaMemset(c->d_err, 0, 4);
    // an interrupted solve may leave partial sums behind: restore the cleared
    // accumulators and recompute every multipole next time
    if (c->have_levels) {
      for (int l = c->lmin; l <= c->lmax; ++l)
        if (c->lev[l].acc.ptr) cudaMemset(c->lev[l].acc.ptr, 0, c->lev[l].acc.bytes);
      for (int l = 2; l <= top_local_level(c); ++l)
        if (c->lev[l].Lm.ptr) cudaMemset(c->lev[l].Lm.ptr, 0, c->lev[l].Lm.bytes);
      c->dirty_lo = c->lmin;
    }
    return FMM_ERR_TIMEOUT;
  }
  return FMM_OK;
}

const char* fmm_last_error(const fmm_ctx* c) { return c ? c->last_error.c_str() : "null context"; }

void fmm_destroy(fmm_ctx* c) {
  if (!c) return;
  if (c->last_stream) cudaStreamSynchronize(c->last_stream);
  drop_batch_graphs_of(c);
  release_tables(c);
  for (auto& T : c->lev) {
    for (DevBuf* b : {&T.oct_key, &T.oct_parent, &T.cell_child, &T.nbr, &T.leaf_cell, &T.rows, &T.rowsL, &T.irows, &T.leafmask, &T.gmass, &T.srcP, &T.srcL, &T.slotL, &T.lslot, &T.anc, &T.tgt, &T.ijk,
                      &T.mass, &T.M, &T.Mhi, &T.Mlo, &T.Chi, &T.Clo, &T.mono, &T.L, &T.Lf, &T.Lm, &T.acc, &T.vel, &T.dS, &T.dQ})
      buf_free(c, *b);
  }
  for (DevBuf* b : {&c->d_m2m_off, &c->d_m2m_g, &c->d_m2m_e, &c->d_m2m_c, &c->d_l2l_off, &c->d_l2l_off8, &c->d_l2l_g,
                    &c->d_l2l_e, &c->d_l2l_c, &c->d_l2l_c32, &c->d_m2m_c32, &c->d_m2m_w0, &c->d_m2m_w0_32, &c->d_m2m_e0,
                    &c->d_m2mT_off, &c->d_m2mT_a, &c->d_m2mT_c, &c->d_l2lT_off, &c->d_l2lT_b, &c->d_l2lT_e,
                    &c->d_l2lT_c, &c->d_m2pT, &c->d_m2lT, &c->d_near64, &c->d_near32, &c->d_l2p64, &c->d_l2p32,
                    &c->op_m2p.f64, &c->op_m2p.hi, &c->op_m2p.lo, &c->op_m2p.klimit, &c->op_m2l.colmap, &c->op_m2l.f64,
                    &c->op_m2l.hi, &c->op_m2l.lo, &c->op_m2l.klimit, &c->op_m2p2.f64, &c->op_m2p2.hi,
                    &c->op_m2p2.lo, &c->op_m2p2.klimit, &c->op_p2pr.f64, &c->op_p2pr.hi, &c->op_p2pr.lo,
                    &c->op_p2pr.klimit, &c->d_lat64, &c->d_lat32, &c->sort_tmp, &c->keys_a, &c->keys_b,
                    &c->vals_a, &c->vals_b, &c->flags, &c->scan, &c->counter, &c->anc_flags, &c->out_stage, &c->in_stage,
                    &c->mass_stage, &c->err_buf, &c->d_alpha})
    buf_free(c, *b);
  c->d_err = nullptr;
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  for (auto& g : c->tree_graphs) cudaGraphExecDestroy(g.exec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->aux_stream) cudaStreamDestroy(c->aux_stream);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->ev_sync) cudaEventDestroy(c->ev_sync);
  for (auto& ev : c->ev)
    if (ev) cudaEventDestroy(ev);
  if (c->h_rb) cudaFreeHost(c->h_rb);
  delete c;
}

fmm_status fmm_tree_counts(const fmm_ctx* c, int64_t* n_oct) {
  if (!c || !n_oct) return FMM_ERR_ARG;
  if (!c->have_levels) return FMM_ERR_STATE;
  for (int l = 0; l <= c->lmax_user; ++l) n_oct[l] = (l == 0 || l > c->lmax) ? 0 : c->lev[l].n_oct;
  return FMM_OK;
}

fmm_status fmm_tree_export(const fmm_ctx* cc, int level, uint64_t* oct_key, int64_t* status, int64_t* nbr) {
  fmm_ctx* c = const_cast<fmm_ctx*>(cc);
  if (!c || !oct_key || !status || !nbr) return FMM_ERR_ARG;
  if (!c->have_levels) return FMM_ERR_STATE;
  if (level < 1 || level > c->lmax_user) return FMM_ERR_ARG;
  if (level > c->lmax) return FMM_OK;  // an empty level: no octs
  const LevelTree& T = c->lev[level];
  int64_t no = T.n_oct;
  std::vector<int32_t> cc32(8 * no), nb32(27 * no);
  CKS(cudaMemcpy(oct_key, T.oct_key.ptr, no * 8, cudaMemcpyDeviceToHost));
  CKS(cudaMemcpy(cc32.data(), T.cell_child.ptr, no * 32, cudaMemcpyDeviceToHost));
  CKS(cudaMemcpy(nb32.data(), T.nbr.ptr, no * 27 * 4, cudaMemcpyDeviceToHost));
  for (int64_t i = 0; i < 8 * no; ++i) {
    int32_t v = cc32[i];
    // the finest level has no refined cells: a non-negative entry cannot occur there
    status[i] = v;
  }
  for (int64_t i = 0; i < 27 * no; ++i) nbr[i] = nb32[i];
  return FMM_OK;
}

fmm_status fmm_host_numerators(int q, const int64_t* u, int64_t* out) {
  if (!u || !out || q < 0 || q > 12) return FMM_ERR_ARG;
  MultiIdx mi;
  mi.build(q);
  std::vector<__int128> P;
  inv_r_numerators(q, u, P, mi);
  for (int k = 0; k < mi.size(); ++k) {
    if (P[k] > (__int128)INT64_MAX || P[k] < (__int128)INT64_MIN) return FMM_ERR_ARG;
    out[k] = (int64_t)P[k];
  }
  return FMM_OK;
}

fmm_status fmm_host_table(int p, int which, double* out, int64_t n) {
  if (p < 1 || p > 8 || !out || which < 0 || which > 9) return FMM_ERR_ARG;
  Tables t;
  t.build(p);
  const int nc = t.nc;
  std::vector<double> v;
  if (which == 6) {  // the lattice tensor, |gamma| <= p
    MultiIdx mq;
    mq.build(p);
    v = lattice_tensor(p, mq);
  }
  if (which == 7) {
    t.build_lattice();
    v = t.lattice;
  }
  if (which == 8 || which == 9) {
    t.build_dl2();
    v = which == 8 ? t.m2p2 : t.p2pr;
  }
  if (which == 0) v = t.m2p;
  if (which == 1) v = t.m2l;
  if (which == 2) v = t.nearop;
  if (which == 3) v = t.l2p;
  if (which == 4 || which == 5) {
    const auto& off = which == 4 ? t.m2m_off : t.l2l_off;
    const auto& g = which == 4 ? t.m2m_g : t.l2l_g;
    const auto& e = which == 4 ? t.m2m_e : t.l2l_e;
    const auto& cf = which == 4 ? t.m2m_c : t.l2l_c;
    v.assign((size_t)8 * nc * nc, 0.0);
    for (int c = 0; c < 8; ++c)
      for (int a = 0; a < nc; ++a)
        for (int j = off[a]; j < off[a + 1]; ++j)
          v[((size_t)c * nc + a) * nc + g[j]] += cf[j] * child_sign(c, e[j]);
  }
  if ((int64_t)v.size() > n) return FMM_ERR_ARG;
  std::memcpy(out, v.data(), v.size() * sizeof(double));
  return FMM_OK;
}

fmm_status fmm_stats(const fmm_ctx* c, int64_t* out4) {
  if (!c || !out4) return FMM_ERR_ARG;
  out4[0] = c->n_launch;
  out4[1] = c->n_cub;
  out4[2] = c->n_solve;
  out4[3] = c->n_set;
  return FMM_OK;
}

fmm_status fmm_set_graphs(fmm_ctx* c, int on) {
  if (!c) return FMM_ERR_ARG;
  c->use_graphs = on != 0;
  return FMM_OK;
}

fmm_status fmm_set_timing(fmm_ctx* c, int on) {
  if (!c) return FMM_ERR_ARG;
  c->timing = on != 0;
  return FMM_OK;
}

fmm_status fmm_stage_times(const fmm_ctx* c, double* ms5) {
  if (!c || !ms5) return FMM_ERR_ARG;
  for (int i = 0; i < 5; ++i) ms5[i] = c->stage_ms[i];
  return FMM_OK;
}

}  // extern "C"
