// gemm_tc.cu -- M2L (Eq. 3) and bottom M2P (Fig. 2, Alg. 4) on the 5th
// generation tensor cores (tcgen05) in split-BF16 with FP32 accumulation.
//
// D[row][n] = sum_k A[row][k] B[n][k] where a row is an oct of the source
// grid, k = (q, s, alpha) runs over the 26 neighbour octs of its parent, their
// 8 cells and the multipole coefficients, and B is the translation operator
// (translation invariant, so one table serves every oct and every level).
// Each operand is split x = hi + lo with hi, lo in BF16; the product keeps
// hi*hi + hi*lo + lo*hi (the lo*lo term is below FP32 rounding).
//
// Per CTA: 128 rows x BN columns, accumulator in tensor memory (TMEM).
//   warps 0-3  gather A rows with cp.async into 64B-swizzled shared memory
//              (the rows are neighbour octs, so TMA tiles cannot fetch them),
//              then run the epilogue (tcgen05.ld, scatter-add to the targets)
//   warp 4     allocates TMEM and loads B tiles with TMA (SWIZZLE_64B)
//   warp 5     one thread issues tcgen05.mma (M=128, N=BN, K=16) per slice
// Split-K over grid.z; partial sums are added with atomics.  Every wait on an
// mbarrier is bounded by a wall-clock limit; on expiry the CTA latches
// kErrTimeout, skips the remaining work and still frees its TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "fmm_internal.cuh"

namespace fmm {
namespace {

constexpr int BM = 128;
constexpr int BK = 32;  // bf16 elements per row per stage = 64 bytes (64-byte swizzle)
constexpr int STAGES = 4;
constexpr int kNbrStride = 27;  // shared-memory row stride of the per-row neighbour table
constexpr int THREADS = 192;
constexpr int kMaxSeg = 24;
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s

__constant__ int c_nbr26[26] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12,
                                14, 15, 16, 17, 18, 19, 20, 21, 22, 23, 24, 25, 26};

// One segment = the rows of one level: its sources, neighbour table and output.
struct TcSeg {
  const __nv_bfloat16* Ahi;
  const __nv_bfloat16* Alo;
  const int32_t* rows;
  const int32_t* nbr;
  const int32_t* cell_child_rows;  // M2P: cell_child of the row level
  const int32_t* cell_child_tgt;   // M2P: cell_child of the target level (refined targets get nothing)
  const int32_t* slot;             // M2L: local-expansion slot of each row oct
  float* out;                      // M2P: [cells of target level][4]; M2L: [slot*8 + cell][nc]
  int nrows;
  int tile0;                       // first M tile of this segment
};

struct TcParams {
  TcSeg seg[kMaxSeg];
  int nseg;
  int KQ;          // K per neighbour offset (8 * nc)
  int Kvalid;      // 26 * KQ
  int nchunks;     // Kpad / BK
  int chunks_per_split;
  int BN, N, nc, mode;
  unsigned* err;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: returns false (and sets *abort) if the phase did not complete
// within kWaitLimitNs or another thread already aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort) {
  if (mbar_try(bar, parity)) return true;
  uint64_t t0 = now_ns();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try(bar, parity)) return true;
    if ((i & 1023) == 0) {
      if (*abort) return false;
      if (now_ns() - t0 > kWaitLimitNs) {
        *abort = 1;
        return false;
      }
    }
  }
}

// K-major operand tile, rows of BK bf16 (64 B), 64-byte swizzle: the 16-byte
// chunk j of row r sits at chunk j ^ ((r >> 1) & 3); 8 rows form a 512 B atom.
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);  // start address
  d |= (uint64_t)1 << 16;                  // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(512 >> 4) << 32;         // stride byte offset: 8 rows x 64 B
  d |= (uint64_t)1 << 46;                  // descriptor version for tcgen05
  d |= (uint64_t)4 << 61;                  // 64-byte swizzle
  return d;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* tm, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"((uint64_t)tm), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum));
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

#define TMEM_LD32(taddr, v)                                                                              \
  asm volatile(                                                                                          \
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"  \
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                        \
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), \
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),        \
        "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),      \
        "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),      \
        "=r"(v[29]), "=r"(v[30]), "=r"(v[31])                                                           \
      : "r"(taddr))

__global__ void __launch_bounds__(THREADS, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_lo, TcParams P) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned carve-up
  uintptr_t base = ((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023;
  unsigned char* sm = (unsigned char*)base;
  const int a_bytes = BM * BK * 2;        // 16 KB
  const int b_bytes = P.BN * BK * 2;      // BN * 128
  unsigned char* Ahi = sm;
  unsigned char* Alo = Ahi + STAGES * a_bytes;
  unsigned char* Bhi = Alo + STAGES * a_bytes;
  unsigned char* Blo = Bhi + STAGES * b_bytes;
  uint64_t* bars = (uint64_t*)(Blo + STAGES * b_bytes);  // full[S], empty[S], done
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * STAGES + 1);
  volatile int* abort = (volatile int*)(tmem_slot + 1);
  int32_t* s_nbr = (int32_t*)(tmem_slot + 4);  // [BM][kNbrStride] source octs of each row

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kc_begin = blockIdx.z * P.chunks_per_split;
  const int kc_end = min(P.nchunks, kc_begin + P.chunks_per_split);
  const int nit = max(0, kc_end - kc_begin);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES), done = smem_u32(bars + 2 * STAGES);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 129);  // 128 gathering threads + 1 TMA arrive
      mbar_init(empty0 + 8 * s, 1);   // tcgen05.commit
    }
    mbar_init(done, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const uint32_t ncols = P.BN <= 32 ? 32 : (P.BN <= 64 ? 64 : (P.BN <= 128 ? 128 : 256));
  if (warp == 4) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  pdl_wait();  // rows, neighbour tables and multipoles come from earlier kernels
  pdl_trigger();

  if (warp < 4) {
    // ---------------- A gather ----------------
    // Thread t owns row t for the epilogue (TMEM lane t) and writes that row's
    // neighbour table.  The copies are spread differently: four lanes fetch the
    // four 16-byte chunks of one row's 64-byte slice, eight rows per
    // instruction, so every 32-byte sector is requested once and whole.
    const int t = threadIdx.x;
    int si = 0;
    while (si + 1 < P.nseg && (int)blockIdx.x >= P.seg[si + 1].tile0) ++si;
    const TcSeg& S = P.seg[si];
    const int64_t row_idx = (int64_t)(blockIdx.x - S.tile0) * BM + t;
    const bool valid = row_idx < S.nrows;
    const int32_t roct = valid ? S.rows[row_idx] : 0;
    int32_t* myn = s_nbr + t * kNbrStride;
    for (int q = 0; q < 26; ++q) myn[q] = valid ? S.nbr[(int64_t)roct * 27 + c_nbr26[q]] : -1;
    __syncwarp();  // each warp gathers its own 32 rows and reads their tables below
    const int jj = lane & 3;  // 16-byte chunk within the row slice
    uint32_t nbr_s[4], dst[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = warp * 32 + i * 8 + (lane >> 2);
      nbr_s[i] = smem_u32(s_nbr + r * kNbrStride);  // read back with ld.shared (a plain pointer would be generic)
      dst[i] = (uint32_t)(r * (BK * 2)) + (uint32_t)((jj ^ ((r >> 1) & 3)) << 4);
    }
    const uint32_t ahi0 = smem_u32(Ahi), alo0 = smem_u32(Alo);
    // Up to three stages of copies in flight: after committing stage it, wait
    // for stage it-2 and mark it full.
    constexpr int kInFlight = 2;
    bool ok = true;
    for (int it = 0; it < nit && ok; ++it) {
      const int s = it % STAGES;
      if (it >= STAGES) ok = mbar_wait(empty0 + 8 * s, ((it / STAGES) - 1) & 1, abort);
      if (!ok) break;
      const int k = (kc_begin + it) * BK + 8 * jj;  // 8 elements never straddle an offset segment (KQ % 8 == 0)
      int qi = -1, off = 0;
      if (k < P.Kvalid) {
        qi = k / P.KQ;
        off = k - qi * P.KQ;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        int32_t src = -1;
        if (qi >= 0) asm volatile("ld.shared.b32 %0, [%1];" : "=r"(src) : "r"(nbr_s[i] + 4 * qi));
        const __nv_bfloat16* gh = src >= 0 ? S.Ahi + (int64_t)src * P.KQ + off : S.Ahi;
        const __nv_bfloat16* gl = src >= 0 ? S.Alo + (int64_t)src * P.KQ + off : S.Alo;
        const uint32_t sz = src >= 0 ? 16u : 0u;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(ahi0 + s * a_bytes + dst[i]), "l"(gh),
                     "r"(sz)
                     : "memory");
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(alo0 + s * a_bytes + dst[i]), "l"(gl),
                     "r"(sz)
                     : "memory");
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
      if (it >= kInFlight) {
        asm volatile("cp.async.wait_group %0;" ::"n"(kInFlight) : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(full0 + 8 * ((it - kInFlight) % STAGES));
      }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (ok)  // the stages committed but not yet marked full
      for (int r = max(0, nit - kInFlight); r < nit; ++r) mbar_arrive(full0 + 8 * (r % STAGES));

    // ---------------- epilogue ----------------
    bool have = ok && nit > 0 && mbar_wait(done, 0, abort);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int nchunk = P.BN / 32;
    for (int j = 0; j < nchunk; ++j) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(j * 32);
      TMEM_LD32(taddr, v);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (!have || !valid) continue;
      const int n0 = blockIdx.y * P.BN + j * 32;
      if (P.mode == kModeM2P) {
        const int f = n0 >> 5;
        const int32_t ch = S.cell_child_rows[(int64_t)roct * 8 + f];
        if (ch >= 0) {
          float* dst = S.out + (int64_t)ch * 32;
          const int32_t* cct = S.cell_child_tgt + (int64_t)ch * 8;
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (cct[u] < 0)  // leaf targets only: the accumulator of refined cells stays zero
              asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst + 4 * u),
                           "f"(__uint_as_float(v[4 * u])), "f"(__uint_as_float(v[4 * u + 1])),
                           "f"(__uint_as_float(v[4 * u + 2])), "f"(__uint_as_float(v[4 * u + 3]))
                           : "memory");
        }
      } else {
        float* dst = S.out + (int64_t)S.slot[roct] * 8 * P.nc + n0;
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (n0 + 4 * u < P.N)
            asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst + 4 * u),
                         "f"(__uint_as_float(v[4 * u])), "f"(__uint_as_float(v[4 * u + 1])),
                         "f"(__uint_as_float(v[4 * u + 2])), "f"(__uint_as_float(v[4 * u + 3]))
                         : "memory");
      }
    }
  } else if (warp == 4) {
    // ---------------- B tiles by TMA ----------------
    if (lane == 0) {
      bool ok = true;
      for (int it = 0; it < nit && ok; ++it) {
        const int s = it % STAGES;
        if (it >= STAGES) ok = mbar_wait(empty0 + 8 * s, ((it / STAGES) - 1) & 1, abort);
        if (!ok) break;
        const int k0 = (kc_begin + it) * BK;
        const int n0 = blockIdx.y * P.BN;
        mbar_arrive_tx(full0 + 8 * s, 2u * (uint32_t)b_bytes);
        tma_load_2d(smem_u32(Bhi + s * b_bytes), &tm_hi, k0, n0, full0 + 8 * s);
        tma_load_2d(smem_u32(Blo + s * b_bytes), &tm_lo, k0, n0, full0 + 8 * s);
      }
    }
    __syncwarp();
  } else {
    // ---------------- MMA issue ----------------
    if (lane == 0) {
      // kind::f16, D = F32, A = B = BF16, both K-major, M = 128, N = BN
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(P.BN >> 3) << 17) |
                             ((uint32_t)(BM >> 4) << 24);
      bool ok = true;
      for (int it = 0; it < nit && ok; ++it) {
        const int s = it % STAGES;
        ok = mbar_wait(full0 + 8 * s, (it / STAGES) & 1, abort);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t ah = smem_u32(Ahi + s * a_bytes), al = smem_u32(Alo + s * a_bytes);
        const uint32_t bh = smem_u32(Bhi + s * b_bytes), bl = smem_u32(Blo + s * b_bytes);
#pragma unroll
        for (int part = 0; part < 3; ++part) {
          const uint32_t a = (part == 2) ? al : ah;
          const uint32_t b = (part == 1) ? bl : bh;
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint32_t accum = (it | part | kk) != 0;
            mma_bf16(tmem, sdesc_sw64(a + kk * 32), sdesc_sw64(b + kk * 32), idesc, accum);
          }
        }
        mma_commit(empty0 + 8 * s);
      }
      if (ok && nit > 0) mma_commit(done);
    }
    __syncwarp();
  }
  if (*abort && threadIdx.x == 0) atomicOr(P.err, kErrTimeout);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 4) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

size_t smem_bytes(int BN) {
  return 1024 + STAGES * (2 * BM * BK * 2 + 2 * BN * BK * 2) + (2 * STAGES + 1) * 8 + 16 + BM * kNbrStride * 4;
}

// split-K factor minimising waves x chunks per CTA
int choose_split(int tiles, int nchunks, int nsm) {
  int best = 1;
  double best_t = 1e30;
  for (int s = 1; s <= 32 && s <= nchunks; ++s) {
    int cps = (nchunks + s - 1) / s;
    int ctas = tiles * ((nchunks + cps - 1) / cps);
    int waves = (ctas + nsm - 1) / nsm;
    double t = (double)waves * (cps + 2);  // +2: pipeline fill and epilogue
    if (t < best_t - 1e-9) {
      best_t = t;
      best = s;
    }
  }
  return best;
}

}  // namespace

fmm_status make_tensor_maps(Ctx* c, GemmOperand& op) {
  auto enc = get_encode();
  if (!enc) {
    c->last_error = "cuTensorMapEncodeTiled unavailable";
    return FMM_ERR_CUDA;
  }
  cuuint64_t dims[2] = {(cuuint64_t)op.Kpad, (cuuint64_t)op.Npad};
  cuuint64_t strides[1] = {(cuuint64_t)op.Kpad * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)op.BN};
  cuuint32_t es[2] = {1, 1};
  for (int w = 0; w < 2; ++w) {
    void* g = w == 0 ? op.hi.ptr : op.lo.ptr;
    CUtensorMap* tm = (CUtensorMap*)(w == 0 ? op.tmap_hi : op.tmap_lo);
    CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, g, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      c->last_error = "cuTensorMapEncodeTiled failed: " + std::to_string((int)r);
      return FMM_ERR_CUDA;
    }
  }
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(256));
    attr_done = true;
  }
  return FMM_OK;
}

void launch_gemm_tc(Ctx* c, const GemmOperand& op, int mode, const int* levels, int nlev, cudaStream_t st,
                    const int32_t* const* rows, const int64_t* nrows) {
  TcParams P;
  int tiles = 0;
  P.nseg = 0;
  for (int i = 0; i < nlev && P.nseg < kMaxSeg; ++i) {
    const int lr = levels[i];  // row level
    LevelTree& R = c->lev[lr];
    // M2P: octs with a refined cell (their children hold the targets);
    // M2L: octs with a cell that has grandchildren (those need a local expansion)
    const int64_t nr = (rows && rows[i]) ? nrows[i] : ((mode == kModeM2P) ? R.n_rows : R.n_rowsL);
    if (!nr) continue;
    TcSeg& S = P.seg[P.nseg++];
    S.Ahi = (const __nv_bfloat16*)R.Mhi.ptr;
    S.Alo = (const __nv_bfloat16*)R.Mlo.ptr;
    S.rows = (rows && rows[i]) ? rows[i] : (const int32_t*)((mode == kModeM2P) ? R.rows.ptr : R.rowsL.ptr);
    S.cell_child_tgt = (mode == kModeM2P) ? (const int32_t*)c->lev[lr + 1].cell_child.ptr : nullptr;
    S.slot = (const int32_t*)R.slotL.ptr;
    S.nbr = (const int32_t*)R.nbr.ptr;
    S.cell_child_rows = (const int32_t*)R.cell_child.ptr;
    S.out = (mode == kModeM2P) ? (float*)c->lev[lr + 1].acc.ptr : (float*)R.Lm.ptr;
    S.nrows = (int)nr;
    S.tile0 = tiles;
    tiles += (int)((nr + BM - 1) / BM);
  }
  if (!tiles) return;
  P.KQ = op.kseg;
  P.Kvalid = op.K;
  P.nchunks = op.Kpad / BK;
  const int tuned = c->tune_split[mode == kModeM2P ? 0 : 1];
  const int split = tuned > 0 ? std::min(tuned, P.nchunks) : choose_split(tiles * op.ntile, P.nchunks, c->num_sms);
  P.chunks_per_split = (P.nchunks + split - 1) / split;
  const int nz = (P.nchunks + P.chunks_per_split - 1) / P.chunks_per_split;
  P.BN = op.BN;
  P.N = op.N;
  P.nc = c->tab.nc;
  P.mode = mode;
  P.err = c->d_err;
  dim3 grid((unsigned)tiles, (unsigned)op.ntile, (unsigned)nz);
  ++c->n_launch;
  launch_pdl(k_gemm_tc, grid, THREADS, smem_bytes(op.BN), st, *(const CUtensorMap*)op.tmap_hi,
             *(const CUtensorMap*)op.tmap_lo, P);
}

}  // namespace fmm
