// gemm_tc.cu -- M2L (Eq. 3) and bottom M2P (Fig. 2, Alg. 4) on the 5th
// generation tensor cores (tcgen05) in split-BF16 with FP32 accumulation.
//
// D[row][n] = sum_k A[row][k] B[n][k] where a row is an oct of the source
// grid, k = (q, s, alpha) runs over the 26 neighbour octs of its parent, their
// 8 cells and the multipole coefficients, and B is the translation operator
// (translation invariant, so one table serves every oct and every level).
// The Delta l = 2 variant (footnote of Sec. 2) adds two modes: M2P from the
// level l-2 grid (2048 columns: the 512 level-l cells under a row oct, found
// through two child links) and the near-field ring, whose "coefficients" are
// the 8 child masses of each source cell (exact P2P as a contraction).
// Each operand is split x = hi + lo with hi, lo in BF16; the product keeps
// hi*hi + hi*lo + lo*hi (the lo*lo term is below FP32 rounding).  In TF32
// precision each operand is one FP32 value rounded to TF32 and each product is
// one kind::tf32 MMA (K = 8): the A stage then holds 32 FP32 values per row
// (32 TMEM columns, as hi + lo do) and the B stage one 128-byte-swizzled tile
// of BN rows x 32 FP32 (the bytes of the hi and lo tiles together).
//
// Per CTA: 128 rows x BN columns.  Tensor memory (TMEM, 512 columns) holds the
// FP32 accumulator (columns 0..255) and SA stages of the A operand (columns
// 256..511, 32 per stage: the hi and lo halves of a BK-wide slice of every
// row, two bf16 per column); the MMA reads A from TMEM and B from shared memory.
//   warps 0-15   producers: the rows are neighbour octs (no TMA tile fetches
//                them), so thread t of warp w loads row 32 (w % 4) + t, i.e.
//                its own TMEM lane, with vector loads and tcgen05.st; the four
//                warps of a lane quarter take every fourth stage, so four
//                stages of loads are in flight per quarter.  Warps 0-3 then
//                run the epilogue (tcgen05.ld, scatter-add to the targets).
//   warp 16      allocates TMEM and loads B tiles with TMA (SWIZZLE_64B)
//   warp 17      one thread issues tcgen05.mma (M=128, N=BN, K=16) per slice
// K is visited slice-major: one BK-wide slice of all 26 offsets, then the
// next (each offset segment is padded to whole slices).  A tile's rows then
// re-read the row slices of the same few hundred neighbour octs across the 26
// offsets, and the shared memory left unused (4 B stages) keeps them in L1.
// Within a segment K runs (alpha, cell), so the coefficients of low degree come
// first; an N tile stops after the slices its columns keep (M2L: |alpha| <=
// p - min |beta| of the tile).  Split-K: grid.y enumerates (N tile, K part)
// pairs from a table, so tiles with few slices get no idle CTAs; partial sums
// are added with atomics.  Every wait on an
// mbarrier is bounded by a wall-clock limit (a launch parameter); on expiry the
// CTA latches kErrTimeout and skips the remaining work, but before it frees its
// TMEM and exits it waits (with a fixed limit of its own) for the TMA loads and
// the MMAs it has already issued: those still write shared and tensor memory.
#include <algorithm>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "fmm_internal.cuh"

namespace fmm {
namespace {

constexpr int BM = 128;
constexpr int BK = kTcBK;  // bf16 elements per row per stage = 64 bytes (64-byte swizzle for B)
constexpr int SB = 4;   // B stages (shared memory; the rest of the SM's 256 KB serves as L1 for the rows)
constexpr int SA = 8;   // A stages (TMEM, 32 columns each)
constexpr int kPhases = 4;                    // producer warps per TMEM lane quarter
constexpr int kProducerWarps = 4 * kPhases;
constexpr int kWarpTma = kProducerWarps;      // also allocates TMEM
constexpr int kWarpMma = kProducerWarps + 1;
constexpr int THREADS = 32 * (kProducerWarps + 2);
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kAcol0 = 256;              // first A column
constexpr int kNbrStride = 27;  // shared-memory row stride of the per-row neighbour table
constexpr int kMaxSeg = 24;
constexpr int kMaxYZ = 64;  // (N tile, K part) pairs of one launch
constexpr uint64_t kDrainLimitNs = 1000000000ull;  // 1 s: waits for a CTA's own copies and MMAs in flight

__constant__ int c_nbr26[26] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12,
                                14, 15, 16, 17, 18, 19, 20, 21, 22, 23, 24, 25, 26};

// One segment = the rows of one level: its sources, neighbour table and output.
struct TcSeg {
  const __nv_bfloat16* Ahi;
  const __nv_bfloat16* Alo;
  const int32_t* rows;
  const int32_t* nbr;
  const int32_t* cell_child_rows;  // M2P: cell_child of the row level
  const int32_t* cell_child_mid;   // M2P2: cell_child of the level between rows and targets
  const int32_t* cell_child_tgt;   // M2P: cell_child of the target level (refined targets get nothing)
  const uint8_t* leafmask_tgt;     // M2P: leaf masks of the target level (or null: use cell_child_tgt)
  const int32_t* slot;             // M2L: local-expansion slot of each row oct
  float* out;                      // M2P: [cells of target level][4]; M2L: [slot*8 + cell][nc]
  int nrows;
  int tile0;                       // first M tile of this segment
};

struct TcParams {
  TcSeg seg[kMaxSeg];
  int nseg;
  int KQ;          // operand row length per neighbour offset (8 * nc)
  int KQP;         // K per neighbour offset in the operator: KQ padded to whole slices
  int chunks_per_split;
  int v8;          // rows load in 32-byte pieces (KQ % 16 == 0 and 32-byte aligned sources)
  int nyz;                  // (N tile, K part) pairs on grid.y
  uint16_t yz_tile[kMaxYZ];  // N tile of pair j
  uint16_t yz_part[kMaxYZ];  // K part of pair j
  uint16_t tile_chunks[kMaxYZ];  // slices the tile visits: 26 x the slices per segment it keeps
  int BN, N, nc, mode;
  unsigned* err;
  uint64_t wait_ns;  // limit of every pipeline wait
  int tf32;          // 1: FP32 operands (Ahi as float), kind::tf32; 0: split-BF16, kind::f16
};

// First K index of the it-th slice a CTA visits.  Slice-major order (slice c of
// every neighbour offset q before slice c + 1) keeps the rows one slice needs,
// about the distinct neighbour octs of the tile, in L1 across the 26 offsets.
__device__ __forceinline__ int slice_k0(int KQP, int it) {
  const int c = it / 26, q = it - 26 * c;
  return q * KQP + c * BK;
}

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
// within limit_ns or another thread already aborted.
// A try_wait may itself suspend the thread for a while, so the clock is read
// on the first retry too, not only every 1024 retries.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort, uint64_t limit_ns) {
  if (mbar_try(bar, parity)) return true;
  uint64_t t0 = now_ns();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try(bar, parity)) return true;
    if ((i & 1023) == 0 || i == 1) {
      if (*abort) return false;
      if (now_ns() - t0 > limit_ns) {
        *abort = 1;
        return false;
      }
    }
  }
}
// Wait for work this CTA itself issued (a TMA load, a tcgen05.commit) to land
// before it leaves; that work completes by itself, so only a fixed limit
// guards it, and the abort flag is ignored.
__device__ __forceinline__ bool mbar_drain(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = now_ns();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try(bar, parity)) return true;
    if ((i & 1023) == 0 && now_ns() - t0 > kDrainLimitNs) return false;
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

// K-major FP32 tile, rows of BK fp32 (128 B), 128-byte swizzle: 8 rows form a 1024 B atom.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);  // start address
  d |= (uint64_t)1 << 16;                  // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                  // descriptor version for tcgen05
  d |= (uint64_t)2 << 61;                  // 128-byte swizzle
  return d;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* tm, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"((uint64_t)tm), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// D (TMEM) += A (TMEM: 128 lanes x 8 columns = 16 bf16 per row) * B (shared memory)
__device__ __forceinline__ void mma_bf16_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t b, uint32_t idesc,
                                            uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "r"(tmem_a), "l"(b), "r"(idesc), "r"(accum));
}

// D (TMEM) += A (TMEM: 128 lanes x 8 columns = 8 tf32 per row) * B (shared memory)
__device__ __forceinline__ void mma_tf32_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t b, uint32_t idesc,
                                            uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "r"(tmem_a), "l"(b), "r"(idesc), "r"(accum));
}

// 16 consecutive columns of this warp's 32 TMEM lanes, one register per lane and column
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
      : "memory");
}

__device__ __forceinline__ void ld_nc_v4(const void* p, uint32_t& a, uint32_t& b, uint32_t& c, uint32_t& d) {
  asm volatile("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(a), "=r"(b), "=r"(c), "=r"(d) : "l"(p));
}
// 32 bytes (one sector) per thread; p must be 32-byte aligned
__device__ __forceinline__ void ld_nc_v8(const void* p, uint32_t* v) {
  asm volatile("ld.global.nc.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "l"(p));
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
  const int b_bytes = P.BN * BK * 2;  // BN * 64
  unsigned char* Bhi = sm;
  unsigned char* Blo = Bhi + SB * b_bytes;
  // fullA[SA], emptyA[SA], fullB[SB], emptyB[SB], done, drain (the MMA issuer's last commit)
  uint64_t* bars = (uint64_t*)(Blo + SB * b_bytes);
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * SA + 2 * SB + 2);
  volatile int* abort = (volatile int*)(tmem_slot + 1);
  int32_t* s_nbr = (int32_t*)(tmem_slot + 4);  // [BM][kNbrStride] source octs of each row

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ytile = P.yz_tile[blockIdx.y];  // N tile
  const int kc_begin = P.yz_part[blockIdx.y] * P.chunks_per_split;
  const int kc_end = min((int)P.tile_chunks[blockIdx.y], kc_begin + P.chunks_per_split);
  const int nit = max(0, kc_end - kc_begin);
  const uint32_t fullA0 = smem_u32(bars), emptyA0 = smem_u32(bars + SA);
  const uint32_t fullB0 = smem_u32(bars + 2 * SA), emptyB0 = smem_u32(bars + 2 * SA + SB);
  const uint32_t done = smem_u32(bars + 2 * SA + 2 * SB);
  const uint32_t drain = smem_u32(bars + 2 * SA + 2 * SB + 1);

  if (threadIdx.x == 0) {
    for (int s = 0; s < SA; ++s) {
      mbar_init(fullA0 + 8 * s, 128);  // the 32 x 4 producer threads of the stage
      mbar_init(emptyA0 + 8 * s, 1);   // tcgen05.commit
    }
    for (int s = 0; s < SB; ++s) {
      mbar_init(fullB0 + 8 * s, 1);    // TMA arrive + transaction bytes
      mbar_init(emptyB0 + 8 * s, 1);   // tcgen05.commit
    }
    mbar_init(done, 1);
    mbar_init(drain, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kWarpTma) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  // Programmatic dependent launch: the row lists and neighbour tables (tree
  // build) and the operator (built at creation) are read before the wait on
  // the previous kernel; only the multipole rows it produces, and the outputs,
  // come after it (the producer warps, which also run the epilogue, wait).
  if (warp < kProducerWarps) {
    // ---------------- A rows into TMEM ----------------
    const int q = warp & 3;             // lane quarter: rows 32 q .. 32 q + 31
    const int t = 32 * q + lane;        // this thread's row (TMEM lane)
    int si = 0;
    while (si + 1 < P.nseg && (int)blockIdx.x >= P.seg[si + 1].tile0) ++si;
    const TcSeg& S = P.seg[si];
    const int64_t row_idx = (int64_t)(blockIdx.x - S.tile0) * BM + t;
    const bool valid = row_idx < S.nrows;
    const int32_t roct = valid ? S.rows[row_idx] : 0;
    if (warp < 4) {
      int32_t* myn = s_nbr + t * kNbrStride;
      for (int qq = 0; qq < 26; ++qq) myn[qq] = valid ? S.nbr[(int64_t)roct * 27 + c_nbr26[qq]] : -1;
    }
    asm volatile("bar.sync 1, %0;" ::"n"(32 * kProducerWarps) : "memory");  // tables of all rows written
    pdl_wait();  // the multipole rows come from the previous kernel
    pdl_trigger();
    const uint32_t myn_s = smem_u32(s_nbr + t * kNbrStride);  // read back with ld.shared
    const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);   // this warp's lanes, column 0
    bool ok = true;
    for (int it = warp >> 2; it < nit && ok; it += kPhases) {
      const int s = it % SA;
      if (it >= SA) ok = mbar_wait(emptyA0 + 8 * s, ((it / SA) - 1) & 1, abort, P.wait_ns);
      if (!ok) break;
      const int k0 = slice_k0(P.KQP, kc_begin + it);
      uint32_t hv[16], lv[16];
      if (P.tf32) {
        // 32 FP32 per row: columns 0..15 take k0..k0+15, columns 16..31 take k0+16..k0+31
        const float* A = reinterpret_cast<const float*>(S.Ahi);
#pragma unroll
        for (int j = 0; j < BK / 8; ++j) {  // 8 fp32 (32 bytes) never straddle an offset segment (KQ % 8 == 0)
          const int k = k0 + 8 * j;
          uint32_t* dst = j < 2 ? hv + 8 * j : lv + 8 * (j - 2);
          int32_t src = -1;
          int off = 0;
          {  // the padding at the end of a segment reads as zeros
            const int qi = k / P.KQP;
            off = k - qi * P.KQP;
            if (off < P.KQ) asm volatile("ld.shared.b32 %0, [%1];" : "=r"(src) : "r"(myn_s + 4 * qi));
          }
          if (src >= 0) {
            ld_nc_v8(A + (int64_t)src * P.KQ + off, dst);
          } else {
#pragma unroll
            for (int u = 0; u < 8; ++u) dst[u] = 0u;
          }
        }
      } else if (P.v8) {
#pragma unroll
        for (int j = 0; j < BK / 16; ++j) {  // 16 bf16 (32 bytes) never straddle an offset segment (KQ % 16 == 0)
          const int k = k0 + 16 * j;
          int32_t src = -1;
          int off = 0;
          {  // the padding at the end of a segment reads as zeros
            const int qi = k / P.KQP;
            off = k - qi * P.KQP;
            if (off < P.KQ) asm volatile("ld.shared.b32 %0, [%1];" : "=r"(src) : "r"(myn_s + 4 * qi));
          }
          if (src >= 0) {
            ld_nc_v8(S.Ahi + (int64_t)src * P.KQ + off, hv + 8 * j);
            ld_nc_v8(S.Alo + (int64_t)src * P.KQ + off, lv + 8 * j);
          } else {
#pragma unroll
            for (int u = 0; u < 8; ++u) hv[8 * j + u] = lv[8 * j + u] = 0u;
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < BK / 8; ++j) {  // 8 bf16 (16 bytes) never straddle an offset segment (KQ % 8 == 0)
          const int k = k0 + 8 * j;
          int32_t src = -1;
          int off = 0;
          {  // the padding at the end of a segment reads as zeros
            const int qi = k / P.KQP;
            off = k - qi * P.KQP;
            if (off < P.KQ) asm volatile("ld.shared.b32 %0, [%1];" : "=r"(src) : "r"(myn_s + 4 * qi));
          }
          if (src >= 0) {
            ld_nc_v4(S.Ahi + (int64_t)src * P.KQ + off, hv[4 * j], hv[4 * j + 1], hv[4 * j + 2], hv[4 * j + 3]);
            ld_nc_v4(S.Alo + (int64_t)src * P.KQ + off, lv[4 * j], lv[4 * j + 1], lv[4 * j + 2], lv[4 * j + 3]);
          } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) hv[4 * j + u] = lv[4 * j + u] = 0u;
          }
        }
      }
      const uint32_t col = kAcol0 + 32u * (uint32_t)s;
      tmem_st16(tl + col, hv);
      tmem_st16(tl + col + 16, lv);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(fullA0 + 8 * s);
    }

    if (warp < 4) {
      // ---------------- epilogue ----------------
      // Everything the scatter needs is loaded before the accumulator is ready:
      // M2P: the child oct under each of the row's cells and which of its cells
      // are leaves (targets); M2L: the row's local-expansion slot.
      const int nchunk = P.BN / 32;
      int32_t ch[8];
      uint32_t tmask[8];
      int64_t slot = 0;
      if (P.mode == kModeM2P2) {
        // 32 columns = the 8 targets of one level-l oct: cell f & 7 of the child
        // oct of cell f >> 3 of the row oct
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          ch[j] = -1;
          const int f = (ytile * P.BN + j * 32) >> 5;
          if (valid && j < nchunk && f < 64) {
            const int32_t mid = S.cell_child_rows[(int64_t)roct * 8 + (f >> 3)];
            if (mid >= 0) ch[j] = S.cell_child_mid[(int64_t)mid * 8 + (f & 7)];
          }
        }
      } else if (P.mode != kModeM2L) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          ch[j] = -1;
          const int f = (ytile * P.BN + j * 32) >> 5;
          if (valid && j < nchunk && f < 8) ch[j] = S.cell_child_rows[(int64_t)roct * 8 + f];
        }
      }
      if (P.mode != kModeM2L) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          tmask[j] = 0;
          if (ch[j] >= 0) {
            if (S.leafmask_tgt) {
              tmask[j] = S.leafmask_tgt[ch[j]];
            } else {
              for (int u = 0; u < 8; ++u) tmask[j] |= (uint32_t)(S.cell_child_tgt[(int64_t)ch[j] * 8 + u] < 0) << u;
            }
          }
        }
      } else if (valid) {
        slot = S.slot[roct];
      }
      bool have = ok && nit > 0 && mbar_wait(done, 0, abort, P.wait_ns);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (j >= nchunk) break;
        uint32_t v[32];
        const uint32_t taddr = tl + (uint32_t)(j * 32);
        TMEM_LD32(taddr, v);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (!have || !valid) continue;
        const int n0 = ytile * P.BN + j * 32;
        if (P.mode != kModeM2L) {
          if (ch[j] >= 0) {
            float* dst = S.out + (int64_t)ch[j] * 32;
#pragma unroll
            for (int u = 0; u < 8; ++u)
              if ((tmask[j] >> u) & 1)  // leaf targets only: the accumulator of refined cells stays zero
                asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst + 4 * u),
                             "f"(__uint_as_float(v[4 * u])), "f"(__uint_as_float(v[4 * u + 1])),
                             "f"(__uint_as_float(v[4 * u + 2])), "f"(__uint_as_float(v[4 * u + 3]))
                             : "memory");
          }
        } else {
          float* dst = S.out + slot * 8 * P.nc + n0;
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (n0 + 4 * u < P.N)
              asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst + 4 * u),
                           "f"(__uint_as_float(v[4 * u])), "f"(__uint_as_float(v[4 * u + 1])),
                           "f"(__uint_as_float(v[4 * u + 2])), "f"(__uint_as_float(v[4 * u + 3]))
                           : "memory");
        }
      }
    }
  } else if (warp == kWarpTma) {
    // ---------------- B tiles by TMA (the operator: no wait) ----------------
    pdl_trigger();
    if (lane == 0) {
      bool ok = true;
      int issued = 0;
      for (int it = 0; it < nit && ok; ++it) {
        const int s = it % SB;
        if (it >= SB) ok = mbar_wait(emptyB0 + 8 * s, ((it / SB) - 1) & 1, abort, P.wait_ns);
        if (!ok) break;
        const int k0 = slice_k0(P.KQP, kc_begin + it);
        const int n0 = ytile * P.BN;
        mbar_arrive_tx(fullB0 + 8 * s, 2u * (uint32_t)b_bytes);
        if (P.tf32) {  // one FP32 tile per stage, laid over the hi and lo regions
          tma_load_2d(smem_u32(Bhi + s * 2 * b_bytes), &tm_hi, k0, n0, fullB0 + 8 * s);
        } else {
          tma_load_2d(smem_u32(Bhi + s * b_bytes), &tm_hi, k0, n0, fullB0 + 8 * s);
          tma_load_2d(smem_u32(Blo + s * b_bytes), &tm_lo, k0, n0, fullB0 + 8 * s);
        }
        ++issued;
      }
      // Loads older than the last SB were consumed by the MMA (it waited for them
      // before freeing their stage); the last SB may still be landing.
      for (int it = max(0, issued - SB); it < issued; ++it)
        if (!mbar_drain(fullB0 + 8 * (it % SB), (it / SB) & 1)) *abort = 1;
    }
    __syncwarp();
  } else if (warp == kWarpMma) {
    // ---------------- MMA issue (shared and tensor memory only) ----------------
    pdl_trigger();
    if (lane == 0) {
      // kind::f16, D = F32, A = B = BF16 (format 1), or kind::tf32, A = B = TF32 (format 2);
      // both K-major, M = 128, N = BN
      const uint32_t fmt = P.tf32 ? 2u : 1u;
      const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(P.BN >> 3) << 17) |
                             ((uint32_t)(BM >> 4) << 24);
      bool ok = true;
      int issued = 0;
      for (int it = 0; it < nit && ok; ++it) {
        const int sa = it % SA, sb = it % SB;
        ok = mbar_wait(fullA0 + 8 * sa, (it / SA) & 1, abort, P.wait_ns) &&
             mbar_wait(fullB0 + 8 * sb, (it / SB) & 1, abort, P.wait_ns);
        if (!ok) break;
        ++issued;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acol = tmem + kAcol0 + 32u * (uint32_t)sa;  // hi at +0, lo at +16
        if (P.tf32) {
          const uint32_t b = smem_u32(Bhi + sb * 2 * b_bytes);
#pragma unroll
          for (int kk = 0; kk < BK / 8; ++kk)  // K = 8 per MMA: 8 TMEM columns, 32 bytes of each B row
            mma_tf32_ta(tmem, acol + 8 * kk, sdesc_sw128(b + kk * 32), idesc, (it | kk) != 0);
        } else {
          const uint32_t bh = smem_u32(Bhi + sb * b_bytes), bl = smem_u32(Blo + sb * b_bytes);
#pragma unroll
          for (int part = 0; part < 3; ++part) {
            const uint32_t a = (part == 2) ? acol + 16 : acol;
            const uint32_t b = (part == 1) ? bl : bh;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
              const uint32_t accum = (it | part | kk) != 0;
              mma_bf16_ta(tmem, a + 8 * kk, sdesc_sw64(b + kk * 32), idesc, accum);
            }
          }
        }
        mma_commit(emptyA0 + 8 * sa);
        mma_commit(emptyB0 + 8 * sb);
      }
      if (ok && nit > 0) mma_commit(done);
      // Every MMA issued must finish before the tensor memory is freed, also when
      // a wait gave up (the epilogue then does not wait for `done`).
      if (issued > 0) {
        mma_commit(drain);
        if (!mbar_drain(drain, 0)) *abort = 1;
      }
    }
    __syncwarp();
  }
  if (*abort && threadIdx.x == 0) atomicOr(P.err, kErrTimeout);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == kWarpTma) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
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
  return 1024 + SB * (2 * BN * BK * 2) + (2 * SA + 2 * SB + 2) * 8 + 16 + BM * kNbrStride * 4;
}

// Split-K: chunks per CTA minimising waves x chunks per CTA, for M tiles that
// each run every N tile y over its own tile_chunks[y] slices.  `split` > 0
// (the autotuner's choice) splits the longest tile in that many parts instead.
int choose_chunks_per_split(int mtiles, const std::vector<int>& chunks, int nsm, int split) {
  const int cmax = *std::max_element(chunks.begin(), chunks.end());
  auto pairs = [&](int cps) {
    int n = 0;
    for (int ch : chunks) n += (ch + cps - 1) / cps;
    return n;
  };
  if (split > 0) {
    int cps = (cmax + split - 1) / split;
    while (pairs(cps) > kMaxYZ) ++cps;
    return cps;
  }
  int best = cmax;
  double best_t = 1e30;
  for (int s = 1; s <= 32 && s <= cmax; ++s) {
    const int cps = (cmax + s - 1) / s;
    const int np = pairs(cps);
    if (np > kMaxYZ) break;
    const int waves = (mtiles * np + nsm - 1) / nsm;
    const double t = (double)waves * (cps + 2);  // +2: pipeline fill and epilogue
    if (t < best_t - 1e-9) {
      best_t = t;
      best = cps;
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
  // split-BF16: two maps of bf16 [Npad][Kpad], 64-byte swizzle (BK bf16 = 64 B per row);
  // TF32: one map of fp32 [Npad][Kpad], 128-byte swizzle (BK fp32 = 128 B per row)
  const bool tf32 = c->cfg.precision == FMM_MIXED_TF32;
  cuuint64_t dims[2] = {(cuuint64_t)op.Kpad, (cuuint64_t)op.Npad};
  cuuint64_t strides[1] = {(cuuint64_t)op.Kpad * (tf32 ? 4 : 2)};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)op.BN};
  cuuint32_t es[2] = {1, 1};
  for (int w = 0; w < 2; ++w) {
    void* g = (w == 0 || tf32) ? op.hi.ptr : op.lo.ptr;
    CUtensorMap* tm = (CUtensorMap*)(w == 0 ? op.tmap_hi : op.tmap_lo);
    CUresult r = enc(tm, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, g, dims,
                     strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     tf32 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
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
                    const int32_t* const* rows, const int64_t* nrows, int sm_budget) {
  TcParams P;
  int tiles = 0;
  P.nseg = 0;
  P.v8 = op.kseg % 16 == 0;
  for (int i = 0; i < nlev && P.nseg < kMaxSeg; ++i) {
    const int lr = levels[i];  // row level
    LevelTree& R = c->lev[lr];
    // M2P (and the ring P2P, Delta l = 2's M2P): octs with a refined cell (their
    // descendants hold the targets); M2L: octs with a cell that has grandchildren
    // (those need a local expansion)
    const bool m2l = mode == kModeM2L;
    const int lt = lr + (mode == kModeM2P2 ? 2 : 1);  // target level of the bottom modes
    const int64_t nr = (rows && rows[i]) ? nrows[i] : (m2l ? R.n_rowsL : R.n_rows);
    if (!nr) continue;
    TcSeg& S = P.seg[P.nseg++];
    S.Ahi = (const __nv_bfloat16*)(mode == kModeP2PR ? R.Chi.ptr : R.Mhi.ptr);
    S.Alo = (const __nv_bfloat16*)(mode == kModeP2PR ? R.Clo.ptr : R.Mlo.ptr);
    S.rows = (rows && rows[i]) ? rows[i] : (const int32_t*)(m2l ? R.rowsL.ptr : R.rows.ptr);
    S.cell_child_tgt = m2l ? nullptr : (const int32_t*)c->lev[lt].cell_child.ptr;
    S.leafmask_tgt = m2l ? nullptr : (const uint8_t*)c->lev[lt].leafmask.ptr;
    S.cell_child_mid = mode == kModeM2P2 ? (const int32_t*)c->lev[lr + 1].cell_child.ptr : nullptr;
    S.slot = (const int32_t*)R.slotL.ptr;
    S.nbr = (const int32_t*)R.nbr.ptr;
    S.cell_child_rows = (const int32_t*)R.cell_child.ptr;
    S.out = m2l ? (float*)R.Lm.ptr : (float*)c->lev[lt].acc.ptr;
    S.nrows = (int)nr;
    S.tile0 = tiles;
    if ((uintptr_t)S.Ahi % 32 || (uintptr_t)S.Alo % 32) P.v8 = 0;
    tiles += (int)((nr + BM - 1) / BM);
  }
  if (!tiles) return;
  P.KQ = op.kseg;
  P.KQP = op.kqp;
  std::vector<int> chunks(op.ntile);
  for (int y = 0; y < op.ntile; ++y) chunks[y] = 26 * op.tile_slices[y];
  const int tuned = c->tune_split[mode == kModeM2L ? 1 : 0];
  P.chunks_per_split = choose_chunks_per_split(tiles, chunks, sm_budget > 0 ? sm_budget : c->num_sms, tuned);
  P.nyz = 0;
  for (int y = 0; y < op.ntile; ++y)
    for (int z = 0; z * P.chunks_per_split < chunks[y]; ++z) {
      P.yz_tile[P.nyz] = (uint16_t)y;
      P.yz_part[P.nyz] = (uint16_t)z;
      P.tile_chunks[P.nyz] = (uint16_t)chunks[y];
      ++P.nyz;
    }
  P.BN = op.BN;
  P.N = op.N;
  P.nc = c->tab.nc;
  P.mode = mode;
  P.err = c->d_err;
  P.wait_ns = (uint64_t)(c->wait_s * 1e9);
  P.tf32 = c->cfg.precision == FMM_MIXED_TF32;
  dim3 grid((unsigned)tiles, (unsigned)P.nyz, 1u);
  ++c->n_launch;
  launch_pdl(k_gemm_tc, grid, THREADS, smem_bytes(op.BN), st, *(const CUtensorMap*)op.tmap_hi,
             *(const CUtensorMap*)op.tmap_lo, P);
}

}  // namespace fmm
