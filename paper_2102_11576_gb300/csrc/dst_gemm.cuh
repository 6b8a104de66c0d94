// dst_gemm.cuh -- the sine transform as a tensor-core GEMM in split BF16.
//
// D = A * S with S = S_n (Section 4.1) symmetric, so both operands are
// K-major rows: D[m][n] = sum_k A[m][k] S[n][k].  NT = 3 (split BF16): every
// operand X is held as a pair of BF16 matrices X = X_hi + X_lo
// (X_lo = bf16(X - X_hi)), and the product is accumulated in FP32 tensor
// memory as
//     A_hi S_hi + A_hi S_lo + A_lo S_hi
// (the split-BF16 product of Henry, Tang & Heinecke, 2019: about 16
// significant bits per operand, the A_lo S_lo term dropped).  NT = 1 (plain
// BF16): only A_hi S_hi, about 8 significant bits per operand.
//
// One CTA computes a 128 x 128 tile of D: a TMA producer thread streams
// 64-wide K slices of the operand tiles (four for NT = 3, two for NT = 1)
// through a 3-stage shared-memory ring (128-byte swizzle), one MMA thread
// issues tcgen05.mma (M=128, N=128, K=16) into a TMEM accumulator, and all
// four warps run the epilogue from TMEM.  NT = 1 needs 97 KB of shared
// memory, so two CTAs share an SM and one's epilogue overlaps the other's
// MMAs.  The epilogue always stores D transposed: TMEM lanes are rows m, so a
// warp's 32 lanes write 32 consecutive addresses of a row of D^T.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"
#include "umma.cuh"

namespace rsfde {

constexpr int kGemmBM = 128, kGemmBK = 64;
// Ring depth: as many stages as fit beside a second CTA on the SM (the TMA
// round trip, not bandwidth, bounds these short-K GEMMs).
__host__ __device__ constexpr int gemm_stages(int NT, int BN) { return (NT == 1 && BN == 64) ? 4 : 3; }
constexpr int kGemmATileBytes = kGemmBM * kGemmBK * 2;  // 16 KB
// B tile: BN rows (64 or 128) of 64 BF16
__host__ __device__ constexpr int gemm_btile_bytes(int BN) { return BN * kGemmBK * 2; }
// per stage: A_hi, A_lo, B_hi, B_lo (NT = 3) or A_hi, B_hi (NT = 1)
__host__ __device__ constexpr int gemm_stage_bytes(int NT, int BN) {
  return (NT == 3 ? 2 : 1) * (kGemmATileBytes + gemm_btile_bytes(BN));
}
__host__ __device__ constexpr int gemm_smem(int NT, int BN) {
  return gemm_stages(NT, BN) * gemm_stage_bytes(NT, BN) + 1024;  // + alignment slack
}
// CTAs that share an SM: shared memory (and TMEM: at most 2 x 256 columns)
__host__ __device__ constexpr int gemm_ctas_per_sm(int NT, int BN) { return NT == 3 ? 1 : 2; }

enum GemmEpi {
  EPI_SPLIT_T = 0,   // out^T (BF16, or split BF16 pair); rows m >= row_b go to the second channel's columns
  EPI_DIVIDE_T = 1,  // two tau divides (Eq. 4.6), both channels out^T
  EPI_COMBINE_T = 2  // masked combine of Eq. 4.6 into z (channel = blockIdx.z)
};

// Symmetric form (SYM): for even n the sine matrix satisfies
//     S[n-1-i][j] = (-1)^j S[i][j]        (0-based i, j),
// so with u_i = sum over even j and e_i = sum over odd j of S[i][j] x_j the
// two outputs i and n-1-i are u_i + e_i and u_i - e_i (i < n/2).  The K
// operand then holds the even-j entries in columns [0, hk) and the odd-j
// entries in [hk, 2 hk) (hk = n/2 rounded up to 64, zero padded), the GEMM
// has n/2 output columns and two TMEM accumulators, and half the MMAs.
__host__ __device__ __forceinline__ int sym_perm(int x, int hk) { return hk ? (x & 1) * hk + (x >> 1) : x; }

struct GemmEpiParams {
  int M, N;       // valid extent of D (N: n/2 in the symmetric form)
  int n_full;     // symmetric form: the transform length n (outputs i and n-1-i); 0 otherwise
  int hk;         // K layout the epilogue writes for the next GEMM: 0 natural, else symmetric halves of hk
  __nv_bfloat16* out_hi;
  __nv_bfloat16* out_lo;
  int ldo;
  int row_b, col_b;     // EPI_SPLIT_T: rows m >= row_b are channel 2, written from column col_b on
  const float* lam_m;   // EPI_DIVIDE_T: tau eigenvalues along D rows (x) and columns (y)
  const float* lam_n;
  float pen;            // dt / eta
  int chb_rows;         // EPI_DIVIDE_T: row offset of channel b in out
  void* z;              // EPI_COMBINE_T: output vector (n2 x n1, x fastest)
  int z_double;
  const uint32_t* phibits;  // EPI_COMBINE_T: Phi transposed and bit-packed, bit y%32 of word
  int wpc;                  //   [x * wpc + y/32] is 1 where (x, y) lies outside Omega
  int ldz;
  const double* zscale;  // EPI_COMBINE_T: if set, z is scaled by *zscale (unscaled first operand)
  int a_koff;           // K offset of channel 1's A operand (EPI_COMBINE_T, blockIdx.z = 1)
  int nch;              // channels (grid z of the one-tile-per-CTA launch)
  long long wait_cycles;  // bound of each pipeline wait (ring slots, accumulator) in SM clock cycles
};

template <int NT>
__device__ __forceinline__ void split_store(__nv_bfloat16* hi, __nv_bfloat16* lo, size_t idx, float v) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  hi[idx] = h;
  if (NT == 3) lo[idx] = __float2bfloat16_rn(v - __bfloat162float(h));
}

// Threads of a CTA: warp 0 lane 0 issues the TMA loads, warp 1 lane 0 the MMAs,
// and every warp runs the epilogue once its role is done (the warps of a TMEM
// lane quarter take alternate 32-column chunks), which is latency-bound: split
// BF16 (one CTA per SM) runs sixteen warps, four per quarter; plain BF16 (two
// CTAs per SM) eight.  With two tiles per CTA (TPC = 2, split BF16 only) the
// second tile's K slices stream into a second pair of TMEM accumulators while
// warps 2..15 run the first tile's epilogue, so the tensor pipe does not wait
// for it; all sixteen run the last one.
__host__ __device__ constexpr int gemm_threads(int NT) { return NT == 3 ? 512 : 256; }
//
// The CTA's work: ntile tiles (at most TPC) of the linear tile order (x
// fastest, then y, then channel), tiles t0 and t0 + tstride; GRID: the one
// tile (blockIdx.x, blockIdx.y, blockIdx.z).  The tensor maps
// may sit in the kernel's parameters or in global memory; the epilogue
// parameters come by value (a kernel parameter, read from the constant bank)
// or by reference (EPT = const GemmEpiParams&, a copy in shared memory).
// THR threads and STG ring stages (defaults: gemm_threads, gemm_stages).
template <int EPI, int NT, bool SYM, int BN, int TPC, bool GRID, typename EPT, int THR = gemm_threads(NT),
          int STG = gemm_stages(NT, BN)>
__device__ __forceinline__ void dst_gemm_body(const CUtensorMap* tA_hi, const CUtensorMap* tA_lo,
                                              const CUtensorMap* tB_hi, const CUtensorMap* tB_lo, int K, EPT ep,
                                              int* err, int t0, int tstride, int ntile_arg) {
  static_assert(NT == 1 || NT == 3, "one or three BF16 products");
  static_assert(BN == 64 || BN == 128, "64- or 128-wide tiles");
  static_assert(TPC == 1 || (TPC == 2 && NT == 3), "two tiles per CTA: split BF16 (one CTA per SM)");
  constexpr int kStageBytes = gemm_stage_bytes(NT, BN);
  constexpr int kB = gemm_btile_bytes(BN);
  constexpr int kGemmStages = STG;
  constexpr uint32_t kCols = SYM ? 2 * BN : BN;  // TMEM columns of a tile: one or two accumulators
  constexpr int kGemmThreads = THR;
  static_assert(THR == 256 || THR == 512, "two or four warps per TMEM lane quarter");
  constexpr int kPerQuarter = kGemmThreads / 128;  // warps per TMEM lane quarter
  extern __shared__ __align__(1024) uint8_t gemm_smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(gemm_smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t full[kGemmStages], empty[kGemmStages], done[TPC];
  __shared__ uint32_t tmem_base;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kGemmStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int i = 0; i < TPC; ++i) mbar_init(&done[i], 1);
    mbar_fence_init();
  }
  if (warp == 0) {
    tmem_alloc(&tmem_base, TPC * kCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = tmem_base;
  // This CTA's tiles: TPC = 1 the grid's (x, y, z) tile; TPC = 2 tiles
  // blockIdx.x and blockIdx.x + gridDim.x of the linear order (x fastest,
  // then y, then channel; the launcher keeps every tile below 2 gridDim.x).
  const int gx = (ep.N + BN - 1) / BN, gy = (ep.M + kGemmBM - 1) / kGemmBM;
  const int ntile = TPC == 1 ? 1 : ntile_arg;
  auto tile_of = [&](int i, int& m0, int& n0, int& ch) {
    if constexpr (GRID) {  // the grid is the tile grid (x, y, channel)
      m0 = blockIdx.y * kGemmBM;
      n0 = blockIdx.x * BN;
      ch = blockIdx.z;
      return;
    }
    const int t = t0 + i * tstride;
    n0 = (t % gx) * BN;
    m0 = ((t / gx) % gy) * kGemmBM;
    ch = t / (gx * gy);
  };
  const int KB = (K + kGemmBK - 1) / kGemmBK;  // SYM: K = 2 hk, KB even
  const int KBh = SYM ? KB / 2 : KB;
  // stage layout: A_hi, [A_lo], B_hi, [B_lo] (all 1024-byte aligned)
  auto a_tile = [&](int s, int lo) { return smem + s * kStageBytes + lo * kGemmATileBytes; };
  auto b_tile = [&](int s, int lo) {
    return smem + s * kStageBytes + (NT == 3 ? 2 : 1) * kGemmATileBytes + lo * kB;
  };

  if (warp == 0 && lane == 0) {  // TMA producer: the K slices of tile 0, then of tile 1
    int issued = 0;  // slices issued, counted over the CTA's tiles (g = i KB + kb)
    bool stop = false;
    for (int i = 0; i < ntile && !stop; ++i) {
      int m0, n0, ch;
      tile_of(i, m0, n0, ch);
      const int a_koff = ch * ep.a_koff;
      for (int kb = 0; kb < KB; ++kb) {
        const int g = i * KB + kb, s = g % kGemmStages, it = g / kGemmStages;
        if (g >= kGemmStages && !mbar_wait(&empty[s], (it - 1) & 1, err, ep.wait_cycles)) {
          stop = true;
          break;
        }
        mbar_expect_tx(&full[s], kStageBytes);
        tma_load_2d(a_tile(s, 0), tA_hi, a_koff + kb * kGemmBK, m0, &full[s]);
        tma_load_2d(b_tile(s, 0), tB_hi, kb * kGemmBK, n0, &full[s]);
        if (NT == 3) {
          tma_load_2d(a_tile(s, 1), tA_lo, a_koff + kb * kGemmBK, m0, &full[s]);
          tma_load_2d(b_tile(s, 1), tB_lo, kb * kGemmBK, n0, &full[s]);
        }
        issued = g + 1;
      }
    }
    // Drain (default bound): slice g was issued only after slice g - stages
    // had landed and been consumed, so at most the last `stages` loads can
    // still be in flight; they land before the block exits, whether the
    // pipeline ran through or a wait gave up.  (Completed phases return at once.)
    for (int g = issued > kGemmStages ? issued - kGemmStages : 0; g < issued; ++g)
      mbar_wait(&full[g % kGemmStages], (g / kGemmStages) & 1, err);
  } else if (warp == 1 && lane == 0) {  // MMA issuer
    constexpr uint32_t idesc = umma_idesc_bf16(kGemmBM, BN);
    int committed = 0;  // tiles whose accumulators are committed to done[]
    bool stop = false;
    for (int i = 0; i < ntile && !stop; ++i) {
    const uint32_t tbase = taddr + (uint32_t)(i * kCols);
    for (int kb = 0; kb < KB; ++kb) {
      const int g = i * KB + kb, s = g % kGemmStages, it = g / kGemmStages;
      if (!mbar_wait(&full[s], it & 1, err, ep.wait_cycles)) {
        stop = true;
        break;
      }
      tc_fence_after();
      // SYM: even-j half into the first accumulator, odd-j half into the second
      const uint32_t acc = (SYM && kb >= KBh) ? tbase + BN : tbase;
      const bool first = SYM ? (kb == 0 || kb == KBh) : (kb == 0);
      const uint64_t a_hi = umma_desc_sw128(smem_u32(a_tile(s, 0)));
      const uint64_t b_hi = umma_desc_sw128(smem_u32(b_tile(s, 0)));
      const uint64_t a_lo = NT == 3 ? umma_desc_sw128(smem_u32(a_tile(s, 1))) : 0;
      const uint64_t b_lo = NT == 3 ? umma_desc_sw128(smem_u32(b_tile(s, 1))) : 0;
#pragma unroll
      for (int k = 0; k < kGemmBK / 16; ++k) {  // 16 BF16 = 32 bytes per MMA: start address + 2
        const uint64_t dk = (uint64_t)(2 * k);
        umma_bf16(acc, a_hi + dk, b_hi + dk, idesc, (!first || k > 0) ? 1u : 0u);
        if (NT == 3) {
          umma_bf16(acc, a_hi + dk, b_lo + dk, idesc, 1u);
          umma_bf16(acc, a_lo + dk, b_hi + dk, idesc, 1u);
        }
      }
      umma_commit(&empty[s]);
    }
    if (!stop) umma_commit(&done[i]);  // tile i's accumulators complete
    committed = stop ? i : i + 1;
    }
    // after a wait gave up: the remaining tiles' done[] too, so that no
    // epilogue wait is left without an arrival (each done[] arrives once)
    for (int i = committed; i < ntile; ++i) umma_commit(&done[i]);
  }
  __syncwarp();
  // Epilogues, tile by tile.  done[i]: every MMA of tile i has completed
  // (the MMA thread commits it after the tile's last issue, also when it gave
  // up early); waited with the default bound, as the tensor memory is freed
  // after the last one.  While warps 0 and 1 still feed the next tile, the
  // other warps of their lane quarters (three each) share its chunks.
#pragma unroll 1
  for (int i = 0; i < ntile; ++i) {
    int m0, n0, ch;
    tile_of(i, m0, n0, ch);
    const uint32_t tb = taddr + (uint32_t)(i * kCols);  // the tile's accumulators
    const bool roles_busy = TPC == 2 && i + 1 < ntile;
    const int q4w = warp & 3;
    const int first_w = (roles_busy && q4w < 2) ? q4w + 4 : q4w;  // first epilogue warp of the quarter
    const int qwarps = (kGemmThreads / 32 - first_w + 3) / 4;      // epilogue warps of the quarter
    bool ok = false;
    if (warp >= first_w) {
      ok = mbar_wait(&done[i], 0, err);
      tc_fence_after();
    }
    // Staged transposed stores (symmetric plain-BF16 split and divide epilogues):
    // the ring's shared memory, idle once the MMAs are done, holds the tile's
    // output rows (each: the tile's 128 rows m as two runs of 64 columns, even
    // and odd m, in the next GEMM's K layout), then the block writes them out as
    // 16-byte vectors.  Runs sit 160 B apart in a 288-B row, so the two halves
    // of a warp's 2-byte writes fall in different banks.  Tiles that straddle
    // the channel boundary or the end of M take the per-element path below.
    constexpr int kStPitch = 144, kStRun = 80;  // BF16 elements
    constexpr int kStRows = (EPI == EPI_DIVIDE_T ? 4 : 2) * BN;
    constexpr bool kCanStage = SYM && NT == 1 && TPC == 1 && EPI != EPI_COMBINE_T &&
                               kStRows * kStPitch * 2 <= kGemmStages * kStageBytes;
    bool staged = false;
    if constexpr (kCanStage) {
      const bool regular =
          m0 + kGemmBM <= ep.M && (ep.ldo & 7) == 0 && (ep.hk & 7) == 0 &&
          (reinterpret_cast<uintptr_t>(ep.out_hi) & 15) == 0 &&
          (EPI != EPI_SPLIT_T || m0 + kGemmBM <= ep.row_b ||
           (m0 >= ep.row_b && ((m0 - ep.row_b) & 15) == 0 && (ep.col_b & 7) == 0));
      staged = __syncthreads_and(regular && ok && !*(volatile int*)err) != 0;  // uniform over the block
    }
    if (staged) {
      const int q4 = warp & 3, half = warp >> 2;
      static_assert(!kCanStage || kPerQuarter == 2, "the staged path runs two warps per quarter");
      const int lc = (lane & 1) * kStRun + q4 * 16 + (lane >> 1);  // this lane's m within a staged row
      __nv_bfloat16* st = reinterpret_cast<__nv_bfloat16*>(smem);
      const float lm = EPI == EPI_DIVIDE_T ? __ldg(ep.lam_m + m0 + q4 * 32 + lane) : 0.0f;
      const uint32_t lane_off = (uint32_t)(q4 * 32) << 16;
      for (int c = half; c < BN / 32; c += 2) {
        float u[32], e[32];
        tmem_ld32x2(tb + lane_off + (uint32_t)(c * 32), tb + lane_off + (uint32_t)(BN + c * 32), u, e);
        const int nb = n0 + c * 32;
        if (nb >= ep.N) continue;  // uniform over the warp
        const int nq = min(32, ep.N - nb);
        if constexpr (EPI == EPI_SPLIT_T) {
  #pragma unroll
          for (int q = 0; q < 32; ++q) {
            if (q < nq) {
              const int r = c * 32 + q;  // staged rows: [n | n_full - 1 - n]
              st[r * kStPitch + lc] = __float2bfloat16_rn(u[q] + e[q]);
              st[(BN + r) * kStPitch + lc] = __float2bfloat16_rn(u[q] - e[q]);
            }
          }
        } else {
          const float ln0 = lane < nq ? __ldg(ep.lam_n + nb + lane) : 0.0f;
          const float ln1 = lane < nq ? __ldg(ep.lam_n + ep.n_full - 1 - (nb + lane)) : 0.0f;
  #pragma unroll
          for (int q = 0; q < 32; ++q) {
            const float base0 = 1.0f - lm - __shfl_sync(0xffffffffu, ln0, q);
            const float base1 = 1.0f - lm - __shfl_sync(0xffffffffu, ln1, q);
            if (q < nq) {
              const int r = c * 32 + q;  // staged rows: [n | mirror | n, penalised | mirror, penalised]
              const float y0 = u[q] + e[q], y1 = u[q] - e[q];
              st[r * kStPitch + lc] = __float2bfloat16_rn(__fdividef(y0, base0));
              st[(BN + r) * kStPitch + lc] = __float2bfloat16_rn(__fdividef(y1, base1));
              st[(2 * BN + r) * kStPitch + lc] = __float2bfloat16_rn(__fdividef(y0, base0 + ep.pen));
              st[(3 * BN + r) * kStPitch + lc] = __float2bfloat16_rn(__fdividef(y1, base1 + ep.pen));
            }
          }
        }
      }
      __syncthreads();
      const int colbase = (EPI == EPI_SPLIT_T && m0 >= ep.row_b) ? ep.col_b + ((m0 - ep.row_b) >> 1) : (m0 >> 1);
      for (int v = threadIdx.x; v < kStRows * 16; v += kGemmThreads) {
        const int r = v >> 4, part = v & 15, run = part >> 3, off = (part & 7) * 8;
        const int sub = r / BN, n = n0 + (r - sub * BN);
        if (n >= ep.N) continue;
        const int grow = ((sub & 1) ? ep.n_full - 1 - n : n) + (sub >= 2 ? ep.chb_rows : 0);
        const uint4 val = *reinterpret_cast<const uint4*>(st + r * kStPitch + run * kStRun + off);
        *reinterpret_cast<uint4*>(ep.out_hi + (size_t)grow * ep.ldo + colbase + run * ep.hk + off) = val;
      }
    } else if (ok && !*(volatile int*)err) {
      const int q4 = q4w, cq = (warp - first_w) >> 2;  // TMEM lane quarter, first chunk
      const int mloc = q4 * 32 + lane;          // TMEM lane = row of the tile
      const int m = m0 + mloc;
      const bool mvalid = m < ep.M;
      const float lm = (EPI == EPI_DIVIDE_T && mvalid) ? __ldg(ep.lam_m + m) : 0.0f;
      // column of D^T that row m goes to, in the next GEMM's K layout
      const int col = (EPI == EPI_SPLIT_T && m >= ep.row_b) ? ep.col_b + sym_perm(m - ep.row_b, ep.hk)
                                                             : sym_perm(m, ep.hk);
      const uint32_t lane_off = (uint32_t)(q4 * 32) << 16;
      // at most two chunks per warp (four chunks over three or four warps)
#pragma unroll 1
      for (int r = 0; r < (BN / 32 + 2) / 3; ++r) {
        const int c = cq + r * qwarps;
        if (c >= BN / 32) break;
        float u[32], e[32];
        if constexpr (SYM) tmem_ld32x2(tb + lane_off + (uint32_t)(c * 32), tb + lane_off + (uint32_t)(BN + c * 32), u, e);
        else tmem_ld32(tb + lane_off + (uint32_t)(c * 32), u);  // whole warp
        const int nb = n0 + c * 32;
        if (nb >= ep.N) continue;  // uniform over the block
        const int nq = min(32, ep.N - nb);
        if (EPI == EPI_SPLIT_T) {
  #pragma unroll
          for (int q = 0; q < 32; ++q) {
            if (q < nq && mvalid) {
              const size_t n = (size_t)(nb + q);
              split_store<NT>(ep.out_hi, ep.out_lo, n * ep.ldo + col, SYM ? u[q] + e[q] : u[q]);
              if constexpr (SYM) split_store<NT>(ep.out_hi, ep.out_lo, (size_t)(ep.n_full - 1 - (nb + q)) * ep.ldo + col,
                                       u[q] - e[q]);
            }
          }
        } else if (EPI == EPI_DIVIDE_T) {
          // rows m: x-frequency i, columns n: y-frequency l (Eq. 4.6 divides);
          // lane l fetches lam_n at its output columns once, the warp shares them
          const float ln0 = lane < nq ? __ldg(ep.lam_n + nb + lane) : 0.0f;
          const float ln1 = (SYM && lane < nq) ? __ldg(ep.lam_n + ep.n_full - 1 - (nb + lane)) : 0.0f;
  #pragma unroll
          for (int q = 0; q < 32; ++q) {
            const float base0 = 1.0f - lm - __shfl_sync(0xffffffffu, ln0, q);
            const float base1 = SYM ? 1.0f - lm - __shfl_sync(0xffffffffu, ln1, q) : 0.0f;
            if (q < nq && mvalid) {
              const size_t n = (size_t)(nb + q);
              const float y0 = SYM ? u[q] + e[q] : u[q];
              // approximate divides (2 ulp): the results are stored in BF16 precision
              split_store<NT>(ep.out_hi, ep.out_lo, n * ep.ldo + col, __fdividef(y0, base0));
              split_store<NT>(ep.out_hi, ep.out_lo, (ep.chb_rows + n) * ep.ldo + col, __fdividef(y0, base0 + ep.pen));
              if constexpr (SYM) {
                const size_t n1 = (size_t)(ep.n_full - 1 - (nb + q));
                const float y1 = u[q] - e[q];
                split_store<NT>(ep.out_hi, ep.out_lo, n1 * ep.ldo + col, __fdividef(y1, base1));
                split_store<NT>(ep.out_hi, ep.out_lo, (ep.chb_rows + n1) * ep.ldo + col, __fdividef(y1, base1 + ep.pen));
              }
            }
          }
        } else {  // EPI_COMBINE_T: z[y][x] from channel ch where phi == ch
          // one mask word holds the 32 y of this chunk for column x = m (nb is a
          // multiple of 32); the mirrored y = n - 1 - nb - q span at most two words
          const uint32_t* colbits = ep.phibits + (size_t)(mvalid ? m : 0) * ep.wpc;
          const uint32_t b0 = mvalid ? __ldg(colbits + (nb >> 5)) : 0u;
          uint32_t bt = 0u, bb = 0u;
          int ytop = 0;
          if constexpr (SYM) {
            ytop = ep.n_full - 1 - nb;
            const int wt = ytop >> 5, wb = max(ytop - 31, 0) >> 5;
            bt = mvalid ? __ldg(colbits + wt) : 0u;
            bb = (mvalid && wb != wt) ? __ldg(colbits + wb) : bt;
          }
          const uint32_t want = (uint32_t)ch;
          const float zs = ep.zscale ? (float)*ep.zscale : 1.0f;
  #pragma unroll
          for (int q = 0; q < 32; ++q) {
            if (q < nq && mvalid) {
              if (((b0 >> q) & 1u) == want) {
                const int p = (nb + q) * ep.ldz + m;
                const float y = zs * (SYM ? u[q] + e[q] : u[q]);
                if (ep.z_double) static_cast<double*>(ep.z)[p] = (double)y;
                else static_cast<float*>(ep.z)[p] = y;
              }
              if constexpr (SYM) {
                const int yy = ytop - q;
                const uint32_t word = ((yy >> 5) == (ytop >> 5)) ? bt : bb;
                if (((word >> (yy & 31)) & 1u) == want) {
                  const int p = yy * ep.ldz + m;
                  if (ep.z_double) static_cast<double*>(ep.z)[p] = (double)(zs * (u[q] - e[q]));
                  else static_cast<float*>(ep.z)[p] = zs * (u[q] - e[q]);
                }
              }
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(taddr, TPC * kCols);
}

template <int EPI, int NT, bool SYM, int BN, int TPC = 1>
__global__ void __launch_bounds__(gemm_threads(NT), gemm_ctas_per_sm(NT, BN))
    dst_gemm_kernel(const __grid_constant__ CUtensorMap tA_hi, const __grid_constant__ CUtensorMap tA_lo,
                    const __grid_constant__ CUtensorMap tB_hi, const __grid_constant__ CUtensorMap tB_lo, int K,
                    GemmEpiParams ep, int* err, const int* gate) {
  pdl_wait();
  pdl_trigger();
  if (gate && *(volatile const int*)gate == 0) return;
  __shared__ GemmEpiParams sep;
  if (threadIdx.x == 0) sep = ep;
  __syncthreads();
  if constexpr (TPC == 1) {  // the grid is the tile grid (x, y, channel)
    dst_gemm_body<EPI, NT, SYM, BN, 1, true, const GemmEpiParams&>(&tA_hi, &tA_lo, &tB_hi, &tB_lo, K, sep, err, 0,
                                                                   0, 1);
  } else {  // one CTA per SM: tiles blockIdx.x and blockIdx.x + gridDim.x
    const int gx = (ep.N + BN - 1) / BN, gy = (ep.M + kGemmBM - 1) / kGemmBM;
    const int ntile = blockIdx.x + gridDim.x < gx * gy * ep.nch ? 2 : 1;
    dst_gemm_body<EPI, NT, SYM, BN, TPC, false, const GemmEpiParams&>(&tA_hi, &tA_lo, &tB_hi, &tB_lo, K, sep, err,
                                                                      blockIdx.x, gridDim.x, ntile);
  }
}


// ---- grouped launches: one GEMM of the chain for many instances -------------
// One instance's GEMM: its operand maps (in global memory, 128-byte aligned
// as the CUtensorMap type is), its epilogue parameters, and for the combine
// epilogue the per-column output: z of Krylov column j at ep.z + j
// z_col_bytes, scaled by s[j] when the instance's first operand is taken
// unscaled from the basis update (fused, columns j > 0).
struct GemmGroupDesc {
  CUtensorMap a_hi, a_lo, b_hi, b_lo;
  GemmEpiParams ep;
  long long z_col_bytes;
  const double* s;
  int fused;
  int K;
  int sym;  // symmetric form (even transform length)
};

// One CTA per tile over every instance's tile grid: instance i owns the CTAs
// [active[i], active[i+1]) (a compacted prefix: finished instances own none),
// local tile t = blockIdx.x - active[i] in the linear tile order.  CTAs past
// active[count] return at once (the grid covers every instance running).
// The instances' K extents are short (a few 64-wide slices), so a tile is
// mostly pipeline fill and epilogue: two CTAs share an SM (eight warps each,
// a two-stage ring) and one's epilogue overlaps the other's MMAs.
constexpr int kGroupThreads = 256, kGroupStages = 2;
__host__ __device__ constexpr int gemm_group_smem(int NT, int BN) {
  return kGroupStages * gemm_stage_bytes(NT, BN) + 1024;
}
template <int EPI, int NT, int BN>
__global__ void __launch_bounds__(kGroupThreads, 2)
    dst_gemm_group_kernel(const GemmGroupDesc* __restrict__ d, const int* __restrict__ active, int count, int j,
                          int* err) {
  const int b = blockIdx.x;
  if (b >= active[count]) return;  // uniform over the block
  int i = 0;  // the last i with active[i] <= b (empty ranges skipped)
  for (int hi = count - 1; i < hi;) {
    const int mid = (i + hi + 1) >> 1;
    if (active[mid] <= b) i = mid;
    else hi = mid - 1;
  }
  const GemmGroupDesc& D = d[i];
  __shared__ GemmEpiParams sep;
  if (threadIdx.x == 0) {
    sep = D.ep;
    if (EPI == EPI_COMBINE_T) {
      sep.z = static_cast<char*>(D.ep.z) + (size_t)j * (size_t)D.z_col_bytes;
      sep.zscale = (D.fused && j > 0) ? D.s + j : nullptr;
    }
  }
  __syncthreads();
  const int t = b - active[i];
  if (D.sym)
    dst_gemm_body<EPI, NT, true, BN, 1, false, const GemmEpiParams&, kGroupThreads, kGroupStages>(
        &D.a_hi, &D.a_lo, &D.b_hi, &D.b_lo, D.K, sep, err, t, 0, 1);
  else
    dst_gemm_body<EPI, NT, false, BN, 1, false, const GemmEpiParams&, kGroupThreads, kGroupStages>(
        &D.a_hi, &D.a_lo, &D.b_hi, &D.b_lo, D.K, sep, err, t, 0, 1);
}

}  // namespace rsfde
