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

// Symmetric form (SYM): the sine matrix satisfies
//     S[n-1-i][j] = (-1)^j S[i][j]        (0-based i, j),
// so with u_i = sum over even j and e_i = sum over odd j of S[i][j] x_j the
// two outputs i and n-1-i are u_i + e_i and u_i - e_i (i < (n+1)/2; for odd n
// the middle row pairs with itself, its odd-j entries are zero and both
// writes of that output, by the same thread, carry u_i).  The K operand then
// holds the even-j entries in columns [0, hk) and the odd-j entries in
// [hk, 2 hk) (hk = (n+1)/2 rounded up to 64, zero padded), the GEMM has
// (n+1)/2 output columns and two TMEM accumulators, and half the MMAs.
__host__ __device__ __forceinline__ int sym_perm(int x, int hk) { return hk ? (x & 1) * hk + (x >> 1) : x; }

struct GemmEpiParams {
  int M, N;       // valid extent of D (N: (n+1)/2 in the symmetric form)
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
// tile (blockIdx.x, blockIdx.y, blockIdx.z).  The body is dst_gemm_tile.inc.
template <int EPI, int NT, bool SYM, int BN, int TPC = 1>
__global__ void __launch_bounds__(gemm_threads(NT), gemm_ctas_per_sm(NT, BN))
    dst_gemm_kernel(const __grid_constant__ CUtensorMap mA_hi, const __grid_constant__ CUtensorMap mA_lo,
                    const __grid_constant__ CUtensorMap mB_hi, const __grid_constant__ CUtensorMap mB_lo, int K,
                    GemmEpiParams ep, int* err, const int* gate) {
  pdl_wait();
  pdl_trigger();
  if (gate && *(volatile const int*)gate == 0) return;
  constexpr bool GRID = TPC == 1;  // one tile per CTA: the grid is the tile grid (x, y, channel)
  constexpr int THR = gemm_threads(NT), STG = gemm_stages(NT, BN);
  const CUtensorMap* tA_hi = &mA_hi;
  const CUtensorMap* tA_lo = &mA_lo;
  const CUtensorMap* tB_hi = &mB_hi;
  const CUtensorMap* tB_lo = &mB_lo;
  int t0 = 0, tstride = 0, ntile_arg = 1;
  if constexpr (TPC == 2) {  // one CTA per SM: tiles blockIdx.x and blockIdx.x + gridDim.x
    const int tx = (ep.N + BN - 1) / BN, ty = (ep.M + kGemmBM - 1) / kGemmBM;
    t0 = blockIdx.x;
    tstride = gridDim.x;
    ntile_arg = blockIdx.x + gridDim.x < tx * ty * ep.nch ? 2 : 1;
  }
#include "dst_gemm_tile.inc"
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
  int sym;  // symmetric form
};

// One CTA per tile over every instance's tile grid: instance i owns the CTAs
// [active[i], active[i+1]) (a compacted prefix: finished instances own none),
// local tile t = blockIdx.x - active[i] in the linear tile order.  CTAs past
// active[count] return at once (the grid covers every instance running).
// The instances' K extents are short (a few 64-wide slices), so a tile is
// mostly pipeline fill and epilogue: two CTAs share an SM (eight warps each,
// a two-stage ring) and one's epilogue overlaps the other's MMAs.
constexpr int kGroupThreads = 256, kGroupStages = 2;
constexpr int kGroupMaxInstances = 1024;  // the compacted prefix a CTA stages in shared memory
__host__ __device__ constexpr int gemm_group_smem(int NT, int BN) {
  return kGroupStages * gemm_stage_bytes(NT, BN) + 1024;
}
// Tile t of instance D's GEMM, epilogue parameters ep (in shared memory).
template <int EPI, int NT, bool SYM, int BN>
__device__ __forceinline__ void group_tile(const GemmGroupDesc& D, const GemmEpiParams& ep, int* err, int t) {
  constexpr int TPC = 1;
  constexpr bool GRID = false;
  constexpr int THR = kGroupThreads, STG = kGroupStages;
  const CUtensorMap* tA_hi = &D.a_hi;
  const CUtensorMap* tA_lo = &D.a_lo;
  const CUtensorMap* tB_hi = &D.b_hi;
  const CUtensorMap* tB_lo = &D.b_lo;
  const int K = D.K;
  const int t0 = t, tstride = 0, ntile_arg = 1;
#include "dst_gemm_tile.inc"
}
template <int EPI, int NT, int BN>
__global__ void __launch_bounds__(kGroupThreads, 2)
    dst_gemm_group_kernel(const GemmGroupDesc* __restrict__ d, const int* __restrict__ active, int count, int j,
                          int* err) {
  const int b = blockIdx.x;
  // the prefix in shared memory first (one coalesced read instead of a chain
  // of dependent global reads in the search)
  __shared__ int sact[kGroupMaxInstances + 1];
  for (int k = threadIdx.x; k <= count; k += blockDim.x) sact[k] = active[k];
  __syncthreads();
  if (b >= sact[count]) return;  // uniform over the block
  int i = 0;  // the last i with sact[i] <= b (empty ranges skipped)
  for (int hi = count - 1; i < hi;) {
    const int mid = (i + hi + 1) >> 1;
    if (sact[mid] <= b) i = mid;
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
  const int t = b - sact[i];
  if (D.sym) group_tile<EPI, NT, true, BN>(D, sep, err, t);
  else group_tile<EPI, NT, false, BN>(D, sep, err, t);
}

}  // namespace rsfde
