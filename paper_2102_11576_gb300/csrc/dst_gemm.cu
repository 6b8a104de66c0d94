// dst_gemm.cu -- the preconditioner of Eq. 4.6 with every sine transform done
// as a tensor-core GEMM (dst_gemm.cuh) in split BF16 (three products) or
// plain BF16 (one product).
//
// P-hat^-1 v = (1-Phi) S W1 + Phi S W2 with S = S_{n2} (x) S_{n1}, W = S v,
// W1 = W / (1 - Lx - Ly), W2 = W / (1 + dt/eta - Lx - Ly).  As matrices
// (rows y, columns x): S v = S_y V S_x.  The passes, each "A times S" with the
// output stored transposed so the next pass again multiplies rows by S:
//   0. split:    A0 = split(scale * V)                      (n2 x n1)
//   1. GEMM:     T1t = (A0 S_x)^T                            (n1 x n2)
//   2. GEMM:     W^T = T1t S_y, epilogue: both tau divides, stored transposed
//                as the stacked [W1; W2]                     (2 n2 x n1)
//   3. GEMM:     Yt = ([W1; W2] S_x)^T, channels side by side (n1 x 2 ld2)
//   4. GEMM x2:  (S_y W_c S_x)^T = Yt_c S_y; the epilogue writes z where the
//                mask selects channel c.
// All BF16 matrices have a leading dimension padded to a multiple of 64 and
// are zeroed once, so tile reads past the valid extent see zeros.  Plain BF16
// keeps only the leading matrix of every pair.
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "dst_gemm.cuh"
#include "internal.h"

namespace rsfde {

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

int pad64(int n) { return (n + 63) / 64 * 64; }

struct Bf16Mat {
  __nv_bfloat16* hi = nullptr;
  __nv_bfloat16* lo = nullptr;
  int rows = 0, cols = 0, ld = 0;
  CUtensorMap map_hi, map_lo;      // tiles of 128 rows (A operands, 128-wide B)
  CUtensorMap map64_hi, map64_lo;  // tiles of 64 rows (64-wide B)
};

bool make_map(CUtensorMap* m, void* p, int rows, int cols, int ld, int box_rows = kGemmBM) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t stride[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)kGemmBK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, p, dim, stride, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// A = scale * V split into a BF16 pair (rows y, columns x, leading dim ld).
// FP64 input is scaled in FP64; FP32 and double-FP32 input in FP32.
__device__ __forceinline__ float scaled_f32(double sc, float, double v) { return (float)(sc * v); }
__device__ __forceinline__ float scaled_f32(double, float scf, df v) { return __fmul_rn(scf, __fadd_rn(v.hi, v.lo)); }
__device__ __forceinline__ float scaled_f32(double, float scf, float v) { return __fmul_rn(scf, v); }

// Column x goes to column sym_perm(x, hk) (the symmetric GEMM's K layout;
// hk = 0: natural order).  FP32 rows whose length is a multiple of 4 move four
// values per thread (one 16-byte load; in the symmetric layout the even and
// the odd pair each land as one 4-byte store).
template <typename Tin, int NT>
__global__ void __launch_bounds__(kBlock) split_kernel(const Tin* __restrict__ v, const double* scale,
                                                       __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                                                       int n1, int n2, int ld, int hk, const int* gate) {
  pdl_wait();
  pdl_trigger();
  if (gate && *(volatile const int*)gate == 0) return;
  const double sc = scale ? *scale : 1.0;
  const float scf = (float)sc;
  if constexpr (std::is_same<Tin, float>::value && NT == 1) {
    if (hk && (n1 & 3) == 0) {
      const int q1 = n1 >> 2;
      for (int j = blockIdx.y; j < n2; j += gridDim.y)
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < q1; i += gridDim.x * blockDim.x) {
          const float4 t = *reinterpret_cast<const float4*>(v + (size_t)j * n1 + 4 * i);
          // x = 4i, 4i+2 (even) -> columns 2i, 2i+1; x = 4i+1, 4i+3 (odd) -> hk + 2i, hk + 2i + 1
          const __nv_bfloat162 ev = __floats2bfloat162_rn(__fmul_rn(scf, t.x), __fmul_rn(scf, t.z));
          const __nv_bfloat162 od = __floats2bfloat162_rn(__fmul_rn(scf, t.y), __fmul_rn(scf, t.w));
          *reinterpret_cast<__nv_bfloat162*>(hi + (size_t)j * ld + 2 * i) = ev;
          *reinterpret_cast<__nv_bfloat162*>(hi + (size_t)j * ld + hk + 2 * i) = od;
        }
      return;
    }
  }
  for (int j = blockIdx.y; j < n2; j += gridDim.y)
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n1; i += gridDim.x * blockDim.x) {
      const float x = scaled_f32(sc, scf, v[(size_t)j * n1 + i]);
      const __nv_bfloat16 h = __float2bfloat16_rn(x);
      const size_t o = (size_t)j * ld + sym_perm(i, hk);
      hi[o] = h;
      if (NT == 3) lo[o] = __float2bfloat16_rn(x - __bfloat162float(h));
    }
}

// The mask for the combine epilogue: bits[x * wpc + y / 32] bit y % 32 = phi[y][x] != 0.
__global__ void __launch_bounds__(kBlock) mask_bits_kernel(const uint8_t* __restrict__ phi, uint32_t* bits, int n1,
                                                           int n2, int wpc) {
  const long total = (long)n1 * wpc;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const int x = (int)(t / wpc), w = (int)(t - (long)x * wpc);
    uint32_t b = 0;
    for (int k = 0; k < 32; ++k) {
      const int y = 32 * w + k;
      if (y < n2 && phi[(size_t)y * n1 + x]) b |= 1u << k;
    }
    bits[t] = b;
  }
}

// Rows over blockIdx.y, columns over blockIdx.x: about 4096 blocks of 256.
static dim3 split_grid(int n1, int n2) {
  const int gx = (n1 + kBlock - 1) / kBlock;
  int gy = 4096 / gx;
  if (gy < 1) gy = 1;
  if (gy > n2) gy = n2;
  return dim3(gx, gy);
}

}  // namespace

struct Bf16Plan {
  int n1 = 0, n2 = 0;
  int ld1 = 0, ld2 = 0;  // K extent (and leading dimension) of an x- and a y-transform operand
  int h1 = 0, h2 = 0;    // symmetric form: half of that extent (0: natural layout, full GEMMs)
  int nt = 3;            // BF16 products per GEMM: 3 (split) or 1 (plain)
  uint32_t* phibits = nullptr;  // the mask, transposed and bit-packed (wpc words per column x)
  int wpc = 0;
  Bf16Mat Sx, Sy, A0, T1t, Wst, Yt;
  const float* lamx = nullptr;
  const float* lamy = nullptr;
  int* err = nullptr;
  void* mem = nullptr;
  long long wait_cycles = kWaitCycles;  // bound of each pipeline wait of the GEMM launches
  int bn[4] = {0, 0, 0, 0};             // tile width of each GEMM of the chain (0: the default rule)
};

// S_n as a split BF16 pair: [S_n]_{ij} = sqrt(2/(n+1)) sin(pi i j/(n+1)), FP64 on the host
// (exactly zero where i j is a multiple of n + 1).  Symmetric form (hk > 0): only
// the rows i <= (n+1)/2 (for odd n the middle row pairs with itself, its
// odd-j entries zero), columns in sym_perm order.
static void host_sine_matrix(int n, int ld, int hk, std::vector<__nv_bfloat16>& hi,
                             std::vector<__nv_bfloat16>& lo) {
  const int rows = hk ? (n + 1) / 2 : n;
  hi.assign((size_t)rows * ld, __float2bfloat16(0.0f));
  lo.assign((size_t)rows * ld, __float2bfloat16(0.0f));
  const long per = 2L * (n + 1);
  const double sc = std::sqrt(2.0 / (n + 1));
  std::vector<double> sn(per);
  for (long m = 0; m < per; ++m)
    sn[m] = m % (n + 1) == 0 ? 0.0 : sc * std::sin(M_PI * (double)m / (double)(n + 1));
  for (int i = 1; i <= rows; ++i)
    for (int j = 1; j <= n; ++j) {
      const float x = (float)sn[((long)i * j) % per];
      const __nv_bfloat16 h = __float2bfloat16(x);
      const size_t o = (size_t)(i - 1) * ld + sym_perm(j - 1, hk);
      hi[o] = h;
      lo[o] = __float2bfloat16(x - __bfloat162float(h));
    }
}

int bf16_plan_create(Bf16Plan** out, int n1, int n2, int nt, const float* lamx, const float* lamy,
                     const uint8_t* phi, cudaStream_t s) {
  *out = nullptr;
  if (!encode_fn()) return RSFDE_ECUDA;
  if (nt != 1 && nt != 3) return RSFDE_EINVAL;
  Bf16Plan* p = new Bf16Plan();
  p->nt = nt;
  p->n1 = n1;
  p->n2 = n2;
  // even n1 and n2: the symmetric form (half the MMAs)
  // the symmetric form (half the MMAs): split BF16 at every n; plain BF16,
  // whose staged epilogue writes the two outputs of a pair from different
  // threads, only where no output pairs with itself (even n)
  const bool sym = nt == 3 || (n1 % 2 == 0 && n2 % 2 == 0);
  p->h1 = sym ? pad64((n1 + 1) / 2) : 0;
  p->h2 = sym ? pad64((n2 + 1) / 2) : 0;
  p->ld1 = sym ? 2 * p->h1 : pad64(n1);
  p->ld2 = sym ? 2 * p->h2 : pad64(n2);
  const int c1 = sym ? p->ld1 : n1, c2 = sym ? p->ld2 : n2;  // K extents of the tensor maps
  p->lamx = lamx;
  p->lamy = lamy;
  struct Spec {
    Bf16Mat* m;
    int rows, cols, ld;
  } specs[] = {{&p->Sx, sym ? (n1 + 1) / 2 : n1, c1, p->ld1}, {&p->Sy, sym ? (n2 + 1) / 2 : n2, c2, p->ld2},
               {&p->A0, n2, c1, p->ld1},                {&p->T1t, n1, c2, p->ld2},
               {&p->Wst, 2 * n2, c1, p->ld1},           {&p->Yt, n1, 2 * p->ld2, 2 * p->ld2}};
  const int parts = nt == 3 ? 2 : 1;
  p->wpc = (n2 + 31) / 32;
  const size_t bits_bytes = ((size_t)n1 * p->wpc * sizeof(uint32_t) + 255) / 256 * 256;
  size_t total = 256 + bits_bytes;
  for (auto& sp : specs) total += parts * ((size_t)sp.rows * sp.ld * sizeof(__nv_bfloat16) + 256);
  cudaError_t e = cudaMalloc(&p->mem, total);
  if (e != cudaSuccess) {
    delete p;
    return e == cudaErrorMemoryAllocation ? RSFDE_ENOMEM : RSFDE_ECUDA;
  }
  cudaMemsetAsync(p->mem, 0, total, s);
  uint8_t* base = static_cast<uint8_t*>(p->mem);
  size_t off = 0;
  p->err = reinterpret_cast<int*>(base);
  off += 256;
  p->phibits = reinterpret_cast<uint32_t*>(base + off);
  off += bits_bytes;
  for (auto& sp : specs) {
    const size_t bytes = (size_t)sp.rows * sp.ld * sizeof(__nv_bfloat16);
    sp.m->rows = sp.rows;
    sp.m->cols = sp.cols;
    sp.m->ld = sp.ld;
    sp.m->hi = reinterpret_cast<__nv_bfloat16*>(base + off);
    off += (bytes + 255) / 256 * 256;
    sp.m->lo = sp.m->hi;  // plain BF16: no second matrix (the kernels never touch it)
    if (nt == 3) {
      sp.m->lo = reinterpret_cast<__nv_bfloat16*>(base + off);
      off += (bytes + 255) / 256 * 256;
    }
    if (!make_map(&sp.m->map_hi, sp.m->hi, sp.rows, sp.cols, sp.ld) ||
        !make_map(&sp.m->map_lo, sp.m->lo, sp.rows, sp.cols, sp.ld) ||
        !make_map(&sp.m->map64_hi, sp.m->hi, sp.rows, sp.cols, sp.ld, 64) ||
        !make_map(&sp.m->map64_lo, sp.m->lo, sp.rows, sp.cols, sp.ld, 64)) {
      cudaFree(p->mem);
      delete p;
      return RSFDE_ECUDA;
    }
  }
  std::vector<__nv_bfloat16> hi, lo;
  host_sine_matrix(n1, p->ld1, p->h1, hi, lo);
  cudaMemcpyAsync(p->Sx.hi, hi.data(), hi.size() * 2, cudaMemcpyHostToDevice, s);
  if (nt == 3) cudaMemcpyAsync(p->Sx.lo, lo.data(), lo.size() * 2, cudaMemcpyHostToDevice, s);
  cudaStreamSynchronize(s);
  mask_bits_kernel<<<vec_grid((size_t)n1 * p->wpc), kBlock, 0, s>>>(phi, p->phibits, n1, n2, p->wpc);
  host_sine_matrix(n2, p->ld2, p->h2, hi, lo);
  cudaMemcpyAsync(p->Sy.hi, hi.data(), hi.size() * 2, cudaMemcpyHostToDevice, s);
  if (nt == 3) cudaMemcpyAsync(p->Sy.lo, lo.data(), lo.size() * 2, cudaMemcpyHostToDevice, s);
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaFree(p->mem);
    delete p;
    return RSFDE_ECUDA;
  }
  *out = p;
  return RSFDE_OK;
}

int bf16_plan_nt(const Bf16Plan* p) { return p ? p->nt : 0; }

void bf16_plan_destroy(Bf16Plan* p) {
  if (!p) return;
  if (p->mem) cudaFree(p->mem);
  delete p;
}

// Reads and clears the give-up flag of the plan's GEMM launches: a wait that
// gave up left that launch's output incomplete (RSFDE_ETIMEOUT), but every
// copy and MMA it had issued completed before it exited, so the plan stays
// usable.
int bf16_plan_error(Bf16Plan* p, cudaStream_t s) {
  int h = 0;
  if (cudaMemcpyAsync(&h, p->err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return RSFDE_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return RSFDE_ECUDA;
  if (h && cudaMemsetAsync(p->err, 0, sizeof(int), s) != cudaSuccess) return RSFDE_ECUDA;
  return h ? RSFDE_ETIMEOUT : RSFDE_OK;
}

void bf16_plan_set_wait(Bf16Plan* p, long long cycles) {
  if (p) p->wait_cycles = cycles > 0 ? cycles : kWaitCycles;
}

// One tile per CTA while the tiles fit one wave; split BF16 with between one
// and two waves of tiles runs one CTA per SM with two tiles each (the second
// tile's main loop overlaps the first one's epilogue; the makespan is two
// main loops and one epilogue instead of two of each).
template <int EPI, int NT, bool SYM, int BN>
static void launch_gemm_t(const Bf16Mat& A, const Bf16Mat& B, int M, int N, int K, int channels,
                          GemmEpiParams ep, int* err, const int* gate, cudaStream_t s) {
  constexpr int smem = gemm_smem(NT, BN);
  const CUtensorMap& bh = BN == 64 ? B.map64_hi : B.map_hi;
  const CUtensorMap& bl = BN == 64 ? B.map64_lo : B.map_lo;
  const int gx = (N + BN - 1) / BN, gy = (M + kGemmBM - 1) / kGemmBM;
  const long tiles = (long)gx * gy * channels;
  ep.nch = channels;
  if constexpr (NT == 3) {
    if (tiles > kNumSMs && tiles <= 2L * kNumSMs) {
      auto k = dst_gemm_kernel<EPI, NT, SYM, BN, 2>;
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      launch_pdl(k, dim3(kNumSMs), dim3(gemm_threads(NT)), smem, s, A.map_hi, A.map_lo, bh, bl, K, ep, err,
                 gate);
      return;
    }
  }
  auto k = dst_gemm_kernel<EPI, NT, SYM, BN, 1>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  launch_pdl(k, dim3(gx, gy, channels), dim3(gemm_threads(NT)), smem, s, A.map_hi, A.map_lo, bh, bl, K, ep, err,
             gate);
}
// Tile width of a GEMM: the plan's recorded choice (autotuner) or the default
// rule.  Plain BF16 (two operand tiles per K slice) takes 64-wide tiles
// while 128-wide ones would leave SMs idle (measured: with at least one
// 128-wide tile per SM the wider tiles are faster).  Split BF16 feeds four
// operand tiles per K slice for three products: a 64-wide tile brings 48 KB
// per slice for 3.1 MFLOP and is bound by the SM's operand inflow, a 128-wide
// one 64 KB for 6.3 MFLOP, so it takes 128 while that keeps 5/8 of the SMs busy.
static int gemm_bn(int nt, int forced, int M, int N, int channels) {
  if (forced == 64 || forced == 128) return forced;
  const long tiles128 = (long)((N + 127) / 128) * ((M + kGemmBM - 1) / kGemmBM) * channels;
  if (nt == 3) return tiles128 * 8 >= 5L * kNumSMs ? 128 : 64;
  return tiles128 < kNumSMs ? 64 : 128;
}
template <int EPI, int NT, bool SYM>
static void launch_gemm_bn(const Bf16Mat& A, const Bf16Mat& B, int M, int N, int K, int channels, int forced,
                           const GemmEpiParams& ep, int* err, const int* gate, cudaStream_t s) {
  if (gemm_bn(NT, forced, M, N, channels) == 64)
    launch_gemm_t<EPI, NT, SYM, 64>(A, B, M, N, K, channels, ep, err, gate, s);
  else
    launch_gemm_t<EPI, NT, SYM, 128>(A, B, M, N, K, channels, ep, err, gate, s);
}
// D = A S for a transform of length n along K; the symmetric form (hk > 0)
// computes the n/2 output pairs from the K operand's two halves.
template <int EPI>
static void launch_gemm(const Bf16Plan* p, int stage, int hk, const Bf16Mat& A, const Bf16Mat& B, int M, int n,
                        int channels, GemmEpiParams ep, const int* gate, cudaStream_t s) {
  ep.M = M;
  ep.N = hk ? (n + 1) / 2 : n;
  ep.n_full = hk ? n : 0;
  const int K = hk ? 2 * hk : n;
  const int f = p->bn[stage];
  if (p->nt == 3) {
    if (hk) launch_gemm_bn<EPI, 3, true>(A, B, M, ep.N, K, channels, f, ep, p->err, gate, s);
    else launch_gemm_bn<EPI, 3, false>(A, B, M, ep.N, K, channels, f, ep, p->err, gate, s);
  } else {
    if (hk) launch_gemm_bn<EPI, 1, true>(A, B, M, ep.N, K, channels, f, ep, p->err, gate, s);
    else launch_gemm_bn<EPI, 1, false>(A, B, M, ep.N, K, channels, f, ep, p->err, gate, s);
  }
}

// GEMM k of the chain (bf16_precond's steps 1-4): operands, the product
// shape (M rows of A, transform length n, hk: the symmetric form's half K
// extent or 0) and the epilogue parameters (for k = 3 without z).
struct ChainGemm {
  const Bf16Mat* A;
  const Bf16Mat* B;
  int M, n, channels, hk;
  GemmEpiParams ep;
};
static void chain_gemm(const Bf16Plan* p, int k, double pen, ChainGemm* g) {
  const int n1 = p->n1, n2 = p->n2;
  GemmEpiParams ep{};
  ep.wait_cycles = p->wait_cycles;
  if (k == 0) {  // 1. T1t = (A0 S_x)^T, columns y in the layout of GEMM 2's K
    *g = ChainGemm{&p->A0, &p->Sx, n2, n1, 1, p->h1, ep};
    g->ep.out_hi = p->T1t.hi;
    g->ep.out_lo = p->T1t.lo;
    g->ep.ldo = p->ld2;
    g->ep.row_b = 1 << 30;
    g->ep.hk = p->h2;
  } else if (k == 1) {  // 2. W^T = T1t S_y; both tau divides (Eq. 4.6), stacked [W1; W2]
    *g = ChainGemm{&p->T1t, &p->Sy, n1, n2, 1, p->h2, ep};
    g->ep.out_hi = p->Wst.hi;
    g->ep.out_lo = p->Wst.lo;
    g->ep.ldo = p->ld1;
    g->ep.lam_m = p->lamx;
    g->ep.lam_n = p->lamy;
    g->ep.pen = (float)pen;
    g->ep.chb_rows = n2;
    g->ep.hk = p->h1;
  } else if (k == 2) {  // 3. Yt = ([W1; W2] S_x)^T, the channels side by side (column offset ld2)
    *g = ChainGemm{&p->Wst, &p->Sx, 2 * n2, n1, 1, p->h1, ep};
    g->ep.out_hi = p->Yt.hi;
    g->ep.out_lo = p->Yt.lo;
    g->ep.ldo = 2 * p->ld2;
    g->ep.row_b = n2;
    g->ep.col_b = p->ld2;
    g->ep.hk = p->h2;
  } else {  // 4. z = (1-Phi) S_y W1 S_x + Phi S_y W2 S_x (channel = blockIdx.z)
    *g = ChainGemm{&p->Yt, &p->Sy, n1, n2, 2, p->h2, ep};
    g->ep.phibits = p->phibits;
    g->ep.wpc = p->wpc;
    g->ep.ldz = n1;
    g->ep.a_koff = p->ld2;
  }
}

bool bf16_plan_a0(const Bf16Plan* p, int vec, Bf16Out* out) {
  if (!p || p->h1 == 0 || vec < 1 || p->n1 % vec != 0) return false;
  *out = Bf16Out{p->A0.hi, p->nt == 3 ? p->A0.lo : nullptr, p->n1, p->ld1, p->h1};
  return true;
}

template <typename Tz, typename Tin>
int bf16_precond(Bf16Plan* p, const Tin* v, const double* vscale, Tz* z, const uint8_t* phi, double pen,
                 const int* gate, cudaStream_t s, bool skip_split, const double* zscale, cudaEvent_t* ev) {
  const int n1 = p->n1, n2 = p->n2;
  if (skip_split) {
    // A0 already holds the unscaled vector (update_kernel); scale at the end
  } else if (p->nt == 3)
    launch_pdl(split_kernel<Tin, 3>, split_grid(n1, n2), dim3(kBlock), 0, s, v, vscale, p->A0.hi, p->A0.lo, n1, n2,
               p->ld1, p->h1, gate);
  else
    launch_pdl(split_kernel<Tin, 1>, split_grid(n1, n2), dim3(kBlock), 0, s, v, vscale, p->A0.hi, p->A0.lo, n1, n2,
               p->ld1, p->h1, gate);
  if (ev) cudaEventRecord(ev[0], s);
  for (int k = 0; k < 4; ++k) {
    ChainGemm g;
    chain_gemm(p, k, pen, &g);
    if (k == 3) {
      g.ep.z = z;
      g.ep.z_double = sizeof(Tz) == 8;
      g.ep.zscale = skip_split ? zscale : nullptr;
    }
    if (k == 1) launch_gemm<EPI_DIVIDE_T>(p, k, g.hk, *g.A, *g.B, g.M, g.n, g.channels, g.ep, gate, s);
    else if (k == 3) launch_gemm<EPI_COMBINE_T>(p, k, g.hk, *g.A, *g.B, g.M, g.n, g.channels, g.ep, gate, s);
    else launch_gemm<EPI_SPLIT_T>(p, k, g.hk, *g.A, *g.B, g.M, g.n, g.channels, g.ep, gate, s);
    if (ev) cudaEventRecord(ev[k + 1], s);
  }
  return cudaGetLastError() == cudaSuccess ? RSFDE_OK : RSFDE_ECUDA;
}

// Times the chain with every GEMM 64 wide, then 128 wide (reps applications
// each, CUDA events between the GEMMs on stream s, the operand v and output z
// the caller's scratch) and records the faster width per GEMM.  bn_out:
// the four widths chosen.
int bf16_plan_autotune(Bf16Plan* p, const double* v, float* z, const uint8_t* phi, double pen, cudaStream_t s,
                       int reps, int* bn_out) {
  if (!p || reps < 1) return RSFDE_EINVAL;
  cudaEvent_t ev[5];
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) return RSFDE_ECUDA;
  float best[4] = {1e30f, 1e30f, 1e30f, 1e30f};
  int pick[4] = {0, 0, 0, 0};
  for (int w : {64, 128}) {
    for (int k = 0; k < 4; ++k) p->bn[k] = w;
    bf16_precond<float, double>(p, v, nullptr, z, phi, pen, nullptr, s, false, nullptr, nullptr);  // warm-up
    float ms[4] = {0, 0, 0, 0};
    for (int r = 0; r < reps; ++r) {
      bf16_precond<float, double>(p, v, nullptr, z, phi, pen, nullptr, s, false, nullptr, ev);
      if (cudaEventSynchronize(ev[4]) != cudaSuccess) break;
      for (int k = 0; k < 4; ++k) {
        float t = 0.f;
        cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
        ms[k] += t;
      }
    }
    for (int k = 0; k < 4; ++k)
      if (ms[k] < best[k]) {
        best[k] = ms[k];
        pick[k] = w;
      }
  }
  for (int k = 0; k < 4; ++k) {
    p->bn[k] = pick[k];
    if (bn_out) bn_out[k] = pick[k];
  }
  for (auto& e : ev) cudaEventDestroy(e);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return RSFDE_ECUDA;
  return bf16_plan_error(p, s);
}

// ---- the batch's lock-step form: every instance's GEMM in one launch ---------
void bf16_plan_a0_any(const Bf16Plan* p, Bf16Out* out) {
  *out = Bf16Out{p->A0.hi, p->nt == 3 ? p->A0.lo : nullptr, p->n1, p->ld1, p->h1};
}

// The descriptors of the four GEMMs of every instance (stage-major: stage k,
// instance i at k * count + i), 64-wide tiles, and their tile counts.
int bf16_group_create(const std::vector<Bf16GroupInst>& in, void** descs, std::vector<int>* tiles) {
  *descs = nullptr;
  const int n = (int)in.size();
  std::vector<GemmGroupDesc> h(4 * (size_t)n);
  for (int k = 0; k < 4; ++k) tiles[k].assign(n, 0);
  for (int i = 0; i < n; ++i) {
    const Bf16Plan* p = in[i].plan;
    if (!p || p->nt != 3) return RSFDE_EINVAL;
    for (int k = 0; k < 4; ++k) {
      ChainGemm g;
      chain_gemm(p, k, in[i].pen, &g);
      GemmGroupDesc& D = h[(size_t)k * n + i];
      std::memset(static_cast<void*>(&D), 0, sizeof(D));
      D.a_hi = g.A->map_hi;
      D.a_lo = g.A->map_lo;
      D.b_hi = g.B->map64_hi;
      D.b_lo = g.B->map64_lo;
      g.ep.M = g.M;
      g.ep.N = g.hk ? (g.n + 1) / 2 : g.n;
      g.ep.n_full = g.hk ? g.n : 0;
      g.ep.nch = g.channels;
      if (k == 3) {
        g.ep.z = in[i].z;
        g.ep.z_double = in[i].z_double;
        D.z_col_bytes = (long long)in[i].z_col_bytes;
        D.s = in[i].s;
        D.fused = in[i].fused;
      }
      D.ep = g.ep;
      D.K = g.hk ? 2 * g.hk : g.n;
      D.sym = g.hk > 0;
      tiles[k][i] = ((g.ep.N + 63) / 64) * ((g.M + kGemmBM - 1) / kGemmBM) * g.channels;
    }
  }
  cudaError_t e = cudaMalloc(descs, h.size() * sizeof(GemmGroupDesc));
  if (e == cudaSuccess) e = cudaMemcpy(*descs, h.data(), h.size() * sizeof(GemmGroupDesc), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (*descs) cudaFree(*descs);
    *descs = nullptr;
    return e == cudaErrorMemoryAllocation ? RSFDE_ENOMEM : RSFDE_ECUDA;
  }
  return RSFDE_OK;
}
void bf16_group_destroy(void* descs) {
  if (descs) cudaFree(descs);
}

// GEMM k of every running instance's chain at Krylov column j: grid = the
// tiles of all instances (max_tiles); the compacted prefix `active` skips
// the finished ones.
template <int EPI>
static void launch_group_t(const GemmGroupDesc* d, int count, const int* active, int max_tiles, int j, int* err,
                           cudaStream_t s) {
  auto k = dst_gemm_group_kernel<EPI, 3, 64>;
  constexpr int smem = gemm_group_smem(3, 64);
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  k<<<max_tiles, kGroupThreads, smem, s>>>(d, active, count, j, err);
}
static_assert(kGroupMaxInstances == kMaxBatchMulti, "the grouped GEMMs stage the batch's whole prefix");
void launch_bf16_group(int k, const void* descs, int count, const int* active, int max_tiles, int j, int* err,
                       cudaStream_t s) {
  if (max_tiles <= 0) return;
  const GemmGroupDesc* d = static_cast<const GemmGroupDesc*>(descs) + (size_t)k * count;
  if (k == 1) launch_group_t<EPI_DIVIDE_T>(d, count, active, max_tiles, j, err, s);
  else if (k == 3) launch_group_t<EPI_COMBINE_T>(d, count, active, max_tiles, j, err, s);
  else launch_group_t<EPI_SPLIT_T>(d, count, active, max_tiles, j, err, s);
}

// A0 = split(s_j V_j) of every running instance (split_kernel's arithmetic,
// element by element); instances whose basis update already wrote A0
// unscaled (fused, j > 0) are skipped.
__global__ void __launch_bounds__(kBlock) split_multi_kernel(const BatchInst* __restrict__ bi,
                                                             const int* __restrict__ prefix,
                                                             const int* __restrict__ active, int count, int j) {
  __shared__ int sact[kMaxBatchMulti + 1];
  for (int k = threadIdx.x; k <= count; k += blockDim.x) sact[k] = active[k];
  __syncthreads();
  const int total = sact[count];
  for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
    const int mi = multi_instance(sact, count, vb);
    const BatchInst& I = bi[mi];
    if (j > 0 && I.a0_fused) continue;  // uniform over the block
    const int lb = vb - sact[mi], nb = __ldg(prefix + mi + 1) - __ldg(prefix + mi);
    const double* v = I.V + (size_t)j * I.N;
    const double sc = I.st->s[j];
    __nv_bfloat16* hi = static_cast<__nv_bfloat16*>(I.a0);
    __nv_bfloat16* lo = static_cast<__nv_bfloat16*>(I.a0_lo);
    for (size_t e = (size_t)lb * blockDim.x + threadIdx.x; e < I.N; e += (size_t)nb * blockDim.x) {
      const int y = (int)(e / (size_t)I.n1), x = (int)(e - (size_t)y * I.n1);
      const float xv = scaled_f32(sc, (float)sc, v[e]);
      const __nv_bfloat16 h = __float2bfloat16_rn(xv);
      const size_t o = (size_t)y * I.a0_ld + sym_perm(x, I.a0_hk);
      hi[o] = h;
      lo[o] = __float2bfloat16_rn(xv - __bfloat162float(h));
    }
  }
}
void launch_split_multi(const BatchInst* bi, const MultiGrid& g, int j, cudaStream_t s) {
  static const int grid = multi_launch_grid(split_multi_kernel, kBlock, 0, 1 << 30);
  split_multi_kernel<<<g.total < grid ? g.total : grid, kBlock, 0, s>>>(bi, g.prefix, g.active, g.count, j);
}

template int bf16_precond<float, double>(Bf16Plan*, const double*, const double*, float*, const uint8_t*, double,
                                         const int*, cudaStream_t, bool, const double*,
                                         cudaEvent_t*);
template int bf16_precond<double, double>(Bf16Plan*, const double*, const double*, double*, const uint8_t*,
                                          double, const int*, cudaStream_t, bool, const double*,
                                         cudaEvent_t*);
template int bf16_precond<float, df>(Bf16Plan*, const df*, const double*, float*, const uint8_t*, double,
                                     const int*, cudaStream_t, bool, const double*,
                                         cudaEvent_t*);
template int bf16_precond<double, df>(Bf16Plan*, const df*, const double*, double*, const uint8_t*, double,
                                      const int*, cudaStream_t, bool, const double*,
                                         cudaEvent_t*);
template int bf16_precond<float, float>(Bf16Plan*, const float*, const double*, float*, const uint8_t*, double,
                                        const int*, cudaStream_t, bool, const double*,
                                         cudaEvent_t*);
template int bf16_precond<double, float>(Bf16Plan*, const float*, const double*, double*, const uint8_t*, double,
                                         const int*, cudaStream_t, bool, const double*,
                                         cudaEvent_t*);

}  // namespace rsfde
