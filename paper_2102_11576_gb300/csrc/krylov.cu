// krylov.cu -- grid-vector kernels of the flexible GMRES solve:
// right side of Eq. 2.17, fused multi-dot and update of the classical
// Gram-Schmidt Arnoldi step, the Givens least squares (single thread, in the
// last block of the norm reduction) and the solution update.
//
// The Krylov basis has the Arnoldi operator's precision: FP64, double-FP32
// (df.cuh) or FP32.  In the last two the Gram-Schmidt arithmetic runs on the
// FP32 pipe as well (GB300 issues FP32 at 58x its FP64 rate) and only the
// per-warp sums, the Hessenberg entries and the Givens step are FP64.
//
// Every reduction is two-level and deterministic: fixed grid, per-block
// partials in block order, summed in a fixed order by the last block.
#include <type_traits>

#include "internal.h"

namespace rsfde {

int vec_grid(size_t N) {
  size_t blocks = (N + kBlock * 4 - 1) / (kBlock * 4);
  const size_t cap = (size_t)kNumSMs * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

static __device__ __forceinline__ bool closed(const int* gate) { return *(volatile const int*)gate == 0; }

__device__ __forceinline__ void init_state_body(SolverState* st, int m, int max_iter, double tol) {
  st->run_iter = 0;
  st->run_cycle = 1;
  st->status = 0;
  st->converged = 0;
  st->jlast = 0;
  st->iters = 0;
  st->cycles = 0;
  st->max_iter = max_iter;
  st->m = m;
  st->zero_solution = 0;
  st->body_runs = 0;
  st->sum_j = 0;
  st->counter = 0;
  st->tol = tol;
  st->bnorm = 0.0;
  st->beta = 0.0;
  st->rel_res = 0.0;
}
__global__ void init_state_kernel(SolverState* st, int m, int max_iter, double tol) {
  init_state_body(st, m, max_iter, tol);
}

__global__ void mask_to_phi_kernel(const uint8_t* __restrict__ in_omega, uint8_t* __restrict__ phi, size_t N) {
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x)
    phi[p] = in_omega[p] ? 0 : 1;
}

// Eq. 2.17 right side with f(u) = u - u^3 + s, zero outside Omega (Section 2),
// and the initial guess of Section 5; ||b||_2 goes to st->bnorm.
__device__ __forceinline__ void rhs_body(const double* __restrict__ u, const double* __restrict__ uu,
                                         const double* __restrict__ src, const uint8_t* __restrict__ phi, double dt,
                                         double* __restrict__ b, double* __restrict__ x0, size_t N, double* partials,
                                         SolverState* st, int bid, int nblk) {
  __shared__ double red[32];
  double acc = 0.0;
  for (size_t p = bid * (size_t)blockDim.x + threadIdx.x; p < N; p += (size_t)nblk * blockDim.x) {
    const double up = u[p];
    const double f = up - up * up * up + (src ? src[p] : 0.0);
    const double bp = up + (phi[p] ? 0.0 : dt * f);
    b[p] = bp;
    x0[p] = uu ? 2.0 * up - uu[p] : up;
    acc += bp * bp;
  }
  const double bs = block_sum(acc, red);
  if (threadIdx.x == 0) partials[bid] = bs;
  if (arrive_last(&st->counter, nblk)) {
    const double tot = sum_partials(partials, nblk, red);
    if (threadIdx.x == 0) st->bnorm = sqrt(tot);
  }
}
__global__ void __launch_bounds__(kBlock) rhs_kernel(const double* __restrict__ u, const double* __restrict__ uu,
                                                     const double* __restrict__ src, const uint8_t* __restrict__ phi,
                                                     double dt, double* __restrict__ b, double* __restrict__ x0,
                                                     size_t N, double* partials, SolverState* st) {
  rhs_body(u, uu, src, phi, dt, b, x0, N, partials, st, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(kBlock) norm_b_kernel(const double* __restrict__ b, size_t N, double* partials,
                                                        SolverState* st) {
  __shared__ double red[32];
  double acc = 0.0;
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x) {
    const double v = b[p];
    acc += v * v;
  }
  const double bs = block_sum(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = bs;
  if (arrive_last(&st->counter, gridDim.x)) {
    const double tot = sum_partials(partials, gridDim.x, red);
    if (threadIdx.x == 0) st->bnorm = sqrt(tot);
  }
}

// ---- Gram-Schmidt over the Krylov basis ---------------------------------------
// Element operations of the basis type: FP64, or double-FP32 (storage and
// arithmetic; the sums leave each warp as FP64).
template <typename Tv>
struct VecOps;
template <>
struct VecOps<double> {
  static __device__ __forceinline__ double zero() { return 0.0; }
  static __device__ __forceinline__ double ld(const double* p) { return *p; }
  static __device__ __forceinline__ void st(double* p, double v) { *p = v; }
  static __device__ __forceinline__ double fma(double acc, double a, double b) { return __fma_rn(a, b, acc); }
  static __device__ __forceinline__ double from(double x) { return x; }
  static __device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
  }
};
template <>
struct VecOps<float> {
  static __device__ __forceinline__ float zero() { return 0.0f; }
  static __device__ __forceinline__ float ld(const float* p) { return *p; }
  static __device__ __forceinline__ void st(float* p, float v) { *p = v; }
  static __device__ __forceinline__ float fma(float acc, float a, float b) { return __fmaf_rn(a, b, acc); }
  static __device__ __forceinline__ float from(double x) { return (float)x; }
  // FP32 within the warp (the basis itself carries FP32 accuracy), FP64 after
  static __device__ __forceinline__ double warp_sum(float v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return (double)v;
  }
};
template <>
struct VecOps<df> {
  static __device__ __forceinline__ df zero() { return df(0.0f, 0.0f); }
  static __device__ __forceinline__ df ld(const df* p) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    return df(v.x, v.y);
  }
  static __device__ __forceinline__ void st(df* p, df v) { *reinterpret_cast<float2*>(p) = make_float2(v.hi, v.lo); }
  static __device__ __forceinline__ df fma(df acc, df a, df b) { return df_fma(acc, a, b); }
  static __device__ __forceinline__ df from(double x) { return df(x); }
  // fixed shuffle order; the result (lane 0) converted to FP64
  static __device__ __forceinline__ double warp_sum(df v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const df u(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
      v = v + u;
    }
    return double(v);
  }
};

constexpr int kWarps = kBlock / 32;

// VEC consecutive elements moved as one 16-byte access (VEC = 16 / sizeof(Tv));
// VEC = 1: one element.  The 16-byte form needs every basis vector 16-byte
// aligned, i.e. N * sizeof(Tv) a multiple of 16.
template <typename Tv, int VEC>
__device__ __forceinline__ void ld_vec(const Tv* p, Tv* o) {
  if constexpr (VEC == 1) {
    o[0] = VecOps<Tv>::ld(p);
  } else if constexpr (std::is_same<Tv, double>::value) {
    const double2 t = *reinterpret_cast<const double2*>(p);
    o[0] = t.x;
    o[1] = t.y;
  } else if constexpr (std::is_same<Tv, df>::value) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    o[0] = df(t.x, t.y);
    o[1] = df(t.z, t.w);
  } else {
    const float4 t = *reinterpret_cast<const float4*>(p);
    o[0] = t.x;
    o[1] = t.y;
    o[2] = t.z;
    o[3] = t.w;
  }
}
template <typename Tv, int VEC>
__device__ __forceinline__ void st_vec(Tv* p, const Tv* v) {
  if constexpr (VEC == 1) {
    VecOps<Tv>::st(p, v[0]);
  } else if constexpr (std::is_same<Tv, double>::value) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  } else if constexpr (std::is_same<Tv, df>::value) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0].hi, v[0].lo, v[1].hi, v[1].lo);
  } else {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
}

// Block sums of cnt <= K accumulators: warp sums, then warp k adds the
// per-warp FP64 sums of accumulator k (fixed order).  Thread 32k returns sum k.
//
// FP64 with all K (2, 4 or 8) accumulators in use: the K warp sums by
// recursive halving -- at the step over lane bit b a lane keeps half of its
// partial sums and adds the partner's matching half, so after log2 K steps
// each lane holds one accumulator's partial and the last 5 - log2 K steps
// finish it: K - 1 + 5 - log2 K additions and shuffles per lane instead of
// 5 K.  The pairs and their order are those of warp_sum (lane bits 4 down to
// 0), so every sum is the same number.
template <int K>
__device__ __forceinline__ void warp_sums_halving(const double* acc, double (*sh)[kWarps], int w, int l) {
  constexpr int R = K == 8 ? 3 : K == 4 ? 2 : 1;
  double v[K];
#pragma unroll
  for (int i = 0; i < K; ++i) v[i] = acc[i];
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int off = 16 >> s;
    constexpr int kMax = K >> 1;
    const bool up = (l & off) != 0;  // keep the upper half of the current K >> s values
#pragma unroll
    for (int i = 0; i < kMax; ++i) {
      const int half = (K >> s) >> 1;
      if (i < half) {
        const double send = up ? v[i] : v[half + i];
        const double keep = up ? v[half + i] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
      }
    }
  }
#pragma unroll
  for (int off = 16 >> R; off; off >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], off);
  if ((l & ((32 >> R) - 1)) == 0) sh[l >> (5 - R)][w] = v[0];  // accumulator l >> (5 - R)
}
template <typename Tv, int K>
__device__ __forceinline__ double block_sums(const Tv* acc, int cnt, double (*sh)[kWarps]) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if constexpr (std::is_same<Tv, double>::value && (K == 2 || K == 4 || K == 8)) {
    if (cnt == K) {
      warp_sums_halving<K>(acc, sh, w, l);
    } else {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (k < cnt) {
          const double ws = VecOps<Tv>::warp_sum(acc[k]);
          if (l == 0) sh[k][w] = ws;
        }
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (k < cnt) {
        const double ws = VecOps<Tv>::warp_sum(acc[k]);
        if (l == 0) sh[k][w] = ws;
      }
    }
  }
  __syncthreads();
  double v = 0.0;
  if (w < cnt) {
    v = l < kWarps ? sh[w][l] : 0.0;
    v = VecOps<double>::warp_sum(v);
  }
  return v;
}

// Partial sums acc[k] += <w, V_{i0+k}> over this thread's packs for exactly
// C vectors (k < C).  C is a compile-time count, so no multiply-add is spent
// on an empty slot (the FP64 forms are bound by the FP64 pipe).  A thread
// takes UNR packs per round, so about eight loads are in flight; the packs are
// visited in grid-stride order.
template <typename Tv, int VEC, int C, int UNR>
__device__ __forceinline__ void dot_rounds(const Tv* __restrict__ V, const Tv* __restrict__ w, size_t N, int i0,
                                           Tv* acc, int bx, int nbx) {
  using Op = VecOps<Tv>;
  const size_t NP = N / VEC;  // VEC divides N (launcher)
  const size_t stride = (size_t)nbx * blockDim.x;
  for (size_t q0 = bx * (size_t)blockDim.x + threadIdx.x; q0 < NP; q0 += UNR * stride) {
    Tv wv[UNR][VEC];
    Tv a[UNR][C][VEC];  // all loads issued before the arithmetic
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      const size_t q = q0 + u * stride;
      const bool in = q < NP;
      if (in) {
        ld_vec<Tv, VEC>(w + q * VEC, wv[u]);
      } else {
#pragma unroll
        for (int e = 0; e < VEC; ++e) wv[u][e] = Op::zero();
      }
#pragma unroll
      for (int k = 0; k < C; ++k) {
        if (in) {
          ld_vec<Tv, VEC>(V + (size_t)(i0 + k) * N + q * VEC, a[u][k]);
        } else {
#pragma unroll
          for (int e = 0; e < VEC; ++e) a[u][k][e] = Op::zero();
        }
      }
    }
#pragma unroll
    for (int u = 0; u < UNR; ++u)
#pragma unroll
      for (int k = 0; k < C; ++k)
#pragma unroll
        for (int e = 0; e < VEC; ++e) acc[k] = Op::fma(acc[k], wv[u][e], a[u][k][e]);
  }
}

// h_i = <w, v_i> = s_i <V_{j+1}, V_i> for i = 0..j  (w is stored in slot j+1).
// blockIdx.y selects a chunk of at most CH basis vectors (the j+1 vectors
// spread evenly over gridDim.y chunks); w is re-read per chunk (it stays in
// L2).  The chunk's exact count selects the unrolled body (dot_rounds).
// accumulate = 1 adds to H (second CGS pass).  The last block finishes the
// j+1 sums, one warp per sum.
template <typename Tv, int VEC, int CH>
__device__ __forceinline__ void multidot_body(const Tv* __restrict__ V, size_t N, int j, int accumulate,
                                              double* partials, SolverState* st, int bx, int nbx, int by, int nby) {
  if (closed(&st->run_iter)) return;
  using Op = VecOps<Tv>;
  constexpr int UNR = kDotChunk / CH;
  __shared__ double wsum[CH][kWarps];
  const int per = (j + 1 + nby - 1) / nby;  // <= CH (launcher)
  const int i0 = by * per;
  const int cnt = min(per, j + 1 - i0);
  const Tv* __restrict__ w = V + (size_t)(j + 1) * N;
  Tv acc[CH];
#pragma unroll
  for (int k = 0; k < CH; ++k) acc[k] = Op::zero();
  switch (cnt) {  // uniform over the block
#define RSFDE_DOT_CASE(C) \
  case C:                \
    if constexpr (C <= CH) dot_rounds<Tv, VEC, C, UNR>(V, w, N, i0, acc, bx, nbx); \
    break;
    RSFDE_DOT_CASE(1)
    RSFDE_DOT_CASE(2)
    RSFDE_DOT_CASE(3)
    RSFDE_DOT_CASE(4)
    RSFDE_DOT_CASE(5)
    RSFDE_DOT_CASE(6)
    RSFDE_DOT_CASE(7)
    RSFDE_DOT_CASE(8)
#undef RSFDE_DOT_CASE
    default:
      break;
  }
  const int G = nbx;
  const double bs = block_sums<Tv, CH>(acc, cnt, wsum);
  const int wk = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0 && wk < cnt) partials[(size_t)(i0 + wk) * G + bx] = bs;
  if (arrive_last(&st->counter, nbx * nby)) {
    for (int i = wk; i <= j; i += kWarps) {
      const double tot = warp_sum_fixed(partials + (size_t)i * G, G);
      if ((threadIdx.x & 31) == 0) {
        const double h = st->s[i] * tot;
        st->hcol[i] = h;
        if (accumulate) st->H[i * kMaxRestart + j] += h;
        else st->H[i * kMaxRestart + j] = h;
      }
    }
  }
}
template <typename Tv, int VEC, int CH>
__global__ void __launch_bounds__(kBlock) multidot_kernel(const Tv* __restrict__ V, size_t N, int j, int accumulate,
                                                          double* partials, SolverState* st) {
  multidot_body<Tv, VEC, CH>(V, N, j, accumulate, partials, st, blockIdx.x, gridDim.x, blockIdx.y, gridDim.y);
}

// Loads chunk k < C of the basis (vectors i0 .. i0+C-1) for UNR packs, then
// subtracts them from val in the order i0, i0+1, ...; every load is issued
// before the dependent chains.
template <typename Tv, int VEC, int C, int UNR>
__device__ __forceinline__ void update_chunk(const Tv* __restrict__ V, size_t N, size_t NP, size_t q0,
                                             size_t stride, int i0, const Tv* ncoef, Tv (&val)[UNR][VEC]) {
  using Op = VecOps<Tv>;
  Tv a[UNR][C][VEC];
#pragma unroll
  for (int u = 0; u < UNR; ++u) {
    const bool in = q0 + u * stride < NP;
#pragma unroll
    for (int k = 0; k < C; ++k) {
      if (in) {
        ld_vec<Tv, VEC>(V + (size_t)(i0 + k) * N + (q0 + u * stride) * VEC, a[u][k]);
      } else {
#pragma unroll
        for (int e = 0; e < VEC; ++e) a[u][k][e] = Op::zero();
      }
    }
  }
#pragma unroll
  for (int u = 0; u < UNR; ++u)
#pragma unroll
    for (int k = 0; k < C; ++k)
#pragma unroll
      for (int e = 0; e < VEC; ++e) val[u][e] = Op::fma(val[u][e], ncoef[i0 + k], a[u][k][e]);
}

// The update's sweep over this block's packs for j + 1 = nfull * CH + R basis
// vectors: nfull chunks of CH, then a tail of R (a compile-time count, so no
// multiply-add is issued for an empty slot -- the FP64 form is bound by the
// FP64 pipe).  Each element takes the terms in the order i = 0..j.  Returns
// this thread's part of ||w||^2.
template <typename Tv, int VEC, int CH, int R>
__device__ __forceinline__ Tv update_rounds(Tv* __restrict__ V, size_t N, int j, int nfull, int final_pass,
                                            const Tv* ncoef, const Bf16Out& bo, int bid, int nblk) {
  using Op = VecOps<Tv>;
  constexpr int UNR = kDotChunk / CH;
  Tv* __restrict__ w = V + (size_t)(j + 1) * N;
  Tv acc = Op::zero();
  const size_t NP = N / VEC;  // VEC divides N (launcher)
  const size_t stride = (size_t)nblk * blockDim.x;
  for (size_t q0 = bid * (size_t)blockDim.x + threadIdx.x; q0 < NP; q0 += UNR * stride) {
    Tv val[UNR][VEC];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      if (q0 + u * stride < NP) {
        ld_vec<Tv, VEC>(w + (q0 + u * stride) * VEC, val[u]);
      } else {
#pragma unroll
        for (int e = 0; e < VEC; ++e) val[u][e] = Op::zero();
      }
    }
    for (int c = 0; c < nfull; ++c) update_chunk<Tv, VEC, CH, UNR>(V, N, NP, q0, stride, c * CH, ncoef, val);
    if constexpr (R > 0) update_chunk<Tv, VEC, R, UNR>(V, N, NP, q0, stride, nfull * CH, ncoef, val);
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      const size_t q = q0 + u * stride;
      if (q >= NP) break;
      const size_t p = q * VEC;
      st_vec<Tv, VEC>(w + p, val[u]);
      if constexpr (std::is_same<Tv, float>::value && VEC == 4) {
        if (bo.a0 && final_pass) {  // x = p mod n1 is a multiple of 4 (n1 is)
          const int y = (int)(p / (size_t)bo.n1), x = (int)(p - (size_t)y * bo.n1);
          const size_t o = (size_t)y * bo.ld + (x >> 1);
          const __nv_bfloat162 ev = __floats2bfloat162_rn(val[u][0], val[u][2]);
          const __nv_bfloat162 od = __floats2bfloat162_rn(val[u][1], val[u][3]);
          *reinterpret_cast<__nv_bfloat162*>(bo.a0 + o) = ev;
          *reinterpret_cast<__nv_bfloat162*>(bo.a0 + o + bo.hk) = od;
          if (bo.lo) {
            const float2 e = __bfloat1622float2(ev), d = __bfloat1622float2(od);
            *reinterpret_cast<__nv_bfloat162*>(bo.lo + o) =
                __floats2bfloat162_rn(val[u][0] - e.x, val[u][2] - e.y);
            *reinterpret_cast<__nv_bfloat162*>(bo.lo + o + bo.hk) =
                __floats2bfloat162_rn(val[u][1] - d.x, val[u][3] - d.y);
          }
        }
      } else if constexpr (std::is_same<Tv, double>::value && VEC == 2) {
        if (bo.a0 && final_pass) {  // x = p mod n1 is even (n1 is): x to column x/2, x+1 to hk + x/2
          const int y = (int)(p / (size_t)bo.n1), x = (int)(p - (size_t)y * bo.n1);
          const size_t o = (size_t)y * bo.ld + (x >> 1);
          const float f0 = f32_trunc(val[u][0]), f1 = f32_trunc(val[u][1]);
          const __nv_bfloat16 h0 = __float2bfloat16_rn(f0), h1 = __float2bfloat16_rn(f1);
          bo.a0[o] = h0;
          bo.a0[o + bo.hk] = h1;
          if (bo.lo) {
            bo.lo[o] = __float2bfloat16_rn(f0 - __bfloat162float(h0));
            bo.lo[o + bo.hk] = __float2bfloat16_rn(f1 - __bfloat162float(h1));
          }
        }
      }
#pragma unroll
      for (int e = 0; e < VEC; ++e) acc = Op::fma(acc, val[u][e], val[u][e]);
    }
  }
  return acc;
}

// V_{j+1} <- V_{j+1} - sum_i (h_i s_i) V_i and ||V_{j+1}||; on the final pass
// the last block runs the Givens step.  The basis vectors are read in chunks
// of CH independent loads for each of kDotChunk / CH packs ahead of the
// dependent update chains (about eight loads in flight for every j).
template <typename Tv, int VEC, int CH>
__device__ __forceinline__ void update_body(Tv* __restrict__ V, size_t N, int j, int final_pass, double* partials,
                                            SolverState* st, const Bf16Out& bo, int bid, int nblk) {
  if (closed(&st->run_iter)) return;
  using Op = VecOps<Tv>;
  __shared__ double wsum[1][kWarps];
  __shared__ Tv ncoef[kMaxRestart + 1];
  for (int i = threadIdx.x; i <= j; i += blockDim.x) ncoef[i] = Op::from(-(st->hcol[i] * st->s[i]));
  __syncthreads();
  const int nfull = (j + 1) / CH;
  Tv acc = Op::zero();
  switch (j + 1 - nfull * CH) {  // uniform over the grid
#define RSFDE_UPD_CASE(R)                                                                            \
  case R:                                                                                            \
    if constexpr (R < CH) acc = update_rounds<Tv, VEC, CH, R>(V, N, j, nfull, final_pass, ncoef, bo, bid, nblk); \
    break;
    RSFDE_UPD_CASE(0)
    RSFDE_UPD_CASE(1)
    RSFDE_UPD_CASE(2)
    RSFDE_UPD_CASE(3)
    RSFDE_UPD_CASE(4)
    RSFDE_UPD_CASE(5)
    RSFDE_UPD_CASE(6)
    RSFDE_UPD_CASE(7)
#undef RSFDE_UPD_CASE
    default:
      break;
  }
  const double bs = block_sums<Tv, 1>(&acc, 1, wsum);
  if (threadIdx.x == 0) partials[bid] = bs;
  if (arrive_last(&st->counter, nblk) && threadIdx.x < 32) {
    const double tot = warp_sum_fixed(partials, nblk);
    if (threadIdx.x == 0 && final_pass) givens_step(st, j, sqrt(tot));
  }
}
template <typename Tv, int VEC, int CH>
__global__ void __launch_bounds__(kBlock) update_kernel(Tv* __restrict__ V, size_t N, int j, int final_pass,
                                                        double* partials, SolverState* st, Bf16Out bo) {
  update_body<Tv, VEC, CH>(V, N, j, final_pass, partials, st, bo, blockIdx.x, gridDim.x);
}

// Back substitution R y = g for the jlast columns of the cycle.
__device__ __forceinline__ void solve_y_body(SolverState* st) {
  if (closed(&st->run_cycle) || threadIdx.x != 0) return;
  const int J = st->jlast;
  for (int i = J - 1; i >= 0; --i) {
    double s = st->g[i];
    for (int k = i + 1; k < J; ++k) s -= st->H[i * kMaxRestart + k] * st->y[k];
    st->y[i] = s / st->H[i * kMaxRestart + i];
  }
}
__global__ void solve_y_kernel(SolverState* st) { solve_y_body(st); }

// x <- x + sum_{i < jlast} y_i z_i  (flexible GMRES keeps the z_i).  With FP32
// z_i the correction sum_i y_i z_i is accumulated in double-FP32 (FP32 pipe;
// FP64 products per basis vector would make the pass FP64-bound on GB300) and
// added to the FP64 x once.  The basis vectors are read in groups of eight
// independent loads.
template <typename Tz>
struct XAcc;
template <>
struct XAcc<double> {
  using C = double;  // coefficient and accumulator type
  static __device__ __forceinline__ double zero() { return 0.0; }
  static __device__ __forceinline__ double coef(double y) { return y; }
  static __device__ __forceinline__ double fma(double acc, double y, double z) { return __fma_rn(y, z, acc); }
  static __device__ __forceinline__ double value(double acc) { return acc; }
};
template <>
struct XAcc<float> {
  using C = df;
  static __device__ __forceinline__ df zero() { return df(0.0f, 0.0f); }
  static __device__ __forceinline__ df coef(double y) { return df(y); }
  static __device__ __forceinline__ df fma(df acc, df y, float z) { return df_fma(acc, y, df(z, 0.0f)); }
  static __device__ __forceinline__ double value(df acc) { return cvt<double>(acc); }
};

template <typename Tz, int VEC>
__device__ __forceinline__ void xupdate_body(double* __restrict__ x, const Tz* __restrict__ Z, size_t N,
                                             SolverState* st, int bid, int nblk) {
  if (closed(&st->run_cycle)) return;
  const int J = st->jlast;
  if (J == 0) return;
  using A = XAcc<Tz>;
  __shared__ typename A::C y[kMaxRestart];
  for (int i = threadIdx.x; i < J; i += blockDim.x) y[i] = A::coef(st->y[i]);
  __syncthreads();
  const size_t NP = N / VEC;  // VEC divides N (launcher)
  for (size_t q = bid * (size_t)blockDim.x + threadIdx.x; q < NP; q += (size_t)nblk * blockDim.x) {
    const size_t p = q * VEC;
    typename A::C acc[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) acc[e] = A::zero();
    for (int i0 = 0; i0 < J; i0 += 8) {
      Tz a[8][VEC];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (i0 + k < J) {
          ld_vec<Tz, VEC>(Z + (size_t)(i0 + k) * N + p, a[k]);
        } else {
#pragma unroll
          for (int e = 0; e < VEC; ++e) a[k][e] = Tz(0);
        }
      }
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (i0 + k < J) {
#pragma unroll
          for (int e = 0; e < VEC; ++e) acc[e] = A::fma(acc[e], y[i0 + k], a[k][e]);
        }
    }
#pragma unroll
    for (int e = 0; e < VEC; ++e) x[p + e] += A::value(acc[e]);
  }
}
template <typename Tz, int VEC>
__global__ void __launch_bounds__(kBlock) xupdate_kernel(double* __restrict__ x, const Tz* __restrict__ Z, size_t N,
                                                         SolverState* st) {
  xupdate_body<Tz, VEC>(x, Z, N, st, blockIdx.x, gridDim.x);
}

__global__ void finalize_kernel(double* __restrict__ x, size_t N, SolverState* st) {
  if (!st->zero_solution) return;
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x)
    x[p] = 0.0;
}

// z = scale * v (the identity preconditioner of plain GMRES).
template <typename Tv, typename Tz>
__global__ void __launch_bounds__(kBlock) scale_copy_kernel(const Tv* __restrict__ v, const double* scale,
                                                            Tz* __restrict__ z, size_t N, const int* gate) {
  if (closed(gate)) return;
  const double sc = *scale;
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x)
    z[p] = Tz(sc * cvt<double>(v[p]));
}

// Condition of the device-side loop over FGMRES cycles (a CUDA graph WHILE
// node): go on while the solve is running.  Each cycle with run_cycle set
// either ends the solve or counts one restart, so the loop is bounded; the
// cap below is a second, independent bound.
__global__ void loop_cond_kernel(cudaGraphConditionalHandle h, SolverState* st) {
  int go = st->run_cycle;
  st->body_runs += 1;
  st->total_body_runs += 1;
  if (go && st->body_runs > st->max_iter + 2) {
    st->status = RSFDE_ENOTCONV;
    st->run_cycle = 0;
    st->run_iter = 0;
    go = 0;
  }
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

// Adjoint step (after M mu = lam is solved): lam_prev, the source gradient and
// the two k-gradient inner products, reduced deterministically; the last
// block adds <mu, A_x u> / k_x and <mu, A_y u> / k_y into grad_k.
__global__ void __launch_bounds__(kBlock)
    adjoint_accum_kernel(const double* __restrict__ u_prev, const double* __restrict__ mu,
                         const double* __restrict__ ax_u, const double* __restrict__ ay_u,
                         const uint8_t* __restrict__ phi, double dt, double ikx, double iky,
                         double* __restrict__ lam_prev, double* __restrict__ grad_src, double* grad_k, size_t N,
                         double* partials, SolverState* st) {
  __shared__ double red[32];
  double sx = 0.0, sy = 0.0;
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x) {
    const double m = mu[p];
    const bool inside = !phi[p];
    const double up = u_prev[p];
    lam_prev[p] = inside ? m + dt * (1.0 - 3.0 * up * up) * m : m;
    if (grad_src && inside) grad_src[p] += dt * m;
    sx += m * ax_u[p];
    sy += m * ay_u[p];
  }
  const int G = gridDim.x;
  const double bx = block_sum(sx, red);
  const double by = block_sum(sy, red);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = bx;
    partials[G + blockIdx.x] = by;
  }
  if (arrive_last(&st->counter, G)) {
    const double tx = sum_partials(partials, G, red);
    const double ty = sum_partials(partials + G, G, red);
    if (threadIdx.x == 0) {
      grad_k[0] += tx * ikx;
      grad_k[1] += ty * iky;
    }
  }
}

// beta = ||v||, then the restart decision (left-preconditioned GMRES, whose
// residual is P^-1 (b - M x) and so is formed by separate kernels).
__global__ void __launch_bounds__(kBlock) restart_norm_kernel(const double* __restrict__ v, size_t N,
                                                              double* partials, SolverState* st, const int* gate) {
  if (closed(gate)) return;
  __shared__ double red[32];
  double acc = 0.0;
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x) {
    const double a = v[p];
    acc += a * a;
  }
  const double bs = block_sum(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = bs;
  if (arrive_last(&st->counter, gridDim.x)) {
    const double tot = sum_partials(partials, gridDim.x, red);
    if (threadIdx.x == 0) restart_prep(st, sqrt(tot));
  }
}

// x <- x + sum_i y_i v_i = x + sum_i (y_i s_i) V_i (left-preconditioned GMRES).
__global__ void __launch_bounds__(kBlock) xupdate_v_kernel(double* __restrict__ x, const double* __restrict__ V,
                                                           size_t N, SolverState* st) {
  if (closed(&st->run_cycle)) return;
  const int J = st->jlast;
  if (J == 0) return;
  __shared__ double y[kMaxRestart];
  for (int i = threadIdx.x; i < J; i += blockDim.x) y[i] = st->y[i] * st->s[i];
  __syncthreads();
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x) {
    double v = x[p];
    for (int i = 0; i < J; ++i) v += y[i] * V[(size_t)i * N + p];
    x[p] = v;
  }
}

// ---- launchers --------------------------------------------------------------
void launch_init_state(SolverState* st, int m, int max_iter, double tol, cudaStream_t s) {
  init_state_kernel<<<1, 1, 0, s>>>(st, m, max_iter, tol);
}
void launch_mask_to_phi(const uint8_t* in_omega, uint8_t* phi, size_t N, cudaStream_t s) {
  mask_to_phi_kernel<<<vec_grid(N), kBlock, 0, s>>>(in_omega, phi, N);
}
void launch_rhs(const double* u, const double* uu, const double* src, const uint8_t* phi, double dt, double* b,
                double* x0, size_t N, double* partials, SolverState* st, cudaStream_t s) {
  rhs_kernel<<<vec_grid(N), kBlock, 0, s>>>(u, uu, src, phi, dt, b, x0, N, partials, st);
}
void launch_norm_b(const double* b, size_t N, double* partials, SolverState* st, cudaStream_t s) {
  norm_b_kernel<<<vec_grid(N), kBlock, 0, s>>>(b, N, partials, st);
}
// Gram-Schmidt grid: one full wave of resident blocks, but no more blocks
// than give every thread eight 16-byte packs (small vectors: the block and
// grid reductions would outweigh the loads).
static int wave_grid(int per_sm, size_t N) {
  const int g = kNumSMs * per_sm;
  size_t c = (N + kBlock * 8 - 1) / (kBlock * 8);
  const int cap = c < 1 ? 1 : (int)c;
  return g < cap ? g : cap;
}
template <typename K>
static int resident_blocks(K kernel) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, kBlock, 0) != cudaSuccess || b < 1) b = 1;
  return b;
}

// Vectors per chunk for the j+1 basis vectors: 2 or 4 while that is enough
// (the kernels then take 4 or 2 packs per round), else 8.
static int dot_chunk(int j) { return j + 1 <= 2 ? 2 : j + 1 <= 4 ? 4 : kDotChunk; }

template <typename Tv, int VEC, int CH>
static dim3 multidot_grid(size_t N, int j) {
  static const int per_sm = resident_blocks(multidot_kernel<Tv, VEC, CH>);
  // the chunks share one wave: each takes 1/chunks of the resident blocks
  const int chunks = (j + 1 + CH - 1) / CH;
  const int gx = wave_grid(per_sm, N / VEC);
  return dim3(gx / chunks > kNumSMs ? gx / chunks : (gx < kNumSMs ? gx : kNumSMs), chunks);
}
template <typename Tv, int VEC, int CH>
static void launch_multidot_t(const Tv* V, size_t N, int j, int accumulate, double* partials, SolverState* st,
                              cudaStream_t s) {
  multidot_kernel<Tv, VEC, CH><<<multidot_grid<Tv, VEC, CH>(N, j), kBlock, 0, s>>>(V, N, j, accumulate, partials, st);
}
// 16-byte accesses when every basis vector is 16-byte aligned, else one element.
template <typename Tv>
void launch_multidot(const Tv* V, size_t N, int j, int accumulate, double* partials, SolverState* st,
                     cudaStream_t s) {
  constexpr int VEC = 16 / sizeof(Tv);
  const int ch = dot_chunk(j);
  if (N % VEC == 0) {
    if (ch == 2) launch_multidot_t<Tv, VEC, 2>(V, N, j, accumulate, partials, st, s);
    else if (ch == 4) launch_multidot_t<Tv, VEC, 4>(V, N, j, accumulate, partials, st, s);
    else launch_multidot_t<Tv, VEC, kDotChunk>(V, N, j, accumulate, partials, st, s);
  } else {
    if (ch == 2) launch_multidot_t<Tv, 1, 2>(V, N, j, accumulate, partials, st, s);
    else if (ch == 4) launch_multidot_t<Tv, 1, 4>(V, N, j, accumulate, partials, st, s);
    else launch_multidot_t<Tv, 1, kDotChunk>(V, N, j, accumulate, partials, st, s);
  }
}
template <typename Tv, int VEC, int CH>
static int update_grid(size_t N) {
  static const int per_sm = resident_blocks(update_kernel<Tv, VEC, CH>);
  return wave_grid(per_sm, N / VEC);
}
template <typename Tv, int VEC, int CH>
static void launch_update_t(Tv* V, size_t N, int j, int final_pass, double* partials, SolverState* st,
                            cudaStream_t s, const Bf16Out& bo) {
  update_kernel<Tv, VEC, CH><<<update_grid<Tv, VEC, CH>(N), kBlock, 0, s>>>(V, N, j, final_pass, partials, st, bo);
}
template <typename Tv>
void launch_update(Tv* V, size_t N, int j, int final_pass, double* partials, SolverState* st, cudaStream_t s,
                   const Bf16Out* bo) {
  constexpr int VEC = 16 / sizeof(Tv);
  const Bf16Out none{nullptr, nullptr, 1, 0, 0};
  const int ch = dot_chunk(j);
  if (N % VEC == 0) {
    const Bf16Out& b = bo ? *bo : none;
    if (ch == 2) launch_update_t<Tv, VEC, 2>(V, N, j, final_pass, partials, st, s, b);
    else if (ch == 4) launch_update_t<Tv, VEC, 4>(V, N, j, final_pass, partials, st, s, b);
    else launch_update_t<Tv, VEC, kDotChunk>(V, N, j, final_pass, partials, st, s, b);
  } else {  // (the BF16 copy is only taken with 16-byte packs)
    if (ch == 2) launch_update_t<Tv, 1, 2>(V, N, j, final_pass, partials, st, s, none);
    else if (ch == 4) launch_update_t<Tv, 1, 4>(V, N, j, final_pass, partials, st, s, none);
    else launch_update_t<Tv, 1, kDotChunk>(V, N, j, final_pass, partials, st, s, none);
  }
}
template void launch_multidot<double>(const double*, size_t, int, int, double*, SolverState*, cudaStream_t);
template void launch_multidot<df>(const df*, size_t, int, int, double*, SolverState*, cudaStream_t);
template void launch_update<double>(double*, size_t, int, int, double*, SolverState*, cudaStream_t,
                                    const Bf16Out*);
template void launch_update<df>(df*, size_t, int, int, double*, SolverState*, cudaStream_t, const Bf16Out*);
template void launch_multidot<float>(const float*, size_t, int, int, double*, SolverState*, cudaStream_t);
template void launch_update<float>(float*, size_t, int, int, double*, SolverState*, cudaStream_t,
                                   const Bf16Out*);
void launch_solve_y(SolverState* st, cudaStream_t s) { solve_y_kernel<<<1, 32, 0, s>>>(st); }
template <typename Tz>
void launch_xupdate(double* x, const Tz* Z, size_t N, SolverState* st, cudaStream_t s) {
  constexpr int VEC = 16 / sizeof(Tz);
  if (N % VEC == 0) xupdate_kernel<Tz, VEC><<<vec_grid(N / VEC), kBlock, 0, s>>>(x, Z, N, st);
  else xupdate_kernel<Tz, 1><<<vec_grid(N), kBlock, 0, s>>>(x, Z, N, st);
}
template void launch_xupdate<double>(double*, const double*, size_t, SolverState*, cudaStream_t);
template void launch_xupdate<float>(double*, const float*, size_t, SolverState*, cudaStream_t);
void launch_adjoint_accum(const double* u_prev, const double* mu, const double* ax_u, const double* ay_u,
                          const uint8_t* phi, double dt, double ikx, double iky, double* lam_prev,
                          double* grad_src, double* grad_k, size_t N, double* partials, SolverState* st,
                          cudaStream_t s) {
  adjoint_accum_kernel<<<vec_grid(N), kBlock, 0, s>>>(u_prev, mu, ax_u, ay_u, phi, dt, ikx, iky, lam_prev,
                                                      grad_src, grad_k, N, partials, st);
}
void launch_restart_norm(const double* v, size_t N, double* partials, SolverState* st, const int* gate,
                         cudaStream_t s) {
  restart_norm_kernel<<<vec_grid(N), kBlock, 0, s>>>(v, N, partials, st, gate);
}
void launch_xupdate_v(double* x, const double* V, size_t N, SolverState* st, cudaStream_t s) {
  xupdate_v_kernel<<<vec_grid(N), kBlock, 0, s>>>(x, V, N, st);
}
void launch_loop_cond(cudaGraphConditionalHandle h, SolverState* st, cudaStream_t s) {
  loop_cond_kernel<<<1, 1, 0, s>>>(h, st);
}
void launch_finalize(double* x, size_t N, SolverState* st, cudaStream_t s) {
  finalize_kernel<<<vec_grid(N), kBlock, 0, s>>>(x, N, st);
}

template <typename Tv, typename Tz>
void launch_scale_copy(const Tv* v, const double* scale, Tz* z, size_t N, const int* gate, cudaStream_t s) {
  scale_copy_kernel<Tv, Tz><<<vec_grid(N), kBlock, 0, s>>>(v, scale, z, N, gate);
}
template void launch_scale_copy<double, double>(const double*, const double*, double*, size_t, const int*,
                                                cudaStream_t);
template void launch_scale_copy<double, float>(const double*, const double*, float*, size_t, const int*,
                                               cudaStream_t);
template void launch_scale_copy<df, double>(const df*, const double*, double*, size_t, const int*, cudaStream_t);
template void launch_scale_copy<df, float>(const df*, const double*, float*, size_t, const int*, cudaStream_t);
template void launch_scale_copy<float, double>(const float*, const double*, double*, size_t, const int*,
                                               cudaStream_t);
template void launch_scale_copy<float, float>(const float*, const double*, float*, size_t, const int*,
                                              cudaStream_t);

// ---- multi-instance launches (batched form) ---------------------------------
// A fixed grid loops over the active virtual blocks (active prefix staged in
// shared memory); each virtual block runs the single-instance body on its
// instance's own virtual grid, so the results are bit-identical to single
// solves.

__global__ void init_multi_kernel(const BatchInst* __restrict__ bi, int count, int m, int max_iter, double tol) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) init_state_body(bi[i].st, m, max_iter, tol);
}
__global__ void __launch_bounds__(kBlock) rhs_multi_kernel(const BatchInst* __restrict__ bi,
                                                           const int* __restrict__ prefix,
                                                           const int* __restrict__ active, int count, int later) {
  multi_loop(bi, prefix, active, count, [&](const BatchInst& I, int lb, int nb) {
    rhs_body(I.u_prev, later ? I.u_pp : nullptr, I.src, I.phi, I.dt, I.b, I.x, I.N, I.partials, I.st, lb, nb);
  });
}
// 64 registers (four blocks per SM), as the single-instance kernels take by
// themselves: the virtual-block loop and the two pack widths would otherwise
// raise them and halve the resident warps of these FP64-pipe-bound loops.
template <typename Tv, int CH>
__global__ void __launch_bounds__(kBlock, 4) multidot_multi_kernel(const BatchInst* __restrict__ bi,
                                                                const int* __restrict__ prefix,
                                                                const int* __restrict__ active, int count, int j,
                                                                int accumulate, int chunks, int* sched) {
  multi_loop(bi, prefix, active, count, [&](const BatchInst& I, int lb, int nb) {
    constexpr int VEC = 16 / sizeof(Tv);
    const int gx = nb / chunks;
    const Tv* V = reinterpret_cast<const Tv*>(I.V);
    if (I.N % VEC == 0)
      multidot_body<Tv, VEC, CH>(V, I.N, j, accumulate, I.partials, I.st, lb % gx, gx, lb / gx, chunks);
    else
      multidot_body<Tv, 1, CH>(V, I.N, j, accumulate, I.partials, I.st, lb % gx, gx, lb / gx, chunks);
  }, sched);
}
template <typename Tv, int CH>
__global__ void __launch_bounds__(kBlock, 4) update_multi_kernel(const BatchInst* __restrict__ bi,
                                                              const int* __restrict__ prefix,
                                                              const int* __restrict__ active, int count, int j,
                                                              int final_pass, int write_a0, int* sched) {
  multi_loop(bi, prefix, active, count, [&](const BatchInst& I, int lb, int nb) {
    constexpr int VEC = 16 / sizeof(Tv);
    const Bf16Out none{nullptr, nullptr, 1, 0, 0};
    Tv* V = reinterpret_cast<Tv*>(I.V);
    if (I.N % VEC == 0) {  // (a0_fused implies N % VEC == 0)
      const bool wr = write_a0 && I.a0_fused;
      const Bf16Out bo{wr ? static_cast<__nv_bfloat16*>(I.a0) : nullptr,
                       wr ? static_cast<__nv_bfloat16*>(I.a0_lo) : nullptr, wr ? I.n1 : 1, I.a0_ld, I.a0_hk};
      update_body<Tv, VEC, CH>(V, I.N, j, final_pass, I.partials, I.st, bo, lb, nb);
    }
    else update_body<Tv, 1, CH>(V, I.N, j, final_pass, I.partials, I.st, none, lb, nb);
  }, sched);
}
__global__ void solve_y_multi_kernel(const BatchInst* __restrict__ bi) { solve_y_body(bi[blockIdx.x].st); }
template <typename Tz>
__global__ void __launch_bounds__(kBlock) xupdate_multi_kernel(const BatchInst* __restrict__ bi,
                                                               const int* __restrict__ prefix,
                                                               const int* __restrict__ active, int count) {
  multi_loop(bi, prefix, active, count, [&](const BatchInst& I, int lb, int nb) {
    constexpr int VEC = 16 / sizeof(Tz);
    const Tz* Z = static_cast<const Tz*>(I.Z);
    if (I.N % VEC == 0) xupdate_body<Tz, VEC>(I.x, Z, I.N, I.st, lb, nb);
    else xupdate_body<Tz, 1>(I.x, Z, I.N, I.st, lb, nb);
  });
}
// End of a batch step: x = 0 where the right side was zero, then the march
// ring moves on (u^{k-2} <- u^{k-1}, u^{k-1} <- u^k).
__global__ void __launch_bounds__(kBlock) finish_rotate_multi_kernel(const BatchInst* __restrict__ bi,
                                                                     const int* __restrict__ prefix,
                                                                     const int* __restrict__ active, int count) {
  multi_loop(bi, prefix, active, count, [&](const BatchInst& I, int lb, int nb) {
    const bool zero = I.st->zero_solution != 0;
    for (size_t p = lb * (size_t)blockDim.x + threadIdx.x; p < I.N; p += (size_t)nb * blockDim.x) {
      const double xv = zero ? 0.0 : I.x[p];
      I.x[p] = xv;
      I.u_pp[p] = I.u_prev[p];
      I.u_prev[p] = xv;
    }
  });
}
// Condition of the batch's device-side loop over FGMRES cycles: go on while
// any instance runs; each running instance counts the cycle and is stopped
// (RSFDE_ENOTCONV) past max_iter + 2 cycles, as in the single-instance loop.
__global__ void loop_cond_multi_kernel(cudaGraphConditionalHandle h, const BatchInst* __restrict__ bi, int count,
                                       int* runs) {
  int go = 0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    SolverState* st = bi[i].st;
    int g = st->run_cycle;
    if (g) {
      st->body_runs += 1;
      st->total_body_runs += 1;
      if (st->body_runs > st->max_iter + 2) {
        st->status = RSFDE_ENOTCONV;
        st->run_cycle = 0;
        st->run_iter = 0;
        g = 0;
      }
    }
    go |= g;
  }
  go = __syncthreads_or(go);
  if (threadIdx.x == 0) {
    *runs += 1;
    cudaGraphSetConditional(h, go ? 1u : 0u);
  }
}
// Active prefixes (one block; count <= kMaxBatchMulti): an inclusive scan per
// family of the instances' virtual-grid sizes, zero where the gate is closed.
__global__ void __launch_bounds__(kMaxBatchMulti) compact_multi_kernel(const BatchInst* __restrict__ bi, int count,
                                                                       int use_cycle, CompactArgs a) {
  __shared__ int sc[kMaxBatchMulti];
  const int i = threadIdx.x;
  int open = 0;
  if (i < count) {
    const SolverState* st = bi[i].st;
    open = use_cycle ? *(volatile const int*)&st->run_cycle : *(volatile const int*)&st->run_iter;
  }
  for (int f = 0; f < a.nfam; ++f) {
    const int v = (i < count && open) ? __ldg(a.prefix[f] + i + 1) - __ldg(a.prefix[f] + i) : 0;
    sc[i] = v;
    __syncthreads();
    for (int d = 1; d < kMaxBatchMulti; d <<= 1) {  // Hillis-Steele inclusive scan
      const int t = i >= d ? sc[i - d] : 0;
      __syncthreads();
      sc[i] += t;
      __syncthreads();
    }
    if (i < count) a.active[f][i] = sc[i] - v;
    if (i == count - 1) a.active[f][count] = sc[i];
    __syncthreads();
  }
}

// 1 in *out while any instance of the batch still runs a cycle (direct launches).
__global__ void any_running_multi_kernel(const BatchInst* __restrict__ bi, int count, int* out) {
  int go = 0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) go |= bi[i].st->run_cycle;
  go = __syncthreads_or(go);
  if (threadIdx.x == 0) *out = go;
}
void launch_any_running_multi(const BatchInst* bi, int count, int* out, cudaStream_t s) {
  any_running_multi_kernel<<<1, 256, 0, s>>>(bi, count, out);
}

void launch_compact_multi(const BatchInst* bi, int count, int use_cycle, const CompactArgs& a, cudaStream_t s) {
  compact_multi_kernel<<<1, kMaxBatchMulti, 0, s>>>(bi, count, use_cycle, a);
}
void launch_init_multi(const BatchInst* bi, int count, int m, int max_iter, double tol, cudaStream_t s) {
  init_multi_kernel<<<(count + 127) / 128, 128, 0, s>>>(bi, count, m, max_iter, tol);
}
void launch_rhs_multi(const BatchInst* bi, const MultiGrid& g, int later, cudaStream_t s) {
  static const int grid = multi_launch_grid(rhs_multi_kernel, kBlock, 0, 1 << 30);
  rhs_multi_kernel<<<g.total < grid ? g.total : grid, kBlock, 0, s>>>(bi, g.prefix, g.active, g.count, later);
}
template <typename Tv, int CH>
static void launch_multidot_multi_t(const BatchInst* bi, const MultiGrid& g, int j, int accumulate, cudaStream_t s) {
  static const int grid = multi_launch_grid(multidot_multi_kernel<Tv, CH>, kBlock, 0, 1 << 30);
  multidot_multi_kernel<Tv, CH><<<g.total < grid ? g.total : grid, kBlock, 0, s>>>(
      bi, g.prefix, g.active, g.count, j, accumulate, (j + CH) / CH, g.sched);
}
template <typename Tv>
void launch_multidot_multi(const BatchInst* bi, const MultiGrid& g, int j, int accumulate, cudaStream_t s) {
  const int ch = dot_chunk(j);
  if (ch == 2) launch_multidot_multi_t<Tv, 2>(bi, g, j, accumulate, s);
  else if (ch == 4) launch_multidot_multi_t<Tv, 4>(bi, g, j, accumulate, s);
  else launch_multidot_multi_t<Tv, kDotChunk>(bi, g, j, accumulate, s);
}
template <typename Tv, int CH>
static void launch_update_multi_t(const BatchInst* bi, const MultiGrid& g, int j, int final_pass, int write_a0,
                                  cudaStream_t s) {
  static const int grid = multi_launch_grid(update_multi_kernel<Tv, CH>, kBlock, 0, 1 << 30);
  update_multi_kernel<Tv, CH><<<g.total < grid ? g.total : grid, kBlock, 0, s>>>(bi, g.prefix, g.active, g.count, j,
                                                                               final_pass, write_a0, g.sched);
}
template <typename Tv>
void launch_update_multi(const BatchInst* bi, const MultiGrid& g, int j, int final_pass, int write_a0, cudaStream_t s) {
  const int ch = dot_chunk(j);
  if (ch == 2) launch_update_multi_t<Tv, 2>(bi, g, j, final_pass, write_a0, s);
  else if (ch == 4) launch_update_multi_t<Tv, 4>(bi, g, j, final_pass, write_a0, s);
  else launch_update_multi_t<Tv, kDotChunk>(bi, g, j, final_pass, write_a0, s);
}
void launch_solve_y_multi(const BatchInst* bi, int count, cudaStream_t s) {
  solve_y_multi_kernel<<<count, 32, 0, s>>>(bi);
}
template <typename Tz>
void launch_xupdate_multi(const BatchInst* bi, const MultiGrid& g, cudaStream_t s) {
  static const int grid = multi_launch_grid(xupdate_multi_kernel<Tz>, kBlock, 0, 1 << 30);
  xupdate_multi_kernel<Tz><<<g.total < grid ? g.total : grid, kBlock, 0, s>>>(bi, g.prefix, g.active, g.count);
}
void launch_finish_rotate_multi(const BatchInst* bi, const MultiGrid& g, cudaStream_t s) {
  static const int grid = multi_launch_grid(finish_rotate_multi_kernel, kBlock, 0, 1 << 30);
  finish_rotate_multi_kernel<<<g.total < grid ? g.total : grid, kBlock, 0, s>>>(bi, g.prefix, g.active, g.count);
}
void launch_loop_cond_multi(cudaGraphConditionalHandle h, const BatchInst* bi, int count, int* runs,
                            cudaStream_t s) {
  loop_cond_multi_kernel<<<1, 256, 0, s>>>(h, bi, count, runs);
}

// The grids of the single-instance launches, for the multi-instance prefixes.
template <typename Tv>
int multidot_blocks(size_t N, int j) {
  constexpr int VEC = 16 / sizeof(Tv);
  const int ch = dot_chunk(j);
  dim3 g;
  if (N % VEC == 0)
    g = ch == 2 ? multidot_grid<Tv, VEC, 2>(N, j) : ch == 4 ? multidot_grid<Tv, VEC, 4>(N, j)
                                                             : multidot_grid<Tv, VEC, kDotChunk>(N, j);
  else
    g = ch == 2 ? multidot_grid<Tv, 1, 2>(N, j) : ch == 4 ? multidot_grid<Tv, 1, 4>(N, j)
                                                           : multidot_grid<Tv, 1, kDotChunk>(N, j);
  return (int)(g.x * g.y);
}
template <typename Tv>
int update_blocks(size_t N, int j) {
  constexpr int VEC = 16 / sizeof(Tv);
  const int ch = dot_chunk(j);
  if (N % VEC == 0)
    return ch == 2 ? update_grid<Tv, VEC, 2>(N) : ch == 4 ? update_grid<Tv, VEC, 4>(N) : update_grid<Tv, VEC, kDotChunk>(N);
  return ch == 2 ? update_grid<Tv, 1, 2>(N) : ch == 4 ? update_grid<Tv, 1, 4>(N) : update_grid<Tv, 1, kDotChunk>(N);
}
int xupdate_blocks(size_t N, int zbytes) {
  const size_t VEC = 16 / (size_t)zbytes;
  return N % VEC == 0 ? vec_grid(N / VEC) : vec_grid(N);
}
#define RSFDE_GS_MULTI(Tv)                                                                              \
  template void launch_multidot_multi<Tv>(const BatchInst*, const MultiGrid&, int, int, cudaStream_t); \
  template void launch_update_multi<Tv>(const BatchInst*, const MultiGrid&, int, int, int, cudaStream_t);   \
  template int multidot_blocks<Tv>(size_t, int);                                                       \
  template int update_blocks<Tv>(size_t, int);
RSFDE_GS_MULTI(double)
RSFDE_GS_MULTI(float)
#undef RSFDE_GS_MULTI
template void launch_xupdate_multi<float>(const BatchInst*, const MultiGrid&, cudaStream_t);

}  // namespace rsfde
