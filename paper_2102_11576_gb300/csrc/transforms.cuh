// transforms.cuh -- the operator M (Eq. 2.14-2.17) and the preconditioner
// P-hat^-1 (Eq. 4.6) as register-Stockham FFT kernels for sm_103a.
//
// Grid functions are x-fastest (u[j*n1 + i]).  A "vector" is a row (x
// direction, contiguous) or a column (y direction, stride n1).  Each vector
// (or pair of vectors) is transformed by a group of L/16 threads (fft16.cuh);
// a block runs F groups.  Row kernels map a group's threads to consecutive
// positions (coalesced rows); column kernels interleave the F groups across
// the lanes of a warp so each access touches F (or 2F) adjacent columns.
//
//  * Arithmetic: T = double, float, or df (double-FP32, df.cuh).
//  * Toeplitz product along an axis: two real vectors are packed as the real
//    and imaginary parts of one complex sequence (the circulant spectrum is
//    real because the Toeplitz matrix of Eq. 2.16 is symmetric), zero padded
//    to L >= 2n-1, transformed, scaled by the spectrum and transformed back.
//  * Sine transform S_n (Section 4.1): with c_k = exp(i pi k^2/(2(n+1))) and
//    jk = (j^2 + k^2 - (k-j)^2)/2,  (S x)_k = sqrt(2/(n+1)) Im(c_k sum_j x_j c_j conj(c_{k-j})),
//    a convolution of length L >= 2n-1 (Bluestein).
//  * P-hat^-1 v = (I-Phi) S (I - Lx - Ly)^-1 S v + Phi S ((1+dt/eta) I - Lx - Ly)^-1 S v
//    (S = S_{n2} (x) S_{n1}; proof of Lemma 4.2) in three passes: rows S_x;
//    columns S_y, the two spectral divides and both inverse S_y; rows S_x
//    of both channels with the masked combine.
#pragma once
#include <type_traits>

#include "common.cuh"
#include "df.cuh"
#include "fft16.cuh"
#include "internal.h"

// Thread cap of one block of the FP32 transform kernels (their register
// budget is 65536 / cap per thread); FP64 and double-FP32 blocks (8-byte
// reals) are capped at 512.
#ifndef RSFDE_FP32_THREADS
#define RSFDE_FP32_THREADS 1024
#endif

namespace rsfde {

template <typename T>
__device__ __forceinline__ bool gate_closed(const int* gate) {
  return gate != nullptr && *(volatile const int*)gate == 0;
}

// Read-only loads of table entries, including double-FP32 pairs.
template <typename T>
__device__ __forceinline__ T ldg_t(const T* p) {
  return __ldg(p);
}
template <>
__device__ __forceinline__ df ldg_t<df>(const df* p) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return {v.x, v.y};
}
template <typename T>
__device__ __forceinline__ cx<T> ldc(const T* p, int k) {
  return {ldg_t(p + 2 * k), ldg_t(p + 2 * k + 1)};
}

// Thread geometry of one block: F groups of G = L/16 threads.
struct GroupIdx {
  int g, t;
};
template <bool COLS>
__device__ __forceinline__ GroupIdx group_idx(int G, int F) {
  // rows: each group's threads consecutive; columns: groups interleaved over lanes
  if (COLS) return {(int)threadIdx.x & (F - 1), (int)threadIdx.x / F};
  return {(int)threadIdx.x / G, (int)threadIdx.x & (G - 1)};
}

// Address of element `pos` of vector `vec`.
template <bool COLS>
__device__ __forceinline__ size_t vaddr(int vec, int pos, int n1) {
  return COLS ? (size_t)pos * n1 + vec : (size_t)vec * n1 + pos;
}


// Bluestein convolution of the 16 chirped values in v: on return v holds
// sum_j a_j conj(c_{k-j}) at the thread's positions (natural order).
template <typename T>
__device__ __forceinline__ void bluestein(cx<T>* v, cx<T>* buf, int t, const AxisTables<T>& ax) {
  const int L = ax.L, Lq = L >> 4;
  const cx<T>* tw = reinterpret_cast<const cx<T>*>(ax.tw);
  fft16_forward<T>(v, buf, t, L, ax.log2L, tw);
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = c_mul(v[k], ldc(ax.bspec, t + k * Lq));  // full spectrum
  fft16_inverse<T>(v, buf, t, L, ax.log2L, tw);
}

// scale * x in the arithmetic type T: FP64 vectors are scaled in FP64 before
// rounding; FP32 and double-FP32 vectors feeding an FP32 transform are scaled
// in FP32, with no FP64 instruction.
template <typename T>
__device__ __forceinline__ T scaled_load(double sc, float, double x) {
  return cvt<T>(sc * x);
}
template <typename T>
__device__ __forceinline__ T scaled_load(double sc, float scf, df x);
template <>
__device__ __forceinline__ float scaled_load<float>(double, float scf, df x) {
  return __fmul_rn(scf, cvt<float>(x));
}
template <>
__device__ __forceinline__ double scaled_load<double>(double sc, float, df x) {
  return sc * double(x);
}
template <>
__device__ __forceinline__ df scaled_load<df>(double sc, float, df x) {
  return df(sc) * x;
}
template <typename T>
__device__ __forceinline__ T scaled_load(double sc, float scf, float x);
template <>
__device__ __forceinline__ float scaled_load<float>(double, float scf, float x) {
  return __fmul_rn(scf, x);
}
template <>
__device__ __forceinline__ double scaled_load<double>(double sc, float, float x) {
  return sc * (double)x;
}
template <>
__device__ __forceinline__ df scaled_load<df>(double sc, float, float x) {
  return df(sc) * df(x, 0.0f);
}

// Im(c_out[pos] * y)
template <typename T>
__device__ __forceinline__ T dst_out(const AxisTables<T>& ax, int pos, cx<T> y) {
  const cx<T> c = ldc(ax.chirp_out, pos);
  return c.r * y.i + c.i * y.r;
}

// Two adjacent elements as one access (8 or 16 bytes; the address is aligned
// to the pair's size).
template <typename X>
struct Pair {
  X x, y;
};
template <typename X>
__device__ __forceinline__ Pair<X> ld_pair(const X* p) {
  if constexpr (std::is_same<X, float>::value) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    return {t.x, t.y};
  } else if constexpr (std::is_same<X, double>::value) {
    const double2 t = *reinterpret_cast<const double2*>(p);
    return {t.x, t.y};
  } else if constexpr (std::is_same<X, df>::value) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    return {df(t.x, t.y), df(t.z, t.w)};
  } else {  // uint8_t
    const uchar2 t = *reinterpret_cast<const uchar2*>(p);
    return {t.x, t.y};
  }
}
template <typename X>
__device__ __forceinline__ void st_pair(X* p, X a, X b) {
  if constexpr (std::is_same<X, float>::value) *reinterpret_cast<float2*>(p) = make_float2(a, b);
  else if constexpr (std::is_same<X, double>::value) *reinterpret_cast<double2*>(p) = make_double2(a, b);
  else *reinterpret_cast<float4*>(p) = make_float4(a.hi, a.lo, b.hi, b.lo);
}

// ---------------------------------------------------------------------------
// Toeplitz product along rows (COLS = false) or columns (COLS = true), two
// vectors per group.  The row pass writes the scratch tmpx in the arithmetic
// type T:
//   MODE_RAW:      tmpx = A_x z
//   other modes:   tmpx = z - A_x z + (dt/eta) phi z   (every term of M z but
//                  A_y z, so the column pass reads one array besides z's
//                  column pairs)
// Column epilogues:
//   MODE_RAW:        out = A_y z
//   MODE_APPLY:      out = tmpx - A_y z  (= M z)
//   MODE_RESID_ONLY: out = b - (tmpx - A_y z)
//   MODE_RESIDUAL:   out = b - (tmpx - A_y z), ||out||^2 reduced, and the
//                    last block restarts the solver.
//
// The residual's ||r||^2 is summed per column pair -- each thread's terms in
// a fixed order, then the group's threads by a fixed tree over t, then the
// pairs in order by one warp -- so the value depends only on the grid, not on
// how many pairs a block holds or how many blocks there are (single and
// batched launches give identical bits).
//
// The body takes its block index and block count explicitly: a kernel
// launch passes blockIdx.x and gridDim.x, a batched launch the instance's
// own block of its virtual grid.
template <typename T, typename Tin, int MODE, bool COLS, typename Tout, int LG = 0>
__device__ __forceinline__ void toeplitz_body(const Tin* __restrict__ z, T* __restrict__ tmpx,
                                              const uint8_t* __restrict__ phi, double pen,
                                              const double* __restrict__ b, Tout* __restrict__ out, int n1, int n2,
                                              const AxisTables<T>& ax, int F, int gstride, const int* gate,
                                              double* partials, SolverState* st, int bid, int nblk) {
  if (gate_closed<T>(gate)) return;
  const T tpen = cvt<T>(pen);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = LG ? (1 << LG) : ax.L, Lq = L >> 4, G = Lq;
  const GroupIdx gi = group_idx<COLS>(G, F);
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw) + (size_t)gi.g * gstride;
  const int nvec = COLS ? n1 : n2, len = COLS ? n2 : n1;
  const int npairs = (nvec + 1) >> 1;
  const int ngroups = (npairs + F - 1) / F;
  // Column passes with even n1: the pair of columns a, a+1 a group transforms
  // is adjacent in memory, so z, A_x z, the mask, b and the output move as
  // pairs (the FP32 and double-FP32 operators on an FP32 z, whatever basis
  // they write, and the double-FP32 true residual).
  constexpr bool kPairIO =
      COLS && ((MODE == MODE_APPLY && !std::is_same<T, double>::value && std::is_same<Tin, float>::value) ||
               (MODE == MODE_RESIDUAL && std::is_same<T, df>::value && std::is_same<Tin, double>::value));
  const bool pair_io = kPairIO && (n1 & 1) == 0;
  for (int grp = bid; grp < ngroups; grp += nblk) {
    const int pr = grp * F + gi.g;
    const int a = 2 * pr;
    const bool live = pr < npairs;
    const bool second = a + 1 < nvec;
    double acc = 0.0;  // this thread's part of the pair's ||r||^2
    cx<T> v[16];  // positions >= L/2 are zero (cleared by the forward transform)
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int pos = gi.t + k * Lq;
      T re = T(0), im = T(0);
      if (live && pos < len) {
        if constexpr (kPairIO) {
          if (pair_io) {
            const Pair<Tin> t2 = ld_pair(z + vaddr<COLS>(a, pos, n1));
            re = cvt<T>(t2.x);
            im = cvt<T>(t2.y);
          } else {
            re = cvt<T>(z[vaddr<COLS>(a, pos, n1)]);
            if (second) im = cvt<T>(z[vaddr<COLS>(a + 1, pos, n1)]);
          }
        } else {
          re = cvt<T>(z[vaddr<COLS>(a, pos, n1)]);
          if (second) im = cvt<T>(z[vaddr<COLS>(a + 1, pos, n1)]);
        }
      }
      v[k] = {re, im};
    }
    const cx<T>* tw = reinterpret_cast<const cx<T>*>(ax.tw);
    fft16_forward<T, LG>(v, buf, gi.t, L, ax.log2L, tw);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const T sg = ldg_t(ax.sigma + gi.t + k * Lq);
      v[k].r *= sg;
      v[k].i *= sg;
    }
    fft16_inverse<T, LG>(v, buf, gi.t, L, ax.log2L, tw);
    if constexpr (kPairIO) {
      if (pair_io) {
        if (live) {
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int pos = gi.t + k * Lq;
            if (pos >= len) continue;
            const size_t p = vaddr<COLS>(a, pos, n1);
            const Pair<T> t2 = ld_pair(tmpx + p);
            const T w0 = t2.x - v[k].r, w1 = t2.y - v[k].i;
            if constexpr (MODE == MODE_APPLY) {
              st_pair(out + p, cvt<Tout>(w0), cvt<Tout>(w1));
            } else {
              const Pair<double> b2 = ld_pair(b + p);
              const double r0 = b2.x - cvt<double>(w0), r1 = b2.y - cvt<double>(w1);
              st_pair(out + p, cvt<Tout>(r0), cvt<Tout>(r1));
              acc += r0 * r0;
              acc += r1 * r1;
            }
          }
        }
      }
    }
    if (!pair_io && live) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int pos = gi.t + k * Lq;
        if (pos >= len) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (h == 1 && !second) break;
          const size_t p = vaddr<COLS>(a + h, pos, n1);
          const T az = h ? v[k].i : v[k].r;
          if (!COLS) {
            if (MODE == MODE_RAW) {
              tmpx[p] = az;  // A_x z, kept in the arithmetic type T
            } else {
              const T zz = cvt<T>(z[p]);  // (the pass read this row at the start: an L1 or L2 hit)
              T sx = zz - az;
              if (phi[p]) sx = sx + tpen * zz;
              tmpx[p] = sx;
            }
          } else {
            // M z = (z - A_x z + (dt/eta) phi z) - A_y z in T; only the result is rounded to Tout
            const T w = MODE == MODE_RAW ? az : tmpx[p] - az;
            if (MODE == MODE_RAW) {
              out[p] = cvt<Tout>(az);
            } else if (MODE == MODE_APPLY) {
              out[p] = cvt<Tout>(w);
            } else if (MODE == MODE_RESID_ONLY) {
              out[p] = cvt<Tout>(b[p] - cvt<double>(w));
            } else {
              const double r = b[p] - cvt<double>(w);
              out[p] = cvt<Tout>(r);
              acc += r * r;
            }
          }
        }
      }
    }
    if constexpr (MODE == MODE_RESIDUAL) {
      // the group's sum by a fixed tree over t in its own buffer (free now)
      double* gsum = reinterpret_cast<double*>(buf);
      __syncthreads();
      gsum[gi.t] = acc;
      __syncthreads();
      for (int h = G >> 1; h > 0; h >>= 1) {
        if (gi.t < h) gsum[gi.t] += gsum[gi.t + h];
        __syncthreads();
      }
      if (gi.t == 0 && live) partials[pr] = gsum[0];
      __syncthreads();  // the next group's transform reuses the buffer
    }
  }
  if constexpr (MODE == MODE_RESIDUAL) {
    if (arrive_last(&st->counter, nblk)) {
      const double tot = block_sum_fixed(partials, npairs);
      if (threadIdx.x == 0) restart_prep(st, sqrt(tot));
    }
  }
}

template <typename T, typename Tin, int MODE, bool COLS, typename Tout>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 512 : RSFDE_FP32_THREADS)
    toeplitz_kernel(const Tin* __restrict__ z, T* __restrict__ tmpx, const uint8_t* __restrict__ phi,
                    double pen, const double* __restrict__ b, Tout* __restrict__ out, int n1, int n2,
                    AxisTables<T> ax, int F, int gstride, const int* gate, double* partials, SolverState* st) {
  // the FP32 operator at length 4096 (n 1025..2048) compiled apart (the same arithmetic)
  if constexpr (std::is_same<T, float>::value && MODE == MODE_APPLY) {
    if (ax.log2L == 12) {
      toeplitz_body<T, Tin, MODE, COLS, Tout, 12>(z, tmpx, phi, pen, b, out, n1, n2, ax, F, gstride, gate, partials,
                                                  st, blockIdx.x, gridDim.x);
      return;
    }
  }
  toeplitz_body<T, Tin, MODE, COLS, Tout>(z, tmpx, phi, pen, b, out, n1, n2, ax, F, gstride, gate, partials, st,
                                          blockIdx.x, gridDim.x);
}

// Sine transform of every row (COLS = false) or column: out = S (scale * in).
template <typename T, typename Tin, typename Tout, bool COLS>
__device__ __forceinline__ void dst_body(const Tin* __restrict__ in, const double* vscale, Tout* __restrict__ out,
                                         int n1, int n2, const AxisTables<T>& ax, int F, int gstride, const int* gate,
                                         int bid, int nblk) {
  if (gate_closed<T>(gate)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = ax.L, Lq = L >> 4, G = Lq;
  const GroupIdx gi = group_idx<COLS>(G, F);
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw) + (size_t)gi.g * gstride;
  const int nvec = COLS ? n1 : n2, len = COLS ? n2 : n1;
  const double sc = vscale ? *vscale : 1.0;
  const float scf = (float)sc;
  const int ngroups = (nvec + F - 1) / F;
  for (int grp = bid; grp < ngroups; grp += nblk) {
    const int vec = grp * F + gi.g;
    const bool live = vec < nvec;
    cx<T> v[16];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int pos = gi.t + k * Lq;
      cx<T> x = {T(0), T(0)};
      if (live && pos < len) {
        const T xv = scaled_load<T>(sc, scf, in[vaddr<COLS>(vec, pos, n1)]);
        const cx<T> c = ldc(ax.chirp, pos);
        x = {xv * c.r, xv * c.i};
      }
      v[k] = x;
    }
    bluestein<T>(v, buf, gi.t, ax);
    if (live) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int pos = gi.t + k * Lq;
        if (pos < len) out[vaddr<COLS>(vec, pos, n1)] = Tout(dst_out(ax, pos, v[k]));
      }
    }
  }
}

template <typename T, typename Tin, typename Tout, bool COLS>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 512 : RSFDE_FP32_THREADS)
    dst_kernel(const Tin* __restrict__ in, const double* vscale, Tout* __restrict__ out, int n1, int n2,
               AxisTables<T> ax, int F, int gstride, const int* gate) {
  dst_body<T, Tin, Tout, COLS>(in, vscale, out, n1, n2, ax, F, gstride, gate, blockIdx.x, gridDim.x);
}

// Preconditioner, column pass.  For each x-frequency i (a column of T1, the
// rows already sine-transformed): W = S_{n2} T1[:, i];
// T2a[:, i] = S_{n2} (W / (1 - lam_x[i] - lam_y)),
// T2b[:, i] = S_{n2} (W / (1 + dt/eta - lam_x[i] - lam_y)).
template <typename T>
__device__ __forceinline__ void precond_cols_body(const T* __restrict__ T1, T* __restrict__ T2a, T* __restrict__ T2b,
                                                  int n1, int n2, const AxisTables<T>& ay, const T* __restrict__ lamx,
                                                  T pen, int F, int gstride, const int* gate, int bid, int nblk) {
  if (gate_closed<T>(gate)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = ay.L, Lq = L >> 4, G = Lq;
  const GroupIdx gi = group_idx<true>(G, F);
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw) + (size_t)gi.g * gstride;
  const int ngroups = (n1 + F - 1) / F;
  for (int grp = bid; grp < ngroups; grp += nblk) {
    const int col = grp * F + gi.g;
    const bool live = col < n1;
    cx<T> v[16];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int pos = gi.t + k * Lq;
      cx<T> x = {T(0), T(0)};
      if (live && pos < n2) {
        const T xv = T1[(size_t)pos * n1 + col];
        const cx<T> c = ldc(ay.chirp, pos);
        x = {xv * c.r, xv * c.i};
      }
      v[k] = x;
    }
    bluestein<T>(v, buf, gi.t, ay);
    const T lx = live ? lamx[col] : T(0);
    T W[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int pos = gi.t + k * Lq;
      W[k] = (live && pos < n2) ? dst_out(ay, pos, v[k]) / (T(1) - lx - __ldg(ay.lam + pos)) : T(0);
    }
#pragma unroll
    for (int ch = 0; ch < 2; ++ch) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int pos = gi.t + k * Lq;
        cx<T> x = {T(0), T(0)};
        if (live && pos < n2) {
          T w = W[k];
          if (ch == 1) {  // W / (1 + pen - l) = W1 * (1 - l) / (1 + pen - l)
            const T base = T(1) - lx - __ldg(ay.lam + pos);
            w = w * base / (base + pen);
          }
          const cx<T> c = ldc(ay.chirp, pos);
          x = {w * c.r, w * c.i};
        }
        v[k] = x;
      }
      bluestein<T>(v, buf, gi.t, ay);
      if (live) {
        T* dst = ch ? T2b : T2a;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int pos = gi.t + k * Lq;
          if (pos < n2) dst[(size_t)pos * n1 + col] = dst_out(ay, pos, v[k]);
        }
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 512 : RSFDE_FP32_THREADS)
    precond_cols_kernel(const T* __restrict__ T1, T* __restrict__ T2a, T* __restrict__ T2b, int n1, int n2,
                        AxisTables<T> ay, const T* __restrict__ lamx, T pen, int F, int gstride, const int* gate) {
  precond_cols_body<T>(T1, T2a, T2b, n1, n2, ay, lamx, pen, F, gstride, gate, blockIdx.x, gridDim.x);
}

// Preconditioner, final row pass:  z[j, :] = (1 - phi) S_{n1} T2a[j, :] + phi S_{n1} T2b[j, :].
template <typename T, typename Tz>
__device__ __forceinline__ void precond_rows_body(const T* __restrict__ T2a, const T* __restrict__ T2b,
                                                  const uint8_t* __restrict__ phi, Tz* __restrict__ z, int n1, int n2,
                                                  const AxisTables<T>& ax, int F, int gstride, const int* gate,
                                                  int bid, int nblk) {
  if (gate_closed<T>(gate)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = ax.L, Lq = L >> 4, G = Lq;
  const GroupIdx gi = group_idx<false>(G, F);
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw) + (size_t)gi.g * gstride;
  const int ngroups = (n2 + F - 1) / F;
  for (int grp = bid; grp < ngroups; grp += nblk) {
    const int row = grp * F + gi.g;
    const bool live = row < n2;
    T res[8];
#pragma unroll
    for (int ch = 0; ch < 2; ++ch) {
      const T* src = ch ? T2b : T2a;
      cx<T> v[16];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int pos = gi.t + k * Lq;
        cx<T> x = {T(0), T(0)};
        if (live && pos < n1) {
          const T xv = src[(size_t)row * n1 + pos];
          const cx<T> c = ldc(ax.chirp, pos);
          x = {xv * c.r, xv * c.i};
        }
        v[k] = x;
      }
      bluestein<T>(v, buf, gi.t, ax);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int pos = gi.t + k * Lq;
        if (ch == 0) {
          res[k] = (pos < n1) ? dst_out(ax, pos, v[k]) : T(0);
        } else if (live && pos < n1) {
          const size_t p = (size_t)row * n1 + pos;
          if (phi[p]) res[k] = dst_out(ax, pos, v[k]);
        }
      }
    }
    if (live) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int pos = gi.t + k * Lq;
        if (pos < n1) z[(size_t)row * n1 + pos] = Tz(res[k]);
      }
    }
  }
}

template <typename T, typename Tz>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 512 : RSFDE_FP32_THREADS)
    precond_rows_kernel(const T* __restrict__ T2a, const T* __restrict__ T2b, const uint8_t* __restrict__ phi,
                        Tz* __restrict__ z, int n1, int n2, AxisTables<T> ax, int F, int gstride, const int* gate) {
  precond_rows_body<T, Tz>(T2a, T2b, phi, z, n1, n2, ax, F, gstride, gate, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// Launch geometry: G = L/16 threads per group; F groups per block, the
// largest power of two within the thread cap (512 FP64 / 1024 FP32), the
// shared-memory budget and the work available (at least ~2 blocks per SM).
// Complex values per 128-byte shared-memory phase: 16 (FP32), 8 (FP64).
template <typename T>
__host__ __device__ static int lanes_per_phase() {
  return 128 / (int)(2 * sizeof(T));
}

// Distance between the groups' buffers (complex values).  Within one access
// phase the lanes cover (t, g) pairs; the offset makes (g * stride + t) hit
// distinct banks: groups interleaved across lanes (columns) need
// stride = P/F mod P, consecutive groups smaller than a phase (rows) need
// stride = G mod P.
template <typename T>
__host__ __device__ static int group_stride(int L, int F, bool cols) {
  const int P = lanes_per_phase<T>();
  const int base = L + L / 16, G = L / 16;
  int target = 0;
  if (cols) target = F >= P ? 1 : P / F;
  else if (G < P) target = G;
  return base + ((target - base) % P + P) % P;
}

// Tile shape (F, the vectors one block transforms) per kernel family,
// transform length and 4/8-byte arithmetic: chosen by measurement
// (rsfde_autotune) when recorded, else by the occupancy heuristic below.
// (the recorded table, the forced shape and the unsupported-launch flag live
// in transforms.cu; tune_forced() returns the shape tune_force_groups set)

// Largest feasible F: the thread cap (512 for 8-byte arithmetic, else
// RSFDE_FP32_THREADS), the shared-memory budget and the work available.
template <typename T>
int max_groups(int L, int items) {
  const int G = L / 16;
  const int cap = sizeof(T) == 8 ? 512 : RSFDE_FP32_THREADS;
  const size_t per = (size_t)(L + L / 16 + lanes_per_phase<T>()) * 2 * sizeof(T);
  int F = 1;
  while (2 * F * G <= cap && per * 2 * F <= (size_t)kSmemBudget && 2 * F <= items) F *= 2;
  return F;
}

template <typename T>
static int pick_groups(int L, int items, int kind) {
  const int Fmax = max_groups<T>(L, items);
  int log2L = 0;
  while ((1 << log2L) < L) ++log2L;
  int F = tune_forced() ? tune_forced() : tune_lookup(kind, log2L, sizeof(T) == 8);
  if (F > 0) return F < Fmax ? F : Fmax;
  F = Fmax;  // heuristic: as wide as fits, but at least ~2 blocks per SM
  while (F > 1 && (items + F - 1) / F < 2 * kNumSMs) F /= 2;
  return F;
}

template <typename T>
static size_t group_smem(int L, int F, bool cols) {
  return (size_t)F * group_stride<T>(L, F, cols) * 2 * sizeof(T);
}

template <typename K>
static void set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// phi != nullptr: tmpx = z - A_x z + pen phi z (ahead of a MODE_APPLY,
// MODE_RESIDUAL or MODE_RESID_ONLY column pass); phi == nullptr: tmpx = A_x z.
template <typename T, typename Tin>
void launch_toeplitz_rows(const Tin* z, void* tmpx, const uint8_t* phi, double pen, int n1, int n2,
                          const AxisTables<T>& ax, const int* gate, cudaStream_t s) {
  const int npairs = (n2 + 1) / 2;
  const int F = pick_groups<T>(ax.L, npairs, TK_TOEP_ROWS);
  const size_t sm = group_smem<T>(ax.L, F, false);
  auto k = phi ? toeplitz_kernel<T, Tin, MODE_APPLY, false, double> : toeplitz_kernel<T, Tin, MODE_RAW, false, double>;
  set_smem(k, sm);
  k<<<(npairs + F - 1) / F, F * (ax.L / 16), sm, s>>>(z, static_cast<T*>(tmpx), phi, pen, nullptr, nullptr,
                                                      n1, n2, ax, F, group_stride<T>(ax.L, F, false), gate,
                                                      nullptr, nullptr);
}


// Only the combinations the solver uses are instantiated: FP32 arithmetic
// runs the operator (MODE_APPLY) alone, double-FP32 the operator and the true
// residual; the raw Toeplitz products and the left variant's residual are FP64.
template <typename T, typename Tin, typename Tout>
void launch_toeplitz_cols(int mode, const Tin* z, void* tmpx, const uint8_t* phi, double pen,
                          const double* b, Tout* out, int n1, int n2, const AxisTables<T>& ay,
                          const int* gate, double* partials, SolverState* st, cudaStream_t s) {
  const int npairs = (n1 + 1) / 2;
  const int F = pick_groups<T>(ay.L, npairs, TK_TOEP_COLS);
  const size_t sm = group_smem<T>(ay.L, F, true);
  const int gs = group_stride<T>(ay.L, F, true);
  int grid = (npairs + F - 1) / F;
  // the true residual: FP64 or double-FP32 arithmetic on an FP64 x
  constexpr bool resid_mode = std::is_same<Tin, double>::value && !std::is_same<T, float>::value;
  constexpr bool fp64_modes = std::is_same<T, double>::value && std::is_same<Tin, double>::value &&
                              std::is_same<Tout, double>::value;
  constexpr bool apply_mode = !std::is_same<T, double>::value || std::is_same<Tout, double>::value;
  if constexpr (resid_mode) {
    if (mode == MODE_RESIDUAL) {  // partials: one per column pair (npairs <= 2048)
      auto k = toeplitz_kernel<T, Tin, MODE_RESIDUAL, true, Tout>;
      set_smem(k, sm);
      k<<<grid, F * (ay.L / 16), sm, s>>>(z, static_cast<T*>(tmpx), phi, pen, b, out, n1, n2, ay, F, gs, gate,
                                          partials, st);
      return;
    }
  }
  if constexpr (fp64_modes) {
    if (mode == MODE_RESID_ONLY || mode == MODE_RAW) {
      auto k = mode == MODE_RAW ? toeplitz_kernel<T, Tin, MODE_RAW, true, Tout>
                                : toeplitz_kernel<T, Tin, MODE_RESID_ONLY, true, Tout>;
      set_smem(k, sm);
      k<<<grid, F * (ay.L / 16), sm, s>>>(z, static_cast<T*>(tmpx), phi, pen, b, out, n1, n2, ay, F, gs, gate,
                                          partials, st);
      return;
    }
  }
  if constexpr (apply_mode) {
    if (mode == MODE_APPLY) {
      auto k = toeplitz_kernel<T, Tin, MODE_APPLY, true, Tout>;
      set_smem(k, sm);
      k<<<grid, F * (ay.L / 16), sm, s>>>(z, static_cast<T*>(tmpx), phi, pen, b, out, n1, n2, ay, F, gs, gate,
                                          partials, st);
      return;
    }
  }
  note_unsupported_launch();  // no kernel for this combination: reported as RSFDE_EINVAL
}

template <typename T, typename Tin, typename Tout>
void launch_dst_rows(const Tin* v, const double* vscale, Tout* out, int n1, int n2, const AxisTables<T>& ax,
                     const int* gate, cudaStream_t s) {
  const int F = pick_groups<T>(ax.L, n2, TK_DST_ROWS);
  const size_t sm = group_smem<T>(ax.L, F, false);
  auto k = dst_kernel<T, Tin, Tout, false>;
  set_smem(k, sm);
  k<<<(n2 + F - 1) / F, F * (ax.L / 16), sm, s>>>(v, vscale, out, n1, n2, ax, F, group_stride<T>(ax.L, F, false),
                                                  gate);
}

template <typename T, typename Tin, typename Tout>
void launch_dst_cols(const Tin* in, Tout* out, int n1, int n2, const AxisTables<T>& ay, cudaStream_t s) {
  const int F = pick_groups<T>(ay.L, n1, TK_DST_COLS);
  const size_t sm = group_smem<T>(ay.L, F, true);
  auto k = dst_kernel<T, Tin, Tout, true>;
  set_smem(k, sm);
  k<<<(n1 + F - 1) / F, F * (ay.L / 16), sm, s>>>(in, nullptr, out, n1, n2, ay, F, group_stride<T>(ay.L, F, true),
                                                  nullptr);
}

template <typename T>
void launch_precond_cols(const T* T1, T* T2a, T* T2b, int n1, int n2, const AxisTables<T>& ay, const T* lamx,
                         double pen, const int* gate, cudaStream_t s) {
  const int F = pick_groups<T>(ay.L, n1, TK_PRE_COLS);
  const size_t sm = group_smem<T>(ay.L, F, true);
  auto k = precond_cols_kernel<T>;
  set_smem(k, sm);
  k<<<(n1 + F - 1) / F, F * (ay.L / 16), sm, s>>>(T1, T2a, T2b, n1, n2, ay, lamx, T(pen), F,
                                                  group_stride<T>(ay.L, F, true), gate);
}

template <typename T, typename Tz>
void launch_precond_rows(const T* T2a, const T* T2b, const uint8_t* phi, Tz* z, int n1, int n2,
                         const AxisTables<T>& ax, const int* gate, cudaStream_t s) {
  const int F = pick_groups<T>(ax.L, n2, TK_PRE_ROWS);
  const size_t sm = group_smem<T>(ax.L, F, false);
  auto k = precond_rows_kernel<T, Tz>;
  set_smem(k, sm);
  k<<<(n2 + F - 1) / F, F * (ax.L / 16), sm, s>>>(T2a, T2b, phi, z, n1, n2, ax, F, group_stride<T>(ax.L, F, false),
                                                  gate);
}

// ---------------------------------------------------------------------------
// Multi-instance transform launches (batched form): every block finds its
// instance by the prefix of block counts and runs the same body as a
// single-instance launch, with F = kMultiThreads / (L/16) transforms per block
// and the instance's own virtual grid, so one launch covers every instance.
template <typename T>
__device__ __forceinline__ const AxisTables<T>& inst_tab(const BatchInst& I, bool y);
template <>
__device__ __forceinline__ const AxisTables<double>& inst_tab<double>(const BatchInst& I, bool y) {
  return y ? I.y64 : I.x64;
}
template <>
__device__ __forceinline__ const AxisTables<float>& inst_tab<float>(const BatchInst& I, bool y) {
  return y ? I.y32 : I.x32;
}
template <>
__device__ __forceinline__ const AxisTables<df>& inst_tab<df>(const BatchInst& I, bool y) {
  return y ? I.ydf : I.xdf;
}

// The multi-instance kernels below ask for the register budget of the
// single-instance kernels (4 blocks of 256 FP32 threads, 2 of FP64 or
// double-FP32, per SM), which their occupancy and latency hiding depend on.

// w_j = M z_j for every instance (MODE_APPLY; rows write z - A_x z + pen phi z
// into the scratch).
template <typename T, typename Tz, typename Tv, bool COLS>
__global__ void __launch_bounds__(kMultiThreads, sizeof(T) == 8 ? 2 : 4) operator_multi_kernel(const BatchInst* __restrict__ bi,
                                                                       const int* __restrict__ prefix,
                                                                       const int* __restrict__ active, int count,
                                                                       int j, int* sched) {
  multi_loop(bi, prefix, active, count, [&](const BatchInst& I, int lb, int nb) {
    const AxisTables<T>& ax = inst_tab<T>(I, COLS);
    const int F = multi_groups(ax.L);
    const Tz* z = static_cast<const Tz*>(I.Z) + (size_t)j * I.N;
    Tv* w = reinterpret_cast<Tv*>(I.V) + (size_t)(j + 1) * I.N;
    toeplitz_body<T, Tz, MODE_APPLY, COLS, Tv>(z, static_cast<T*>(I.tmpx), I.phi, I.pen, nullptr, w, I.n1, I.n2, ax,
                                               F, group_stride<T>(ax.L, F, COLS), &I.st->run_iter, nullptr, nullptr,
                                               lb, nb);
  }, sched);
}

// V_0 = b - M x and the restart decision (rows: x - A_x x + pen phi x into the
// scratch).
template <typename T, typename Tv, bool COLS>
__global__ void __launch_bounds__(kMultiThreads, sizeof(T) == 8 ? 2 : 4) residual_multi_kernel(const BatchInst* __restrict__ bi,
                                                                       const int* __restrict__ prefix,
                                                                       const int* __restrict__ active, int count, int* sched) {
  multi_loop(bi, prefix, active, count, [&](const BatchInst& I, int lb, int nb) {
    const AxisTables<T>& ax = inst_tab<T>(I, COLS);
    const int F = multi_groups(ax.L);
    const int gs = group_stride<T>(ax.L, F, COLS);
    if constexpr (COLS)
      toeplitz_body<T, double, MODE_RESIDUAL, true, Tv>(I.x, static_cast<T*>(I.tmpx), I.phi, I.pen, I.b,
                                                        reinterpret_cast<Tv*>(I.V), I.n1, I.n2, ax, F, gs,
                                                        &I.st->run_cycle, I.partials, I.st, lb, nb);
    else
      toeplitz_body<T, double, MODE_APPLY, false, double>(I.x, static_cast<T*>(I.tmpx), I.phi, I.pen, nullptr,
                                                          nullptr, I.n1, I.n2, ax, F, gs, &I.st->run_cycle, nullptr,
                                                          nullptr, lb, nb);
  }, sched);
}

// The three passes of the FFT preconditioner, z_j = P-hat^-1 (s_j V_j).
template <typename T, typename Tv>
__global__ void __launch_bounds__(kMultiThreads, sizeof(T) == 8 ? 2 : 4) dst_rows_multi_kernel(const BatchInst* __restrict__ bi,
                                                                       const int* __restrict__ prefix,
                                                                       const int* __restrict__ active, int count,
                                                                       int j, int* sched) {
  multi_loop(bi, prefix, active, count, [&](const BatchInst& I, int lb, int nb) {
    const AxisTables<T>& ax = inst_tab<T>(I, false);
    const int F = multi_groups(ax.L);
    dst_body<T, Tv, T, false>(reinterpret_cast<const Tv*>(I.V) + (size_t)j * I.N, &I.st->s[j],
                              static_cast<T*>(I.T1), I.n1, I.n2, ax, F, group_stride<T>(ax.L, F, false),
                              &I.st->run_iter, lb, nb);
  }, sched);
}
template <typename T>
__global__ void __launch_bounds__(kMultiThreads, sizeof(T) == 8 ? 2 : 4) precond_cols_multi_kernel(const BatchInst* __restrict__ bi,
                                                                           const int* __restrict__ prefix,
                                                                           const int* __restrict__ active,
                                                                           int count, int* sched) {
  multi_loop(bi, prefix, active, count, [&](const BatchInst& I, int lb, int nb) {
    const AxisTables<T>& ay = inst_tab<T>(I, true);
    const int F = multi_groups(ay.L);
    precond_cols_body<T>(static_cast<const T*>(I.T1), static_cast<T*>(I.T2a), static_cast<T*>(I.T2b), I.n1, I.n2,
                         ay, inst_tab<T>(I, false).lam, T(I.pen), F, group_stride<T>(ay.L, F, true),
                         &I.st->run_iter, lb, nb);
  }, sched);
}
template <typename T, typename Tz>
__global__ void __launch_bounds__(kMultiThreads, sizeof(T) == 8 ? 2 : 4) precond_rows_multi_kernel(const BatchInst* __restrict__ bi,
                                                                           const int* __restrict__ prefix,
                                                                           const int* __restrict__ active, int count,
                                                                           int j, int* sched) {
  multi_loop(bi, prefix, active, count, [&](const BatchInst& I, int lb, int nb) {
    const AxisTables<T>& ax = inst_tab<T>(I, false);
    const int F = multi_groups(ax.L);
    precond_rows_body<T, Tz>(static_cast<const T*>(I.T2a), static_cast<const T*>(I.T2b), I.phi,
                             static_cast<Tz*>(I.Z) + (size_t)j * I.N, I.n1, I.n2, ax, F,
                             group_stride<T>(ax.L, F, false), &I.st->run_iter, lb, nb);
  }, sched);
}

// Dynamic shared memory of a multi-instance transform launch: the largest any
// of its transform lengths needs.
template <typename T>
static size_t multi_smem(const MultiGrid& g, bool cols) {
  size_t m = 0;
  for (int k = 4; k <= 12; ++k)
    if (g.l2mask & (1u << k)) {
      const int L = 1 << k, F = multi_groups(L);
      const size_t b = group_smem<T>(L, F, cols);
      if (b > m) m = b;
    }
  return m;
}

template <typename T, typename Tz, typename Tv>
void launch_operator_multi(const BatchInst* bi, const MultiGrid& rows, const MultiGrid& cols, int j, cudaStream_t s) {
  auto kr = operator_multi_kernel<T, Tz, Tv, false>;
  auto kc = operator_multi_kernel<T, Tz, Tv, true>;
  const size_t sr = multi_smem<T>(rows, false), sc = multi_smem<T>(cols, true);
  set_smem(kr, sr);
  set_smem(kc, sc);
  kr<<<multi_launch_grid(kr, kMultiThreads, sr, rows.total), kMultiThreads, sr, s>>>(bi, rows.prefix, rows.active,
                                                                                   rows.count, j, rows.sched);
  kc<<<multi_launch_grid(kc, kMultiThreads, sc, cols.total), kMultiThreads, sc, s>>>(bi, cols.prefix, cols.active,
                                                                                   cols.count, j, cols.sched);
}

template <typename T, typename Tv>
void launch_residual_multi(const BatchInst* bi, const MultiGrid& rows, const MultiGrid& cols, cudaStream_t s) {
  auto kr = residual_multi_kernel<T, Tv, false>;
  auto kc = residual_multi_kernel<T, Tv, true>;
  const size_t sr = multi_smem<T>(rows, false), sc = multi_smem<T>(cols, true);
  set_smem(kr, sr);
  set_smem(kc, sc);
  kr<<<multi_launch_grid(kr, kMultiThreads, sr, rows.total), kMultiThreads, sr, s>>>(bi, rows.prefix, rows.active,
                                                                                   rows.count, rows.sched);
  kc<<<multi_launch_grid(kc, kMultiThreads, sc, cols.total), kMultiThreads, sc, s>>>(bi, cols.prefix, cols.active,
                                                                                   cols.count, cols.sched);
}

template <typename T, typename Tz, typename Tv>
void launch_precond_multi(const BatchInst* bi, const MultiGrid& drows, const MultiGrid& pcols, const MultiGrid& prows,
                          int j, cudaStream_t s) {
  auto k1 = dst_rows_multi_kernel<T, Tv>;
  auto k2 = precond_cols_multi_kernel<T>;
  auto k3 = precond_rows_multi_kernel<T, Tz>;
  const size_t s1 = multi_smem<T>(drows, false), s2 = multi_smem<T>(pcols, true), s3 = multi_smem<T>(prows, false);
  set_smem(k1, s1);
  set_smem(k2, s2);
  set_smem(k3, s3);
  k1<<<multi_launch_grid(k1, kMultiThreads, s1, drows.total), kMultiThreads, s1, s>>>(bi, drows.prefix, drows.active,
                                                                                    drows.count, j, drows.sched);
  k2<<<multi_launch_grid(k2, kMultiThreads, s2, pcols.total), kMultiThreads, s2, s>>>(bi, pcols.prefix, pcols.active,
                                                                                    pcols.count, pcols.sched);
  k3<<<multi_launch_grid(k3, kMultiThreads, s3, prows.total), kMultiThreads, s3, s>>>(bi, prows.prefix, prows.active,
                                                                                    prows.count, j, prows.sched);
}

}  // namespace rsfde
