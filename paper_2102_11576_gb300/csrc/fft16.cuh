// fft16.cuh -- register-resident Stockham FFTs of power-of-two length L >= 16.
//
// A transform is done by a "group" of G = L/16 threads; thread t of the group
// holds the 16 complex values at positions t + k*L/16 (k = 0..15) in
// registers.  Each pass applies radix-R DFTs (R = 16, or 2/4/8 for the one
// pass that L = 16^a * R needs) to values L/R apart, after the Stockham
// twiddles, and the values move through a padded shared-memory buffer only
// between passes.  The forward transform runs [R_small, 16, ..., 16] and
// leaves thread t holding the spectrum in natural order at its own positions
// t + k*L/16; the inverse runs [16, ..., 16, R_small] and starts from exactly
// those registers.  A convolution (Toeplitz product, Bluestein sine transform)
// therefore needs no shared-memory round trip for the pointwise spectral
// product, and its output ends up at the positions its input came from.
//
// Shared memory: one buffer of L + L/16 (+ a few) complex values per group;
// one pad value every 16 and a per-mapping offset between the groups' buffers
// keep the exchanges free of bank conflicts.  Twiddles:
// tw[m] = exp(-2 pi i m / L), m in [0, L), interleaved (re, im).
#pragma once

namespace rsfde {

template <typename T>
struct cx {
  T r, i;
};

template <typename T>
__device__ __forceinline__ cx<T> c_add(cx<T> a, cx<T> b) {
  return {a.r + b.r, a.i + b.i};
}
template <typename T>
__device__ __forceinline__ cx<T> c_sub(cx<T> a, cx<T> b) {
  return {a.r - b.r, a.i - b.i};
}
template <typename T>
__device__ __forceinline__ cx<T> c_mul(cx<T> a, cx<T> b) {
  return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r};
}
// times -i (forward) or +i (inverse)
template <typename T, bool INV>
__device__ __forceinline__ cx<T> c_mi(cx<T> a) {
  return INV ? cx<T>{-a.i, a.r} : cx<T>{a.i, -a.r};
}
// times exp(-+ 2 pi i k / 16) for the fixed k of the radix-16/8 kernels
template <typename T, bool INV, int K>
__device__ __forceinline__ cx<T> rot16(cx<T> a) {
  const T c1 = T(0.92387953251128675612818318939678828682241662586364);  // cos(pi/8)
  const T s1 = T(0.38268343236508977172845998403039886676134456248563);  // sin(pi/8)
  const T h = T(0.70710678118654752440084436210484903928483593768847);   // cos(pi/4)
  T wr, wi;
  if (K == 1) { wr = c1; wi = -s1; }
  else if (K == 2) { wr = h; wi = -h; }
  else if (K == 3) { wr = s1; wi = -c1; }
  else if (K == 4) { return c_mi<T, INV>(a); }
  else if (K == 6) { wr = -h; wi = -h; }
  else { wr = -c1; wi = s1; }  // K == 9
  if (INV) wi = -wi;
  return {a.r * wr - a.i * wi, a.r * wi + a.i * wr};
}

// Natural-order DFTs on v[0], v[S], ..., v[(R-1)S] (compile-time stride).
template <typename T, bool INV, int S>
__device__ __forceinline__ void dft2(cx<T>* v) {
  const cx<T> a = v[0], b = v[S];
  v[0] = c_add(a, b);
  v[S] = c_sub(a, b);
}
template <typename T, bool INV, int S>
__device__ __forceinline__ void dft4(cx<T>* v) {
  const cx<T> t0 = c_add(v[0], v[2 * S]), t1 = c_sub(v[0], v[2 * S]);
  const cx<T> t2 = c_add(v[S], v[3 * S]), t3 = c_mi<T, INV>(c_sub(v[S], v[3 * S]));
  v[0] = c_add(t0, t2);
  v[2 * S] = c_sub(t0, t2);
  v[S] = c_add(t1, t3);
  v[3 * S] = c_sub(t1, t3);
}
// 8 = 4 x 2: q = 2 q1 + q2, r = r1 + 4 r2
template <typename T, bool INV, int S>
__device__ __forceinline__ void dft8(cx<T>* v) {
  dft4<T, INV, 2 * S>(v);
  dft4<T, INV, 2 * S>(v + S);
  // v[(2 r1 + q2) S] = b[q2][r1]; twiddle W8^{q2 r1} = W16^{2 q2 r1}
  v[3 * S] = rot16<T, INV, 2>(v[3 * S]);
  v[5 * S] = rot16<T, INV, 4>(v[5 * S]);
  v[7 * S] = rot16<T, INV, 6>(v[7 * S]);
  cx<T> o[8];
#pragma unroll
  for (int r1 = 0; r1 < 4; ++r1) {
    o[r1] = c_add(v[2 * r1 * S], v[(2 * r1 + 1) * S]);
    o[r1 + 4] = c_sub(v[2 * r1 * S], v[(2 * r1 + 1) * S]);
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) v[r * S] = o[r];
}
// 16 = 4 x 4: q = 4 q1 + q2, r = r1 + 4 r2
template <typename T, bool INV>
__device__ __forceinline__ void dft16(cx<T>* v) {
  dft4<T, INV, 4>(v);
  dft4<T, INV, 4>(v + 1);
  dft4<T, INV, 4>(v + 2);
  dft4<T, INV, 4>(v + 3);
  // v[4 r1 + q2] = b[q2][r1]; twiddle W16^{q2 r1}
  v[5] = rot16<T, INV, 1>(v[5]);
  v[9] = rot16<T, INV, 2>(v[9]);
  v[13] = rot16<T, INV, 3>(v[13]);
  v[6] = rot16<T, INV, 2>(v[6]);
  v[10] = rot16<T, INV, 4>(v[10]);
  v[14] = rot16<T, INV, 6>(v[14]);
  v[7] = rot16<T, INV, 3>(v[7]);
  v[11] = rot16<T, INV, 6>(v[11]);
  v[15] = rot16<T, INV, 9>(v[15]);
  dft4<T, INV, 1>(v);
  dft4<T, INV, 1>(v + 4);
  dft4<T, INV, 1>(v + 8);
  dft4<T, INV, 1>(v + 12);
  // position 4 r1 + r2 holds output r1 + 4 r2: transpose the 4 x 4
  cx<T> o[16];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) o[a + 4 * b] = v[4 * a + b];
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = o[r];
}

template <typename T, bool INV, int R, int S>
__device__ __forceinline__ void dft_r(cx<T>* v) {
  if (R == 16) dft16<T, INV>(v);
  else if (R == 8) dft8<T, INV, S>(v);
  else if (R == 4) dft4<T, INV, S>(v);
  else dft2<T, INV, S>(v);
}

__device__ __forceinline__ int fft_pad(int i) { return i + (i >> 4); }

// Twiddle w^q for q = 1..R-1 with w = tw[step].  FP64 reads every power from
// the table (the FP64 units are the scarce resource); FP32 reads w (read-only
// path), squares it into w^2, w^4, w^8, and forms each other power, as it is
// applied, from the factors of q's binary digits (at most three products;
// ~15 ulp at worst, inside the FP32 transforms' error) -- the FP32 transforms
// wait on loads, not arithmetic, and four base powers and one product live at
// a time (64 registers).
template <typename T, bool INV, int R>
__device__ __forceinline__ void twiddle_apply(cx<T>* v, int i, int step, const cx<T>* __restrict__ tw) {
  constexpr int S = 16 / R;
  if (sizeof(T) == 8) {
#pragma unroll
    for (int q = 1; q < R; ++q) {
      cx<T> w = tw[q * step];
      if (INV) w.i = -w.i;
      v[i + q * S] = c_mul(v[i + q * S], w);
    }
  } else {
    cx<T> b[4];  // w^1, w^2, w^4, w^8
    auto ld = [&](int idx) {
      const float2 t = __ldg(reinterpret_cast<const float2*>(tw) + idx);
      return cx<T>{t.x, t.y};
    };
    b[0] = ld(step);
    if (R > 2) b[1] = c_mul(b[0], b[0]);
    if (R > 4) b[2] = c_mul(b[1], b[1]);
    if (R > 8) b[3] = c_mul(b[2], b[2]);
    if (INV) {
#pragma unroll
      for (int k = 0; k < 4; ++k) b[k].i = -b[k].i;
    }
#pragma unroll
    for (int q = 1; q < R; ++q) {
      cx<T> w;
      bool have = false;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (q & (1 << k)) {
          w = have ? c_mul(w, b[k]) : b[k];
          have = true;
        }
      }
      v[i + q * S] = c_mul(v[i + q * S], w);
    }
  }
}

// One Stockham pass: twiddles for sub-transforms of length Ns * R, radix-R
// DFTs of the 16/R items this thread owns (item i = position t + i L/16).
// LG > 0: the transform length 2^LG is a compile-time constant (the index
// arithmetic folds); LG = 0: L is the runtime argument.  Both give the same
// arithmetic in the same order.
template <typename T, bool INV, int R, int LG = 0>
__device__ __forceinline__ void fft_pass(cx<T>* v, int t, int Lrt, int Ns, const cx<T>* __restrict__ tw) {
  constexpr int S = 16 / R;
  const int L = LG ? (1 << LG) : Lrt;
  const int Lq = L >> 4;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    if (Ns > 1) {
      const int j = t + i * Lq;
      const int jm = j & (Ns - 1);
      twiddle_apply<T, INV, R>(v, i, jm * (L / (Ns * R)), tw);
    }
    dft_r<T, INV, R, S>(v + i);
  }
}

// Moves the pass outputs through shared memory so that every thread again
// holds the positions t + k L/16 that the next pass reads.
template <typename T, int R, int LG = 0>
__device__ __forceinline__ void fft_exchange(cx<T>* v, cx<T>* buf, int t, int Lrt, int Ns) {
  constexpr int S = 16 / R;
  const int L = LG ? (1 << LG) : Lrt;
  const int Lq = L >> 4;
  __syncthreads();
#pragma unroll
  for (int i = 0; i < S; ++i) {
    const int j = t + i * Lq;
    const int jm = j & (Ns - 1);
    const int d = (j - jm) * R + jm;
#pragma unroll
    for (int r = 0; r < R; ++r) buf[fft_pad(d + r * Ns)] = v[i + r * S];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = buf[fft_pad(t + k * Lq)];
}

// Forward transform: input positions t + k L/16 in v, output spectrum (natural
// order) at the same positions.  Every input of this library's convolutions
// is zero on the upper half (positions >= L/2, i.e. k >= 8): those registers
// are cleared here so the first pass's arithmetic on them folds away.  All
// threads of the block must call it with the same L (it synchronises).
template <typename T, int LG = 0>
__device__ __forceinline__ void fft16_forward(cx<T>* v, cx<T>* buf, int t, int Lrt, int lgrt,
                                              const cx<T>* __restrict__ tw) {
#pragma unroll
  for (int k = 8; k < 16; ++k) v[k] = {T(0), T(0)};
  const int L = LG ? (1 << LG) : Lrt, log2L = LG ? LG : lgrt;
  const int small = log2L & 3;
  const int n16 = log2L >> 2;
  int Ns = 1;
  if (small == 1) {
    fft_pass<T, false, 2, LG>(v, t, L, Ns, tw);
    fft_exchange<T, 2, LG>(v, buf, t, L, Ns);
    Ns = 2;
  } else if (small == 2) {
    fft_pass<T, false, 4, LG>(v, t, L, Ns, tw);
    fft_exchange<T, 4, LG>(v, buf, t, L, Ns);
    Ns = 4;
  } else if (small == 3) {
    fft_pass<T, false, 8, LG>(v, t, L, Ns, tw);
    fft_exchange<T, 8, LG>(v, buf, t, L, Ns);
    Ns = 8;
  }
#pragma unroll 1
  for (int p = 0; p < n16; ++p) {
    fft_pass<T, false, 16, LG>(v, t, L, Ns, tw);
    if (p + 1 < n16) fft_exchange<T, 16, LG>(v, buf, t, L, Ns);
    Ns <<= 4;
  }
}

// Inverse transform (unnormalised, times L) from the forward's register layout;
// output in natural order at positions t + k L/16.  Callers read only k < 8
// (positions < L/2), so the last pass's other outputs are never formed.
template <typename T, int LG = 0>
__device__ __forceinline__ void fft16_inverse(cx<T>* v, cx<T>* buf, int t, int Lrt, int lgrt,
                                              const cx<T>* __restrict__ tw) {
  const int L = LG ? (1 << LG) : Lrt, log2L = LG ? LG : lgrt;
  const int small = log2L & 3;
  const int n16 = log2L >> 2;
  int Ns = 1;
#pragma unroll 1
  for (int p = 0; p < n16; ++p) {
    fft_pass<T, true, 16, LG>(v, t, L, Ns, tw);
    if (p + 1 < n16 || small) fft_exchange<T, 16, LG>(v, buf, t, L, Ns);
    Ns <<= 4;
  }
  if (small == 1) fft_pass<T, true, 2, LG>(v, t, L, Ns, tw);
  else if (small == 2) fft_pass<T, true, 4, LG>(v, t, L, Ns, tw);
  else if (small == 3) fft_pass<T, true, 8, LG>(v, t, L, Ns, tw);
}

}  // namespace rsfde
