// fft.cuh -- in-place power-of-two complex FFTs in shared memory.
//
// The two transforms used on the hot path are both convolutions:
//   * the Toeplitz products A_x z, A_y z of Eq. 2.15-2.16, by embedding the
//     symmetric Toeplitz matrix in a circulant of length L >= 2n-1;
//   * the sine transform S_n of Section 4.1, by the chirp-z (Bluestein)
//     identity jk = (j^2 + k^2 - (k-j)^2)/2, a convolution of length L >= 2n-1.
// A convolution needs no output ordering, so the forward transform is
// decimation-in-frequency (natural order in, bit-reversed out), the pointwise
// product uses a spectrum stored in bit-reversed order, and the inverse is
// decimation-in-time (bit-reversed in, natural out).  No permutation pass.
//
// Data: B transforms, real parts re[b*L + l], imaginary parts im[b*L + l].
// Twiddles: tw[2*j], tw[2*j+1] = cos, sin of -2 pi j / L for j in [0, L).
// Stages are radix 4 (three twiddle products per four points) with one
// radix-2 stage when log2 L is odd.  The inverse is unnormalised (times L).
#pragma once

namespace rsfde {

// One radix-2 DIF butterfly of the first stage (span L/2), k in [0, L/2).
template <typename T>
__host__ __device__ __forceinline__ void dif_r2(T* re, T* im, int L, int k, const T* tw) {
  const int h = L >> 1;
  T ar = re[k], ai = im[k], br = re[k + h], bi = im[k + h];
  T wr = tw[2 * k], wi = tw[2 * k + 1];
  re[k] = ar + br;
  im[k] = ai + bi;
  T dr = ar - br, di = ai - bi;
  re[k + h] = dr * wr - di * wi;
  im[k + h] = dr * wi + di * wr;
}

// One radix-4 DIF butterfly: quarter span s, butterfly q in [0, L/4).
// Equals two radix-2 DIF stages of spans 2s and s.
template <typename T>
__host__ __device__ __forceinline__ void dif_r4(T* re, T* im, int L, int s, int q, const T* tw) {
  const int k0 = q & (s - 1);
  const int base = ((q - k0) << 2) + k0;
  const int step = L / (4 * s);  // W_{4s}^{k0} = W_L^{k0 * L/(4s)}
  const int j1 = k0 * step;
  T x0r = re[base], x0i = im[base];
  T x1r = re[base + s], x1i = im[base + s];
  T x2r = re[base + 2 * s], x2i = im[base + 2 * s];
  T x3r = re[base + 3 * s], x3i = im[base + 3 * s];
  T t0r = x0r + x2r, t0i = x0i + x2i;
  T t1r = x1r + x3r, t1i = x1i + x3i;
  T t2r = x0r - x2r, t2i = x0i - x2i;
  T t3r = x1i - x3i, t3i = x3r - x1r;  // (x1 - x3) * (-i)
  re[base] = t0r + t1r;
  im[base] = t0i + t1i;
  T ar = t0r - t1r, ai = t0i - t1i;
  T br = t2r + t3r, bi = t2i + t3i;
  T cr = t2r - t3r, ci = t2i - t3i;
  T w1r = tw[2 * j1], w1i = tw[2 * j1 + 1];
  T w2r = tw[4 * j1], w2i = tw[4 * j1 + 1];
  T w3r = tw[6 * j1], w3i = tw[6 * j1 + 1];
  re[base + s] = ar * w2r - ai * w2i;
  im[base + s] = ar * w2i + ai * w2r;
  re[base + 2 * s] = br * w1r - bi * w1i;
  im[base + 2 * s] = br * w1i + bi * w1r;
  re[base + 3 * s] = cr * w3r - ci * w3i;
  im[base + 3 * s] = cr * w3i + ci * w3r;
}

// One radix-4 DIT butterfly with conjugate twiddles (inverse transform):
// two radix-2 DIT stages of spans s and 2s.
template <typename T>
__host__ __device__ __forceinline__ void dit_r4(T* re, T* im, int L, int s, int q, const T* tw) {
  const int k0 = q & (s - 1);
  const int base = ((q - k0) << 2) + k0;
  const int step = L / (4 * s);
  const int j1 = k0 * step;
  // v = conj(W_{4s}^{k0}); u1 = y1 v^2, u2 = y2 v, u3 = y3 v^3
  T v1r = tw[2 * j1], v1i = -tw[2 * j1 + 1];
  T v2r = tw[4 * j1], v2i = -tw[4 * j1 + 1];
  T v3r = tw[6 * j1], v3i = -tw[6 * j1 + 1];
  T y0r = re[base], y0i = im[base];
  T y1r = re[base + s], y1i = im[base + s];
  T y2r = re[base + 2 * s], y2i = im[base + 2 * s];
  T y3r = re[base + 3 * s], y3i = im[base + 3 * s];
  T u1r = y1r * v2r - y1i * v2i, u1i = y1r * v2i + y1i * v2r;
  T u2r = y2r * v1r - y2i * v1i, u2i = y2r * v1i + y2i * v1r;
  T u3r = y3r * v3r - y3i * v3i, u3i = y3r * v3i + y3i * v3r;
  T p0r = y0r + u1r, p0i = y0i + u1i;
  T p1r = y0r - u1r, p1i = y0i - u1i;
  T q0r = u2r + u3r, q0i = u2i + u3i;
  T q1r = u3i - u2i, q1i = u2r - u3r;  // (u2 - u3) * i
  re[base] = p0r + q0r;
  im[base] = p0i + q0i;
  re[base + 2 * s] = p0r - q0r;
  im[base + 2 * s] = p0i - q0i;
  re[base + s] = p1r + q1r;
  im[base + s] = p1i + q1i;
  re[base + 3 * s] = p1r - q1r;
  im[base + 3 * s] = p1i - q1i;
}

// Last radix-2 DIT butterfly (span L/2) with conjugate twiddle, k in [0, L/2).
template <typename T>
__host__ __device__ __forceinline__ void dit_r2(T* re, T* im, int L, int k, const T* tw) {
  const int h = L >> 1;
  T wr = tw[2 * k], wi = -tw[2 * k + 1];
  T ar = re[k], ai = im[k];
  T xr = re[k + h], xi = im[k + h];
  T br = xr * wr - xi * wi, bi = xr * wi + xi * wr;
  re[k] = ar + br;
  im[k] = ai + bi;
  re[k + h] = ar - br;
  im[k + h] = ai - bi;
}

#ifdef __CUDACC__
// Forward DIF of B transforms of length L = 2^log2L held in shared memory.
// Every thread of the block must call it; it ends with __syncthreads().
template <typename T>
__device__ __forceinline__ void fft_dif(T* re, T* im, int L, int log2L, int B, const T* __restrict__ tw) {
  int s;
  if (log2L & 1) {
    const int h = L >> 1;
    for (int t = threadIdx.x; t < B * h; t += blockDim.x) {
      const int b = t >> (log2L - 1);
      dif_r2(re + b * L, im + b * L, L, t & (h - 1), tw);
    }
    __syncthreads();
    s = L >> 3;
  } else {
    s = L >> 2;
  }
  const int quarter = L >> 2;
  for (; s >= 1; s >>= 2) {
    for (int t = threadIdx.x; t < B * quarter; t += blockDim.x) {
      const int b = t >> (log2L - 2);
      dif_r4(re + b * L, im + b * L, L, s, t & (quarter - 1), tw);
    }
    __syncthreads();
  }
}

// Inverse DIT (unnormalised) of B transforms; bit-reversed in, natural out.
template <typename T>
__device__ __forceinline__ void ifft_dit(T* re, T* im, int L, int log2L, int B, const T* __restrict__ tw) {
  const int quarter = L >> 2;
  const int smax = (log2L & 1) ? (L >> 3) : (L >> 2);
  for (int s = 1; s <= smax; s <<= 2) {
    for (int t = threadIdx.x; t < B * quarter; t += blockDim.x) {
      const int b = t >> (log2L - 2);
      dit_r4(re + b * L, im + b * L, L, s, t & (quarter - 1), tw);
    }
    __syncthreads();
  }
  if (log2L & 1) {
    const int h = L >> 1;
    for (int t = threadIdx.x; t < B * h; t += blockDim.x) {
      const int b = t >> (log2L - 1);
      dit_r2(re + b * L, im + b * L, L, t & (h - 1), tw);
    }
    __syncthreads();
  }
}
#endif

}  // namespace rsfde
