// exact.cuh -- the Toeplitz products of the true residual b - M x (Eq. 2.14-
// 2.17) computed exactly in integer arithmetic on GB300's integer pipes.
//
// GB300 executes FP64 at 1/64 of its FP32/INT32 rate, so an FP64 FFT of the
// residual is bound by the FP64 pipe.  Here each vector x (a row or a column
// of the grid) is scaled by a power of two to integers x_q below 2^55 in
// magnitude (E the largest biased exponent in the vector: x_q = trunc(x
// 2^(1077-E))), the Toeplitz column t on the host to integers t_q =
// round(t 2^St) whose row sum T1_q = |t_q[0]| + 2 sum_k |t_q[k]| is below
// 2^63, so the convolution sum_l t_q[|i-l|] x_q[l] is an integer below 2^118
// in magnitude.  It is computed exactly modulo four primes p < 2^30 (product
// > 2^119.99) by number-theoretic transforms of length L >= 2n-1, then
// reconstructed by Garner's mixed-radix form of the Chinese remainder theorem
// and scaled back to FP64 (truncated to 53 bits).  The product's only errors
// are the two scalings (|x - x_q 2^(E-1077)| < 2^-54 max|x|; each t_k within
// 2^-63 T1) and the final truncation -- below the rounding error bounds of
// FP64 evaluation, direct or by FFT.  What follows the product (x - A_x x +
// (dt/eta) phi x, b - ..., ||r||^2) is FP64 arithmetic.
//
// Transforms: the register-resident Stockham layout of fft16.cuh (a group of
// L/16 threads, thread t holding positions t + k L/16), with values in
// [0, p), Shoup's multiplication by precomputed constants (w, floor(w 2^32 /
// p)) and radix-16/8/4/2 butterflies.  NTT_p(x)[k] = sum_j x_j w^(jk) with
// w = g^((p-1)/L), g a generator of Z_p^*.
#pragma once
#include <stdint.h>

#include "transforms.cuh"

namespace rsfde {

constexpr int kNttPrimes = 4;
// primes k 2^16 + 1 just below 2^30 (L up to 2^16), and generators of Z_p^*
constexpr uint32_t kNttP[kNttPrimes] = {1073479681u, 1072496641u, 1071513601u, 1070727169u};
constexpr uint32_t kNttG[kNttPrimes] = {11u, 11u, 23u, 11u};

__host__ __device__ constexpr uint32_t ntt_pow(uint32_t b, uint64_t e, uint32_t p) {
  uint64_t r = 1, x = b % p;
  while (e) {
    if (e & 1) r = r * x % p;
    x = x * x % p;
    e >>= 1;
  }
  return (uint32_t)r;
}
// Shoup's companion of a constant w < p: floor(w 2^32 / p)
__host__ __device__ constexpr uint32_t ntt_shoup(uint32_t w, uint32_t p) {
  return (uint32_t)(((uint64_t)w << 32) / p);
}

// a w mod p for any 32-bit a (w < p < 2^31, wq = ntt_shoup(w, p)): with
// q = floor(a wq / 2^32), a w - q p lies in [0, 2p) and is exact mod 2^32.
__device__ __forceinline__ uint32_t mulq(uint32_t a, uint32_t w, uint32_t wq, uint32_t p) {
  const uint32_t q = __umulhi(a, wq);
  const uint32_t r = a * w - q * p;
  return min(r, r - p);  // r - p wraps above r when r < p
}
__device__ __forceinline__ uint32_t addq(uint32_t a, uint32_t b, uint32_t p) {  // a, b < p
  const uint32_t s = a + b;
  return min(s, s - p);
}
__device__ __forceinline__ uint32_t subq(uint32_t a, uint32_t b, uint32_t p) {  // a, b < p
  const uint32_t d = a - b + p;
  return min(d, d - p);
}
__device__ __forceinline__ uint32_t redq(uint32_t a, uint32_t p) {  // a < 2p
  return min(a, a - p);
}

// Table entry through the read-only path, issued where it is written: the
// twiddle and spectrum reads are the same for every vector a block
// transforms, and hoisting them out of the vector loops would hold ~100
// registers.
__device__ __forceinline__ uint2 ld_tab(const uint2* p) {
  uint2 r;
  asm volatile("ld.global.nc.v2.u32 {%0, %1}, [%2];" : "=r"(r.x), "=r"(r.y) : "l"(p));
  return r;
}

// Constants of each prime: p, 2^32 mod p and floor(2^32/p) (for residues),
// and the powers W16^K (K = 1, 2, 3, 4, 6, 9: the radix-16/8/4 butterflies'
// internal roots) of W16 = g^((p-1)/16) = w^(L/16), forward and inverse, with
// Shoup companions, all evaluated at compile time.
struct NttPrimeConsts {
  uint32_t p, r32, r32q, oneq;
  uint32_t w[2][6], wq[2][6];
};
struct NttConstTable {
  NttPrimeConsts c[kNttPrimes];
};
constexpr NttConstTable make_ntt_consts() {
  NttConstTable t{};
  const int ks[6] = {1, 2, 3, 4, 6, 9};
  for (int i = 0; i < kNttPrimes; ++i) {
    const uint32_t p = kNttP[i];
    const uint32_t w16 = ntt_pow(kNttG[i], (p - 1) / 16, p);
    t.c[i].p = p;
    t.c[i].r32 = (uint32_t)((1ull << 32) % p);
    t.c[i].r32q = ntt_shoup(t.c[i].r32, p);
    t.c[i].oneq = ntt_shoup(1u, p);
    for (int j = 0; j < 6; ++j)
      for (int inv = 0; inv < 2; ++inv) {
        const uint32_t w = ntt_pow(w16, (uint64_t)(inv ? (16 - ks[j]) % 16 : ks[j]), p);
        t.c[i].w[inv][j] = w;
        t.c[i].wq[inv][j] = ntt_shoup(w, p);
      }
  }
  return t;
}

// One direction's butterfly constants of one prime (compile-time values: the
// multiplications take them as immediates).
struct NttK {
  uint32_t p;
  uint32_t w[6], wq[6];
};
template <int PI, bool INV>
__device__ __forceinline__ NttK ntt_consts() {
  constexpr NttConstTable T = make_ntt_consts();
  NttK k;
  k.p = T.c[PI].p;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    k.w[j] = T.c[PI].w[INV][j];
    k.wq[j] = T.c[PI].wq[INV][j];
  }
  return k;
}
// times W16^K (K in 1, 2, 3, 4, 6, 9) in the direction K holds
template <int K>
__device__ __forceinline__ uint32_t nrot(uint32_t a, const NttK& c) {
  constexpr int j = K == 1 ? 0 : K == 2 ? 1 : K == 3 ? 2 : K == 4 ? 3 : K == 6 ? 4 : 5;
  static_assert(K == 1 || K == 2 || K == 3 || K == 4 || K == 6 || K == 9, "stored powers");
  return mulq(a, c.w[j], c.wq[j], c.p);
}

// Natural-order DFTs over Z_p on v[0], v[S], ..., v[(R-1)S] (the factorings of
// fft16.cuh with W4 = W16^4 in place of -i).
template <int S>
__device__ __forceinline__ void ndft2(uint32_t* v, const NttK& c) {
  const uint32_t a = v[0], b = v[S];
  v[0] = addq(a, b, c.p);
  v[S] = subq(a, b, c.p);
}
template <int S>
__device__ __forceinline__ void ndft4(uint32_t* v, const NttK& c) {
  const uint32_t p = c.p;
  const uint32_t t0 = addq(v[0], v[2 * S], p), t1 = subq(v[0], v[2 * S], p);
  const uint32_t t2 = addq(v[S], v[3 * S], p), t3 = nrot<4>(subq(v[S], v[3 * S], p), c);
  v[0] = addq(t0, t2, p);
  v[2 * S] = subq(t0, t2, p);
  v[S] = addq(t1, t3, p);
  v[3 * S] = subq(t1, t3, p);
}
template <int S>
__device__ __forceinline__ void ndft8(uint32_t* v, const NttK& c) {
  const uint32_t p = c.p;
  ndft4<2 * S>(v, c);
  ndft4<2 * S>(v + S, c);
  v[3 * S] = nrot<2>(v[3 * S], c);
  v[5 * S] = nrot<4>(v[5 * S], c);
  v[7 * S] = nrot<6>(v[7 * S], c);
  uint32_t o[8];
#pragma unroll
  for (int r1 = 0; r1 < 4; ++r1) {
    o[r1] = addq(v[2 * r1 * S], v[(2 * r1 + 1) * S], p);
    o[r1 + 4] = subq(v[2 * r1 * S], v[(2 * r1 + 1) * S], p);
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) v[r * S] = o[r];
}
__device__ __forceinline__ void ndft16(uint32_t* v, const NttK& c) {
  ndft4<4>(v, c);
  ndft4<4>(v + 1, c);
  ndft4<4>(v + 2, c);
  ndft4<4>(v + 3, c);
  v[5] = nrot<1>(v[5], c);
  v[9] = nrot<2>(v[9], c);
  v[13] = nrot<3>(v[13], c);
  v[6] = nrot<2>(v[6], c);
  v[10] = nrot<4>(v[10], c);
  v[14] = nrot<6>(v[14], c);
  v[7] = nrot<3>(v[7], c);
  v[11] = nrot<6>(v[11], c);
  v[15] = nrot<9>(v[15], c);
  ndft4<1>(v, c);
  ndft4<1>(v + 4, c);
  ndft4<1>(v + 8, c);
  ndft4<1>(v + 12, c);
  uint32_t o[16];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) o[a + 4 * b] = v[4 * a + b];
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = o[r];
}
// The same DFTs when the upper half of the inputs is zero (the forward
// transform's first pass: positions >= L/2 of every input are zero).
template <int S>
__device__ __forceinline__ void ndft4h(uint32_t* v, const NttK& c) {  // v[2S] = v[3S] = 0
  const uint32_t p = c.p, a = v[0], b = v[S], t3 = nrot<4>(b, c);
  v[0] = addq(a, b, p);
  v[2 * S] = subq(a, b, p);
  v[S] = addq(a, t3, p);
  v[3 * S] = subq(a, t3, p);
}
template <int S>
__device__ __forceinline__ void ndft8h(uint32_t* v, const NttK& c) {
  const uint32_t p = c.p;
  ndft4h<2 * S>(v, c);
  ndft4h<2 * S>(v + S, c);
  v[3 * S] = nrot<2>(v[3 * S], c);
  v[5 * S] = nrot<4>(v[5 * S], c);
  v[7 * S] = nrot<6>(v[7 * S], c);
  uint32_t o[8];
#pragma unroll
  for (int r1 = 0; r1 < 4; ++r1) {
    o[r1] = addq(v[2 * r1 * S], v[(2 * r1 + 1) * S], p);
    o[r1 + 4] = subq(v[2 * r1 * S], v[(2 * r1 + 1) * S], p);
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) v[r * S] = o[r];
}
__device__ __forceinline__ void ndft16h(uint32_t* v, const NttK& c) {
  ndft4h<4>(v, c);
  ndft4h<4>(v + 1, c);
  ndft4h<4>(v + 2, c);
  ndft4h<4>(v + 3, c);
  v[5] = nrot<1>(v[5], c);
  v[9] = nrot<2>(v[9], c);
  v[13] = nrot<3>(v[13], c);
  v[6] = nrot<2>(v[6], c);
  v[10] = nrot<4>(v[10], c);
  v[14] = nrot<6>(v[14], c);
  v[7] = nrot<3>(v[7], c);
  v[11] = nrot<6>(v[11], c);
  v[15] = nrot<9>(v[15], c);
  ndft4<1>(v, c);
  ndft4<1>(v + 4, c);
  ndft4<1>(v + 8, c);
  ndft4<1>(v + 12, c);
  uint32_t o[16];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) o[a + 4 * b] = v[4 * a + b];
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = o[r];
}

template <int R, int S, bool HALF>
__device__ __forceinline__ void ndft_r(uint32_t* v, const NttK& c) {
  if (HALF) {
    if (R == 16) ndft16h(v, c);
    else if (R == 8) ndft8h<S>(v, c);
    else if (R == 4) ndft4h<S>(v, c);
    else v[S] = v[0];  // radix 2 with a zero second input
  } else {
    if (R == 16) ndft16(v, c);
    else if (R == 8) ndft8<S>(v, c);
    else if (R == 4) ndft4<S>(v, c);
    else ndft2<S>(v, c);
  }
}

// One Stockham pass (the index arithmetic of fft_pass); tw: {w^m, Shoup} of
// the forward (w) or inverse (w^-1) root, matching the direction of c.
// LG > 0: the transform length 2^LG is a compile-time constant (the index
// arithmetic folds); LG = 0: L is the runtime argument.
template <int R, bool HALF = false, int LG = 0>
__device__ __forceinline__ void ntt_pass(uint32_t* v, int t, int Lrt, int Ns, const uint2* __restrict__ tw,
                                         const NttK& c) {
  constexpr int S = 16 / R;
  const int L = LG ? (1 << LG) : Lrt;
  const int Lq = L >> 4;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    if (Ns > 1) {
      const int j = t + i * Lq;
      const int step = (j & (Ns - 1)) * (L / (Ns * R));
#pragma unroll
      for (int q = 1; q < R; ++q) {
        const uint2 w = ld_tab(tw + q * step);
        v[i + q * S] = mulq(v[i + q * S], w.x, w.y, c.p);
      }
    }
    ndft_r<R, S, HALF>(v + i, c);
  }
}

template <int R, int LG = 0>
__device__ __forceinline__ void ntt_exchange(uint32_t* v, uint32_t* buf, int t, int Lrt, int Ns) {
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

// Forward transform of a sequence that is zero on positions >= L/2 (k >= 8);
// spectrum in natural order at the thread's positions.  Block-uniform L.
template <int LG = 0>
__device__ __forceinline__ void ntt16_forward(uint32_t* v, uint32_t* buf, int t, int Lrt, int lgrt,
                                              const uint2* __restrict__ tw, const NttK& c) {
#pragma unroll
  for (int k = 8; k < 16; ++k) v[k] = 0u;
  const int L = LG ? (1 << LG) : Lrt, log2L = LG ? LG : lgrt;
  const int small = log2L & 3, n16 = log2L >> 2;
  int Ns = 1, q = 0;
  // the first pass (Ns = 1, no twiddles) sees the zero upper half
  if (small == 1) {
    ntt_pass<2, true, LG>(v, t, L, Ns, tw, c);
    ntt_exchange<2, LG>(v, buf, t, L, Ns);
    Ns = 2;
  } else if (small == 2) {
    ntt_pass<4, true, LG>(v, t, L, Ns, tw, c);
    ntt_exchange<4, LG>(v, buf, t, L, Ns);
    Ns = 4;
  } else if (small == 3) {
    ntt_pass<8, true, LG>(v, t, L, Ns, tw, c);
    ntt_exchange<8, LG>(v, buf, t, L, Ns);
    Ns = 8;
  } else {
    ntt_pass<16, true, LG>(v, t, L, Ns, tw, c);
    if (n16 > 1) ntt_exchange<16, LG>(v, buf, t, L, Ns);
    Ns = 16;
    q = 1;
  }
#pragma unroll 1
  for (; q < n16; ++q) {
    ntt_pass<16, false, LG>(v, t, L, Ns, tw, c);
    if (q + 1 < n16) ntt_exchange<16, LG>(v, buf, t, L, Ns);
    Ns <<= 4;
  }
}
// Inverse (unnormalised) from the forward's layout; positions < L/2 are read.
template <int LG = 0>
__device__ __forceinline__ void ntt16_inverse(uint32_t* v, uint32_t* buf, int t, int Lrt, int lgrt,
                                              const uint2* __restrict__ twi, const NttK& c) {
  const int L = LG ? (1 << LG) : Lrt, log2L = LG ? LG : lgrt;
  const int small = log2L & 3, n16 = log2L >> 2;
  int Ns = 1;
#pragma unroll 1
  for (int q = 0; q < n16; ++q) {
    ntt_pass<16, false, LG>(v, t, L, Ns, twi, c);
    if (q + 1 < n16 || small) ntt_exchange<16, LG>(v, buf, t, L, Ns);
    Ns <<= 4;
  }
  if (small == 1) ntt_pass<2, false, LG>(v, t, L, Ns, twi, c);
  else if (small == 2) ntt_pass<4, false, LG>(v, t, L, Ns, twi, c);
  else if (small == 3) ntt_pass<8, false, LG>(v, t, L, Ns, twi, c);
}

// x_q = trunc(|x| 2^(1077 - E)) for E >= the biased exponent of x (E >= 1):
// the 53-bit significand (e the biased exponent, taken as 1 for subnormals)
// times 2^(e - E + 2), below 2^55.
__device__ __forceinline__ uint64_t quantize(double x, int E) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  const unsigned long long mag = e ? (m | (1ull << 52)) : m;
  const int sh = E - (e ? e : 1) - 2;
  if (sh < 0) return mag << (-sh);
  return sh < 64 ? mag >> sh : 0ull;
}
__device__ __forceinline__ int biased_exponent(double x) {
  return (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FF);
}

// q mod p for q < 2^55 (negated when neg): q = h 2^32 + l, h < 2^23 < p.
template <int PI>
__device__ __forceinline__ uint32_t residue(uint64_t q, bool neg) {
  constexpr NttConstTable T = make_ntt_consts();
  constexpr uint32_t p = T.c[PI].p;
  const uint32_t r = addq(mulq((uint32_t)(q >> 32), T.c[PI].r32, T.c[PI].r32q, p),
                          mulq((uint32_t)q, 1u, T.c[PI].oneq, p), p);
  return (neg && r) ? p - r : r;
}

// Garner: the integer V with V = r_i mod p_i and |V| < P/2 (P = p0 p1 p2 p3),
// as a double times 2^scale (truncated to 53 bits).  V = a0 + p0 (a1 + p1 (a2 +
// p2 a3)), a_i in [0, p_i) from the residues; a3 > p3/2 means V < 0, and then
// V = a0 + p0 (a1 + p1 (a2 + p2 (a3 - p3))).
__device__ __forceinline__ double crt_to_double(uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3, int scale) {
  constexpr uint32_t p0 = kNttP[0], p1 = kNttP[1], p2 = kNttP[2], p3 = kNttP[3];
  constexpr uint32_t i01 = ntt_pow(p0 % p1, p1 - 2, p1), i01q = ntt_shoup(i01, p1);
  constexpr uint32_t i02 = ntt_pow(p0 % p2, p2 - 2, p2), i02q = ntt_shoup(i02, p2);
  constexpr uint32_t i12 = ntt_pow(p1 % p2, p2 - 2, p2), i12q = ntt_shoup(i12, p2);
  constexpr uint32_t i03 = ntt_pow(p0 % p3, p3 - 2, p3), i03q = ntt_shoup(i03, p3);
  constexpr uint32_t i13 = ntt_pow(p1 % p3, p3 - 2, p3), i13q = ntt_shoup(i13, p3);
  constexpr uint32_t i23 = ntt_pow(p2 % p3, p3 - 2, p3), i23q = ntt_shoup(i23, p3);
  static_assert(p0 > p1 && p1 > p2 && p2 > p3, "descending primes (a_i mod p_j by one subtraction)");
  const uint32_t a0 = r0;
  const uint32_t a1 = mulq(subq(r1, redq(a0, p1), p1), i01, i01q, p1);
  uint32_t u = mulq(subq(r2, redq(a0, p2), p2), i02, i02q, p2);
  const uint32_t a2 = mulq(subq(u, redq(a1, p2), p2), i12, i12q, p2);
  u = mulq(subq(r3, redq(a0, p3), p3), i03, i03q, p3);
  u = mulq(subq(u, redq(a1, p3), p3), i13, i13q, p3);
  const uint32_t a3 = mulq(subq(u, redq(a2, p3), p3), i23, i23q, p3);
  const bool neg = a3 > (p3 >> 1);
  const long long t2 = (long long)(neg ? (long long)a3 - (long long)p3 : (long long)a3) * p2 + a2;
  // magnitude (|t2| p1 +- a1) p0 +- a0, + for V >= 0 (t2 >= 0), - otherwise
  const unsigned long long m = (unsigned long long)(t2 < 0 ? -t2 : t2);
  unsigned long long lo = m * p1, hi = __umul64hi(m, (unsigned long long)p1);
  if (!neg) {
    const unsigned long long l2 = lo + a1;
    hi += l2 < lo;
    lo = l2;
  } else {
    hi -= lo < a1;
    lo -= a1;
  }
  unsigned long long h2 = __umul64hi(lo, (unsigned long long)p0) + hi * p0;
  lo *= p0;
  if (!neg) {
    const unsigned long long l2 = lo + a0;
    h2 += l2 < lo;
    lo = l2;
  } else {
    h2 -= lo < a0;
    lo -= a0;
  }
  hi = h2;
  if ((hi | lo) == 0ull) return 0.0;
  const int bl = hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)lo);  // bit length
  unsigned long long mant;
  if (bl > 53) {
    const int sh = bl - 53;
    mant = sh >= 64 ? hi >> (sh - 64) : (hi << (64 - sh)) | (lo >> sh);
  } else {
    mant = lo << (53 - bl);
  }
  const int be = bl - 1 + scale + 1023;  // biased exponent of the result
  if (be <= 0) return 0.0;
  const unsigned long long bits = ((unsigned long long)neg << 63) |
                                  ((unsigned long long)(be < 2047 ? be : 2047) << 52) |
                                  (be < 2047 ? (mant & 0xFFFFFFFFFFFFFull) : 0ull);
  return __longlong_as_double((long long)bits);
}

// Largest biased exponent over one group's values: shuffles over the lanes of
// this warp in the group (rows: G consecutive lanes; columns: lanes F apart),
// then the warps' maxima by a shared-memory atomic.  slot: this group's word,
// zero on entry.  Called by every thread of the block.
template <bool COLS>
__device__ __forceinline__ int group_max(int e, int* slot, int G, int F) {
  if (COLS) {
    for (int o = F; o < 32; o <<= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  } else {
    const int w = G < 32 ? G : 32;
    for (int o = 1; o < w; o <<= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  }
  atomicMax(slot, e);
  __syncthreads();
  const int r = *slot;
  __syncthreads();
  return r;
}

// Pass 1 of an exact Toeplitz product along rows (COLS = false) or columns:
// for prime PI, every vector's product modulo p at every position, into
// sc.res[PI] (the grid's layout), and (PI = 0) each vector's largest biased
// exponent E into sc.ebuf[vector] (2047: the vector holds an infinity or
// NaN).  One vector per group of L/16 threads; the block takes the vector
// groups grp0, grp0 + gstep, ...
template <int PI, bool COLS, int LG>
__device__ __forceinline__ void ntt_body(const double* __restrict__ x, const ExactScratch& sc, int n1, int n2,
                                         const ExactAxis& ax, int F, int gstride, int grp0, int gstep) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = LG ? (1 << LG) : ax.L, Lq = L >> 4, G = Lq;
  const GroupIdx gi = group_idx<COLS>(G, F);
  uint32_t* buf = reinterpret_cast<uint32_t*>(smem_raw) + (size_t)gi.g * gstride;
  int* slot = reinterpret_cast<int*>(buf);
  const int nvec = COLS ? n1 : n2, len = COLS ? n2 : n1;
  const int ngroups = (nvec + F - 1) / F;
  const uint2* tw = ax.tab + (size_t)3 * PI * L;
  uint32_t* __restrict__ res = sc.res[PI];
  for (int grp = grp0; grp < ngroups; grp += gstep) {
    const int vec = grp * F + gi.g;
    const bool has = vec < nvec;
    double xv[8];
    int e = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int pos = gi.t + k * Lq;
      xv[k] = (has && pos < len) ? x[vaddr<COLS>(vec, pos, n1)] : 0.0;
      e = max(e, biased_exponent(xv[k]));
    }
    if (gi.t == 0) slot[0] = 0;
    __syncthreads();
    const int E = group_max<COLS>(e, slot, G, F);
    if (PI == 0 && gi.t == 0 && has) sc.ebuf[vec] = E;
    const int Ee = E ? E : 1;
    uint32_t v[16];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = residue<PI>(quantize(xv[k], Ee), __double_as_longlong(xv[k]) < 0);
    {
      const NttK c = ntt_consts<PI, false>();
      ntt16_forward<LG>(v, buf, gi.t, L, ax.log2L, tw, c);
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const uint2 s = ld_tab(tw + 2 * L + gi.t + k * Lq);
        v[k] = mulq(v[k], s.x, s.y, c.p);
      }
    }
    ntt16_inverse<LG>(v, buf, gi.t, L, ax.log2L, tw + L, ntt_consts<PI, true>());
    if (has) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int pos = gi.t + k * Lq;
        if (pos < len) res[vaddr<COLS>(vec, pos, n1)] = v[k];
      }
    }
    __syncthreads();  // the next vector's exponent slot reuses the buffer
  }
}

// 64 registers: at least 32 warps per SM (the transforms wait on shared
// memory and the twiddle reads; at 16 warps they ran 1.3x longer)
template <bool COLS>
__global__ void __launch_bounds__(COLS ? 1024 : 512, COLS ? 1 : 2)
    ntt_kernel(const double* __restrict__ x, ExactScratch sc, int n1, int n2, ExactAxis ax, int F, int gstride,
               const int* gate) {
  if (gate_closed<double>(gate)) return;
  // the prime (uniform over the block), and the length 4096 (n 1025..2048) compiled apart
  if (ax.log2L == 12) {
    switch (blockIdx.y) {
      case 0: ntt_body<0, COLS, 12>(x, sc, n1, n2, ax, F, gstride, blockIdx.x, gridDim.x); break;
      case 1: ntt_body<1, COLS, 12>(x, sc, n1, n2, ax, F, gstride, blockIdx.x, gridDim.x); break;
      case 2: ntt_body<2, COLS, 12>(x, sc, n1, n2, ax, F, gstride, blockIdx.x, gridDim.x); break;
      default: ntt_body<3, COLS, 12>(x, sc, n1, n2, ax, F, gstride, blockIdx.x, gridDim.x); break;
    }
    return;
  }
  switch (blockIdx.y) {
    case 0: ntt_body<0, COLS, 0>(x, sc, n1, n2, ax, F, gstride, blockIdx.x, gridDim.x); break;
    case 1: ntt_body<1, COLS, 0>(x, sc, n1, n2, ax, F, gstride, blockIdx.x, gridDim.x); break;
    case 2: ntt_body<2, COLS, 0>(x, sc, n1, n2, ax, F, gstride, blockIdx.x, gridDim.x); break;
    default: ntt_body<3, COLS, 0>(x, sc, n1, n2, ax, F, gstride, blockIdx.x, gridDim.x); break;
  }
}

// Pass 2, elementwise over the grid: the product at p from its four residues
// (Garner), scaled by its vector's exponent, then the FP64 epilogue of
// toeplitz_body with T = double:
//   rows:  tmpx = x - A_x x + pen phi x
//   cols   MODE_RESID_ONLY: out = b - (tmpx - A_y x);  MODE_RESIDUAL: that,
//          and ||out||^2 by a fixed-order block sum per block and
//          block_sum_fixed over the blocks (the grid is a function of N), the
//          last block restarting the solver.
// (bid, nblk): this block's index in the pass's grid and the grid's size.
template <int MODE, bool COLS, typename Tout>
__device__ __forceinline__ void crt_body(const double* __restrict__ x, const ExactScratch& sc,
                                         double* __restrict__ tmpx, const uint8_t* __restrict__ phi, double pen,
                                         const double* __restrict__ b, Tout* __restrict__ out, int n1, int n2, int St,
                                         double* partials, SolverState* st, int bid, int nblk) {
  const size_t N = (size_t)n1 * n2;
  double acc = 0.0;
  for (size_t p = bid * (size_t)blockDim.x + threadIdx.x; p < N; p += (size_t)nblk * blockDim.x) {
    const int vec = COLS ? (int)(p % (size_t)n1) : (int)(p / (size_t)n1);
    const int E = __ldg(sc.ebuf + vec);
    const double az = E == 2047 ? __longlong_as_double(0x7FF8000000000000ll)
                                : crt_to_double(__ldg(sc.res[0] + p), __ldg(sc.res[1] + p), __ldg(sc.res[2] + p),
                                                __ldg(sc.res[3] + p), (E ? E : 1) - 1077 - St);
    if (!COLS) {
      const double xx = x[p];
      double sx = xx - az;
      if (phi[p]) sx = sx + pen * xx;
      tmpx[p] = sx;
    } else {
      const double r = b[p] - (tmpx[p] - az);
      out[p] = (Tout)r;
      if (MODE == MODE_RESIDUAL) acc += r * r;
    }
  }
  if constexpr (MODE == MODE_RESIDUAL) {
    __shared__ double sh[kBlock / 32];
    const double bs = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[bid] = bs;
    if (arrive_last(&st->counter, nblk)) {
      const double tot = block_sum_fixed(partials, nblk);
      if (threadIdx.x == 0) restart_prep(st, sqrt(tot));
    }
  }
}
template <int MODE, bool COLS, typename Tout>
__global__ void __launch_bounds__(kBlock)
    crt_kernel(const double* __restrict__ x, ExactScratch sc, double* __restrict__ tmpx,
               const uint8_t* __restrict__ phi, double pen, const double* __restrict__ b, Tout* __restrict__ out,
               int n1, int n2, int St, const int* gate, double* partials, SolverState* st) {
  if (gate_closed<double>(gate)) return;
  crt_body<MODE, COLS, Tout>(x, sc, tmpx, phi, pen, b, out, n1, n2, St, partials, st, blockIdx.x, gridDim.x);
}

// Groups per block (a power of two) of the transform kernel: at least 128
// threads per block; columns at least four groups (four adjacent columns
// fill a 32-byte sector of x); at most 1024 threads.
__host__ __device__ inline int exact_groups(int L, bool cols) {
  const int G = L >> 4;
  int F = G >= 128 ? 1 : 128 / G;
  if (cols && F < 4) F = 4;
  while (F > 1 && F * G > 1024) F >>= 1;
  return F;
}
// words per group exchange buffer: the padded exchange buffer (the largest
// padded index is L - 1 + (L - 1)/16), 16 mod 32 so that the buffers of
// neighbouring groups start half a bank row apart
__host__ __device__ inline int exact_stride(int L) {
  const int w = L + (L >> 4) + 1;
  return (w + 31) / 32 * 32 + 16;
}

}  // namespace rsfde
