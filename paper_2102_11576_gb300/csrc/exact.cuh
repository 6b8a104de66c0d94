// exact.cuh -- the Toeplitz products of the true residual b - M x (Eq. 2.14-
// 2.17) computed exactly in integer arithmetic on GB300's integer pipes.
//
// GB300 executes FP64 at 1/64 of its FP32/INT32 rate, so an FP64 FFT of the
// residual is bound by the FP64 pipe.  Here each vector x (a row or a column
// of the grid) is scaled by a power of two to integers below 2^52 in
// magnitude (x_q = trunc(x 2^(1074-E)), E the largest biased exponent in the
// vector), the Toeplitz column t likewise on the host (t_q = round(t 2^St),
// |t_q| < 2^52), and the convolution sum_l t_q[|i-l|] x_q[l] -- an integer
// below n 2^104 <= 2^116 in magnitude for n <= 4096 -- is computed exactly
// modulo four primes p < 2^30 (product ~2^120) by number-theoretic transforms
// of length L >= 2n-1, then reconstructed by Garner's mixed-radix form of the
// Chinese remainder theorem and scaled back to FP64 (truncated to 53 bits).
// The product's only errors are the two quantisations (|x - x_q 2^(E-1074)|
// < 2^-51 max|x|, t likewise) and the final truncation: smaller than the
// rounding of an FP64 FFT, whose error grows with log2 L.  What follows the
// product (z - A_x z + (dt/eta) phi z, b - ..., ||r||^2) is FP64 arithmetic.
//
// Transforms: the register-resident Stockham layout of fft16.cuh (a group of
// L/16 threads, thread t holding positions t + k L/16), with values in
// [0, p), Shoup's multiplication by precomputed constants (w, floor(w 2^32 /
// p)) and radix-16/8/4/2 butterflies whose internal roots of unity are
// compile-time constants of each prime.  NTT_p(x)[k] = sum_j x_j w^(jk) with
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

// times W16^K (forward) or W16^-K (inverse), W16 = g^((p-1)/16) = w^(L/16)
template <int PI, bool INV, int K>
__device__ __forceinline__ uint32_t nrot(uint32_t a) {
  constexpr uint32_t p = kNttP[PI];
  constexpr uint32_t w16 = ntt_pow(kNttG[PI], (p - 1) / 16, p);
  constexpr uint32_t w = ntt_pow(w16, INV ? (16 - K) % 16 : K, p);
  constexpr uint32_t wq = ntt_shoup(w, p);
  return mulq(a, w, wq, p);
}

// Natural-order DFTs over Z_p on v[0], v[S], ..., v[(R-1)S] (the factorings of
// fft16.cuh with W4 = W16^4 in place of -i).
template <int PI, bool INV, int S>
__device__ __forceinline__ void ndft2(uint32_t* v) {
  constexpr uint32_t p = kNttP[PI];
  const uint32_t a = v[0], b = v[S];
  v[0] = addq(a, b, p);
  v[S] = subq(a, b, p);
}
template <int PI, bool INV, int S>
__device__ __forceinline__ void ndft4(uint32_t* v) {
  constexpr uint32_t p = kNttP[PI];
  const uint32_t t0 = addq(v[0], v[2 * S], p), t1 = subq(v[0], v[2 * S], p);
  const uint32_t t2 = addq(v[S], v[3 * S], p), t3 = nrot<PI, INV, 4>(subq(v[S], v[3 * S], p));
  v[0] = addq(t0, t2, p);
  v[2 * S] = subq(t0, t2, p);
  v[S] = addq(t1, t3, p);
  v[3 * S] = subq(t1, t3, p);
}
template <int PI, bool INV, int S>
__device__ __forceinline__ void ndft8(uint32_t* v) {
  constexpr uint32_t p = kNttP[PI];
  ndft4<PI, INV, 2 * S>(v);
  ndft4<PI, INV, 2 * S>(v + S);
  v[3 * S] = nrot<PI, INV, 2>(v[3 * S]);
  v[5 * S] = nrot<PI, INV, 4>(v[5 * S]);
  v[7 * S] = nrot<PI, INV, 6>(v[7 * S]);
  uint32_t o[8];
#pragma unroll
  for (int r1 = 0; r1 < 4; ++r1) {
    o[r1] = addq(v[2 * r1 * S], v[(2 * r1 + 1) * S], p);
    o[r1 + 4] = subq(v[2 * r1 * S], v[(2 * r1 + 1) * S], p);
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) v[r * S] = o[r];
}
template <int PI, bool INV>
__device__ __forceinline__ void ndft16(uint32_t* v) {
  ndft4<PI, INV, 4>(v);
  ndft4<PI, INV, 4>(v + 1);
  ndft4<PI, INV, 4>(v + 2);
  ndft4<PI, INV, 4>(v + 3);
  v[5] = nrot<PI, INV, 1>(v[5]);
  v[9] = nrot<PI, INV, 2>(v[9]);
  v[13] = nrot<PI, INV, 3>(v[13]);
  v[6] = nrot<PI, INV, 2>(v[6]);
  v[10] = nrot<PI, INV, 4>(v[10]);
  v[14] = nrot<PI, INV, 6>(v[14]);
  v[7] = nrot<PI, INV, 3>(v[7]);
  v[11] = nrot<PI, INV, 6>(v[11]);
  v[15] = nrot<PI, INV, 9>(v[15]);
  ndft4<PI, INV, 1>(v);
  ndft4<PI, INV, 1>(v + 4);
  ndft4<PI, INV, 1>(v + 8);
  ndft4<PI, INV, 1>(v + 12);
  uint32_t o[16];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) o[a + 4 * b] = v[4 * a + b];
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = o[r];
}
template <int PI, bool INV, int R, int S>
__device__ __forceinline__ void ndft_r(uint32_t* v) {
  if (R == 16) ndft16<PI, INV>(v);
  else if (R == 8) ndft8<PI, INV, S>(v);
  else if (R == 4) ndft4<PI, INV, S>(v);
  else ndft2<PI, INV, S>(v);
}

// One Stockham pass (the index arithmetic of fft_pass); tw: {w^m, Shoup} of
// the forward (w) or inverse (w^-1) root.
template <int PI, bool INV, int R>
__device__ __forceinline__ void ntt_pass(uint32_t* v, int t, int L, int Ns, const uint2* __restrict__ tw) {
  constexpr uint32_t p = kNttP[PI];
  constexpr int S = 16 / R;
  const int Lq = L >> 4;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    if (Ns > 1) {
      const int j = t + i * Lq;
      const int step = (j & (Ns - 1)) * (L / (Ns * R));
#pragma unroll
      for (int q = 1; q < R; ++q) {
        const uint2 w = __ldg(tw + q * step);
        v[i + q * S] = mulq(v[i + q * S], w.x, w.y, p);
      }
    }
    ndft_r<PI, INV, R, S>(v + i);
  }
}

template <int R>
__device__ __forceinline__ void ntt_exchange(uint32_t* v, uint32_t* buf, int t, int L, int Ns) {
  constexpr int S = 16 / R;
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
template <int PI>
__device__ __forceinline__ void ntt16_forward(uint32_t* v, uint32_t* buf, int t, int L, int log2L,
                                              const uint2* __restrict__ tw) {
#pragma unroll
  for (int k = 8; k < 16; ++k) v[k] = 0u;
  const int small = log2L & 3, n16 = log2L >> 2;
  int Ns = 1;
  if (small == 1) {
    ntt_pass<PI, false, 2>(v, t, L, Ns, tw);
    ntt_exchange<2>(v, buf, t, L, Ns);
    Ns = 2;
  } else if (small == 2) {
    ntt_pass<PI, false, 4>(v, t, L, Ns, tw);
    ntt_exchange<4>(v, buf, t, L, Ns);
    Ns = 4;
  } else if (small == 3) {
    ntt_pass<PI, false, 8>(v, t, L, Ns, tw);
    ntt_exchange<8>(v, buf, t, L, Ns);
    Ns = 8;
  }
  for (int q = 0; q < n16; ++q) {
    ntt_pass<PI, false, 16>(v, t, L, Ns, tw);
    if (q + 1 < n16) ntt_exchange<16>(v, buf, t, L, Ns);
    Ns <<= 4;
  }
}
// Inverse (unnormalised) from the forward's layout; positions < L/2 are read.
template <int PI>
__device__ __forceinline__ void ntt16_inverse(uint32_t* v, uint32_t* buf, int t, int L, int log2L,
                                              const uint2* __restrict__ twi) {
  const int small = log2L & 3, n16 = log2L >> 2;
  int Ns = 1;
  for (int q = 0; q < n16; ++q) {
    ntt_pass<PI, true, 16>(v, t, L, Ns, twi);
    if (q + 1 < n16 || small) ntt_exchange<16>(v, buf, t, L, Ns);
    Ns <<= 4;
  }
  if (small == 1) ntt_pass<PI, true, 2>(v, t, L, Ns, twi);
  else if (small == 2) ntt_pass<PI, true, 4>(v, t, L, Ns, twi);
  else if (small == 3) ntt_pass<PI, true, 8>(v, t, L, Ns, twi);
}

// x_q = trunc(|x| 2^(1074 - E)) with E >= the biased exponent of x (E >= 1):
// the significand shifted right by E - e + 1 (e the biased exponent, taken
// as 1 for subnormals), below 2^52.
__device__ __forceinline__ uint64_t quantize(double x, int E) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  const unsigned long long mag = e ? (m | (1ull << 52)) : m;
  const int sh = E - (e ? e : 1) + 1;
  return sh < 64 ? mag >> sh : 0ull;
}
__device__ __forceinline__ int biased_exponent(double x) {
  return (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FF);
}

// q mod p for q < 2^52 (negated when neg): q = h 2^32 + l, h < 2^20.
template <int PI>
__device__ __forceinline__ uint32_t residue(uint64_t q, bool neg) {
  constexpr uint32_t p = kNttP[PI];
  constexpr uint32_t r32 = (uint32_t)((1ull << 32) % p);
  constexpr uint32_t r32q = ntt_shoup(r32, p), oneq = ntt_shoup(1u, p);
  const uint32_t r = addq(mulq((uint32_t)(q >> 32), r32, r32q, p), mulq((uint32_t)q, 1u, oneq, p), p);
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

// The residues mod prime PI of the Toeplitz product of one vector at the
// thread's output positions t + k L/16 (k < 8): transform, times the scaled
// spectrum of the quantised Toeplitz column, inverse transform.
template <int PI>
__device__ __forceinline__ void ntt_conv(const uint64_t* xq, unsigned negmask, uint32_t* buf, int t,
                                         const ExactAxis& ax, uint32_t* out) {
  constexpr uint32_t p = kNttP[PI];
  uint32_t v[16];
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = residue<PI>(xq[k], (negmask >> k) & 1u);
  ntt16_forward<PI>(v, buf, t, ax.L, ax.log2L, ax.tw[PI]);
  const int Lq = ax.L >> 4;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const uint2 s = __ldg(ax.spec[PI] + t + k * Lq);
    v[k] = mulq(v[k], s.x, s.y, p);
  }
  ntt16_inverse<PI>(v, buf, t, ax.L, ax.log2L, ax.twi[PI]);
#pragma unroll
  for (int k = 0; k < 8; ++k) out[k] = v[k];
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

// Exact Toeplitz pass over an FP64 vector field (rows: COLS = false; columns:
// COLS = true); two vectors (a, a+1) per group, one after the other, as in
// toeplitz_body, whose modes and epilogues this follows with T = double:
//   rows  MODE_RAW: tmpx = A_x x;  other modes: tmpx = x - A_x x + pen phi x
//   cols  MODE_RAW: out = A_y x;  MODE_APPLY: out = tmpx - A_y x;
//         MODE_RESID_ONLY: out = b - (tmpx - A_y x);  MODE_RESIDUAL: that and
//         ||out||^2 per column pair by a fixed tree, the last block summing
//         the pairs in order and restarting the solver.
// A vector holding an infinity or NaN yields NaN products.
template <int MODE, bool COLS, typename Tout>
__device__ __forceinline__ void exact_body(const double* __restrict__ x, double* __restrict__ tmpx,
                                           const uint8_t* __restrict__ phi, double pen,
                                           const double* __restrict__ b, Tout* __restrict__ out, int n1, int n2,
                                           const ExactAxis& ax, int F, int gstride, const int* gate,
                                           double* partials, SolverState* st, int bid, int nblk) {
  if (gate_closed<double>(gate)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = ax.L, Lq = L >> 4, G = Lq;
  const GroupIdx gi = group_idx<COLS>(G, F);
  uint32_t* buf = reinterpret_cast<uint32_t*>(smem_raw) + (size_t)gi.g * gstride;
  int* slot = reinterpret_cast<int*>(buf);
  const int nvec = COLS ? n1 : n2, len = COLS ? n2 : n1;
  const int npairs = (nvec + 1) >> 1;
  const int ngroups = (npairs + F - 1) / F;
  for (int grp = bid; grp < ngroups; grp += nblk) {
    const int pr = grp * F + gi.g;
    const int a = 2 * pr;
    const bool live = pr < npairs;
    const bool second = a + 1 < nvec;
    double acc = 0.0;
    for (int h = 0; h < 2; ++h) {  // uniform over the block (every group runs both)
      const bool has = live && (h == 0 || second);
      double xv[8];
      int e = 0;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int pos = gi.t + k * Lq;
        xv[k] = (has && pos < len) ? x[vaddr<COLS>(a + h, pos, n1)] : 0.0;
        e = max(e, biased_exponent(xv[k]));
      }
      if (gi.t == 0) slot[0] = 0;
      __syncthreads();
      const int E = group_max<COLS>(e, slot, G, F);
      const int Ee = E ? E : 1;
      uint64_t xq[8];
      unsigned negm = 0;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        xq[k] = quantize(xv[k], Ee);
        negm |= (unsigned)(__double_as_longlong(xv[k]) < 0) << k;
      }  // (x is read again in the epilogue: an L1 or L2 hit)
      uint32_t res[4][8];
      ntt_conv<0>(xq, negm, buf, gi.t, ax, res[0]);
      ntt_conv<1>(xq, negm, buf, gi.t, ax, res[1]);
      ntt_conv<2>(xq, negm, buf, gi.t, ax, res[2]);
      ntt_conv<3>(xq, negm, buf, gi.t, ax, res[3]);
      __syncthreads();  // the next vector's exponent slot reuses the buffer
      if (!has) continue;
      const int scale = Ee - 1074 - ax.St;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int pos = gi.t + k * Lq;
        if (pos >= len) continue;
        const double az = E == 2047 ? __longlong_as_double(0x7FF8000000000000ll)
                                    : crt_to_double(res[0][k], res[1][k], res[2][k], res[3][k], scale);
        const size_t p = vaddr<COLS>(a + h, pos, n1);
        if (!COLS) {
          if (MODE == MODE_RAW) {
            tmpx[p] = az;
          } else {
            const double xx = x[p];
            double sx = xx - az;
            if (phi[p]) sx = sx + pen * xx;
            tmpx[p] = sx;
          }
        } else {
          const double w = MODE == MODE_RAW ? az : tmpx[p] - az;
          if (MODE == MODE_RAW || MODE == MODE_APPLY) {
            out[p] = (Tout)w;
          } else if (MODE == MODE_RESID_ONLY) {
            out[p] = (Tout)(b[p] - w);
          } else {
            const double r = b[p] - w;
            out[p] = (Tout)r;
            acc += r * r;
          }
        }
      }
    }
    if constexpr (MODE == MODE_RESIDUAL) {
      double* gsum = reinterpret_cast<double*>(buf);
      __syncthreads();
      gsum[gi.t] = acc;
      __syncthreads();
      for (int hh = G >> 1; hh > 0; hh >>= 1) {
        if (gi.t < hh) gsum[gi.t] += gsum[gi.t + hh];
        __syncthreads();
      }
      if (gi.t == 0 && live) partials[pr] = gsum[0];
      __syncthreads();
    }
  }
  if constexpr (MODE == MODE_RESIDUAL) {
    if (arrive_last(&st->counter, nblk)) {
      const double tot = block_sum_fixed(partials, npairs);
      if (threadIdx.x == 0) restart_prep(st, sqrt(tot));
    }
  }
}

template <int MODE, bool COLS, typename Tout>
__global__ void __launch_bounds__(512)
    exact_kernel(const double* __restrict__ x, double* __restrict__ tmpx, const uint8_t* __restrict__ phi,
                 double pen, const double* __restrict__ b, Tout* __restrict__ out, int n1, int n2, ExactAxis ax,
                 int F, int gstride, const int* gate, double* partials, SolverState* st) {
  exact_body<MODE, COLS, Tout>(x, tmpx, phi, pen, b, out, n1, n2, ax, F, gstride, gate, partials, st, blockIdx.x,
                               gridDim.x);
}

// Groups per block (a power of two): at least 128 threads per block, columns
// at least two groups (two adjacent column pairs fill a 32-byte sector), at
// most 512 threads.
__host__ __device__ inline int exact_groups(int L, bool cols) {
  const int G = L >> 4;
  int F = G >= 128 ? 1 : 128 / G;
  if (cols && F < 2) F = 2;
  while (F > 1 && F * G > 512) F >>= 1;
  return F;
}
// words per group buffer: the padded exchange buffer, odd so that the groups'
// buffers start in different banks; at least G doubles for the norm tree
__host__ __device__ inline int exact_stride(int L) {
  const int w = L + (L >> 4) + 1;
  return w | 1;
}

}  // namespace rsfde
