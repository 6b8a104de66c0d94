// exact.cu -- host tables and launchers of the exact Toeplitz products of the
// true residual (the transforms and kernels are in exact.cuh).
#include <cmath>
#include <vector>

#include "exact.cuh"

namespace rsfde {

namespace {

uint32_t mulmod(uint32_t a, uint32_t b, uint32_t p) { return (uint32_t)((uint64_t)a * b % p); }

// Natural-order transform sum_j a_j w^(jk) mod p (iterative radix-2 after a
// bit-reversal permutation).
void host_ntt(std::vector<uint32_t>& a, uint32_t w, uint32_t p) {
  const int L = (int)a.size();
  for (int i = 1, j = 0; i < L; ++i) {
    int bit = L >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i], a[j]);
  }
  for (int len = 2; len <= L; len <<= 1) {
    const uint32_t wl = ntt_pow(w, (uint64_t)(L / len), p);
    for (int i = 0; i < L; i += len) {
      uint32_t wk = 1;
      for (int k = 0; k < len / 2; ++k) {
        const uint32_t u = a[i + k], v = mulmod(a[i + k + len / 2], wk, p);
        a[i + k] = (uint32_t)(((uint64_t)u + v) % p);
        a[i + k + len / 2] = (uint32_t)(((uint64_t)u + p - v) % p);
        wk = mulmod(wk, wl, p);
      }
    }
  }
}

uint2 with_shoup(uint32_t w, uint32_t p) { return make_uint2(w, ntt_shoup(w, p)); }

}  // namespace

std::vector<uint2> build_exact_tables(const std::vector<double>& t, int L, int* St) {
  const int n = (int)t.size();
  // largest St with T1_q = |t_q[0]| + 2 sum_{k>=1} |t_q[k]| < 2^63 (a bound on
  // every row's absolute sum), so that |sum_l t_q x_q| < 2^63 2^55 = 2^118,
  // below half the primes' product
  double t1 = std::fabs(t[0]);
  for (int k = 1; k < n; ++k) t1 += 2.0 * std::fabs(t[k]);
  std::vector<long long> tq(n, 0);
  *St = 0;
  if (t1 > 0.0) {
    for (int s = 62 - std::ilogb(t1);; --s) {
      unsigned __int128 sum = 0;
      for (int k = 0; k < n; ++k) {
        tq[k] = std::llround(std::ldexp(t[k], s));
        const unsigned long long a = (unsigned long long)(tq[k] < 0 ? -tq[k] : tq[k]);
        sum += (unsigned __int128)a * (k ? 2u : 1u);
      }
      if (sum < ((unsigned __int128)1 << 63)) {
        *St = s;
        break;
      }
    }
  }
  std::vector<uint2> out((size_t)kNttPrimes * 3 * L);
  for (int pi = 0; pi < kNttPrimes; ++pi) {
    const uint32_t p = kNttP[pi];
    const uint32_t w = ntt_pow(kNttG[pi], (uint64_t)(p - 1) / (uint64_t)L, p);
    const uint32_t wi = ntt_pow(w, (uint64_t)(p - 2), p);
    uint2* tw = out.data() + (size_t)pi * 3 * L;
    uint2* twi = tw + L;
    uint2* spec = twi + L;
    uint32_t a = 1, ai = 1;
    for (int m = 0; m < L; ++m) {
      tw[m] = with_shoup(a, p);
      twi[m] = with_shoup(ai, p);
      a = mulmod(a, w, p);
      ai = mulmod(ai, wi, p);
    }
    // circulant embedding of the symmetric Toeplitz column, residues mod p
    std::vector<uint32_t> c(L, 0u);
    auto res = [&](long long v) { return (uint32_t)(((v % (long long)p) + (long long)p) % (long long)p); };
    c[0] = res(tq[0]);
    for (int k = 1; k < n; ++k) c[k] = c[L - k] = res(tq[k]);
    host_ntt(c, w, p);
    const uint32_t linv = ntt_pow((uint32_t)L % p, (uint64_t)(p - 2), p);
    for (int k = 0; k < L; ++k) spec[k] = with_shoup(mulmod(c[k], linv, p), p);
  }
  return out;
}

template <typename K>
static void exact_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// The transform kernel for rows or columns: blockIdx.y is the prime.
template <bool COLS>
static void launch_ntt(const double* x, const ExactScratch& sc, int n1, int n2, const ExactAxis& ax,
                       const int* gate, cudaStream_t s) {
  const int nvec = COLS ? n1 : n2;
  const int F = exact_groups(ax.L, COLS), gs = exact_stride(ax.L);
  const size_t sm = (size_t)F * gs * sizeof(uint32_t);
  auto k = ntt_kernel<COLS>;
  exact_smem(k, sm);
  k<<<dim3((nvec + F - 1) / F, kNttPrimes), F * (ax.L / 16), sm, s>>>(x, sc, n1, n2, ax, F, gs, gate);
}

void launch_exact_rows(const double* x, double* tmpx, const uint8_t* phi, double pen, int n1, int n2,
                       const ExactAxis& ax, const ExactScratch& sc, const int* gate, cudaStream_t s) {
  launch_ntt<false>(x, sc, n1, n2, ax, gate, s);
  crt_kernel<MODE_APPLY, false, double><<<vec_grid((size_t)n1 * n2), kBlock, 0, s>>>(
      x, sc, tmpx, phi, pen, nullptr, nullptr, n1, n2, ax.St, gate, nullptr, nullptr);
}

template <typename Tout>
void launch_exact_cols(int mode, const double* x, double* tmpx, const uint8_t* phi, double pen, const double* b,
                       Tout* out, int n1, int n2, const ExactAxis& ay, const ExactScratch& sc, const int* gate,
                       double* partials, SolverState* st, cudaStream_t s) {
  ExactScratch sy = sc;
  sy.ebuf = sc.ebuf + n2;  // the rows' exponents stay apart
  const int grid = vec_grid((size_t)n1 * n2);
  if (mode == MODE_RESIDUAL) {
    launch_ntt<true>(x, sy, n1, n2, ay, gate, s);
    crt_kernel<MODE_RESIDUAL, true, Tout><<<grid, kBlock, 0, s>>>(x, sy, tmpx, phi, pen, b, out, n1, n2, ay.St,
                                                                  gate, partials, st);
    return;
  }
  if constexpr (std::is_same<Tout, double>::value) {
    if (mode == MODE_RESID_ONLY) {
      launch_ntt<true>(x, sy, n1, n2, ay, gate, s);
      crt_kernel<MODE_RESID_ONLY, true, double><<<grid, kBlock, 0, s>>>(x, sy, tmpx, phi, pen, b, out, n1, n2,
                                                                        ay.St, gate, partials, st);
      return;
    }
  }
  note_unsupported_launch();
}
// ---- the lock-step batch: every instance's residual in four launches --------
// Transforms: 256-thread blocks (the multi-instance transform width), F =
// 256 / (L/16) vector groups per block; each virtual block is one group of
// vectors for one prime.  The arithmetic of a vector does not depend on F, so
// the residues equal the single-instance launch's.
int exact_multi_ntt_blocks(int L, int nvec) {
  const int F = kMultiThreads / (L / 16);
  return (nvec + F - 1) / F * kNttPrimes;
}
template <bool COLS>
__global__ void __launch_bounds__(kMultiThreads, 3)
    ntt_multi_kernel(const BatchInst* __restrict__ bi, const int* __restrict__ prefix,
                     const int* __restrict__ active, int count, int* sched) {
  multi_loop(bi, prefix, active, count, [&](const BatchInst& I, int lb, int) {
    const ExactAxis& ax = COLS ? I.ey : I.ex;
    const int F = kMultiThreads / (ax.L / 16), gs = exact_stride(ax.L);
    const int ngroups = ((COLS ? I.n1 : I.n2) + F - 1) / F;
    const int prime = lb / ngroups, grp = lb - prime * ngroups;
    ExactScratch sc = I.esc;
    if (COLS) sc.ebuf += I.n2;  // the rows' exponents stay apart
    switch (prime) {  // uniform over the block
      case 0: ntt_body<0, COLS, 0>(I.x, sc, I.n1, I.n2, ax, F, gs, grp, ngroups); break;
      case 1: ntt_body<1, COLS, 0>(I.x, sc, I.n1, I.n2, ax, F, gs, grp, ngroups); break;
      case 2: ntt_body<2, COLS, 0>(I.x, sc, I.n1, I.n2, ax, F, gs, grp, ngroups); break;
      default: ntt_body<3, COLS, 0>(I.x, sc, I.n1, I.n2, ax, F, gs, grp, ngroups); break;
    }
  }, sched);
}
// Chinese remaindering and the FP64 epilogue (FP64 basis): rows write the
// scratch, columns b - (scratch - A_y x) into V_0 with the norm and restart.
template <bool COLS>
__global__ void __launch_bounds__(kBlock)
    crt_multi_kernel(const BatchInst* __restrict__ bi, const int* __restrict__ prefix,
                     const int* __restrict__ active, int count, int* sched) {
  multi_loop(bi, prefix, active, count, [&](const BatchInst& I, int lb, int nb) {
    ExactScratch sc = I.esc;
    if (COLS) {
      sc.ebuf += I.n2;
      crt_body<MODE_RESIDUAL, true, double>(I.x, sc, static_cast<double*>(I.tmpx), I.phi, I.pen, I.b, I.V, I.n1,
                                            I.n2, I.ey.St, I.partials, I.st, lb, nb);
    } else {
      crt_body<MODE_APPLY, false, double>(I.x, sc, static_cast<double*>(I.tmpx), I.phi, I.pen, nullptr, nullptr,
                                          I.n1, I.n2, I.ex.St, nullptr, nullptr, lb, nb);
    }
  }, sched);
}
// dynamic shared memory of a transform launch: the largest any of its lengths needs
static size_t exact_multi_smem(const MultiGrid& g) {
  size_t m = 0;
  for (int k = 4; k <= 12; ++k)
    if (g.l2mask & (1u << k)) {
      const int L = 1 << k;
      const size_t b = (size_t)(kMultiThreads / (L / 16)) * exact_stride(L) * sizeof(uint32_t);
      if (b > m) m = b;
    }
  return m;
}
void launch_exact_multi(const BatchInst* bi, const MultiGrid& nrows, const MultiGrid& crows, const MultiGrid& ncols,
                        const MultiGrid& ccols, cudaStream_t s) {
  auto nr = ntt_multi_kernel<false>;
  auto nc = ntt_multi_kernel<true>;
  auto cr = crt_multi_kernel<false>;
  auto cc = crt_multi_kernel<true>;
  const size_t sr = exact_multi_smem(nrows), sc = exact_multi_smem(ncols);
  exact_smem(nr, sr);
  exact_smem(nc, sc);
  nr<<<multi_launch_grid(nr, kMultiThreads, sr, nrows.total), kMultiThreads, sr, s>>>(bi, nrows.prefix, nrows.active,
                                                                                   nrows.count, nrows.sched);
  cr<<<multi_launch_grid(cr, kBlock, 0, crows.total), kBlock, 0, s>>>(bi, crows.prefix, crows.active, crows.count,
                                                                     crows.sched);
  nc<<<multi_launch_grid(nc, kMultiThreads, sc, ncols.total), kMultiThreads, sc, s>>>(bi, ncols.prefix, ncols.active,
                                                                                   ncols.count, ncols.sched);
  cc<<<multi_launch_grid(cc, kBlock, 0, ccols.total), kBlock, 0, s>>>(bi, ccols.prefix, ccols.active, ccols.count,
                                                                     ccols.sched);
}

template void launch_exact_cols<double>(int, const double*, double*, const uint8_t*, double, const double*,
                                        double*, int, int, const ExactAxis&, const ExactScratch&, const int*,
                                        double*, SolverState*, cudaStream_t);
template void launch_exact_cols<float>(int, const double*, double*, const uint8_t*, double, const double*, float*,
                                       int, int, const ExactAxis&, const ExactScratch&, const int*, double*,
                                       SolverState*, cudaStream_t);

}  // namespace rsfde
