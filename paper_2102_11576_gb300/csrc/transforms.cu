// transforms.cu -- the operator M (Eq. 2.14-2.17) and the preconditioner
// P-hat^-1 (Eq. 4.6) as shared-memory FFT kernels for sm_103a.
//
// Grid functions are x-fastest (u[j*n1 + i]).  Row kernels (x direction)
// read whole contiguous rows; column kernels (y direction) take a panel of
// adjacent columns so every global access is a run of consecutive addresses.
//
//  * Toeplitz product along an axis: two real vectors are packed as the real
//    and imaginary parts of one complex sequence (the circulant spectrum is
//    real because the Toeplitz matrix of Eq. 2.16 is symmetric), zero padded
//    to L, transformed, scaled by the spectrum and transformed back.
//  * Sine transform S_n (Section 4.1): with c_k = exp(i pi k^2/(2(n+1))) and
//    jk = (j^2 + k^2 - (k-j)^2)/2,  (S x)_k = sqrt(2/(n+1)) Im(c_k sum_j x_j c_j conj(c_{k-j})),
//    a convolution of length L >= 2n-1 (Bluestein).
//  * P-hat^-1 v = (I-Phi) S (I - Lx - Ly)^-1 S v + Phi S ((1+dt/eta) I - Lx - Ly)^-1 S v
//    (S = S_{n2} (x) S_{n1}; proof of Lemma 4.2) in three passes: rows S_x;
//    columns S_y, the two spectral divides and both inverse S_y; rows S_x
//    of both channels with the masked combine.
#include "common.cuh"
#include "fft.cuh"
#include "internal.h"

namespace rsfde {

template <typename T>
__device__ __forceinline__ void chirp_in(T x, const T* __restrict__ c, int k, T& re, T& im) {
  re = x * __ldg(c + 2 * k);
  im = x * __ldg(c + 2 * k + 1);
}
// Im(c_k * (yr + i yi))
template <typename T>
__device__ __forceinline__ T chirp_out_im(const T* __restrict__ c, int k, T yr, T yi) {
  return __ldg(c + 2 * k) * yi + __ldg(c + 2 * k + 1) * yr;
}

template <typename T>
__device__ __forceinline__ void spectral_mul_complex(T* re, T* im, int count, int L, const T* __restrict__ spec) {
  for (int t = threadIdx.x; t < count; t += blockDim.x) {
    const int l = t & (L - 1);
    const T sr = __ldg(spec + 2 * l), si = __ldg(spec + 2 * l + 1);
    const T ar = re[t], ai = im[t];
    re[t] = ar * sr - ai * si;
    im[t] = ar * si + ai * sr;
  }
  __syncthreads();
}

template <typename T>
__device__ __forceinline__ bool gate_closed(const int* gate) {
  return gate != nullptr && *(volatile const int*)gate == 0;
}

// ---------------------------------------------------------------------------
// (I (x) A_x) z for all rows, two rows per complex transform.
template <typename T, typename Tin>
__global__ void __launch_bounds__(kBlock) toeplitz_rows_kernel(const Tin* __restrict__ z, double* __restrict__ out,
                                                               int n1, int n2, AxisTables<T> ax, int B,
                                                               const int* gate) {
  if (gate_closed<T>(gate)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = ax.L;
  T* re = reinterpret_cast<T*>(smem_raw);
  T* im = re + (size_t)B * L;
  const int npairs = (n2 + 1) >> 1;
  const int ngroups = (npairs + B - 1) / B;
  for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const int p0 = grp * B;
    for (int b = 0; b < B; ++b) {
      const int r0 = 2 * (p0 + b), r1 = r0 + 1;
      for (int l = threadIdx.x; l < L; l += blockDim.x) {
        T a = T(0), c = T(0);
        if (l < n1 && r0 < n2) {
          a = T(z[(size_t)r0 * n1 + l]);
          if (r1 < n2) c = T(z[(size_t)r1 * n1 + l]);
        }
        re[b * L + l] = a;
        im[b * L + l] = c;
      }
    }
    __syncthreads();
    fft_dif(re, im, L, ax.log2L, B, ax.tw);
    for (int t = threadIdx.x; t < B * L; t += blockDim.x) {
      const T sg = __ldg(ax.sigma + (t & (L - 1)));
      re[t] *= sg;
      im[t] *= sg;
    }
    __syncthreads();
    ifft_dit(re, im, L, ax.log2L, B, ax.tw);
    for (int b = 0; b < B; ++b) {
      const int r0 = 2 * (p0 + b), r1 = r0 + 1;
      if (r0 >= n2) break;
      for (int l = threadIdx.x; l < n1; l += blockDim.x) {
        out[(size_t)r0 * n1 + l] = double(re[b * L + l]);
        if (r1 < n2) out[(size_t)r1 * n1 + l] = double(im[b * L + l]);
      }
    }
    __syncthreads();
  }
}

// (A_y (x) I) z over panels of 2B adjacent columns, fused with the rest of M:
//   MODE_APPLY:    out = z - tmpx - A_y z + (dt/eta) phi z
//   MODE_RESIDUAL: out = b - (z - tmpx - A_y z + (dt/eta) phi z), and
//                  ||out||^2 is reduced; the last block restarts the solver.
template <typename T, typename Tin, int MODE>
__global__ void __launch_bounds__(kBlock) toeplitz_cols_kernel(const Tin* __restrict__ z, const double* __restrict__ tmpx,
                                                               const uint8_t* __restrict__ phi, double pen,
                                                               const double* __restrict__ b, double* __restrict__ out,
                                                               int n1, int n2, AxisTables<T> ay, int B, const int* gate,
                                                               double* partials, SolverState* st) {
  if (gate_closed<T>(gate)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  const int L = ay.L;
  T* re = reinterpret_cast<T*>(smem_raw);
  T* im = re + (size_t)B * L;
  const int W = 2 * B;  // columns per panel
  const int ngroups = (n1 + W - 1) / W;
  double acc = 0.0;
  for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const int c0 = grp * W;
    for (int t = threadIdx.x; t < W * L; t += blockDim.x) {
      const int l = t / W, c = t - l * W;
      const int col = c0 + c;
      T v = T(0);
      if (l < n2 && col < n1) v = T(z[(size_t)l * n1 + col]);
      T* dst = (c & 1) ? im : re;
      dst[(c >> 1) * L + l] = v;
    }
    __syncthreads();
    fft_dif(re, im, L, ay.log2L, B, ay.tw);
    for (int t = threadIdx.x; t < B * L; t += blockDim.x) {
      const T sg = __ldg(ay.sigma + (t & (L - 1)));
      re[t] *= sg;
      im[t] *= sg;
    }
    __syncthreads();
    ifft_dit(re, im, L, ay.log2L, B, ay.tw);
    for (int t = threadIdx.x; t < W * n2; t += blockDim.x) {
      const int l = t / W, c = t - l * W;
      const int col = c0 + c;
      if (col < n1) {
        const size_t p = (size_t)l * n1 + col;
        const double ayz = double(((c & 1) ? im : re)[(c >> 1) * L + l]);
        const double zz = double(z[p]);
        const double w = zz - tmpx[p] - ayz + (phi[p] ? pen * zz : 0.0);
        if (MODE == MODE_APPLY) {
          out[p] = w;
        } else {
          const double r = b[p] - w;
          out[p] = r;
          acc += r * r;
        }
      }
    }
    __syncthreads();
  }
  if (MODE == MODE_RESIDUAL) {
    double bs = block_sum(acc, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = bs;
    if (arrive_last(&st->counter, gridDim.x)) {
      double tot = sum_partials(partials, gridDim.x, red);
      if (threadIdx.x == 0) restart_prep(st, sqrt(tot));
    }
  }
}

// ---------------------------------------------------------------------------
// Row sine transform:  out[j, :] = S_{n1} (scale * v[j, :]);  B rows at once.
template <typename T, typename Tout>
__global__ void __launch_bounds__(kBlock) dst_rows_kernel(const double* __restrict__ v, const double* vscale,
                                                          Tout* __restrict__ out, int n1, int n2,
                                                          AxisTables<T> ax, int B, const int* gate) {
  if (gate_closed<T>(gate)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = ax.L;
  T* re = reinterpret_cast<T*>(smem_raw);
  T* im = re + (size_t)B * L;
  const double sc = vscale ? *vscale : 1.0;
  const int ngroups = (n2 + B - 1) / B;
  for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const int r0 = grp * B;
    for (int bb = 0; bb < B; ++bb) {
      const int r = r0 + bb;
      for (int l = threadIdx.x; l < L; l += blockDim.x) {
        T xr = T(0), xi = T(0);
        if (l < n1 && r < n2) chirp_in(T(sc * v[(size_t)r * n1 + l]), ax.chirp, l, xr, xi);
        re[bb * L + l] = xr;
        im[bb * L + l] = xi;
      }
    }
    __syncthreads();
    fft_dif(re, im, L, ax.log2L, B, ax.tw);
    spectral_mul_complex(re, im, B * L, L, ax.bspec);
    ifft_dit(re, im, L, ax.log2L, B, ax.tw);
    for (int bb = 0; bb < B; ++bb) {
      const int r = r0 + bb;
      if (r >= n2) break;
      for (int l = threadIdx.x; l < n1; l += blockDim.x)
        out[(size_t)r * n1 + l] = Tout(chirp_out_im(ax.chirp_out, l, re[bb * L + l], im[bb * L + l]));
    }
    __syncthreads();
  }
}

// Column sine transform: out[:, i] = S_{n2} in[:, i]; panels of B columns.
template <typename T, typename Tin, typename Tout>
__global__ void __launch_bounds__(kBlock) dst_cols_kernel(const Tin* __restrict__ in, Tout* __restrict__ out, int n1,
                                                          int n2, AxisTables<T> ay, int B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = ay.L;
  T* re = reinterpret_cast<T*>(smem_raw);
  T* im = re + (size_t)B * L;
  const int ngroups = (n1 + B - 1) / B;
  for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const int c0 = grp * B;
    for (int t = threadIdx.x; t < B * L; t += blockDim.x) {
      const int l = t / B, c = t - l * B;
      const int col = c0 + c;
      T xr = T(0), xi = T(0);
      if (l < n2 && col < n1) chirp_in(T(in[(size_t)l * n1 + col]), ay.chirp, l, xr, xi);
      re[c * L + l] = xr;
      im[c * L + l] = xi;
    }
    __syncthreads();
    fft_dif(re, im, L, ay.log2L, B, ay.tw);
    spectral_mul_complex(re, im, B * L, L, ay.bspec);
    ifft_dit(re, im, L, ay.log2L, B, ay.tw);
    for (int t = threadIdx.x; t < B * n2; t += blockDim.x) {
      const int l = t / B, c = t - l * B;
      const int col = c0 + c;
      if (col < n1) out[(size_t)l * n1 + col] = Tout(chirp_out_im(ay.chirp_out, l, re[c * L + l], im[c * L + l]));
    }
    __syncthreads();
  }
}

// Preconditioner, column pass.  For each x-frequency i (a column of T1 = rows
// already sine-transformed): W = S_{n2} T1[:, i];
// W1 = W / (1 - lam_x[i] - lam_y[:]),  W2 = W / (1 + dt/eta - lam_x[i] - lam_y[:]);
// T2a[:, i] = S_{n2} W1,  T2b[:, i] = S_{n2} W2.  B columns, 2B buffers.
template <typename T>
__global__ void __launch_bounds__(kBlock) precond_cols_kernel(const T* __restrict__ T1, T* __restrict__ T2a,
                                                              T* __restrict__ T2b, int n1, int n2,
                                                              AxisTables<T> ay, const T* __restrict__ lamx, T pen,
                                                              int B, const int* gate) {
  if (gate_closed<T>(gate)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = ay.L;
  T* re = reinterpret_cast<T*>(smem_raw);
  T* im = re + (size_t)2 * B * L;
  T* reB = re + (size_t)B * L;  // second channel
  T* imB = im + (size_t)B * L;
  const int ngroups = (n1 + B - 1) / B;
  for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const int c0 = grp * B;
    for (int t = threadIdx.x; t < B * L; t += blockDim.x) {
      const int l = t / B, c = t - l * B;
      const int col = c0 + c;
      T xr = T(0), xi = T(0);
      if (l < n2 && col < n1) chirp_in(T1[(size_t)l * n1 + col], ay.chirp, l, xr, xi);
      re[c * L + l] = xr;
      im[c * L + l] = xi;
    }
    __syncthreads();
    fft_dif(re, im, L, ay.log2L, B, ay.tw);
    spectral_mul_complex(re, im, B * L, L, ay.bspec);
    ifft_dit(re, im, L, ay.log2L, B, ay.tw);
    for (int t = threadIdx.x; t < B * L; t += blockDim.x) {
      const int c = t / L, l = t - c * L;
      const int col = c0 + c;
      T ar = T(0), ai = T(0), br = T(0), bi = T(0);
      if (l < n2 && col < n1) {
        const T w = chirp_out_im(ay.chirp_out, l, re[t], im[t]);
        const T base = T(1) - __ldg(lamx + col) - __ldg(ay.lam + l);
        chirp_in(w / base, ay.chirp, l, ar, ai);
        chirp_in(w / (base + pen), ay.chirp, l, br, bi);
      }
      re[t] = ar;
      im[t] = ai;
      reB[t] = br;
      imB[t] = bi;
    }
    __syncthreads();
    fft_dif(re, im, L, ay.log2L, 2 * B, ay.tw);
    spectral_mul_complex(re, im, 2 * B * L, L, ay.bspec);
    ifft_dit(re, im, L, ay.log2L, 2 * B, ay.tw);
    for (int t = threadIdx.x; t < B * n2; t += blockDim.x) {
      const int l = t / B, c = t - l * B;
      const int col = c0 + c;
      if (col < n1) {
        const size_t p = (size_t)l * n1 + col;
        T2a[p] = chirp_out_im(ay.chirp_out, l, re[c * L + l], im[c * L + l]);
        T2b[p] = chirp_out_im(ay.chirp_out, l, reB[c * L + l], imB[c * L + l]);
      }
    }
    __syncthreads();
  }
}

// Preconditioner, final row pass:  z[j, :] = (1 - phi) S_{n1} T2a[j, :] + phi S_{n1} T2b[j, :].
template <typename T, typename Tz>
__global__ void __launch_bounds__(kBlock) precond_rows_kernel(const T* __restrict__ T2a, const T* __restrict__ T2b,
                                                              const uint8_t* __restrict__ phi, Tz* __restrict__ z,
                                                              int n1, int n2, AxisTables<T> ax, int B,
                                                              const int* gate) {
  if (gate_closed<T>(gate)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = ax.L;
  T* re = reinterpret_cast<T*>(smem_raw);
  T* im = re + (size_t)2 * B * L;
  T* reB = re + (size_t)B * L;
  T* imB = im + (size_t)B * L;
  const int ngroups = (n2 + B - 1) / B;
  for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const int r0 = grp * B;
    for (int bb = 0; bb < B; ++bb) {
      const int r = r0 + bb;
      for (int l = threadIdx.x; l < L; l += blockDim.x) {
        T ar = T(0), ai = T(0), br = T(0), bi = T(0);
        if (l < n1 && r < n2) {
          chirp_in(T2a[(size_t)r * n1 + l], ax.chirp, l, ar, ai);
          chirp_in(T2b[(size_t)r * n1 + l], ax.chirp, l, br, bi);
        }
        re[bb * L + l] = ar;
        im[bb * L + l] = ai;
        reB[bb * L + l] = br;
        imB[bb * L + l] = bi;
      }
    }
    __syncthreads();
    fft_dif(re, im, L, ax.log2L, 2 * B, ax.tw);
    spectral_mul_complex(re, im, 2 * B * L, L, ax.bspec);
    ifft_dit(re, im, L, ax.log2L, 2 * B, ax.tw);
    for (int bb = 0; bb < B; ++bb) {
      const int r = r0 + bb;
      if (r >= n2) break;
      for (int l = threadIdx.x; l < n1; l += blockDim.x) {
        const size_t p = (size_t)r * n1 + l;
        const T va = chirp_out_im(ax.chirp_out, l, re[bb * L + l], im[bb * L + l]);
        const T vb = chirp_out_im(ax.chirp_out, l, reB[bb * L + l], imB[bb * L + l]);
        z[p] = Tz(phi[p] ? vb : va);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Launchers.  The batch B of each kernel is the largest power of two whose
// buffers fit the shared-memory budget (capped so small grids still spread
// over the SMs).

static int pick_batch(int L, int elem_bytes, int buffers_per_item, int items) {
  const size_t per = (size_t)L * 2 * elem_bytes * buffers_per_item;
  int B = 1;
  while (B < 8 && per * (size_t)(2 * B) <= (size_t)kSmemBudget && 2 * B <= items) B *= 2;
  // keep at least ~2 groups per SM when the grid is small
  while (B > 1 && (items + B - 1) / B < 2 * kNumSMs) B /= 2;
  return B;
}

static int grid_for(int groups) { return groups < 1 ? 1 : groups; }

template <typename K>
static void set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, typename Tin>
void launch_toeplitz_rows(const Tin* z, double* out, int n1, int n2, const AxisTables<T>& ax, const int* gate,
                          cudaStream_t s) {
  const int npairs = (n2 + 1) / 2;
  const int B = pick_batch(ax.L, sizeof(T), 1, npairs);
  const size_t sm = (size_t)B * ax.L * 2 * sizeof(T);
  auto k = toeplitz_rows_kernel<T, Tin>;
  set_smem(k, sm);
  k<<<grid_for((npairs + B - 1) / B), kBlock, sm, s>>>(z, out, n1, n2, ax, B, gate);
}

template <typename T, typename Tin>
void launch_toeplitz_cols(int mode, const Tin* z, const double* tmpx, const uint8_t* phi, double pen,
                          const double* b, double* out, int n1, int n2, const AxisTables<T>& ay,
                          const int* gate, double* partials, SolverState* st, cudaStream_t s) {
  const int npairs = (n1 + 1) / 2;
  const int B = pick_batch(ay.L, sizeof(T), 1, npairs);
  const size_t sm = (size_t)B * ay.L * 2 * sizeof(T);
  int grid = grid_for((n1 + 2 * B - 1) / (2 * B));
  if (mode == MODE_APPLY) {
    auto k = toeplitz_cols_kernel<T, Tin, MODE_APPLY>;
    set_smem(k, sm);
    k<<<grid, kBlock, sm, s>>>(z, tmpx, phi, pen, b, out, n1, n2, ay, B, gate, partials, st);
  } else {
    if (grid > kMaxPartials) grid = kMaxPartials;
    auto k = toeplitz_cols_kernel<T, Tin, MODE_RESIDUAL>;
    set_smem(k, sm);
    k<<<grid, kBlock, sm, s>>>(z, tmpx, phi, pen, b, out, n1, n2, ay, B, gate, partials, st);
  }
}

template <typename T, typename Tout>
void launch_dst_rows(const double* v, const double* vscale, Tout* out, int n1, int n2, const AxisTables<T>& ax,
                     const int* gate, cudaStream_t s) {
  const int B = pick_batch(ax.L, sizeof(T), 1, n2);
  const size_t sm = (size_t)B * ax.L * 2 * sizeof(T);
  auto k = dst_rows_kernel<T, Tout>;
  set_smem(k, sm);
  k<<<grid_for((n2 + B - 1) / B), kBlock, sm, s>>>(v, vscale, out, n1, n2, ax, B, gate);
}

template <typename T, typename Tin, typename Tout>
void launch_dst_cols(const Tin* in, Tout* out, int n1, int n2, const AxisTables<T>& ay, cudaStream_t s) {
  const int B = pick_batch(ay.L, sizeof(T), 1, n1);
  const size_t sm = (size_t)B * ay.L * 2 * sizeof(T);
  auto k = dst_cols_kernel<T, Tin, Tout>;
  set_smem(k, sm);
  k<<<grid_for((n1 + B - 1) / B), kBlock, sm, s>>>(in, out, n1, n2, ay, B);
}

template <typename T>
void launch_precond_cols(const T* T1, T* T2a, T* T2b, int n1, int n2, const AxisTables<T>& ay, const T* lamx,
                         double pen, const int* gate, cudaStream_t s) {
  const int B = pick_batch(ay.L, sizeof(T), 2, n1);
  const size_t sm = (size_t)2 * B * ay.L * 2 * sizeof(T);
  auto k = precond_cols_kernel<T>;
  set_smem(k, sm);
  k<<<grid_for((n1 + B - 1) / B), kBlock, sm, s>>>(T1, T2a, T2b, n1, n2, ay, lamx, T(pen), B, gate);
}

template <typename T, typename Tz>
void launch_precond_rows(const T* T2a, const T* T2b, const uint8_t* phi, Tz* z, int n1, int n2,
                         const AxisTables<T>& ax, const int* gate, cudaStream_t s) {
  const int B = pick_batch(ax.L, sizeof(T), 2, n2);
  const size_t sm = (size_t)2 * B * ax.L * 2 * sizeof(T);
  auto k = precond_rows_kernel<T, Tz>;
  set_smem(k, sm);
  k<<<grid_for((n2 + B - 1) / B), kBlock, sm, s>>>(T2a, T2b, phi, z, n1, n2, ax, B, gate);
}

// explicit instantiations used by the solver
template void launch_toeplitz_rows<double, double>(const double*, double*, int, int, const AxisTables<double>&,
                                                   const int*, cudaStream_t);
template void launch_toeplitz_rows<double, float>(const float*, double*, int, int, const AxisTables<double>&,
                                                  const int*, cudaStream_t);
template void launch_toeplitz_cols<double, double>(int, const double*, const double*, const uint8_t*, double,
                                                   const double*, double*, int, int, const AxisTables<double>&,
                                                   const int*, double*, SolverState*, cudaStream_t);
template void launch_toeplitz_cols<double, float>(int, const float*, const double*, const uint8_t*, double,
                                                  const double*, double*, int, int, const AxisTables<double>&,
                                                  const int*, double*, SolverState*, cudaStream_t);
template void launch_dst_rows<double, double>(const double*, const double*, double*, int, int,
                                              const AxisTables<double>&, const int*, cudaStream_t);
template void launch_dst_rows<float, float>(const double*, const double*, float*, int, int,
                                            const AxisTables<float>&, const int*, cudaStream_t);
template void launch_dst_rows<double, float>(const double*, const double*, float*, int, int,
                                             const AxisTables<double>&, const int*, cudaStream_t);
template void launch_dst_cols<double, double, double>(const double*, double*, int, int, const AxisTables<double>&,
                                                      cudaStream_t);
template void launch_precond_cols<double>(const double*, double*, double*, int, int, const AxisTables<double>&,
                                          const double*, double, const int*, cudaStream_t);
template void launch_precond_cols<float>(const float*, float*, float*, int, int, const AxisTables<float>&,
                                         const float*, double, const int*, cudaStream_t);
template void launch_precond_rows<double, double>(const double*, const double*, const uint8_t*, double*, int, int,
                                                  const AxisTables<double>&, const int*, cudaStream_t);
template void launch_precond_rows<double, float>(const double*, const double*, const uint8_t*, float*, int, int,
                                                 const AxisTables<double>&, const int*, cudaStream_t);
template void launch_precond_rows<float, float>(const float*, const float*, const uint8_t*, float*, int, int,
                                                const AxisTables<float>&, const int*, cudaStream_t);
template void launch_precond_rows<float, double>(const float*, const float*, const uint8_t*, double*, int, int,
                                                 const AxisTables<float>&, const int*, cudaStream_t);

}  // namespace rsfde
