// common.cuh -- shared types of the GB300 solver library (internal).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rsfde {

constexpr int kMaxRestart = 64;  // largest m of FGMRES(m)

// Programmatic dependent launch (the BF16 preconditioner's split and GEMM
// chain).  A kernel launched by launch_pdl may be scheduled while the previous
// kernel in the stream (or graph) still runs; it must call pdl_wait() before
// touching memory, which returns once that grid has completed and its writes
// are visible (a no-op after an ordinary launch).  pdl_trigger() lets the next
// kernel be scheduled as soon as every block of this grid has issued it (all of
// them are then resident).  Measured: it hides the launch gaps of the GEMM
// chain; issued by the transform and Gram-Schmidt kernels too, the early
// trigger made the graph-replayed step ~4 % slower, so those launch normally.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k, args...);  // errors surface through cudaGetLastError
}
constexpr int kBlock = 256;      // threads per block of the grid-vector kernels

// Device-resident control state of one FGMRES solve.  Every kernel of an
// Arnoldi iteration is gated by run_iter, every cycle-end kernel by
// run_cycle, so a whole cycle can be enqueued (or replayed as a graph)
// without the host reading anything between iterations.
struct SolverState {
  int run_iter;   // 1 while the current cycle keeps iterating
  int run_cycle;  // 1 until the solve is finished
  int status;     // 0, or RSFDE_ENOTCONV / RSFDE_ENONFINITE
  int converged;
  int jlast;      // Arnoldi columns built in the current cycle
  int iters, cycles, max_iter, m;
  int zero_solution;  // b == 0: x must be zeroed
  int body_runs;      // FGMRES cycles replayed by the device-side graph loop (this solve)
  long long total_body_runs;  // the same over the context's lifetime (never reset)
  long long sum_j;            // sum of the Arnoldi column index j over the solve's iterations
  unsigned int counter;  // arrivals for the last-block reductions
  unsigned int pad;
  double tol, bnorm, beta, rel_res;
  double s[kMaxRestart + 1];  // v_i = s_i * V_i (normalisation deferred into the readers)
  double H[(kMaxRestart + 1) * kMaxRestart];  // rotated Hessenberg, H[i*kMaxRestart + j]
  double hcol[kMaxRestart + 1];
  double cs[kMaxRestart], sn[kMaxRestart], g[kMaxRestart + 1], y[kMaxRestart];
};

// Per-axis tables of one precision T (double or float), all device pointers.
// L is the power-of-two convolution length >= 2n-1 used by both transforms.
template <typename T>
struct AxisTables {
  int n, L, log2L;
  const T* tw;         // 2L: cos, sin of -2 pi j/L
  const T* sigma;      // L: circulant spectrum of the Toeplitz column / L, natural order
  const T* chirp;      // 2n: exp(i pi k^2 / (2(n+1))), k = 1..n
  const T* chirp_out;  // 2n: sqrt(2/(n+1)) exp(i pi k^2 / (2(n+1)))
  const T* bspec;      // 2L: spectrum of exp(-i pi d^2/(2(n+1))) / L, natural order
  const T* lam;        // n: eigenvalues of tau(A_axis)
};

// Tables of the exact Toeplitz product along one axis (exact.cuh): for each of
// the four primes i, at tab + 3 i L: the L Stockham twiddles of w =
// g^((p-1)/L), then those of w^-1, then the transform of the quantised
// circulant column times L^-1 (natural order); each entry {value, Shoup
// companion floor(value 2^32 / p)}.
struct ExactAxis {
  int n, L, log2L;
  int St;  // the Toeplitz column was quantised as round(t 2^St), |t_q| < 2^52
  const uint2* tab;
};
// Scratch of an exact Toeplitz pass: the product's residues modulo each prime
// (N words each, the grid's layout) and each vector's exponent.
struct ExactScratch {
  uint32_t* res[4];
  int* ebuf;
};

__device__ __forceinline__ double block_sum(double v, double* sh) {
  if (blockDim.x < 32) {  // blocks smaller than a warp (tiny grids): serial sum in a fixed order
    sh[threadIdx.x] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
      for (int i = 0; i < (int)blockDim.x; ++i) s += sh[i];
    __syncthreads();
    return s;  // valid in thread 0
  }
  // blockDim.x is a multiple of 32 here
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (w == 0) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  __syncthreads();
  return v;  // valid in thread 0
}

// Last-block-done pattern: returns true in exactly one block, after every
// block has published its partial results.  That block resets the counter.
__device__ __forceinline__ bool arrive_last(unsigned int* counter, unsigned int total) {
  __shared__ int is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int prev = atomicAdd(counter, 1u);
    is_last = (prev == total - 1);
    if (is_last) *counter = 0;
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last != 0;
}

// Sum of the `count` values p[0..count) by one warp in an order fixed by count
// alone (lane 0 returns it): each lane takes every 32nd value, sixteen loads
// in flight before they are added into four fixed accumulators, then a fixed
// butterfly over the lanes.
__device__ __forceinline__ double warp_sum_fixed(const double* p, int count) {
  const int l = threadIdx.x & 31;
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  for (int q0 = l; q0 < count; q0 += 16 * 32) {
    double t[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int q = q0 + 32 * k;
      t[k] = q < count ? __ldcg(p + q) : 0.0;
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k & 3] += t[k];
  }
  double v = (a[0] + a[1]) + (a[2] + a[3]);
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// The same sum for a block of any size: a block narrower than a warp (tiny
// grids) runs the warp's lanes and butterfly one after another in thread 0,
// in the identical order, so the value never depends on the block size.
// Valid in thread 0; every thread of the block must call it.
__device__ __forceinline__ double block_sum_fixed(const double* p, int count) {
  double v = 0.0;
  if (blockDim.x >= 32) {
    if (threadIdx.x < 32) v = warp_sum_fixed(p, count);
    return v;
  }
  if (threadIdx.x != 0) return 0.0;
  double s[32];
  for (int l = 0; l < 32; ++l) {
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int q0 = l; q0 < count; q0 += 16 * 32)
      for (int k = 0; k < 16; ++k) {
        const int q = q0 + 32 * k;
        a[k & 3] += q < count ? __ldcg(p + q) : 0.0;
      }
    s[l] = (a[0] + a[1]) + (a[2] + a[3]);
  }
  for (int o = 16; o; o >>= 1) {
    double t[32];
    for (int l = 0; l < 32; ++l) t[l] = s[l] + s[l ^ o];
    for (int l = 0; l < 32; ++l) s[l] = t[l];
  }
  return s[0];
}

// Deterministic sum of `count` partials (fixed order for a fixed count).
__device__ __forceinline__ double sum_partials(const double* p, int count, double* sh) {
  double v = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) v += __ldcg(p + i);
  return block_sum(v, sh);
}

}  // namespace rsfde
