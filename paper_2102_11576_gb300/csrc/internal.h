// internal.h -- declarations shared by the library's translation units.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/rsfde.h"
#include "common.cuh"
#include "df.cuh"

namespace rsfde {

constexpr int kNumSMs = 152;              // GB300: 2 dies x 76 SMs
constexpr int kSmemBudget = 200 * 1024;   // dynamic shared memory per block we allow
constexpr int kMaxPartials = 4096;        // per-block partial sums of one reduction
constexpr int kDotChunk = 8;              // basis vectors per block row of the multi-dot
constexpr int MODE_APPLY = 0;
constexpr int MODE_RESIDUAL = 1;
constexpr int MODE_RAW = 2;         // column pass writes A_y z alone
constexpr int MODE_RESID_ONLY = 3;  // column pass writes b - M z, no reduction

// ---- device-side solver control (single thread) ---------------------------
// Called by the last block of the true-residual kernel with beta = ||b - M x||:
// either finishes the solve or starts the next FGMRES cycle with v_0 = r / beta.
__device__ __forceinline__ void restart_prep(SolverState* st, double beta) {
  st->beta = beta;
  st->jlast = 0;
  if (st->bnorm == 0.0) {  // b = 0: the solution is x = 0
    st->zero_solution = 1;
    st->converged = 1;
    st->rel_res = 0.0;
    st->run_cycle = 0;
    st->run_iter = 0;
    return;
  }
  st->rel_res = beta / st->bnorm;
  if (!isfinite(beta) || !isfinite(st->bnorm)) {
    st->status = RSFDE_ENONFINITE;
    st->run_cycle = 0;
    st->run_iter = 0;
    return;
  }
  if (beta <= st->tol * st->bnorm) {
    st->converged = 1;
    st->run_cycle = 0;
    st->run_iter = 0;
    return;
  }
  if (st->iters >= st->max_iter) {
    st->status = RSFDE_ENOTCONV;
    st->run_cycle = 0;
    st->run_iter = 0;
    return;
  }
  st->s[0] = 1.0 / beta;
  st->g[0] = beta;
  for (int i = 1; i <= st->m; ++i) st->g[i] = 0.0;
  st->run_iter = 1;
  st->cycles += 1;
}

// Arnoldi column j is complete (H[0..j][j] and hnorm = H[j+1][j]): apply the
// stored Givens rotations, form the new one, update g and decide whether the
// cycle goes on (Section 5: GMRES with restart).
__device__ __forceinline__ void givens_step(SolverState* st, int j, double hnorm) {
  constexpr int KM = kMaxRestart;
  double* H = st->H;
  H[(j + 1) * KM + j] = hnorm;
  for (int i = 0; i < j; ++i) {
    const double a = H[i * KM + j], b = H[(i + 1) * KM + j];
    H[i * KM + j] = st->cs[i] * a + st->sn[i] * b;
    H[(i + 1) * KM + j] = -st->sn[i] * a + st->cs[i] * b;
  }
  const double a = H[j * KM + j], b = hnorm;
  double c = 1.0, s = 0.0;
  if (b != 0.0) {
    const double r = hypot(a, b);
    c = a / r;
    s = b / r;
  }
  st->cs[j] = c;
  st->sn[j] = s;
  H[j * KM + j] = c * a + s * b;
  H[(j + 1) * KM + j] = 0.0;
  st->g[j + 1] = -s * st->g[j];
  st->g[j] = c * st->g[j];
  st->iters += 1;
  st->sum_j += j;
  st->jlast = j + 1;
  st->s[j + 1] = hnorm > 0.0 ? 1.0 / hnorm : 0.0;
  if (!isfinite(hnorm) || !isfinite(st->g[j + 1]) || !isfinite(H[j * KM + j])) {
    st->status = RSFDE_ENONFINITE;
    st->jlast = 0;
    st->run_iter = 0;
    st->run_cycle = 0;
    return;
  }
  if (fabs(st->g[j + 1]) <= st->tol * st->bnorm || hnorm == 0.0 || j + 1 >= st->m ||
      st->iters >= st->max_iter)
    st->run_iter = 0;
}

// ---- tile-shape autotuning (transforms.cu) -----------------------------------
enum TuneKind { TK_TOEP_ROWS, TK_TOEP_COLS, TK_DST_ROWS, TK_DST_COLS, TK_PRE_COLS, TK_PRE_ROWS, TK_COUNT };
void tune_force_groups(int F);  // 0: use the recorded choice / heuristic
int tune_forced();              // the shape tune_force_groups set (0: none)
void tune_record(int kind, int log2L, int wide, int F);
int tune_lookup(int kind, int log2L, int wide);
template <typename T>
int max_groups(int L, int items);

// ---- launchers (transforms.cu) ---------------------------------------------
// A launcher asked for a (type, mode) pair it has no kernel for launches
// nothing and raises a flag that the next launch check reports.
void note_unsupported_launch();
bool take_unsupported_launch();
// tmpx: scratch of N values of the arithmetic type T between the passes:
// z - A_x z + pen phi z when phi is given, else A_x z
template <typename T, typename Tin>
void launch_toeplitz_rows(const Tin* z, void* tmpx, const uint8_t* phi, double pen, int n1, int n2,
                          const AxisTables<T>& ax, const int* gate, cudaStream_t s);
// out: Tout = double, or df for a double-FP32 Krylov basis
template <typename T, typename Tin, typename Tout>
void launch_toeplitz_cols(int mode, const Tin* z, void* tmpx, const uint8_t* phi, double pen,
                          const double* b, Tout* out, int n1, int n2, const AxisTables<T>& ay,
                          const int* gate, double* partials, SolverState* st, cudaStream_t s);
// Exact Toeplitz products of the true residual (exact.cuh), two launches per
// pass (the transforms for the four primes, then the Chinese remaindering
// with the epilogue): the row pass writes tmpx = x - A_x x + pen phi x; the
// column pass MODE_RESIDUAL (Tout double or float, with the norm and restart)
// or MODE_RESID_ONLY (double).  sc: four arrays of N words and n1 + n2 ints.
// build_exact_tables: the host tables of one axis (Toeplitz column t, length
// L), 3 L entries per prime in the order tw, twi, spec; *St the quantisation
// exponent of t.
std::vector<uint2> build_exact_tables(const std::vector<double>& t, int L, int* St);
void launch_exact_rows(const double* x, double* tmpx, const uint8_t* phi, double pen, int n1, int n2,
                       const ExactAxis& ax, const ExactScratch& sc, const int* gate, cudaStream_t s);
template <typename Tout>
void launch_exact_cols(int mode, const double* x, double* tmpx, const uint8_t* phi, double pen, const double* b,
                       Tout* out, int n1, int n2, const ExactAxis& ay, const ExactScratch& sc, const int* gate,
                       double* partials, SolverState* st, cudaStream_t s);
template <typename T, typename Tin, typename Tout>
void launch_dst_rows(const Tin* v, const double* vscale, Tout* out, int n1, int n2, const AxisTables<T>& ax,
                     const int* gate, cudaStream_t s);
template <typename T, typename Tin, typename Tout>
void launch_dst_cols(const Tin* in, Tout* out, int n1, int n2, const AxisTables<T>& ay, cudaStream_t s);
template <typename T>
void launch_precond_cols(const T* T1, T* T2a, T* T2b, int n1, int n2, const AxisTables<T>& ay, const T* lamx,
                         double pen, const int* gate, cudaStream_t s);
template <typename T, typename Tz>
void launch_precond_rows(const T* T2a, const T* T2b, const uint8_t* phi, Tz* z, int n1, int n2,
                         const AxisTables<T>& ax, const int* gate, cudaStream_t s);

// Optional second output of the final update pass (FP32 or FP64 basis): the
// new vector rounded to BF16 in the symmetric GEMM's K layout (row y at
// a0 + y*ld, even x at x/2, odd x at hk + x/2), the next preconditioner's first
// operand; with lo set (split BF16) also the remainder bf16(x - hi) at the
// same place of lo.
struct Bf16Out {
  __nv_bfloat16* a0;
  __nv_bfloat16* lo;
  int n1, ld, hk;
};

// ---- split-BF16 tensor-core preconditioner (dst_gemm.cu) --------------------
struct Bf16Plan;
// nt: BF16 products per GEMM, 3 (split BF16) or 1 (plain BF16)
// phi: the context's mask (device, n2 x n1, 1 outside Omega), fixed for the plan's life
int bf16_plan_create(Bf16Plan** out, int n1, int n2, int nt, const float* lamx, const float* lamy,
                     const uint8_t* phi, cudaStream_t s);
int bf16_plan_nt(const Bf16Plan* p);
void bf16_plan_destroy(Bf16Plan* p);
int bf16_plan_error(Bf16Plan* p, cudaStream_t s);  // reads and clears the give-up flag
void bf16_plan_set_wait(Bf16Plan* p, long long cycles);  // <= 0: the default bound
// skip_split: the first operand was already written (update_kernel's Bf16Out,
// unscaled), and zscale multiplies the result instead.
// ev: if set, five events recorded before the first GEMM and after each (timing).
template <typename Tz, typename Tin>
int bf16_precond(Bf16Plan* p, const Tin* v, const double* vscale, Tz* z, const uint8_t* phi, double pen,
                 const int* gate, cudaStream_t s, bool skip_split = false, const double* zscale = nullptr,
                 cudaEvent_t* ev = nullptr);
// Measured tile width (64 or 128) per GEMM of the chain, recorded in the plan.
int bf16_plan_autotune(Bf16Plan* p, const double* v, float* z, const uint8_t* phi, double pen, cudaStream_t s,
                       int reps, int* bn_out);
// The Bf16Out target of the plan's first operand, if the plan can take it
// (symmetric layout, n1 a multiple of vec); returns false otherwise.
bool bf16_plan_a0(const Bf16Plan* p, int vec, Bf16Out* out);

// ---- batched instances: one launch per phase over every instance -------------
// One instance of a batch as the multi-instance kernels see it (an array of
// these lives in device memory).  Every buffer is the instance's own
// context's; u_prev, u_pp and src are its time-march ring.
struct BatchInst {
  int n1, n2;
  size_t N;
  double pen, dt;
  const uint8_t* phi;
  double* V;   // Krylov basis, in the basis type
  void* Z;     // preconditioned vectors
  void* tmpx;  // operator scratch
  void* T1;
  void* T2a;
  void* T2b;
  double* b;
  double* x;
  double* partials;
  SolverState* st;
  double* u_prev;
  double* u_pp;
  const double* src;
  AxisTables<double> x64, y64;
  AxisTables<float> x32, y32;
  AxisTables<df> xdf, ydf;
  // split-BF16 preconditioner (lock-step form): the instance's first GEMM
  // operand (BF16 pair, leading dimension a0_ld, symmetric half a0_hk), and
  // whether the basis update writes it for columns j > 0 (a0_fused)
  void* a0;
  void* a0_lo;
  int a0_ld, a0_hk, a0_fused;
  // exact true residual (lock-step form): the instance's tables and scratch
  ExactAxis ex, ey;
  ExactScratch esc;
};

// The blocks of one multi-instance launch: instance i owns the blocks
// [prefix[i], prefix[i+1]) -- exactly the grid a launch for that instance
// alone would have, so every reduction is split the same way and the results
// are bit-identical to single-instance solves.  l2mask (transform kernels):
// bit k is set when an instance's transform length along the kernel's axis
// is 2^k (it sizes the shared memory).
//
// A launch does not run every virtual block: a compaction kernel first writes
// `active`, the same prefix with the counts of instances whose gate is
// closed set to zero, and a fixed grid of `grid` blocks loops over the
// active virtual blocks only (so finished instances cost nothing).
struct MultiGrid {
  const int* prefix = nullptr;  // device, count + 1 entries
  int* active = nullptr;        // device, count + 1 entries (compaction output)
  int count = 0, total = 0;
  unsigned l2mask = 0;
  // device, 2 ints, zero between launches: if set, the launch hands its
  // virtual blocks out one at a time (next block, finished blocks) instead
  // of round robin; the last block to finish zeroes both again
  int* sched = nullptr;
};
// Threads of a multi-instance transform block: F = kMultiThreads / (L/16)
// transforms per block, for every L up to 4096.
constexpr int kMultiThreads = 256;
__host__ __device__ constexpr int multi_groups(int L) { return kMultiThreads / (L / 16); }
// Largest batch of the multi-instance form: a block holds the active prefix
// (kMaxBatchMulti + 1 ints) in shared memory.
constexpr int kMaxBatchMulti = 1024;

// The last i in [0, count) with p[i] <= b (the instance owning virtual block b;
// empty ranges are skipped because the next instance starts at the same value).
__device__ __forceinline__ int multi_instance(const int* p, int count, int b) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// The loop of a multi-instance kernel over the active virtual blocks (the
// active prefix staged in shared memory): each virtual block runs the
// single-instance body on its instance's own virtual grid, so the results do
// not depend on which block of the launch runs it.  sched (MultiGrid::sched):
// hand the virtual blocks out dynamically, else round robin.
template <typename Fn>
__device__ __forceinline__ void multi_loop(const BatchInst* __restrict__ bi, const int* __restrict__ prefix,
                                           const int* __restrict__ active, int count, Fn&& fn,
                                           int* sched = nullptr) {
  __shared__ int sact[kMaxBatchMulti + 1];
  __shared__ int snext;
  for (int k = threadIdx.x; k <= count; k += blockDim.x) sact[k] = active[k];
  __syncthreads();
  const int total = sact[count];
  if (sched) {  // dynamic hand-out: blocks that finish early take the remaining virtual blocks
    for (;;) {
      if (threadIdx.x == 0) snext = atomicAdd(sched, 1);
      __syncthreads();
      const int vb = snext;
      if (vb >= total) break;  // uniform over the block
      const int mi = multi_instance(sact, count, vb);
      const int b0 = __ldg(prefix + mi);
      fn(bi[mi], vb - sact[mi], __ldg(prefix + mi + 1) - b0);
      __syncthreads();  // shared memory (and snext) reused by the next virtual block
    }
    // every block counts itself out after its last hand-out; the last one
    // zeroes the counters for the next launch on the stream
    if (threadIdx.x == 0) {
      __threadfence();
      if (atomicAdd(sched + 1, 1) == (int)gridDim.x - 1) {
        sched[0] = 0;
        sched[1] = 0;
        __threadfence();
      }
    }
    return;
  }
  for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
    const int mi = multi_instance(sact, count, vb);
    const int b0 = __ldg(prefix + mi);
    fn(bi[mi], vb - sact[mi], __ldg(prefix + mi + 1) - b0);
    __syncthreads();  // the next virtual block reuses the block's shared memory
  }
}

// Compaction: for up to kMaxCompact families, active[f][i] = sum over k < i of
// the virtual-grid size of instance k if its gate (run_iter, or run_cycle with
// use_cycle) is open, else 0; active[f][count] the total.
constexpr int kMaxCompact = 16;
struct CompactArgs {
  const int* prefix[kMaxCompact];
  int* active[kMaxCompact];
  int nfam;
};
void launch_compact_multi(const BatchInst* bi, int count, int use_cycle, const CompactArgs& a, cudaStream_t s);
void launch_any_running_multi(const BatchInst* bi, int count, int* out, cudaStream_t s);
// Blocks of a multi-instance launch: every SM filled with resident blocks, at
// most the total virtual blocks.
template <typename K>
int multi_launch_grid(K kernel, int threads, size_t smem, int total) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  const int g = kNumSMs * per_sm;
  return total < g ? (total > 0 ? total : 1) : g;
}

// multi-instance launchers (transforms.cuh, instantiated per arithmetic type)
template <typename T, typename Tz, typename Tv>
void launch_operator_multi(const BatchInst* bi, const MultiGrid& rows, const MultiGrid& cols, int j, cudaStream_t s);
template <typename T, typename Tv>
void launch_residual_multi(const BatchInst* bi, const MultiGrid& rows, const MultiGrid& cols, cudaStream_t s);
template <typename T, typename Tz, typename Tv>
void launch_precond_multi(const BatchInst* bi, const MultiGrid& drows, const MultiGrid& pcols, const MultiGrid& prows,
                          int j, cudaStream_t s);
// multi-instance launchers (krylov.cu)
void launch_init_multi(const BatchInst* bi, int count, int m, int max_iter, double tol, cudaStream_t s);
void launch_rhs_multi(const BatchInst* bi, const MultiGrid& g, int later, cudaStream_t s);
template <typename Tv>
void launch_multidot_multi(const BatchInst* bi, const MultiGrid& g, int j, int accumulate, cudaStream_t s);
// write_a0: instances with a0_fused also write V_{j+1} as their BF16 operand
template <typename Tv>
void launch_update_multi(const BatchInst* bi, const MultiGrid& g, int j, int final_pass, int write_a0, cudaStream_t s);
// Split-BF16 preconditioner of the lock-step form (dst_gemm.cu): one launch
// per pass over every running instance.
struct Bf16GroupInst {
  const Bf16Plan* plan;
  double pen;
  void* z;             // Z, the instance's preconditioned vectors (column j at z + j z_col_bytes)
  size_t z_col_bytes;
  int z_double;
  const double* s;     // the basis scales s_j
  int fused;           // A0 of columns j > 0 written unscaled by the basis update
};
// descs: device array of the four GEMMs of every instance; tiles[4]: the tile
// counts per instance of each GEMM (the grids of the grouped launches).
int bf16_group_create(const std::vector<Bf16GroupInst>& in, void** descs, std::vector<int>* tiles);
void bf16_group_destroy(void* descs);
void launch_bf16_group(int k, const void* descs, int count, const int* active, int max_tiles, int j, int* err,
                       cudaStream_t s);
void launch_split_multi(const BatchInst* bi, const MultiGrid& g, int j, cudaStream_t s);
// The exact true residual of every instance whose cycle ends (exact.cu): the
// transforms of the row pass (nrows: vector groups x 4 primes per instance),
// its Chinese remaindering (crows: vec_grid(N) per instance, as the
// single-instance launch), then the same for the columns with b - M x, the
// norm and the restart decision.
void launch_exact_multi(const BatchInst* bi, const MultiGrid& nrows, const MultiGrid& crows, const MultiGrid& ncols,
                        const MultiGrid& ccols, cudaStream_t s);
int exact_multi_ntt_blocks(int L, int nvec);  // virtual blocks of one instance's transform launch
void bf16_plan_a0_any(const Bf16Plan* p, Bf16Out* out);
void launch_solve_y_multi(const BatchInst* bi, int count, cudaStream_t s);
template <typename Tz>
void launch_xupdate_multi(const BatchInst* bi, const MultiGrid& g, cudaStream_t s);
void launch_finish_rotate_multi(const BatchInst* bi, const MultiGrid& g, cudaStream_t s);
void launch_loop_cond_multi(cudaGraphConditionalHandle h, const BatchInst* bi, int count, int* runs,
                            cudaStream_t s);
// The grid a single-instance launch uses (and a multi-instance launch gives
// each instance): Gram-Schmidt at column j, the vector kernels.
template <typename Tv>
int multidot_blocks(size_t N, int j);  // grid.x * grid.y
template <typename Tv>
int update_blocks(size_t N, int j);
int xupdate_blocks(size_t N, int zbytes);

// ---- launchers (krylov.cu) -------------------------------------------------
int vec_grid(size_t N);
void launch_init_state(SolverState* st, int m, int max_iter, double tol, cudaStream_t s);
void launch_mask_to_phi(const uint8_t* in_omega, uint8_t* phi, size_t N, cudaStream_t s);
void launch_rhs(const double* u, const double* uu, const double* src, const uint8_t* phi, double dt, double* b,
                double* x0, size_t N, double* partials, SolverState* st, cudaStream_t s);
void launch_norm_b(const double* b, size_t N, double* partials, SolverState* st, cudaStream_t s);
// Gram-Schmidt over the Krylov basis V (Tv = double, or df: double-FP32
// storage and arithmetic)
template <typename Tv>
void launch_multidot(const Tv* V, size_t N, int j, int accumulate, double* partials, SolverState* st,
                     cudaStream_t s);
template <typename Tv>
void launch_update(Tv* V, size_t N, int j, int final_pass, double* partials, SolverState* st, cudaStream_t s,
                   const Bf16Out* bo = nullptr);
void launch_solve_y(SolverState* st, cudaStream_t s);
template <typename Tz>
void launch_xupdate(double* x, const Tz* Z, size_t N, SolverState* st, cudaStream_t s);
void launch_finalize(double* x, size_t N, SolverState* st, cudaStream_t s);
void launch_loop_cond(cudaGraphConditionalHandle h, SolverState* st, cudaStream_t s);
void launch_restart_norm(const double* v, size_t N, double* partials, SolverState* st, const int* gate,
                         cudaStream_t s);
void launch_xupdate_v(double* x, const double* V, size_t N, SolverState* st, cudaStream_t s);
void launch_adjoint_accum(const double* u_prev, const double* mu, const double* ax_u, const double* ay_u,
                          const uint8_t* phi, double dt, double ikx, double iky, double* lam_prev,
                          double* grad_src, double* grad_k, size_t N, double* partials, SolverState* st,
                          cudaStream_t s);
template <typename Tv, typename Tz>
void launch_scale_copy(const Tv* v, const double* scale, Tz* z, size_t N, const int* gate, cudaStream_t s);

}  // namespace rsfde
