// api.cu -- the C ABI (include/rsfde.h): context, FP64 host setup of the
// Toeplitz and tau tables, and the orchestration of flexible GMRES on one
// CUDA stream.
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <type_traits>
#include <functional>
#include <vector>

#include <nvtx3/nvToolsExt.h>  // header-only: ranges reach a profiler when one is attached

#include "fft.cuh"  // host butterflies for the setup spectra

#include "internal.h"

using namespace rsfde;

namespace {

// ---- host setup (FP64) -----------------------------------------------------
// Section 1: c_alpha = -1 / (2 cos(alpha pi / 2)).
double riesz_c(double alpha) { return -1.0 / (2.0 * std::cos(alpha * M_PI / 2.0)); }

// Eq. 2.16 first column of c * G_n^(alpha), from the weights of Eq. 2.6.
std::vector<double> toeplitz_first_column(double alpha, double c, int n) {
  std::vector<double> g(n + 2);
  g[0] = 1.0;
  for (int l = 1; l < n + 2; ++l) g[l] = g[l - 1] * (1.0 - (alpha + 1.0) / l);
  std::vector<double> t(n);
  for (int k = 0; k < n; ++k) t[k] = c * (k == 0 ? 2.0 * g[1] : k == 1 ? g[0] + g[2] : g[k + 1]);
  return t;
}

// Section 4.1: eigenvalues of tau(T_n) for symmetric Toeplitz T_n with first
// column t: lambda_k = t_0 + 2 sum_{j=1}^{n-1} t_j cos(pi j k / (n+1)), the
// values S_n tau(T_n) S_n takes on its diagonal.
std::vector<double> tau_eigenvalues(const std::vector<double>& t) {
  const int n = (int)t.size();
  const long period = 2L * (n + 1);
  std::vector<double> cosv(period);
  for (long m = 0; m < period; ++m) cosv[m] = std::cos(M_PI * (double)m / (double)(n + 1));
  std::vector<double> lam(n);
  for (int k = 1; k <= n; ++k) {
    double s = 0.0;
    for (int j = n - 1; j >= 1; --j) s += t[j] * cosv[((long)j * k) % period];
    lam[k - 1] = t[0] + 2.0 * s;
  }
  return lam;
}

void host_dif(std::vector<double>& re, std::vector<double>& im, int L, int log2L, const std::vector<double>& tw) {
  int s;
  if (log2L & 1) {
    for (int k = 0; k < L / 2; ++k) dif_r2(re.data(), im.data(), L, k, tw.data());
    s = L >> 3;
  } else {
    s = L >> 2;
  }
  for (; s >= 1; s >>= 2)
    for (int q = 0; q < L / 4; ++q) dif_r4(re.data(), im.data(), L, s, q, tw.data());
  // the DIF leaves the spectrum in bit-reversed order; the kernels want it natural
  std::vector<double> r2(L), i2(L);
  for (int l = 0; l < L; ++l) {
    int b = 0;
    for (int x = l, k = 0; k < log2L; ++k, x >>= 1) b = (b << 1) | (x & 1);
    r2[b] = re[l];
    i2[b] = im[l];
  }
  re.swap(r2);
  im.swap(i2);
}

struct HostAxis {
  int n = 0, L = 0, log2L = 0;
  std::vector<double> t, lam, tw, sigma, chirp, chirp_out, bspec;
};

HostAxis build_axis(int n, double alpha, double c) {
  HostAxis a;
  a.n = n;
  a.L = 16;  // the register FFT's smallest length
  a.log2L = 4;
  while (a.L < 2 * n - 1) {
    a.L <<= 1;
    a.log2L++;
  }
  const int L = a.L;
  a.t = toeplitz_first_column(alpha, c, n);
  a.lam = tau_eigenvalues(a.t);
  a.tw.resize(2 * L);
  for (int j = 0; j < L; ++j) {
    a.tw[2 * j] = std::cos(2.0 * M_PI * j / L);
    a.tw[2 * j + 1] = -std::sin(2.0 * M_PI * j / L);
  }
  // circulant embedding of the symmetric Toeplitz matrix; its spectrum is real
  std::vector<double> re(L, 0.0), im(L, 0.0);
  re[0] = a.t[0];
  for (int k = 1; k < n; ++k) re[k] = re[L - k] = a.t[k];
  host_dif(re, im, L, a.log2L, a.tw);
  a.sigma.resize(L);
  for (int l = 0; l < L; ++l) a.sigma[l] = re[l] / L;
  // Bluestein chirps for S_n: exp(i pi k^2 / (2(n+1))), phase reduced mod 4(n+1)
  const long per = 4L * (n + 1);
  const double nrm = std::sqrt(2.0 / (n + 1));
  a.chirp.resize(2 * n);
  a.chirp_out.resize(2 * n);
  for (int k = 1; k <= n; ++k) {
    const long m = ((long)k * k) % per;
    const double ang = M_PI * (double)m / (2.0 * (n + 1));
    a.chirp[2 * (k - 1)] = std::cos(ang);
    a.chirp[2 * (k - 1) + 1] = std::sin(ang);
    a.chirp_out[2 * (k - 1)] = nrm * std::cos(ang);
    a.chirp_out[2 * (k - 1) + 1] = nrm * std::sin(ang);
  }
  std::fill(re.begin(), re.end(), 0.0);
  std::fill(im.begin(), im.end(), 0.0);
  for (int d = 0; d < n; ++d) {
    const long m = ((long)d * d) % per;
    const double ang = -M_PI * (double)m / (2.0 * (n + 1));
    re[d] = std::cos(ang);
    im[d] = std::sin(ang);
    if (d > 0) {
      re[L - d] = re[d];
      im[L - d] = im[d];
    }
  }
  host_dif(re, im, L, a.log2L, a.tw);
  a.bspec.resize(2 * L);
  for (int l = 0; l < L; ++l) {
    a.bspec[2 * l] = re[l] / L;
    a.bspec[2 * l + 1] = im[l] / L;
  }
  return a;
}

// Device copy of one axis' tables in precision T (one allocation).
template <typename T>
struct DevAxis {
  void* mem = nullptr;
  AxisTables<T> tab{};
  void release() {
    if (mem) cudaFree(mem);
    mem = nullptr;
  }
  cudaError_t upload(const HostAxis& h, cudaStream_t s) {
    const size_t L = h.L, n = h.n;
    const size_t count = 2 * L + L + 2 * n + 2 * n + 2 * L + n;
    std::vector<T> buf(count);
    size_t o = 0;
    auto put = [&](const std::vector<double>& v) {
      size_t start = o;
      for (double d : v) buf[o++] = T(d);
      return start;
    };
    size_t o_tw = put(h.tw), o_sig = put(h.sigma), o_ch = put(h.chirp), o_cho = put(h.chirp_out),
           o_bs = put(h.bspec), o_lam = put(h.lam);
    if (!mem) {
      cudaError_t e = cudaMalloc(&mem, count * sizeof(T));
      if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaMemcpyAsync(mem, buf.data(), count * sizeof(T), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(s);
    const T* b = static_cast<const T*>(mem);
    tab.n = h.n;
    tab.L = h.L;
    tab.log2L = h.log2L;
    tab.tw = b + o_tw;
    tab.sigma = b + o_sig;
    tab.chirp = b + o_ch;
    tab.chirp_out = b + o_cho;
    tab.bspec = b + o_bs;
    tab.lam = b + o_lam;
    return e;
  }
};

// Device copy of one axis' exact-product tables (one allocation).
struct DevExact {
  void* mem = nullptr;
  size_t bytes = 0;
  ExactAxis tab{};
  void release() {
    if (mem) cudaFree(mem);
    mem = nullptr;
    bytes = 0;
  }
  cudaError_t upload(const HostAxis& h, cudaStream_t s) {
    int St = 0;
    const std::vector<uint2> t = build_exact_tables(h.t, h.L, &St);
    const size_t need = t.size() * sizeof(uint2);
    if (mem && bytes != need) release();
    if (!mem) {
      cudaError_t e = cudaMalloc(&mem, need);
      if (e != cudaSuccess) return e;
      bytes = need;
    }
    cudaError_t e = cudaMemcpyAsync(mem, t.data(), need, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(s);
    tab.n = h.n;
    tab.L = h.L;
    tab.log2L = h.log2L;
    tab.St = St;
    tab.tab = static_cast<const uint2*>(mem);
    return e;
  }
};

}  // namespace

struct rsfde_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int n1 = 0, n2 = 0;
  size_t N = 0;
  double ax = 0, bx = 0, ay = 0, by = 0;
  double alpha1 = 0, alpha2 = 0, kx = 0, ky = 0, dt = 0, eta = 0;
  double hx = 0, hy = 0, cx = 0, cy = 0, pen = 0;
  rsfde_opts opts{};
  int m_alloc = 0;
  HostAxis hx_axis, hy_axis;
  DevAxis<double> x64, y64;
  DevExact xex, yex;  // exact Toeplitz products of the true residual
  DevAxis<float> x32, y32;
  DevAxis<df> xdf, ydf;
  uint8_t* phi = nullptr;
  double* V = nullptr;      // (m+1) x N
  void* Z = nullptr;        // m x N (double or float)
  double* tmpx = nullptr;   // N
  void* T1 = nullptr;       // N (double-sized)
  void* T2a = nullptr;
  void* T2b = nullptr;
  double* b = nullptr;
  double* x = nullptr;
  double* hbuf = nullptr;   // 3N for the host-array step
  double* partials = nullptr;
  size_t npartials = 0;
  SolverState* st = nullptr;
  SolverState* st_host = nullptr;  // pinned
  int64_t launches = 0;
  Bf16Plan* bf16 = nullptr;  // tensor-core preconditioner, made when first needed
  long long wait_cycles = 0;  // its pipeline wait bound (0: the default)
  // one FGMRES cycle captured as the body of a device-side WHILE loop
  cudaStream_t cap_stream = nullptr;  // private stream used only for capture
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  int graph_key = -1;
  int64_t launches_per_body = 0;
  // profiler: event pairs per kernel class, recorded while prof_on
  bool prof_on = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
  double prof_ms[RSFDE_K_COUNT] = {0};
  int64_t prof_n[RSFDE_K_COUNT] = {0};
  double prof_call0[RSFDE_K_COUNT] = {0};  // prof_ms when the current public call began
  double call_bytes = 0;                   // right side bytes of the current call (rsfde_step)
};

namespace {

bool bad_alpha(double a) { return !(a > 1.0 && a < 2.0); }

// Largest grid side: the transform kernels take convolution lengths up to
// 8192 (a group of L/16 = 512 threads, the FP64 and double-FP32 block cap).
constexpr int kMaxN = 4096;

int cuda_fail(cudaError_t e) {
  if (e == cudaSuccess) return RSFDE_OK;
  if (e == cudaErrorMemoryAllocation) return RSFDE_ENOMEM;
  return RSFDE_ECUDA;
}

int check_launch(rsfde_ctx* c) {
  if (take_unsupported_launch()) return RSFDE_EINVAL;
  return cuda_fail(cudaGetLastError());
}

cudaEvent_t prof_event(rsfde_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets one launch of kernel class k with events when profiling is on.
// A named NVTX range over a host-side scope (an entry point, or the enqueue
// of one kernel of a class), for timeline profilers.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

struct ProfScope {
  rsfde_ctx* c;
  int k;
  cudaEvent_t a = nullptr, b = nullptr;
  NvtxRange range;
  ProfScope(rsfde_ctx* c_, int k_) : c(c_), k(k_), range(rsfde_kernel_class_name(k_)) {
    c->launches += 1;
    if (!c->prof_on) return;
    a = prof_event(c);
    b = prof_event(c);
    cudaEventRecord(a, c->stream);
  }
  ~ProfScope() {
    if (!a) return;
    cudaEventRecord(b, c->stream);
    c->ev_pending.push_back({k, {a, b}});
  }
};

void prof_harvest(rsfde_ctx* c) {
  for (auto& p : c->ev_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.second.first, p.second.second) == cudaSuccess) c->prof_ms[p.first] += ms;
    c->prof_n[p.first] += 1;
    c->ev_pool.push_back(p.second.first);
    c->ev_pool.push_back(p.second.second);
  }
  c->ev_pending.clear();
}

int build_tables(rsfde_ctx* c) {
  c->hx = (c->bx - c->ax) / (c->n1 + 1);  // Section 2
  c->hy = (c->by - c->ay) / (c->n2 + 1);
  c->cx = c->dt * c->kx * riesz_c(c->alpha1) / std::pow(c->hx, c->alpha1);
  c->cy = c->dt * c->ky * riesz_c(c->alpha2) / std::pow(c->hy, c->alpha2);
  c->pen = c->dt / c->eta;
  c->hx_axis = build_axis(c->n1, c->alpha1, c->cx);
  c->hy_axis = build_axis(c->n2, c->alpha2, c->cy);
  cudaError_t e;
  if ((e = c->x64.upload(c->hx_axis, c->stream)) != cudaSuccess) return cuda_fail(e);
  if ((e = c->y64.upload(c->hy_axis, c->stream)) != cudaSuccess) return cuda_fail(e);
  if ((e = c->x32.upload(c->hx_axis, c->stream)) != cudaSuccess) return cuda_fail(e);
  if ((e = c->y32.upload(c->hy_axis, c->stream)) != cudaSuccess) return cuda_fail(e);
  if ((e = c->xdf.upload(c->hx_axis, c->stream)) != cudaSuccess) return cuda_fail(e);
  if ((e = c->ydf.upload(c->hy_axis, c->stream)) != cudaSuccess) return cuda_fail(e);
  if ((e = c->xex.upload(c->hx_axis, c->stream)) != cudaSuccess) return cuda_fail(e);
  if ((e = c->yex.upload(c->hy_axis, c->stream)) != cudaSuccess) return cuda_fail(e);
  return RSFDE_OK;
}

void free_ctx(rsfde_ctx* c) {
  if (!c) return;
  for (auto& p : c->ev_pending) {
    cudaEventDestroy(p.second.first);
    cudaEventDestroy(p.second.second);
  }
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  c->x64.release();
  c->y64.release();
  c->x32.release();
  c->y32.release();
  c->xdf.release();
  c->ydf.release();
  c->xex.release();
  c->yex.release();
  void* ptrs[] = {c->phi, c->V, c->Z, c->tmpx, c->T1, c->T2a, c->T2b, c->b, c->x, c->hbuf, c->partials, c->st};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->st_host) cudaFreeHost(c->st_host);
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  bf16_plan_destroy(c->bf16);
  delete c;
}

// Z (the preconditioned vectors) is FP32 for the FP32 and split-BF16 preconditioners.
bool fp32_precond(const rsfde_ctx* c) {
  const int p = c->opts.precond_prec;
  return p == RSFDE_FP32 || p == RSFDE_BF16X3 || p == RSFDE_BF16;
}
bool bf16_precond_on(const rsfde_ctx* c) {
  return c->opts.precond_prec == RSFDE_BF16X3 || c->opts.precond_prec == RSFDE_BF16;
}

// The tensor-core plan of the current preconditioner precision (three BF16
// products per GEMM for BF16X3, one for BF16).
int ensure_bf16(rsfde_ctx* c) {
  if (!bf16_precond_on(c)) return RSFDE_OK;
  const int nt = c->opts.precond_prec == RSFDE_BF16X3 ? 3 : 1;
  if (c->bf16 && bf16_plan_nt(c->bf16) == nt) return RSFDE_OK;
  if (c->bf16) {
    cudaStreamSynchronize(c->stream);
    bf16_plan_destroy(c->bf16);
    c->bf16 = nullptr;
  }
  const int rc = bf16_plan_create(&c->bf16, c->n1, c->n2, nt, c->x32.tab.lam, c->y32.tab.lam, c->phi, c->stream);
  if (rc == RSFDE_OK) bf16_plan_set_wait(c->bf16, c->wait_cycles);
  return rc;
}

// The tensor-core preconditioner z = P-hat^-1 (scale * v) (five launches).
template <typename Tz, typename Tin>
void enqueue_precond_bf16(rsfde_ctx* c, const Tin* v, const double* vscale, Tz* z, const int* gate,
                          bool first_operand_ready = false) {
  ProfScope ps(c, RSFDE_K_DST_GEMM);
  c->launches += first_operand_ready ? 4 : 5;
  bf16_precond<Tz, Tin>(c->bf16, v, vscale, z, c->phi, c->pen, gate, c->stream, first_operand_ready, vscale);
}

// ---- enqueue helpers ---------------------------------------------------------
// w = M z (Eq. 2.17), z in precision Tz, arithmetic T (double or df), w
// stored as Tw (double, or df for a double-FP32 Krylov basis).
template <typename T, typename Tz, typename Tw>
void enqueue_apply_M_t(rsfde_ctx* c, const Tz* z, Tw* w, const int* gate, const AxisTables<T>& tx,
                       const AxisTables<T>& ty) {
  {
    ProfScope ps(c, RSFDE_K_TOEPLITZ_ROWS);
    launch_toeplitz_rows<T, Tz>(z, c->tmpx, c->phi, c->pen, c->n1, c->n2, tx, gate, c->stream);
  }
  {
    ProfScope ps(c, RSFDE_K_TOEPLITZ_COLS);
    launch_toeplitz_cols<T, Tz, Tw>(MODE_APPLY, z, c->tmpx, c->phi, c->pen, nullptr, w, c->n1, c->n2, ty, gate,
                                    nullptr, nullptr, c->stream);
  }
}

template <typename Tz>
void enqueue_apply_M(rsfde_ctx* c, const Tz* z, double* w, const int* gate) {
  if (c->opts.matvec_prec == RSFDE_DF32) enqueue_apply_M_t<df, Tz, double>(c, z, w, gate, c->xdf.tab, c->ydf.tab);
  else if (c->opts.matvec_prec == RSFDE_FP32)
    enqueue_apply_M_t<float, Tz, double>(c, z, w, gate, c->x32.tab, c->y32.tab);
  else enqueue_apply_M_t<double, Tz, double>(c, z, w, gate, c->x64.tab, c->y64.tab);
}

bool left_variant(const rsfde_ctx* c) { return c->opts.variant == RSFDE_GMRES_LEFT; }

// The right-preconditioned FGMRES keeps its Krylov basis, and runs its
// Gram-Schmidt, in basis_prec: FP64 (FP64 arithmetic, whatever the operator's
// arithmetic), or -- with an operator of the same precision, whose output is
// then stored without a conversion -- double-FP32 or FP32 on the FP32 pipe.
// Paper mode keeps FP64.
enum BasisKind { BASIS_FP64, BASIS_DF32, BASIS_FP32 };
BasisKind basis_kind(const rsfde_ctx* c) {
  if (left_variant(c)) return BASIS_FP64;
  if (c->opts.basis_prec == RSFDE_DF32) return BASIS_DF32;
  if (c->opts.basis_prec == RSFDE_FP32) return BASIS_FP32;
  return BASIS_FP64;
}

template <typename T, typename Tz, typename Tin>
void enqueue_precond_t(rsfde_ctx* c, const Tin* v, const double* vscale, Tz* z, const int* gate,
                       const AxisTables<T>& tx, const AxisTables<T>& ty);

// z = P-hat^-1 (scale * v) into an FP64 vector, in the context's preconditioner precision.
template <typename Tz, typename Tin>
void enqueue_precond_bf16(rsfde_ctx* c, const Tin* v, const double* vscale, Tz* z, const int* gate,
                          bool first_operand_ready);

void enqueue_precond64(rsfde_ctx* c, const double* v, const double* vscale, double* z, const int* gate) {
  if (bf16_precond_on(c)) enqueue_precond_bf16<double, double>(c, v, vscale, z, gate);
  else if (fp32_precond(c)) enqueue_precond_t<float, double, double>(c, v, vscale, z, gate, c->x32.tab, c->y32.tab);
  else enqueue_precond_t<double, double, double>(c, v, vscale, z, gate, c->x64.tab, c->y64.tab);
}

// Left-preconditioned GMRES: V_0 = P^-1 (b - M x) (or b - M x without a
// preconditioner), beta = ||V_0||, then restart_prep.
// Scratch of the exact residual: the FFT preconditioner's work arrays T1 and
// T2a (8 N bytes each: two residue arrays each) and T2b (the exponents),
// free whenever a residual runs.
ExactScratch exact_scratch(rsfde_ctx* c) {
  ExactScratch sc;
  sc.res[0] = static_cast<uint32_t*>(c->T1);
  sc.res[1] = sc.res[0] + c->N;
  sc.res[2] = static_cast<uint32_t*>(c->T2a);
  sc.res[3] = sc.res[2] + c->N;
  sc.ebuf = static_cast<int*>(c->T2b);
  return sc;
}

// r = b - M x (no norm) with M x in FP64 or, for resid_prec RSFDE_EXACT, exact
// Toeplitz products.
void enqueue_resid_only(rsfde_ctx* c, const double* x, const double* b, double* r, const int* gate) {
  const bool exact = c->opts.resid_prec == RSFDE_EXACT;
  {
    ProfScope ps(c, RSFDE_K_RESID_ROWS);
    if (exact)
      launch_exact_rows(x, c->tmpx, c->phi, c->pen, c->n1, c->n2, c->xex.tab, exact_scratch(c), gate, c->stream);
    else launch_toeplitz_rows<double, double>(x, c->tmpx, c->phi, c->pen, c->n1, c->n2, c->x64.tab, gate, c->stream);
  }
  ProfScope ps(c, RSFDE_K_RESID_COLS);
  if (exact)
    launch_exact_cols<double>(MODE_RESID_ONLY, x, c->tmpx, c->phi, c->pen, b, r, c->n1, c->n2, c->yex.tab,
                              exact_scratch(c), gate, nullptr, nullptr, c->stream);
  else
    launch_toeplitz_cols<double, double>(MODE_RESID_ONLY, x, c->tmpx, c->phi, c->pen, b, r, c->n1, c->n2,
                                         c->y64.tab, gate, nullptr, nullptr, c->stream);
}

void enqueue_residual_left(rsfde_ctx* c, const int* gate) {
  double* r = c->opts.use_precond ? static_cast<double*>(c->Z) : c->V;
  enqueue_resid_only(c, c->x, c->b, r, gate);
  if (c->opts.use_precond) enqueue_precond64(c, r, nullptr, c->V, gate);
  ProfScope ps(c, RSFDE_K_OTHER);
  launch_restart_norm(c->V, c->N, c->partials, c->st, gate, c->stream);
}

// ||b|| for the stop test: ||P^-1 b|| for left-preconditioned GMRES (st->bnorm).
void enqueue_bnorm(rsfde_ctx* c) {
  const double* v = c->b;
  if (left_variant(c) && c->opts.use_precond) {
    enqueue_precond64(c, c->b, nullptr, static_cast<double*>(c->Z), nullptr);
    v = static_cast<double*>(c->Z);
  }
  ProfScope ps(c, RSFDE_K_OTHER);
  launch_norm_b(v, c->N, c->partials, c->st, c->stream);
}

// V_0 = b - M x, beta = ||V_0||, then restart_prep (device); M x in FP64 or
// (resid_prec = RSFDE_DF32) double-FP32, b - M x and its norm in FP64.
template <typename T>
void enqueue_residual_t(rsfde_ctx* c, const int* gate, const AxisTables<T>& tx, const AxisTables<T>& ty) {
  {
    ProfScope ps(c, RSFDE_K_RESID_ROWS);
    launch_toeplitz_rows<T, double>(c->x, c->tmpx, c->phi, c->pen, c->n1, c->n2, tx, gate, c->stream);
  }
  ProfScope ps(c, RSFDE_K_RESID_COLS);
  if (basis_kind(c) == BASIS_DF32)
    launch_toeplitz_cols<T, double, df>(MODE_RESIDUAL, c->x, c->tmpx, c->phi, c->pen, c->b,
                                        reinterpret_cast<df*>(c->V), c->n1, c->n2, ty, gate, c->partials, c->st,
                                        c->stream);
  else if (basis_kind(c) == BASIS_FP32)
    launch_toeplitz_cols<T, double, float>(MODE_RESIDUAL, c->x, c->tmpx, c->phi, c->pen, c->b,
                                           reinterpret_cast<float*>(c->V), c->n1, c->n2, ty, gate, c->partials,
                                           c->st, c->stream);
  else
    launch_toeplitz_cols<T, double, double>(MODE_RESIDUAL, c->x, c->tmpx, c->phi, c->pen, c->b, c->V, c->n1, c->n2,
                                            ty, gate, c->partials, c->st, c->stream);
}

// V_0 = b - M x with exact Toeplitz products, beta = ||V_0||, restart_prep.
void enqueue_residual_exact(rsfde_ctx* c, const int* gate) {
  {
    ProfScope ps(c, RSFDE_K_RESID_ROWS);
    launch_exact_rows(c->x, c->tmpx, c->phi, c->pen, c->n1, c->n2, c->xex.tab, exact_scratch(c), gate, c->stream);
  }
  ProfScope ps(c, RSFDE_K_RESID_COLS);
  if (basis_kind(c) == BASIS_FP32)
    launch_exact_cols<float>(MODE_RESIDUAL, c->x, c->tmpx, c->phi, c->pen, c->b, reinterpret_cast<float*>(c->V),
                             c->n1, c->n2, c->yex.tab, exact_scratch(c), gate, c->partials, c->st, c->stream);
  else
    launch_exact_cols<double>(MODE_RESIDUAL, c->x, c->tmpx, c->phi, c->pen, c->b, c->V, c->n1, c->n2, c->yex.tab,
                              exact_scratch(c), gate, c->partials, c->st, c->stream);
}

void enqueue_residual(rsfde_ctx* c, const int* gate) {
  if (left_variant(c)) {
    enqueue_residual_left(c, gate);
    return;
  }
  if (c->opts.resid_prec == RSFDE_DF32) enqueue_residual_t<df>(c, gate, c->xdf.tab, c->ydf.tab);
  else if (c->opts.resid_prec == RSFDE_EXACT) enqueue_residual_exact(c, gate);
  else enqueue_residual_t<double>(c, gate, c->x64.tab, c->y64.tab);
}

// z = P-hat^-1 (scale * v) (Eq. 4.6) into z of precision Tz.
template <typename T, typename Tz, typename Tin>
void enqueue_precond_t(rsfde_ctx* c, const Tin* v, const double* vscale, Tz* z, const int* gate,
                       const AxisTables<T>& tx, const AxisTables<T>& ty) {
  T* t1 = static_cast<T*>(c->T1);
  T* t2a = static_cast<T*>(c->T2a);
  T* t2b = static_cast<T*>(c->T2b);
  {
    ProfScope ps(c, RSFDE_K_DST_ROWS);
    launch_dst_rows<T, Tin, T>(v, vscale, t1, c->n1, c->n2, tx, gate, c->stream);
  }
  {
    ProfScope ps(c, RSFDE_K_PRECOND_COLS);
    launch_precond_cols<T>(t1, t2a, t2b, c->n1, c->n2, ty, tx.lam, c->pen, gate, c->stream);
  }
  {
    ProfScope ps(c, RSFDE_K_PRECOND_ROWS);
    launch_precond_rows<T, Tz>(t2a, t2b, c->phi, z, c->n1, c->n2, tx, gate, c->stream);
  }
}

// The right side and guess of a step (a1): read u^{k-1}, u^{k-2} and s when
// given, the mask bits; write b and x0.
double rhs_bytes(const rsfde_ctx* c, bool has_uu, bool has_src) {
  const double N = (double)c->N;
  return (8.0 + (has_uu ? 8.0 : 0.0) + (has_src ? 8.0 : 0.0) + 16.0) * N + N / 8.0;
}

void enqueue_init(rsfde_ctx* c) {
  ProfScope ps(c, RSFDE_K_OTHER);
  launch_init_state(c->st, c->opts.restart, c->opts.max_iter, c->opts.tol, c->stream);
}

void enqueue_rhs(rsfde_ctx* c, const double* u, const double* uu, const double* src, double* b, double* x0) {
  ProfScope ps(c, RSFDE_K_OTHER);
  launch_rhs(u, uu, src, c->phi, c->dt, b, x0, c->N, c->partials, c->st, c->stream);
}

// One FGMRES(m) cycle: m gated Arnoldi iterations, the solution update and
// the true residual with the restart decision.  Nothing is read on the host.
// Krylov basis element type Tv: double, df or float (basis_kind).
template <typename Tz, typename Tv>
void enqueue_cycle_t(rsfde_ctx* c) {
  const size_t N = c->N;
  const int m = c->opts.restart;
  const int* gi = &c->st->run_iter;
  const int* gc = &c->st->run_cycle;
  Tz* Z = static_cast<Tz*>(c->Z);
  Tv* V = reinterpret_cast<Tv*>(c->V);
  // Tensor-core preconditioner with an FP32 or FP64 basis: the final update
  // pass of iteration j also writes V_{j+1} rounded to BF16 (split BF16: the
  // pair hi, lo) as the first GEMM operand of iteration j+1, whose split pass
  // is then skipped.
  Bf16Out bo{};
  constexpr int kVec = 16 / sizeof(Tv);
  const bool fused = (std::is_same<Tv, float>::value || std::is_same<Tv, double>::value) &&
                     c->opts.use_precond && bf16_precond_on(c) && N % kVec == 0 &&
                     bf16_plan_a0(c->bf16, kVec, &bo);
  for (int j = 0; j < m; ++j) {
    const Tv* vj = V + (size_t)j * N;
    Tz* zj = Z + (size_t)j * N;
    if (c->opts.use_precond) {
      if (bf16_precond_on(c))
        enqueue_precond_bf16<Tz, Tv>(c, vj, &c->st->s[j], zj, gi, fused && j > 0);
      else if (fp32_precond(c))
        enqueue_precond_t<float, Tz, Tv>(c, vj, &c->st->s[j], zj, gi, c->x32.tab, c->y32.tab);
      else
        enqueue_precond_t<double, Tz, Tv>(c, vj, &c->st->s[j], zj, gi, c->x64.tab, c->y64.tab);
    } else {
      ProfScope ps(c, RSFDE_K_OTHER);
      launch_scale_copy<Tv, Tz>(vj, &c->st->s[j], zj, N, gi, c->stream);  // P = I: z_j = v_j
    }
    Tv* w = V + (size_t)(j + 1) * N;
    if constexpr (std::is_same<Tv, df>::value) enqueue_apply_M_t<df, Tz, df>(c, zj, w, gi, c->xdf.tab, c->ydf.tab);
    else if constexpr (std::is_same<Tv, float>::value)
      enqueue_apply_M_t<float, Tz, float>(c, zj, w, gi, c->x32.tab, c->y32.tab);
    else enqueue_apply_M<Tz>(c, zj, w, gi);
    const bool cgs2 = c->opts.arnoldi == RSFDE_CGS2;
    for (int pass = 0; pass < (cgs2 ? 2 : 1); ++pass) {
      {
        ProfScope ps(c, RSFDE_K_MULTIDOT);
        launch_multidot<Tv>(V, N, j, pass, c->partials, c->st, c->stream);
      }
      ProfScope ps(c, RSFDE_K_UPDATE);
      launch_update<Tv>(V, N, j, (!cgs2 || pass == 1) ? 1 : 0, c->partials, c->st, c->stream,
                        fused && j + 1 < m ? &bo : nullptr);
    }
  }
  {
    ProfScope ps(c, RSFDE_K_SOLVE_Y);
    launch_solve_y(c->st, c->stream);
  }
  {
    ProfScope ps(c, RSFDE_K_XUPDATE);
    launch_xupdate<Tz>(c->x, Z, N, c->st, c->stream);
  }
  enqueue_residual(c, gc);
}

// One cycle of left-preconditioned GMRES(m) (Section 5): w = P^-1 M v_j,
// the same Gram-Schmidt and Givens kernels, x += V y, residual P^-1 (b - M x).
void enqueue_cycle_left(rsfde_ctx* c) {
  const size_t N = c->N;
  const int m = c->opts.restart;
  const int* gi = &c->st->run_iter;
  double* tmp = static_cast<double*>(c->Z);  // Z is unused by this variant
  for (int j = 0; j < m; ++j) {
    const double* vj = c->V + (size_t)j * N;
    double* w = c->V + (size_t)(j + 1) * N;
    if (c->opts.use_precond) {
      enqueue_apply_M<double>(c, vj, tmp, gi);    // M V_j
      enqueue_precond64(c, tmp, &c->st->s[j], w, gi);  // P^-1 M v_j
    } else {
      {
        ProfScope ps(c, RSFDE_K_OTHER);
        launch_scale_copy<double, double>(vj, &c->st->s[j], tmp, N, gi, c->stream);
      }
      enqueue_apply_M<double>(c, tmp, w, gi);
    }
    const bool cgs2 = c->opts.arnoldi == RSFDE_CGS2;
    for (int pass = 0; pass < (cgs2 ? 2 : 1); ++pass) {
      {
        ProfScope ps(c, RSFDE_K_MULTIDOT);
        launch_multidot<double>(c->V, N, j, pass, c->partials, c->st, c->stream);
      }
      ProfScope ps(c, RSFDE_K_UPDATE);
      launch_update<double>(c->V, N, j, (!cgs2 || pass == 1) ? 1 : 0, c->partials, c->st, c->stream);
    }
  }
  {
    ProfScope ps(c, RSFDE_K_SOLVE_Y);
    launch_solve_y(c->st, c->stream);
  }
  {
    ProfScope ps(c, RSFDE_K_XUPDATE);
    launch_xupdate_v(c->x, c->V, N, c->st, c->stream);
  }
  enqueue_residual_left(c, &c->st->run_cycle);
}

void enqueue_cycle(rsfde_ctx* c) {
  if (left_variant(c)) enqueue_cycle_left(c);
  else if (basis_kind(c) == BASIS_DF32) {
    if (fp32_precond(c) && c->opts.use_precond) enqueue_cycle_t<float, df>(c);
    else enqueue_cycle_t<double, df>(c);
  } else if (basis_kind(c) == BASIS_FP32) {
    if (fp32_precond(c) && c->opts.use_precond) enqueue_cycle_t<float, float>(c);
    else enqueue_cycle_t<double, float>(c);
  } else if (fp32_precond(c) && c->opts.use_precond) enqueue_cycle_t<float, double>(c);
  else enqueue_cycle_t<double, double>(c);
}

int graph_key(const rsfde_ctx* c) {
  const rsfde_opts& o = c->opts;
  int k = o.basis_prec;
  k = k * 3 + (o.resid_prec == RSFDE_DF32 ? 1 : o.resid_prec == RSFDE_EXACT ? 2 : 0);
  k = k * 65 + o.restart;
  k = k * 5 + o.precond_prec;
  k = k * 4 + o.matvec_prec;
  k = k * 2 + o.arnoldi;
  k = k * 2 + o.use_precond;
  return k * 2 + o.variant;
}

// Captures one FGMRES cycle into the body of a CUDA graph WHILE node whose
// condition the device sets after every cycle (loop_cond_kernel).
int build_cycle_graph(rsfde_ctx* c) {
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->graph_exec = nullptr;
  c->graph = nullptr;
  c->graph_key = -1;
  cudaError_t e;
  if (!c->cap_stream && (e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(e);
  if ((e = cudaGraphCreate(&c->graph, 0)) != cudaSuccess) return cuda_fail(e);
  cudaGraphConditionalHandle h;
  if ((e = cudaGraphConditionalHandleCreate(&h, c->graph, 1, cudaGraphCondAssignDefault)) != cudaSuccess)
    return cuda_fail(e);
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  if ((e = cudaGraphAddNode(&node, c->graph, nullptr, nullptr, 0, &np)) != cudaSuccess) return cuda_fail(e);
  cudaGraph_t body = np.conditional.phGraph_out[0];
  cudaStream_t user = c->stream;
  const bool prof = c->prof_on;
  const int64_t l0 = c->launches;
  c->stream = c->cap_stream;
  c->prof_on = false;
  e = cudaStreamBeginCaptureToGraph(c->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    enqueue_cycle(c);
    launch_loop_cond(h, c->st, c->stream);
    e = cudaStreamEndCapture(c->stream, &body);
  }
  c->launches_per_body = c->launches - l0 + 1;
  c->launches = l0;
  c->stream = user;
  c->prof_on = prof;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph_exec, c->graph, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e);
  }
  c->graph_key = graph_key(c);
  return RSFDE_OK;
}

// Start of a public solve or step: with the profiler on, every earlier launch
// is harvested so that the call's phase times are its own.
void begin_call(rsfde_ctx* c) {
  c->call_bytes = 0;
  if (!c->prof_on) return;
  cudaStreamSynchronize(c->stream);
  prof_harvest(c);
  for (int k = 0; k < RSFDE_K_COUNT; ++k) c->prof_call0[k] = c->prof_ms[k];
}

// Algorithmic HBM bytes of a solve (each grid vector the method reads or
// writes once per use, in the configured precisions): per Arnoldi iteration j
// the preconditioner (read v, write z), the operator (read z, write w, the
// mask bits) and Gram-Schmidt (e_v N (2j + 4) per pass: the j+1 basis vectors
// and w read by the dots and again by the update, the new vector written);
// per cycle the solution update (read the z of the cycle, read and write x);
// per true residual read x and b and the mask bits, write r.
double solve_bytes(const rsfde_ctx* c, const SolverState& h) {
  const double N = (double)c->N;
  const double ev = left_variant(c) ? 8.0 : (basis_kind(c) == BASIS_FP32 ? 4.0 : 8.0);
  const double ez = (left_variant(c) || !fp32_precond(c)) ? 8.0 : 4.0;
  const double it = (double)h.iters, sj = (double)h.sum_j, cyc = (double)h.cycles;
  const double passes = c->opts.arnoldi == RSFDE_CGS2 ? 2.0 : 1.0;
  double b = 0.0;
  if (c->opts.use_precond) b += it * (ev + ez) * N;
  b += it * ((ez + ev) * N + N / 8.0);
  b += passes * ev * N * (2.0 * sj + 4.0 * it);
  b += ez * it * N + 16.0 * N * cyc;
  b += (cyc + 1.0) * ((16.0 + ev) * N + N / 8.0);
  return b;
}

// Solve M x = b with b = c->b, x = c->x (initial guess), st->bnorm set.
int run_solver(rsfde_ctx* c, rsfde_stats* stats) {
  int rc = ensure_bf16(c);
  if (rc) return rc;
  enqueue_residual(c, &c->st->run_cycle);
  rc = check_launch(c);
  if (rc) return rc;
  if (c->opts.use_graph && !c->prof_on) {
    if (c->graph_key != graph_key(c) && (rc = build_cycle_graph(c))) return rc;
    cudaError_t e = cudaGraphLaunch(c->graph_exec, c->stream);
    if (e != cudaSuccess) return cuda_fail(e);
  } else {
    const size_t head = offsetof(SolverState, counter);
    // each cycle does at least one iteration, so max_iter + 1 cycles bound the loop
    for (long guard = 0;; ++guard) {
      if (guard > (long)c->opts.max_iter + 1) return RSFDE_ENOTCONV;
      cudaError_t e = cudaMemcpyAsync(c->st_host, c->st, head, cudaMemcpyDeviceToHost, c->stream);
      if (e != cudaSuccess) return cuda_fail(e);
      if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(e);
      if (c->prof_on) prof_harvest(c);
      if (!c->st_host->run_cycle) break;
      enqueue_cycle(c);
      if ((rc = check_launch(c))) return rc;
    }
  }
  {
    ProfScope ps(c, RSFDE_K_OTHER);
    launch_finalize(c->x, c->N, c->st, c->stream);
  }
  cudaError_t e = cudaMemcpyAsync(c->st_host, c->st, sizeof(SolverState), cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(e);
  const SolverState& h = *c->st_host;
  if (c->opts.use_graph && !c->prof_on) c->launches += (int64_t)h.body_runs * c->launches_per_body;
  if (c->bf16 && bf16_precond_on(c) && (rc = bf16_plan_error(c->bf16, c->stream))) return rc;
  if (stats) {
    stats->iters = h.iters;
    stats->restarts = h.cycles > 0 ? h.cycles - 1 : 0;
    stats->converged = h.converged;
    stats->status = h.status;
    stats->rel_res = h.rel_res;
    stats->bnorm = h.bnorm;
    stats->bytes = c->call_bytes + solve_bytes(c, h);
    // phases: [0] right side, norms, loop control; [1] operator; [2]
    // preconditioner; [3] Gram-Schmidt and Givens; [4] back substitution;
    // [5] solution update and true residual
    static const int phase[RSFDE_K_COUNT] = {1, 1, 2, 2, 2, 3, 3, 5, 0, 2, 5, 5, 4};
    for (int k = 0; k < 6; ++k) stats->t_ms[k] = 0.0;
    if (c->prof_on) {
      prof_harvest(c);
      for (int k = 0; k < RSFDE_K_COUNT; ++k) stats->t_ms[phase[k]] += c->prof_ms[k] - c->prof_call0[k];
    }
  }
  return h.status;
}

// ---- tile-shape autotuning ----------------------------------------------------
template <typename Fn>
float time_calls(rsfde_ctx* c, int reps, Fn fn) {
  fn();  // warm-up (also sets the kernel's shared-memory attribute)
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a, c->stream);
  for (int r = 0; r < reps; ++r) fn();
  cudaEventRecord(b, c->stream);
  cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms / reps;
}

int log2_of(int L) {
  int k = 0;
  while ((1 << k) < L) ++k;
  return k;
}

// Tries every feasible tile shape F of one kernel family and records the fastest.
template <typename T, typename Fn>
int tune_one(rsfde_ctx* c, int kind, int L, int items, int reps, Fn run) {
  const int Fmax = max_groups<T>(L, items);
  int best = 1;
  float best_ms = 1e30f;
  for (int F = 1; F <= Fmax; F *= 2) {
    tune_force_groups(F);
    const float ms = time_calls(c, reps, run);
    if (ms < best_ms) {
      best_ms = ms;
      best = F;
    }
  }
  tune_force_groups(0);
  tune_record(kind, log2_of(L), sizeof(T) == 8, best);
  return best;
}

// Times the operator in the types the solver uses: FP64 z and w, or (FP32 or
// double-FP32 arithmetic) an FP32 z and a w of the basis type Tw.
template <typename T, typename Tw>
void tune_operator(rsfde_ctx* c, int reps, const AxisTables<T>& tx, const AxisTables<T>& ty, int* chosen) {
  using Tz = typename std::conditional<std::is_same<T, double>::value, double, float>::type;
  const Tz* z = reinterpret_cast<const Tz*>(c->V);
  Tw* w = reinterpret_cast<Tw*>(c->V + c->N);
  chosen[TK_TOEP_ROWS] = tune_one<T>(c, TK_TOEP_ROWS, tx.L, (c->n2 + 1) / 2, reps, [&] {
    launch_toeplitz_rows<T, Tz>(z, c->tmpx, c->phi, c->pen, c->n1, c->n2, tx, nullptr, c->stream);
  });
  chosen[TK_TOEP_COLS] = tune_one<T>(c, TK_TOEP_COLS, ty.L, (c->n1 + 1) / 2, reps, [&] {
    launch_toeplitz_cols<T, Tz, Tw>(MODE_APPLY, z, c->tmpx, c->phi, c->pen, nullptr, w, c->n1, c->n2, ty, nullptr,
                                    nullptr, nullptr, c->stream);
  });
}

// Times the true residual's two passes (FP64 x and b; the residual written
// into the first basis vector) in arithmetic T.  x, b, the basis and the
// solver state are scratch here: every solve re-initialises them.
template <typename T>
void tune_residual(rsfde_ctx* c, int reps, const AxisTables<T>& tx, const AxisTables<T>& ty, int* chosen) {
  cudaMemsetAsync(c->x, 0, c->N * sizeof(double), c->stream);
  cudaMemsetAsync(c->b, 0, c->N * sizeof(double), c->stream);
  chosen[TK_TOEP_ROWS] = tune_one<T>(c, TK_TOEP_ROWS, tx.L, (c->n2 + 1) / 2, reps, [&] {
    launch_toeplitz_rows<T, double>(c->x, c->tmpx, c->phi, c->pen, c->n1, c->n2, tx, nullptr, c->stream);
  });
  chosen[TK_TOEP_COLS] = tune_one<T>(c, TK_TOEP_COLS, ty.L, (c->n1 + 1) / 2, reps, [&] {
    if (basis_kind(c) == BASIS_FP32)
      launch_toeplitz_cols<T, double, float>(MODE_RESIDUAL, c->x, c->tmpx, c->phi, c->pen, c->b,
                                             reinterpret_cast<float*>(c->V), c->n1, c->n2, ty, nullptr, c->partials,
                                             c->st, c->stream);
    else
      launch_toeplitz_cols<T, double, double>(MODE_RESIDUAL, c->x, c->tmpx, c->phi, c->pen, c->b, c->V, c->n1,
                                              c->n2, ty, nullptr, c->partials, c->st, c->stream);
  });
}

template <typename T>
void tune_precond(rsfde_ctx* c, int reps, const AxisTables<T>& tx, const AxisTables<T>& ty, int* chosen) {
  T* t1 = static_cast<T*>(c->T1);
  T* t2a = static_cast<T*>(c->T2a);
  T* t2b = static_cast<T*>(c->T2b);
  chosen[TK_DST_ROWS] = tune_one<T>(c, TK_DST_ROWS, tx.L, c->n2, reps, [&] {
    if (basis_kind(c) == BASIS_DF32)
      launch_dst_rows<T, df, T>(reinterpret_cast<const df*>(c->V), nullptr, t1, c->n1, c->n2, tx, nullptr,
                                c->stream);
    else if (basis_kind(c) == BASIS_FP32)
      launch_dst_rows<T, float, T>(reinterpret_cast<const float*>(c->V), nullptr, t1, c->n1, c->n2, tx, nullptr,
                                   c->stream);
    else launch_dst_rows<T, double, T>(c->V, nullptr, t1, c->n1, c->n2, tx, nullptr, c->stream);
  });
  chosen[TK_PRE_COLS] = tune_one<T>(c, TK_PRE_COLS, ty.L, c->n1, reps, [&] {
    launch_precond_cols<T>(t1, t2a, t2b, c->n1, c->n2, ty, tx.lam, c->pen, nullptr, c->stream);
  });
  chosen[TK_PRE_ROWS] = tune_one<T>(c, TK_PRE_ROWS, tx.L, c->n2, reps, [&] {
    launch_precond_rows<T, double>(t2a, t2b, c->phi, c->V + c->N, c->n1, c->n2, tx, nullptr, c->stream);
  });
}

int autotune_ctx(rsfde_ctx* c, int reps, int32_t* chosen_out) {
  int chosen[TK_COUNT] = {0};
  const size_t bytes = c->N * sizeof(double);
  cudaMemsetAsync(c->V, 0, 2 * bytes, c->stream);  // defined inputs for the timing runs
  cudaMemsetAsync(c->T1, 0, bytes, c->stream);
  cudaMemsetAsync(c->T2a, 0, bytes, c->stream);
  cudaMemsetAsync(c->T2b, 0, bytes, c->stream);
  const bool b64 = basis_kind(c) == BASIS_FP64;
  if (c->opts.matvec_prec == RSFDE_DF32) {
    if (b64) tune_operator<df, double>(c, reps, c->xdf.tab, c->ydf.tab, chosen);
    else tune_operator<df, df>(c, reps, c->xdf.tab, c->ydf.tab, chosen);
  } else if (c->opts.matvec_prec == RSFDE_FP32) {
    if (b64) tune_operator<float, double>(c, reps, c->x32.tab, c->y32.tab, chosen);
    else tune_operator<float, float>(c, reps, c->x32.tab, c->y32.tab, chosen);
  } else {
    tune_operator<double, double>(c, reps, c->x64.tab, c->y64.tab, chosen);
  }
  // the double-FP32 true residual runs the same transform families in 8-byte
  // arithmetic (recorded separately from the 4-byte shapes): timed as itself
  if (c->opts.resid_prec == RSFDE_DF32 && c->opts.matvec_prec != RSFDE_DF32 && !left_variant(c)) {
    int unused[TK_COUNT] = {0};
    tune_residual<df>(c, reps, c->xdf.tab, c->ydf.tab, unused);
  }
  if (c->opts.precond_prec == RSFDE_FP32) tune_precond<float>(c, reps, c->x32.tab, c->y32.tab, chosen);
  else if (c->opts.precond_prec == RSFDE_FP64) tune_precond<double>(c, reps, c->x64.tab, c->y64.tab, chosen);
  int bn[4] = {0, 0, 0, 0};
  int rc = RSFDE_OK;
  if (bf16_precond_on(c) && (rc = ensure_bf16(c)) == RSFDE_OK)
    rc = bf16_plan_autotune(c->bf16, c->V, static_cast<float*>(c->Z), c->phi, c->pen, c->stream, reps, bn);
  if (rc != RSFDE_OK) return rc;
  c->graph_key = -1;  // captured launches carry the old shapes
  if (chosen_out) {
    for (int k = 0; k < TK_COUNT; ++k) chosen_out[k] = chosen[k];
    for (int k = 0; k < 4; ++k) chosen_out[TK_COUNT + k] = bn[k];
  }
  rc = check_launch(c);
  if (rc == RSFDE_OK) rc = cuda_fail(cudaStreamSynchronize(c->stream));
  return rc;
}

// ---- batched instances: one CUDA graph advances every instance by a step ---

// Captures fn(c) (work enqueued on c->stream) into a child-graph node of g.
template <typename Fn>
cudaError_t add_captured(rsfde_ctx* c, cudaGraph_t g, const cudaGraphNode_t* deps, size_t ndeps, Fn fn,
                         cudaGraphNode_t* out) {
  cudaError_t e;
  if (!c->cap_stream && (e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return e;
  cudaGraph_t child;
  if ((e = cudaGraphCreate(&child, 0)) != cudaSuccess) return e;
  cudaStream_t user = c->stream;
  const bool prof = c->prof_on;
  c->stream = c->cap_stream;
  c->prof_on = false;
  e = cudaStreamBeginCaptureToGraph(c->stream, child, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    fn(c);
    e = cudaStreamEndCapture(c->stream, &child);
  }
  c->stream = user;
  c->prof_on = prof;
  if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(out, g, deps, ndeps, child);
  cudaGraphDestroy(child);
  return e;
}

// The instance's device-side loop over FGMRES cycles (a WHILE node) after deps.
cudaError_t add_cycle_loop(rsfde_ctx* c, cudaGraph_t g, const cudaGraphNode_t* deps, size_t ndeps,
                           cudaGraphNode_t* out) {
  cudaGraphConditionalHandle h;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  if ((e = cudaGraphAddNode(out, g, deps, nullptr, ndeps, &np)) != cudaSuccess) return e;
  cudaGraph_t body = np.conditional.phGraph_out[0];
  cudaStream_t user = c->stream;
  const bool prof = c->prof_on;
  const int64_t l0 = c->launches;
  c->stream = c->cap_stream;
  c->prof_on = false;
  e = cudaStreamBeginCaptureToGraph(c->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    enqueue_cycle(c);
    launch_loop_cond(h, c->st, c->stream);
    e = cudaStreamEndCapture(c->stream, &body);
  }
  c->launches_per_body = c->launches - l0 + 1;
  c->launches = l0;
  c->stream = user;
  c->prof_on = prof;
  return e;
}

}  // namespace

struct rsfde_batch {
  int count = 0;
  std::vector<rsfde_ctx*> ctx;
  std::vector<double*> ring;  // per instance: u^{k-1}, u^{k-2}, source (3 N doubles)
  std::vector<int> has_src;
  cudaStream_t stream = nullptr;
  cudaGraphExec_t exec[2] = {nullptr, nullptr};  // [0]: first step (no u^{k-2}), [1]: later steps
  int64_t launches_pro[2] = {0, 0}, launches_epi = 0;
  int steps_done = 0;
  int64_t launches = 0;
  // Multi-instance form: every phase of every instance in one launch.
  bool multi = false;
  BatchInst* inst = nullptr;  // device array of count descriptors
  int* prefixes = nullptr;    // device: every MultiGrid's block offsets
  int* runs = nullptr;        // device: loop-body runs of the current step's graph
  MultiGrid g_trows, g_tcols, g_drows, g_pcols, g_prows, g_rhs, g_xupd, g_fin, g_rrows, g_rcols;
  std::vector<MultiGrid> g_dot, g_upd;  // per Arnoldi column j (one active array shared by all j)
  int* actives = nullptr;               // device: the active prefixes
  // split-BF16 preconditioner of the lock-step form: the split and the four
  // grouped GEMMs, their descriptors, and the GEMM launches' give-up flag
  bool bf16 = false;
  MultiGrid g_split, g_gemm[4];
  // exact true residual (resid_prec RSFDE_EXACT): transforms and Chinese
  // remaindering of the row and the column pass
  bool exact = false;
  MultiGrid g_nrows, g_crows, g_ncols, g_ccols;
  void* gdesc = nullptr;
  int* gemm_err = nullptr;
  int* sched = nullptr;  // device: the dynamic hand-out counters of the Gram-Schmidt launches
  int64_t launches_per_body = 0;
  cudaStream_t cap = nullptr;
};

namespace {

void free_batch(rsfde_batch* b) {
  if (!b) return;
  if (b->inst) cudaFree(b->inst);
  if (b->prefixes) cudaFree(b->prefixes);
  if (b->actives) cudaFree(b->actives);
  if (b->runs) cudaFree(b->runs);
  bf16_group_destroy(b->gdesc);
  if (b->gemm_err) cudaFree(b->gemm_err);
  if (b->sched) cudaFree(b->sched);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (auto& x : b->exec)
    if (x) cudaGraphExecDestroy(x);
  for (double* r : b->ring)
    if (r) cudaFree(r);
  for (rsfde_ctx* c : b->ctx) free_ctx(c);
  delete b;
}

// ---- multi-instance form ------------------------------------------------------
// The batch advances in lock step: every kernel of the FGMRES cycle is one
// launch over all instances (each on its own virtual grid, gated by its own
// solver flags), and the cycles repeat while any instance still runs.  It
// covers the FFT preconditioner in FP32 with the FP32 operator, an FP64 or
// FP32 basis and the FP64 true residual, and the split-BF16 tensor-core
// preconditioner with the FP32 operator, the FP64 basis and the FP64 true
// residual; other options use the graph of per-instance branches
// (build_batch_graph).
enum { MV_FP32_B64, MV_FP32_B32, MV_BF16X3_B64, MV_NONE };
int multi_form(const rsfde_opts& o) {
  if (o.variant != RSFDE_FGMRES_RIGHT || !o.use_precond || o.matvec_prec != RSFDE_FP32) return MV_NONE;
  if (o.resid_prec == RSFDE_EXACT && o.basis_prec != RSFDE_FP64) return MV_NONE;
  if (o.resid_prec != RSFDE_FP64 && o.resid_prec != RSFDE_EXACT) return MV_NONE;
  if (o.precond_prec == RSFDE_BF16X3) return o.basis_prec == RSFDE_FP64 ? MV_BF16X3_B64 : MV_NONE;
  if (o.precond_prec != RSFDE_FP32) return MV_NONE;
  return o.basis_prec == RSFDE_FP64 ? MV_FP32_B64 : MV_FP32_B32;
}

// One FGMRES cycle of every instance: operator arithmetic Tm, basis Tv,
// true-residual arithmetic (FP64 or double-FP32).
template <typename Tm, typename Tv>
void enqueue_multi_residual(rsfde_batch* b, cudaStream_t s) {
  if (b->exact) launch_exact_multi(b->inst, b->g_nrows, b->g_crows, b->g_ncols, b->g_ccols, s);
  else launch_residual_multi<double, Tv>(b->inst, b->g_rrows, b->g_rcols, s);
}
// Active prefixes of the families a phase uses: the Arnoldi iteration at
// column j (gate run_iter), or the cycle end (gate run_cycle).
void enqueue_compact_iter(rsfde_batch* b, int j, cudaStream_t s) {
  CompactArgs a{};
  const MultiGrid* fft[] = {&b->g_drows, &b->g_pcols, &b->g_prows, &b->g_trows, &b->g_tcols, &b->g_dot[j],
                            &b->g_upd[j]};
  const MultiGrid* gem[] = {&b->g_split,    &b->g_gemm[0], &b->g_gemm[1], &b->g_gemm[2], &b->g_gemm[3],
                            &b->g_trows,    &b->g_tcols,   &b->g_dot[j],  &b->g_upd[j]};
  const MultiGrid* const* fam = b->bf16 ? gem : fft;
  a.nfam = b->bf16 ? 9 : 7;
  for (int f = 0; f < a.nfam; ++f) {
    a.prefix[f] = fam[f]->prefix;
    a.active[f] = fam[f]->active;
  }
  launch_compact_multi(b->inst, b->count, 0, a, s);
}
void enqueue_compact_cycle(rsfde_batch* b, cudaStream_t s) {
  CompactArgs a{};
  const MultiGrid* fft[] = {&b->g_xupd, &b->g_rrows, &b->g_rcols};
  const MultiGrid* ex[] = {&b->g_xupd, &b->g_nrows, &b->g_crows, &b->g_ncols, &b->g_ccols};
  const MultiGrid* const* fam = b->exact ? ex : fft;
  a.nfam = b->exact ? 5 : 3;
  for (int f = 0; f < a.nfam; ++f) {
    a.prefix[f] = fam[f]->prefix;
    a.active[f] = fam[f]->active;
  }
  launch_compact_multi(b->inst, b->count, 1, a, s);
}

template <typename Tm, typename Tv>
void enqueue_multi_cycle(rsfde_batch* b, cudaStream_t s) {
  const rsfde_opts& o = b->ctx[0]->opts;
  const bool cgs2 = o.arnoldi == RSFDE_CGS2;
  for (int j = 0; j < o.restart; ++j) {
    enqueue_compact_iter(b, j, s);
    if (b->bf16) {
      launch_split_multi(b->inst, b->g_split, j, s);
      for (int k = 0; k < 4; ++k)
        launch_bf16_group(k, b->gdesc, b->count, b->g_gemm[k].active, b->g_gemm[k].total, j, b->gemm_err, s);
    } else {
      launch_precond_multi<float, float, Tv>(b->inst, b->g_drows, b->g_pcols, b->g_prows, j, s);
    }
    launch_operator_multi<Tm, float, Tv>(b->inst, b->g_trows, b->g_tcols, j, s);
    for (int pass = 0; pass < (cgs2 ? 2 : 1); ++pass) {
      launch_multidot_multi<Tv>(b->inst, b->g_dot[j], j, pass, s);
      launch_update_multi<Tv>(b->inst, b->g_upd[j], j, (!cgs2 || pass == 1) ? 1 : 0,
                              b->bf16 && j + 1 < o.restart ? 1 : 0, s);
    }
  }
  launch_solve_y_multi(b->inst, b->count, s);
  enqueue_compact_cycle(b, s);
  launch_xupdate_multi<float>(b->inst, b->g_xupd, s);
  enqueue_multi_residual<Tm, Tv>(b, s);
}
void enqueue_multi_cycle_any(rsfde_batch* b, cudaStream_t s) {
  if (multi_form(b->ctx[0]->opts) != MV_FP32_B32) enqueue_multi_cycle<float, double>(b, s);
  else enqueue_multi_cycle<float, float>(b, s);
}
void enqueue_multi_residual_any(rsfde_batch* b, cudaStream_t s) {
  if (multi_form(b->ctx[0]->opts) != MV_FP32_B32) enqueue_multi_residual<float, double>(b, s);
  else enqueue_multi_residual<float, float>(b, s);
}
// Launches of one loop-body run: per Arnoldi column the compaction, the
// preconditioner (three FFT passes, or the split and four GEMMs), two
// operator passes, multi-dot and update (two more with CGS2); then the back
// substitution, compaction, solution update, residual (2) and loop condition.
int64_t multi_body_launches(const rsfde_batch* b) {
  const rsfde_opts& o = b->ctx[0]->opts;
  const int per_col = 1 + (b->bf16 ? 5 : 3) + 2 + (o.arnoldi == RSFDE_CGS2 ? 4 : 2);
  return (int64_t)o.restart * per_col + 6 + (b->exact ? 2 : 0);  // the exact residual: four launches
}

// Device descriptors and the prefixes of every multi-instance grid.
int setup_multi(rsfde_batch* b) {
  const rsfde_opts& o = b->ctx[0]->opts;
  if (multi_form(o) == MV_NONE) return RSFDE_OK;
  if (b->count > kMaxBatchMulti) return RSFDE_OK;  // the active prefix is held in shared memory
  for (rsfde_ctx* c : b->ctx)
    if (c->x64.tab.L > 4096 || c->y64.tab.L > 4096) return RSFDE_OK;  // one 256-thread group per transform at most
  const int n = b->count, m = o.restart;
  const bool bf16 = multi_form(o) == MV_BF16X3_B64;
  if (bf16)
    for (rsfde_ctx* c : b->ctx) {
      const int rc = ensure_bf16(c);
      if (rc != RSFDE_OK) return rc;
    }
  std::vector<BatchInst> hi(n);
  std::vector<Bf16GroupInst> gin;
  for (int i = 0; i < n; ++i) {
    rsfde_ctx* c = b->ctx[i];
    BatchInst& I = hi[i];
    I.n1 = c->n1;
    I.n2 = c->n2;
    I.N = c->N;
    I.pen = c->pen;
    I.dt = c->dt;
    I.phi = c->phi;
    I.V = c->V;
    I.Z = c->Z;
    I.tmpx = c->tmpx;
    I.T1 = c->T1;
    I.T2a = c->T2a;
    I.T2b = c->T2b;
    I.b = c->b;
    I.x = c->x;
    I.partials = c->partials;
    I.st = c->st;
    I.u_prev = b->ring[i];
    I.u_pp = b->ring[i] + c->N;
    I.src = b->has_src[i] ? b->ring[i] + 2 * c->N : nullptr;
    I.x64 = c->x64.tab;
    I.y64 = c->y64.tab;
    I.x32 = c->x32.tab;
    I.y32 = c->y32.tab;
    I.xdf = c->xdf.tab;
    I.ydf = c->ydf.tab;
    I.a0 = I.a0_lo = nullptr;
    I.a0_ld = I.a0_hk = I.a0_fused = 0;
    I.ex = c->xex.tab;
    I.ey = c->yex.tab;
    I.esc = exact_scratch(c);
    if (bf16) {
      // as the single-instance cycle: the basis update writes the next
      // operand when the plan takes it (enqueue_cycle_t's `fused`)
      Bf16Out bo{};
      I.a0_fused = (c->N % 2 == 0 && bf16_plan_a0(c->bf16, 2, &bo)) ? 1 : 0;
      bf16_plan_a0_any(c->bf16, &bo);
      I.a0 = bo.a0;
      I.a0_lo = bo.lo;
      I.a0_ld = bo.ld;
      I.a0_hk = bo.hk;
      gin.push_back(Bf16GroupInst{c->bf16, c->pen, c->Z, c->N * sizeof(float), 0, c->st->s, I.a0_fused});
    }
  }
  // block counts of every family, instance by instance
  const bool b64 = o.basis_prec == RSFDE_FP64;
  auto ceil_div = [](long a, long q) { return (int)((a + q - 1) / q); };
  std::vector<std::vector<int>> counts;
  std::vector<MultiGrid*> grids;
  auto family = [&](MultiGrid* g, std::function<int(rsfde_ctx*)> blocks, std::function<int(rsfde_ctx*)> log2L) {
    std::vector<int> v(n);
    g->l2mask = 0;
    for (int i = 0; i < n; ++i) {
      v[i] = blocks(b->ctx[i]);
      if (log2L) g->l2mask |= 1u << log2L(b->ctx[i]);
    }
    counts.push_back(v);
    grids.push_back(g);
  };
  auto lx = [](rsfde_ctx* c) { return c->x64.tab.log2L; };
  auto ly = [](rsfde_ctx* c) { return c->y64.tab.log2L; };
  family(&b->g_trows, [&](rsfde_ctx* c) { return ceil_div((c->n2 + 1) / 2, multi_groups(c->x64.tab.L)); }, lx);
  family(&b->g_tcols, [&](rsfde_ctx* c) { return ceil_div((c->n1 + 1) / 2, multi_groups(c->y64.tab.L)); }, ly);
  family(&b->g_drows, [&](rsfde_ctx* c) { return ceil_div(c->n2, multi_groups(c->x64.tab.L)); }, lx);
  family(&b->g_pcols, [&](rsfde_ctx* c) { return ceil_div(c->n1, multi_groups(c->y64.tab.L)); }, ly);
  family(&b->g_prows, [&](rsfde_ctx* c) { return ceil_div(c->n2, multi_groups(c->x64.tab.L)); }, lx);
  family(&b->g_rrows, [&](rsfde_ctx* c) { return ceil_div((c->n2 + 1) / 2, multi_groups(c->x64.tab.L)); }, lx);
  family(&b->g_rcols, [&](rsfde_ctx* c) { return ceil_div((c->n1 + 1) / 2, multi_groups(c->y64.tab.L)); }, ly);
  family(&b->g_rhs, [&](rsfde_ctx* c) { return vec_grid(c->N); }, nullptr);
  family(&b->g_xupd, [&](rsfde_ctx* c) { return xupdate_blocks(c->N, 4); }, nullptr);
  family(&b->g_fin, [&](rsfde_ctx* c) { return vec_grid(c->N); }, nullptr);
  b->g_dot.assign(m, MultiGrid{});
  b->g_upd.assign(m, MultiGrid{});
  for (int j = 0; j < m; ++j) {
    family(&b->g_dot[j], [&](rsfde_ctx* c) {
      return b64 ? multidot_blocks<double>(c->N, j) : multidot_blocks<float>(c->N, j);
    }, nullptr);
    family(&b->g_upd[j], [&](rsfde_ctx* c) {
      return b64 ? update_blocks<double>(c->N, j) : update_blocks<float>(c->N, j);
    }, nullptr);
  }
  const bool exact = o.resid_prec == RSFDE_EXACT;
  if (exact) {  // the exact residual's transforms (vector groups x primes) and remaindering
    family(&b->g_nrows, [&](rsfde_ctx* c) { return exact_multi_ntt_blocks(c->xex.tab.L, c->n2); },
           [](rsfde_ctx* c) { return c->xex.tab.log2L; });
    family(&b->g_crows, [&](rsfde_ctx* c) { return vec_grid(c->N); }, nullptr);
    family(&b->g_ncols, [&](rsfde_ctx* c) { return exact_multi_ntt_blocks(c->yex.tab.L, c->n1); },
           [](rsfde_ctx* c) { return c->yex.tab.log2L; });
    family(&b->g_ccols, [&](rsfde_ctx* c) { return vec_grid(c->N); }, nullptr);
  }
  if (bf16) {  // the split (four elements a thread) and each GEMM's tiles
    std::vector<int> tiles[4];
    const int rc = bf16_group_create(gin, &b->gdesc, tiles);
    if (rc != RSFDE_OK) return rc;
    family(&b->g_split, [&](rsfde_ctx* c) { return ceil_div((long)c->N, 4L * kBlock); }, nullptr);
    for (int k = 0; k < 4; ++k) {
      int next = 0;  // family() visits the instances in order
      family(&b->g_gemm[k], [&](rsfde_ctx*) { return tiles[k][next++]; }, nullptr);
    }
  }
  std::vector<int> all;
  std::vector<size_t> off;
  for (auto& v : counts) {
    off.push_back(all.size());
    int acc = 0;
    all.push_back(0);
    for (int c : v) all.push_back(acc += c);
  }
  cudaError_t e = cudaMalloc((void**)&b->inst, sizeof(BatchInst) * n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->prefixes, sizeof(int) * all.size());
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->runs, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(b->runs, 0, sizeof(int));  // loop runs over the batch's life
  if (e == cudaSuccess) e = cudaMemcpy(b->inst, hi.data(), sizeof(BatchInst) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->prefixes, all.data(), sizeof(int) * all.size(), cudaMemcpyHostToDevice);
  // active prefixes: the iteration families (drows, pcols, prows, trows, tcols,
  // dot, upd) and the cycle-end ones (xupd, rrows, rcols); the right side and
  // the epilogue run every instance (active = the full prefix)
  const int nact = 10 + (bf16 ? 5 : 0) + (exact ? 4 : 0);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->actives, sizeof(int) * (size_t)nact * (n + 1));
  if (e == cudaSuccess && bf16) e = cudaMalloc((void**)&b->gemm_err, sizeof(int));
  if (e == cudaSuccess && bf16) e = cudaMemset(b->gemm_err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->sched, 4 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(b->sched, 0, 4 * sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e);
  for (size_t k = 0; k < grids.size(); ++k) {
    grids[k]->prefix = b->prefixes + off[k];
    grids[k]->active = const_cast<int*>(grids[k]->prefix);
    grids[k]->count = n;
    grids[k]->total = all[off[k] + n];
  }
  MultiGrid* own[] = {&b->g_drows, &b->g_pcols, &b->g_prows, &b->g_trows, &b->g_tcols, &b->g_xupd, &b->g_rrows,
                      &b->g_rcols};
  for (int k = 0; k < 8; ++k) own[k]->active = b->actives + (size_t)k * (n + 1);
  // the transform launches hand out their virtual blocks dynamically too (one
  // launch at a time on the batch's stream, so they share one counter pair)
  for (MultiGrid* g : {&b->g_drows, &b->g_pcols, &b->g_prows, &b->g_trows, &b->g_tcols, &b->g_rrows, &b->g_rcols})
    g->sched = b->sched + 2;
  for (int j = 0; j < m; ++j) {  // the Gram-Schmidt launches hand their virtual blocks out dynamically
    b->g_dot[j].active = b->actives + (size_t)8 * (n + 1);
    b->g_upd[j].active = b->actives + (size_t)9 * (n + 1);
    b->g_dot[j].sched = b->sched;
    b->g_upd[j].sched = b->sched + 2;
  }
  if (bf16) {
    b->g_split.active = b->actives + (size_t)10 * (n + 1);
    for (int k = 0; k < 4; ++k) b->g_gemm[k].active = b->actives + (size_t)(11 + k) * (n + 1);
  }
  if (exact) {
    MultiGrid* eg[] = {&b->g_nrows, &b->g_crows, &b->g_ncols, &b->g_ccols};
    for (int k = 0; k < 4; ++k) {
      eg[k]->active = b->actives + (size_t)(nact - 4 + k) * (n + 1);
      eg[k]->sched = b->sched + 2;
    }
  }
  b->bf16 = bf16;
  b->exact = exact;
  b->multi = true;
  return RSFDE_OK;
}

// The source pointer of instance i's descriptor follows has_src.
int update_multi_src(rsfde_batch* b, int i) {
  if (!b->multi) return RSFDE_OK;
  const double* src = b->has_src[i] ? b->ring[i] + 2 * b->ctx[i]->N : nullptr;
  return cuda_fail(cudaMemcpyAsync(reinterpret_cast<char*>(b->inst + i) + offsetof(BatchInst, src), &src,
                                   sizeof(src), cudaMemcpyHostToDevice, b->stream));
}

// Captures fn (work enqueued on stream cap) into a child-graph node of g.
template <typename Fn>
cudaError_t capture_child(cudaStream_t cap, cudaGraph_t g, const cudaGraphNode_t* deps, size_t ndeps, Fn fn,
                          cudaGraphNode_t* out) {
  cudaGraph_t child;
  cudaError_t e = cudaGraphCreate(&child, 0);
  if (e != cudaSuccess) return e;
  e = cudaStreamBeginCaptureToGraph(cap, child, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    fn(cap);
    e = cudaStreamEndCapture(cap, &child);
  }
  if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(out, g, deps, ndeps, child);
  cudaGraphDestroy(child);
  return e;
}

// One time step of every instance as one graph: [reset, right sides, initial
// residuals] -> WHILE(any instance runs: one FGMRES cycle of all) -> [finish,
// rotate the march rings].
int build_batch_graph_multi(rsfde_batch* b, int later) {
  cudaError_t e;
  if (!b->cap && (e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e);
  const rsfde_opts& o = b->ctx[0]->opts;
  cudaGraph_t g;
  if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) return cuda_fail(e);
  cudaGraphNode_t pro, loop, epi;
  e = capture_child(b->cap, g, nullptr, 0, [&](cudaStream_t s) {
    launch_init_multi(b->inst, b->count, o.restart, o.max_iter, o.tol, s);
    launch_rhs_multi(b->inst, b->g_rhs, later, s);
    enqueue_compact_cycle(b, s);
    enqueue_multi_residual_any(b, s);
  }, &pro);
  cudaGraphConditionalHandle h;
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) {
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    e = cudaGraphAddNode(&loop, g, &pro, nullptr, 1, &np);
    if (e == cudaSuccess) {
      cudaGraph_t body = np.conditional.phGraph_out[0];
      e = cudaStreamBeginCaptureToGraph(b->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
      if (e == cudaSuccess) {
        enqueue_multi_cycle_any(b, b->cap);
        launch_loop_cond_multi(h, b->inst, b->count, b->runs, b->cap);
        e = cudaStreamEndCapture(b->cap, &body);
      }
    }
  }
  if (e == cudaSuccess)
    e = capture_child(b->cap, g, &loop, 1, [&](cudaStream_t s) { launch_finish_rotate_multi(b->inst, b->g_fin, s); },
                      &epi);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec[later], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e);
  }
  // launches: 5 in the prologue (reset, right sides, compaction, residual
  // row and column pass), per loop run 8 per Arnoldi column (compaction,
  // three preconditioner passes, two operator passes, multi-dot and update;
  // two more with CGS2) plus the back substitution, compaction, solution
  // update, residual (2) and loop condition, and 1 in the epilogue
  b->launches_pro[later] = b->exact ? 7 : 5;
  b->launches_epi = 1;
  b->launches_per_body = multi_body_launches(b);
  return RSFDE_OK;
}

// The same time step with direct launches and one host check per cycle
// (use_graph = 0: the kernels are ordinary launches, which profilers see).
int run_batch_step_direct(rsfde_batch* b, int later) {
  const rsfde_opts& o = b->ctx[0]->opts;
  cudaStream_t s = b->stream;
  launch_init_multi(b->inst, b->count, o.restart, o.max_iter, o.tol, s);
  launch_rhs_multi(b->inst, b->g_rhs, later, s);
  enqueue_compact_cycle(b, s);
  enqueue_multi_residual_any(b, s);
  int* flag = b->runs;  // reused as the host-read flag in this mode
  int any = 0;
  for (long guard = 0;; ++guard) {
    launch_any_running_multi(b->inst, b->count, flag, s);
    cudaError_t e = cudaMemcpyAsync(&any, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e);
    if (!any || guard > (long)o.max_iter + 1) break;
    enqueue_multi_cycle_any(b, s);
    b->launches += b->launches_per_body;  // the body, its loop check counted as the condition kernel
  }
  launch_finish_rotate_multi(b->inst, b->g_fin, s);
  return cuda_fail(cudaGetLastError());
}

// Builds the graph of one time step of every instance: per instance the
// chain [right side, initial residual] -> WHILE(FGMRES cycle) -> [finalise,
// u^{k-2} <- u^{k-1}, u^{k-1} <- u^k]; the instances' chains are independent.
int build_batch_graph(rsfde_batch* b, int later) {
  if (b->multi) return build_batch_graph_multi(b, later);
  cudaGraph_t g;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return cuda_fail(e);
  for (int i = 0; i < b->count && e == cudaSuccess; ++i) {
    rsfde_ctx* c = b->ctx[i];
    double* u_prev = b->ring[i];
    double* u_pp = u_prev + c->N;
    double* src = b->has_src[i] ? u_prev + 2 * c->N : nullptr;
    cudaGraphNode_t pro, loop, epi;
    const int64_t l0 = c->launches;
    e = add_captured(c, g, nullptr, 0,
                     [&](rsfde_ctx* cc) {
                       enqueue_init(cc);
                       enqueue_rhs(cc, u_prev, later ? u_pp : nullptr, src, cc->b, cc->x);
                       if (left_variant(cc)) enqueue_bnorm(cc);
                       enqueue_residual(cc, &cc->st->run_cycle);
                     },
                     &pro);
    if (i == 0) b->launches_pro[later] = c->launches - l0;
    if (e == cudaSuccess) e = add_cycle_loop(c, g, &pro, 1, &loop);
    const int64_t l1 = c->launches;
    if (e == cudaSuccess)
      e = add_captured(c, g, &loop, 1,
                       [&](rsfde_ctx* cc) {
                         ProfScope ps(cc, RSFDE_K_OTHER);
                         launch_finalize(cc->x, cc->N, cc->st, cc->stream);
                         cudaMemcpyAsync(u_pp, u_prev, cc->N * sizeof(double), cudaMemcpyDeviceToDevice,
                                         cc->stream);
                         cudaMemcpyAsync(u_prev, cc->x, cc->N * sizeof(double), cudaMemcpyDeviceToDevice,
                                         cc->stream);
                       },
                       &epi);
    if (i == 0) b->launches_epi = c->launches - l1;
    c->launches = l0;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec[later], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e);
  }
  return RSFDE_OK;
}

}  // namespace

// ============================================================================
extern "C" {

void rsfde_opts_default(rsfde_opts* o) {
  if (!o) return;
  o->restart = 20;
  o->max_iter = 10000;
  o->tol = 1e-10;
  o->precond_prec = RSFDE_FP64;
  o->arnoldi = RSFDE_CGS;
  o->use_precond = 1;
  o->matvec_prec = RSFDE_FP64;
  o->variant = RSFDE_FGMRES_RIGHT;
  o->use_graph = 1;
  o->stream = nullptr;
  o->resid_prec = RSFDE_FP64;
  o->basis_prec = RSFDE_FP64;
}

const char* rsfde_strerror(int code) {
  switch (code) {
    case RSFDE_OK: return "ok";
    case RSFDE_EINVAL: return "invalid argument";
    case RSFDE_ENOMEM: return "out of memory";
    case RSFDE_ECUDA: return "CUDA error";
    case RSFDE_ENOTCONV: return "GMRES did not converge within max_iter";
    case RSFDE_ENONFINITE: return "non-finite value in the right side or the Arnoldi process";
    case RSFDE_ETIMEOUT: return "device-side wait timed out";
    default: return "unknown error";
  }
}

static int valid_opts(const rsfde_opts* o) {
  if (o->restart < 1 || o->restart > kMaxRestart || o->max_iter < 1 || !(o->tol > 0.0)) return 0;
  if (o->precond_prec != RSFDE_FP64 && o->precond_prec != RSFDE_FP32 && o->precond_prec != RSFDE_BF16X3 &&
      o->precond_prec != RSFDE_BF16)
    return 0;
  if (o->arnoldi != RSFDE_CGS && o->arnoldi != RSFDE_CGS2) return 0;
  if (o->matvec_prec != RSFDE_FP64 && o->matvec_prec != RSFDE_DF32 && o->matvec_prec != RSFDE_FP32) return 0;
  if (o->variant != RSFDE_FGMRES_RIGHT && o->variant != RSFDE_GMRES_LEFT) return 0;
  if (o->resid_prec != RSFDE_FP64 && o->resid_prec != RSFDE_DF32 && o->resid_prec != RSFDE_EXACT) return 0;
  // the exact residual writes an FP64 or FP32 first basis vector
  if (o->resid_prec == RSFDE_EXACT && o->basis_prec == RSFDE_DF32) return 0;
  // the basis stores the operator's output: FP64 takes any operator, the
  // double-FP32 and FP32 bases only their own
  if (o->basis_prec != RSFDE_FP64 && o->basis_prec != o->matvec_prec) return 0;
  if (o->basis_prec != RSFDE_FP64 && o->basis_prec != RSFDE_DF32 && o->basis_prec != RSFDE_FP32) return 0;
  return 1;
}

int rsfde_setup(rsfde_ctx** out, const rsfde_grid* g, const uint8_t* mask, double alpha1, double alpha2,
                double kx, double ky, double dt, double eta, const rsfde_opts* opts) {
  if (!out) return RSFDE_EINVAL;
  *out = nullptr;
  if (!g || !mask || bad_alpha(alpha1) || bad_alpha(alpha2) || !(kx > 0) || !(ky > 0) || !(dt > 0) ||
      !(eta > 0) || g->n1 < 1 || g->n2 < 1 || g->n1 > kMaxN || g->n2 > kMaxN || !(g->bx > g->ax) ||
      !(g->by > g->ay))
    return RSFDE_EINVAL;
  rsfde_opts o;
  rsfde_opts_default(&o);
  if (opts) o = *opts;
  if (!valid_opts(&o)) return RSFDE_EINVAL;
  rsfde_ctx* c = new (std::nothrow) rsfde_ctx();
  if (!c) return RSFDE_ENOMEM;
  cudaGetDevice(&c->device);
  c->stream = static_cast<cudaStream_t>(o.stream);
  c->opts = o;
  c->m_alloc = o.restart;
  c->n1 = g->n1;
  c->n2 = g->n2;
  c->N = (size_t)g->n1 * g->n2;
  c->ax = g->ax;
  c->bx = g->bx;
  c->ay = g->ay;
  c->by = g->by;
  c->alpha1 = alpha1;
  c->alpha2 = alpha2;
  c->kx = kx;
  c->ky = ky;
  c->dt = dt;
  c->eta = eta;
  const size_t N = c->N, m = o.restart;
  c->npartials = (size_t)(kMaxRestart + 2) * (size_t)vec_grid(N);
  if (c->npartials < (size_t)kMaxPartials) c->npartials = kMaxPartials;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  alloc((void**)&c->phi, N);
  alloc((void**)&c->V, (m + 1) * N * sizeof(double));
  alloc(&c->Z, m * N * sizeof(double));
  alloc((void**)&c->tmpx, N * sizeof(double));
  alloc(&c->T1, N * sizeof(double));
  alloc(&c->T2a, N * sizeof(double));
  alloc(&c->T2b, N * sizeof(double));
  alloc((void**)&c->b, N * sizeof(double));
  alloc((void**)&c->x, N * sizeof(double));
  alloc((void**)&c->partials, c->npartials * sizeof(double));
  alloc((void**)&c->st, sizeof(SolverState));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->st_host, sizeof(SolverState));
  if (e != cudaSuccess) {
    free_ctx(c);
    return cuda_fail(e);
  }
  cudaMemsetAsync(c->st, 0, sizeof(SolverState), c->stream);
  {
    ProfScope ps(c, RSFDE_K_OTHER);
    launch_mask_to_phi(mask, c->phi, N, c->stream);
  }
  int rc = build_tables(c);
  if (rc == RSFDE_OK) rc = ensure_bf16(c);
  if (rc == RSFDE_OK) rc = check_launch(c);
  if (rc == RSFDE_OK) rc = cuda_fail(cudaStreamSynchronize(c->stream));
  if (rc != RSFDE_OK) {
    free_ctx(c);
    return rc;
  }
  *out = c;
  return RSFDE_OK;
}

int rsfde_set_params(rsfde_ctx* c, double kx, double ky, double dt) {
  if (!c || !(kx > 0) || !(ky > 0) || !(dt > 0)) return RSFDE_EINVAL;
  c->kx = kx;
  c->ky = ky;
  c->dt = dt;
  return build_tables(c);
}

int rsfde_set_opts(rsfde_ctx* c, const rsfde_opts* o) {
  if (!c || !o || !valid_opts(o) || o->restart > c->m_alloc) return RSFDE_EINVAL;
  c->opts = *o;
  c->stream = static_cast<cudaStream_t>(o->stream);
  return ensure_bf16(c);
}

int rsfde_set_stream(rsfde_ctx* c, void* stream) {
  if (!c) return RSFDE_EINVAL;
  c->stream = static_cast<cudaStream_t>(stream);
  c->opts.stream = stream;
  return RSFDE_OK;
}

int rsfde_solve(rsfde_ctx* c, const double* b, double* x, rsfde_stats* stats) {
  NvtxRange range("rsfde_solve");
  if (!c || !b || !x) return RSFDE_EINVAL;
  const size_t bytes = c->N * sizeof(double);
  begin_call(c);
  cudaMemcpyAsync(c->b, b, bytes, cudaMemcpyDeviceToDevice, c->stream);
  cudaMemcpyAsync(c->x, x, bytes, cudaMemcpyDeviceToDevice, c->stream);
  c->call_bytes = 8.0 * c->N;  // ||b||
  enqueue_init(c);
  enqueue_bnorm(c);
  int rc = check_launch(c);
  if (rc) return rc;
  rc = run_solver(c, stats);
  if (rc == RSFDE_ECUDA || rc == RSFDE_ENOMEM) return rc;
  cudaError_t e = cudaMemcpyAsync(x, c->x, bytes, cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  return rc;
}

int rsfde_rhs(rsfde_ctx* c, const double* u_prev, const double* u_prevprev, const double* src, double* b,
              double* x0) {
  if (!c || !u_prev || !b || !x0) return RSFDE_EINVAL;
  enqueue_init(c);
  enqueue_rhs(c, u_prev, u_prevprev, src, b, x0);
  return check_launch(c);
}

int rsfde_step(rsfde_ctx* c, const double* u_prev, const double* u_prevprev, const double* src, double* u_next,
               rsfde_stats* stats) {
  NvtxRange range("rsfde_step");
  if (!c || !u_prev || !u_next) return RSFDE_EINVAL;
  begin_call(c);
  c->call_bytes = rhs_bytes(c, u_prevprev != nullptr, src != nullptr);
  enqueue_init(c);
  enqueue_rhs(c, u_prev, u_prevprev, src, c->b, c->x);
  if (left_variant(c)) enqueue_bnorm(c);
  int rc = check_launch(c);
  if (rc) return rc;
  rc = run_solver(c, stats);
  if (rc == RSFDE_ECUDA || rc == RSFDE_ENOMEM) return rc;
  cudaError_t e = cudaMemcpyAsync(u_next, c->x, c->N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  return rc;
}

int rsfde_step_host(rsfde_ctx* c, const double* u_prev_h, const double* u_prevprev_h, const double* src_h,
                    double* u_next_h, rsfde_stats* stats) {
  NvtxRange range("rsfde_step_host");
  if (!c || !u_prev_h || !u_next_h) return RSFDE_EINVAL;
  const size_t bytes = c->N * sizeof(double);
  if (!c->hbuf) {
    cudaError_t e = cudaMalloc((void**)&c->hbuf, 3 * bytes);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  double* d_u = c->hbuf;
  double* d_uu = u_prevprev_h ? c->hbuf + c->N : nullptr;
  double* d_src = src_h ? c->hbuf + 2 * c->N : nullptr;
  cudaMemcpyAsync(d_u, u_prev_h, bytes, cudaMemcpyHostToDevice, c->stream);
  if (d_uu) cudaMemcpyAsync(d_uu, u_prevprev_h, bytes, cudaMemcpyHostToDevice, c->stream);
  if (d_src) cudaMemcpyAsync(d_src, src_h, bytes, cudaMemcpyHostToDevice, c->stream);
  begin_call(c);
  c->call_bytes = rhs_bytes(c, d_uu != nullptr, d_src != nullptr);
  enqueue_init(c);
  enqueue_rhs(c, d_u, d_uu, d_src, c->b, c->x);
  if (left_variant(c)) enqueue_bnorm(c);
  int rc = check_launch(c);
  if (rc) return rc;
  rc = run_solver(c, stats);
  if (rc == RSFDE_ECUDA || rc == RSFDE_ENOMEM) return rc;
  cudaError_t e = cudaMemcpyAsync(u_next_h, c->x, bytes, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  return rc;
}

int rsfde_adjoint(rsfde_ctx* c, const double* lam, double* mu, rsfde_stats* stats) {
  NvtxRange range("rsfde_adjoint");
  // M is symmetric (Lemma 2.3): M^T mu = lam is the forward system.
  return rsfde_solve(c, lam, mu, stats);
}

int rsfde_adjoint_step(rsfde_ctx* c, const double* u_prev, const double* u_k, const double* lam, double* mu,
                       double* lam_prev, double* grad_src, double* grad_k, rsfde_stats* stats) {
  NvtxRange range("rsfde_adjoint_step");
  if (!c || !u_prev || !u_k || !lam || !mu || !lam_prev || !grad_k) return RSFDE_EINVAL;
  int rc = rsfde_solve(c, lam, mu, stats);  // M^T = M (Lemma 2.3)
  if (rc == RSFDE_ECUDA || rc == RSFDE_ENOMEM || rc == RSFDE_EINVAL) return rc;
  if (rc != RSFDE_OK) return rc;
  double* ay_u = static_cast<double*>(c->T2a);  // scratch, free after the solve
  {
    ProfScope ps(c, RSFDE_K_TOEPLITZ_ROWS);
    launch_toeplitz_rows<double, double>(u_k, c->tmpx, nullptr, 0.0, c->n1, c->n2, c->x64.tab, nullptr, c->stream);
  }
  {
    ProfScope ps(c, RSFDE_K_TOEPLITZ_COLS);
    launch_toeplitz_cols<double, double>(MODE_RAW, u_k, c->tmpx, c->phi, c->pen, nullptr, ay_u, c->n1, c->n2,
                                         c->y64.tab, nullptr, nullptr, nullptr, c->stream);
  }
  {
    ProfScope ps(c, RSFDE_K_OTHER);
    launch_adjoint_accum(u_prev, mu, c->tmpx, ay_u, c->phi, c->dt, 1.0 / c->kx, 1.0 / c->ky, lam_prev, grad_src,
                         grad_k, c->N, c->partials, c->st, c->stream);
  }
  if ((rc = check_launch(c))) return rc;
  return cuda_fail(cudaStreamSynchronize(c->stream));
}

int rsfde_apply_M(rsfde_ctx* c, const double* z, double* w) {
  NvtxRange range("rsfde_apply_M");
  if (!c || !z || !w) return RSFDE_EINVAL;
  enqueue_apply_M<double>(c, z, w, nullptr);
  return check_launch(c);
}

int rsfde_residual(rsfde_ctx* c, const double* x, const double* b, double* r) {
  NvtxRange range("rsfde_residual");
  if (!c || !x || !b || !r || r == x || r == b) return RSFDE_EINVAL;
  if (c->opts.resid_prec == RSFDE_DF32) return RSFDE_EINVAL;
  enqueue_resid_only(c, x, b, r, nullptr);
  return check_launch(c);
}

int rsfde_apply_precond(rsfde_ctx* c, const double* v, double* z) {
  NvtxRange range("rsfde_apply_precond");
  if (!c || !v || !z) return RSFDE_EINVAL;
  if (bf16_precond_on(c)) {
    int rc = ensure_bf16(c);
    if (rc) return rc;
    enqueue_precond_bf16<double, double>(c, v, nullptr, z, nullptr);
    if ((rc = check_launch(c))) return rc;
    return bf16_plan_error(c->bf16, c->stream);
  }
  if (fp32_precond(c)) enqueue_precond_t<float, double, double>(c, v, nullptr, z, nullptr, c->x32.tab, c->y32.tab);
  else enqueue_precond_t<double, double, double>(c, v, nullptr, z, nullptr, c->x64.tab, c->y64.tab);
  return check_launch(c);
}

int rsfde_dst2(rsfde_ctx* c, const double* v, double* out) {
  NvtxRange range("rsfde_dst2");
  if (!c || !v || !out) return RSFDE_EINVAL;
  {
    ProfScope ps(c, RSFDE_K_DST_ROWS);
    launch_dst_rows<double, double, double>(v, nullptr, c->tmpx, c->n1, c->n2, c->x64.tab, nullptr, c->stream);
  }
  {
    ProfScope ps(c, RSFDE_K_PRECOND_COLS);
    launch_dst_cols<double, double, double>(c->tmpx, out, c->n1, c->n2, c->y64.tab, c->stream);
  }
  return check_launch(c);
}

int rsfde_get_tables(rsfde_ctx* c, double* lam_x, double* lam_y, double* t_x, double* t_y) {
  if (!c) return RSFDE_EINVAL;
  if (lam_x) std::memcpy(lam_x, c->hx_axis.lam.data(), sizeof(double) * c->n1);
  if (lam_y) std::memcpy(lam_y, c->hy_axis.lam.data(), sizeof(double) * c->n2);
  if (t_x) std::memcpy(t_x, c->hx_axis.t.data(), sizeof(double) * c->n1);
  if (t_y) std::memcpy(t_y, c->hy_axis.t.data(), sizeof(double) * c->n2);
  return RSFDE_OK;
}

int rsfde_get_params(rsfde_ctx* c, double* out5) {
  if (!c || !out5) return RSFDE_EINVAL;
  out5[0] = c->cx;
  out5[1] = c->cy;
  out5[2] = c->pen;
  out5[3] = c->hx;
  out5[4] = c->hy;
  return RSFDE_OK;
}

int64_t rsfde_kernel_launches(const rsfde_ctx* c) { return c ? c->launches : 0; }

int rsfde_set_wait_cycles(rsfde_ctx* c, int64_t cycles) {
  if (!c || cycles < 0) return RSFDE_EINVAL;
  c->wait_cycles = cycles;
  bf16_plan_set_wait(c->bf16, cycles);
  return RSFDE_OK;
}

int rsfde_autotune(rsfde_ctx* c, int32_t reps, int32_t* chosen) {
  NvtxRange range("rsfde_autotune");
  if (!c || reps < 1) return RSFDE_EINVAL;
  return autotune_ctx(c, reps, chosen);
}

int rsfde_profile_enable(rsfde_ctx* c, int on) {
  if (!c) return RSFDE_EINVAL;
  c->prof_on = on != 0;
  return RSFDE_OK;
}

int rsfde_profile_read(rsfde_ctx* c, double* ms, int64_t* launches) {
  if (!c) return RSFDE_EINVAL;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  prof_harvest(c);
  for (int k = 0; k < RSFDE_K_COUNT; ++k) {
    if (ms) ms[k] = c->prof_ms[k];
    if (launches) launches[k] = c->prof_n[k];
    c->prof_ms[k] = 0.0;
    c->prof_n[k] = 0;
  }
  return RSFDE_OK;
}

const char* rsfde_kernel_class_name(int k) {
  static const char* names[RSFDE_K_COUNT] = {"toeplitz_rows", "toeplitz_cols", "dst_rows",   "precond_cols",
                                             "precond_rows",  "multidot",      "update",     "xupdate",
                                             "other",         "dst_gemm",      "resid_rows", "resid_cols",
                                             "solve_y"};
  return (k >= 0 && k < RSFDE_K_COUNT) ? names[k] : "unknown";
}

void rsfde_destroy(rsfde_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free_ctx(c);
}

// ---- batched instances -------------------------------------------------------
int rsfde_batch_create(rsfde_batch** out, int32_t count, const rsfde_grid* grids, const uint8_t* const* masks,
                       const double* alpha1, const double* alpha2, const double* kx, const double* ky,
                       const double* dt, const double* eta, const rsfde_opts* opts) {
  if (!out) return RSFDE_EINVAL;
  *out = nullptr;
  if (count < 1 || !grids || !masks || !alpha1 || !alpha2 || !kx || !ky || !dt || !eta) return RSFDE_EINVAL;
  rsfde_batch* b = new (std::nothrow) rsfde_batch();
  if (!b) return RSFDE_ENOMEM;
  b->count = count;
  b->stream = opts ? static_cast<cudaStream_t>(opts->stream) : nullptr;
  for (int i = 0; i < count; ++i) {
    rsfde_ctx* c = nullptr;
    int rc = rsfde_setup(&c, &grids[i], masks[i], alpha1[i], alpha2[i], kx[i], ky[i], dt[i], eta[i], opts);
    if (rc) {
      free_batch(b);
      return rc;
    }
    b->ctx.push_back(c);
    double* r = nullptr;
    cudaError_t e = cudaMalloc(&r, 3 * c->N * sizeof(double));
    if (e != cudaSuccess) {
      free_batch(b);
      return cuda_fail(e);
    }
    cudaMemsetAsync(r, 0, 3 * c->N * sizeof(double), b->stream);
    b->ring.push_back(r);
    b->has_src.push_back(0);
  }
  int rc = cuda_fail(cudaStreamSynchronize(b->stream));
  if (rc == RSFDE_OK) rc = setup_multi(b);
  if (rc != RSFDE_OK) {
    free_batch(b);
    return rc;
  }
  *out = b;
  return RSFDE_OK;
}

int rsfde_batch_set(rsfde_batch* b, int32_t i, const double* u0, const double* src) {
  if (!b || i < 0 || i >= b->count || !u0) return RSFDE_EINVAL;
  rsfde_ctx* c = b->ctx[i];
  const size_t bytes = c->N * sizeof(double);
  cudaMemcpyAsync(b->ring[i], u0, bytes, cudaMemcpyDeviceToDevice, b->stream);
  if (src) cudaMemcpyAsync(b->ring[i] + 2 * c->N, src, bytes, cudaMemcpyDeviceToDevice, b->stream);
  if ((src != nullptr) != (b->has_src[i] != 0)) {  // the graphs (or the descriptor) read the source or not
    b->has_src[i] = src != nullptr;
    int rc = update_multi_src(b, i);
    if (rc != RSFDE_OK) return rc;
    if (!b->multi)
      for (auto& x : b->exec)
        if (x) {
          cudaGraphExecDestroy(x);
          x = nullptr;
        }
  }
  b->steps_done = 0;
  return cuda_fail(cudaStreamSynchronize(b->stream));
}

int rsfde_batch_run(rsfde_batch* b, int32_t steps, rsfde_stats* stats) {
  NvtxRange range("rsfde_batch_run");
  if (!b || steps < 0) return RSFDE_EINVAL;
  const bool direct = b->multi && !b->ctx[0]->opts.use_graph;
  for (int k = 0; k < steps; ++k) {
    const int later = b->steps_done > 0;
    if (direct) {
      if (b->launches_per_body == 0) {
        b->launches_pro[0] = b->launches_pro[1] = b->exact ? 7 : 5;
        b->launches_epi = 1;
        b->launches_per_body = multi_body_launches(b);
      }
      int rc = run_batch_step_direct(b, later);
      if (rc) return rc;
      b->steps_done += 1;
      b->launches += b->launches_pro[later] + b->launches_epi;
      continue;
    }
    if (!b->exec[later]) {
      int rc = build_batch_graph(b, later);
      if (rc) return rc;
    }
    cudaError_t e = cudaGraphLaunch(b->exec[later], b->stream);
    if (e != cudaSuccess) return cuda_fail(e);
    b->steps_done += 1;
    b->launches += (int64_t)(b->multi ? 1 : b->count) * (b->launches_pro[later] + b->launches_epi);
  }
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  const size_t head = offsetof(SolverState, counter);
  int worst = RSFDE_OK;
  if (b->bf16) {  // a GEMM pipeline wait gave up: that launch's output is incomplete
    int flag = 0;
    e = cudaMemcpy(&flag, b->gemm_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && flag) e = cudaMemset(b->gemm_err, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e);
    if (flag) worst = RSFDE_ETIMEOUT;
  }
  for (int i = 0; i < b->count; ++i) {
    rsfde_ctx* c = b->ctx[i];
    e = cudaMemcpy(c->st_host, c->st, head, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e);
    const SolverState& h = *c->st_host;
    if (stats) {
      stats[i].iters = h.iters;
      stats[i].restarts = h.cycles > 0 ? h.cycles - 1 : 0;
      stats[i].converged = h.converged;
      stats[i].status = h.status;
      stats[i].rel_res = 0.0;
      stats[i].bnorm = 0.0;
      for (int k = 0; k < 6; ++k) stats[i].t_ms[k] = 0.0;
      stats[i].bytes = rhs_bytes(c, b->steps_done > 1, b->has_src[i] != 0) + solve_bytes(c, h);
    }
    if (h.status != RSFDE_OK && worst == RSFDE_OK) worst = h.status;
  }
  if (stats) {  // the residual fields follow the counter in the state
    for (int i = 0; i < b->count; ++i) {
      rsfde_ctx* c = b->ctx[i];
      double rr[4];
      e = cudaMemcpy(rr, &c->st->tol, sizeof(rr), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(e);
      stats[i].bnorm = rr[1];
      stats[i].rel_res = rr[3];
    }
  }
  return worst;
}

int rsfde_batch_get(rsfde_batch* b, int32_t i, double* u_out) {
  if (!b || i < 0 || i >= b->count || !u_out) return RSFDE_EINVAL;
  rsfde_ctx* c = b->ctx[i];
  cudaError_t e = cudaMemcpyAsync(u_out, b->ring[i], c->N * sizeof(double), cudaMemcpyDeviceToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return cuda_fail(e);
}

int64_t rsfde_batch_kernel_launches(rsfde_batch* b) {
  if (!b) return 0;
  if (b->multi && !b->ctx[0]->opts.use_graph) return b->launches;  // counted as launched
  if (b->multi) {  // per step the prologue and epilogue, plus every run of the loop body
    int runs = 0;
    if (cudaMemcpy(&runs, b->runs, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return b->launches;
    return b->launches + (int64_t)runs * b->launches_per_body;
  }
  // prologue and epilogue launches per instance-step, plus every replayed cycle
  int64_t n = b->launches;
  for (rsfde_ctx* c : b->ctx) {
    long long runs = 0;
    if (cudaMemcpy(&runs, &c->st->total_body_runs, sizeof(runs), cudaMemcpyDeviceToHost) == cudaSuccess)
      n += (int64_t)runs * c->launches_per_body;
  }
  return n;
}

int rsfde_batch_autotune(rsfde_batch* b, int32_t reps) {
  if (!b || reps < 1) return RSFDE_EINVAL;
  // the recorded shapes are keyed by transform length: tune one instance per length pair
  std::vector<std::pair<int, int>> seen;
  for (rsfde_ctx* c : b->ctx) {
    const std::pair<int, int> key(c->x64.tab.L, c->y64.tab.L);
    bool done = false;
    for (auto& k : seen) done |= (k == key);
    if (done) continue;
    seen.push_back(key);
    int rc = autotune_ctx(c, reps, nullptr);
    if (rc) return rc;
  }
  for (auto& x : b->exec)
    if (x) {
      cudaGraphExecDestroy(x);
      x = nullptr;
    }
  return RSFDE_OK;
}

void rsfde_batch_destroy(rsfde_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  free_batch(b);
}

}  // extern "C"
