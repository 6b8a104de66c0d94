// noalloc.cu -- rsfde_dst2_noalloc: the 2D orthonormal sine transform
// (S_{n2} (x) S_{n1}) v without any device allocation.
//
// Who needs it: code that must not call cudaMalloc -- for example a host
// application or framework that owns every device allocation through its own
// pool, where a stray cudaMalloc would bypass its accounting or fragment the
// memory it manages.  Such callers cannot create an rsfde_ctx, because
// rsfde_setup allocates the context's workspace and tables.
//
// Instead, the intermediate of the two passes (rows, then columns) and the
// per-axis transform tables live in file-scope static __device__ arrays of a
// fixed maximum size (n1, n2 <= RSFDE_NOALLOC_MAX_N).  They are part of the
// library's module, so every GPU that loads the library holds them
// (about 2.1 MB) until the process exits.
#include <cmath>
#include <mutex>

#include "fft.cuh"
#include "internal.h"

using namespace rsfde;

namespace {

constexpr int kMaxN = RSFDE_NOALLOC_MAX_N;
constexpr int kMaxL = 1024;  // power of two >= 2*kMaxN - 1
constexpr int kTableDoubles = 2 * kMaxL + 2 * kMaxN + 2 * kMaxN + 2 * kMaxL;  // tw, chirp, chirp_out, bspec
constexpr int kMaxDevices = 64;

// Intermediate after the row pass (up to kMaxN^2 values) and the two axes' tables.
static __device__ __align__(256) double g_noalloc_scratch[(size_t)kMaxN * kMaxN];
static __device__ __align__(256) double g_noalloc_tables[2 * kTableDoubles];

// Host-side device addresses of the two arrays, looked up once per device,
// and the sizes and stream of the tables last copied to each device.
static double* s_scratch_addr[kMaxDevices];
static double* s_tables_addr[kMaxDevices];
static bool s_ready[kMaxDevices];
static int s_last_n1[kMaxDevices], s_last_n2[kMaxDevices];
static cudaStream_t s_last_stream[kMaxDevices];

// Host staging of the tables: fixed-size, so the call allocates nothing on
// the host either.  cudaMemcpyAsync from pageable memory returns once the
// bytes are staged, so the buffers may be refilled by the next call.  One
// mutex serialises the host side of all calls (the staging buffers and the
// per-device records are process-wide).
static double h_tables[2 * kTableDoubles];
static double h_re[kMaxL], h_im[kMaxL];
static std::mutex s_host_mutex;

int pow2_at_least(int v, int* log2v) {
  int L = 16, lg = 4;
  while (L < v) {
    L <<= 1;
    ++lg;
  }
  *log2v = lg;
  return L;
}

// Fills one axis' sine-transform tables (twiddles, chirps, Bluestein kernel
// spectrum in natural order) at
// h_tables + axis * kTableDoubles.
void fill_axis(int axis, int n, int L, int log2L) {
  double* base = h_tables + (size_t)axis * kTableDoubles;
  double* tw = base;
  double* chirp = tw + 2 * kMaxL;
  double* chirp_out = chirp + 2 * kMaxN;
  double* bspec = chirp_out + 2 * kMaxN;
  for (int j = 0; j < L; ++j) {
    tw[2 * j] = std::cos(2.0 * M_PI * j / L);
    tw[2 * j + 1] = -std::sin(2.0 * M_PI * j / L);
  }
  const long per = 4L * (n + 1);
  const double nrm = std::sqrt(2.0 / (n + 1));
  for (int k = 1; k <= n; ++k) {
    const double ang = M_PI * (double)(((long)k * k) % per) / (2.0 * (n + 1));
    chirp[2 * (k - 1)] = std::cos(ang);
    chirp[2 * (k - 1) + 1] = std::sin(ang);
    chirp_out[2 * (k - 1)] = nrm * std::cos(ang);
    chirp_out[2 * (k - 1) + 1] = nrm * std::sin(ang);
  }
  for (int l = 0; l < L; ++l) h_re[l] = h_im[l] = 0.0;
  for (int d = 0; d < n; ++d) {
    const double ang = -M_PI * (double)(((long)d * d) % per) / (2.0 * (n + 1));
    h_re[d] = std::cos(ang);
    h_im[d] = std::sin(ang);
    if (d > 0) {
      h_re[L - d] = h_re[d];
      h_im[L - d] = h_im[d];
    }
  }
  int s;
  if (log2L & 1) {
    for (int k = 0; k < L / 2; ++k) dif_r2(h_re, h_im, L, k, tw);
    s = L >> 3;
  } else {
    s = L >> 2;
  }
  for (; s >= 1; s >>= 2)
    for (int q = 0; q < L / 4; ++q) dif_r4(h_re, h_im, L, s, q, tw);
  // the DIF leaves the spectrum in bit-reversed order; the kernels want it natural
  for (int l = 0; l < L; ++l) {
    int b = 0;
    for (int x = l, k = 0; k < log2L; ++k, x >>= 1) b = (b << 1) | (x & 1);
    bspec[2 * b] = h_re[l] / L;
    bspec[2 * b + 1] = h_im[l] / L;
  }
}

AxisTables<double> device_axis(const double* dev_tables, int axis, int n, int L, int log2L) {
  const double* base = dev_tables + (size_t)axis * kTableDoubles;
  AxisTables<double> t{};
  t.n = n;
  t.L = L;
  t.log2L = log2L;
  t.tw = base;
  t.chirp = base + 2 * kMaxL;
  t.chirp_out = t.chirp + 2 * kMaxN;
  t.bspec = t.chirp_out + 2 * kMaxN;
  t.sigma = nullptr;  // not used by the sine transform
  t.lam = nullptr;
  return t;
}

}  // namespace

extern "C" int rsfde_dst2_noalloc(int32_t n1, int32_t n2, const double* v, double* out, void* stream) {
  if (n1 < 1 || n2 < 1 || n1 > kMaxN || n2 > kMaxN || !v || !out || v == out) return RSFDE_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RSFDE_ECUDA;
  std::lock_guard<std::mutex> lock(s_host_mutex);
  if (!s_ready[dev]) {
    // once per device, with that device current: the arrays' device addresses
    if (cudaGetSymbolAddress((void**)&s_scratch_addr[dev], g_noalloc_scratch) != cudaSuccess) return RSFDE_ECUDA;
    if (cudaGetSymbolAddress((void**)&s_tables_addr[dev], g_noalloc_tables) != cudaSuccess) return RSFDE_ECUDA;
    s_ready[dev] = true;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int lg1 = 0, lg2 = 0;
  const int L1 = pow2_at_least(2 * n1 - 1, &lg1);
  const int L2 = pow2_at_least(2 * n2 - 1, &lg2);
  // The tables depend only on (n1, n2).  When the previous call on this
  // device had the same sizes and the same stream, the copy it enqueued
  // before its kernels still holds them (stream order); otherwise they are
  // rebuilt and every value the kernels read is rewritten, so nothing else
  // from an earlier call (the arrays keep the last call's contents) is used.
  if (s_last_n1[dev] != n1 || s_last_n2[dev] != n2 || s_last_stream[dev] != s) {
    fill_axis(0, n1, L1, lg1);
    fill_axis(1, n2, L2, lg2);
    s_last_n1[dev] = 0;  // unknown until the copy is enqueued
    if (cudaMemcpyAsync(s_tables_addr[dev], h_tables, sizeof(h_tables), cudaMemcpyHostToDevice, s) != cudaSuccess)
      return RSFDE_ECUDA;
    s_last_n1[dev] = n1;
    s_last_n2[dev] = n2;
    s_last_stream[dev] = s;
  }
  const AxisTables<double> tx = device_axis(s_tables_addr[dev], 0, n1, L1, lg1);
  const AxisTables<double> ty = device_axis(s_tables_addr[dev], 1, n2, L2, lg2);
  launch_dst_rows<double, double>(v, nullptr, s_scratch_addr[dev], n1, n2, tx, nullptr, s);
  launch_dst_cols<double, double, double>(s_scratch_addr[dev], out, n1, n2, ty, s);
  return cudaGetLastError() == cudaSuccess ? RSFDE_OK : RSFDE_ECUDA;
}
