// lbw_spectrum.cu -- mode frequencies of probe series, on the device, in FP64.
//
// The paper reads normal modes off driven frequency sweeps (Sec. IV.A, Fig. Fig.Frequencies;
// Sec. IV.C, Fig. FreqTorus).  For a pulse-excited run the same modes are the peaks of the
// probe signal's spectrum, estimated here:
//   1. mean removed, Hann window w_t = 1/2 - 1/2 cos(2 pi t / (T - 1));
//   2. zero padding to M = smallest power of two >= 4 T; radix-2 Stockham FFT
//      (log2 M passes through global memory, natural-order output);
//   3. |X_j|^2, local maxima above 1e-3 of the largest bin; the k strongest are chosen with
//      warp-shuffle arg-max reductions (ties: lower bin) and sorted by frequency;
//   4. each peak is refined by a parabola through log-power at j-1, j, j+1 and 40
//      golden-section steps on the windowed DTFT over +-1 bin (one CTA per peak; the DTFT
//      sum uses per-thread chunks with a rotation recurrence for e^{-i omega t}).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "lbw_internal.h"

namespace lbw {
namespace {

constexpr int kThreads = 512;
constexpr double kGolden = 0.6180339887498949;

__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) red[0] = s;
  }
  __syncthreads();
  return red[0];
}

// mean of the (summed) series and sum of the window weights
__global__ void stats_kernel(const double* __restrict__ x, long long T, int nser, long long stride,
                             double* out) {
  __shared__ double red[32];
  double s = 0.0, sw = 0.0;
  for (long long t = threadIdx.x; t < T; t += blockDim.x) {
    double v = 0.0;
    for (int p = 0; p < nser; ++p) v += x[(long long)p * stride + t];
    s += v;
    sw += 0.5 - 0.5 * cospi(2.0 * (double)t / (double)(T - 1));
  }
  s = block_sum(s, red);
  sw = block_sum(sw, red);
  if (threadIdx.x == 0) {
    out[0] = s / (double)T;
    out[1] = sw;
  }
}

// xw_t = w_t (x_t - mean) as complex, zero-padded to M
__global__ void window_kernel(const double* __restrict__ x, long long T, int nser, long long stride,
                              const double* __restrict__ stats, long long M, double2* a,
                              double* xw) {
  const double mean = stats[0];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < M;
       t += (long long)gridDim.x * blockDim.x) {
    double v = 0.0;
    if (t < T) {
      for (int p = 0; p < nser; ++p) v += x[(long long)p * stride + t];
      v = (0.5 - 0.5 * cospi(2.0 * (double)t / (double)(T - 1))) * (v - mean);
      xw[t] = v;
    }
    a[t] = make_double2(v, 0.0);
  }
}

// one radix-2 Stockham pass: sub-transforms of size ns are combined into size 2 ns
__global__ void stockham_kernel(const double2* __restrict__ in, double2* __restrict__ out,
                                long long M, long long ns) {
  const long long half = M >> 1;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < half;
       j += (long long)gridDim.x * blockDim.x) {
    const long long k = j & (ns - 1);
    const double2 a0 = in[j], b = in[j + half];
    double s, c;
    sincospi((double)k / (double)ns, &s, &c);  // w = e^{-i pi k / ns}
    const double2 a1 = make_double2(b.x * c + b.y * s, b.y * c - b.x * s);
    const long long d = (j / ns) * 2 * ns + k;
    out[d] = make_double2(a0.x + a1.x, a0.y + a1.y);
    out[d + ns] = make_double2(a0.x - a1.x, a0.y - a1.y);
  }
}

__global__ void power_kernel(const double2* __restrict__ X, long long M, double* P) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j <= M / 2;
       j += (long long)gridDim.x * blockDim.x)
    P[j] = X[j].x * X[j].x + X[j].y * X[j].y;
}

__global__ void max_kernel(const double* __restrict__ P, long long M, double* out) {
  __shared__ double red[32];
  double m = 0.0;
  for (long long j = 1 + threadIdx.x; j <= M / 2; j += blockDim.x) m = fmax(m, P[j]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) out[2] = m;
  }
}

__global__ void candidates_kernel(const double* __restrict__ P, long long M,
                                  const double* __restrict__ stats, double thresh,
                                  long long* cand, unsigned long long* count) {
  const double lim = thresh * stats[2];
  for (long long j = 1 + blockIdx.x * (long long)blockDim.x + threadIdx.x; j < M / 2;
       j += (long long)gridDim.x * blockDim.x) {
    const double p = P[j];
    if (p > P[j - 1] && p >= P[j + 1] && p >= lim) {
      unsigned long long s = atomicAdd(count, 1ULL);
      cand[s] = j;
    }
  }
}

// better(a, b): higher power wins, equal power -> lower bin
__device__ __forceinline__ bool better(double pa, long long ja, double pb, long long jb) {
  return pa > pb || (pa == pb && ja < jb);
}

// lowest-frequency selection: the lower bin wins
__device__ __forceinline__ bool lower(double, long long ja, double, long long jb) { return ja < jb; }

// k rounds of a block-wide arg-max over the candidate list (warp shuffles), then sort; the
// winner of a round is the strongest candidate, or with `lowest` the lowest-frequency one
__global__ void select_kernel(const double* __restrict__ P, long long* cand,
                              const unsigned long long* __restrict__ count, int k,
                              long long* chosen, int* n_chosen, bool lowest) {
  auto wins = [&](double pa, long long ja, double pb, long long jb) {
    return lowest ? lower(pa, ja, pb, jb) : better(pa, ja, pb, jb);
  };
  __shared__ double sp[32];
  __shared__ long long sj[32];
  __shared__ long long pick[64];
  const long long n = (long long)*count;
  int got = 0;
  for (int r = 0; r < k; ++r) {
    double bp = -1.0;
    long long bj = -1;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
      const long long j = cand[i];
      if (j < 0) continue;
      if (bj < 0 || wins(P[j], j, bp, bj)) { bp = P[j]; bj = j; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double op = __shfl_down_sync(0xffffffffu, bp, o);
      const long long oj = __shfl_down_sync(0xffffffffu, bj, o);
      if (oj >= 0 && (bj < 0 || wins(op, oj, bp, bj))) { bp = op; bj = oj; }
    }
    if ((threadIdx.x & 31) == 0) { sp[threadIdx.x >> 5] = bp; sj[threadIdx.x >> 5] = bj; }
    __syncthreads();
    if (threadIdx.x < 32) {
      bp = threadIdx.x < (blockDim.x >> 5) ? sp[threadIdx.x] : -1.0;
      bj = threadIdx.x < (blockDim.x >> 5) ? sj[threadIdx.x] : -1;
      for (int o = 16; o > 0; o >>= 1) {
        const double op = __shfl_down_sync(0xffffffffu, bp, o);
        const long long oj = __shfl_down_sync(0xffffffffu, bj, o);
        if (oj >= 0 && (bj < 0 || wins(op, oj, bp, bj))) { bp = op; bj = oj; }
      }
      if (threadIdx.x == 0) sj[0] = bj;
    }
    __syncthreads();
    const long long win = sj[0];
    __syncthreads();
    if (win < 0) break;
    for (long long i = threadIdx.x; i < n; i += blockDim.x)
      if (cand[i] == win) cand[i] = -1;
    if (threadIdx.x == 0) pick[got] = win;
    ++got;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    for (int a = 1; a < got; ++a) {  // insertion sort by frequency
      long long v = pick[a];
      int b = a - 1;
      while (b >= 0 && pick[b] > v) { pick[b + 1] = pick[b]; --b; }
      pick[b + 1] = v;
    }
    for (int a = 0; a < got; ++a) chosen[a] = pick[a];
    *n_chosen = got;
  }
}

// |sum_t xw_t e^{-i omega t}|^2 over the block
__device__ double dtft_power(const double* __restrict__ xw, long long T, double omega, double* red) {
  const long long chunk = (T + blockDim.x - 1) / blockDim.x;
  const long long t0 = threadIdx.x * chunk, t1 = min(T, t0 + chunk);
  double re = 0.0, im = 0.0;
  if (t0 < t1) {
    double s, c, ds, dc;
    sincos(omega * (double)t0, &s, &c);
    sincos(omega, &ds, &dc);
    for (long long t = t0; t < t1; ++t) {
      re += xw[t] * c;
      im -= xw[t] * s;
      const double cn = c * dc - s * ds;
      s = s * dc + c * ds;
      c = cn;
    }
  }
  re = block_sum(re, red);
  im = block_sum(im, red);
  return re * re + im * im;
}

__global__ void refine_kernel(const double* __restrict__ xw, long long T, const double* __restrict__ P,
                              long long M, const long long* __restrict__ chosen,
                              const int* __restrict__ n_chosen, const double* __restrict__ stats,
                              double* freq, double* amp) {
  __shared__ double red[32];
  const int p = blockIdx.x;
  if (p >= *n_chosen) return;
  const long long j = chosen[p];
  const double la = log(P[j - 1]), lb = log(P[j]), lc = log(P[j + 1]);
  const double den = la - 2.0 * lb + lc;
  double delta = (den < 0.0) ? 0.5 * (la - lc) / den : 0.0;
  if (!isfinite(delta)) delta = 0.0;
  const double pi = 3.141592653589793238462643383279502884;
  const double om = 2.0 * pi * ((double)j + delta) / (double)M;
  const double halfw = 2.0 * pi / (double)M;
  double a = om - halfw, b = om + halfw;
  for (int it = 0; it < 40; ++it) {
    const double c = b - kGolden * (b - a);
    const double d = a + kGolden * (b - a);
    const double fc = dtft_power(xw, T, c, red);
    const double fd = dtft_power(xw, T, d, red);
    if (fc > fd) b = d; else a = c;
  }
  const double w = 0.5 * (a + b);
  const double pw = dtft_power(xw, T, w, red);
  if (threadIdx.x == 0) {
    freq[p] = w;
    amp[p] = 2.0 * sqrt(pw) / stats[1];
  }
}

// Workspace of one estimate, carved from one block of device memory sized for series of up to
// T samples and transforms of up to M points: stats(4) | a(M) | b(M) | xw(T) | P(M/2+1) |
// cand(M/4+1) | count | chosen(64) | n_chosen | freq(64) | amp(64).
struct Workspace {
  double* stats;
  double2 *A, *B;
  double* xw;
  double* P;
  long long* cand;
  unsigned long long* count;
  long long* chosen;
  int* n_chosen;
  double *freq, *amp;
};

constexpr size_t round16(size_t n) { return (n + 15) / 16 * 16; }

constexpr size_t workspace_bytes(size_t M, size_t T) {
  return round16(4 * 8) + 2 * round16(M * 16) + round16(T * 8) + round16((M / 2 + 1) * 8) +
         round16((M / 4 + 1) * 8) + round16(8) + round16(64 * 8) + round16(8) + round16(64 * 8) +
         round16(64 * 8);
}

Workspace carve(unsigned char* base, size_t M, size_t T) {
  unsigned char* p = base;
  auto take = [&](size_t n) { unsigned char* q = p; p += round16(n); return q; };
  Workspace w;
  w.stats = (double*)take(4 * 8);
  w.A = (double2*)take(M * 16);
  w.B = (double2*)take(M * 16);
  w.xw = (double*)take(T * 8);
  w.P = (double*)take((M / 2 + 1) * 8);
  w.cand = (long long*)take((M / 4 + 1) * 8);
  w.count = (unsigned long long*)take(8);
  w.chosen = (long long*)take(64 * 8);
  w.n_chosen = (int*)take(8);
  w.freq = (double*)take(64 * 8);
  w.amp = (double*)take(64 * 8);
  return w;
}

// The estimator's launches on stream s and the copy of its results to the host (synchronous).
// Every workspace value is written before it is read except the candidate counter, which is
// cleared here, so a workspace may hold anything from an earlier call.  *finite is false when
// the series' mean is not finite (a NaN or infinity in the series: an unstable run).
cudaError_t run_estimator(const Workspace& w, const double* d_x, int64_t T, int nser,
                          int32_t stride_series, int32_t k, bool lowest, double rel_power,
                          cudaStream_t s, double* h_freq, double* h_amp, int32_t* h_n,
                          bool* finite) {
  long long M = 1;
  while (M < 4 * T) M <<= 1;
  // a launch error left behind by an unrelated earlier runtime call on this thread would
  // otherwise be read back below as this call's failure
  (void)cudaGetLastError();
  cudaError_t e = cudaMemsetAsync(w.count, 0, 8, s);
  const int blocks = 152 * 4;
  if (e == cudaSuccess) {
    stats_kernel<<<1, 1024, 0, s>>>(d_x, T, nser, stride_series, w.stats);
    window_kernel<<<blocks, 256, 0, s>>>(d_x, T, nser, stride_series, w.stats, M, w.A, w.xw);
    double2 *in = w.A, *out = w.B;
    for (long long ns = 1; ns < M; ns <<= 1) {
      stockham_kernel<<<blocks, 256, 0, s>>>(in, out, M, ns);
      std::swap(in, out);
    }
    power_kernel<<<blocks, 256, 0, s>>>(in, M, w.P);
    max_kernel<<<1, 1024, 0, s>>>(w.P, M, w.stats);
    candidates_kernel<<<blocks, 256, 0, s>>>(w.P, M, w.stats, rel_power, w.cand, w.count);
    select_kernel<<<1, 1024, 0, s>>>(w.P, w.cand, w.count, k, w.chosen, w.n_chosen, lowest);
    refine_kernel<<<k, kThreads, 0, s>>>(w.xw, T, w.P, M, w.chosen, w.n_chosen, w.stats, w.freq, w.amp);
    e = cudaGetLastError();
  }
  int nfound = 0;
  double mean = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&nfound, w.n_chosen, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&mean, w.stats, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  *finite = std::isfinite(mean);
  if (!*finite) nfound = 0;
  if (e == cudaSuccess && nfound > 0) {
    e = cudaMemcpyAsync(h_freq, w.freq, sizeof(double) * nfound, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_amp, w.amp, sizeof(double) * nfound, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (e == cudaSuccess) *h_n = nfound;
  return e;
}

}  // namespace

lbw_status spectrum_device(const double* d_x, int64_t T, int32_t n_series, int32_t stride_series,
                           bool sum_all, int32_t k, cudaStream_t s, double* h_freq,
                           double* h_amp, int32_t* h_n, bool lowest, double rel_power) {
  long long M = 1;
  while (M < 4 * T) M <<= 1;
  unsigned char* base = nullptr;
  LBW_CUDA(cudaMallocAsync((void**)&base, workspace_bytes((size_t)M, (size_t)T), s));
  const Workspace w = carve(base, (size_t)M, (size_t)T);
  int32_t nfound = 0;
  bool finite = true;
  const cudaError_t e = run_estimator(w, d_x, T, sum_all ? n_series : 1, stride_series, k, lowest,
                                      rel_power, s, h_freq, h_amp, &nfound, &finite);
  cudaFreeAsync(base, s);
  if (e != cudaSuccess) return cuda_fail(e, "spectrum");
  if (!finite) return fail(LBW_EUNSTABLE, "spectrum: the series holds a non-finite value (unstable run)");
  *h_n = nfound;
  return LBW_OK;
}

}  // namespace lbw

// ---------------------------------------------------------------- no-allocation variant -----
//
// lbw_spectrum_series_static: the estimator above on a caller-owned device series, with all of
// its workspace in one file-scope device array instead of stream-ordered allocations, for
// callers that must not allocate device memory.  The array is sized for series of up to
// kStaticMaxT samples and is held by every GPU that loads the library until the process exits.

namespace lbw {
namespace {
constexpr int64_t kStaticMaxT = 16384;
constexpr size_t kStaticMaxM = 4 * (size_t)kStaticMaxT;  // a power of two: M of the largest T
}  // namespace
}  // namespace lbw

// The workspace.  In host code this name is only a host-side handle: its device address comes
// from cudaGetSymbolAddress, looked up once per device context (static_workspace below).
static __device__ __align__(256) unsigned char
    g_spectrum_scratch[lbw::workspace_bytes(lbw::kStaticMaxM, lbw::kStaticMaxT)];

namespace {

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// Unique ID of the calling thread's current context (0 when there is none or the driver does
// not say).  IDs are never reused within a process, so a context created after a device reset
// never matches an ID cached before it.
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(fn);
    fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(fn);
    (void)cudaGetLastError();
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

struct StaticAddr {
  unsigned long long ctx_id = 0;
  void* ptr = nullptr;
};
std::mutex g_static_mu;
StaticAddr g_static_addr[256];

// Device address of the workspace on the current device.  Set-up, with that device current:
// cudaGetSymbolAddress, once per device context; the address is cached under the context's ID
// and looked up again when the device's context has changed (after cudaDeviceReset).
cudaError_t static_workspace(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_static_mu);
  StaticAddr& a = g_static_addr[dev];
  const unsigned long long id = current_context_id();
  if (id == 0 || a.ptr == nullptr || a.ctx_id != id) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_spectrum_scratch);
    if (e != cudaSuccess) return e;
    a.ptr = ptr;
    a.ctx_id = current_context_id();  // the look-up makes the device's primary context current
  }
  *out = static_cast<unsigned char*>(a.ptr);
  return cudaSuccess;
}

}  // namespace

extern "C" lbw_status lbw_spectrum_series_static(const double* dev_x, int64_t T, int32_t k,
                                                 void* stream, double* host_freq, double* host_amp,
                                                 int32_t* host_n_found) {
  using namespace lbw;
  if (!dev_x || !host_freq || !host_amp || !host_n_found) return fail(LBW_EINVAL, "NULL argument");
  if (T < 4 || T > kStaticMaxT)
    return fail(LBW_EINVAL, "lbw_spectrum_series_static: T must be in [4, " + std::to_string(kStaticMaxT) +
                                "] (the fixed workspace holds " + std::to_string(kStaticMaxT) + " samples)");
  if (k < 1 || k > 64) return fail(LBW_EINVAL, "1 <= k <= 64");
  int dev = 0;
  LBW_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return fail(LBW_EINVAL, "device ordinal out of range");
  unsigned char* base = nullptr;
  cudaError_t e = static_workspace(dev, &base);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_spectrum_scratch)");
  const Workspace w = carve(base, kStaticMaxM, (size_t)kStaticMaxT);
  int32_t nfound = 0;
  bool finite = true;
  e = run_estimator(w, dev_x, T, 1, (int32_t)T, k, false, 1e-3,
                    reinterpret_cast<cudaStream_t>(stream), host_freq, host_amp, &nfound, &finite);
  if (e != cudaSuccess) return cuda_fail(e, "lbw_spectrum_series_static");
  if (!finite) return fail(LBW_EUNSTABLE, "spectrum: the series holds a non-finite value");
  *host_n_found = nfound;
  return LBW_OK;
}

