// lbw_batch.cu -- an ensemble of lattices of uneven sizes advanced together.
//
// Every member is an independent lattice of the paper's scheme (its own geometry, sizes and
// probes).  All members' populations live in one pair of allocations; one time step of the
// whole ensemble is one launch of a persistent kernel whose CTAs walk a work list of
// (member, q2 tile, q1 tile, q3 segment) items and run the same register-pipelined tile march
// as the single-lattice kernel (lbw_march.cuh), so a member's numbers do not depend on the
// batching.  Steps are captured in CUDA-graph chains.  lbw_batch_tune times candidate tile
// shapes (rows per tile, planes per q3 segment, CTAs per SM) on the ensemble and keeps the
// fastest, optionally persisting it in a JSON-lines cache keyed by the ensemble's signature.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "lbw_internal.h"
#include "lbw_march.cuh"

namespace lbw {
namespace {

using namespace dev;

constexpr int kBatchBX = 32;  // q2 columns per tile (one warp per tile row)

template <typename S>
__global__ void __launch_bounds__(512) batch_step_kernel(const StepArgs<S>* __restrict__ members,
                                                         const int4* __restrict__ items, int n_items,
                                                         int lz, unsigned long long* counters,
                                                         int nprobe, long long cap) {
  using R = typename Store<S>::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) StepArgs<S> A;
  __shared__ int probe_list[kMaxProbes];
  __shared__ int probe_cnt;
  __shared__ unsigned long long t_sample;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nthr = blockDim.x * blockDim.y;
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int4 item = items[it];  // member, x0, y0, z0
    const unsigned* src = reinterpret_cast<const unsigned*>(members + item.x);
    unsigned* dst = reinterpret_cast<unsigned*>(&A);
    for (int k = tid; k < (int)(sizeof(StepArgs<S>) / 4); k += nthr) dst[k] = src[k];
    if (tid == 0) {
      probe_cnt = 0;
      t_sample = counters[1];
    }
    __syncthreads();
    const int z1 = min(item.w + lz, A.n3);
    scan_probes(A, item.y, item.z, item.w, z1, probe_list, &probe_cnt);
    march_tile(A, item.y, item.z, item.w, z1, reinterpret_cast<R*>(smem_raw), probe_list, probe_cnt,
               t_sample);
    __syncthreads();  // shared memory is reused by the next item
  }
  finish_step(counters, nprobe, cap, gridDim.x);
}

struct Shape {
  int by = 8;    // tile rows (CTA = 32 x by threads)
  int lz = 32;   // planes per q3 segment
  int cps = 2;   // CTAs per SM of the persistent grid
};

}  // namespace
}  // namespace lbw

using namespace lbw;

struct lbw_batch {
  int n = 0, prec = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<Grid> views;               // per member, pointing into the shared allocations
  std::vector<size_t> foff, toff;        // element offsets of each member's populations / table
  void* f[2] = {nullptr, nullptr};
  void* table = nullptr;
  unsigned long long* counters = nullptr;
  int32_t* probe_q = nullptr;
  double* series = nullptr;
  int nprobe = 0;
  int64_t cap = 0;
  void* members[2] = {nullptr, nullptr};  // StepArgs arrays for source buffer 0 / 1
  int4* items = nullptr;
  int n_items = 0, blocks = 0;
  Shape shape;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int graph_len = 0, cur = 0;
  int64_t steps = 0;
  bool initialised = false;
  long long total_nodes = 0;
};

namespace {

size_t es_of(int prec) { return prec == LBW_F64 ? 8 : prec == LBW_F32 ? 4 : 2; }
size_t rs_of(int prec) { return prec == LBW_F64 ? 8 : 4; }

void drop_graphs(lbw_batch* b) {
  for (int k = 0; k < 2; ++k)
    if (b->graph[k]) {
      cudaGraphExecDestroy(b->graph[k]);
      b->graph[k] = nullptr;
    }
  b->graph_len = 0;
}

template <typename S>
void fill_args(lbw_batch* b, int m, int src, StepArgs<S>& a) {
  using R = typename Store<S>::R;
  const Grid& g = b->views[m];
  std::memset(&a, 0, sizeof(a));
  a.fin = reinterpret_cast<const S*>(g.f[src]);
  a.fout = reinterpret_cast<S*>(g.f[1 - src]);
  a.tab = reinterpret_cast<const R*>(g.table);
  a.n1 = g.d.n[0]; a.n2 = g.d.n[1]; a.n3 = g.d.n[2];
  a.lz = b->shape.lz;
  a.nn = g.nn;
  for (int k = 0; k < 6; ++k) a.bc[k] = g.d.bc[k];
  a.damping = (R)g.d.damping;
  a.cs2 = (R)g.d.cs2;
  a.two_w0 = (R)(2.0 * g.w0);
  for (int i = 0; i < 7; ++i) {
    const double w = i == 0 ? g.w0 : g.w1;
    a.w[i] = (R)w;
    a.inv_w[i] = (R)(1.0 / w);
  }
  a.s2lo = g.d.bc[2] == LBW_BC_ANTIBOUNCE ? R(-1) : R(1);
  a.s2hi = g.d.bc[3] == LBW_BC_ANTIBOUNCE ? R(-1) : R(1);
  a.nprobe = b->nprobe;
  a.probe_q = b->probe_q ? b->probe_q + (size_t)m * b->nprobe * 3 : nullptr;
  a.series = b->series ? b->series + (size_t)m * b->nprobe * b->cap : nullptr;
  a.cap = b->cap;
  a.counters = b->counters;
  a.nblocks = 0;
}

template <typename S>
lbw_status upload_args(lbw_batch* b) {
  std::vector<StepArgs<S>> host(b->n);
  for (int src = 0; src < 2; ++src) {
    for (int m = 0; m < b->n; ++m) fill_args<S>(b, m, src, host[m]);
    if (!b->members[src]) LBW_CUDA(cudaMallocAsync(&b->members[src], sizeof(StepArgs<S>) * b->n, b->stream));
    LBW_CUDA(cudaMemcpyAsync(b->members[src], host.data(), sizeof(StepArgs<S>) * b->n,
                             cudaMemcpyHostToDevice, b->stream));
  }
  return LBW_OK;
}

template <typename S>
int max_cps() {
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_step_kernel<S>, 512, 4096) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return std::max(1, per);
}

// work list for the current shape: items of each member in (q3 segment, q1 tile, q2 tile)
// order, so consecutive CTAs hold spatial neighbours
lbw_status build_items(lbw_batch* b) {
  std::vector<int4> items;
  for (int m = 0; m < b->n; ++m) {
    const lbw_grid_desc& d = b->views[m].d;
    for (int z0 = 0; z0 < d.n[2]; z0 += b->shape.lz)
      for (int y0 = 0; y0 < d.n[0]; y0 += b->shape.by)
        for (int x0 = 0; x0 < d.n[1]; x0 += kBatchBX) items.push_back(make_int4(m, x0, y0, z0));
  }
  if (b->items) cudaFreeAsync(b->items, b->stream);
  b->items = nullptr;
  LBW_CUDA(cudaMallocAsync((void**)&b->items, sizeof(int4) * items.size(), b->stream));
  LBW_CUDA(cudaMemcpyAsync(b->items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice,
                           b->stream));
  b->n_items = (int)items.size();
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  b->blocks = std::max(1, std::min(b->n_items, sms * b->shape.cps));
  drop_graphs(b);
  return LBW_OK;
}

lbw_status refresh(lbw_batch* b) {
  lbw_status st = build_items(b);
  if (st != LBW_OK) return st;
  switch (b->prec) {
    case LBW_F64: return upload_args<double>(b);
    case LBW_F32: return upload_args<float>(b);
    case LBW_F16S: return upload_args<__half>(b);
    default: return upload_args<__nv_bfloat16>(b);
  }
}

template <typename S>
cudaError_t launch_batch_t(lbw_batch* b, int src) {
  using R = typename Store<S>::R;
  const dim3 block(kBatchBX, b->shape.by);
  const size_t smem = 3 * (size_t)(kBatchBX + 2) * (b->shape.by + 2) * sizeof(R);
  batch_step_kernel<S><<<b->blocks, block, smem, b->stream>>>(
      reinterpret_cast<const StepArgs<S>*>(b->members[src]), b->items, b->n_items, b->shape.lz,
      b->counters, b->nprobe, b->cap);
  return cudaGetLastError();
}

cudaError_t launch_batch(lbw_batch* b, int src) {
  switch (b->prec) {
    case LBW_F64: return launch_batch_t<double>(b, src);
    case LBW_F32: return launch_batch_t<float>(b, src);
    case LBW_F16S: return launch_batch_t<__half>(b, src);
    default: return launch_batch_t<__nv_bfloat16>(b, src);
  }
}

lbw_status ensure_graph(lbw_batch* b, int start, int len) {
  if (b->graph[start] && b->graph_len == len) return LBW_OK;
  if (b->graph_len != len) drop_graphs(b);
  cudaGraph_t graph;
  LBW_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  int src = start;
  cudaError_t e = cudaSuccess;
  for (int s = 0; s < len && e == cudaSuccess; ++s) {
    e = launch_batch(b, src);
    src = 1 - src;
  }
  cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
  if (e != cudaSuccess) return cuda_fail(e, "batch launch during capture");
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&b->graph[start], graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  b->graph_len = len;
  return LBW_OK;
}

lbw_status advance(lbw_batch* b, int64_t n_steps) {
  const int chain = 64;
  int64_t left = n_steps;
  if (left >= chain) {
    for (int start = 0; start < 2; ++start) {
      lbw_status st = ensure_graph(b, start, chain);
      if (st != LBW_OK) return st;
    }
    while (left >= chain) {
      LBW_CUDA(cudaGraphLaunch(b->graph[b->cur], b->stream));
      left -= chain;
    }
  }
  while (left > 0) {
    LBW_CUDA(launch_batch(b, b->cur));
    b->cur = 1 - b->cur;
    --left;
  }
  b->steps += n_steps;
  return LBW_OK;
}

std::string signature(const lbw_batch* b) {
  unsigned long long h = 1469598103934665603ULL;  // FNV-1a over the members' sizes
  for (const Grid& g : b->views)
    for (int a = 0; a < 3; ++a) {
      h ^= (unsigned long long)g.d.n[a];
      h *= 1099511628211ULL;
    }
  std::ostringstream s;
  s << "n" << b->n << "-p" << b->prec << "-nodes" << b->total_nodes << "-h" << std::hex << h;
  return s.str();
}

}  // namespace

extern "C" {

lbw_status lbw_batch_create(const lbw_grid_desc* descs, int32_t n, void* stream, lbw_batch** out) {
  if (!descs || !out) return fail(LBW_EINVAL, "descs and out must not be NULL");
  *out = nullptr;
  if (n < 1 || n > 65536) return fail(LBW_EINVAL, "1 <= n <= 65536 members");
  lbw_batch* b = new (std::nothrow) lbw_batch();
  if (!b) return fail(LBW_ENOMEM, "host allocation failed");
  auto cleanup = [&](lbw_status s) {
    lbw_batch_destroy(b);
    return s;
  };
  b->n = n;
  b->prec = descs[0].prec;
  b->stream = reinterpret_cast<cudaStream_t>(stream);
  if (!b->stream) {
    cudaError_t es = cudaStreamCreate(&b->stream);
    if (es != cudaSuccess) {
      delete b;
      return cuda_fail(es, "cudaStreamCreate");
    }
    b->own_stream = true;
  }
  b->views.resize(n);
  b->foff.resize(n);
  b->toff.resize(n);
  std::vector<double> tab_all;
  size_t ftot = 0;
  for (int m = 0; m < n; ++m) {
    lbw_grid_desc d = descs[m];
    if (d.prec != b->prec) return cleanup(fail(LBW_EINVAL, "all members must share the storage precision"));
    lbw_status st = validate_desc(d);
    if (st != LBW_OK) return cleanup(fail(st, "member " + std::to_string(m) + ": " + lbw_last_error()));
    std::vector<double> tab;
    st = build_force_table(d, tab);
    if (st != LBW_OK) return cleanup(fail(st, "member " + std::to_string(m) + ": " + lbw_last_error()));
    Grid& g = b->views[m];
    g.d = d;
    g.stream = b->stream;
    g.nn = (int64_t)d.n[0] * d.n[1] * d.n[2];
    g.elem = es_of(d.prec);
    g.w0 = 1.0 - 3.0 * d.cs2;
    g.w1 = 0.5 * d.cs2;
    b->foff[m] = ftot;
    // 256-byte aligned member slices
    const size_t align = 256 / g.elem;
    ftot += (7 * (size_t)g.nn + align - 1) / align * align;
    b->toff[m] = tab_all.size();
    tab_all.insert(tab_all.end(), tab.begin(), tab.end());
    while (tab_all.size() % 64) tab_all.push_back(0.0);
    b->total_nodes += g.nn;
  }
  const size_t es = es_of(b->prec), rs = rs_of(b->prec);
  for (int k = 0; k < 2; ++k) {
    cudaError_t e = cudaMallocAsync(&b->f[k], ftot * es, b->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cleanup(fail(LBW_ENOMEM, std::string("ensemble populations: ") + cudaGetErrorString(e)));
    }
  }
  cudaError_t e = cudaMallocAsync(&b->table, tab_all.size() * rs, b->stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&b->counters, 4 * sizeof(unsigned long long), b->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cleanup(fail(LBW_ENOMEM, "ensemble tables"));
  }
  std::vector<float> tf;
  const void* src = tab_all.data();
  if (rs == 4) {
    tf.assign(tab_all.begin(), tab_all.end());
    src = tf.data();
  }
  e = cudaMemcpyAsync(b->table, src, tab_all.size() * rs, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->counters, 0, 4 * sizeof(unsigned long long), b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->f[0], 0, ftot * es, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->f[1], 0, ftot * es, b->stream);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "ensemble upload"));
  for (int m = 0; m < n; ++m) {
    Grid& g = b->views[m];
    g.f[0] = static_cast<unsigned char*>(b->f[0]) + b->foff[m] * es;
    g.f[1] = static_cast<unsigned char*>(b->f[1]) + b->foff[m] * es;
    g.table = static_cast<unsigned char*>(b->table) + b->toff[m] * rs;
    g.counters = b->counters;
  }
  b->shape.cps = std::min(2, b->prec == LBW_F32 ? max_cps<float>() : 2);
  lbw_status st = refresh(b);
  if (st != LBW_OK) return cleanup(st);
  LBW_CUDA(cudaStreamSynchronize(b->stream));
  *out = b;
  return LBW_OK;
}

void lbw_batch_destroy(lbw_batch* b) {
  if (!b) return;
  drop_graphs(b);
  for (int k = 0; k < 2; ++k) {
    if (b->f[k]) cudaFreeAsync(b->f[k], b->stream);
    if (b->members[k]) cudaFreeAsync(b->members[k], b->stream);
  }
  if (b->table) cudaFreeAsync(b->table, b->stream);
  if (b->counters) cudaFreeAsync(b->counters, b->stream);
  if (b->items) cudaFreeAsync(b->items, b->stream);
  if (b->probe_q) cudaFreeAsync(b->probe_q, b->stream);
  if (b->series) cudaFreeAsync(b->series, b->stream);
  cudaStreamSynchronize(b->stream);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
}

lbw_status lbw_batch_init(lbw_batch* b, const lbw_pulse* host_pulses, const int32_t* host_counts) {
  if (!b || !host_counts) return fail(LBW_EINVAL, "NULL argument");
  size_t total = 0;
  for (int m = 0; m < b->n; ++m) {
    if (host_counts[m] < 0) return fail(LBW_EINVAL, "negative pulse count");
    total += host_counts[m];
  }
  if (total > 0 && !host_pulses) return fail(LBW_EINVAL, "host_pulses is NULL");
  std::vector<double> hp(5 * std::max<size_t>(1, total), 0.0);
  for (size_t k = 0; k < total; ++k) {
    if (!(host_pulses[k].sigma > 0)) return fail(LBW_EINVAL, "pulse sigma must be > 0");
    hp[5 * k] = host_pulses[k].x[0];
    hp[5 * k + 1] = host_pulses[k].x[1];
    hp[5 * k + 2] = host_pulses[k].x[2];
    hp[5 * k + 3] = host_pulses[k].sigma;
    hp[5 * k + 4] = host_pulses[k].amp;
  }
  double* d_p = nullptr;
  LBW_CUDA(cudaMallocAsync(&d_p, hp.size() * sizeof(double), b->stream));
  cudaError_t e = cudaMemcpyAsync(d_p, hp.data(), hp.size() * sizeof(double), cudaMemcpyHostToDevice, b->stream);
  size_t off = 0;
  for (int m = 0; m < b->n && e == cudaSuccess; ++m) {
    b->views[m].cur = b->cur;
    e = launch_init(&b->views[m], d_p + 5 * off, host_counts[m]);
    off += host_counts[m];
  }
  cudaFreeAsync(d_p, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->counters, 0, 4 * sizeof(unsigned long long), b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch init");
  b->steps = 0;
  b->initialised = true;
  return LBW_OK;
}

lbw_status lbw_batch_probe(lbw_batch* b, const int32_t* host_q, int32_t per_member, int64_t capacity) {
  if (!b) return fail(LBW_EINVAL, "batch is NULL");
  if (per_member < 0 || per_member > kMaxProbes) return fail(LBW_EINVAL, "0 <= per_member <= 64");
  if (per_member > 0 && (!host_q || capacity < 1)) return fail(LBW_EINVAL, "probes need nodes and capacity");
  for (int m = 0; m < b->n; ++m)
    for (int k = 0; k < per_member; ++k)
      for (int a = 0; a < 3; ++a) {
        const int v = host_q[((size_t)m * per_member + k) * 3 + a];
        if (v < 0 || v >= b->views[m].d.n[a]) return fail(LBW_EINVAL, "probe node outside its member's lattice");
      }
  if ((double)b->n * per_member * capacity * 8.0 > 64e9) return fail(LBW_EINVAL, "probe series too large");
  if (b->probe_q) { cudaFreeAsync(b->probe_q, b->stream); b->probe_q = nullptr; }
  if (b->series) { cudaFreeAsync(b->series, b->stream); b->series = nullptr; }
  b->nprobe = 0;
  b->cap = 0;
  if (per_member > 0) {
    const size_t nq = (size_t)b->n * per_member;
    LBW_CUDA(cudaMallocAsync((void**)&b->probe_q, sizeof(int32_t) * 3 * nq, b->stream));
    LBW_CUDA(cudaMallocAsync((void**)&b->series, sizeof(double) * nq * capacity, b->stream));
    LBW_CUDA(cudaMemcpyAsync(b->probe_q, host_q, sizeof(int32_t) * 3 * nq, cudaMemcpyHostToDevice, b->stream));
    LBW_CUDA(cudaMemsetAsync(b->series, 0, sizeof(double) * nq * capacity, b->stream));
    b->nprobe = per_member;
    b->cap = capacity;
  }
  LBW_CUDA(cudaMemsetAsync(b->counters + 1, 0, sizeof(unsigned long long), b->stream));
  lbw_status st = refresh(b);
  if (st != LBW_OK) return st;
  LBW_CUDA(cudaStreamSynchronize(b->stream));
  return LBW_OK;
}

lbw_status lbw_batch_step(lbw_batch* b, int64_t n_steps) {
  if (!b) return fail(LBW_EINVAL, "batch is NULL");
  if (!b->initialised) return fail(LBW_ESTATE, "lbw_batch_step before lbw_batch_init");
  if (n_steps < 0) return fail(LBW_EINVAL, "n_steps must be >= 0");
  return advance(b, n_steps);
}

lbw_status lbw_batch_probe_read(lbw_batch* b, double* host_out, int64_t* n_steps) {
  if (!b || !n_steps) return fail(LBW_EINVAL, "NULL argument");
  unsigned long long rec = 0;
  LBW_CUDA(cudaMemcpyAsync(&rec, b->counters + 1, sizeof(rec), cudaMemcpyDeviceToHost, b->stream));
  LBW_CUDA(cudaStreamSynchronize(b->stream));
  *n_steps = (int64_t)rec;
  if (b->nprobe == 0 || rec == 0) return LBW_OK;
  if (!host_out) return fail(LBW_EINVAL, "host_out is NULL");
  LBW_CUDA(cudaMemcpyAsync(host_out, b->series, sizeof(double) * b->n * b->nprobe * b->cap,
                           cudaMemcpyDeviceToHost, b->stream));
  LBW_CUDA(cudaStreamSynchronize(b->stream));
  return LBW_OK;
}

lbw_status lbw_batch_spectrum(lbw_batch* b, int32_t k, double* host_freq, double* host_amp,
                              int32_t* host_n_found) {
  if (!b || !host_freq || !host_amp || !host_n_found) return fail(LBW_EINVAL, "NULL argument");
  if (k < 1 || k > 64) return fail(LBW_EINVAL, "1 <= k <= 64");
  if (b->nprobe == 0) return fail(LBW_ESTATE, "no probes registered");
  unsigned long long rec = 0;
  LBW_CUDA(cudaMemcpyAsync(&rec, b->counters + 1, sizeof(rec), cudaMemcpyDeviceToHost, b->stream));
  LBW_CUDA(cudaStreamSynchronize(b->stream));
  if (rec < 4) return fail(LBW_ESTATE, "fewer than 4 recorded samples");
  for (int m = 0; m < b->n; ++m) {
    lbw_status st = spectrum_device(b->series + (size_t)m * b->nprobe * b->cap, (int64_t)rec, b->nprobe,
                                    (int32_t)b->cap, true, k, b->stream, host_freq + (size_t)m * k,
                                    host_amp + (size_t)m * k, host_n_found + m);
    if (st != LBW_OK) return st;
  }
  return LBW_OK;
}

lbw_status lbw_batch_get_populations(lbw_batch* b, int32_t member, double* host_f) {
  if (!b || !host_f) return fail(LBW_EINVAL, "NULL argument");
  if (member < 0 || member >= b->n) return fail(LBW_EINVAL, "member out of range");
  Grid& g = b->views[member];
  g.cur = b->cur;
  double* d = nullptr;
  LBW_CUDA(cudaMallocAsync(&d, sizeof(double) * 7 * g.nn, b->stream));
  cudaError_t e = launch_to_double(&g, d);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(host_f, d, sizeof(double) * 7 * g.nn, cudaMemcpyDeviceToHost, b->stream);
  cudaFreeAsync(d, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch populations");
  return LBW_OK;
}

lbw_status lbw_batch_tune(lbw_batch* b, int32_t trial_steps, const char* cache_path, char* report,
                          int32_t report_cap) {
  if (!b) return fail(LBW_EINVAL, "batch is NULL");
  if (trial_steps < 1 || trial_steps > 1000) return fail(LBW_EINVAL, "1 <= trial_steps <= 1000");
  const std::string sig = signature(b);
  std::string line;
  bool cached = false;
  Shape best = b->shape;
  if (cache_path) {  // JSON lines: {"signature": "...", "by": 8, "lz": 32, "cps": 2, "ms": ...}
    std::ifstream in(cache_path);
    while (in && std::getline(in, line)) {
      if (line.find("\"" + sig + "\"") == std::string::npos) continue;
      Shape s;
      if (sscanf(line.c_str() + line.find("\"by\""), "\"by\": %d, \"lz\": %d, \"cps\": %d", &s.by, &s.lz,
                 &s.cps) == 3) {
        best = s;
        cached = true;
      }
    }
  }
  double best_ms = -1.0;
  std::ostringstream rep;
  if (!cached) {
    const int cps_max = b->prec == LBW_F32 ? max_cps<float>() : 2;
    const int bys[3] = {4, 8, 16}, lzs[3] = {16, 32, 64}, cpss[3] = {1, 2, 4};
    cudaEvent_t e0, e1;
    LBW_CUDA(cudaEventCreate(&e0));
    LBW_CUDA(cudaEventCreate(&e1));
    for (int by : bys)
      for (int lz : lzs)
        for (int cps : cpss) {
          if (cps > cps_max) continue;
          b->shape = Shape{by, lz, cps};
          lbw_status st = refresh(b);
          if (st != LBW_OK) return st;
          for (int w = 0; w < 2; ++w) {  // warm-up
            LBW_CUDA(launch_batch(b, b->cur));
            b->cur = 1 - b->cur;
          }
          LBW_CUDA(cudaEventRecord(e0, b->stream));
          for (int s = 0; s < trial_steps; ++s) {
            LBW_CUDA(launch_batch(b, b->cur));
            b->cur = 1 - b->cur;
          }
          LBW_CUDA(cudaEventRecord(e1, b->stream));
          LBW_CUDA(cudaEventSynchronize(e1));
          float ms = 0.f;
          LBW_CUDA(cudaEventElapsedTime(&ms, e0, e1));
          ms /= trial_steps;
          rep << "by=" << by << " lz=" << lz << " cps=" << cps << " ms=" << ms << "\n";
          if (best_ms < 0 || ms < best_ms) {
            best_ms = ms;
            best = b->shape;
          }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cache_path) {
      std::ofstream o(cache_path, std::ios::app);
      o << "{\"signature\": \"" << sig << "\", \"by\": " << best.by << ", \"lz\": " << best.lz
        << ", \"cps\": " << best.cps << ", \"ms\": " << best_ms << "}\n";
    }
  }
  b->shape = best;
  lbw_status st = refresh(b);
  if (st != LBW_OK) return st;
  // trial steps ran on the ensemble's buffers: callers tune before lbw_batch_init
  LBW_CUDA(cudaMemsetAsync(b->counters, 0, 4 * sizeof(unsigned long long), b->stream));
  LBW_CUDA(cudaStreamSynchronize(b->stream));
  rep << (cached ? "cached " : "chosen ") << "by=" << best.by << " lz=" << best.lz << " cps=" << best.cps
      << " signature=" << sig << "\n";
  if (report && report_cap > 0) {
    const std::string r = rep.str();
    std::strncpy(report, r.c_str(), (size_t)report_cap - 1);
    report[report_cap - 1] = '\0';
  }
  return LBW_OK;
}

lbw_status lbw_batch_info(lbw_batch* b, int64_t* total_nodes, int32_t* tile_rows, int32_t* seg_planes,
                          int32_t* ctas_per_sm) {
  if (!b) return fail(LBW_EINVAL, "batch is NULL");
  if (total_nodes) *total_nodes = b->total_nodes;
  if (tile_rows) *tile_rows = b->shape.by;
  if (seg_planes) *seg_planes = b->shape.lz;
  if (ctas_per_sm) *ctas_per_sm = b->shape.cps;
  return LBW_OK;
}

}  // extern "C"
