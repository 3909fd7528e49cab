// lbw_api.cu -- host side of the C ABI: descriptor validation, the FP64 geometry table,
// device memory, CUDA-graph step chains, probes and read-out.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "lbw_internal.h"

namespace lbw {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

lbw_status fail(lbw_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

lbw_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return LBW_ECUDA;
}

namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;
// Flat-space stability of the step: spectral radius 1 while
// sum_a (c^2 g_q^{aa} + cs^2) <= 4 (measured on the step operator); keep a margin.
constexpr double kStabilityLimit = 3.0;

// Metric of Sec. IV in lattice coordinates: x^a = x0^a + (q^a + 1/2) h^a, so
// g_q^{ab} = g^{ab} / (h_a h_b), sqrt(g_q) = h1 h2 h3 sqrt(g), G_q^a = G^a / h_a, with
// G^a = g^{bc} Gamma^a_{bc} = -(1/sqrt g) d_b (sqrt g g^{ab}).
struct Metric {
  double sg, g11, g22, g33, g13, G1, G3;
  bool ok;
};

Metric metric_at(const lbw_grid_desc& d, double q1, double q2, double q3) {
  (void)q2;
  const double r = d.x0[0] + (q1 + 0.5) * d.h[0];
  const double w = d.x0[2] + (q3 + 0.5) * d.h[2];
  Metric m{};
  m.ok = true;
  double sg = 1, g11 = 1, g22 = 1, g33 = 1, g13 = 0, G1 = 0, G3 = 0;
  switch (d.kind) {
    case LBW_CARTESIAN: break;
    case LBW_POLAR:
    case LBW_CYLINDRICAL:  // Eqs. MetricCylindrical, CylindricalChr
      if (!(r > 0)) m.ok = false;
      sg = r; g22 = 1.0 / (r * r); G1 = -1.0 / r;
      break;
    case LBW_TRUMPET: {  // Eqs. coordinatesTrumpet, MetricTrumpet with a general flare s(z)
      double s, ds, dds;
      if (d.horn_profile == 0) {
        const double Z = d.geom[0] - w, lam = d.geom[1];
        if (!(Z > 0)) m.ok = false;
        s = std::pow(Z, -lam);
        ds = lam * s / Z;
        dds = lam * (lam + 1.0) * s / (Z * Z);
      } else {
        const double a0 = d.geom[0], b = d.geom[1], al = d.geom[2], e = std::exp(al * w);
        s = (a0 + b * e) / (a0 + b);
        ds = b * al * e / (a0 + b);
        dds = al * ds;
      }
      if (!(r > 0) || !(s > 0)) m.ok = false;
      sg = r * s * s;
      g11 = (1.0 + r * r * ds * ds) / (s * s);
      g13 = -r * ds / s;
      g22 = 1.0 / (r * r * s * s);
      G1 = (r * r * s * dds - 2.0 * r * r * ds * ds - 1.0) / (r * s * s);
      break;
    }
    default: {  // torus, Eqs. CoordinatesTorus, AMetricTorus, AChristoffelTorus
      const double R = d.geom[0], cp = std::cos(w), Rr = R + r * cp;
      if (!(r > 0) || !(Rr > 0)) m.ok = false;
      sg = r * Rr;
      g22 = 1.0 / (Rr * Rr);
      g33 = 1.0 / (r * r);
      G1 = -(R + 2.0 * r * cp) / (r * Rr);
      G3 = std::sin(w) / (r * Rr);
    }
  }
  const double *h = d.h;
  m.sg = sg * h[0] * h[1] * h[2];
  m.g11 = g11 / (h[0] * h[0]);
  m.g22 = g22 / (h[1] * h[1]);
  m.g33 = g33 / (h[2] * h[2]);
  m.g13 = g13 / (h[0] * h[2]);
  m.G1 = G1 / h[0];
  m.G3 = G3 / h[2];
  return m;
}

bool is_angle(const lbw_grid_desc& d, int axis) {
  if (d.kind == LBW_CARTESIAN) return false;
  if (axis == 1) return true;
  return axis == 2 && d.kind == LBW_TOROIDAL;
}

lbw_status validate(lbw_grid_desc& d) {
  if (d.kind < 0 || d.kind > 4) return fail(LBW_EINVAL, "kind must be a lbw_metric value");
  if (d.tau != 0.5)
    return fail(LBW_EINVAL, "tau must be 0.5: the scheme is derived for tau = 1/2 only");
  for (int a = 0; a < 3; ++a)
    if (d.n[a] < 1 || d.n[a] > (1 << 20)) return fail(LBW_EINVAL, "n[a] must be in [1, 2^20]");
  if ((long long)d.n[0] * d.n[1] * d.n[2] > (1LL << 34))
    return fail(LBW_EINVAL, "lattice larger than 2^34 nodes");
  if (d.kind == LBW_POLAR && d.n[2] != 1) return fail(LBW_EINVAL, "polar grids need n[2] == 1");
  if (!(d.cs2 > 0.0 && d.cs2 < 1.0 / 3.0)) return fail(LBW_EINVAL, "cs2 must be in (0, 1/3)");
  if (!(d.c > 0.0)) return fail(LBW_EINVAL, "c must be > 0");
  if (!(d.damping > 0.0 && d.damping <= 1.0)) return fail(LBW_EINVAL, "damping must be in (0, 1]");
  if (d.prec < 0 || d.prec > 3) return fail(LBW_EINVAL, "prec must be a lbw_prec value");
  if (d.geom_mode < LBW_GEOM_AUTO || d.geom_mode > LBW_GEOM_ANALYTIC)
    return fail(LBW_EINVAL, "geom_mode must be a lbw_geom_mode value");
  if (d.reserved != 0) return fail(LBW_EINVAL, "reserved must be 0");
  if (d.geom_mode == LBW_GEOM_ANALYTIC && d.prec != LBW_F64 && d.prec != LBW_F32)
    return fail(LBW_EINVAL, "geom_mode ANALYTIC is built for FP32 and FP64 storage");
  if (d.equilibrium < LBW_EQ_CURVILINEAR || d.equilibrium > LBW_EQ_HERMITE)
    return fail(LBW_EINVAL, "equilibrium must be a lbw_equilibrium value");
  if (d.equilibrium != LBW_EQ_CURVILINEAR &&
      (d.kind != LBW_CARTESIAN || (d.prec != LBW_F64 && d.prec != LBW_F32) || d.geom_mode == LBW_GEOM_ANALYTIC))
    return fail(LBW_EINVAL, "the moment-matching and Hermite equilibria are the Cartesian schemes of Sec. II: "
                            "kind CARTESIAN, FP32 or FP64 storage, table geometry");
  if (d.equilibrium != LBW_EQ_CURVILINEAR) {
    double E, two0;
    equilibrium_coefs(d, &E, &two0);
    if (!(E > 0.0 && E <= 1.0 / 3.0))
      return fail(LBW_EINVAL, "equilibrium: the rest population's weight 1 - 3 E must stay in [0, 1) "
                              "(E = c^2 for moment matching, the Hermite form's stress coefficient otherwise)");
  }
  if (d.kind == LBW_TRUMPET && d.horn_profile != 0 && d.horn_profile != 1)
    return fail(LBW_EINVAL, "horn_profile must be 0 (Bessel) or 1 (exponential)");
  for (int k = 0; k < 6; ++k)
    if (d.bc[k] < 0 || d.bc[k] > 3) return fail(LBW_EINVAL, "bc must be lbw_bc values");
  for (int a = 0; a < 3; ++a) {
    const bool p0 = d.bc[2 * a] == LBW_BC_PERIODIC, p1 = d.bc[2 * a + 1] == LBW_BC_PERIODIC;
    if (p0 != p1) return fail(LBW_EINVAL, "periodic faces come in pairs");
    if (is_angle(d, a)) {
      if (!p0) return fail(LBW_EINVAL, "angular axes must be periodic");
      if (d.h[a] == 0.0) d.h[a] = kTwoPi / d.n[a];
      if (std::fabs(d.h[a] * d.n[a] - kTwoPi) > 1e-9)
        return fail(LBW_EINVAL, "an angular axis must span 2 pi: h = 2 pi / n");
    }
    if (!(d.h[a] > 0.0)) return fail(LBW_EINVAL, "h must be > 0");
  }
  if (d.kind == LBW_POLAR && d.bc[4] != LBW_BC_PERIODIC)
    return fail(LBW_EINVAL, "polar grids need periodic q3 faces");
  if (d.kind == LBW_TOROIDAL && !(d.geom[0] > 0)) return fail(LBW_EINVAL, "torus needs R > 0");
  if (d.kind == LBW_TRUMPET && d.horn_profile == 1 && !(d.geom[0] + d.geom[1] > 0))
    return fail(LBW_EINVAL, "exponential horn needs a0 + b > 0");
  return LBW_OK;
}

// Coefficient table of the forcing term (see TableSlot).  Ghost rule at a non-periodic face:
// free -> rho copied; bounce-back (rigid) -> P mirrored; anti-bounce-back (Dirichlet) -> P
// mirrored with opposite sign; the ghost's metric is taken at the ghost position.
lbw_status build_table(const lbw_grid_desc& d, std::vector<double>& tab) {
  const int n1 = d.n[0], n3 = d.n[2];
  const double c2 = d.c * d.c, cs2 = d.cs2;
  tab.assign((size_t)n1 * n3 * T_SLOTS, 0.0);
  double worst = 0.0;
  for (int q3 = 0; q3 < n3; ++q3)
    for (int q1 = 0; q1 < n1; ++q1) {
      double* e = &tab[((size_t)q3 * n1 + q1) * T_SLOTS];
      const Metric m = metric_at(d, q1, 0, q3);
      if (!m.ok) return fail(LBW_EINVAL, "metric undefined on the lattice (r, s or R + r cos phi <= 0)");
      worst = std::max(worst, c2 * (m.g11 + m.g22 + m.g33) + 3.0 * cs2);
      e[T_SG] = m.sg;
      e[T_INVSG] = 1.0 / m.sg;
      if (d.equilibrium != LBW_EQ_CURVILINEAR) continue;  // the Cartesian schemes have no force
      e[T_H22] = 0.5 * (c2 * m.g22 - cs2);
      e[T_MG1] = -c2 * m.G1;
      e[T_MG3] = -c2 * m.G3;
      // neighbours along q1 (axis 0) and q3 (axis 2)
      for (int axis = 0; axis < 3; axis += 2)
        for (int s = -1; s <= 1; s += 2) {
          int p1 = q1 + (axis == 0 ? s : 0), p3 = q3 + (axis == 2 ? s : 0);
          const int n = d.n[axis], pos = axis == 0 ? p1 : p3;
          const int face = 2 * axis + (s > 0 ? 1 : 0);
          double K11 = 0, K13 = 0, K33 = 0, self = 1.0;
          bool ghost = false;
          if (pos < 0 || pos >= n) {
            if (d.bc[face] == LBW_BC_PERIODIC) {
              if (axis == 0) p1 = (p1 + n) % n; else p3 = (p3 + n) % n;
            } else {
              ghost = true;
            }
          }
          const Metric mn = metric_at(d, p1, 0, p3);
          if (!mn.ok) return fail(LBW_EINVAL, "metric undefined at a ghost node (move r_in or Zmax)");
          K11 = c2 * mn.g11 - cs2;
          K13 = c2 * mn.g13;
          K33 = c2 * mn.g33 - cs2;
          if (ghost) {
            if (d.bc[face] == LBW_BC_FREE) self = 1.0;
            else self = (d.bc[face] == LBW_BC_BOUNCE ? 1.0 : -1.0) * mn.sg / m.sg;
          }
          // D1 gets +-(1/2) K^{1b} rho(x +- e_b); D3 gets +-(1/2) K^{3b} rho(x +- e_b)
          const double k1 = axis == 0 ? K11 : K13;   // K^{1b}
          const double k3 = axis == 0 ? K13 : K33;   // K^{3b}
          if (ghost) {
            e[T_S1] += 0.5 * s * k1 * self;
            e[T_S3] += 0.5 * s * k3 * self;
          } else if (axis == 0) {
            e[s > 0 ? T_A1P : T_A1M] = 0.5 * k1;
            e[s > 0 ? T_B13P : T_B13M] = 0.5 * k3;
          } else {
            e[s > 0 ? T_C13P : T_C13M] = 0.5 * k1;
            e[s > 0 ? T_C33P : T_C33M] = 0.5 * k3;
          }
        }
    }
  if (worst > kStabilityLimit)
    return fail(LBW_EINVAL, "lattice too coarse for c: max c^2 (g^11 + g^22 + g^33) + 3 cs^2 = " +
                                std::to_string(worst) + " > 3 (raise r_in or lower c)");
  return LBW_OK;
}

}  // namespace

lbw_status validate_desc(lbw_grid_desc& d) { return validate(d); }
lbw_status build_force_table(const lbw_grid_desc& d, std::vector<double>& tab) { return build_table(d, tab); }

double lattice_sqrtg(const lbw_grid_desc& d, int q1, int q3) { return metric_at(d, q1, 0, q3).sg; }

namespace {

size_t elem_size(int prec) { return prec == LBW_F64 ? 8 : prec == LBW_F32 ? 4 : 2; }
size_t real_size(int prec) { return prec == LBW_F64 ? 8 : 4; }

void drop_graphs(Grid* g) {
  for (int k = 0; k < 2; ++k)
    if (g->graph[k]) {
      cudaGraphExecDestroy(g->graph[k]);
      g->graph[k] = nullptr;
    }
  g->graph_len = 0;
}

// Harmonic sources on the state just written to buffer `buf` (no-op without sources).
cudaError_t apply_sources(Grid* g, int buf) {
  if (g->nsrc == 0) return cudaSuccess;
  return launch_sources(g->d.prec, g->f[buf], static_cast<const SourceEntry*>(g->src), g->nsrc,
                        g->src_kind, g->src_amp, g->counters, g->stream);
}

// A chain of `len` steps starting from buffer `start`, captured once and replayed.
lbw_status ensure_graph(Grid* g, int start, int len) {
  if (g->graph[start] && g->graph_len == len) return LBW_OK;
  if (g->graph_len != len) drop_graphs(g);
  cudaGraph_t graph;
  LBW_CUDA(cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
  int src = start;
  cudaError_t e = cudaSuccess;
  for (int s = 0; s < len && e == cudaSuccess; ++s) {
    e = launch_step(g, src);
    if (e == cudaSuccess) e = apply_sources(g, 1 - src);
    src = 1 - src;
  }
  cudaError_t e2 = cudaStreamEndCapture(g->stream, &graph);
  if (e != cudaSuccess) return cuda_fail(e, "step launch during capture");
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&g->graph[start], graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  g->graph_len = len;
  return LBW_OK;
}

// Samples recorded so far (counters[1]) and the wait flag (counters[3]): a step whose bounded
// wait for staged data ran out raises the flag and leaves the state undefined.
lbw_status read_counters(Grid* g, unsigned long long* recorded) {
  unsigned long long c[3] = {0, 0, 0};
  LBW_CUDA(cudaMemcpyAsync(c, g->counters + 1, sizeof(c), cudaMemcpyDeviceToHost, g->stream));
  LBW_CUDA(cudaStreamSynchronize(g->stream));
  if (recorded) *recorded = c[0];
  if (c[2]) return fail(LBW_ETIMEOUT, "a time step's bounded wait for staged data ran out; the state is "
                                      "undefined until lbw_init");
  return LBW_OK;
}

}  // namespace
}  // namespace lbw

using namespace lbw;

struct lbw_grid : Grid {};

extern "C" {

const char* lbw_last_error(void) { return g_last_error.c_str(); }

lbw_status lbw_create_grid(const lbw_grid_desc* desc, void* stream, lbw_grid** out) {
  if (!desc || !out) return fail(LBW_EINVAL, "desc and out must not be NULL");
  *out = nullptr;
  lbw_grid_desc d = *desc;
  lbw_status st = validate(d);
  if (st != LBW_OK) return st;
  std::vector<double> tab;
  st = build_table(d, tab);
  if (st != LBW_OK) return st;

  lbw_grid* g = new (std::nothrow) lbw_grid();
  if (!g) return fail(LBW_ENOMEM, "host allocation failed");
  g->d = d;
  g->stream = reinterpret_cast<cudaStream_t>(stream);
  if (!g->stream) {
    // the legacy default stream cannot be captured into a graph; a blocking stream created
    // here stays ordered with it (legacy-stream semantics)
    cudaError_t es = cudaStreamCreate(&g->stream);
    if (es != cudaSuccess) {
      delete g;
      return cuda_fail(es, "cudaStreamCreate");
    }
    g->own_stream = true;
  }
  g->nn = (int64_t)d.n[0] * d.n[1] * d.n[2];
  g->elem = elem_size(d.prec);
  g->w0 = 1.0 - 3.0 * d.cs2;
  g->w1 = 0.5 * d.cs2;
  auto cleanup = [&](lbw_status s) {
    lbw_destroy(g);
    return s;
  };
  const size_t fbytes = (size_t)7 * g->nn * g->elem;
  for (int k = 0; k < 2; ++k) {
    cudaError_t e = cudaMallocAsync(&g->f[k], fbytes, g->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cleanup(fail(LBW_ENOMEM, std::string("population buffers: ") + cudaGetErrorString(e)));
    }
  }
  const size_t rs = real_size(d.prec);
  const size_t tbytes = tab.size() * rs;
  cudaError_t e = cudaMallocAsync(&g->table, tbytes, g->stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&g->counters, 5 * sizeof(unsigned long long), g->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cleanup(fail(LBW_ENOMEM, "table allocation failed"));
  }
  std::vector<float> tf;
  const void* src = tab.data();
  if (rs == 4) {
    tf.assign(tab.begin(), tab.end());
    src = tf.data();
  }
  e = cudaMemcpyAsync(g->table, src, tbytes, cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->counters, 0, 5 * sizeof(unsigned long long), g->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->f[0], 0, fbytes, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "create: upload"));
  step_launch_shape(g);
  if (d.geom_mode == LBW_GEOM_ANALYTIC && g->tma_by == 0)
    return cleanup(fail(LBW_EINVAL, "geom_mode ANALYTIC needs the tile kernel: q2 extent a multiple of "
                                    "the tile width (64, or 128 for 16-bit storage) and non-periodic q1"));
  *out = g;
  return LBW_OK;
}

void lbw_destroy(lbw_grid* g) {
  if (!g) return;
  drop_graphs(g);
  for (int k = 0; k < 2; ++k)
    if (g->f[k]) cudaFreeAsync(g->f[k], g->stream);
  if (g->table) cudaFreeAsync(g->table, g->stream);
  if (g->counters) cudaFreeAsync(g->counters, g->stream);
  if (g->probe_q) cudaFreeAsync(g->probe_q, g->stream);
  if (g->series) cudaFreeAsync(g->series, g->stream);
  if (g->src) cudaFreeAsync(g->src, g->stream);
  cudaStreamSynchronize(g->stream);
  if (g->own_stream) cudaStreamDestroy(g->stream);
  delete g;
}

lbw_status lbw_init(lbw_grid* g, const lbw_pulse* host_pulses, int32_t n_pulses) {
  if (!g) return fail(LBW_EINVAL, "grid is NULL");
  if (n_pulses < 0 || n_pulses > (1 << 20)) return fail(LBW_EINVAL, "n_pulses out of range");
  if (n_pulses > 0 && !host_pulses) return fail(LBW_EINVAL, "host_pulses is NULL");
  for (int k = 0; k < n_pulses; ++k)
    if (!(host_pulses[k].sigma > 0)) return fail(LBW_EINVAL, "pulse sigma must be > 0");
  double* d_p = nullptr;
  const size_t pb = sizeof(double) * 5 * std::max(1, n_pulses);
  LBW_CUDA(cudaMallocAsync(&d_p, pb, g->stream));
  std::vector<double> hp(5 * std::max(1, n_pulses), 0.0);
  for (int k = 0; k < n_pulses; ++k) {
    hp[5 * k] = host_pulses[k].x[0];
    hp[5 * k + 1] = host_pulses[k].x[1];
    hp[5 * k + 2] = host_pulses[k].x[2];
    hp[5 * k + 3] = host_pulses[k].sigma;
    hp[5 * k + 4] = host_pulses[k].amp;
  }
  cudaError_t e = cudaMemcpyAsync(d_p, hp.data(), pb, cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess) e = launch_init(g, d_p, n_pulses);
  cudaFreeAsync(d_p, g->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->counters, 0, 5 * sizeof(unsigned long long), g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) return cuda_fail(e, "init");
  g->steps = 0;
  g->initialised = true;
  return LBW_OK;
}

lbw_status lbw_step(lbw_grid* g, int64_t n_steps) {
  if (!g) return fail(LBW_EINVAL, "grid is NULL");
  if (!g->initialised) return fail(LBW_ESTATE, "lbw_step before lbw_init");
  if (n_steps < 0) return fail(LBW_EINVAL, "n_steps must be >= 0");
  const int chain = 64;
  int64_t left = n_steps;
  if (left >= chain) {
    for (int start = 0; start < 2; ++start) {
      lbw_status st = ensure_graph(g, start, chain);
      if (st != LBW_OK) return st;
    }
    while (left >= chain) {
      LBW_CUDA(cudaGraphLaunch(g->graph[g->cur], g->stream));
      // an even chain ends on the buffer it started from
      left -= chain;
    }
  }
  while (left > 0) {
    LBW_CUDA(launch_step(g, g->cur));
    LBW_CUDA(apply_sources(g, 1 - g->cur));
    g->cur = 1 - g->cur;
    --left;
  }
  g->steps += n_steps;
  return LBW_OK;
}

lbw_status lbw_inject_wait_timeout(lbw_grid* g) {
  if (!g) return fail(LBW_EINVAL, "grid is NULL");
  if (!g->initialised) return fail(LBW_ESTATE, "lbw_inject_wait_timeout before lbw_init");
  if (g->tma_by == 0)
    return fail(LBW_EINVAL, "this lattice runs the register-pipelined step kernel, which has no device waits");
  // any non-zero value requests the injected timeout; lbw_init clears it
  LBW_CUDA(cudaMemsetAsync(g->counters + 4, 0xff, sizeof(unsigned long long), g->stream));
  LBW_CUDA(cudaStreamSynchronize(g->stream));
  return LBW_OK;
}

lbw_status lbw_step_count(lbw_grid* g, int64_t* out) {
  if (!g || !out) return fail(LBW_EINVAL, "NULL argument");
  *out = g->steps;
  return LBW_OK;
}

lbw_status lbw_source(lbw_grid* g, const int32_t* host_q, int32_t n, int32_t kind, double amp,
                      double omega) {
  if (!g) return fail(LBW_EINVAL, "grid is NULL");
  if (n < 0 || n > (1 << 24)) return fail(LBW_EINVAL, "0 <= n <= 2^24 source nodes");
  if (n > 0 && !host_q) return fail(LBW_EINVAL, "host_q is NULL");
  if (kind != 0 && kind != 1) return fail(LBW_EINVAL, "kind must be 0 (P) or 1 (J'_z)");
  if (!std::isfinite(amp) || !std::isfinite(omega)) return fail(LBW_EINVAL, "amp and omega must be finite");
  std::vector<SourceEntry> h((size_t)std::max(n, 0));
  for (int k = 0; k < n; ++k) {
    const int q1 = host_q[3 * k], q2 = host_q[3 * k + 1], q3 = host_q[3 * k + 2];
    if (q1 < 0 || q1 >= g->d.n[0] || q2 < 0 || q2 >= g->d.n[1] || q3 < 0 || q3 >= g->d.n[2])
      return fail(LBW_EINVAL, "source node outside the lattice");
    h[k].off = ((long long)q3 * g->d.n[0] + q1) * g->d.n[1] + q2;
    h[k].ps = g->nn;
    h[k].ghost = 0;
    h[k].pad = 0;
    h[k].sg = lattice_sqrtg(g->d, q1, q3);
    h[k].omega = omega;
    double eq_two0;
    equilibrium_coefs(g->d, &h[k].cs2, &eq_two0);  // the equilibrium the source imposes
  }
  drop_graphs(g);  // captured chains carry the source list
  if (g->src) { cudaFreeAsync(g->src, g->stream); g->src = nullptr; }
  g->nsrc = 0;
  if (n > 0) {
    LBW_CUDA(cudaMallocAsync(&g->src, sizeof(SourceEntry) * n, g->stream));
    LBW_CUDA(cudaMemcpyAsync(g->src, h.data(), sizeof(SourceEntry) * n, cudaMemcpyHostToDevice, g->stream));
    LBW_CUDA(cudaStreamSynchronize(g->stream));
    g->nsrc = n;
    g->src_kind = kind;
    g->src_amp = amp;
  }
  return LBW_OK;
}

lbw_status lbw_probe(lbw_grid* g, const int32_t* host_q, int32_t n, int64_t capacity) {
  if (!g) return fail(LBW_EINVAL, "grid is NULL");
  if (n < 0 || n > kMaxProbes) return fail(LBW_EINVAL, "0 <= n <= 64 probes");
  if (n > 0 && (!host_q || capacity < 1)) return fail(LBW_EINVAL, "probes need nodes and capacity >= 1");
  for (int k = 0; k < n; ++k)
    for (int a = 0; a < 3; ++a)
      if (host_q[3 * k + a] < 0 || host_q[3 * k + a] >= g->d.n[a])
        return fail(LBW_EINVAL, "probe node outside the lattice");
  if ((double)n * (double)capacity * 8.0 > 64e9) return fail(LBW_EINVAL, "probe series too large");
  if (g->probe_q) { cudaFreeAsync(g->probe_q, g->stream); g->probe_q = nullptr; }
  if (g->series) { cudaFreeAsync(g->series, g->stream); g->series = nullptr; }
  drop_graphs(g);  // the captured launches carry the probe pointers
  g->nprobe = 0;
  g->cap = 0;
  if (n > 0) {
    LBW_CUDA(cudaMallocAsync((void**)&g->probe_q, sizeof(int32_t) * 3 * n, g->stream));
    LBW_CUDA(cudaMallocAsync((void**)&g->series, sizeof(double) * n * capacity, g->stream));
    LBW_CUDA(cudaMemcpyAsync(g->probe_q, host_q, sizeof(int32_t) * 3 * n, cudaMemcpyHostToDevice,
                             g->stream));
    LBW_CUDA(cudaMemsetAsync(g->series, 0, sizeof(double) * n * capacity, g->stream));
    g->nprobe = n;
    g->cap = capacity;
  }
  // restart the sample counter (counters[1]); the step count is kept
  LBW_CUDA(cudaMemsetAsync(g->counters + 1, 0, sizeof(unsigned long long), g->stream));
  LBW_CUDA(cudaStreamSynchronize(g->stream));
  return LBW_OK;
}

lbw_status lbw_probe_read(lbw_grid* g, double* host_out, int64_t cap_per_probe, int64_t* n_steps) {
  if (!g || !n_steps) return fail(LBW_EINVAL, "NULL argument");
  unsigned long long rec = 0;
  lbw_status st = read_counters(g, &rec);
  if (st != LBW_OK) return st;
  *n_steps = (int64_t)rec;
  if (g->nprobe == 0) return LBW_OK;
  if (!host_out || cap_per_probe < (int64_t)rec)
    return fail(LBW_EINVAL, "host_out must hold n_probes x recorded samples");
  if (rec > 0)
    LBW_CUDA(cudaMemcpy2DAsync(host_out, sizeof(double) * cap_per_probe, g->series,
                               sizeof(double) * g->cap, sizeof(double) * rec, g->nprobe,
                               cudaMemcpyDeviceToHost, g->stream));
  LBW_CUDA(cudaStreamSynchronize(g->stream));
  for (int k = 0; k < g->nprobe; ++k)
    for (unsigned long long t = 0; t < rec; ++t)
      if (!std::isfinite(host_out[(size_t)k * cap_per_probe + t]))
        return fail(LBW_EUNSTABLE, "probe series holds a non-finite value (unstable run)");
  return LBW_OK;
}

lbw_status lbw_spectrum(lbw_grid* g, int32_t probe, int32_t k, double* host_freq, double* host_amp,
                        int32_t* n_found) {
  if (!g || !host_freq || !host_amp || !n_found) return fail(LBW_EINVAL, "NULL argument");
  if (probe < -1 || probe >= g->nprobe) return fail(LBW_EINVAL, "probe index out of range");
  if (k < 1 || k > 64) return fail(LBW_EINVAL, "1 <= k <= 64");
  unsigned long long rec = 0;
  lbw_status st = read_counters(g, &rec);
  if (st != LBW_OK) return st;
  if (rec < 4) return fail(LBW_ESTATE, "fewer than 4 recorded samples");
  const double* base = g->series + (probe >= 0 ? (size_t)probe * g->cap : 0);
  return spectrum_device(base, (int64_t)rec, probe >= 0 ? 1 : g->nprobe, (int32_t)g->cap,
                         probe < 0, k, g->stream, host_freq, host_amp, n_found);
}

lbw_status lbw_spectrum_lowest(lbw_grid* g, int32_t probe, int32_t k, double rel_power,
                               double* host_freq, double* host_amp, int32_t* n_found) {
  if (!g || !host_freq || !host_amp || !n_found) return fail(LBW_EINVAL, "NULL argument");
  if (probe < -1 || probe >= g->nprobe) return fail(LBW_EINVAL, "probe index out of range");
  if (k < 1 || k > 64) return fail(LBW_EINVAL, "1 <= k <= 64");
  if (!(rel_power > 0.0 && rel_power <= 1.0)) return fail(LBW_EINVAL, "0 < rel_power <= 1");
  unsigned long long rec = 0;
  lbw_status st = read_counters(g, &rec);
  if (st != LBW_OK) return st;
  if (rec < 4) return fail(LBW_ESTATE, "fewer than 4 recorded samples");
  const double* base = g->series + (probe >= 0 ? (size_t)probe * g->cap : 0);
  return spectrum_device(base, (int64_t)rec, probe >= 0 ? 1 : g->nprobe, (int32_t)g->cap,
                         probe < 0, k, g->stream, host_freq, host_amp, n_found, true, rel_power);
}

lbw_status lbw_spectrum_series(const double* host_x, int64_t T, int32_t n_series, int32_t k,
                               void* stream, double* host_freq, double* host_amp,
                               int32_t* host_n_found) {
  if (!host_x || !host_freq || !host_amp || !host_n_found) return fail(LBW_EINVAL, "NULL argument");
  if (T < 4 || T > (1LL << 26) || n_series < 1 || n_series > 1024)
    return fail(LBW_EINVAL, "need 4 <= T <= 2^26 and 1 <= n_series <= 1024");
  if (k < 1 || k > 64) return fail(LBW_EINVAL, "1 <= k <= 64");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  double* d_x = nullptr;
  LBW_CUDA(cudaMallocAsync(&d_x, sizeof(double) * T * n_series, s));
  cudaError_t e = cudaMemcpyAsync(d_x, host_x, sizeof(double) * T * n_series, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    cudaFreeAsync(d_x, s);
    return cuda_fail(e, "spectrum upload");
  }
  lbw_status st = LBW_OK;
  for (int j = 0; j < n_series && st == LBW_OK; ++j)
    st = spectrum_device(d_x + (size_t)j * T, T, 1, (int32_t)T, false, k, s, host_freq + (size_t)j * k,
                         host_amp + (size_t)j * k, host_n_found + j);
  cudaFreeAsync(d_x, s);
  cudaStreamSynchronize(s);
  return st;
}

lbw_status lbw_get_field(lbw_grid* g, double* host_P) {
  if (!g || !host_P) return fail(LBW_EINVAL, "NULL argument");
  double* d = nullptr;
  LBW_CUDA(cudaMallocAsync(&d, sizeof(double) * g->nn, g->stream));
  cudaError_t e = launch_field(g, d);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(host_P, d, sizeof(double) * g->nn, cudaMemcpyDeviceToHost, g->stream);
  cudaFreeAsync(d, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) return cuda_fail(e, "get_field");
  const lbw_status st = read_counters(g, nullptr);
  if (st != LBW_OK) return st;
  for (int64_t x = 0; x < g->nn; ++x)
    if (!std::isfinite(host_P[x])) return fail(LBW_EUNSTABLE, "field holds a non-finite value (unstable run)");
  return LBW_OK;
}

lbw_status lbw_get_populations(lbw_grid* g, double* host_f) {
  if (!g || !host_f) return fail(LBW_EINVAL, "NULL argument");
  double* d = nullptr;
  LBW_CUDA(cudaMallocAsync(&d, sizeof(double) * 7 * g->nn, g->stream));
  cudaError_t e = launch_to_double(g, d);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(host_f, d, sizeof(double) * 7 * g->nn, cudaMemcpyDeviceToHost, g->stream);
  cudaFreeAsync(d, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) return cuda_fail(e, "get_populations");
  return read_counters(g, nullptr);
}

lbw_status lbw_set_populations(lbw_grid* g, const double* host_f) {
  if (!g || !host_f) return fail(LBW_EINVAL, "NULL argument");
  double* d = nullptr;
  LBW_CUDA(cudaMallocAsync(&d, sizeof(double) * 7 * g->nn, g->stream));
  cudaError_t e = cudaMemcpyAsync(d, host_f, sizeof(double) * 7 * g->nn, cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess) e = launch_from_double(g, d);
  cudaFreeAsync(d, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) return cuda_fail(e, "set_populations");
  g->initialised = true;
  return LBW_OK;
}

}  // extern "C"
