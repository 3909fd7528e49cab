// lbw_internal.h -- types shared by the translation units of liblbw (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "lbw.h"

namespace lbw {

// Per-(q1, q3) coefficients of the geometric forcing term, built on the host in FP64 from
// the metric in lattice coordinates (Sec. IV) and rounded to the arithmetic type R.
// With K^{ab} = c^2 g_q^{ab} - cs^2 delta^{ab} and rho the post-stream density, the
// divergence of A^{ab} = rho K^{ab} by central differences (Eq. DerivativeFromTaylor) is
//   D1 = A1p rho(q1+1) - A1m rho(q1-1) + C13p rho(q3+1) - C13m rho(q3-1) + S1 rho
//   D2 = H22 (rho(q2+1) - rho(q2-1))
//   D3 = B13p rho(q1+1) - B13m rho(q1-1) + C33p rho(q3+1) - C33m rho(q3-1) + S3 rho
// where every coefficient already holds the factor 1/2, and a non-periodic face's ghost
// (whose rho is a multiple of the node's own rho) is folded into S1 / S3 with the
// neighbour coefficient set to zero.  mG1, mG3 = -c^2 G_q^1, -c^2 G_q^3.
enum TableSlot {
  T_A1P = 0, T_A1M, T_B13P, T_B13M, T_C13P, T_C13M, T_C33P, T_C33M,
  T_S1, T_S3, T_H22, T_MG1, T_MG3, T_INVSG, T_SG, T_PAD, T_SLOTS
};

constexpr int kMaxProbes = 64;

struct Grid {
  lbw_grid_desc d;
  cudaStream_t stream = nullptr;
  bool own_stream = false;  // created here when the caller passed the legacy stream 0
  int64_t nn = 0;          // nodes
  size_t elem = 0;         // bytes per stored population value
  void* f[2] = {nullptr, nullptr};  // ping-pong population buffers, 7 planes each
  int cur = 0;             // which buffer holds the current post-collision state
  void* table = nullptr;   // n3 * n1 * T_SLOTS values of R (float or double)
  // probes
  int32_t nprobe = 0;
  int32_t* probe_q = nullptr;     // device, nprobe x 3
  double* series = nullptr;       // device, nprobe x cap
  int64_t cap = 0;
  // device counters: [0] steps since init, [1] samples recorded, [2] last-block ticket,
  // [3] timeout flag of a bounded wait, [4] injected-timeout request (tests)
  unsigned long long* counters = nullptr;
  int64_t steps = 0;       // host mirror of counters[0]
  bool initialised = false;
  // launch shape of the step kernel
  int bx = 0, by = 0, lz = 0;
  int tma_by = 0;          // 0: register-pipelined kernel; 4 or 7: TMA tile kernel rows
  int tma_npt = 2;         // TMA tile kernel: nodes per lane (tile width 32 x tma_npt)
  // padded storage (ensembles on the tile kernel): row length and first data column in
  // elements; pitch 0 means dense rows of n2 values
  int pitch = 0, col0 = 0;
  // harmonic sources: device SourceEntry array, applied after every step
  int32_t nsrc = 0;
  void* src = nullptr;
  int32_t src_kind = 0;
  double src_amp = 0.0;
  alignas(64) unsigned char tmaps[5 * 128];  // tensor maps: f[0] main/halo, f[1] main/halo, table
  dim3 grid_dim;
  // captured step chains, one per parity of the starting buffer
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int graph_len = 0;
  // 16-bit storage scale: stored value = f_i * inv_w[i]
  double w0 = 0, w1 = 0;
};

// error plumbing ---------------------------------------------------------------------------
void set_error(const std::string& msg);
lbw_status fail(lbw_status s, const std::string& msg);
lbw_status cuda_fail(cudaError_t e, const char* what);

#define LBW_CUDA(call)                                      \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return ::lbw::cuda_fail(e_, #call); \
  } while (0)

// descriptor validation (fills default angular spacings) and the FP64 force-coefficient table
lbw_status validate_desc(lbw_grid_desc& d);
lbw_status build_force_table(const lbw_grid_desc& d, std::vector<double>& tab);

// One harmonic source node: element offset of its population 0 from the buffer base, the
// population stride, the column shift of its ghost copy (0: none), sqrt(g) in lattice
// coordinates, the angular frequency (rad / step) and the lattice's cs^2.
struct SourceEntry {
  long long off, ps;
  int ghost, pad;
  double sg, omega, cs2;
};

// sqrt(g) of lattice node (q1, q3) of desc in lattice coordinates (FP64, as in the table)
double lattice_sqrtg(const lbw_grid_desc& d, int q1, int q3);

// Collision constants of the equilibrium: 2 f_i^eq = E rho + xi_i . j' (i >= 1, unscaled storage)
// and 2 f_0^eq = two0 rho.  The paper's method has E = cs^2 (two0 = 2 w0); the Cartesian
// schemes of Sec. II (lbw_equilibrium) change E and have no forcing term.
inline void equilibrium_coefs(const lbw_grid_desc& d, double* E, double* two0) {
  const double cs2 = d.cs2, c2 = d.c * d.c;
  double e = cs2;
  if (d.equilibrium == LBW_EQ_MOMENT_MATCHING) e = c2;
  if (d.equilibrium == LBW_EQ_HERMITE) e = cs2 + (c2 - cs2) * (1.0 - 3.0 * cs2) / (2.0 * cs2);
  *E = e;
  *two0 = 2.0 - 6.0 * e;
}

// population stride of a lattice's storage in elements
inline long long pop_stride(const Grid* g) {
  return g->pitch ? (long long)g->d.n[0] * g->d.n[2] * g->pitch : g->nn;
}

// kernels (lbw_step.cu) ---------------------------------------------------------------------
cudaError_t launch_step(Grid* g, int src);             // one time step, buffer src -> 1-src
cudaError_t launch_init(Grid* g, const double* d_pulses, int npulse);
cudaError_t launch_field(Grid* g, double* d_P);        // P of the current state
cudaError_t launch_to_double(Grid* g, double* d_f);    // current populations -> doubles
cudaError_t launch_from_double(Grid* g, const double* d_f);
void step_launch_shape(Grid* g);                       // choose bx, by, lz, grid_dim
// After step t (counters[0] = t): every source node's populations become the equilibrium that
// carries amp sin(omega t) as P (kind 0) or as J'_z (kind 1).
cudaError_t launch_sources(int prec, void* base, const SourceEntry* d_entries, int n, int kind,
                           double amp, const unsigned long long* d_counters, cudaStream_t stream);
// 128-byte CUtensorMap for a tiled TMA view: element type from lbw_prec, dims / box innermost
// first, strides in bytes of dimensions 1 .. rank - 1; false when the driver refuses it
bool encode_tiled_map(void* map, int prec, int rank, void* base, const uint64_t* dims,
                      const uint64_t* strides, const uint32_t* box);

// spectrum (lbw_spectrum.cu) ----------------------------------------------------------------
// The k strongest peaks (lowest = false) or the k lowest-frequency peaks (lowest = true)
// whose power is at least rel_power of the strongest.
lbw_status spectrum_device(const double* d_x, int64_t T, int32_t n_series, int32_t stride_series,
                           bool sum_all, int32_t k, cudaStream_t s, double* h_freq,
                           double* h_amp, int32_t* h_n, bool lowest = false,
                           double rel_power = 1e-3);

}  // namespace lbw
