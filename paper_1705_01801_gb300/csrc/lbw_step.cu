// lbw_step.cu -- the fused stream + collide time step and the state kernels.
//
// One launch advances the whole lattice by one time step of the paper's scheme
// (Sec. III "Summarizing"): pull streaming along xi_i with the face rules of Sec. IV.A,
// rho = sum f (Eq. PressureCurvedSystem), the geometric forcing term with its divergence by
// central differences of the post-stream rho (Eqs. JCorrectionForce, DerivativeFromTaylor),
// the shifted momentum (Eq. JShifted), the corrected equilibrium
// (Eq. EquilibriumCurvedSystemHermiteCorrected) and BGK relaxation at tau = 1/2
// (f* = 2 f^eq - f, Eq. SecondOrder).
//
// Work decomposition (GB300): a CTA owns a (q2, q1) tile of BX x BY columns and marches
// along q3 over a segment of LZ planes.  For each plane it pulls the seven populations of
// the plane ahead, so the post-stream rho of plane z+1 is known before plane z collides:
// rho along q3 stays in registers, rho of the current plane (tile plus a one-node halo) sits
// in a triple-buffered shared-memory plane, so each plane costs one __syncthreads.  All
// loads and stores are coalesced along q2 (the fastest axis).  The q3 segments make the
// grid a multiple of the resident CTA count on the 152 SMs.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "lbw_internal.h"

namespace lbw {
namespace {

// storage <-> arithmetic conversion; 16-bit formats store f_i / w_i
template <typename S> struct Store;
template <> struct Store<double> {
  using R = double;
  static constexpr bool kScaled = false;
  __device__ static R ld(const double* p) { return __ldg(p); }
  __device__ static void st(double* p, R v) { *p = v; }
};
template <> struct Store<float> {
  using R = float;
  static constexpr bool kScaled = false;
  __device__ static R ld(const float* p) { return __ldg(p); }
  __device__ static void st(float* p, R v) { *p = v; }
};
template <> struct Store<__half> {
  using R = float;
  static constexpr bool kScaled = true;
  __device__ static R ld(const __half* p) { return __half2float(__ldg(p)); }
  __device__ static void st(__half* p, R v) { *p = __float2half_rn(v); }
};
template <> struct Store<__nv_bfloat16> {
  using R = float;
  static constexpr bool kScaled = true;
  __device__ static R ld(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
  __device__ static void st(__nv_bfloat16* p, R v) { *p = __float2bfloat16_rn(v); }
};

template <typename S>
struct StepArgs {
  using R = typename Store<S>::R;
  const S* __restrict__ fin;
  S* __restrict__ fout;
  const R* __restrict__ tab;
  int n1, n2, n3, lz;
  long long nn;
  int bc[6];
  R damping, cs2, two_w0;
  R w[7], inv_w[7];      // storage scale (16-bit formats)
  R s2lo, s2hi;          // rho ghost factor of a non-periodic q2 face
  int nprobe;
  const int* __restrict__ probe_q;
  double* __restrict__ series;
  long long cap;
  unsigned long long* counters;
  unsigned int nblocks;
};

__device__ __forceinline__ long long node(int q1, int q2, int q3, int n1, int n2) {
  return ((long long)q3 * n1 + q1) * n2 + q2;
}

template <typename S>
__device__ __forceinline__ typename Store<S>::R ldf(const StepArgs<S>& a, int i, long long x) {
  typename Store<S>::R v = Store<S>::ld(a.fin + (long long)i * a.nn + x);
  if (Store<S>::kScaled) v *= a.w[i];
  return v;
}

// Value of population i streamed into node x across face `face` (source outside the lattice).
template <typename S>
__device__ __forceinline__ typename Store<S>::R across(const StepArgs<S>& a, int face, int i,
                                                       int opp, long long x, long long wrap) {
  switch (a.bc[face]) {
    case LBW_BC_PERIODIC: return ldf(a, i, x + wrap);
    case LBW_BC_BOUNCE: return a.damping * ldf(a, opp, x);   // f_out = D f_in
    case LBW_BC_ANTIBOUNCE: return -ldf(a, opp, x);          // P = 0 wall
    default: return ldf(a, i, x);                            // free: copy of the node
  }
}

// Pull streaming of all seven populations into the in-range node (q1, q2, q3).
template <typename S>
__device__ __forceinline__ void pull(const StepArgs<S>& a, int q1, int q2, int q3,
                                     typename Store<S>::R f[7]) {
  const int n1 = a.n1, n2 = a.n2, n3 = a.n3;
  const long long x = node(q1, q2, q3, n1, n2);
  const long long s1 = n2, s3 = (long long)n1 * n2;
  f[0] = ldf(a, 0, x);
  f[1] = (q1 > 0) ? ldf(a, 1, x - s1) : across(a, 0, 1, 2, x, (long long)(n1 - 1) * s1);
  f[2] = (q1 < n1 - 1) ? ldf(a, 2, x + s1) : across(a, 1, 2, 1, x, -(long long)(n1 - 1) * s1);
  f[3] = (q2 > 0) ? ldf(a, 3, x - 1) : across(a, 2, 3, 4, x, (long long)(n2 - 1));
  f[4] = (q2 < n2 - 1) ? ldf(a, 4, x + 1) : across(a, 3, 4, 3, x, -(long long)(n2 - 1));
  f[5] = (q3 > 0) ? ldf(a, 5, x - s3) : across(a, 4, 5, 6, x, (long long)(n3 - 1) * s3);
  f[6] = (q3 < n3 - 1) ? ldf(a, 6, x + s3) : across(a, 5, 6, 5, x, -(long long)(n3 - 1) * s3);
}

// Map a possibly out-of-range coordinate to the lattice: periodic wrap, or -1 for a ghost.
__device__ __forceinline__ int resolve(int q, int n, bool periodic) {
  if (q >= 0 && q < n) return q;
  if (!periodic) return -1;
  const int m = q % n;  // tiles may be wider than the lattice (e.g. n = 1)
  return m < 0 ? m + n : m;
}

// Post-stream rho at a possibly out-of-range position; ghosts give 0 (their contribution
// to the force is folded into the coefficient table).
template <typename S>
__device__ __forceinline__ typename Store<S>::R rho_at(const StepArgs<S>& a, int q1, int q2,
                                                       int q3) {
  q1 = resolve(q1, a.n1, a.bc[0] == LBW_BC_PERIODIC);
  q2 = resolve(q2, a.n2, a.bc[2] == LBW_BC_PERIODIC);
  q3 = resolve(q3, a.n3, a.bc[4] == LBW_BC_PERIODIC);
  if (q1 < 0 || q2 < 0 || q3 < 0) return 0;
  typename Store<S>::R f[7];
  pull(a, q1, q2, q3, f);
  return ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + f[6]);
}

template <typename S>
__global__ void __launch_bounds__(512) step_kernel(const StepArgs<S> a) {
  using R = typename Store<S>::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* planes = reinterpret_cast<R*>(smem_raw);
  __shared__ int probe_list[kMaxProbes];
  __shared__ int probe_cnt;
  __shared__ unsigned long long t_sample;

  const int BX = blockDim.x, BY = blockDim.y;
  const int PW = BX + 2, PS = PW * (BY + 2);
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
  const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
  const int z0 = blockIdx.z * a.lz, z1 = min(z0 + a.lz, a.n3);
  const int q2 = x0 + tx, q1 = y0 + ty;
  const bool valid = (q2 < a.n2) && (q1 < a.n1);
  const int nhalo = 2 * BX + 2 * BY;
  const bool p1 = a.bc[0] == LBW_BC_PERIODIC, p2 = a.bc[2] == LBW_BC_PERIODIC;

  if (tid == 0) {
    probe_cnt = 0;
    t_sample = a.counters[1];
  }
  __syncthreads();
  if (tid < a.nprobe) {
    const int pq1 = a.probe_q[3 * tid], pq2 = a.probe_q[3 * tid + 1], pq3 = a.probe_q[3 * tid + 2];
    if (pq1 >= y0 && pq1 < y0 + BY && pq2 >= x0 && pq2 < x0 + BX && pq3 >= z0 && pq3 < z1) {
      int slot = atomicAdd(&probe_cnt, 1);
      probe_list[slot] = tid;
    }
  }

  // the halo slot this thread fills (rows q1 = y0-1 / y0+BY, columns q2 = x0-1 / x0+BX)
  int h1 = 0, h2 = 0, hslot = -1;
  if (tid < nhalo) {
    if (tid < BX) { h1 = y0 - 1; h2 = x0 + tid; hslot = tid + 1; }
    else if (tid < 2 * BX) { h1 = y0 + BY; h2 = x0 + tid - BX; hslot = (BY + 1) * PW + tid - BX + 1; }
    else if (tid < 2 * BX + BY) { h1 = y0 + tid - 2 * BX; h2 = x0 - 1; hslot = (tid - 2 * BX + 1) * PW; }
    else { h1 = y0 + tid - 2 * BX - BY; h2 = x0 + BX; hslot = (tid - 2 * BX - BY + 1) * PW + BX + 1; }
  }
  const int own = (ty + 1) * PW + tx + 1;
  // position this thread's own slot stands for (ragged tiles resolve through the faces)
  const int o1 = resolve(q1, a.n1, p1), o2 = resolve(q2, a.n2, p2);

  R fc[7], fn[7];
  R rp = rho_at(a, q1, q2, z0 - 1);  // plane below the segment: rho of own column only
  R rc;
  {
    // plane z0: own populations (valid threads) and the plane's rho into buffer 0
    if (valid) {
      pull(a, q1, q2, z0, fc);
      rc = ((fc[0] + fc[1]) + (fc[2] + fc[3])) + ((fc[4] + fc[5]) + fc[6]);
    } else {
      rc = (o1 >= 0 && o2 >= 0) ? rho_at(a, o1, o2, z0) : R(0);
    }
    planes[own] = rc;
    if (hslot >= 0) planes[hslot] = rho_at(a, h1, h2, z0);
  }

  for (int z = z0; z < z1; ++z) {
    const int b = (z - z0) % 3;
    R* cur = planes + b * PS;
    R* nxt = planes + ((b + 1) % 3) * PS;
    R rn;
    if (z + 1 < z1) {
      if (valid) {
        pull(a, q1, q2, z + 1, fn);
        rn = ((fn[0] + fn[1]) + (fn[2] + fn[3])) + ((fn[4] + fn[5]) + fn[6]);
      } else {
        rn = (o1 >= 0 && o2 >= 0) ? rho_at(a, o1, o2, z + 1) : R(0);
      }
      nxt[own] = rn;
      if (hslot >= 0) nxt[hslot] = rho_at(a, h1, h2, z + 1);
    } else {
      rn = valid ? rho_at(a, q1, q2, z + 1) : R(0);
    }
    __syncthreads();

    if (valid) {
      const R* T = a.tab + ((long long)z * a.n1 + q1) * T_SLOTS;
      R c[T_SLOTS];
#pragma unroll
      for (int k = 0; k < T_SLOTS; k += 4) {
        if (sizeof(R) == 4) {
          float4 v = __ldg(reinterpret_cast<const float4*>(T + k));
          c[k] = v.x; c[k + 1] = v.y; c[k + 2] = v.z; c[k + 3] = v.w;
        } else {
          double2 v0 = __ldg(reinterpret_cast<const double2*>(T + k));
          double2 v1 = __ldg(reinterpret_cast<const double2*>(T + k + 2));
          c[k] = v0.x; c[k + 1] = v0.y; c[k + 2] = v1.x; c[k + 3] = v1.y;
        }
      }
      const R rho = rc;
      const R rd = cur[own - PW], ru = cur[own + PW];
      R rl = cur[own - 1], rr = cur[own + 1];
      if (q2 == 0 && !p2) rl = a.s2lo * rho;
      if (q2 == a.n2 - 1 && !p2) rr = a.s2hi * rho;
      const R D1 = c[T_A1P] * ru - c[T_A1M] * rd + c[T_C13P] * rn - c[T_C13M] * rp + c[T_S1] * rho;
      const R D3 = c[T_B13P] * ru - c[T_B13M] * rd + c[T_C33P] * rn - c[T_C33M] * rp + c[T_S3] * rho;
      const R D2 = c[T_H22] * (rr - rl);
      const R half = R(0.5);
      const R j1 = (fc[1] - fc[2]) + half * (c[T_MG1] * rho - D1);
      const R j2 = (fc[3] - fc[4]) - half * D2;
      const R j3 = (fc[5] - fc[6]) + half * (c[T_MG3] * rho - D3);
      const R e = a.cs2 * rho;
      R o[7];
      o[0] = a.two_w0 * rho - fc[0];
      o[1] = e + j1 - fc[1];
      o[2] = e - j1 - fc[2];
      o[3] = e + j2 - fc[3];
      o[4] = e - j2 - fc[4];
      o[5] = e + j3 - fc[5];
      o[6] = e - j3 - fc[6];
      const long long x = node(q1, q2, z, a.n1, a.n2);
#pragma unroll
      for (int i = 0; i < 7; ++i) {
        R v = o[i];
        if (Store<S>::kScaled) v *= a.inv_w[i];
        Store<S>::st(a.fout + (long long)i * a.nn + x, v);
      }
      if (probe_cnt > 0 && t_sample < (unsigned long long)a.cap) {
        for (int s = 0; s < probe_cnt; ++s) {
          const int k = probe_list[s];
          if (a.probe_q[3 * k] == q1 && a.probe_q[3 * k + 1] == q2 && a.probe_q[3 * k + 2] == z)
            a.series[(long long)k * a.cap + t_sample] = (double)rho * (double)c[T_INVSG];
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 7; ++i) fc[i] = fn[i];
    rp = rc;
    rc = rn;
  }

  // the last CTA to finish advances the step and sample counters (no spin-wait)
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    unsigned int ticket = atomicAdd(reinterpret_cast<unsigned int*>(&a.counters[2]), 1u);
    if (ticket == a.nblocks - 1) {
      a.counters[0] += 1;
      if (a.nprobe > 0 && a.counters[1] < (unsigned long long)a.cap) a.counters[1] += 1;
      a.counters[2] = 0;
      __threadfence();
    }
  }
}

template <typename S>
StepArgs<S> make_args(Grid* g, int src) {
  using R = typename Store<S>::R;
  StepArgs<S> a;
  a.fin = reinterpret_cast<const S*>(g->f[src]);
  a.fout = reinterpret_cast<S*>(g->f[1 - src]);
  a.tab = reinterpret_cast<const R*>(g->table);
  a.n1 = g->d.n[0]; a.n2 = g->d.n[1]; a.n3 = g->d.n[2];
  a.lz = g->lz;
  a.nn = g->nn;
  for (int k = 0; k < 6; ++k) a.bc[k] = g->d.bc[k];
  a.damping = (R)g->d.damping;
  a.cs2 = (R)g->d.cs2;
  a.two_w0 = (R)(2.0 * g->w0);
  for (int i = 0; i < 7; ++i) {
    double w = i == 0 ? g->w0 : g->w1;
    a.w[i] = (R)w;
    a.inv_w[i] = (R)(1.0 / w);
  }
  a.s2lo = g->d.bc[2] == LBW_BC_ANTIBOUNCE ? R(-1) : R(1);
  a.s2hi = g->d.bc[3] == LBW_BC_ANTIBOUNCE ? R(-1) : R(1);
  a.nprobe = g->nprobe;
  a.probe_q = g->probe_q;
  a.series = g->series;
  a.cap = g->cap;
  a.counters = g->counters;
  a.nblocks = g->grid_dim.x * g->grid_dim.y * g->grid_dim.z;
  return a;
}

template <typename S>
cudaError_t launch_step_t(Grid* g, int src) {
  using R = typename Store<S>::R;
  StepArgs<S> a = make_args<S>(g, src);
  dim3 block(g->bx, g->by);
  size_t smem = 3 * (size_t)(g->bx + 2) * (g->by + 2) * sizeof(R);
  step_kernel<S><<<g->grid_dim, block, smem, g->stream>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- initial state ----------

struct InitGeom {
  int kind, profile;
  double h[3], x0[3], geom[4];
};

__device__ void embed_dev(const InitGeom& G, double u1, double u2, double u3, double X[3]) {
  switch (G.kind) {
    case LBW_CARTESIAN: X[0] = u1; X[1] = u2; X[2] = u3; break;
    case LBW_POLAR:
    case LBW_CYLINDRICAL: X[0] = u1 * cos(u2); X[1] = u1 * sin(u2); X[2] = u3; break;
    case LBW_TRUMPET: {
      double s;
      if (G.profile == 0) s = pow(G.geom[0] - u3, -G.geom[1]);
      else s = (G.geom[0] + G.geom[1] * exp(G.geom[2] * u3)) / (G.geom[0] + G.geom[1]);
      X[0] = u1 * s * cos(u2); X[1] = u1 * s * sin(u2); X[2] = u3;
      break;
    }
    default: {
      double rr = G.geom[0] + u1 * cos(u3);
      X[0] = rr * cos(u2); X[1] = rr * sin(u2); X[2] = u1 * sin(u3);
    }
  }
}

// rho0 = sqrt(g) P0, P0 a sum of Gaussian pulses in the embedding distance (FP64 math).
template <typename R>
__global__ void init_rho_kernel(InitGeom G, const double* __restrict__ pulses, int npulse,
                                const R* __restrict__ tab, int n1, int n2, int n3, R* rho0) {
  const long long nn = (long long)n1 * n2 * n3;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < nn;
       x += (long long)gridDim.x * blockDim.x) {
    const int q2 = (int)(x % n2);
    const int q1 = (int)((x / n2) % n1);
    const int q3 = (int)(x / ((long long)n1 * n2));
    double X[3];
    embed_dev(G, G.x0[0] + (q1 + 0.5) * G.h[0], G.x0[1] + (q2 + 0.5) * G.h[1],
              G.x0[2] + (q3 + 0.5) * G.h[2], X);
    double P0 = 0.0;
    for (int k = 0; k < npulse; ++k) {
      const double* p = pulses + 5 * k;
      const double d2 = (X[0] - p[0]) * (X[0] - p[0]) + (X[1] - p[1]) * (X[1] - p[1]) +
                        (X[2] - p[2]) * (X[2] - p[2]);
      P0 += p[4] * exp(-d2 / (2.0 * p[3] * p[3]));
    }
    rho0[x] = (R)((double)tab[((long long)q3 * n1 + q1) * T_SLOTS + T_SG] * P0);
  }
}

// Post-collision state at rest: f*_i = f_i^eq(rho0, F(rho0) / 2), F from the same table.
template <typename S>
__global__ void init_f_kernel(const StepArgs<S> a, const typename Store<S>::R* __restrict__ rho0) {
  using R = typename Store<S>::R;
  const bool p1 = a.bc[0] == LBW_BC_PERIODIC, p2 = a.bc[2] == LBW_BC_PERIODIC,
             p3 = a.bc[4] == LBW_BC_PERIODIC;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < a.nn;
       x += (long long)gridDim.x * blockDim.x) {
    const int q2 = (int)(x % a.n2);
    const int q1 = (int)((x / a.n2) % a.n1);
    const int q3 = (int)(x / ((long long)a.n1 * a.n2));
    auto at = [&](int r1, int r2, int r3) -> R {
      r1 = resolve(r1, a.n1, p1); r2 = resolve(r2, a.n2, p2); r3 = resolve(r3, a.n3, p3);
      if (r1 < 0 || r2 < 0 || r3 < 0) return R(0);
      return rho0[node(r1, r2, r3, a.n1, a.n2)];
    };
    const R* c = a.tab + ((long long)q3 * a.n1 + q1) * T_SLOTS;
    const R rho = rho0[x];
    const R ru = at(q1 + 1, q2, q3), rd = at(q1 - 1, q2, q3);
    const R rn = at(q1, q2, q3 + 1), rp = at(q1, q2, q3 - 1);
    R rr = at(q1, q2 + 1, q3), rl = at(q1, q2 - 1, q3);
    if (q2 == 0 && !p2) rl = a.s2lo * rho;
    if (q2 == a.n2 - 1 && !p2) rr = a.s2hi * rho;
    const R D1 = c[T_A1P] * ru - c[T_A1M] * rd + c[T_C13P] * rn - c[T_C13M] * rp + c[T_S1] * rho;
    const R D3 = c[T_B13P] * ru - c[T_B13M] * rd + c[T_C33P] * rn - c[T_C33M] * rp + c[T_S3] * rho;
    const R D2 = c[T_H22] * (rr - rl);
    const R j1 = R(0.5) * (c[T_MG1] * rho - D1), j2 = R(-0.5) * D2,
            j3 = R(0.5) * (c[T_MG3] * rho - D3);
    const R e = R(0.5) * a.cs2 * rho;
    R o[7] = {R(0.5) * a.two_w0 * rho, e + R(0.5) * j1, e - R(0.5) * j1, e + R(0.5) * j2,
              e - R(0.5) * j2, e + R(0.5) * j3, e - R(0.5) * j3};
#pragma unroll
    for (int i = 0; i < 7; ++i) {
      R v = o[i];
      if (Store<S>::kScaled) v *= a.inv_w[i];
      Store<S>::st(a.fout + (long long)i * a.nn + x, v);
    }
  }
}

template <typename S>
cudaError_t launch_init_t(Grid* g, const double* d_pulses, int npulse) {
  using R = typename Store<S>::R;
  InitGeom G;
  G.kind = g->d.kind;
  G.profile = g->d.horn_profile;
  for (int a = 0; a < 3; ++a) { G.h[a] = g->d.h[a]; G.x0[a] = g->d.x0[a]; }
  for (int k = 0; k < 4; ++k) G.geom[k] = g->d.geom[k];
  // rho0 goes to the scratch bytes of the other population buffer (>= N values of R)
  R* rho0 = reinterpret_cast<R*>(g->f[1 - g->cur]);
  const int threads = 256;
  const int blocks = (int)std::min<long long>((g->nn + threads - 1) / threads, 152LL * 16);
  init_rho_kernel<R><<<blocks, threads, 0, g->stream>>>(
      G, d_pulses, npulse, reinterpret_cast<const R*>(g->table), g->d.n[0], g->d.n[1],
      g->d.n[2], rho0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  StepArgs<S> a = make_args<S>(g, 1 - g->cur);  // fout = current buffer
  init_f_kernel<S><<<blocks, threads, 0, g->stream>>>(a, rho0);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- read-out ---------------

template <typename S>
__global__ void field_kernel(const S* __restrict__ f, long long nn, int n1, int n2,
                             const typename Store<S>::R* __restrict__ tab, double w0,
                             double w1, double* __restrict__ P) {
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < nn;
       x += (long long)gridDim.x * blockDim.x) {
    const int q1 = (int)((x / n2) % n1);
    const int q3 = (int)(x / ((long long)n1 * n2));
    double r = 0.0;
    for (int i = 0; i < 7; ++i) {
      double v = (double)Store<S>::ld(f + (long long)i * nn + x);
      if (Store<S>::kScaled) v *= (i == 0 ? w0 : w1);
      r += v;
    }
    P[x] = r * (double)tab[((long long)q3 * n1 + q1) * T_SLOTS + T_INVSG];
  }
}

template <typename S>
__global__ void to_double_kernel(const S* __restrict__ f, long long nn, double w0, double w1,
                                 double* __restrict__ out) {
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < 7 * nn;
       x += (long long)gridDim.x * blockDim.x) {
    double v = (double)Store<S>::ld(f + x);
    if (Store<S>::kScaled) v *= (x < nn ? w0 : w1);
    out[x] = v;
  }
}

template <typename S>
__global__ void from_double_kernel(const double* __restrict__ in, long long nn, double w0,
                                   double w1, S* __restrict__ f) {
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < 7 * nn;
       x += (long long)gridDim.x * blockDim.x) {
    double v = in[x];
    if (Store<S>::kScaled) v /= (x < nn ? w0 : w1);
    Store<S>::st(f + x, (typename Store<S>::R)v);
  }
}

template <typename S>
cudaError_t launch_readout_t(Grid* g, int what, double* d_out, const double* d_in) {
  const int threads = 256;
  const int blocks = 152 * 8;
  const S* f = reinterpret_cast<const S*>(g->f[g->cur]);
  if (what == 0)
    field_kernel<S><<<blocks, threads, 0, g->stream>>>(
        f, g->nn, g->d.n[0], g->d.n[1], reinterpret_cast<const typename Store<S>::R*>(g->table),
        g->w0, g->w1, d_out);
  else if (what == 1)
    to_double_kernel<S><<<blocks, threads, 0, g->stream>>>(f, g->nn, g->w0, g->w1, d_out);
  else
    from_double_kernel<S><<<blocks, threads, 0, g->stream>>>(
        d_in, g->nn, g->w0, g->w1, reinterpret_cast<S*>(g->f[g->cur]));
  return cudaGetLastError();
}

template <typename F>
cudaError_t dispatch(int prec, F&& fn) {
  switch (prec) {
    case LBW_F64: return fn(double());
    case LBW_F32: return fn(float());
    case LBW_F16S: return fn(__half());
    default: return fn(__nv_bfloat16());
  }
}

}  // namespace

cudaError_t launch_step(Grid* g, int src) {
  return dispatch(g->d.prec, [&](auto tag) { return launch_step_t<decltype(tag)>(g, src); });
}

cudaError_t launch_init(Grid* g, const double* d_pulses, int npulse) {
  return dispatch(g->d.prec,
                  [&](auto tag) { return launch_init_t<decltype(tag)>(g, d_pulses, npulse); });
}

cudaError_t launch_field(Grid* g, double* d_P) {
  return dispatch(g->d.prec,
                  [&](auto tag) { return launch_readout_t<decltype(tag)>(g, 0, d_P, nullptr); });
}

cudaError_t launch_to_double(Grid* g, double* d_f) {
  return dispatch(g->d.prec,
                  [&](auto tag) { return launch_readout_t<decltype(tag)>(g, 1, d_f, nullptr); });
}

cudaError_t launch_from_double(Grid* g, const double* d_f) {
  return dispatch(g->d.prec,
                  [&](auto tag) { return launch_readout_t<decltype(tag)>(g, 2, nullptr, d_f); });
}

// CTA tile: BX columns along q2 (a multiple of 32, at most 128) by BY rows along q1 with
// BX * BY = 512; q3 segments so the grid fills every resident CTA slot on the device.
void step_launch_shape(Grid* g) {
  const int n1 = g->d.n[0], n2 = g->d.n[1], n3 = g->d.n[2];
  int bx = std::min(128, ((n2 + 31) / 32) * 32);
  int by = 512 / bx;
  g->bx = bx;
  g->by = by;
  const long long cols = (long long)((n2 + bx - 1) / bx) * ((n1 + by - 1) / by);
  int dev = 0, sms = 152, per_sm = 2;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long slots = (long long)sms * per_sm;
  long long segs = std::max<long long>(1, (slots + cols - 1) / cols);
  segs = std::min<long long>(segs, n3);
  int lz = (int)((n3 + segs - 1) / segs);
  g->lz = lz;
  g->grid_dim = dim3((n2 + bx - 1) / bx, (n1 + by - 1) / by, (n3 + lz - 1) / lz);
}

}  // namespace lbw
