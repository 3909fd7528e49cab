// lbw_march.cuh -- per-node arithmetic of the fused step and the register-pipelined tile march,
// shared by the single-lattice kernels (lbw_step.cu) and the batched ensemble (lbw_batch.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lbw_internal.h"

namespace lbw {
namespace dev {

// storage <-> arithmetic conversion; 16-bit formats store f_i / w_i
template <typename S> struct Store;
template <> struct Store<double> {
  using R = double;
  static constexpr bool kScaled = false;
  __device__ static R ld(const double* p) { return __ldg(p); }
  __device__ static R ld_smem(const double* p) { return *p; }
  __device__ static void st(double* p, R v) { *p = v; }
};
template <> struct Store<float> {
  using R = float;
  static constexpr bool kScaled = false;
  __device__ static R ld(const float* p) { return __ldg(p); }
  __device__ static R ld_smem(const float* p) { return *p; }
  __device__ static void st(float* p, R v) { *p = v; }
};
template <> struct Store<__half> {
  using R = float;
  static constexpr bool kScaled = true;
  __device__ static R ld(const __half* p) { return __half2float(__ldg(p)); }
  __device__ static R ld_smem(const __half* p) { return __half2float(*p); }
  __device__ static void st(__half* p, R v) { *p = __float2half_rn(v); }
};
template <> struct Store<__nv_bfloat16> {
  using R = float;
  static constexpr bool kScaled = true;
  __device__ static R ld(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
  __device__ static R ld_smem(const __nv_bfloat16* p) { return __bfloat162float(*p); }
  __device__ static void st(__nv_bfloat16* p, R v) { *p = __float2bfloat16_rn(v); }
};

// Closed-form geometry of the lattice for the analytic geometry mode: the metric of Sec. IV in
// lattice coordinates (x^a = x0^a + (q^a + 1/2) h^a), evaluated in the arithmetic type R.
template <typename R>
struct GeomArgs {
  int kind, profile;
  R x0r, x0w, h0, h1, h2;  // r (or x) and the third coordinate's origin, spacings
  R g0, g1, g2;            // torus R | Bessel horn Zmax, lambda | exponential a0, b, alpha
  R c2, cs2;
};

template <typename R>
struct MetricR {
  R sg, g11, g22, g33, g13, G1, G3;
};

// sqrt(g), g^{ab} and the contracted Christoffel symbols G^a at lattice position (q1, q3)
// (Eqs. MetricCylindrical, CylindricalChr; coordinatesTrumpet, MetricTrumpet with a general
// flare s(z); CoordinatesTorus, AMetricTorus, AChristoffelTorus), written in lattice units.
template <typename R>
__device__ MetricR<R> metric_q(const GeomArgs<R>& G, int q1, int q3) {
  const R r = G.x0r + (R(q1) + R(0.5)) * G.h0;
  const R w = G.x0w + (R(q3) + R(0.5)) * G.h2;
  R sg = 1, g11 = 1, g22 = 1, g33 = 1, g13 = 0, G1 = 0, G3 = 0;
  if (G.kind == LBW_POLAR || G.kind == LBW_CYLINDRICAL) {
    sg = r; g22 = R(1) / (r * r); G1 = R(-1) / r;
  } else if (G.kind == LBW_TRUMPET) {
    R s, ds, dds;
    if (G.profile == 0) {
      const R Z = G.g0 - w, lam = G.g1;
      s = pow(Z, -lam);
      ds = lam * s / Z;
      dds = lam * (lam + R(1)) * s / (Z * Z);
    } else {
      const R e = exp(G.g2 * w), A = G.g0 + G.g1;
      s = (G.g0 + G.g1 * e) / A;
      ds = G.g1 * G.g2 * e / A;
      dds = G.g2 * ds;
    }
    sg = r * s * s;
    g11 = (R(1) + r * r * ds * ds) / (s * s);
    g13 = -r * ds / s;
    g22 = R(1) / (r * r * s * s);
    G1 = (r * r * s * dds - R(2) * r * r * ds * ds - R(1)) / (r * s * s);
  } else if (G.kind == LBW_TOROIDAL) {
    const R cp = cos(w), Rr = G.g0 + r * cp;
    sg = r * Rr;
    g22 = R(1) / (Rr * Rr);
    g33 = R(1) / (r * r);
    G1 = -(G.g0 + R(2) * r * cp) / (r * Rr);
    G3 = sin(w) / (r * Rr);
  }
  MetricR<R> m;
  m.sg = sg * G.h0 * G.h1 * G.h2;
  m.g11 = g11 / (G.h0 * G.h0);
  m.g22 = g22 / (G.h1 * G.h1);
  m.g33 = g33 / (G.h2 * G.h2);
  m.g13 = g13 / (G.h0 * G.h2);
  m.G1 = G1 / G.h0;
  m.G3 = G3 / G.h2;
  return m;
}

// The 16 force coefficients (TableSlot) of row (q1, q3) from the metric at the row, m, and at
// its four neighbours nb = (q1 - 1, q1 + 1, q3 - 1, q3 + 1), each taken at the wrapped position
// across a periodic face and at the ghost position across any other face.  Ghost rules as in
// the host-built table: free -> rho copied; bounce-back -> P mirrored; anti-bounce-back -> P
// mirrored with opposite sign.
template <typename R>
__device__ void table_row(const GeomArgs<R>& G, const int (&bc)[6], int n1, int n3, int q1, int q3,
                          const MetricR<R>& m, const MetricR<R> (&nb)[4], R* out) {
  R e[T_SLOTS];
#pragma unroll
  for (int k = 0; k < T_SLOTS; ++k) e[k] = R(0);
  e[T_H22] = R(0.5) * (G.c2 * m.g22 - G.cs2);
  e[T_MG1] = -G.c2 * m.G1;
  e[T_MG3] = -G.c2 * m.G3;
  e[T_SG] = m.sg;
  e[T_INVSG] = R(1) / m.sg;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int axis = k < 2 ? 0 : 2, s = (k & 1) ? 1 : -1;
    const int pos = (axis == 0 ? q1 : q3) + s, n = axis == 0 ? n1 : n3;
    const int face = 2 * axis + (s > 0 ? 1 : 0);
    const bool ghost = (pos < 0 || pos >= n) && bc[face] != LBW_BC_PERIODIC;
    const MetricR<R>& mn = nb[k];
    const R K11 = G.c2 * mn.g11 - G.cs2, K13 = G.c2 * mn.g13, K33 = G.c2 * mn.g33 - G.cs2;
    const R k1 = axis == 0 ? K11 : K13, k3 = axis == 0 ? K13 : K33;
    if (ghost) {
      const R self = bc[face] == LBW_BC_FREE ? R(1) : (bc[face] == LBW_BC_BOUNCE ? R(1) : R(-1)) * mn.sg / m.sg;
      e[T_S1] += R(0.5) * R(s) * k1 * self;
      e[T_S3] += R(0.5) * R(s) * k3 * self;
    } else if (axis == 0) {
      e[s > 0 ? T_A1P : T_A1M] = R(0.5) * k1;
      e[s > 0 ? T_B13P : T_B13M] = R(0.5) * k3;
    } else {
      e[s > 0 ? T_C13P : T_C13M] = R(0.5) * k1;
      e[s > 0 ? T_C33P : T_C33M] = R(0.5) * k3;
    }
  }
#pragma unroll
  for (int k = 0; k < T_SLOTS; ++k) out[k] = e[k];
}

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
  // storage geometry of the populations: row length, first data column and population stride
  // in elements (dense lattices: n2, 0, nn; ensembles on the tile kernel pad every row with
  // ghost columns that mirror the periodic wrap)
  int pitch, col0;
  long long ps;
  GeomArgs<R> geo;  // closed-form geometry (used by the tile kernel in the analytic mode)
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

// Register-pipelined march of one (q2, q1) tile over planes z0 .. z1 - 1 of the lattice a
// (one time step of the paper's scheme for those nodes).  The CTA is BX x BY threads (blockDim);
// `planes` holds three rho planes of (BX + 2) x (BY + 2) values; the caller has filled
// probe_list / probe_cnt with the probes inside this tile and segment.  For each plane the
// CTA pulls the populations of the plane ahead, so the post-stream rho of plane z + 1 is known
// before plane z collides: rho along q3 stays in registers, rho of the current plane (tile plus
// a one-node halo) in shared memory, one __syncthreads per plane.
template <typename S>
__device__ __forceinline__ void march_tile(const StepArgs<S>& a, int x0, int y0, int z0, int z1,
                                           typename Store<S>::R* planes, const int* probe_list,
                                           const int& probe_cnt, unsigned long long t_sample) {
  using R = typename Store<S>::R;
  const int BX = blockDim.x, BY = blockDim.y;
  const int PW = BX + 2, PS = PW * (BY + 2);
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
  const int q2 = x0 + tx, q1 = y0 + ty;
  const bool valid = (q2 < a.n2) && (q1 < a.n1);
  const int nhalo = 2 * BX + 2 * BY;
  const bool p1 = a.bc[0] == LBW_BC_PERIODIC, p2 = a.bc[2] == LBW_BC_PERIODIC;

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

}

// Probes of lattice a that fall in the tile [x0, x0 + BX) x [y0, y0 + BY) x [z0, z1).
template <typename S>
__device__ __forceinline__ void scan_probes(const StepArgs<S>& a, int x0, int y0, int z0, int z1,
                                            int* probe_list, int* probe_cnt) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if (tid < a.nprobe) {
    const int pq1 = a.probe_q[3 * tid], pq2 = a.probe_q[3 * tid + 1], pq3 = a.probe_q[3 * tid + 2];
    if (pq1 >= y0 && pq1 < y0 + (int)blockDim.y && pq2 >= x0 && pq2 < x0 + (int)blockDim.x &&
        pq3 >= z0 && pq3 < z1)
      probe_list[atomicAdd(probe_cnt, 1)] = tid;
  }
}

// The last CTA to finish a step advances the step and sample counters (no spin-wait).
__device__ __forceinline__ void finish_step(unsigned long long* counters, int nprobe, long long cap,
                                            unsigned int nblocks) {
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    __threadfence();
    unsigned int ticket = atomicAdd(reinterpret_cast<unsigned int*>(&counters[2]), 1u);
    if (ticket == nblocks - 1) {
      counters[0] += 1;
      if (nprobe > 0 && counters[1] < (unsigned long long)cap) counters[1] += 1;
      counters[2] = 0;
      __threadfence();
    }
  }
}

}  // namespace dev
}  // namespace lbw
