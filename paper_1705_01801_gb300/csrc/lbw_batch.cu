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
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "lbw_internal.h"
#include "lbw_march.cuh"
#include "lbw_tma.cuh"

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

// ---------------------------------------------------------------- TMA-staged ensemble ------
//
// Members whose q2 axis is periodic are stored with padded rows: G = 16 / sizeof(S) ghost
// columns on each side of the n2 data columns (ghost-left = the last G data columns,
// ghost-right = the first G), the row rounded up to 16 bytes.  A 64-column tile's box
// [x0, x0 + 64 + 2 G) in stored columns starts 16-byte aligned; past the row end it reads
// zeros (outside the tensor, no memory traffic).  A tile therefore stages each population with
// ONE tensor copy whatever n2 is (ragged last tiles and the periodic wrap included), and the
// step writes the ghost copies of the G nodes next to the wrap.  The persistent CTA walks (member, q2 tile, q1 tile, q3 segment) items; per item it
// copies the member's StepArgs into shared memory, re-initialises its mbarriers and runs the
// same producer / consumer pipeline as the single-lattice tile kernel (lbw_step.cu:
// step_tma_kernel), two nodes per lane.  Tiles start at q1 = -1 instead of 0 when
// (n1 - 1) is a multiple of BY, so no halo row ever sits on a q1 face.
constexpr int kTmaBatchBX = 64;

template <typename S, int BY>
struct BatchTmaLayout {
  static constexpr int G = 16 / (int)sizeof(S);
  static constexpr int RW = kTmaBatchBX + 2 * G;  // staged row: G | 64 data columns | G
  static constexpr int POPB = (((BY + 2) * RW * (int)sizeof(S)) + 127) / 128 * 128;
  static constexpr int SLOTB = 7 * POPB;
};

template <typename S, int BY>
constexpr size_t batch_tma_smem() {
  using R = typename Store<S>::R;
  constexpr int NB = 5, PS = (BY + 2) * (kTmaBatchBX + 4);
  constexpr int TABB = ((BY * T_SLOTS * (int)sizeof(R)) + 127) / 128 * 128;
  return 128 + 128 + (size_t)NB * BatchTmaLayout<S, BY>::SLOTB + ((3 * PS * sizeof(R) + 127) / 128) * 128 +
         (size_t)NB * TABB;
}

__device__ __forceinline__ void mbar_inval(unsigned bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(bar) : "memory");
}

template <typename S, int BY>
__global__ void __launch_bounds__(32 * (BY + 3)) batch_tma_kernel(
    const StepArgs<S>* __restrict__ members, const CUtensorMap* __restrict__ maps, int src,
    const int4* __restrict__ items, int n_items, int lz, unsigned long long* counters, int nprobe,
    long long cap) {
  using R = typename Store<S>::R;
  using L = BatchTmaLayout<S, BY>;
  constexpr int NPT = 2, BX = kTmaBatchBX, NB = 5, ROWS = BY + 2, NCW = ROWS;
  constexpr int ES = (int)sizeof(S), RS = (int)sizeof(R);
  constexpr int G = L::G, RW = L::RW, POPB = L::POPB, SLOTB = L::SLOTB;
  constexpr int C0 = NPT, PW = BX + 2 * NPT, PS = ROWS * PW;
  constexpr int TABB = ((BY * T_SLOTS * RS) + 127) / 128 * 128;
  constexpr int RHOB = ((3 * PS * RS) + 127) / 128 * 128;
  constexpr bool SC = Store<S>::kScaled;
  // slot grouping as in step_tma_kernel: 32- and 64-bit storage carry population 6 of plane
  // p + 1 in plane p's slot, 16-bit storage keeps whole planes
  constexpr bool RG = sizeof(S) >= 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) StepArgs<S> A;
  __shared__ int probe_list[kMaxProbes];
  __shared__ int probe_cnt;
  __shared__ int abort_flag;
  __shared__ int next_it;
  __shared__ unsigned long long t_sample;

  const int lane = threadIdx.x, w = threadIdx.y, tid = w * 32 + lane, nthr = 32 * (BY + 3);
  // items are claimed from a step-wide counter (the upper half of counters[2], cleared with
  // the ticket by the step's last CTA): CTAs that draw small items take more of them, so the
  // step ends when the work does (a fixed stride over the list left CTAs idle behind others
  // with larger items; the 512-trumpet ensemble ran 20% slower).  The producer claims the
  // next item once it has issued the current item's last copies, a few planes before the
  // CTA is free: neighbouring items (consecutive in the list) then start within a few
  // microseconds of each other and march in step, so the rows and planes they share are
  // read from DRAM once and found in L2 by the other.
  unsigned* const claim = reinterpret_cast<unsigned*>(&counters[2]) + 1;
  const unsigned sbase = smem_u32(smem_raw);
  const unsigned OFF = (128u - (sbase & 127u)) & 127u;
  const unsigned SL = OFF + 128, RHO = SL + NB * SLOTB, TAB = RHO + RHOB;
  auto full_at = [&](int k) { return sbase + OFF + 8u * k; };
  auto empty_at = [&](int k) { return sbase + OFF + 8u * (NB + k); };
  if (tid == 0) {
    abort_flag = 0;
    t_sample = counters[1];
    next_it = (int)atomicAdd(claim, 1u);
  }
  __syncthreads();

  bool fresh = true;
  for (int it = next_it; it < n_items;) {
    const int4 item = items[it];  // member, x0 (data column), y0 (may be -1), z0
    {
      const unsigned* from = reinterpret_cast<const unsigned*>(members + item.x);
      unsigned* to = reinterpret_cast<unsigned*>(&A);
      for (int k = tid; k < (int)(sizeof(StepArgs<S>) / 4); k += nthr) to[k] = from[k];
    }
    if (tid == 0) {
      for (int k = 0; k < NB; ++k) {
        if (!fresh) {  // the previous item left its phases behind
          mbar_inval(full_at(k));
          mbar_inval(empty_at(k));
        }
        mbar_init_count(full_at(k), 1);
        mbar_init_count(empty_at(k), NCW);
      }
      asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
      probe_cnt = 0;
    }
    fresh = false;
    __syncthreads();  // every thread has read next_it for this item
    const int x0 = item.y, y0 = item.z, z0 = item.w;
    const int z1 = min(z0 + lz, A.n3);
    const bool p3 = A.bc[4] == LBW_BC_PERIODIC;
    if (tid < A.nprobe) {
      const int pq1 = A.probe_q[3 * tid], pq2 = A.probe_q[3 * tid + 1], pq3 = A.probe_q[3 * tid + 2];
      if (pq1 >= y0 && pq1 < y0 + BY && pq2 >= x0 && pq2 < x0 + BX && pq3 >= z0 && pq3 < z1)
        probe_list[atomicAdd(&probe_cnt, 1)] = tid;
    }
    __syncthreads();
    const CUtensorMap* tm_f = maps + 3 * item.x + src;
    const CUtensorMap* tm_t = maps + 3 * item.x + 2;

    auto wait_bar = [&](unsigned bar, unsigned parity) -> bool {
      long long n = 0;
      while (!mbar_try_wait(bar, parity)) {
        if (++n > kWaitLimit) {
          abort_flag = 1;
          A.counters[3] = 1;
          return false;
        }
      }
      return true;
    };

    if (w == ROWS) {  // ---------------------------------------------------------- producer
      if (lane == 0) {
        // the previous item's generic-proxy reads of the slots come before these copies
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        const unsigned tx_pop = (unsigned)(ROWS * RW * ES);
        int s = 0, use = 0, issued = z0 - 3;
        for (int p = z0 - 2; p <= z1 + (RG ? 0 : 1); ++p) {
          if (use > 0 && !wait_bar(empty_at(s), (unsigned)((use - 1) & 1))) break;
          const unsigned bar = full_at(s);
          const unsigned base = sbase + SL + s * SLOTB;
          const int pg = resolve(p, A.n3, p3);
          if (p == z0 - 2) {
            // only population 5 of this plane streams into the segment; when the first pulled
            // plane z0 - 1 is the q3 = 0 face of a wall, its reflected population 6 rides here
            const int pn = (RG && !p3 && z0 == 1) ? 0 : -1;
            mbar_expect_tx(bar, (pg < 0 ? 0u : tx_pop) + (pn >= 0 ? tx_pop : 0u));
            if (pg >= 0) tma_load_4d(base + 5 * POPB, tm_f, x0, y0 - 1, pg, 5, bar);
            if (pn >= 0) tma_load_4d(base + 6 * POPB, tm_f, x0, y0 - 1, pn, 6, bar);
          } else {
            const int pn = RG ? resolve(p + 1, A.n3, p3) : pg;
            const bool tab = pg >= 0 && p >= z0 && p < z1;
            mbar_expect_tx(bar, (pg >= 0 ? 6 * tx_pop : 0u) + (pn >= 0 ? tx_pop : 0u) +
                                    (tab ? (unsigned)(BY * T_SLOTS * RS) : 0u));
#pragma unroll 1
            for (int i = 0; i < 7; ++i) {
              const int pi = i == 6 ? pn : pg;
              if (pi >= 0) tma_load_4d(base + i * POPB, tm_f, x0, y0 - 1 - xi1_of(i), pi, i, bar);
            }
            if (tab) tma_load_3d(sbase + TAB + s * TABB, tm_t, 0, y0, pg, bar);
          }
          issued = p;
          if (++s == NB) { s = 0; ++use; }
        }
        next_it = (int)atomicAdd(claim, 1u);  // read by every thread after the item's last barrier
        for (int p = max(z0 - 2, issued - NB + 1); p <= issued; ++p) {
          const int k = p - (z0 - 2);
          wait_bar(full_at(k % NB), (unsigned)((k / NB) & 1));
        }
      }
    } else {  // -------------------------------------------------------------------- consumers
      const int q1 = y0 - 1 + w;
      const bool interior = w >= 1 && w <= BY;
      const bool rowin = q1 >= 0 && q1 < A.n1;
      const bool owner = interior && rowin;
      const int c0 = lane * NPT, q2 = x0 + c0;
      const int n2 = A.n2;
      auto wall = [&](int b) -> R { return b == LBW_BC_BOUNCE ? A.damping : R(-1); };
      auto ld1 = [&](unsigned off) -> R { return Store<S>::ld_smem(reinterpret_cast<const S*>(smem_raw + off)); };
      auto ldv = [&](unsigned off, R (&o)[NPT]) { VecN<S, NPT>::ld(reinterpret_cast<const S*>(smem_raw + off), o); };
      auto ldr = [&](unsigned off) -> R { return *reinterpret_cast<const R*>(smem_raw + off); };

      const unsigned own = (unsigned)((w * RW + G + c0) * ES);
      unsigned o1 = POPB + own, o2 = 2 * POPB + own;
      R m1 = R(1), m2 = R(1);
      if (rowin && q1 == 0) {
        const int b = A.bc[0];
        if (b == LBW_BC_FREE) o1 = POPB + own + RW * ES;
        else { o1 = 2 * POPB + own - RW * ES; m1 = wall(b); }
      }
      if (rowin && q1 == A.n1 - 1) {
        const int b = A.bc[1];
        if (b == LBW_BC_FREE) o2 = 2 * POPB + own - RW * ES;
        else { o2 = POPB + own + RW * ES; m2 = wall(b); }
      }
      const unsigned o3e = 3 * POPB + own - ES, o4e = 4 * POPB + own + NPT * ES;
      const bool f5_own = A.bc[4] == LBW_BC_FREE, f6_own = A.bc[5] == LBW_BC_FREE;
      const unsigned f5_face = (f5_own ? 5 : 6) * POPB, f6_face = (f6_own ? 6 : 5) * POPB;
      const R m5_face = A.bc[4] == LBW_BC_FREE ? R(1) : wall(A.bc[4]);
      const R m6_face = A.bc[5] == LBW_BC_FREE ? R(1) : wall(A.bc[5]);

      // halo column node of a halo warp: warp 0 lane l -> (y0 + l, x0 - 1), warp BY + 1 ->
      // (y0 + l, x0 + BX), lanes l < BY; both live inside the staged rows (ghost columns)
      const bool hwarp = !interior;
      const int hl = lane < BY ? lane : BY - 1;
      const int hq1 = y0 + hl;
      const bool hcol = hwarp && lane < BY;
      const bool hin = hq1 >= 0 && hq1 < A.n1;
      unsigned h0, h1, h2, h3, h4;
      R hm1 = R(1), hm2 = R(1);
      {
        const int hw = hl + 1, hc = (w == 0) ? G - 1 : G + BX;  // staged column of the node
        auto hat = [&](int pop, int row, int col) { return (unsigned)(pop * POPB + (row * RW + col) * ES); };
        h0 = hat(0, hw, hc);
        h1 = hat(1, hw, hc);
        h2 = hat(2, hw, hc);
        h3 = hat(3, hw, hc - 1);
        h4 = hat(4, hw, hc + 1);
        if (hq1 == 0) {
          const int b = A.bc[0];
          if (b == LBW_BC_FREE) h1 = hat(1, hw + 1, hc);
          else { h1 = hat(2, hw - 1, hc); hm1 = wall(b); }
        }
        if (hq1 == A.n1 - 1) {
          const int b = A.bc[1];
          if (b == LBW_BC_FREE) h2 = hat(2, hw - 1, hc);
          else { h2 = hat(1, hw + 1, hc); hm2 = wall(b); }
        }
      }
      const unsigned hrho = (unsigned)(((hl + 1) * PW + ((w == 0) ? C0 - 1 : C0 + BX)) * RS);
      const unsigned myrho = (unsigned)((w * PW + C0 + c0) * RS);

      bool has_probe = false;
      if (owner && t_sample < (unsigned long long)A.cap)
        for (int s = 0; s < probe_cnt; ++s) has_probe |= A.probe_q[3 * probe_list[s]] == q1;

      R fA[7][NPT], fB[7][NPT], rA[NPT], rB[NPT], rC[NPT];
      // storage of this lane's nodes (padded rows) and their ghost copies near the wrap
      const long long row_stride = (long long)A.n1 * A.pitch;
      S* const dst_z0 = A.fout + ((long long)z0 * A.n1 + (owner ? q1 : 0)) * A.pitch + G + q2;
      const int nvalid = q2 + 1 < n2 ? 2 : (q2 < n2 ? 1 : 0);
      const int gh0 = q2 < G ? n2 : (q2 >= n2 - G ? -n2 : 0);          // column shift of the
      const int gh1 = q2 + 1 < G ? n2 : (q2 + 1 >= n2 - G ? -n2 : 0);  // ghost copy, 0: none

      auto stepA = [&](int u, R (&f)[7][NPT], R (&rr)[NPT], int slm, int sl0, int slp, int rbu,
                       bool wr) {
        const bool zlo = !p3 && u == 0, zhi = !p3 && u == A.n3 - 1;
        const bool zghost = !p3 && (u < 0 || u >= A.n3);
        const unsigned S0 = SL + sl0 * SLOTB, SM = SL + slm * SLOTB;
        unsigned B5, B6;
        if constexpr (RG) {  // slot sl0: pops 0-5 of u, pop 6 of u + 1; slm: pop 6 of u
          B5 = zlo ? (f5_own ? S0 + 5 * POPB : SM + 6 * POPB) : SM + 5 * POPB;
          B6 = zhi ? (f6_own ? SM + 6 * POPB : S0 + 5 * POPB) : S0 + 6 * POPB;
        } else {
          B5 = zlo ? S0 + f5_face : SM + 5 * POPB;
          B6 = zhi ? S0 + f6_face : SL + slp * SLOTB + 6 * POPB;
        }
        const R m5 = zlo ? m5_face : R(1), m6 = zhi ? m6_face : R(1);
        R t3[NPT], t4[NPT];
        ldv(S0 + own, f[0]);
        ldv(S0 + o1, f[1]);
        ldv(S0 + o2, f[2]);
        ldv(S0 + 3 * POPB + own, t3);
        ldv(S0 + 4 * POPB + own, t4);
        ldv(B5 + own, f[5]);
        ldv(B6 + own, f[6]);
        f[3][0] = ld1(S0 + o3e);
        f[3][1] = t3[0];
        f[4][0] = t4[1];
        f[4][1] = ld1(S0 + o4e);
        const bool ghost = zghost || !rowin;
        if constexpr (sizeof(R) == 4) {
          float2 F[7];
#pragma unroll
          for (int i = 0; i < 7; ++i) F[i] = f2(f[i][0], f[i][1]);
          F[1] = mul2(bc2(m1), F[1]);
          F[2] = mul2(bc2(m2), F[2]);
          F[5] = mul2(bc2(m5), F[5]);
          F[6] = mul2(bc2(m6), F[6]);
          f[1][0] = F[1].x; f[1][1] = F[1].y;
          f[2][0] = F[2].x; f[2][1] = F[2].y;
          f[5][0] = F[5].x; f[5][1] = F[5].y;
          f[6][0] = F[6].x; f[6][1] = F[6].y;
          float2 sum;
          if constexpr (SC)
            sum = fma2(bc2(A.w[0]), F[0],
                       mul2(bc2(A.w[1]), add2(add2(add2(F[1], F[2]), add2(F[3], F[4])), add2(F[5], F[6]))));
          else
            sum = add2(add2(add2(F[0], F[1]), add2(F[2], F[3])), add2(add2(F[4], F[5]), F[6]));
          rr[0] = ghost ? R(0) : sum.x;
          rr[1] = ghost ? R(0) : sum.y;
        } else {
#pragma unroll
          for (int k = 0; k < NPT; ++k) {
            f[1][k] *= m1; f[2][k] *= m2; f[5][k] *= m5; f[6][k] *= m6;
            const R sum = ((f[0][k] + f[1][k]) + (f[2][k] + f[3][k])) + ((f[4][k] + f[5][k]) + f[6][k]);
            rr[k] = ghost ? R(0) : sum;
          }
        }
        if (wr) {
          const unsigned pl = RHO + rbu * (PS * RS);
          VecN<R, NPT>::st(reinterpret_cast<R*>(smem_raw + pl + myrho), rr);
          if (hwarp) {
            R g[7];
            g[0] = ld1(S0 + h0);
            g[1] = hm1 * ld1(S0 + h1);
            g[2] = hm2 * ld1(S0 + h2);
            g[3] = ld1(S0 + h3);
            g[4] = ld1(S0 + h4);
            g[5] = m5 * ld1(B5 + h0);  // h0 addresses population 0: B5 / B6 add their own
            g[6] = m6 * ld1(B6 + h0);
            const R h = SC ? A.w[0] * g[0] + A.w[1] * (((g[1] + g[2]) + (g[3] + g[4])) + (g[5] + g[6]))
                           : ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + g[6]);
            if (hcol) *reinterpret_cast<R*>(smem_raw + pl + hrho) = (hin && !zghost) ? h : R(0);
          }
        }
      };

      auto stepB = [&](int zc, R (&fc)[7][NPT], const R (&rp)[NPT], const R (&rc)[NPT],
                       const R (&rn)[NPT], int slz, int rbz) {
        const unsigned cur = RHO + rbz * (PS * RS) + myrho;
        R ru[NPT], rd[NPT];
        VecN<R, NPT>::ld(reinterpret_cast<const R*>(smem_raw + cur + PW * RS), ru);
        VecN<R, NPT>::ld(reinterpret_cast<const R*>(smem_raw + cur - PW * RS), rd);
        const R rl[NPT] = {ldr(cur - RS), rc[0]};
        const R rrt[NPT] = {rc[1], ldr(cur + NPT * RS)};
        const unsigned T = TAB + slz * TABB + (w - 1) * (T_SLOTS * RS);
        R c[T_SLOTS];
#pragma unroll
        for (int k = 0; k < T_SLOTS; k += 4) {
          if (RS == 4) {
            const float4 v = *reinterpret_cast<const float4*>(smem_raw + T + k * RS);
            c[k] = v.x; c[k + 1] = v.y; c[k + 2] = v.z; c[k + 3] = v.w;
          } else {
            const double2 v0 = *reinterpret_cast<const double2*>(smem_raw + T + k * RS);
            const double2 v1 = *reinterpret_cast<const double2*>(smem_raw + T + (k + 2) * RS);
            c[k] = v0.x; c[k + 1] = v0.y; c[k + 2] = v1.x; c[k + 3] = v1.y;
          }
        }
        if constexpr (sizeof(R) == 4) {
          const float2 A1P = bc2(-c[T_A1P]), A1M = bc2(c[T_A1M]), C13P = bc2(-c[T_C13P]),
                       C13M = bc2(c[T_C13M]), S1 = bc2(-c[T_S1]), B13P = bc2(-c[T_B13P]),
                       B13M = bc2(c[T_B13M]), C33P = bc2(-c[T_C33P]), C33M = bc2(c[T_C33M]),
                       S3 = bc2(-c[T_S3]), H22 = bc2(c[T_H22]), MG1 = bc2(c[T_MG1]),
                       MG3 = bc2(c[T_MG3]), CS2 = bc2(A.cs2), W0 = bc2(A.two_w0),
                       HALF = bc2(SC ? 1.f / A.cs2 : 0.5f), MHALF = bc2(SC ? -1.f / A.cs2 : -0.5f);
          const float2 rho = f2(rc[0], rc[1]);
          const float2 u = f2(ru[0], ru[1]), d = f2(rd[0], rd[1]);
          const float2 n = f2(rn[0], rn[1]), p = f2(rp[0], rp[1]);
          const float2 nD1 = fma2(S1, rho, fma2(C13M, p, fma2(C13P, n, fma2(A1M, d, mul2(A1P, u)))));
          const float2 nD3 = fma2(S3, rho, fma2(C33M, p, fma2(C33P, n, fma2(B13M, d, mul2(B13P, u)))));
          const float2 D2 = mul2(H22, sub2(f2(rrt[0], rrt[1]), f2(rl[0], rl[1])));
          float2 F[7];
#pragma unroll
          for (int i = 0; i < 7; ++i) F[i] = f2(fc[i][0], fc[i][1]);
          const float2 j1 = fma2(HALF, fma2(MG1, rho, nD1), sub2(F[1], F[2]));
          const float2 j2 = fma2(MHALF, D2, sub2(F[3], F[4]));
          const float2 j3 = fma2(HALF, fma2(MG3, rho, nD3), sub2(F[5], F[6]));
          const float2 e = SC ? add2(rho, rho) : mul2(CS2, rho);
          float2 o[7];
          o[0] = SC ? sub2(e, F[0]) : sub2(mul2(W0, rho), F[0]);
          o[1] = sub2(add2(e, j1), F[1]);
          o[2] = sub2(sub2(e, j1), F[2]);
          o[3] = sub2(add2(e, j2), F[3]);
          o[4] = sub2(sub2(e, j2), F[4]);
          o[5] = sub2(add2(e, j3), F[5]);
          o[6] = sub2(sub2(e, j3), F[6]);
#pragma unroll
          for (int i = 0; i < 7; ++i) {
            fc[i][0] = o[i].x;
            fc[i][1] = o[i].y;
          }
        } else {
#pragma unroll
          for (int k = 0; k < NPT; ++k) {
            const R rho = rc[k];
            const R D1 = c[T_A1P] * ru[k] - c[T_A1M] * rd[k] + c[T_C13P] * rn[k] - c[T_C13M] * rp[k] +
                         c[T_S1] * rho;
            const R D3 = c[T_B13P] * ru[k] - c[T_B13M] * rd[k] + c[T_C33P] * rn[k] - c[T_C33M] * rp[k] +
                         c[T_S3] * rho;
            const R D2 = c[T_H22] * (rrt[k] - rl[k]);
            const R j1 = (fc[1][k] - fc[2][k]) + R(0.5) * (c[T_MG1] * rho - D1);
            const R j2 = (fc[3][k] - fc[4][k]) - R(0.5) * D2;
            const R j3 = (fc[5][k] - fc[6][k]) + R(0.5) * (c[T_MG3] * rho - D3);
            const R e = A.cs2 * rho;
            fc[0][k] = A.two_w0 * rho - fc[0][k];
            fc[1][k] = e + j1 - fc[1][k];
            fc[2][k] = e - j1 - fc[2][k];
            fc[3][k] = e + j2 - fc[3][k];
            fc[4][k] = e - j2 - fc[4][k];
            fc[5][k] = e + j3 - fc[5][k];
            fc[6][k] = e - j3 - fc[6][k];
          }
        }
        S* dst = dst_z0 + (long long)(zc - z0) * row_stride;
#pragma unroll
        for (int i = 0; i < 7; ++i) {
          if (nvalid == 2) VecN<S, NPT>::st(dst, fc[i]);
          else if (nvalid == 1) Store<S>::st(dst, fc[i][0]);
          if (gh0 != 0 && nvalid >= 1) Store<S>::st(dst + gh0, fc[i][0]);
          if (gh1 != 0 && nvalid == 2) Store<S>::st(dst + 1 + gh1, fc[i][1]);
          dst += A.ps;
        }
        if (has_probe) {
          for (int s = 0; s < probe_cnt; ++s) {
            const int k = probe_list[s];
            const int dq = A.probe_q[3 * k + 1] - q2;
            if (A.probe_q[3 * k] == q1 && dq >= 0 && dq < NPT && A.probe_q[3 * k + 2] == zc)
              A.series[(long long)k * A.cap + t_sample] = (double)(dq == 0 ? rc[0] : rc[1]) * (double)c[T_INVSG];
          }
        }
      };

      constexpr int AHEAD = RG ? 0 : 1;
      bool ok = wait_bar(full_at(0), 0) && wait_bar(full_at(1), 0) && (RG || wait_bar(full_at(2), 0));
      if (ok && owner) stepA(z0 - 1, fB, rA, 0, 1, 2, 2, false);
      if (lane == 0) mbar_arrive(empty_at(0));
      ok = ok && wait_bar(full_at(2 + AHEAD), 0);
      if (ok) stepA(z0, fA, rB, 1, 2, 3, 0, true);
      if (lane == 0) mbar_arrive(empty_at(1));
      ok = !named_sync_or(1, NCW * 32, !ok || abort_flag);
      int sz = 2, s1 = 3, s2 = 4, uw = 0, rbz = 0, rb1 = 1;
      auto advance = [&]() {
        rbz = rb1;
        rb1 = rb1 == 2 ? 0 : rb1 + 1;
        sz = s1;
        s1 = s2;
        s2 = s2 == NB - 1 ? 0 : s2 + 1;
        if ((RG ? s1 : s2) == 0) ++uw;
      };
      auto iter = [&](int zz, R (&fc)[7][NPT], R (&fn)[7][NPT], const R (&rp)[NPT],
                      const R (&rc)[NPT], R (&rn)[NPT], bool collide) {
        const bool in = wait_bar(full_at(RG ? s1 : s2), (unsigned)(uw & 1));
        if (in) stepA(zz + 1, fn, rn, sz, s1, s2, rb1, true);
        const bool go = !named_sync_or(1, NCW * 32, !in || abort_flag);
        if (go && collide) stepB(zz, fc, rp, rc, rn, sz, rbz);
        if (lane == 0) mbar_arrive(empty_at(sz));
        advance();
        return go;
      };
      int z = z0;
      if (!owner) {
        for (; ok && z < z1; ++z) ok = iter(z, fA, fB, rA, rB, rC, false);
      } else {
        for (; ok && z + 1 < z1; z += 2) {
          ok = iter(z, fA, fB, rA, rB, rC, true);
          if (!ok) break;
          ok = iter(z + 1, fB, fA, rB, rC, rA, true);
#pragma unroll
          for (int k = 0; k < NPT; ++k) {
            const R t = rA[k];
            rA[k] = rC[k];
            rB[k] = t;
          }
        }
        if (ok && z < z1) ok = iter(z, fA, fB, rA, rB, rC, true);
      }
    }
    __syncthreads();  // item done: the producer has drained, the next item re-uses everything
    if (abort_flag) break;
    it = next_it;
  }
  finish_step(counters, nprobe, cap, gridDim.x);
}

// ---------------------------------------------------------------- full-row ensemble --------
//
// When every member's row fits a tile, a tile spans whole rows: ROWS = BY_m + 2 staged rows
// of the member's n2 data columns, with the tile's nodes laid out row-major over the consumer
// lanes (two q2-adjacent nodes per lane; with an odd n2 the last pair of a row carries one
// phantom node, computed and discarded).  The periodic q2 wrap then lies inside the tile: the
// pulls across it and the q2 gradient read the other end of the same staged row, so no ghost
// column is read or written, one tensor copy stages a population (ROWS x n2 rounded up to 16
// bytes, the box of the member's own tensor map), and no lane is left idle by a ragged last
// q2 tile.  The tile height follows the member (narrow rows give tall tiles).  The staging
// pipeline, slot regrouping, faces and collision are those of batch_tma_kernel.  32- and
// 64-bit storage.
constexpr int kRowWarps = 9;                   // consumer warps
constexpr int kRowNodes = kRowWarps * 32 * 2;  // nodes of a tile plane
constexpr int kRowCap = 648;                   // staged elements of a population plane
constexpr int kRowMaxBY = 16;                  // tile rows at most (coefficient slots)
constexpr int kRowMinBY = 3;                   // fewer would put a halo row on a q1 face

// Staged rows of a member's full-row tile (BY_m + 2), 0 when the member cannot use one.
inline int row_tile_rows(int n2, size_t es) {
  const int v = (int)(16 / es), n2w = n2 + (n2 & 1), bw = (n2 + v - 1) / v * v;
  if (bw > 256) return 0;
  const int rows = std::min(std::min(kRowNodes / n2w, kRowCap / bw), kRowMaxBY + 2);
  return rows - 2 >= kRowMinBY ? rows : 0;
}

template <typename S>
struct BatchRowLayout {
  using R = typename Store<S>::R;
  static constexpr int POPB = ((kRowCap * (int)sizeof(S)) + 127) / 128 * 128;
  static constexpr int SLOTB = 7 * POPB;
  static constexpr int TABB = ((kRowMaxBY * T_SLOTS * (int)sizeof(R)) + 127) / 128 * 128;
  static constexpr int RHOB = ((3 * kRowNodes * (int)sizeof(R)) + 127) / 128 * 128;
};

template <typename S>
constexpr size_t batch_row_smem() {
  using L = BatchRowLayout<S>;
  return 128 + 128 + 5 * (size_t)L::SLOTB + L::RHOB + 5 * (size_t)L::TABB;
}

// items: (member, BY_m, first interior row y0 (may be -1), z0)
template <typename S>
__global__ void __launch_bounds__(32 * (kRowWarps + 1), sizeof(S) == 4 ? 2 : 1) batch_row_kernel(
    const StepArgs<S>* __restrict__ members, const CUtensorMap* __restrict__ maps, int src,
    const int4* __restrict__ items, int n_items, int lz, unsigned long long* counters, int nprobe,
    long long cap) {
  using R = typename Store<S>::R;
  using L = BatchRowLayout<S>;
  static_assert(sizeof(S) >= 4, "the full-row tile regroups slots: 32- and 64-bit storage");
  constexpr int NPT = 2, NB = 5, NCW = kRowWarps;
  constexpr int ES = (int)sizeof(S), RS = (int)sizeof(R), V = 16 / ES;
  constexpr int POPB = L::POPB, SLOTB = L::SLOTB, TABB = L::TABB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) StepArgs<S> A;
  __shared__ int probe_list[kMaxProbes];
  __shared__ int probe_cnt;
  __shared__ int abort_flag;
  __shared__ int next_it;
  __shared__ unsigned long long t_sample;

  const int lane = threadIdx.x, w = threadIdx.y, tid = w * 32 + lane, nthr = 32 * (NCW + 1);
  // items are claimed as in batch_tma_kernel (the producer claims the next one once it has
  // issued the current item's last copies)
  unsigned* const claim = reinterpret_cast<unsigned*>(&counters[2]) + 1;
  const unsigned sbase = smem_u32(smem_raw);
  const unsigned OFF = (128u - (sbase & 127u)) & 127u;
  const unsigned SL = OFF + 128, RHO = SL + NB * SLOTB, TAB = RHO + L::RHOB;
  auto full_at = [&](int k) { return sbase + OFF + 8u * k; };
  auto empty_at = [&](int k) { return sbase + OFF + 8u * (NB + k); };
  if (tid == 0) {
    abort_flag = 0;
    t_sample = counters[1];
    next_it = (int)atomicAdd(claim, 1u);
  }
  __syncthreads();

  bool fresh = true;
  for (int it = next_it; it < n_items;) {
    const int4 item = items[it];
    {
      const unsigned* from = reinterpret_cast<const unsigned*>(members + item.x);
      unsigned* to = reinterpret_cast<unsigned*>(&A);
      for (int k = tid; k < (int)(sizeof(StepArgs<S>) / 4); k += nthr) to[k] = from[k];
    }
    if (tid == 0) {
      for (int k = 0; k < NB; ++k) {
        if (!fresh) {
          mbar_inval(full_at(k));
          mbar_inval(empty_at(k));
        }
        mbar_init_count(full_at(k), 1);
        mbar_init_count(empty_at(k), NCW);
      }
      asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
      probe_cnt = 0;
    }
    fresh = false;
    __syncthreads();  // every thread has read next_it for this item
    const int BYm = item.y, y0 = item.z, z0 = item.w, ROWS = BYm + 2;
    const int z1 = min(z0 + lz, A.n3);
    const bool p3 = A.bc[4] == LBW_BC_PERIODIC;
    const int n2 = A.n2, n2w = n2 + (n2 & 1), BW = (n2 + V - 1) / V * V;
    if (tid < A.nprobe) {
      const int pq1 = A.probe_q[3 * tid], pq3 = A.probe_q[3 * tid + 2];
      if (pq1 >= y0 && pq1 < y0 + BYm && pq3 >= z0 && pq3 < z1) probe_list[atomicAdd(&probe_cnt, 1)] = tid;
    }
    __syncthreads();
    const CUtensorMap* tm_f = maps + 3 * item.x + src;
    const CUtensorMap* tm_t = maps + 3 * item.x + 2;

    auto wait_bar = [&](unsigned bar, unsigned parity) -> bool {
      long long n = 0;
      while (!mbar_try_wait(bar, parity)) {
        if (++n > kWaitLimit) {
          abort_flag = 1;
          A.counters[3] = 1;
          return false;
        }
      }
      return true;
    };

    if (w == NCW) {  // ---------------------------------------------------------- producer
      if (lane == 0) {
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        const unsigned tx_pop = (unsigned)(ROWS * BW * ES);
        const int xg = A.col0;  // the first data column of a stored row
        int s = 0, use = 0, issued = z0 - 3;
        for (int p = z0 - 2; p <= z1; ++p) {
          if (use > 0 && !wait_bar(empty_at(s), (unsigned)((use - 1) & 1))) break;
          const unsigned bar = full_at(s);
          const unsigned base = sbase + SL + s * SLOTB;
          const int pg = resolve(p, A.n3, p3);
          if (p == z0 - 2) {
            // population 5 of this plane; population 6 of the q3 = 0 face when z0 - 1 is it
            const int pn = (!p3 && z0 == 1) ? 0 : -1;
            mbar_expect_tx(bar, (pg < 0 ? 0u : tx_pop) + (pn >= 0 ? tx_pop : 0u));
            if (pg >= 0) tma_load_4d(base + 5 * POPB, tm_f, xg, y0 - 1, pg, 5, bar);
            if (pn >= 0) tma_load_4d(base + 6 * POPB, tm_f, xg, y0 - 1, pn, 6, bar);
          } else {
            const int pn = resolve(p + 1, A.n3, p3);
            const bool tab = pg >= 0 && p >= z0 && p < z1;
            mbar_expect_tx(bar, (pg >= 0 ? 6 * tx_pop : 0u) + (pn >= 0 ? tx_pop : 0u) +
                                    (tab ? (unsigned)(BYm * T_SLOTS * RS) : 0u));
#pragma unroll 1
            for (int i = 0; i < 7; ++i) {
              const int pi = i == 6 ? pn : pg;
              if (pi >= 0) tma_load_4d(base + i * POPB, tm_f, xg, y0 - 1 - xi1_of(i), pi, i, bar);
            }
            if (tab) tma_load_3d(sbase + TAB + s * TABB, tm_t, 0, y0, pg, bar);
          }
          issued = p;
          if (++s == NB) { s = 0; ++use; }
        }
        next_it = (int)atomicAdd(claim, 1u);  // read by every thread after the item's last barrier
        for (int p = max(z0 - 2, issued - NB + 1); p <= issued; ++p) {
          const int k = p - (z0 - 2);
          wait_bar(full_at(k % NB), (unsigned)((k / NB) & 1));
        }
      }
    } else {  // -------------------------------------------------------------------- consumers
      // this lane's node pair: flattened index 2 (w * 32 + lane) over ROWS x n2w, row-major
      const int nd = 2 * (w * 32 + lane);
      const bool active = nd < ROWS * n2w;
      const int row = active ? nd / n2w : ROWS - 1, col = active ? nd % n2w : 0;
      const int q1 = y0 - 1 + row;
      const bool interior = row >= 1 && row <= BYm;
      const bool rowin = q1 >= 0 && q1 < A.n1;
      const bool owner = active && interior && rowin;
      const bool odd_last = col + 1 == n2;  // the pair's second node is a phantom (odd n2)
      auto wall = [&](int b) -> R { return b == LBW_BC_BOUNCE ? A.damping : R(-1); };
      auto ld1 = [&](unsigned off) -> R { return Store<S>::ld_smem(reinterpret_cast<const S*>(smem_raw + off)); };
      auto ldv = [&](unsigned off, R (&o)[NPT]) { VecN<S, NPT>::ld(reinterpret_cast<const S*>(smem_raw + off), o); };
      auto ldr = [&](unsigned off) -> R { return *reinterpret_cast<const R*>(smem_raw + off); };

      // staged offsets: populations 0, 3, 4, 5, 6 at (row, col); 1 / 2 at the pull or at the
      // q1-face rule (a face row reads the staged row next to it, never a halo row: tiles
      // have >= 3 interior rows and start at q1 = -1 where a halo row would sit on a face)
      const unsigned own = (unsigned)((row * BW + col) * ES);
      unsigned o1 = POPB + own, o2 = 2 * POPB + own;
      R m1 = R(1), m2 = R(1);
      if (rowin && q1 == 0) {
        const int b = A.bc[0];
        if (b == LBW_BC_FREE) o1 = POPB + own + BW * ES;
        else { o1 = 2 * POPB + own - BW * ES; m1 = wall(b); }
      }
      if (rowin && q1 == A.n1 - 1) {
        const int b = A.bc[1];
        if (b == LBW_BC_FREE) o2 = 2 * POPB + own - BW * ES;
        else { o2 = POPB + own + BW * ES; m2 = wall(b); }
      }
      // q2 neighbours across the periodic wrap, inside the same staged row: column cl left of
      // the pair, cr right of it, column 0 for the last node of an odd row
      const int cl = col == 0 ? n2 - 1 : col - 1;
      const int cr = col + 2 >= n2 ? col + 2 - n2 : col + 2;
      const unsigned o3e = (unsigned)(3 * POPB + (row * BW + cl) * ES);
      const unsigned o4e = (unsigned)(4 * POPB + (row * BW + cr) * ES);
      const unsigned o4w = (unsigned)(4 * POPB + row * BW * ES);
      const bool f5_own = A.bc[4] == LBW_BC_FREE, f6_own = A.bc[5] == LBW_BC_FREE;
      const R m5_face = A.bc[4] == LBW_BC_FREE ? R(1) : wall(A.bc[4]);
      const R m6_face = A.bc[5] == LBW_BC_FREE ? R(1) : wall(A.bc[5]);
      // rho planes: ROWS rows of n2w values (the phantom column included, never read)
      const unsigned myrho = (unsigned)((row * n2w + col) * RS);
      const unsigned lrho = (unsigned)((row * n2w + cl) * RS), rrho = (unsigned)((row * n2w + cr) * RS);
      const unsigned wrho = (unsigned)(row * n2w * RS);
      constexpr unsigned PLANE = (unsigned)(kRowNodes * RS);

      bool has_probe = false;
      if (owner && t_sample < (unsigned long long)A.cap)
        for (int s = 0; s < probe_cnt; ++s) has_probe |= A.probe_q[3 * probe_list[s]] == q1;

      R fA[7][NPT], fB[7][NPT], rA[NPT], rB[NPT], rC[NPT];
      const long long row_stride = (long long)A.n1 * A.pitch;
      S* const dst_z0 = A.fout + ((long long)z0 * A.n1 + (owner ? q1 : 0)) * A.pitch + A.col0 + col;

      // step A of pulled plane u (slot sl0: populations 0-5 of u and 6 of u + 1; slot slm:
      // population 5 of u - 1 and 6 of u), rho into rr and (wr) into rho plane rbu
      auto stepA = [&](int u, R (&f)[7][NPT], R (&rr)[NPT], int slm, int sl0, int rbu, bool wr) {
        const bool zlo = !p3 && u == 0, zhi = !p3 && u == A.n3 - 1;
        const bool zghost = !p3 && (u < 0 || u >= A.n3);
        const unsigned S0 = SL + sl0 * SLOTB, SM = SL + slm * SLOTB;
        const unsigned B5 = zlo ? (f5_own ? S0 + 5 * POPB : SM + 6 * POPB) : SM + 5 * POPB;
        const unsigned B6 = zhi ? (f6_own ? SM + 6 * POPB : S0 + 5 * POPB) : S0 + 6 * POPB;
        const R m5 = zlo ? m5_face : R(1), m6 = zhi ? m6_face : R(1);
        R t3[NPT], t4[NPT];
        ldv(S0 + own, f[0]);
        ldv(S0 + o1, f[1]);
        ldv(S0 + o2, f[2]);
        ldv(S0 + 3 * POPB + own, t3);
        ldv(S0 + 4 * POPB + own, t4);
        ldv(B5 + own, f[5]);
        ldv(B6 + own, f[6]);
        f[3][0] = ld1(S0 + o3e);
        f[3][1] = t3[0];
        f[4][0] = odd_last ? ld1(S0 + o4w) : t4[1];
        f[4][1] = ld1(S0 + o4e);
        const bool ghost = zghost || !rowin;
        if constexpr (sizeof(R) == 4) {
          float2 F[7];
#pragma unroll
          for (int i = 0; i < 7; ++i) F[i] = f2(f[i][0], f[i][1]);
          F[1] = mul2(bc2(m1), F[1]);
          F[2] = mul2(bc2(m2), F[2]);
          F[5] = mul2(bc2(m5), F[5]);
          F[6] = mul2(bc2(m6), F[6]);
          f[1][0] = F[1].x; f[1][1] = F[1].y;
          f[2][0] = F[2].x; f[2][1] = F[2].y;
          f[5][0] = F[5].x; f[5][1] = F[5].y;
          f[6][0] = F[6].x; f[6][1] = F[6].y;
          const float2 sum = add2(add2(add2(F[0], F[1]), add2(F[2], F[3])), add2(add2(F[4], F[5]), F[6]));
          rr[0] = ghost ? R(0) : sum.x;
          rr[1] = ghost ? R(0) : sum.y;
        } else {
#pragma unroll
          for (int k = 0; k < NPT; ++k) {
            f[1][k] *= m1; f[2][k] *= m2; f[5][k] *= m5; f[6][k] *= m6;
            const R sum = ((f[0][k] + f[1][k]) + (f[2][k] + f[3][k])) + ((f[4][k] + f[5][k]) + f[6][k]);
            rr[k] = ghost ? R(0) : sum;
          }
        }
        if (wr && active) VecN<R, NPT>::st(reinterpret_cast<R*>(smem_raw + RHO + rbu * PLANE + myrho), rr);
      };

      // step B: collide plane zc (populations fc, rho rp / rc / rn of planes zc - 1 / zc / zc + 1)
      auto stepB = [&](int zc, R (&fc)[7][NPT], const R (&rp)[NPT], const R (&rc)[NPT],
                       const R (&rn)[NPT], int slz, int rbz) {
        const unsigned pl = RHO + rbz * PLANE;
        R ru[NPT], rd[NPT];
        VecN<R, NPT>::ld(reinterpret_cast<const R*>(smem_raw + pl + myrho + n2w * RS), ru);
        VecN<R, NPT>::ld(reinterpret_cast<const R*>(smem_raw + pl + myrho - n2w * RS), rd);
        const R rl[NPT] = {ldr(pl + lrho), rc[0]};
        const R rrt[NPT] = {odd_last ? ldr(pl + wrho) : rc[1], ldr(pl + rrho)};
        const unsigned T = TAB + slz * TABB + (row - 1) * (T_SLOTS * RS);
        R c[T_SLOTS];
#pragma unroll
        for (int k = 0; k < T_SLOTS; k += 4) {
          if (RS == 4) {
            const float4 v = *reinterpret_cast<const float4*>(smem_raw + T + k * RS);
            c[k] = v.x; c[k + 1] = v.y; c[k + 2] = v.z; c[k + 3] = v.w;
          } else {
            const double2 v0 = *reinterpret_cast<const double2*>(smem_raw + T + k * RS);
            const double2 v1 = *reinterpret_cast<const double2*>(smem_raw + T + (k + 2) * RS);
            c[k] = v0.x; c[k + 1] = v0.y; c[k + 2] = v1.x; c[k + 3] = v1.y;
          }
        }
        if constexpr (sizeof(R) == 4) {
          const float2 A1P = bc2(-c[T_A1P]), A1M = bc2(c[T_A1M]), C13P = bc2(-c[T_C13P]),
                       C13M = bc2(c[T_C13M]), S1 = bc2(-c[T_S1]), B13P = bc2(-c[T_B13P]),
                       B13M = bc2(c[T_B13M]), C33P = bc2(-c[T_C33P]), C33M = bc2(c[T_C33M]),
                       S3 = bc2(-c[T_S3]), H22 = bc2(c[T_H22]), MG1 = bc2(c[T_MG1]),
                       MG3 = bc2(c[T_MG3]), CS2 = bc2(A.cs2), W0 = bc2(A.two_w0), HALF = bc2(0.5f),
                       MHALF = bc2(-0.5f);
          const float2 rho = f2(rc[0], rc[1]);
          const float2 u = f2(ru[0], ru[1]), d = f2(rd[0], rd[1]);
          const float2 n = f2(rn[0], rn[1]), p = f2(rp[0], rp[1]);
          const float2 nD1 = fma2(S1, rho, fma2(C13M, p, fma2(C13P, n, fma2(A1M, d, mul2(A1P, u)))));
          const float2 nD3 = fma2(S3, rho, fma2(C33M, p, fma2(C33P, n, fma2(B13M, d, mul2(B13P, u)))));
          const float2 D2 = mul2(H22, sub2(f2(rrt[0], rrt[1]), f2(rl[0], rl[1])));
          float2 F[7];
#pragma unroll
          for (int i = 0; i < 7; ++i) F[i] = f2(fc[i][0], fc[i][1]);
          const float2 j1 = fma2(HALF, fma2(MG1, rho, nD1), sub2(F[1], F[2]));
          const float2 j2 = fma2(MHALF, D2, sub2(F[3], F[4]));
          const float2 j3 = fma2(HALF, fma2(MG3, rho, nD3), sub2(F[5], F[6]));
          const float2 e = mul2(CS2, rho);
          float2 o[7];
          o[0] = sub2(mul2(W0, rho), F[0]);
          o[1] = sub2(add2(e, j1), F[1]);
          o[2] = sub2(sub2(e, j1), F[2]);
          o[3] = sub2(add2(e, j2), F[3]);
          o[4] = sub2(sub2(e, j2), F[4]);
          o[5] = sub2(add2(e, j3), F[5]);
          o[6] = sub2(sub2(e, j3), F[6]);
#pragma unroll
          for (int i = 0; i < 7; ++i) {
            fc[i][0] = o[i].x;
            fc[i][1] = o[i].y;
          }
        } else {
#pragma unroll
          for (int k = 0; k < NPT; ++k) {
            const R rho = rc[k];
            const R D1 = c[T_A1P] * ru[k] - c[T_A1M] * rd[k] + c[T_C13P] * rn[k] - c[T_C13M] * rp[k] +
                         c[T_S1] * rho;
            const R D3 = c[T_B13P] * ru[k] - c[T_B13M] * rd[k] + c[T_C33P] * rn[k] - c[T_C33M] * rp[k] +
                         c[T_S3] * rho;
            const R D2 = c[T_H22] * (rrt[k] - rl[k]);
            const R j1 = (fc[1][k] - fc[2][k]) + R(0.5) * (c[T_MG1] * rho - D1);
            const R j2 = (fc[3][k] - fc[4][k]) - R(0.5) * D2;
            const R j3 = (fc[5][k] - fc[6][k]) + R(0.5) * (c[T_MG3] * rho - D3);
            const R e = A.cs2 * rho;
            fc[0][k] = A.two_w0 * rho - fc[0][k];
            fc[1][k] = e + j1 - fc[1][k];
            fc[2][k] = e - j1 - fc[2][k];
            fc[3][k] = e + j2 - fc[3][k];
            fc[4][k] = e - j2 - fc[4][k];
            fc[5][k] = e + j3 - fc[5][k];
            fc[6][k] = e - j3 - fc[6][k];
          }
        }
        S* dst = dst_z0 + (long long)(zc - z0) * row_stride;
#pragma unroll
        for (int i = 0; i < 7; ++i) {
          if (odd_last) Store<S>::st(dst, fc[i][0]);
          else VecN<S, NPT>::st(dst, fc[i]);
          dst += A.ps;
        }
        if (has_probe) {
          for (int s = 0; s < probe_cnt; ++s) {
            const int k = probe_list[s];
            const int dq = A.probe_q[3 * k + 1] - col;
            if (A.probe_q[3 * k] == q1 && dq >= 0 && dq < NPT && col + dq < n2 && A.probe_q[3 * k + 2] == zc)
              A.series[(long long)k * A.cap + t_sample] = (double)(dq == 0 ? rc[0] : rc[1]) * (double)c[T_INVSG];
          }
        }
      };

      // every lane runs the same loop (halo, interior and idle lanes share warps); step B runs
      // on the lanes that own lattice nodes
      bool ok = wait_bar(full_at(0), 0) && wait_bar(full_at(1), 0);
      if (ok && owner) stepA(z0 - 1, fB, rA, 0, 1, 2, false);
      if (lane == 0) mbar_arrive(empty_at(0));
      ok = ok && wait_bar(full_at(2), 0);
      if (ok) stepA(z0, fA, rB, 1, 2, 0, true);
      if (lane == 0) mbar_arrive(empty_at(1));
      ok = !named_sync_or(1, NCW * 32, !ok || abort_flag);
      int sz = 2, s1 = 3, s2 = 4, uw = 0, rbz = 0, rb1 = 1;
      auto advance = [&]() {
        rbz = rb1;
        rb1 = rb1 == 2 ? 0 : rb1 + 1;
        sz = s1;
        s1 = s2;
        s2 = s2 == NB - 1 ? 0 : s2 + 1;
        if (s1 == 0) ++uw;
      };
      auto iter = [&](int zz, R (&fc)[7][NPT], R (&fn)[7][NPT], const R (&rp)[NPT],
                      const R (&rc)[NPT], R (&rn)[NPT]) {
        const bool in = wait_bar(full_at(s1), (unsigned)(uw & 1));
        if (in) stepA(zz + 1, fn, rn, sz, s1, rb1, true);
        const bool go = !named_sync_or(1, NCW * 32, !in || abort_flag);
        if (go && owner) stepB(zz, fc, rp, rc, rn, sz, rbz);
        if (lane == 0) mbar_arrive(empty_at(sz));
        advance();
        return go;
      };
      int z = z0;
      for (; ok && z + 1 < z1; z += 2) {
        ok = iter(z, fA, fB, rA, rB, rC);
        if (!ok) break;
        ok = iter(z + 1, fB, fA, rB, rC, rA);
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
          const R t = rA[k];
          rA[k] = rC[k];
          rB[k] = t;
        }
      }
      if (ok && z < z1) ok = iter(z, fA, fB, rA, rB, rC);
    }
    __syncthreads();  // item done: the producer has drained, the next item re-uses everything
    if (abort_flag) break;
    it = next_it;
  }
  finish_step(counters, nprobe, cap, gridDim.x);
}

// Ghost columns of padded rows from the data columns they copy (G on each side: ghost-left =
// the last G data columns, ghost-right = the first G), for a member's buffer f: the full-row
// kernel does not keep them, the 64-column kernel reads them.
template <typename S>
__global__ void ghost_fill_kernel(S* __restrict__ f, long long rows, int pitch, int n2, int G) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < rows * 2 * G;
       k += (long long)gridDim.x * blockDim.x) {
    S* row = f + (k / (2 * G)) * pitch;
    const int j = (int)(k % (2 * G));
    if (j < G) row[j] = row[n2 + j];
    else row[n2 + j] = row[j];
  }
}

struct Shape {
  int by = 8;    // tile rows (register-pipelined: CTA = 32 x by threads; TMA: 4 or 7, 0 = full rows)
  int lz = 32;   // planes per q3 segment
  int cps = 2;   // CTAs per SM of the persistent grid
};

}  // namespace
namespace {
// Largest |x| of each series over its samples [t0, t1): one CTA per series, series s at
// x + s * stride; NaN when a sample is not finite (so the host sees the instability).
__global__ void series_peak_kernel(const double* __restrict__ x, long long stride, long long t0, long long t1,
                                   double* __restrict__ out) {
  __shared__ double red[32];
  const double* p = x + (long long)blockIdx.x * stride;
  double m = 0.0;
  bool bad = false;
  for (long long t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
    const double v = fabs(p[t]);
    bad |= !isfinite(v);
    m = fmax(m, v);
  }
  for (int o = 16; o > 0; o >>= 1) {
    m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    bad |= __shfl_down_sync(0xffffffffu, (int)bad, o) != 0;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = bad ? NAN : m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    bool anybad = false;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      anybad |= !isfinite(red[k]);
      r = fmax(r, red[k]);
    }
    out[blockIdx.x] = anybad ? NAN : r;
  }
}
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
  bool tma = false;              // padded members on the TMA-staged kernel
  bool rowk = false;             // ... and every member fits a full-row tile (shape.by == 0)
  void* maps = nullptr;          // device: per member tensor maps (buffer 0, buffer 1, table)
  // harmonic sources of all members (offsets from the buffer base), applied after each step
  int nsrc = 0, src_kind = 0;
  double src_amp = 0.0;
  void* src = nullptr;
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
  a.pitch = g.pitch ? g.pitch : g.d.n[1];
  a.col0 = g.col0;
  a.ps = pop_stride(&g);
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

// The TMA-staged kernel for (storage type, tile rows): f(kernel, dynamic shared bytes).
template <typename S, typename F>
auto batch_tma_dispatch(int by, F&& f) {
  return by == 7 ? f(batch_tma_kernel<S, 7>, batch_tma_smem<S, 7>())
                 : f(batch_tma_kernel<S, 4>, batch_tma_smem<S, 4>());
}

template <typename F>
auto prec_dispatch(int prec, F&& f) {
  switch (prec) {
    case LBW_F64: return f(double());
    case LBW_F32: return f(float());
    case LBW_F16S: return f(__half());
    default: return f(__nv_bfloat16());
  }
}

// resident CTAs per SM of the full-row kernel (0 when it cannot run)
int row_cps(int prec) {
  auto occ = [](auto kern, size_t smem) {
    int per = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 32 * (kRowWarps + 1), smem) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return per;
  };
  if (prec == LBW_F32) return occ(batch_row_kernel<float>, batch_row_smem<float>());
  if (prec == LBW_F64) return occ(batch_row_kernel<double>, batch_row_smem<double>());
  return 0;
}

// resident CTAs per SM of the TMA-staged kernel with `by` rows (0 when it cannot run; by = 0:
// the full-row kernel)
int tma_cps(int prec, int by) {
  if (by == 0) return row_cps(prec);
  return prec_dispatch(prec, [&](auto tag) {
    using S = decltype(tag);
    return batch_tma_dispatch<S>(by, [&](auto kern, size_t smem) {
      int per = 0;
      if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 32 * (by + 3), smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
      }
      return per;
    });
  });
}

// Ghost columns of a padded member row and the row length (elements) for storage size es:
// G | n2 data | G, rounded up to 16 bytes.  The last tile's box may reach past the row end;
// those columns are outside the tensor and arrive as zeros without touching memory.
// (Rows rounded up to 128-byte lines instead read 21% more from DRAM, measured on the
// 32-trumpet ensemble, probably because power-of-two row strides crowd the same L2 sets.)
int ghost_cols(size_t es) { return (int)(16 / es); }
int padded_pitch(int n2, size_t es) {
  const int v = (int)(16 / es);
  return (n2 + 2 * ghost_cols(es) + v - 1) / v * v;
}

// Tensor maps of every member for tile rows `by`: 4-D views (stored column, q1, q3,
// population) of both buffers with (64 + 2 G) x (by + 2) boxes, 3-D view of the table.
lbw_status build_batch_maps(lbw_batch* b, int by) {
  const size_t es = es_of(b->prec);
  const int rprec = b->prec == LBW_F64 ? LBW_F64 : LBW_F32;
  const size_t rs = rs_of(b->prec);
  std::vector<CUtensorMap> h(3 * (size_t)b->n);
  for (int m = 0; m < b->n; ++m) {
    const Grid& g = b->views[m];
    const uint64_t P = (uint64_t)g.pitch, n1 = (uint64_t)g.d.n[0], n3 = (uint64_t)g.d.n[2];
    const uint64_t dims[4] = {P, n1, n3, 7};
    const uint64_t strides[3] = {P * es, P * n1 * es, P * n1 * n3 * es};
    // by = 0: full-row tiles, the member's n2 data columns (rounded up to 16 bytes) x its rows
    const int v = (int)(16 / es), rows = by == 0 ? row_tile_rows(g.d.n[1], es) : by + 2;
    if (rows < 3) return fail(LBW_EINVAL, "ensemble member " + std::to_string(m) + " does not fit a full-row tile");
    const uint32_t box[4] = {(uint32_t)(by == 0 ? (g.d.n[1] + v - 1) / v * v : kTmaBatchBX + 2 * g.col0),
                             (uint32_t)rows, 1, 1};
    for (int k = 0; k < 2; ++k)
      if (!encode_tiled_map(&h[3 * m + k], b->prec, 4, g.f[k], dims, strides, box))
        return fail(LBW_ECUDA, "tensor map of ensemble member " + std::to_string(m));
    const uint64_t tdims[3] = {(uint64_t)T_SLOTS, n1, n3};
    const uint64_t tstr[2] = {(uint64_t)T_SLOTS * rs, (uint64_t)T_SLOTS * rs * n1};
    const uint32_t tbox[3] = {(uint32_t)T_SLOTS, (uint32_t)(rows - 2), 1};
    if (!encode_tiled_map(&h[3 * m + 2], rprec, 3, g.table, tdims, tstr, tbox))
      return fail(LBW_ECUDA, "table tensor map of ensemble member " + std::to_string(m));
  }
  if (!b->maps) LBW_CUDA(cudaMallocAsync(&b->maps, sizeof(CUtensorMap) * h.size(), b->stream));
  LBW_CUDA(cudaMemcpyAsync(b->maps, h.data(), sizeof(CUtensorMap) * h.size(), cudaMemcpyHostToDevice,
                           b->stream));
  LBW_CUDA(cudaStreamSynchronize(b->stream));  // h is released on return
  return LBW_OK;
}

// work list for the current shape: items of each member in (q3 segment, q1 tile, q2 tile)
// order, so consecutive CTAs hold spatial neighbours.  TMA tiles are 64 columns wide and
// start at q1 = -1 when (n1 - 1) is a multiple of the tile rows (no halo row on a face).
// Full-row tiles (shape.by == 0) have the member's own row count: items (member, rows, y0, z0).
lbw_status build_items(lbw_batch* b) {
  std::vector<int4> items;
  for (int m = 0; m < b->n; ++m) {
    const lbw_grid_desc& d = b->views[m].d;
    if (b->tma && b->shape.by == 0) {
      const int by = row_tile_rows(d.n[1], b->views[m].elem) - 2;
      if (by < kRowMinBY) return fail(LBW_EINVAL, "ensemble member does not fit a full-row tile");
      const int y_start = (d.n[0] - 1) % by == 0 ? -1 : 0;
      for (int z0 = 0; z0 < d.n[2]; z0 += b->shape.lz)
        for (int y0 = y_start; y0 < d.n[0]; y0 += by) items.push_back(make_int4(m, by, y0, z0));
      continue;
    }
    const int bx = b->tma ? kTmaBatchBX : kBatchBX;
    const int y_start = (b->tma && (d.n[0] - 1) % b->shape.by == 0) ? -1 : 0;
    for (int z0 = 0; z0 < d.n[2]; z0 += b->shape.lz)
      for (int y0 = y_start; y0 < d.n[0]; y0 += b->shape.by)
        for (int x0 = 0; x0 < d.n[1]; x0 += bx) items.push_back(make_int4(m, x0, y0, z0));
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
  if (b->tma) {
    st = build_batch_maps(b, b->shape.by);
    if (st != LBW_OK) return st;
  }
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
  if constexpr (sizeof(S) >= 4) {
    if (b->tma && b->shape.by == 0) {
      batch_row_kernel<S><<<b->blocks, dim3(32, kRowWarps + 1), batch_row_smem<S>(), b->stream>>>(
          reinterpret_cast<const StepArgs<S>*>(b->members[src]), reinterpret_cast<const CUtensorMap*>(b->maps),
          src, b->items, b->n_items, b->shape.lz, b->counters, b->nprobe, b->cap);
      return cudaGetLastError();
    }
  }
  if (b->tma) {
    return batch_tma_dispatch<S>(b->shape.by, [&](auto kern, size_t smem) {
      kern<<<b->blocks, dim3(32, b->shape.by + 3), smem, b->stream>>>(
          reinterpret_cast<const StepArgs<S>*>(b->members[src]), reinterpret_cast<const CUtensorMap*>(b->maps),
          src, b->items, b->n_items, b->shape.lz, b->counters, b->nprobe, b->cap);
      return cudaGetLastError();
    });
  }
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

cudaError_t batch_sources(lbw_batch* b, int buf) {
  if (b->nsrc == 0) return cudaSuccess;
  return launch_sources(b->prec, b->f[buf], static_cast<const SourceEntry*>(b->src), b->nsrc, b->src_kind,
                        b->src_amp, b->counters, b->stream);
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
    if (e == cudaSuccess) e = batch_sources(b, 1 - src);
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
    LBW_CUDA(batch_sources(b, 1 - b->cur));
    b->cur = 1 - b->cur;
    --left;
  }
  b->steps += n_steps;
  return LBW_OK;
}

// Samples recorded (counters[1]) and the wait flag (counters[3]) of the ensemble.
lbw_status batch_counters(lbw_batch* b, unsigned long long* recorded) {
  unsigned long long c[3] = {0, 0, 0};
  LBW_CUDA(cudaMemcpyAsync(c, b->counters + 1, sizeof(c), cudaMemcpyDeviceToHost, b->stream));
  LBW_CUDA(cudaStreamSynchronize(b->stream));
  if (recorded) *recorded = c[0];
  if (c[2]) return fail(LBW_ETIMEOUT, "a time step's bounded wait for staged data ran out; the state is "
                                      "undefined until lbw_batch_init");
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
  s << "n" << b->n << "-p" << b->prec << (b->tma ? "-tma" : "-reg") << "-nodes" << b->total_nodes << "-h"
    << std::hex << h;
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
  // the TMA-staged kernel takes ensembles whose members all wrap in q2 (ghost columns), have
  // walls in q1, at least 2 G columns and 32-bit population offsets
  {
    const size_t es = es_of(b->prec);
    b->tma = tma_cps(b->prec, 7) > 0 && tma_cps(b->prec, 4) > 0;
    for (int m = 0; m < n && b->tma; ++m) {
      const lbw_grid_desc& d = descs[m];
      const long long ps = (long long)d.n[0] * d.n[2] * padded_pitch(d.n[1], es);
      if (d.bc[2] != LBW_BC_PERIODIC || d.bc[3] != LBW_BC_PERIODIC || d.bc[0] == LBW_BC_PERIODIC ||
          d.n[1] < 2 * ghost_cols(es) || 7 * ps >= (1LL << 31) || d.n[0] < 2)
        b->tma = false;
    }
    // full-row tiles: 32- or 64-bit storage and every member's row in a tile
    b->rowk = b->tma && row_cps(b->prec) > 0;
    for (int m = 0; m < n && b->rowk; ++m)
      if (row_tile_rows(descs[m].n[1], es) == 0) b->rowk = false;
  }
  std::vector<double> tab_all;
  size_t ftot = 0;
  for (int m = 0; m < n; ++m) {
    lbw_grid_desc d = descs[m];
    if (d.prec != b->prec) return cleanup(fail(LBW_EINVAL, "all members must share the storage precision"));
    lbw_status st = validate_desc(d);
    if (st != LBW_OK) return cleanup(fail(st, "member " + std::to_string(m) + ": " + lbw_last_error()));
    if (d.equilibrium != LBW_EQ_CURVILINEAR)
      return cleanup(fail(LBW_EINVAL, "member " + std::to_string(m) + ": ensembles run the paper's equilibrium"));
    if (d.geom_mode == LBW_GEOM_ANALYTIC)
      return cleanup(fail(LBW_EINVAL, "member " + std::to_string(m) +
                                          ": ensembles take the geometry from the table (geom_mode ANALYTIC is "
                                          "for single lattices)"));
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
    if (b->tma) {
      g.pitch = padded_pitch(d.n[1], g.elem);
      g.col0 = ghost_cols(g.elem);
    }
    b->foff[m] = ftot;
    // 256-byte aligned member slices
    const size_t align = 256 / g.elem;
    ftot += (7 * (size_t)pop_stride(&g) + align - 1) / align * align;
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
  if (b->rowk) {  // full-row tiles where every member fits one (the autotuner's pick on trumpets)
    b->shape.by = 0;
    b->shape.lz = 16;
    b->shape.cps = std::min(2, row_cps(b->prec));
  } else if (b->tma) {
    b->shape.by = 7;
    b->shape.cps = std::min(2, tma_cps(b->prec, 7));
  } else {
    b->shape.cps = std::min(2, b->prec == LBW_F32 ? max_cps<float>() : 2);
  }
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
  if (b->maps) cudaFreeAsync(b->maps, b->stream);
  if (b->src) cudaFreeAsync(b->src, b->stream);
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

lbw_status lbw_batch_source(lbw_batch* b, const int32_t* host_q, int32_t per_member, int32_t kind,
                            double amp, const double* host_omega) {
  if (!b) return fail(LBW_EINVAL, "batch is NULL");
  if (per_member < 0 || (long long)per_member * b->n > (1 << 24)) return fail(LBW_EINVAL, "too many source nodes");
  if (per_member > 0 && (!host_q || !host_omega)) return fail(LBW_EINVAL, "sources need nodes and frequencies");
  if (kind != 0 && kind != 1) return fail(LBW_EINVAL, "kind must be 0 (P) or 1 (J'_z)");
  if (!std::isfinite(amp)) return fail(LBW_EINVAL, "amp must be finite");
  const bool p_all = b->tma;  // padded members carry ghost copies of nodes near the wrap
  std::vector<SourceEntry> h;
  h.reserve((size_t)b->n * per_member);
  for (int m = 0; m < b->n && per_member > 0; ++m) {
    const Grid& g = b->views[m];
    if (!std::isfinite(host_omega[m])) return fail(LBW_EINVAL, "omega must be finite");
    const int pitch = g.pitch ? g.pitch : g.d.n[1], col0 = g.col0, n2 = g.d.n[1];
    for (int k = 0; k < per_member; ++k) {
      const int32_t* q = host_q + ((size_t)m * per_member + k) * 3;
      if (q[0] < 0 || q[0] >= g.d.n[0] || q[1] < 0 || q[1] >= n2 || q[2] < 0 || q[2] >= g.d.n[2])
        return fail(LBW_EINVAL, "source node outside its member's lattice");
      SourceEntry e{};
      e.off = (long long)b->foff[m] + ((long long)q[2] * g.d.n[0] + q[0]) * pitch + col0 + q[1];
      e.ps = pop_stride(&g);
      e.ghost = 0;
      if (p_all && col0 > 0 && g.d.bc[2] == LBW_BC_PERIODIC) {
        if (q[1] < col0) e.ghost = n2;
        else if (q[1] >= n2 - col0) e.ghost = -n2;
      }
      e.sg = lattice_sqrtg(g.d, q[0], q[2]);
      e.omega = host_omega[m];
      e.cs2 = g.d.cs2;
      h.push_back(e);
    }
  }
  drop_graphs(b);  // captured chains carry the source list
  if (b->src) { cudaFreeAsync(b->src, b->stream); b->src = nullptr; }
  b->nsrc = 0;
  if (!h.empty()) {
    LBW_CUDA(cudaMallocAsync(&b->src, sizeof(SourceEntry) * h.size(), b->stream));
    LBW_CUDA(cudaMemcpyAsync(b->src, h.data(), sizeof(SourceEntry) * h.size(), cudaMemcpyHostToDevice, b->stream));
    LBW_CUDA(cudaStreamSynchronize(b->stream));
    b->nsrc = (int)h.size();
    b->src_kind = kind;
    b->src_amp = amp;
  }
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
  lbw_status st = batch_counters(b, &rec);
  if (st != LBW_OK) return st;
  *n_steps = (int64_t)rec;
  if (b->nprobe == 0 || rec == 0) return LBW_OK;
  if (!host_out) return fail(LBW_EINVAL, "host_out is NULL");
  LBW_CUDA(cudaMemcpyAsync(host_out, b->series, sizeof(double) * b->n * b->nprobe * b->cap,
                           cudaMemcpyDeviceToHost, b->stream));
  LBW_CUDA(cudaStreamSynchronize(b->stream));
  return LBW_OK;
}

lbw_status lbw_batch_probe_peak(lbw_batch* b, int64_t tail, double* host_out) {
  if (!b || !host_out) return fail(LBW_EINVAL, "NULL argument");
  if (tail < 1) return fail(LBW_EINVAL, "tail must be >= 1");
  if (b->nprobe == 0) return fail(LBW_ESTATE, "no probes registered");
  unsigned long long rec = 0;
  lbw_status st = batch_counters(b, &rec);
  if (st != LBW_OK) return st;
  if ((unsigned long long)tail > rec) return fail(LBW_EINVAL, "tail longer than the recorded series");
  const int nser = b->n * b->nprobe;
  double* d = nullptr;
  LBW_CUDA(cudaMallocAsync(&d, sizeof(double) * nser, b->stream));
  series_peak_kernel<<<nser, 256, 0, b->stream>>>(b->series, (long long)b->cap, (long long)(rec - tail),
                                                  (long long)rec, d);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, d, sizeof(double) * nser, cudaMemcpyDeviceToHost, b->stream);
  cudaFreeAsync(d, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "probe_peak");
  for (int k = 0; k < nser; ++k)
    if (!std::isfinite(host_out[k])) return fail(LBW_EUNSTABLE, "probe series holds a non-finite value (unstable run)");
  return LBW_OK;
}

lbw_status lbw_batch_spectrum(lbw_batch* b, int32_t k, double* host_freq, double* host_amp,
                              int32_t* host_n_found) {
  if (!b || !host_freq || !host_amp || !host_n_found) return fail(LBW_EINVAL, "NULL argument");
  if (k < 1 || k > 64) return fail(LBW_EINVAL, "1 <= k <= 64");
  if (b->nprobe == 0) return fail(LBW_ESTATE, "no probes registered");
  unsigned long long rec = 0;
  lbw_status st0 = batch_counters(b, &rec);
  if (st0 != LBW_OK) return st0;
  if (rec < 4) return fail(LBW_ESTATE, "fewer than 4 recorded samples");
  for (int m = 0; m < b->n; ++m) {
    lbw_status st = spectrum_device(b->series + (size_t)m * b->nprobe * b->cap, (int64_t)rec, b->nprobe,
                                    (int32_t)b->cap, true, k, b->stream, host_freq + (size_t)m * k,
                                    host_amp + (size_t)m * k, host_n_found + m);
    if (st != LBW_OK) return st;
  }
  return LBW_OK;
}

lbw_status lbw_batch_spectrum_lowest(lbw_batch* b, int32_t k, double rel_power, double* host_freq,
                                     double* host_amp, int32_t* host_n_found) {
  if (!b || !host_freq || !host_amp || !host_n_found) return fail(LBW_EINVAL, "NULL argument");
  if (k < 1 || k > 64) return fail(LBW_EINVAL, "1 <= k <= 64");
  if (!(rel_power > 0.0 && rel_power <= 1.0)) return fail(LBW_EINVAL, "0 < rel_power <= 1");
  if (b->nprobe == 0) return fail(LBW_ESTATE, "no probes registered");
  unsigned long long rec = 0;
  lbw_status st0 = batch_counters(b, &rec);
  if (st0 != LBW_OK) return st0;
  if (rec < 4) return fail(LBW_ESTATE, "fewer than 4 recorded samples");
  for (int m = 0; m < b->n; ++m) {
    lbw_status st = spectrum_device(b->series + (size_t)m * b->nprobe * b->cap, (int64_t)rec, b->nprobe,
                                    (int32_t)b->cap, true, k, b->stream, host_freq + (size_t)m * k,
                                    host_amp + (size_t)m * k, host_n_found + m, true, rel_power);
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
  return batch_counters(b, nullptr);
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
    // register-pipelined kernel: rows {4, 8, 16} x CTAs per SM {1, 2, 4}; TMA-staged kernel:
    // rows {4, 7} and full-row tiles (by = 0, where every member fits one) x CTAs per SM
    // {1, 2}; both x segment planes {16, 32, 64}
    std::vector<int> bys = b->tma ? std::vector<int>{4, 7} : std::vector<int>{4, 8, 16};
    if (b->rowk) bys.push_back(0);
    std::vector<int> cpss = b->tma ? std::vector<int>{1, 2} : std::vector<int>{1, 2, 4};
    const int lzs[3] = {16, 32, 64};
    cudaEvent_t e0, e1;
    LBW_CUDA(cudaEventCreate(&e0));
    LBW_CUDA(cudaEventCreate(&e1));
    for (int by : bys)
      for (int lz : lzs)
        for (int cps : cpss) {
          const int cps_max = b->tma ? tma_cps(b->prec, by) : (b->prec == LBW_F32 ? max_cps<float>() : 2);
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

lbw_status lbw_batch_set_shape(lbw_batch* b, int32_t tile_rows, int32_t seg_planes, int32_t ctas_per_sm) {
  if (!b) return fail(LBW_EINVAL, "batch is NULL");
  const bool ok_rows = b->tma ? (tile_rows == 4 || tile_rows == 7 || (tile_rows == 0 && b->rowk))
                              : (tile_rows == 4 || tile_rows == 8 || tile_rows == 16);
  if (!ok_rows) return fail(LBW_EINVAL, "tile_rows is not a shape this ensemble's kernel offers");
  if (seg_planes < 1) return fail(LBW_EINVAL, "seg_planes must be >= 1");
  const int cps_max = b->tma ? tma_cps(b->prec, tile_rows) : (b->prec == LBW_F32 ? max_cps<float>() : 2);
  if (ctas_per_sm < 1 || ctas_per_sm > std::max(1, cps_max) || (b->tma && cps_max == 0))
    return fail(LBW_EINVAL, "ctas_per_sm must be in [1, what the kernel keeps resident]");
  const Shape old = b->shape;
  b->shape = Shape{tile_rows, seg_planes, ctas_per_sm};
  lbw_status st = refresh(b);
  if (st != LBW_OK) {
    b->shape = old;
    refresh(b);
    return st;
  }
  if (b->tma && old.by == 0 && tile_rows != 0) {  // the 64-column kernel reads ghost columns
    for (int m = 0; m < b->n; ++m) {
      const Grid& g = b->views[m];
      const long long rows = 7LL * g.d.n[0] * g.d.n[2];
      const int blocks = (int)std::min<long long>((rows * 2 * g.col0 + 255) / 256, 1024);
      prec_dispatch(b->prec, [&](auto tag) {
        using S = decltype(tag);
        ghost_fill_kernel<S><<<blocks, 256, 0, b->stream>>>(reinterpret_cast<S*>(g.f[b->cur]), rows, g.pitch,
                                                             g.d.n[1], g.col0);
        return 0;
      });
    }
    LBW_CUDA(cudaGetLastError());
  }
  LBW_CUDA(cudaStreamSynchronize(b->stream));
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
