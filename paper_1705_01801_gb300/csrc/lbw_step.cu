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
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "lbw_internal.h"
#include "lbw_march.cuh"
#include "lbw_tma.cuh"

namespace lbw {
namespace {

using namespace dev;

template <typename S>
__global__ void __launch_bounds__(512) step_kernel(const StepArgs<S> a) {
  using R = typename Store<S>::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int probe_list[kMaxProbes];
  __shared__ int probe_cnt;
  __shared__ unsigned long long t_sample;
  const int x0 = blockIdx.x * blockDim.x, y0 = blockIdx.y * blockDim.y;
  const int z0 = blockIdx.z * a.lz, z1 = min(z0 + a.lz, a.n3);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    probe_cnt = 0;
    t_sample = a.counters[1];
  }
  __syncthreads();
  scan_probes(a, x0, y0, z0, z1, probe_list, &probe_cnt);
  march_tile(a, x0, y0, z0, z1, reinterpret_cast<R*>(smem_raw), probe_list, probe_cnt, t_sample);
  finish_step(a.counters, a.nprobe, a.cap, a.nblocks);
}

// ---------------------------------------------------------------- TMA tile kernel -------
//
// Raw post-collision planes are staged in shared memory by the Tensor Memory Accelerator and
// consumed plane by plane along q3 (see step_tma_kernel).

__host__ __device__ constexpr int round128(int b) { return (b + 127) / 128 * 128; }

// 16-bit storage (whole-plane slots): ONE box per plane holds all seven populations over the
// BY + 4 rows that the pulls of the BY + 2 consumer rows read (lattice rows y0 - 2 .. y0 + BY
// + 1, the same rows for every population) and BX + 2V columns (the tile and its 16-byte halo
// columns, V = 8 elements); a tile on a periodic q2 edge takes its wrapped halo columns (all
// seven populations) in one more V-column box per wrapped side.  At 16-bit byte rates the
// per-population boxes (22 copies per plane) bound the kernel by the copies issued, not by
// the bytes (measured: FP16 trumpet 136 -> 165 GLUPS with the plane box).
template <int BY, int BX>
struct PlaneLayout {
  static constexpr int V = 8, WX = BX + 2 * V, PR = BY + 4;
  __host__ __device__ static constexpr int row_bytes() { return WX * 2; }
  __host__ __device__ static constexpr int pop_bytes() { return PR * WX * 2; }
  __host__ __device__ static constexpr int plane_bytes() { return 7 * pop_bytes(); }
  __host__ __device__ static constexpr int hpop_bytes() { return PR * 16; }
  __host__ __device__ static constexpr int halo_bytes() { return 7 * hpop_bytes(); }
  __host__ __device__ static constexpr int slot_bytes() {
    return round128(plane_bytes()) + 2 * round128(halo_bytes());
  }
};

template <int BY, int BX>
struct TmaLayout {
  // per population: main box (BY+2) x BX, left / right halo boxes (BY+2) x V, 128-B aligned
  template <typename S>
  __host__ __device__ static constexpr int main_bytes() { return (BY + 2) * BX * (int)sizeof(S); }
  __host__ __device__ static constexpr int halo_bytes() { return (((BY + 2) * 16) + 127) / 128 * 128; }
  template <typename S>
  __host__ __device__ static constexpr int pop_bytes() { return main_bytes<S>() + 2 * halo_bytes(); }
  template <typename S>
  __host__ __device__ static constexpr int slot_bytes() { return 7 * pop_bytes<S>(); }
};

// Fused step, TMA-staged.  CTA = BY + 2 consumer warps + 1 producer warp.  Consumer warp w
// stands for lattice row q1 = y0 - 1 + w (warps 0 and BY + 1 are halo rows; they also compute
// rho of the tile's two halo columns), lane l owns the NPT nodes q2 = x0 + NPT l ...
// (BX = 32 NPT columns).  The producer's lane 0 stages raw plane p into slot
// (p - z0 + 2) mod NB: with 32- or 64-bit storage, per population a main box of BX columns x
// BY + 2 rows (rows shifted by the population's xi1, so the pull of tile row w reads staged
// row w of every population) and two V-column halo boxes at x0 - V and x0 + BX (periodic
// wraps in the coordinates); with 16-bit storage the plane box of PlaneLayout (the pull of
// tile row w reads staged row w + 1 - xi1) and, on a periodic q2 edge, the wrapped halo box;
// then the tile's coefficient rows.  With 32- or 64-bit storage a slot holds populations 0-5 of its plane
// and population 6 of the next one (the population that streams down into the plane), so
// pulling plane u needs the slots of planes u and u - 1 only and the last slot is plane z1;
// with 16-bit storage a slot holds its whole plane, pulling plane u needs planes u - 1 .. u + 1
// and the last slot is plane z1 + 1.  The plane below the segment carries population 5 only
// (16-bit: its plane box without halo boxes).
// The slot's full mbarrier completes on the bytes, and a slot is refilled only after every
// consumer warp has released it (empty mbarrier), so the producer runs up to NB - 2 (16-bit:
// NB - 3) planes ahead.  Per plane u the consumers read step B's shared inputs of plane
// u - 1, pull the populations of plane u and write its rho into one of three rotating rho
// planes (step A), collide plane u - 1 (step B, rows of the tile only), release the slot of
// plane u - 1 and synchronise among themselves (named barrier).  Face rules are reads of other staged values (bounce-back /
// anti-bounce-back: the node's own opposite population; free: the node's own population),
// chosen by selects so the per-plane code has no data-dependent branches; the launch shape
// keeps halo rows off the q1 faces and halo columns off the q2 faces.  Shared memory is
// addressed by 32-bit offsets from the dynamic array.  Every mbarrier wait is bounded: on
// expiry counters[3] is raised and the CTA stops.
template <typename S, int BY, int NPT, bool ANA>
__global__ void __launch_bounds__(32 * (BY + 3)) step_tma_kernel(
    const StepArgs<S> a, const __grid_constant__ CUtensorMap tm_main,
    const __grid_constant__ CUtensorMap tm_halo, const __grid_constant__ CUtensorMap tm_tab) {
  using R = typename Store<S>::R;
  constexpr int BX = 32 * NPT, NB = 5, ROWS = BY + 2, NCW = ROWS;  // consumer warps
  // 32- and 64-bit storage: population 6 of plane p + 1 rides in plane p's slot (measured:
  // FP32 trumpet 6% and cylinder 2% faster); 16-bit storage keeps whole planes per slot (the
  // regrouped form measured 7-8% slower there)
  constexpr bool RG = sizeof(S) >= 4;
  constexpr int ES = (int)sizeof(S), RS = (int)sizeof(R);
  constexpr int V = 16 / ES;
  using PL = PlaneLayout<BY, BX>;
  static_assert(RG || !ANA, "the analytic geometry is built for 32- and 64-bit storage only");
  // 32/64-bit: per population a main box and two halo boxes; 16-bit: the plane box layout
  constexpr int MB = TmaLayout<BY, BX>::template main_bytes<S>();
  constexpr int HB = TmaLayout<BY, BX>::halo_bytes();
  constexpr int POPB = RG ? TmaLayout<BY, BX>::template pop_bytes<S>() : PL::pop_bytes();
  constexpr int SLOTB = RG ? TmaLayout<BY, BX>::template slot_bytes<S>() : PL::slot_bytes();
  constexpr int WXB = PL::row_bytes(), HPOP = PL::hpop_bytes();
  constexpr int HL = round128(PL::plane_bytes()), HR = HL + round128(PL::halo_bytes());
  // rho row: nodes at NPT .. NPT + BX - 1 (vector aligned), halo columns at NPT - 1, NPT + BX
  constexpr int C0 = NPT, PW = BX + 2 * NPT;
  constexpr int PS = ROWS * PW;
  constexpr int TABB = ((BY * T_SLOTS * RS) + 127) / 128 * 128;
  constexpr int RHOB = ((3 * PS * RS) + 127) / 128 * 128;  // three rho planes
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int probe_list[kMaxProbes];
  __shared__ int probe_cnt;
  __shared__ int abort_flag;
  __shared__ int stall_req;
  __shared__ unsigned long long t_sample;

  // Programmatic dependent launch: this grid may be scheduled while the previous step drains;
  // nothing of the previous step's output (populations, counters) is touched before its
  // completion, and the next step may be scheduled from here on.
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
  const int lane = threadIdx.x, w = threadIdx.y, tid = w * 32 + lane;
  const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY, z0 = blockIdx.z * a.lz;
  const int z1 = min(z0 + a.lz, a.n3);
  const bool p2 = a.bc[2] == LBW_BC_PERIODIC, p3 = a.bc[4] == LBW_BC_PERIODIC;
  // 16-bit: the tile's halo column on this side wraps around the periodic q2 axis
  const bool wrapL = p2 && x0 == 0, wrapR = p2 && x0 + BX == a.n2;

  // byte offsets from smem_raw (TMA destinations want 128-byte alignment): barriers, NB
  // slots, three rho planes, NB coefficient blocks
  const unsigned sbase = smem_u32(smem_raw);
  const unsigned OFF = (128u - (sbase & 127u)) & 127u;
  const unsigned SL = OFF + 128, RHO = SL + NB * SLOTB, TAB = RHO + RHOB, MSC = TAB + NB * TABB;
  auto full_at = [&](int k) { return sbase + OFF + 8u * k; };
  auto empty_at = [&](int k) { return sbase + OFF + 8u * (NB + k); };
  // a barrier that no thread or copy ever completes: the target of the injected timeout
  const unsigned stall_bar = sbase + OFF + 8u * (2 * NB);

  if (tid == 0) {
    for (int k = 0; k < NB; ++k) {
      mbar_init_count(full_at(k), ANA ? 2 : 1);  // analytic: the producer's rows arrive too
      mbar_init_count(empty_at(k), NCW);
    }
    mbar_init_count(stall_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    probe_cnt = 0;
    abort_flag = 0;
    stall_req = a.counters[4] != 0ull;  // failure injection (lbw_inject_wait_timeout)
    t_sample = a.counters[1];
  }
  __syncthreads();
  if (tid < a.nprobe) {
    const int pq1 = a.probe_q[3 * tid], pq2 = a.probe_q[3 * tid + 1], pq3 = a.probe_q[3 * tid + 2];
    if (pq1 >= y0 && pq1 < y0 + BY && pq2 >= x0 && pq2 < x0 + BX && pq3 >= z0 && pq3 < z1)
      probe_list[atomicAdd(&probe_cnt, 1)] = tid;
  }
  __syncthreads();

  // Bounded wait for a phase of `bar`: after `limit` tries the CTA's abort flag and the step's
  // timeout flag (counters[3]) are raised.  With `watch`, the wait also gives up (raising
  // nothing) as soon as another warp of the CTA has raised the abort flag.
  auto wait_bar = [&](unsigned bar, unsigned parity, long long limit = kWaitLimit,
                      bool watch = false) -> bool {
    long long it = 0;
    while (!mbar_try_wait(bar, parity)) {
      if (watch && *reinterpret_cast<volatile int*>(&abort_flag)) return false;
      if (++it > limit) {
        abort_flag = 1;
        a.counters[3] = 1;
        return false;
      }
    }
    return true;
  };

  if (w == ROWS) {  // ------------------------------------------------------------ producer
    if constexpr (!ANA) {
      // Lane 0 waits for free slots and issues the copies (this loop as written measured 4%
      // faster on the torus than one shared with the analytic mode below).
      if (lane == 0) {
        int xl = x0 - V, xr = x0 + BX;
        const bool hl = xl >= 0 || p2, hr = xr < a.n2 || p2;
        if (xl < 0) xl += a.n2;
        if (xr >= a.n2) xr -= a.n2;
        const unsigned tx_pop = (unsigned)(ROWS * BX * ES) + (hl ? ROWS * 16u : 0u) + (hr ? ROWS * 16u : 0u);
        int s = 0, use = 0;
        int issued = z0 - 3;
        for (int p = z0 - 2; p <= z1 + (RG ? 0 : 1); ++p) {
          if (use > 0 && !wait_bar(empty_at(s), (unsigned)((use - 1) & 1), kWaitLimit, true)) break;
          const unsigned bar = full_at(s);
          const unsigned base = sbase + SL + s * SLOTB;
          const int pg = resolve(p, a.n3, p3);
          if constexpr (!RG) {  // whole planes: the plane box and the wrapped halo boxes
            if (pg < 0) {
              mbar_expect_tx(bar, 0);
            } else {
              // plane z0 - 2 only gives population 5 at the tile's own columns
              const bool tab = p >= z0 && p < z1, side = p != z0 - 2;
              mbar_expect_tx(bar, (unsigned)PL::plane_bytes() +
                                      (side && wrapL ? (unsigned)PL::halo_bytes() : 0u) +
                                      (side && wrapR ? (unsigned)PL::halo_bytes() : 0u) +
                                      (tab ? (unsigned)(BY * T_SLOTS * RS) : 0u));
              tma_load_4d(base, &tm_main, x0 - PL::V, y0 - 2, pg, 0, bar);
              if (side && wrapL) tma_load_4d(base + HL, &tm_halo, a.n2 - PL::V, y0 - 2, pg, 0, bar);
              if (side && wrapR) tma_load_4d(base + HR, &tm_halo, 0, y0 - 2, pg, 0, bar);
              if (tab) tma_load_3d(sbase + TAB + s * TABB, &tm_tab, 0, y0, pg, bar);
            }
          } else if (p == z0 - 2) {
            // only population 5 of this plane streams into the segment; when the first pulled
            // plane z0 - 1 is the q3 = 0 face of a wall, its reflected population 6 rides here
            const int pn = (!p3 && z0 == 1) ? 0 : -1;
            mbar_expect_tx(bar, (pg < 0 ? 0u : (unsigned)(ROWS * BX * ES)) + (pn >= 0 ? tx_pop : 0u));
            if (pg >= 0) tma_load_4d(base + 5 * POPB, &tm_main, x0, y0 - 1, pg, 5, bar);
            if (pn >= 0) {
              tma_load_4d(base + 6 * POPB, &tm_main, x0, y0 - 1, pn, 6, bar);
              if (hl) tma_load_4d(base + 6 * POPB + MB, &tm_halo, xl, y0 - 1, pn, 6, bar);
              if (hr) tma_load_4d(base + 6 * POPB + MB + HB, &tm_halo, xr, y0 - 1, pn, 6, bar);
            }
          } else {
            // populations 0-5 of plane p and population 6 of plane p + 1 (which streams into
            // plane p), so a pulled plane needs its own slot and the one before it only
            const int pn = resolve(p + 1, a.n3, p3);
            const bool tab = pg >= 0 && p >= z0 && p < z1;
            mbar_expect_tx(bar, (pg >= 0 ? 6 * tx_pop : 0u) + (pn >= 0 ? tx_pop : 0u) +
                                    (tab ? (unsigned)(BY * T_SLOTS * RS) : 0u));
#pragma unroll 1
            for (int i = 0; i < 7; ++i) {
              const int pi = i == 6 ? pn : pg;
              if (pi < 0) continue;
              const int row = y0 - 1 - xi1_of(i);
              tma_load_4d(base + i * POPB, &tm_main, x0, row, pi, i, bar);
              if (hl) tma_load_4d(base + i * POPB + MB, &tm_halo, xl, row, pi, i, bar);
              if (hr) tma_load_4d(base + i * POPB + MB + HB, &tm_halo, xr, row, pi, i, bar);
            }
            if (tab) tma_load_3d(sbase + TAB + s * TABB, &tm_tab, 0, y0, pg, bar);
          }
          issued = p;
          if (++s == NB) { s = 0; ++use; }
        }
        // drain: the last NB staged planes have landed before the CTA exits (bounded)
        for (int p = max(z0 - 2, issued - NB + 1); p <= issued; ++p) {
          const int k = p - (z0 - 2);
          wait_bar(full_at(k % NB), (unsigned)((k / NB) & 1));
        }
      }
    } else {
      // Analytic geometry: lane 0 waits for free slots and issues the population copies; the
      // other lanes follow it through the loop, and after each slot wait they write the
      // coefficient rows of a collided plane into the slot's table block, after which lane 0
      // adds the slot's second arrival.
      int xl = x0 - V, xr = x0 + BX;
      const bool hl = xl >= 0 || p2, hr = xr < a.n2 || p2;
      if (xl < 0) xl += a.n2;
      if (xr >= a.n2) xr -= a.n2;
      const unsigned tx_pop = (unsigned)(ROWS * BX * ES) + (hl ? ROWS * 16u : 0u) + (hr ? ROWS * 16u : 0u);
      int s = 0, use = 0;
      int issued = z0 - 3;
      for (int p = z0 - 2; p <= z1 + (RG ? 0 : 1); ++p) {
        int free_slot = 1;
        if (lane == 0 && use > 0) free_slot = wait_bar(empty_at(s), (unsigned)((use - 1) & 1), kWaitLimit, true);
        free_slot = __shfl_sync(0xffffffffu, free_slot, 0);
        __syncwarp();  // orders lane 0's acquire of the free slot before the others' row writes
        if (!free_slot) break;
        const unsigned bar = full_at(s);
        const unsigned base = sbase + SL + s * SLOTB;
        const int pg = resolve(p, a.n3, p3);
        bool tab = false;  // this plane is collided here: its coefficient rows ride in the slot
        if (p == z0 - 2) {
          // only population 5 of this plane streams into the segment; when the first pulled
          // plane z0 - 1 is the q3 = 0 face of a wall, its reflected population 6 rides here
          if (lane == 0) {
            const int pn = (!p3 && z0 == 1) ? 0 : -1;
            mbar_expect_tx(bar, (pg < 0 ? 0u : (unsigned)(ROWS * BX * ES)) + (pn >= 0 ? tx_pop : 0u));
            if (pg >= 0) tma_load_4d(base + 5 * POPB, &tm_main, x0, y0 - 1, pg, 5, bar);
            if (pn >= 0) {
              tma_load_4d(base + 6 * POPB, &tm_main, x0, y0 - 1, pn, 6, bar);
              if (hl) tma_load_4d(base + 6 * POPB + MB, &tm_halo, xl, y0 - 1, pn, 6, bar);
              if (hr) tma_load_4d(base + 6 * POPB + MB + HB, &tm_halo, xr, y0 - 1, pn, 6, bar);
            }
          }
        } else {
          // populations 0-5 of plane p and population 6 of plane p + 1 (which streams into
          // plane p), so a pulled plane needs its own slot and the one before it only
          tab = pg >= 0 && p >= z0 && p < z1;
          if (lane == 0) {
            const int pn = resolve(p + 1, a.n3, p3);
            mbar_expect_tx(bar, (pg >= 0 ? 6 * tx_pop : 0u) + (pn >= 0 ? tx_pop : 0u) + 0u);
#pragma unroll 1
            for (int i = 0; i < 7; ++i) {
              const int pi = i == 6 ? pn : pg;
              if (pi < 0) continue;
              const int row = y0 - 1 - xi1_of(i);
              tma_load_4d(base + i * POPB, &tm_main, x0, row, pi, i, bar);
              if (hl) tma_load_4d(base + i * POPB + MB, &tm_halo, xl, row, pi, i, bar);
              if (hr) tma_load_4d(base + i * POPB + MB + HB, &tm_halo, xr, row, pi, i, bar);
            }
          }
        }
        {
          if (tab) {
            // the metric at rows y0 - 1 .. y0 + BY of planes pg - 1, pg, pg + 1, one position per
            // lane (wrapped across a periodic q3 face, at the ghost position across any other),
            // then lanes 0 .. BY - 1 assemble the tile's rows from it
            MetricR<R>* msc = reinterpret_cast<MetricR<R>*>(smem_raw + MSC);
            for (int k = lane; k < 3 * ROWS; k += 32) {
              int q3n = pg + k / ROWS - 1;
              if (p3) q3n = q3n < 0 ? q3n + a.n3 : (q3n >= a.n3 ? q3n - a.n3 : q3n);
              msc[k] = metric_q(a.geo, y0 - 1 + k % ROWS, q3n);
            }
            __syncwarp();
            if (lane < BY) {
              R* rowp = reinterpret_cast<R*>(smem_raw + TAB + s * TABB) + lane * T_SLOTS;
              const MetricR<R> nb[4] = {msc[ROWS + lane], msc[ROWS + lane + 2], msc[lane + 1],
                                        msc[2 * ROWS + lane + 1]};
              table_row(a.geo, a.bc, a.n1, a.n3, y0 + lane, pg, msc[ROWS + lane + 1], nb, rowp);
            }
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(bar);  // the rows are written (second arrival of the phase)
        }
        issued = p;
        if (++s == NB) { s = 0; ++use; }
      }
      // drain: the last NB staged planes have landed before the CTA exits (bounded)
      if (lane == 0)
        for (int p = max(z0 - 2, issued - NB + 1); p <= issued; ++p) {
          const int k = p - (z0 - 2);
          wait_bar(full_at(k % NB), (unsigned)((k / NB) & 1));
        }
    }
  } else {  // ------------------------------------------------------------------- consumers
    const int q1 = y0 - 1 + w;
    const bool interior = w >= 1 && w <= BY;
    const bool rowin = q1 >= 0 && q1 < a.n1;  // a lattice row, not a ghost beyond a q1 face
    const bool owner = interior && rowin;
    const int c0 = lane * NPT;
    const int q2 = x0 + c0;
    const bool q2lo = !p2 && q2 == 0, q2hi = !p2 && q2 + NPT - 1 == a.n2 - 1;
    // 16-bit formats store h_i = f_i / w_i and the step works on h directly (rho = w0 h0 +
    // w1 (h1 + ... + h6), h* = 2 f^eq / w - h), so no per-population scaling; the face and
    // wall factors are the same for f and h (all moving populations share w1)
    constexpr bool SC = Store<S>::kScaled;
    const R sc0 = R(1), sc1 = R(1);
    auto wall = [&](int b) -> R { return b == LBW_BC_BOUNCE ? a.damping : R(-1); };
    auto ld1 = [&](unsigned off) -> R { return Store<S>::ld_smem(reinterpret_cast<const S*>(smem_raw + off)); };
    auto ldv = [&](unsigned off, R (&o)[NPT]) { VecN<S, NPT>::ld(reinterpret_cast<const S*>(smem_raw + off), o); };
    auto ldr = [&](unsigned off) -> R { return *reinterpret_cast<const R*>(smem_raw + off); };

    unsigned own, o1, o2, o3e, o4e;
    R m1 = sc1, m2 = sc1;
    if constexpr (RG) {
      // offsets within a slot of this lane's vectors: pops 0, 3, 4, 5, 6 at (w, c0); pops 1 / 2
      // at the pull or at the q1-face rule (the face rows read the staged rows next to them)
      own = (unsigned)(w * BX * ES + c0 * ES);
      o1 = POPB + own;
      o2 = 2 * POPB + own;
      if (rowin && q1 == 0) {
        const int b = a.bc[0];
        if (b == LBW_BC_FREE) o1 = POPB + own + BX * ES;
        else { o1 = 2 * POPB + own - BX * ES; m1 = sc1 * wall(b); }
      }
      if (rowin && q1 == a.n1 - 1) {
        const int b = a.bc[1];
        if (b == LBW_BC_FREE) o2 = 2 * POPB + own - BX * ES;
        else { o2 = POPB + own + BX * ES; m2 = sc1 * wall(b); }
      }
      // pop 3 of node c0 reads column c0 - 1 (left halo box for lane 0), pop 4 of node
      // c0 + NPT - 1 reads column c0 + NPT (right halo box for lane 31)
      o3e = lane == 0 ? 3 * POPB + MB + w * 16 + (V - 1) * ES : 3 * POPB + own - ES;
      o4e = lane == 31 ? 4 * POPB + MB + HB + w * 16 : 4 * POPB + own + NPT * ES;
    } else {
      // plane box: lattice row q1 + dr sits in staged row w + 1 + dr of every population,
      // tile column c at V + c; pop 1 pulls from row q1 - 1, pop 2 from q1 + 1, and the
      // q1-face rules read the node's own row
      own = (unsigned)((w + 1) * WXB + (PL::V + c0) * ES);
      o1 = POPB + own - WXB;
      o2 = 2 * POPB + own + WXB;
      if (rowin && q1 == 0) {
        const int b = a.bc[0];
        if (b == LBW_BC_FREE) o1 = POPB + own;
        else { o1 = 2 * POPB + own; m1 = sc1 * wall(b); }
      }
      if (rowin && q1 == a.n1 - 1) {
        const int b = a.bc[1];
        if (b == LBW_BC_FREE) o2 = 2 * POPB + own;
        else { o2 = POPB + own; m2 = sc1 * wall(b); }
      }
      // columns -1 and BX come from the wrapped halo boxes on a periodic q2 edge
      o3e = (lane == 0 && wrapL) ? HL + 3 * HPOP + (w + 1) * 16 + (PL::V - 1) * ES : 3 * POPB + own - ES;
      o4e = (lane == 31 && wrapR) ? HR + 4 * HPOP + (w + 1) * 16 : 4 * POPB + own + NPT * ES;
    }
    // q2 faces (non-periodic q2): free copies the node's own value, walls reflect the opposite
    const bool q2lo_free = a.bc[2] == LBW_BC_FREE, q2hi_free = a.bc[3] == LBW_BC_FREE;
    const R q2lo_m = sc1 * wall(a.bc[2]), q2hi_m = sc1 * wall(a.bc[3]);
    // q3 faces: populations 5 / 6 at the first / last plane take the node's own value (free)
    // or its opposite population (walls), with these factors
    const bool f5_own = a.bc[4] == LBW_BC_FREE, f6_own = a.bc[5] == LBW_BC_FREE;
    const R m5_face = a.bc[4] == LBW_BC_FREE ? sc1 : sc1 * wall(a.bc[4]);
    const R m6_face = a.bc[5] == LBW_BC_FREE ? sc1 : sc1 * wall(a.bc[5]);

    // halo column node of a halo warp: warp 0 lane l -> (y0 + l, x0 - 1), warp BY+1 ->
    // (y0 + l, x0 + BX), lanes l < BY; the other lanes mirror lane BY - 1 and store nothing
    const bool hwarp = !interior;
    const int hl = lane < BY ? lane : BY - 1;
    const int hq1 = y0 + hl, hq2 = (w == 0) ? x0 - 1 : x0 + BX;
    const bool hcol = hwarp && lane < BY;
    const bool hin = hq1 < a.n1 && (p2 || (hq2 >= 0 && hq2 < a.n2));
    unsigned h0, h1, h2, h3, h4;
    unsigned hps = POPB;  // population stride at the halo column node
    R hm1 = sc1, hm2 = sc1;
    if constexpr (!RG) {
      // plane box: lattice row y0 + hl is staged row hl + 2; the column node lies in a
      // wrapped halo box on a periodic q2 edge, else in the plane box
      const int hr2 = hl + 2;
      const bool hh = (w == 0) ? wrapL : wrapR;
      hps = hh ? HPOP : POPB;
      auto hat = [&](int pop, int r) -> unsigned {
        return hh ? (unsigned)(((w == 0) ? HL : HR) + pop * HPOP + r * 16 + ((w == 0) ? (PL::V - 1) * ES : 0))
                  : (unsigned)(pop * POPB + r * WXB + (PL::V + ((w == 0) ? -1 : BX)) * ES);
      };
      h0 = hat(0, hr2);
      h1 = hat(1, hr2 - 1);
      h2 = hat(2, hr2 + 1);
      // pop 3 from column -2 / BX - 1, pop 4 from column 0 / BX + 1
      h3 = (w == 0) ? (wrapL ? HL + 3 * HPOP + hr2 * 16 + (PL::V - 2) * ES : 3 * POPB + hr2 * WXB + (PL::V - 2) * ES)
                    : 3 * POPB + hr2 * WXB + (PL::V + BX - 1) * ES;
      h4 = (w == 0) ? 4 * POPB + hr2 * WXB + PL::V * ES
                    : (wrapR ? HR + 4 * HPOP + hr2 * 16 + ES : 4 * POPB + hr2 * WXB + (PL::V + BX + 1) * ES);
      if (hq1 == 0) {
        const int b = a.bc[0];
        if (b == LBW_BC_FREE) h1 = hat(1, hr2);
        else { h1 = hat(2, hr2); hm1 = sc1 * wall(b); }
      }
      if (hq1 == a.n1 - 1) {
        const int b = a.bc[1];
        if (b == LBW_BC_FREE) h2 = hat(2, hr2);
        else { h2 = hat(1, hr2); hm2 = sc1 * wall(b); }
      }
    } else {
      const int hw = hl + 1;
      // column -1 lives in the left halo box (index V - 1), column BX in the right one (0)
      const unsigned hbox = (w == 0) ? MB : MB + HB, hcolb = (w == 0) ? (V - 1) * ES : 0;
      auto hat = [&](int pop, int row) { return (unsigned)(pop * POPB) + hbox + row * 16 + hcolb; };
      h0 = hat(0, hw);
      h1 = hat(1, hw);
      h2 = hat(2, hw);
      // pop 3 from column -2 / BX - 1, pop 4 from column 0 / BX + 1
      h3 = (w == 0) ? 3 * POPB + MB + hw * 16 + (V - 2) * ES : 3 * POPB + hw * BX * ES + (BX - 1) * ES;
      h4 = (w == 0) ? 4 * POPB + hw * BX * ES : 4 * POPB + MB + HB + hw * 16 + ES;
      if (hq1 == 0) {
        const int b = a.bc[0];
        if (b == LBW_BC_FREE) h1 = hat(1, hw + 1);
        else { h1 = hat(2, hw - 1); hm1 = sc1 * wall(b); }
      }
      if (hq1 == a.n1 - 1) {
        const int b = a.bc[1];
        if (b == LBW_BC_FREE) h2 = hat(2, hw - 1);
        else { h2 = hat(1, hw + 1); hm2 = sc1 * wall(b); }
      }
    }
    const unsigned hrho = (unsigned)(((hl + 1) * PW + ((w == 0) ? C0 - 1 : C0 + BX)) * RS);
    const unsigned myrho = (unsigned)((w * PW + C0 + c0) * RS);

    // probes of this warp's row (recorded while the sample counter is below capacity)
    bool has_probe = false;
    if (owner && t_sample < (unsigned long long)a.cap)
      for (int s = 0; s < probe_cnt; ++s) has_probe |= a.probe_q[3 * probe_list[s]] == q1;

    R fA[7][NPT], fB[7][NPT], rA[NPT], rB[NPT], rC[NPT];
    const long long n12 = (long long)a.n1 * a.n2;
    S* const dst_z0 = a.fout + node(owner ? q1 : 0, q2, z0, a.n1, a.n2);

    // step A of pulled plane u: populations into f, rho into rr and (wr) the rho plane
    // slots of planes u - 1, u, u + 1.  Regrouped (RG): slot sl0 holds populations 0-5 of
    // plane u and population 6 of plane u + 1, slot slm population 5 of plane u - 1 and
    // population 6 of plane u (the faces' own values), slot slp is not read.  Otherwise each
    // slot holds its whole plane.
    auto stepA = [&](int u, R (&f)[7][NPT], R (&rr)[NPT], int slm, int sl0, int slp, int rbu,
                     bool wr) {
      const bool zlo = !p3 && u == 0, zhi = !p3 && u == a.n3 - 1;
      const bool zghost = !p3 && (u < 0 || u >= a.n3);
      const unsigned S0 = SL + sl0 * SLOTB, SM = SL + slm * SLOTB;
      unsigned B5, B6, H5, H6;
      if constexpr (RG) {
        B5 = zlo ? (f5_own ? S0 + 5 * POPB : SM + 6 * POPB) : SM + 5 * POPB;
        B6 = zhi ? (f6_own ? SM + 6 * POPB : S0 + 5 * POPB) : S0 + 6 * POPB;
        H5 = B5;
        H6 = B6;
      } else {
        const unsigned s5 = zlo ? S0 : SM, s6 = zhi ? S0 : SL + slp * SLOTB;
        const int p5 = zlo ? (f5_own ? 5 : 6) : 5, p6 = zhi ? (f6_own ? 6 : 5) : 6;
        B5 = s5 + p5 * POPB;
        B6 = s6 + p6 * POPB;
        H5 = s5 + p5 * hps;
        H6 = s6 + p6 * hps;
      }
      const R m5 = zlo ? m5_face : sc1, m6 = zhi ? m6_face : sc1;
      R t3[NPT], t4[NPT];
      ldv(S0 + own, f[0]);
      ldv(S0 + o1, f[1]);
      ldv(S0 + o2, f[2]);
      ldv(S0 + 3 * POPB + own, t3);
      ldv(S0 + 4 * POPB + own, t4);
      ldv(B5 + own, f[5]);
      ldv(B6 + own, f[6]);
      f[3][0] = sc1 * ld1(S0 + o3e);
      f[4][NPT - 1] = sc1 * ld1(S0 + o4e);
#pragma unroll
      for (int k = 0; k + 1 < NPT; ++k) {
        f[3][k + 1] = sc1 * t3[k];
        f[4][k] = sc1 * t4[k + 1];
      }
      if (!p2) {
        f[3][0] = q2lo ? (q2lo_free ? sc1 * t3[0] : q2lo_m * t4[0]) : f[3][0];
        f[4][NPT - 1] = q2hi ? (q2hi_free ? sc1 * t4[NPT - 1] : q2hi_m * t3[NPT - 1]) : f[4][NPT - 1];
      }
      const bool ghost = zghost || !rowin;
      if constexpr (sizeof(R) == 4) {
        const float2 W0S = bc2(a.w[0]), W1S = bc2(a.w[1]);
#pragma unroll
        for (int k = 0; k < NPT; k += 2) {
          float2 F[7];
#pragma unroll
          for (int i = 0; i < 7; ++i) F[i] = f2(f[i][k], f[i][k + 1]);
          F[1] = mul2(bc2(m1), F[1]);
          F[2] = mul2(bc2(m2), F[2]);
          F[5] = mul2(bc2(m5), F[5]);
          F[6] = mul2(bc2(m6), F[6]);
          f[1][k] = F[1].x; f[1][k + 1] = F[1].y;
          f[2][k] = F[2].x; f[2][k + 1] = F[2].y;
          f[5][k] = F[5].x; f[5][k + 1] = F[5].y;
          f[6][k] = F[6].x; f[6][k + 1] = F[6].y;
          float2 sum;
          if constexpr (SC)
            sum = fma2(W0S, F[0], mul2(W1S, add2(add2(add2(F[1], F[2]), add2(F[3], F[4])), add2(F[5], F[6]))));
          else
            sum = add2(add2(add2(F[0], F[1]), add2(F[2], F[3])), add2(add2(F[4], F[5]), F[6]));
          rr[k] = ghost ? R(0) : sum.x;
          rr[k + 1] = ghost ? R(0) : sum.y;
        }
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
          g[0] = sc0 * ld1(S0 + h0);
          g[1] = hm1 * ld1(S0 + h1);
          g[2] = hm2 * ld1(S0 + h2);
          g[3] = sc1 * ld1(S0 + h3);
          g[4] = sc1 * ld1(S0 + h4);
          g[5] = m5 * ld1(H5 + h0);  // h0 addresses population 0: H5 / H6 add their own
          g[6] = m6 * ld1(H6 + h0);
          const R h = SC ? a.w[0] * g[0] + a.w[1] * (((g[1] + g[2]) + (g[3] + g[4])) + (g[5] + g[6]))
                         : ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + g[6]);
          if (hcol) *reinterpret_cast<R*>(smem_raw + pl + hrho) = (hin && !zghost) ? h : R(0);
        }
      }
    };

    // step B's shared-memory inputs for plane zc: rho of plane zc at the neighbours in q1 and
    // q2 (rho plane rbz) and the tile row's coefficients (slot slz).  They are read before
    // step A of the plane ahead, which writes another rho plane, so their latency overlaps
    // with step A's work.
    struct BIn {
      R ru[NPT], rd[NPT], lft, rgt;
      int slz;
    };
    auto loadB = [&](BIn& b, int slz, int rbz) {
      const unsigned cur = RHO + rbz * (PS * RS) + myrho;
      VecN<R, NPT>::ld(reinterpret_cast<const R*>(smem_raw + cur + PW * RS), b.ru);
      VecN<R, NPT>::ld(reinterpret_cast<const R*>(smem_raw + cur - PW * RS), b.rd);
      b.lft = ldr(cur - RS);
      b.rgt = ldr(cur + NPT * RS);
      b.slz = slz;
    };

    // step B: collide plane zc with populations fc, rho (rp, rc, rn) and the inputs in bi
    auto stepB = [&](int zc, R (&fc)[7][NPT], const R (&rp)[NPT], const R (&rc)[NPT],
                     const R (&rn)[NPT], const BIn& bi) {
      const R (&ru)[NPT] = bi.ru;
      const R (&rd)[NPT] = bi.rd;
      const unsigned T = TAB + bi.slz * TABB + (w - 1) * (T_SLOTS * RS);
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
      R rl[NPT], rrt[NPT];
      rl[0] = q2lo ? a.s2lo * rc[0] : bi.lft;
      rrt[NPT - 1] = q2hi ? a.s2hi * rc[NPT - 1] : bi.rgt;
#pragma unroll
      for (int k = 0; k + 1 < NPT; ++k) {
        rl[k + 1] = rc[k];
        rrt[k] = rc[k + 1];
      }
      if constexpr (sizeof(R) == 4) {
        // node pairs (k, k + 1) in paired FP32 instructions; negated coefficients give -D1 and
        // -D3 directly
        const float2 A1P = bc2(-c[T_A1P]), A1M = bc2(c[T_A1M]), C13P = bc2(-c[T_C13P]),
                     C13M = bc2(c[T_C13M]), S1 = bc2(-c[T_S1]), B13P = bc2(-c[T_B13P]),
                     B13M = bc2(c[T_B13M]), C33P = bc2(-c[T_C33P]), C33M = bc2(c[T_C33M]),
                     S3 = bc2(-c[T_S3]), H22 = bc2(c[T_H22]), MG1 = bc2(c[T_MG1]),
                     MG3 = bc2(c[T_MG3]), CS2 = bc2(a.cs2), W0 = bc2(a.two_w0),
                     HALF = bc2(SC ? 1.f / a.cs2 : 0.5f), MHALF = bc2(SC ? -1.f / a.cs2 : -0.5f);
#pragma unroll
        for (int k = 0; k < NPT; k += 2) {
          const float2 rho = f2(rc[k], rc[k + 1]);
          const float2 u = f2(ru[k], ru[k + 1]), d = f2(rd[k], rd[k + 1]);
          const float2 n = f2(rn[k], rn[k + 1]), p = f2(rp[k], rp[k + 1]);
          const float2 nD1 = fma2(S1, rho, fma2(C13M, p, fma2(C13P, n, fma2(A1M, d, mul2(A1P, u)))));
          const float2 nD3 = fma2(S3, rho, fma2(C33M, p, fma2(C33P, n, fma2(B13M, d, mul2(B13P, u)))));
          const float2 D2 = mul2(H22, sub2(f2(rrt[k], rrt[k + 1]), f2(rl[k], rl[k + 1])));
          float2 F[7];
#pragma unroll
          for (int i = 0; i < 7; ++i) F[i] = f2(fc[i][k], fc[i][k + 1]);
          // unscaled: j = m + F/2, f* = 2 f^eq - f with 2 f^eq = cs2 rho +- j (2 w0 rho at rest);
          // scaled (h = f / w): J = 2 j / cs2, h* = 2 rho +- J - h
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
            fc[i][k] = o[i].x;
            fc[i][k + 1] = o[i].y;
          }
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
          const R e = a.cs2 * rho;
          fc[0][k] = a.two_w0 * rho - fc[0][k];
          fc[1][k] = e + j1 - fc[1][k];
          fc[2][k] = e - j1 - fc[2][k];
          fc[3][k] = e + j2 - fc[3][k];
          fc[4][k] = e - j2 - fc[4][k];
          fc[5][k] = e + j3 - fc[5][k];
          fc[6][k] = e - j3 - fc[6][k];
        }
      }
      S* dst = dst_z0 + (long long)(zc - z0) * n12;
#pragma unroll
      for (int i = 0; i < 7; ++i) {
        VecN<S, NPT>::st(dst, fc[i]);
        dst += a.nn;
      }
      if (has_probe) {
        for (int s = 0; s < probe_cnt; ++s) {
          const int k = probe_list[s];
          const int dq = a.probe_q[3 * k + 1] - q2;
          if (a.probe_q[3 * k] == q1 && dq >= 0 && dq < NPT && a.probe_q[3 * k + 2] == zc) {
            R v = rc[0];
#pragma unroll
            for (int j = 1; j < NPT; ++j) v = dq == j ? rc[j] : v;
            a.series[(long long)k * a.cap + t_sample] = (double)v * (double)c[T_INVSG];
          }
        }
      }
    };

    if (stall_req) {
      // Injected timeout: every consumer warp waits on the barrier nothing completes, so the
      // bounded wait runs out and raises the flags.  No slot is consumed or released, hence
      // the producer never re-fills a slot whose copy may still be in flight; it stops at its
      // first wait for a released slot and drains the copies it issued.
      wait_bar(stall_bar, 0, kStallTries);
    } else {
      // rho of plane z0 - 1 at the own nodes, from the staged planes z0 - 2 (population 5 only),
      // z0 - 1 and z0; then step A of plane z0
      // the slot that completes what step A of plane u needs: u's own (RG) or u + 1's
      constexpr int AHEAD = RG ? 0 : 1;
      bool ok = wait_bar(full_at(0), 0) && wait_bar(full_at(1), 0) && (RG || wait_bar(full_at(2), 0));
      if (ok && owner) stepA(z0 - 1, fB, rA, 0, 1, 2, 2, false);
      if (lane == 0) mbar_arrive(empty_at(0));  // plane z0 - 2 is no longer needed
      ok = ok && wait_bar(full_at(2 + AHEAD), 0);
      if (ok) stepA(z0, fA, rB, 1, 2, 3, 0, true);
      if (lane == 0) mbar_arrive(empty_at(1));  // nor is plane z0 - 1
      ok = !named_sync_or(1, NCW * 32, !ok || abort_flag);
      // slots of raw planes z, z + 1, z + 2 (plane z0 - 2 sits in slot 0) and the fill count of
      // the awaited slot (plane z + 1's or z + 2's), advanced plane by plane.  rho planes rotate
      // through three buffers: a warp writing plane z + 1's buffer has passed the barrier that
      // follows every read of that buffer (plane z - 2); the rows of plane z0 - 1 in buffer 2
      // are never written or read.
      int sz = 2, s1 = 3, s2 = 4, uw = 0, rbz = 0, rb1 = 1;
      auto advance = [&]() {
        rbz = rb1;
        rb1 = rb1 == 2 ? 0 : rb1 + 1;
        sz = s1;
        s1 = s2;
        s2 = s2 == NB - 1 ? 0 : s2 + 1;
        if ((RG ? s1 : s2) == 0) ++uw;
      };
      // iteration z: raw plane z + 1 (RG) or z + 2 in, B(z)'s shared-memory reads, A(z + 1),
      // B(z), release raw plane z, barrier.  B(z) needs rho of plane z + 1 only at the warp's
      // own nodes (its own A(z + 1)) and rho plane z, which every warp wrote before the previous
      // iteration's barrier; A(z + 1) writes rho plane z + 1, whose buffer was last read by
      // B(z - 2), two barriers back.  Every warp passes the same barriers; the barrier ORs the
      // warps' abort states (a timed-out wait here, or the producer's flag), so all warps leave
      // after the same iteration.
      auto iter = [&](int zz, R (&fc)[7][NPT], R (&fn)[7][NPT], const R (&rp)[NPT],
                      const R (&rc)[NPT], R (&rn)[NPT], bool collide) {
        const bool in = wait_bar(full_at(RG ? s1 : s2), (unsigned)(uw & 1));
        if (in) {
          BIn bi;
          if (collide) loadB(bi, sz, rbz);
          stepA(zz + 1, fn, rn, sz, s1, s2, rb1, true);
          if (collide) stepB(zz, fc, rp, rc, rn, bi);
        }
        if (lane == 0) mbar_arrive(empty_at(sz));  // raw plane zz is no longer needed
        const bool go = !named_sync_or(1, NCW * 32, !in || abort_flag);
        advance();
        return go;
      };
      int z = z0;
      if (!owner) {  // halo rows and rows beyond the lattice: rho only
        for (; ok && z < z1; ++z) ok = iter(z, fA, fB, rA, rB, rC, false);
      } else {
        for (; ok && z + 1 < z1; z += 2) {
          ok = iter(z, fA, fB, rA, rB, rC, true);
          if (!ok) break;
          ok = iter(z + 1, fB, fA, rB, rC, rA, true);
          // next pair expects rho(z+1), rho(z+2) in rA, rB
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
  }

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
  double eq_e, eq_two0;
  equilibrium_coefs(g->d, &eq_e, &eq_two0);
  a.cs2 = (R)eq_e;  // cs^2 for the paper's method; the Cartesian equilibria change it
  a.two_w0 = (R)eq_two0;
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
  a.pitch = g->pitch ? g->pitch : g->d.n[1];
  a.col0 = g->col0;
  a.ps = pop_stride(g);
  a.geo.kind = g->d.kind;
  a.geo.profile = g->d.horn_profile;
  a.geo.x0r = (R)g->d.x0[0];
  a.geo.x0w = (R)g->d.x0[2];
  a.geo.h0 = (R)g->d.h[0];
  a.geo.h1 = (R)g->d.h[1];
  a.geo.h2 = (R)g->d.h[2];
  a.geo.g0 = (R)g->d.geom[0];
  a.geo.g1 = (R)g->d.geom[1];
  a.geo.g2 = (R)g->d.geom[2];
  a.geo.c2 = (R)(g->d.c * g->d.c);
  a.geo.cs2 = (R)g->d.cs2;
  return a;
}

template <typename S, int BY, int NPT, bool ANA>
constexpr size_t tma_smem_bytes() {
  using R = typename Store<S>::R;
  constexpr int BX = 32 * NPT, NB = 5, PS = (BY + 2) * (BX + 2 * NPT);
  constexpr int TABB = ((BY * T_SLOTS * (int)sizeof(R)) + 127) / 128 * 128;
  constexpr int SLOTB = sizeof(S) == 2 ? PlaneLayout<BY, BX>::slot_bytes()
                                       : TmaLayout<BY, BX>::template slot_bytes<S>();
  return 128 /* alignment slack */ + 128 /* barriers */ + (size_t)NB * SLOTB +
         ((3 * PS * sizeof(R) + 127) / 128) * 128 + (size_t)NB * TABB +
         (ANA ? ((3 * (BY + 2) * sizeof(MetricR<R>) + 127) / 128) * 128 : 0);  // see step_tma_kernel
}

// The tile kernel for (rows BY, nodes per lane NPT, analytic geometry or not): f(kernel,
// dynamic shared bytes).  Four nodes per lane (128-column tiles) exist for the 16-bit storage
// formats only, the analytic geometry for 32- and 64-bit storage only; the table-geometry
// kernels carry none of the analytic code.
template <typename S, typename F>
auto tma_dispatch(int by, int npt, bool ana, F&& f) {
  if constexpr (sizeof(S) == 2) {
    if (npt == 4)
      return by == 7 ? f(step_tma_kernel<S, 7, 4, false>, tma_smem_bytes<S, 7, 4, false>())
                     : f(step_tma_kernel<S, 4, 4, false>, tma_smem_bytes<S, 4, 4, false>());
  } else {
    if (ana)
      return by == 7 ? f(step_tma_kernel<S, 7, 2, true>, tma_smem_bytes<S, 7, 2, true>())
                     : f(step_tma_kernel<S, 4, 2, true>, tma_smem_bytes<S, 4, 2, true>());
  }
  return by == 7 ? f(step_tma_kernel<S, 7, 2, false>, tma_smem_bytes<S, 7, 2, false>())
                 : f(step_tma_kernel<S, 4, 2, false>, tma_smem_bytes<S, 4, 2, false>());
}

template <typename S>
cudaError_t launch_step_t(Grid* g, int src) {
  using R = typename Store<S>::R;
  StepArgs<S> a = make_args<S>(g, src);
  if (g->tma_by > 0) {
    const CUtensorMap* m = reinterpret_cast<const CUtensorMap*>(g->tmaps);
    // consecutive steps overlap launch and prologue with the previous step's tail
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = g->grid_dim;
    cfg.blockDim = dim3(32, g->tma_by + 3);
    cfg.stream = g->stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return tma_dispatch<S>(g->tma_by, g->tma_npt, g->d.geom_mode == LBW_GEOM_ANALYTIC, [&](auto kern, size_t smem) {
      cfg.dynamicSmemBytes = smem;
      return cudaLaunchKernelEx(&cfg, kern, a, m[2 * src], m[2 * src + 1], m[4]);
    });
  }
  dim3 block(g->bx, g->by);
  size_t smem = 3 * (size_t)(g->bx + 2) * (g->by + 2) * sizeof(R);
  step_kernel<S><<<g->grid_dim, block, smem, g->stream>>>(a);
  return cudaGetLastError();
}

struct TmaInfo {
  int regs;
  size_t smem;
};

template <typename S>
TmaInfo tma_info_t(int by, int npt, bool ana) {
  return tma_dispatch<S>(by, npt, ana, [&](auto kern, size_t smem) {
    cudaFuncAttributes at;
    int regs = 255;
    if (cudaFuncGetAttributes(&at, kern) == cudaSuccess) regs = at.numRegs;
    else cudaGetLastError();
    return TmaInfo{regs, smem};
  });
}

template <typename S>
cudaError_t tma_prepare_t(int by, int npt, bool ana) {
  return tma_dispatch<S>(by, npt, ana, [&](auto kern, size_t smem) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
}

TmaInfo tma_info(int prec, int by, int npt, bool ana) {
  switch (prec) {
    case LBW_F64: return tma_info_t<double>(by, npt, ana);
    case LBW_F32: return tma_info_t<float>(by, npt, ana);
    case LBW_F16S: return tma_info_t<__half>(by, npt, ana);
    default: return tma_info_t<__nv_bfloat16>(by, npt, ana);
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

EncodeTiledFn tiled_encoder() {
  static EncodeTiledFn encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return nullptr;
    }
    encode = reinterpret_cast<EncodeTiledFn>(fn);
  }
  return encode;
}

// Tensor maps of the two population buffers (4-D: q2, q1, q3, population) with the main
// (bx x BY+2) and halo (V x BY+2) boxes, and of the coefficient table (3-D: slot, q1, q3).
bool build_tmaps(Grid* g, int by, int bx) {
  const EncodeTiledFn encode = tiled_encoder();
  if (!encode) return false;
  const int es = (int)g->elem, rs = g->d.prec == LBW_F64 ? 8 : 4;
  CUtensorMapDataType dt = g->d.prec == LBW_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                           : g->d.prec == LBW_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                           : g->d.prec == LBW_F16S ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                   : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const cuuint64_t dims[4] = {(cuuint64_t)g->d.n[1], (cuuint64_t)g->d.n[0], (cuuint64_t)g->d.n[2], 7};
  const cuuint64_t strides[3] = {(cuuint64_t)g->d.n[1] * es, (cuuint64_t)g->d.n[1] * g->d.n[0] * es,
                                 (cuuint64_t)g->nn * es};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  // 32/64-bit: one population's main (bx x BY+2) and halo (V x BY+2) boxes; 16-bit: the plane
  // box (bx + 2V x BY+4, all seven populations) and the wrapped halo box (V x BY+4, seven)
  const bool plane = es == 2;
  const cuuint32_t box_main[4] = {(cuuint32_t)(plane ? bx + 2 * (16 / es) : bx),
                                  (cuuint32_t)(by + (plane ? 4 : 2)), 1, plane ? 7u : 1u};
  const cuuint32_t box_halo[4] = {(cuuint32_t)(16 / es), (cuuint32_t)(by + (plane ? 4 : 2)), 1,
                                  plane ? 7u : 1u};
  CUtensorMap* m = reinterpret_cast<CUtensorMap*>(g->tmaps);
  for (int b = 0; b < 2; ++b) {
    if (encode(&m[2 * b], dt, 4, g->f[b], dims, strides, box_main, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
    if (encode(&m[2 * b + 1], dt, 4, g->f[b], dims, strides, box_halo, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  const cuuint64_t tdims[3] = {(cuuint64_t)T_SLOTS, (cuuint64_t)g->d.n[0], (cuuint64_t)g->d.n[2]};
  const cuuint64_t tstr[2] = {(cuuint64_t)T_SLOTS * rs, (cuuint64_t)T_SLOTS * rs * g->d.n[0]};
  const cuuint32_t tbox[3] = {(cuuint32_t)T_SLOTS, (cuuint32_t)by, 1};
  const cuuint32_t testr[3] = {1, 1, 1};
  return encode(&m[4], rs == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                g->table, tdims, tstr, tbox, testr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// ---------------------------------------------------------------- initial state ----------

struct InitGeom {
  int kind, profile;
  double h[3], x0[3], geom[4];
};

__device__ void embed_dev(const InitGeom& G, double u1, double u2, double u3, double X[3]) {
  double s2, c2;
  switch (G.kind) {
    case LBW_CARTESIAN: X[0] = u1; X[1] = u2; X[2] = u3; break;
    case LBW_POLAR:
    case LBW_CYLINDRICAL:
      sincos(u2, &s2, &c2);
      X[0] = u1 * c2; X[1] = u1 * s2; X[2] = u3;
      break;
    case LBW_TRUMPET: {
      double s;
      if (G.profile == 0) s = pow(G.geom[0] - u3, -G.geom[1]);
      else s = (G.geom[0] + G.geom[1] * exp(G.geom[2] * u3)) / (G.geom[0] + G.geom[1]);
      sincos(u2, &s2, &c2);
      X[0] = u1 * s * c2; X[1] = u1 * s * s2; X[2] = u3;
      break;
    }
    default: {
      double s3, c3;
      sincos(u3, &s3, &c3);
      sincos(u2, &s2, &c2);
      const double rr = G.geom[0] + u1 * c3;
      X[0] = rr * c2; X[1] = rr * s2; X[2] = u1 * s3;
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
      const double e = d2 / (2.0 * p[3] * p[3]);
      if (e < 80.0) P0 += p[4] * exp(-e);  // beyond: below 2e-35 of the amplitude
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
    const long long px = ((long long)q3 * a.n1 + q1) * a.pitch + a.col0 + q2;
    // ghost copy of a node near the periodic wrap (padded storage only)
    int gq = -1;
    if (a.col0 > 0 && p2) gq = q2 < a.col0 ? a.col0 + a.n2 + q2 : (q2 >= a.n2 - a.col0 ? q2 - a.n2 + a.col0 : -1);
#pragma unroll
    for (int i = 0; i < 7; ++i) {
      R v = o[i];
      if (Store<S>::kScaled) v *= a.inv_w[i];
      Store<S>::st(a.fout + (long long)i * a.ps + px, v);
      if (gq >= 0) Store<S>::st(a.fout + (long long)i * a.ps + (px - a.col0 - q2) + gq, v);
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

// ---------------------------------------------------------------- harmonic sources -------

// Reading of the paper's sources (ring, plate and point sources of Sec. IV impose P, or J'_z
// for the plate, as C sin(omega t)): after step t the source node's post-collision
// populations are replaced by the equilibrium carrying the imposed value; kind 0:
// f_i = f_i^eq(sqrt(g) C sin(omega t), 0); kind 1: f_i = f_i^eq(rho, (0, 0, sqrt(g) C sin(omega t)))
// with the node's own rho.  16-bit formats store f_i / w_i.
template <typename S>
__global__ void source_kernel(S* __restrict__ base, const SourceEntry* __restrict__ e, int n, int kind,
                              double amp, const unsigned long long* __restrict__ counters) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const SourceEntry s = e[k];
  const double cs2 = s.cs2;
  const double w0 = 1.0 - 3.0 * cs2, w1 = 0.5 * cs2;
  const double v = amp * sin(s.omega * (double)counters[0]);
  S* f = base + s.off;
  double rho = 0.0, j3 = 0.0;
  if (kind == 0) {
    rho = s.sg * v;
  } else {
    for (int i = 0; i < 7; ++i) {
      double x = (double)Store<S>::ld(f + (long long)i * s.ps);
      if (Store<S>::kScaled) x *= (i == 0 ? w0 : w1);
      rho += x;
    }
    j3 = s.sg * v;
  }
  for (int i = 0; i < 7; ++i) {
    const double xi3 = i == 5 ? 1.0 : (i == 6 ? -1.0 : 0.0);
    double val = i == 0 ? w0 * rho : w1 * (rho + xi3 * j3 / cs2);
    if (Store<S>::kScaled) val /= (i == 0 ? w0 : w1);
    const typename Store<S>::R r = (typename Store<S>::R)val;
    Store<S>::st(f + (long long)i * s.ps, r);
    if (s.ghost != 0) Store<S>::st(f + (long long)i * s.ps + s.ghost, r);
  }
}

// ---------------------------------------------------------------- read-out ---------------

// Storage address of dense node x (q2 fastest) in a possibly padded layout.
struct Pad {
  int n2, pitch, col0;
  __device__ long long at(long long x) const {
    return (x / n2) * pitch + col0 + (x % n2);
  }
};

template <typename S>
__global__ void field_kernel(const S* __restrict__ f, long long nn, long long ps, Pad pad, int n1,
                             const typename Store<S>::R* __restrict__ tab, double w0, double w1,
                             double* __restrict__ P) {
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < nn;
       x += (long long)gridDim.x * blockDim.x) {
    const int q1 = (int)((x / pad.n2) % n1);
    const int q3 = (int)(x / ((long long)n1 * pad.n2));
    const long long px = pad.at(x);
    double r = 0.0;
    for (int i = 0; i < 7; ++i) {
      double v = (double)Store<S>::ld(f + (long long)i * ps + px);
      if (Store<S>::kScaled) v *= (i == 0 ? w0 : w1);
      r += v;
    }
    P[x] = r * (double)tab[((long long)q3 * n1 + q1) * T_SLOTS + T_INVSG];
  }
}

template <typename S>
__global__ void to_double_kernel(const S* __restrict__ f, long long nn, long long ps, Pad pad,
                                 double w0, double w1, double* __restrict__ out) {
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < 7 * nn;
       x += (long long)gridDim.x * blockDim.x) {
    const long long i = x / nn, node = x - i * nn;
    double v = (double)Store<S>::ld(f + i * ps + pad.at(node));
    if (Store<S>::kScaled) v *= (i == 0 ? w0 : w1);
    out[x] = v;
  }
}

// Dense doubles into storage; padded storage also gets the ghost copies of a periodic q2.
template <typename S>
__global__ void from_double_kernel(const double* __restrict__ in, long long nn, long long ps,
                                   Pad pad, bool p2, double w0, double w1, S* __restrict__ f) {
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < 7 * nn;
       x += (long long)gridDim.x * blockDim.x) {
    const long long i = x / nn, node = x - i * nn;
    double v = in[x];
    if (Store<S>::kScaled) v /= (i == 0 ? w0 : w1);
    const long long px = pad.at(node);
    const typename Store<S>::R r = (typename Store<S>::R)v;
    Store<S>::st(f + i * ps + px, r);
    if (pad.col0 > 0 && p2) {
      const int q2 = (int)(node % pad.n2);
      const long long row = px - pad.col0 - q2;
      if (q2 < pad.col0) Store<S>::st(f + i * ps + row + pad.col0 + pad.n2 + q2, r);
      if (q2 >= pad.n2 - pad.col0) Store<S>::st(f + i * ps + row + q2 - pad.n2 + pad.col0, r);
    }
  }
}

template <typename S>
cudaError_t launch_readout_t(Grid* g, int what, double* d_out, const double* d_in) {
  const int threads = 256;
  const int blocks = 152 * 8;
  const S* f = reinterpret_cast<const S*>(g->f[g->cur]);
  const Pad pad{g->d.n[1], g->pitch ? g->pitch : g->d.n[1], g->col0};
  const long long ps = pop_stride(g);
  if (what == 0)
    field_kernel<S><<<blocks, threads, 0, g->stream>>>(
        f, g->nn, ps, pad, g->d.n[0], reinterpret_cast<const typename Store<S>::R*>(g->table),
        g->w0, g->w1, d_out);
  else if (what == 1)
    to_double_kernel<S><<<blocks, threads, 0, g->stream>>>(f, g->nn, ps, pad, g->w0, g->w1, d_out);
  else
    from_double_kernel<S><<<blocks, threads, 0, g->stream>>>(
        d_in, g->nn, ps, pad, g->d.bc[2] == LBW_BC_PERIODIC, g->w0, g->w1,
        reinterpret_cast<S*>(g->f[g->cur]));
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

cudaError_t launch_sources(int prec, void* base, const SourceEntry* d_entries, int n, int kind,
                           double amp, const unsigned long long* d_counters, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int threads = 128, blocks = (n + threads - 1) / threads;
  return dispatch(prec, [&](auto tag) {
    using S = decltype(tag);
    source_kernel<S><<<blocks, threads, 0, stream>>>(reinterpret_cast<S*>(base), d_entries, n, kind, amp,
                                                     d_counters);
    return cudaGetLastError();
  });
}

bool encode_tiled_map(void* map, int prec, int rank, void* base, const uint64_t* dims,
                      const uint64_t* strides, const uint32_t* box) {
  const EncodeTiledFn encode = tiled_encoder();
  if (!encode) return false;
  const CUtensorMapDataType dt = prec == LBW_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                 : prec == LBW_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : prec == LBW_F16S ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                    : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  cuuint64_t d[5], st[4];
  cuuint32_t bx[5], es[5];
  for (int k = 0; k < rank; ++k) {
    d[k] = dims[k];
    bx[k] = box[k];
    es[k] = 1;
    if (k + 1 < rank) st[k] = strides[k];
  }
  return encode(reinterpret_cast<CUtensorMap*>(map), dt, (cuuint32_t)rank, base, d, st, bx, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

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

// Launch shape.  TMA tile kernel (q2 extent a multiple of the tile width, non-periodic q1):
// tiles of BX = 64 columns (two nodes per lane) or, for 16-bit storage when the q2 extent is
// a multiple of 128, BX = 128 (four nodes per lane: at 16-bit byte rates the two-node form
// runs out of instruction issue); BY in {4, 7} rows, never with a halo row on the q1 = n1 - 1
// face.  The resident CTAs per SM follow from shared memory and the kernel's register count;
// the number of q3 segments minimises waves x CTAs per SM x (planes per segment + 3) x
// (BY + 2) x BX, the node-planes an SM stages with whole waves counted.  Otherwise the
// register-pipelined kernel with 512-thread tiles.
void step_launch_shape(Grid* g) {
  const int n1 = g->d.n[0], n2 = g->d.n[1], n3 = g->d.n[2];
  int dev = 0, sms = 152, smem_max = 227 * 1024;
  if (cudaGetDevice(&dev) == cudaSuccess) {
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  }
  g->tma_by = 0;
  const int npt = (g->elem == 2 && n2 % 128 == 0) ? 4 : 2, bx = 32 * npt;
  const bool ana = g->d.geom_mode == LBW_GEOM_ANALYTIC;
  if (n2 % bx == 0 && g->d.bc[0] != LBW_BC_PERIODIC && g->nn * 7 < (1LL << 31)) {
    const int bys[2] = {4, 7};
    int per_sm_of[2] = {0, 0};
    for (int c = 0; c < 2; ++c) {
      const int by = bys[c], threads = 32 * (by + 3);
      const TmaInfo ti = tma_info(g->d.prec, by, npt, ana);
      if ((long long)ti.smem > smem_max || ti.regs > 255) continue;
      if ((n1 - 1) % by == 0) continue;  // a halo row would sit on the q1 = n1 - 1 face
      const int rr = (ti.regs + 7) & ~7;
      const int per_sm = std::min<int>(2048 / threads, (int)((228LL * 1024) / (ti.smem + 1024)));
      per_sm_of[c] = std::max(1, std::min(per_sm, 65536 / (rr * threads)));
    }
    // a lone CTA per SM idles the SM at every plane barrier (measured: 16-bit trumpet 8% slower
    // than two CTAs of fewer rows), so shapes with two or more resident CTAs come first
    const bool two = per_sm_of[0] >= 2 || per_sm_of[1] >= 2;
    double best = 1e300;
    for (int c = 0; c < 2; ++c) {
      const int by = bys[c], per_sm = per_sm_of[c];
      if (per_sm == 0 || (two && per_sm < 2)) continue;
      const long long tiles = (long long)(n2 / bx) * ((n1 + by - 1) / by);
      const long long slots = (long long)sms * per_sm;
      for (long long segs = 1; segs <= n3; ++segs) {
        const int lz = (int)((n3 + segs - 1) / segs);
        const long long blocks = tiles * ((n3 + lz - 1) / lz);
        const long long waves = (blocks + slots - 1) / slots;
        const double cost = (double)waves * per_sm * (lz + 3) * (by + 2) * bx;
        if (cost < best) {
          best = cost;
          g->tma_by = by;
          g->lz = lz;
        }
      }
    }
    if (g->tma_by > 0) {
      g->tma_npt = npt;
      cudaError_t e = dispatch(g->d.prec, [&](auto tag) { return tma_prepare_t<decltype(tag)>(g->tma_by, npt, ana); });
      if (e == cudaSuccess && build_tmaps(g, g->tma_by, bx)) {
        g->grid_dim = dim3(n2 / bx, (n1 + g->tma_by - 1) / g->tma_by, (n3 + g->lz - 1) / g->lz);
        return;
      }
      cudaGetLastError();
      g->tma_by = 0;
    }
  }
  int bx2 = std::min(128, ((n2 + 31) / 32) * 32);
  int by2 = 512 / bx2;
  g->bx = bx2;
  g->by = by2;
  const long long cols = (long long)((n2 + bx2 - 1) / bx2) * ((n1 + by2 - 1) / by2);
  const long long slots = (long long)sms * 2;
  long long segs = std::max<long long>(1, slots / cols);
  segs = std::min<long long>(segs, n3);
  g->lz = (int)((n3 + segs - 1) / segs);
  g->grid_dim = dim3((n2 + bx2 - 1) / bx2, (n1 + by2 - 1) / by2, (n3 + g->lz - 1) / g->lz);
}

}  // namespace lbw
