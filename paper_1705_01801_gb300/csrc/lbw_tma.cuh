// lbw_tma.cuh -- device helpers of the TMA-staged step kernels (single lattice and
// ensemble): vector moves of NPT consecutive nodes, paired FP32 arithmetic, mbarrier and
// tensor-copy wrappers (inline PTX), and a named barrier with an OR reduction.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace lbw {
namespace dev {

__device__ __forceinline__ int xi1_of(int i) { return i == 1 ? 1 : (i == 2 ? -1 : 0); }

// N consecutive nodes along q2 per lane, moved as one vector: FP32 8 / 16 bytes, FP64 16
// bytes, 16-bit formats 4 / 8 bytes (converted to and from FP32 in pairs).
template <typename S, int N> struct VecN;
template <> struct VecN<float, 2> {
  __device__ static void ld(const float* p, float (&o)[2]) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    o[0] = v.x; o[1] = v.y;
  }
  __device__ static void st(float* p, const float (&o)[2]) {
    *reinterpret_cast<float2*>(p) = make_float2(o[0], o[1]);
  }
};
template <> struct VecN<float, 4> {
  __device__ static void ld(const float* p, float (&o)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  }
  __device__ static void st(float* p, const float (&o)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
  }
};
template <> struct VecN<double, 2> {
  __device__ static void ld(const double* p, double (&o)[2]) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    o[0] = v.x; o[1] = v.y;
  }
  __device__ static void st(double* p, const double (&o)[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
  }
};
// 16-bit pairs <-> float2
__device__ __forceinline__ float2 to_f2(__half2 v) { return __half22float2(v); }
__device__ __forceinline__ float2 to_f2(__nv_bfloat162 v) { return __bfloat1622float2(v); }
template <typename P> __device__ __forceinline__ P from_f2(float a, float b);
template <> __device__ __forceinline__ __half2 from_f2<__half2>(float a, float b) { return __floats2half2_rn(a, b); }
template <> __device__ __forceinline__ __nv_bfloat162 from_f2<__nv_bfloat162>(float a, float b) {
  return __floats2bfloat162_rn(a, b);
}
template <typename S> struct Pair16;
template <> struct Pair16<__half> { using T = __half2; };
template <> struct Pair16<__nv_bfloat16> { using T = __nv_bfloat162; };
template <typename S> struct Vec16 {
  using P = typename Pair16<S>::T;
  __device__ static void ld(const S* p, float (&o)[2]) {
    const float2 a = to_f2(*reinterpret_cast<const P*>(p));
    o[0] = a.x; o[1] = a.y;
  }
  __device__ static void st(S* p, const float (&o)[2]) {
    *reinterpret_cast<P*>(p) = from_f2<P>(o[0], o[1]);
  }
  __device__ static void ld(const S* p, float (&o)[4]) {
    const uint2 u = *reinterpret_cast<const uint2*>(p);
    const float2 a = to_f2(*reinterpret_cast<const P*>(&u.x)), b = to_f2(*reinterpret_cast<const P*>(&u.y));
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
  }
  __device__ static void st(S* p, const float (&o)[4]) {
    const P a = from_f2<P>(o[0], o[1]), b = from_f2<P>(o[2], o[3]);
    uint2 u;
    u.x = *reinterpret_cast<const unsigned*>(&a);
    u.y = *reinterpret_cast<const unsigned*>(&b);
    *reinterpret_cast<uint2*>(p) = u;
  }
};
template <int N> struct VecN<__half, N> : Vec16<__half> {};
template <int N> struct VecN<__nv_bfloat16, N> : Vec16<__nv_bfloat16> {};

// Paired FP32 arithmetic (one instruction for two lanes' values of a node pair), the same
// IEEE round-to-nearest operations as the scalar forms.
__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 bc2(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 add2(float2 x, float2 y) { return __fadd2_rn(x, y); }
__device__ __forceinline__ float2 mul2(float2 x, float2 y) { return __fmul2_rn(x, y); }
__device__ __forceinline__ float2 fma2(float2 x, float2 y, float2 z) { return __ffma2_rn(x, y, z); }
__device__ __forceinline__ float2 sub2(float2 x, float2 y) { return __ffma2_rn(y, bc2(-1.f), x); }

constexpr long long kWaitLimit = 1LL << 20;  // x up to 2 us per try: about 2 s
constexpr long long kStallTries = 256;       // the injected timeout: under a millisecond

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
  unsigned done;
  // the thread may sleep up to 2 us inside try_wait until the phase completes
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 2000;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done) : "r"(bar), "r"(parity) : "memory");
  return done != 0;
}
__device__ __forceinline__ void tma_load_4d(unsigned dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];\n"
      ::"r"(dst), "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
        "r"(bar) : "memory");
}
__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];\n"
      ::"r"(dst), "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2),
        "r"(bar) : "memory");
}


__device__ __forceinline__ void mbar_init_count(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}
// Named barrier that also returns the OR of v over the participating threads, so every
// thread takes the same decision.
__device__ __forceinline__ bool named_sync_or(int id, int threads, bool v) {
  unsigned r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n"
      " barrier.cta.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r) : "r"((unsigned)v), "r"(id), "r"(threads) : "memory");
  return r != 0;
}

}  // namespace dev
}  // namespace lbw
