// Device helpers shared by the fused Sinkhorn sweep kernels: element
// widening of the Gibbs kernel K, packed fp32 pairs for the paired FMA,
// mbarrier / bulk-copy / cluster PTX wrappers and the bounded mbarrier wait.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include "fa_internal.cuh"

namespace fa {

// ------------------------------------------------------------ K element types
template <typename TK> struct KT;
template <> struct KT<float> {
  static constexpr int V = 4;
  __device__ static __forceinline__ void unpack(const uint4& u, float (&f)[4]) {
    f[0] = __uint_as_float(u.x); f[1] = __uint_as_float(u.y);
    f[2] = __uint_as_float(u.z); f[3] = __uint_as_float(u.w);
  }
};
template <> struct KT<__nv_bfloat16> {
  static constexpr int V = 8;
  // bf16 is the upper half of an fp32: widen by shifting, register-only.
  __device__ static __forceinline__ void unpack(const uint4& u, float (&f)[8]) {
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      f[2 * q] = __uint_as_float(w[q] << 16);
      f[2 * q + 1] = __uint_as_float(w[q] & 0xffff0000u);
    }
  }
};

// Packed pairs of fp32 in one 64-bit register pair, for the paired FMA of
// sm_100+ (fma.rn.f32x2): one instruction per two elements.
typedef unsigned long long f2_t;
__device__ __forceinline__ f2_t pk2(float lo, float hi) {
  f2_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ f2_t pk2u(uint32_t lo, uint32_t hi) {
  f2_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(lo), "r"(hi));
  return r;
}
__device__ __forceinline__ float2 upk2(f2_t v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
__device__ __forceinline__ f2_t fadd2(f2_t a, f2_t b) {
  f2_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2_t ffma2(f2_t a, f2_t b, f2_t c) {
  f2_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
// the 16 bytes of K as V/2 packed fp32 pairs (columns 2k, 2k+1)
__device__ __forceinline__ void pairs(const uint4& u, f2_t (&p)[2], float) {
  p[0] = pk2u(u.x, u.y);
  p[1] = pk2u(u.z, u.w);
}
__device__ __forceinline__ void pairs(const uint4& u, f2_t (&p)[4], __nv_bfloat16) {
  // bf16 is the upper half of an fp32: widen by shift / mask
  p[0] = pk2u(u.x << 16, u.x & 0xffff0000u);
  p[1] = pk2u(u.y << 16, u.y & 0xffff0000u);
  p[2] = pk2u(u.z << 16, u.z & 0xffff0000u);
  p[3] = pk2u(u.w << 16, u.w & 0xffff0000u);
}

// One 16-byte shared-memory load (a single LDS.128 per thread).
__device__ __forceinline__ uint4 lds128(const void* p) {
  uint4 r;
  asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "r"((uint32_t)__cvta_generic_to_shared(p)));
  return r;
}

// The same load from a 32-bit shared-memory address (no generic-to-shared
// conversion; constant offsets fold into the instruction).
__device__ __forceinline__ uint4 lds128a(uint32_t a) {
  uint4 r;
  asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "r"(a));
  return r;
}

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// The same test, letting the hardware suspend the thread (up to the hint,
// in ns) until the phase completes instead of returning at once: waiting
// warps then issue almost nothing.
constexpr uint32_t kSuspendNs = 10000;
__device__ __forceinline__ bool mbar_try_suspend(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(a), "r"(parity), "n"(kSuspendNs)
      : "memory");
  return ok != 0;
}
// Bounded wait on an mbarrier phase: false after about 2 s (the caller then
// records ST_TIMEOUT and stops depending on that data).
constexpr uint64_t kWaitNs = 2000000000ull;
__device__ inline bool mbar_wait_bounded(uint32_t a, uint32_t parity) {
  if (mbar_try(a, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0; it < (1u << 28); ++it) {
    if (mbar_try_suspend(a, parity)) return true;
    if ((it & 63u) == 0 && global_ns() - t0 > kWaitNs) return false;
  }
  return false;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_size() {
  uint32_t r;
  asm volatile("mov.u32 %0, %cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t map_cluster(uint32_t local_smem_addr, uint32_t cta) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local_smem_addr), "r"(cta));
  return r;
}
// 4-byte store into a peer CTA's shared memory that completes as 4
// transaction bytes on the peer's mbarrier (no fence needed on either side).
__device__ __forceinline__ void st_async_f32(uint32_t remote_addr, float v, uint32_t remote_mbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(
                   remote_addr),
               "r"(__float_as_uint(v)), "r"(remote_mbar)
               : "memory");
}

}  // namespace fa
