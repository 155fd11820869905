// Node-similarity cost on the 5th-generation tensor cores (Algorithm 1, node cost):
//   C[i,j] = alpha exp(-<R1_i, R2_j>) + (1-alpha) exp(-<X1h_i, X2h_j>)
//
// Both products are "A B^T" with K-major operands, so they share one
// kernel: the operands are concatenated along K, A = [R1 | X1h] and
// B = [R2 | X2h], and the K chunks of the first part accumulate into one
// TMEM accumulator, those of the second part into another.
//
// Persistent and warp-specialised: one CTA per SM walks the 128 x 128
// output tiles t = blockIdx.x, blockIdx.x + gridDim.x, ... in a grouped
// order (16 tile rows share each tile column while it is in L2, so B is
// read from HBM once per group, not once per tile row).
//   - warp 0 (one thread) streams 128-byte K chunks of A and B into a
//     shared-memory ring with TMA (128-byte swizzle), across tiles;
//   - warp 1 (one thread) issues tcgen05.mma (M = 128, N = 128) into one of
//     two TMEM buffers (256 columns each: product 1 | product 2), releases
//     each ring stage with tcgen05.commit and signals the buffer full;
//   - warps 2-9 read a full buffer back with tcgen05.ld (warp w reads TMEM
//     lanes 32 (w mod 4) .. + 31, i.e. rows of the tile, and one half of
//     its columns), apply the exp epilogue, write their part of the tile
//     of C once and hand the buffer back.
// So one tile's epilogue runs while the next tile's MMAs fill the other
// buffer.  Every mbarrier wait is bounded; a timeout sets ST_TIMEOUT, every
// role leaves its loop, copies in flight and MMAs are waited for (bounded)
// and TMEM is freed.
// Precision: BF16 operands with FP32 accumulation for the BF16 form; for the
// FP32 form each operand is split into two TF32 parts, x = hi + lo, and
// three products (hi hi + hi lo + lo hi) keep the dot products at about FP32
// accuracy (the lo lo term is below 2^-21 relative).
#include <cuda.h>
#include <math.h>

#include "fa_internal.cuh"

namespace fa {

constexpr int kTM = 128, kTN = 128;         // output tile
constexpr int kEpiWarps = 8;                // two per TMEM lane quadrant
constexpr int kGemmThreads = 32 * (2 + kEpiWarps);   // TMA warp, MMA warp, epilogue warps
constexpr int kAccCols = 2 * kTN;           // one TMEM buffer: product 1 | product 2
constexpr int kGroupM = 16;                 // tile rows per raster group

template <bool TF32> struct TcCfg {
  static constexpr int ELEM = TF32 ? 4 : 2;
  static constexpr int KC = 128 / ELEM;          // elements per 128-byte chunk
  static constexpr int A_BYTES = kTM * 128;      // 16 KB
  static constexpr int B_BYTES = kTN * 128;      // 16 KB
  static constexpr int NOPS = TF32 ? 2 : 1;      // hi (and lo) operand sets
  static constexpr int STAGE = NOPS * (A_BYTES + B_BYTES);
  static constexpr int NSTAGE = TF32 ? 3 : 6;
  static constexpr int SMEM = NSTAGE * STAGE + 1024;   // + alignment slack
  // instruction descriptor: D f32, A/B tf32 (2) or bf16 (1), K-major,
  // N = 128 (n_dim = N >> 3 at bit 17), M = 128 (m_dim = M >> 4 at bit 24)
  static constexpr uint32_t IDESC = (1u << 4) | ((TF32 ? 2u : 1u) << 7) |
                                    ((TF32 ? 2u : 1u) << 10) | ((uint32_t)(kTN >> 3) << 17) |
                                    ((uint32_t)(kTM >> 4) << 24);
};

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t s_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void tc_mbar_init(uint32_t a, uint32_t c) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(c) : "memory");
}
__device__ __forceinline__ void tc_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tc_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ bool tc_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t tc_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// bounded wait (about 2 s), false on timeout
__device__ bool tc_wait(uint32_t a, uint32_t parity) {
  if (tc_try(a, parity)) return true;
  const uint64_t t0 = tc_ns();
  for (uint32_t it = 0; it < (1u << 28); ++it) {
    if (tc_try(a, parity)) return true;
    if ((it & 63u) == 0 && tc_ns() - t0 > 2000000000ull) return false;
  }
  return false;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}
// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;                 // leading byte offset (unused when swizzled)
  d |= (uint64_t)(1024u >> 4) << 32;       // stride byte offset
  d |= (uint64_t)1u << 46;                 // version
  d |= (uint64_t)2u << 61;                 // SWIZZLE_128B
  return d;
}
template <bool TF32>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  if constexpr (TF32) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(TcCfg<true>::IDESC), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(TcCfg<false>::IDESC), "r"(accumulate)
        : "memory");
  }
}
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   mbar)
               : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------ main kernel
// tile t -> (tile row mb, tile column nb): groups of kGroupM tile rows, the
// row index fastest inside a group, so the CTAs working at one time share a
// few tile columns of B and the group's rows of A
__device__ __forceinline__ void tile_coords(int t, int tiles_m, int tiles_n, int& mb, int& nb) {
  const int per_group = kGroupM * tiles_n;
  const int g = t / per_group, r = t - g * per_group;
  const int m0 = g * kGroupM;
  const int gm = min(tiles_m - m0, kGroupM);
  mb = m0 + r % gm;
  nb = r / gm;
}

template <bool TF32>
__global__ void __launch_bounds__(kGemmThreads, 1) k_node_cost_tc(
    const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mA_lo,
    const __grid_constant__ CUtensorMap mB, const __grid_constant__ CUtensorMap mB_lo,
    int n1, int n2, int64_t ldc, int cR, int cX, int ldr, float alpha, int tiles_m,
    int tiles_n, float* __restrict__ C, int* __restrict__ status) {
  using Cf = TcCfg<TF32>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full[Cf::NSTAGE], empty[Cf::NSTAGE], tfull[2], tempty[2], done;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_fail;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int total = cR + cX;
  const int ntiles = tiles_m * tiles_n;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     s_addr(&tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < Cf::NSTAGE; ++s) {
      tc_mbar_init(s_addr(&full[s]), 1);
      tc_mbar_init(s_addr(&empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc_mbar_init(s_addr(&tfull[b]), 1);
      tc_mbar_init(s_addr(&tempty[b]), kEpiWarps);   // one arrival per epilogue warp
    }
    tc_mbar_init(s_addr(&done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  auto a_off = [](int op) { return op * (Cf::A_BYTES + Cf::B_BYTES); };
  auto b_off = [](int op) { return op * (Cf::A_BYTES + Cf::B_BYTES) + Cf::A_BYTES; };

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer: chunk c of the CTA goes to stage c % NSTAGE
      int c = 0;
      for (int t = blockIdx.x; t < ntiles && !s_fail; t += gridDim.x) {
        int mb, nb;
        tile_coords(t, tiles_m, tiles_n, mb, nb);
        for (int kc = 0; kc < total; ++kc) {
          const int s = c % Cf::NSTAGE, k = c / Cf::NSTAGE;
          if (k > 0 && !tc_wait(s_addr(&empty[s]), (uint32_t)((k - 1) & 1))) {
            s_fail = 1;
            break;
          }
          unsigned char* st = smem + (size_t)s * Cf::STAGE;
          const uint32_t fb = s_addr(&full[s]);
          tc_expect_tx(fb, (uint32_t)Cf::STAGE);
          const int x = kc < cR ? kc * Cf::KC : ldr + (kc - cR) * Cf::KC;
          tma_load_2d(s_addr(st + a_off(0)), &mA, x, mb * kTM, fb);
          tma_load_2d(s_addr(st + b_off(0)), &mB, x, nb * kTN, fb);
          if constexpr (TF32) {
            tma_load_2d(s_addr(st + a_off(1)), &mA_lo, x, mb * kTM, fb);
            tma_load_2d(s_addr(st + b_off(1)), &mB_lo, x, nb * kTN, fb);
          }
          ++c;
        }
      }
      if (s_fail) {
        // let copies still in flight into the ring land before the CTA exits
        for (int cc = c - Cf::NSTAGE; cc < c; ++cc)
          if (cc >= 0) tc_wait(s_addr(&full[cc % Cf::NSTAGE]), (uint32_t)((cc / Cf::NSTAGE) & 1));
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer: local tile lt fills TMEM buffer lt & 1
      int c = 0, lt = 0;
      for (int t = blockIdx.x; t < ntiles && !s_fail; t += gridDim.x, ++lt) {
        const int b = lt & 1, use = lt >> 1;
        if (use > 0 && !tc_wait(s_addr(&tempty[b]), (uint32_t)((use - 1) & 1))) {
          s_fail = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc = tmem + (uint32_t)(b * kAccCols);
        bool ok = true;
        for (int kc = 0; kc < total; ++kc, ++c) {
          const int s = c % Cf::NSTAGE;
          if (!tc_wait(s_addr(&full[s]), (uint32_t)((c / Cf::NSTAGE) & 1))) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          unsigned char* st = smem + (size_t)s * Cf::STAGE;
          const uint32_t d = acc + (kc < cR ? 0u : (uint32_t)kTN);
          const bool first = (kc == 0) || (kc == cR);
          const uint32_t a_hi = s_addr(st + a_off(0)), b_hi = s_addr(st + b_off(0));
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {   // 4 x 32 bytes of K per 128-byte chunk
            const uint32_t accum = (first && kk == 0) ? 0u : 1u;
            mma<TF32>(d, smem_desc(a_hi + kk * 32), smem_desc(b_hi + kk * 32), accum);
            if constexpr (TF32) {
              const uint32_t a_lo = s_addr(st + a_off(1)), b_lo = s_addr(st + b_off(1));
              mma<TF32>(d, smem_desc(a_hi + kk * 32), smem_desc(b_lo + kk * 32), 1u);
              mma<TF32>(d, smem_desc(a_lo + kk * 32), smem_desc(b_hi + kk * 32), 1u);
            }
          }
          tc_commit(s_addr(&empty[s]));
        }
        if (!ok) {
          s_fail = 1;
          break;
        }
        tc_commit(s_addr(&tfull[b]));   // fires once this tile's MMAs have completed
      }
      tc_commit(s_addr(&done));         // fires once every MMA issued above has completed
    }
  } else {
    // ---------------- epilogue: warp w owns TMEM lanes (rows) 32 (w % 4) .. + 31
    // and one half of the tile's 32-column chunks (kChunks of them)
    const int quad = warp & 3, half = (warp - 2) >> 2;
    constexpr int kChunks = kTN / 32 / (kEpiWarps / 4);
    const float beta = 1.0f - alpha;
    int lt = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++lt) {
      if (s_fail) break;
      const int b = lt & 1, use = lt >> 1;
      const bool ok = __all_sync(0xffffffffu, tc_wait(s_addr(&tfull[b]), (uint32_t)(use & 1)));
      if (!ok) {
        if (lane == 0) s_fail = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      int mb, nb;
      tile_coords(t, tiles_m, tiles_n, mb, nb);
      const int row = mb * kTM + quad * 32 + lane;
      const uint32_t base = tmem + (uint32_t)(b * kAccCols) + ((uint32_t)(quad * 32) << 16);
#pragma unroll 1
      for (int c2 = 0; c2 < kChunks; ++c2) {
        const int cc = half * kChunks + c2;
        float d1[32], d2[32];
        if (cR > 0) {
          tmem_ld32(base + cc * 32, d1);
        } else {
#pragma unroll
          for (int i = 0; i < 32; ++i) d1[i] = 0.f;
        }
        if (cX > 0) {
          tmem_ld32(base + kTN + cc * 32, d2);
        } else {
#pragma unroll
          for (int i = 0; i < 32; ++i) d2[i] = 0.f;
        }
        const int col0 = nb * kTN + cc * 32;
        if (row < n1 && col0 < ldc) {
          float* dst = C + (int64_t)row * ldc + col0;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            float o[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int j = col0 + q * 4 + e;
              // __expf: relative error of a few ulp for the |d| <= ~2 of
              // unit-norm attributes and RWR rows
              o[e] = j < n2 ? alpha * __expf(-d1[q * 4 + e]) + beta * __expf(-d2[q * 4 + e]) : 0.f;
            }
            reinterpret_cast<float4*>(dst)[q] = make_float4(o[0], o[1], o[2], o[3]);
          }
        }
      }
      // buffer b read out: hand it back to the MMA issuer
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) tc_arrive(s_addr(&tempty[b]));
    }
  }
  __syncwarp();
  __syncthreads();   // every role has left its loop
  if (warp == 0) {
    // every MMA this CTA issued has completed before TMEM is freed
    const bool ok = __all_sync(0xffffffffu, tc_wait(s_addr(&done), 0u));
    if (lane == 0 && (!ok || s_fail)) atomicOr(status, ST_TIMEOUT);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// ------------------------------------------------------------ operands
// A = [R | X] (n x KT, KT = ldr + ldx) as TF32 hi/lo parts (stored as fp32
// bit patterns with the low 13 mantissa bits zero) or as bf16.
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__global__ void k_split_tf32(int n, int64_t ldr, int64_t ldx, const float* __restrict__ R,
                             const float* __restrict__ X, float* __restrict__ hi,
                             float* __restrict__ lo) {
  const int64_t KT = ldr + ldx;
  const int64_t total = (int64_t)n * KT;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / KT, k = t % KT;
    const float v = k < ldr ? R[i * ldr + k] : X[i * ldx + (k - ldr)];
    const float h = to_tf32(v);
    hi[t] = h;
    lo[t] = to_tf32(v - h);
  }
}

__global__ void k_pack_bf16(int n, int64_t ldr, int64_t ldx, const float* __restrict__ R,
                            const float* __restrict__ X, __nv_bfloat16* __restrict__ out) {
  const int64_t KT = ldr + ldx;
  const int64_t total = (int64_t)n * KT;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / KT, k = t % KT;
    out[t] = __float2bfloat16_rn(k < ldr ? R[i * ldr + k] : X[i * ldx + (k - ldr)]);
  }
}

// ------------------------------------------------------------ host
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

bool tc_gemm_available() {
  int dev = 0, major = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess)
    return false;
  return major >= 10 && encode_fn() != nullptr;
}

static size_t ld_of(int k) { return (size_t)round_up(k < 1 ? 1 : k, 64); }

size_t node_cost_tc_workspace(int n1, int n2, int L, int d, bool bf16) {
  const size_t KT = ld_of(L) + ld_of(d);
  const size_t e = bf16 ? 2 : 4, parts = bf16 ? 1 : 2;
  return ((size_t)n1 + (size_t)n2) * KT * e * parts + 256;
}

static fa_status make_map(CUtensorMap* m, const void* base, bool bf16, int rows, int64_t KT,
                          int box_rows) {
  const int e = bf16 ? 2 : 4;
  cuuint64_t dims[2] = {(cuuint64_t)KT, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(KT * e)};
  cuuint32_t box[2] = {(cuuint32_t)(128 / e), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_fn()(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                           2, const_cast<void*>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return FA_ERR_CUDA;
  }
  return FA_OK;
}

fa_status launch_node_cost_tc(int n1, int n2, int L, int64_t ldr, const float* R1,
                              const float* R2, int d, int64_t ldx, const float* X1h,
                              const float* X2h, float alpha, bool bf16, float* C, int64_t ldc,
                              void* ws, size_t ws_bytes, int* status, cudaStream_t s) {
  if (!encode_fn()) {
    set_error("tcgen05 GEMM: cuTensorMapEncodeTiled unavailable");
    return FA_ERR_UNSUPPORTED;
  }
  const int64_t KT = ldr + ldx;
  const size_t e = bf16 ? 2 : 4;
  if (ws_bytes < ((size_t)n1 + n2) * KT * e * (bf16 ? 1 : 2)) {
    set_error("tcgen05 GEMM: workspace too small");
    return FA_ERR_ARG;
  }
  unsigned char* w = static_cast<unsigned char*>(ws);
  // operand layout in the workspace: A (hi), B (hi), A lo, B lo
  void* A = w;
  void* B = w + (size_t)n1 * KT * e;
  void* Alo = w + ((size_t)n1 + n2) * KT * e;
  void* Blo = static_cast<unsigned char*>(Alo) + (size_t)n1 * KT * e;
  const unsigned blocks = 4096;
  if (bf16) {
    k_pack_bf16<<<blocks, 256, 0, s>>>(n1, ldr, ldx, R1, X1h, static_cast<__nv_bfloat16*>(A));
    FA_LAUNCHED("k_pack_bf16");
    k_pack_bf16<<<blocks, 256, 0, s>>>(n2, ldr, ldx, R2, X2h, static_cast<__nv_bfloat16*>(B));
    FA_LAUNCHED("k_pack_bf16");
  } else {
    k_split_tf32<<<blocks, 256, 0, s>>>(n1, ldr, ldx, R1, X1h, static_cast<float*>(A),
                                        static_cast<float*>(Alo));
    FA_LAUNCHED("k_split_tf32");
    k_split_tf32<<<blocks, 256, 0, s>>>(n2, ldr, ldx, R2, X2h, static_cast<float*>(B),
                                        static_cast<float*>(Blo));
    FA_LAUNCHED("k_split_tf32");
  }
  CUtensorMap mA, mB, mAl, mBl;
  FA_TRY(make_map(&mA, A, bf16, n1, KT, kTM));
  FA_TRY(make_map(&mB, B, bf16, n2, KT, kTN));
  if (bf16) {
    mAl = mA;
    mBl = mB;
  } else {
    FA_TRY(make_map(&mAl, Alo, bf16, n1, KT, kTM));
    FA_TRY(make_map(&mBl, Blo, bf16, n2, KT, kTN));
  }
  const int kc = bf16 ? TcCfg<false>::KC : TcCfg<true>::KC;
  const int cR = L > 0 ? (L + kc - 1) / kc : 0;
  const int cX = d > 0 ? (d + kc - 1) / kc : 0;
  const int tiles_m = (n1 + kTM - 1) / kTM;
  const int tiles_n = (int)((ldc + kTN - 1) / kTN);
  const int64_t ntiles = (int64_t)tiles_m * tiles_n;
  if (ntiles <= 0) return FA_OK;
  if (ntiles > INT32_MAX) {
    set_error("tcgen05 GEMM: %lld output tiles exceed the tile index range", (long long)ntiles);
    return FA_ERR_UNSUPPORTED;
  }
  // one persistent CTA per SM (TMEM: all 512 columns per CTA);
  // FA_GEMM_CTAS caps the count (tuning, and tests that walk many tiles per CTA)
  int dev = 0, sms = 0;
  FA_CUDA(cudaGetDevice(&dev));
  FA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const char* ctas_str = getenv("FA_GEMM_CTAS");
  const int ctas_env = ctas_str ? atoi(ctas_str) : 0;
  int64_t ctas = sms > 0 ? sms : 1;
  if (ctas_env > 0 && ctas_env < ctas) ctas = ctas_env;
  if (ctas > ntiles) ctas = ntiles;
  const dim3 grid((unsigned)ctas);
  const int ldr_i = (int)ldr;
  if (bf16) {
    const int smem = TcCfg<false>::SMEM;
    FA_CUDA(cudaFuncSetAttribute(k_node_cost_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    k_node_cost_tc<false><<<grid, kGemmThreads, smem, s>>>(mA, mAl, mB, mBl, n1, n2, ldc, cR, cX,
                                                           ldr_i, alpha, tiles_m, tiles_n, C,
                                                           status);
  } else {
    const int smem = TcCfg<true>::SMEM;
    FA_CUDA(cudaFuncSetAttribute(k_node_cost_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    k_node_cost_tc<true><<<grid, kGemmThreads, smem, s>>>(mA, mAl, mB, mBl, n1, n2, ldc, cR, cX,
                                                          ldr_i, alpha, tiles_m, tiles_n, C,
                                                          status);
  }
  FA_LAUNCHED("k_node_cost_tc");
  return FA_OK;
}

}  // namespace fa
