// Phase 3 of Algorithm 1 (Eq. 3) split by column ranges of the plan: the
// data path of a sweep whose columns are sharded over devices.
//
// A device owning columns [j0, j1) of K cannot finish a row sum alone, so
// one iteration runs in three steps instead of the fused single pass:
//
//   rows     partial row sums r_ib = sum_{j in block b} K_ij v_j for every
//            fixed column block b (kShardBlock columns) of the range
//   combine  u_i = mu_i / sum_b r_ib, the blocks added in block order
//            (all blocks of all ranges: on several devices the blocks are
//            gathered first -- n1 floats per block, the only exchange)
//   cols     column sums sum_i K_ij u_i of the range, in a fixed order of
//            row groups, and the next column scaling v_j = nu_j / (.)
//
// Block boundaries do not depend on how the columns are split, and every
// sum runs in a fixed order, so any split into ranges that are multiples of
// the block gives bit-identical results.  The range reads its columns of K
// twice per iteration (rows, then cols): the price of not exchanging row
// sums inside the pass.
#include <cuda_bf16.h>
#include <stdint.h>

#include "fa_internal.cuh"

namespace fa {

namespace {

constexpr int kRowsPerCta = 16;     // rows of a row-partial CTA (2 per warp)
constexpr int kColGroups = 128;     // row groups of the column pass (fixed)

__device__ __forceinline__ void widen8(const uint4& u, float (&f)[8], __nv_bfloat16) {
  const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    f[2 * q] = __uint_as_float(w[q] << 16);
    f[2 * q + 1] = __uint_as_float(w[q] & 0xffff0000u);
  }
}

// r[b][i] = sum over the kShardBlock columns of block b of K_ij v_j: warp
// per row (2 rows per warp), lane l takes the 8-column vectors l, l + 32,
// ... of the block in order, then a fixed butterfly.
template <typename TK>
__global__ void __launch_bounds__(256) k_shard_rows(int n1, int n2, int64_t ld, int b0,
                                                   const TK* __restrict__ K,
                                                   const float* __restrict__ v,
                                                   float* __restrict__ rowpart) {
  constexpr int V = 16 / sizeof(TK);               // elements per 16-byte vector
  const int b = b0 + blockIdx.y;                   // global column block
  const int64_t jb = (int64_t)b * kShardBlock;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int rr = 0; rr < kRowsPerCta / 8; ++rr) {
    const int i = blockIdx.x * kRowsPerCta + warp * (kRowsPerCta / 8) + rr;
    if (i >= n1) break;
    const TK* krow = K + (int64_t)i * ld + jb;
    float acc = 0.f;
    for (int e = lane * V; e < kShardBlock; e += 32 * V) {
      const int64_t j = jb + e;
      if (j >= n2) break;                          // padding columns hold 0 anyway
      const uint4 raw = __ldg(reinterpret_cast<const uint4*>(krow + e));
      float k[V];
      if constexpr (sizeof(TK) == 2) {
        widen8(raw, *reinterpret_cast<float(*)[8]>(k), __nv_bfloat16());
      } else {
        k[0] = __uint_as_float(raw.x); k[1] = __uint_as_float(raw.y);
        k[2] = __uint_as_float(raw.z); k[3] = __uint_as_float(raw.w);
      }
#pragma unroll
      for (int t = 0; t < V; ++t) acc = fmaf(k[t], j + t < n2 ? v[j + t] : 0.f, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) rowpart[(int64_t)b * n1 + i] = acc;
  }
}

// u_i = mu / sum_b r[b][i] in block order; log u_i = log mu - log(sum)
__global__ void k_shard_combine(int n1, int nblocks, const float* __restrict__ rowpart, float mu,
                                float log_mu, float* __restrict__ u, float* __restrict__ log_u,
                                int* __restrict__ status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n1) return;
  float s = 0.f;
  for (int b = 0; b < nblocks; ++b) s += rowpart[(int64_t)b * n1 + i];
  if (s > 0.f && isfinite(s)) {
    u[i] = mu / s;
    log_u[i] = log_mu - logf(s);
  } else {
    atomicOr(status, ST_NUMERIC);
    u[i] = 0.f;
    log_u[i] = log_mu;
  }
}

// colpart[g][j] = sum over rows i = g, g + G, ... of K_ij u_i for the
// columns [j0, j1) (thread per 4 columns, rows in order)
template <typename TK>
__global__ void __launch_bounds__(256) k_shard_cols(int n1, int64_t ld, int64_t j0, int64_t j1,
                                                    const TK* __restrict__ K,
                                                    const float* __restrict__ u,
                                                    float* __restrict__ colpart) {
  const int64_t j = j0 + ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (j >= j1) return;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int i = blockIdx.y; i < n1; i += gridDim.y) {
    const float ui = u[i];
    float k[4];
    if constexpr (sizeof(TK) == 2) {
      const uint2 raw = __ldg(reinterpret_cast<const uint2*>(K + (int64_t)i * ld + j));
      k[0] = __uint_as_float(raw.x << 16); k[1] = __uint_as_float(raw.x & 0xffff0000u);
      k[2] = __uint_as_float(raw.y << 16); k[3] = __uint_as_float(raw.y & 0xffff0000u);
    } else {
      const float4 raw = __ldg(reinterpret_cast<const float4*>(K + (int64_t)i * ld + j));
      k[0] = raw.x; k[1] = raw.y; k[2] = raw.z; k[3] = raw.w;
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) acc[t] = fmaf(k[t], ui, acc[t]);
  }
  *reinterpret_cast<float4*>(colpart + (int64_t)blockIdx.y * ld + j) =
      make_float4(acc[0], acc[1], acc[2], acc[3]);
}

}  // namespace

fa_status launch_shard_rows(int n1, int n2, int64_t ld, int64_t j0, int64_t j1, const void* K,
                            bool bf16, const float* v, float* rowpart, cudaStream_t s) {
  const int b0 = (int)(j0 / kShardBlock);
  const int nb = (int)((j1 - j0 + kShardBlock - 1) / kShardBlock);
  if (nb <= 0 || n1 <= 0) return FA_OK;
  dim3 grid((unsigned)((n1 + kRowsPerCta - 1) / kRowsPerCta), (unsigned)nb);
  if (bf16)
    k_shard_rows<__nv_bfloat16><<<grid, 256, 0, s>>>(
        n1, n2, ld, b0, static_cast<const __nv_bfloat16*>(K), v, rowpart);
  else
    k_shard_rows<float><<<grid, 256, 0, s>>>(n1, n2, ld, b0, static_cast<const float*>(K), v,
                                            rowpart);
  FA_LAUNCHED("k_shard_rows");
  return FA_OK;
}

fa_status launch_shard_combine(int n1, int nblocks, const float* rowpart, float mu, float* u,
                               float* log_u, int* status, cudaStream_t s) {
  k_shard_combine<<<(n1 + 255) / 256, 256, 0, s>>>(n1, nblocks, rowpart, mu, logf(mu), u, log_u,
                                                   status);
  FA_LAUNCHED("k_shard_combine");
  return FA_OK;
}

int shard_col_groups(int n1) { return n1 < kColGroups ? n1 : kColGroups; }

fa_status launch_shard_cols(int n1, int64_t ld, int64_t j0, int64_t j1, const void* K, bool bf16,
                            const float* u, float* colpart, cudaStream_t s) {
  const int64_t ncol = j1 - j0;
  if (ncol <= 0 || n1 <= 0) return FA_OK;
  dim3 grid((unsigned)((ncol / 4 + 255) / 256), (unsigned)shard_col_groups(n1));
  if (bf16)
    k_shard_cols<__nv_bfloat16><<<grid, 256, 0, s>>>(n1, ld, j0, j1,
                                                     static_cast<const __nv_bfloat16*>(K), u, colpart);
  else
    k_shard_cols<float><<<grid, 256, 0, s>>>(n1, ld, j0, j1, static_cast<const float*>(K), u,
                                            colpart);
  FA_LAUNCHED("k_shard_cols");
  return FA_OK;
}

}  // namespace fa
