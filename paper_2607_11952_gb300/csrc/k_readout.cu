// Alignment read-out (Eq. 4 plan, Section 4.1.1 metrics): per-row top-k of
// T_ij = u_i K_ij v_j and the rank of given (row, column) pairs.  The row
// factor u_i does not change the order inside a row, so both kernels score
// s_ij = K_ij * v_j in float32 with identical rounding.  Order: larger
// score first, equal scores by lower column index.
#include <limits.h>
#include <math.h>

#include "fa_internal.cuh"

namespace fa {

__device__ __forceinline__ float kval(const float* K, int64_t t) { return K[t]; }
__device__ __forceinline__ float kval(const __nv_bfloat16* K, int64_t t) {
  return __bfloat162float(K[t]);
}

// (a_val, a_idx) ranks before (b_val, b_idx)?
__device__ __forceinline__ bool better(float av, int ai, float bv, int bi) {
  return av > bv || (av == bv && ai < bi);
}

constexpr int kTopkThreads = 256;

// One CTA per row.  Every thread keeps a sorted list of its KMAX best
// (score, column) pairs in registers (insertion by a compare-swap chain with
// static indices), then k rounds of a block-wide arg-max pop the winners.
template <typename TK, int KMAX>
__global__ void __launch_bounds__(kTopkThreads) k_topk(
    int n2, int64_t ld, const TK* __restrict__ K, const float* __restrict__ v,
    int k, int32_t* __restrict__ idx, float* __restrict__ score) {
  __shared__ float sv[kTopkThreads / 32];
  __shared__ int si[kTopkThreads / 32];
  __shared__ int win;
  const int row = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float vals[KMAX];
  int ids[KMAX];
#pragma unroll
  for (int t = 0; t < KMAX; ++t) { vals[t] = -INFINITY; ids[t] = INT_MAX; }
  const TK* Kr = K + (int64_t)row * ld;
  for (int j = tid; j < n2; j += kTopkThreads) {
    const float s = kval(Kr, j) * v[j];
    if (s > vals[KMAX - 1]) {
      float cv = s;
      int cj = j;
#pragma unroll
      for (int t = 0; t < KMAX; ++t) {
        if (better(cv, cj, vals[t], ids[t])) {
          float tv = vals[t]; int ti = ids[t];
          vals[t] = cv; ids[t] = cj;
          cv = tv; cj = ti;
        }
      }
    }
  }
  for (int r = 0; r < k; ++r) {
    float bv = vals[0];
    int bi = ids[0];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      float ov = __shfl_xor_sync(0xffffffffu, bv, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (better(ov, oi, bv, bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { sv[warp] = bv; si[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      float wv = sv[0];
      int wi = si[0];
      for (int w = 1; w < kTopkThreads / 32; ++w)
        if (better(sv[w], si[w], wv, wi)) { wv = sv[w]; wi = si[w]; }
      const bool ok = wi != INT_MAX;
      idx[(int64_t)row * k + r] = ok ? wi : -1;
      if (score) score[(int64_t)row * k + r] = ok ? wv : -INFINITY;
      win = wi;
    }
    __syncthreads();
    if (ids[0] == win && win != INT_MAX) {
#pragma unroll
      for (int t = 0; t + 1 < KMAX; ++t) { vals[t] = vals[t + 1]; ids[t] = ids[t + 1]; }
      vals[KMAX - 1] = -INFINITY;
      ids[KMAX - 1] = INT_MAX;
    }
    __syncthreads();
  }
}

fa_status launch_topk(int n1, int n2, int64_t ld, const void* K, bool bf16,
                      const float* v, int k, int32_t* idx, float* score,
                      cudaStream_t s) {
#define FA_TOPK(KM)                                                              \
  if (bf16)                                                                     \
    k_topk<__nv_bfloat16, KM><<<n1, kTopkThreads, 0, s>>>(                     \
        n2, ld, static_cast<const __nv_bfloat16*>(K), v, k, idx, score);       \
  else                                                                          \
    k_topk<float, KM><<<n1, kTopkThreads, 0, s>>>(                             \
        n2, ld, static_cast<const float*>(K), v, k, idx, score);
  if (k <= 8) {
    FA_TOPK(8)
  } else if (k <= 16) {
    FA_TOPK(16)
  } else {
    FA_TOPK(32)
  }
#undef FA_TOPK
  FA_LAUNCHED("k_topk");
  return FA_OK;
}

// rank = 1 + #{j : s_j > s_c} + #{j < c : s_j == s_c}; one CTA per query.
template <typename TK>
__global__ void __launch_bounds__(kTopkThreads) k_rank(
    int n2, int64_t ld, const TK* __restrict__ K, const float* __restrict__ v,
    const int32_t* __restrict__ rows, const int32_t* __restrict__ cols,
    int32_t* __restrict__ rank) {
  __shared__ int sc[kTopkThreads / 32];
  const int t = blockIdx.x;
  const int i = rows[t], c = cols[t];
  const TK* Kr = K + (int64_t)i * ld;
  const float ref = kval(Kr, c) * v[c];
  int cnt = 0;
  for (int j = threadIdx.x; j < n2; j += kTopkThreads) {
    const float s = kval(Kr, j) * v[j];
    cnt += (s > ref) || (s == ref && j < c);
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0) sc[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int tot = 0;
    for (int w = 0; w < kTopkThreads / 32; ++w) tot += sc[w];
    rank[t] = 1 + tot;
  }
}

fa_status launch_rank(int n2, int64_t ld, const void* K, bool bf16,
                      const float* v, int nq, const int32_t* rows,
                      const int32_t* cols, int32_t* rank, cudaStream_t s) {
  if (nq <= 0) return FA_OK;
  if (bf16)
    k_rank<__nv_bfloat16><<<nq, kTopkThreads, 0, s>>>(
        n2, ld, static_cast<const __nv_bfloat16*>(K), v, rows, cols, rank);
  else
    k_rank<float><<<nq, kTopkThreads, 0, s>>>(
        n2, ld, static_cast<const float*>(K), v, rows, cols, rank);
  FA_LAUNCHED("k_rank");
  return FA_OK;
}

// ------------------------------------------------------------ plan change
// sum_ij |T_a,ij - T_b,ij| with T = diag(exp(log_u)) K diag(exp(log_v)):
// each element's two plan values in float32, their absolute difference
// accumulated in float64.  Block b sums rows b, b + gridDim.x, ...; a
// one-block kernel adds the block sums in index order (deterministic).
constexpr int kDiffThreads = 256;

template <typename TK>
__global__ void __launch_bounds__(kDiffThreads) k_plan_l1diff(
    int n1, int n2, int64_t ld, const TK* __restrict__ Ka, const float* __restrict__ lua,
    const float* __restrict__ lva, const TK* __restrict__ Kb, const float* __restrict__ lub,
    const float* __restrict__ lvb, double* __restrict__ part) {
  __shared__ double red[kDiffThreads / 32];
  double acc = 0.0;
  for (int i = blockIdx.x; i < n1; i += gridDim.x) {
    const float ua = expf(lua[i]), ub = expf(lub[i]);
    const int64_t row = (int64_t)i * ld;
    for (int j = threadIdx.x; j < n2; j += kDiffThreads) {
      const float ta = ua * kval(Ka, row + j) * expf(lva[j]);
      const float tb = ub * kval(Kb, row + j) * expf(lvb[j]);
      acc += (double)fabsf(ta - tb);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kDiffThreads / 32; ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

__global__ void k_sum_in_order(int n, const double* __restrict__ part, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int b = 0; b < n; ++b) t += part[b];
    *out = t;
  }
}

fa_status launch_plan_l1diff(int n1, int n2, int64_t ld, bool bf16, const void* Ka,
                             const float* lua, const float* lva, const void* Kb,
                             const float* lub, const float* lvb, double* part, int nblocks,
                             double* out, cudaStream_t s) {
  const int blocks = n1 < nblocks ? (n1 > 0 ? n1 : 1) : nblocks;
  if (bf16)
    k_plan_l1diff<__nv_bfloat16><<<blocks, kDiffThreads, 0, s>>>(
        n1, n2, ld, static_cast<const __nv_bfloat16*>(Ka), lua, lva,
        static_cast<const __nv_bfloat16*>(Kb), lub, lvb, part);
  else
    k_plan_l1diff<float><<<blocks, kDiffThreads, 0, s>>>(
        n1, n2, ld, static_cast<const float*>(Ka), lua, lva, static_cast<const float*>(Kb),
        lub, lvb, part);
  FA_LAUNCHED("k_plan_l1diff");
  k_sum_in_order<<<1, 32, 0, s>>>(blocks, part, out);
  FA_LAUNCHED("k_sum_in_order");
  return FA_OK;
}

}  // namespace fa
