// Node-similarity cost on CUDA cores (Algorithm 1, node cost):
//   C[i,j] = alpha exp(-<R1_i, R2_j>) + (1-alpha) exp(-<X1h_i, X2h_j>)
// Plain FP32 tiled GEMM (64x64 tile, 4x4 outputs per thread, two
// accumulators).  It is the cross-check for the tcgen05 kernel and the
// FA_GEMM_SIMT mode; operands are row-major with zero-padded leading
// dimensions that are multiples of 64.
#include <math.h>

#include "fa_internal.cuh"

namespace fa {

__global__ void __launch_bounds__(256) k_node_cost_simt(
    int n1, int n2, int L, int64_t ldr, const float* __restrict__ R1,
    const float* __restrict__ R2, int d, int64_t ldx,
    const float* __restrict__ X1, const float* __restrict__ X2, float alpha,
    float* __restrict__ C, int64_t ldc) {
  __shared__ float As[16][68];
  __shared__ float Bs[16][68];
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[2][4][4];
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[p][r][c] = 0.f;

  const int row = threadIdx.x >> 2, kq = (threadIdx.x & 3) * 4;
  const int ia = min(i0 + row, n1 - 1), jb = min(j0 + row, n2 - 1);
#pragma unroll
  for (int pass = 0; pass < 2; ++pass) {
    const float* A = pass == 0 ? R1 : X1;
    const float* B = pass == 0 ? R2 : X2;
    const int Kd = pass == 0 ? L : d;
    const int64_t lda = pass == 0 ? ldr : ldx;
    for (int k0 = 0; k0 < Kd; k0 += 16) {
      const float4 a = *reinterpret_cast<const float4*>(A + (int64_t)ia * lda + k0 + kq);
      const float4 b = *reinterpret_cast<const float4*>(B + (int64_t)jb * lda + k0 + kq);
      As[kq + 0][row] = a.x; As[kq + 1][row] = a.y; As[kq + 2][row] = a.z; As[kq + 3][row] = a.w;
      Bs[kq + 0][row] = b.x; Bs[kq + 1][row] = b.y; Bs[kq + 2][row] = b.z; Bs[kq + 3][row] = b.w;
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) {
        float af[4], bf[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) af[r] = As[kk][ty * 4 + r];
#pragma unroll
        for (int c = 0; c < 4; ++c) bf[c] = Bs[kk][tx * 4 + c];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[pass][r][c] += af[r] * bf[c];
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = i0 + ty * 4 + r;
    if (i >= n1) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = j0 + tx * 4 + c;
      if (j < ldc)
        C[(int64_t)i * ldc + j] =
            j < n2 ? alpha * expf(-acc[0][r][c]) + (1.f - alpha) * expf(-acc[1][r][c])
                   : 0.f;
    }
  }
}

fa_status launch_node_cost_simt(int n1, int n2, int L, int64_t ldr,
                                const float* R1, const float* R2, int d,
                                int64_t ldx, const float* X1h,
                                const float* X2h, float alpha, float* C,
                                int64_t ldc, cudaStream_t s) {
  dim3 grid((unsigned)(ldc / 64), (unsigned)((n1 + 63) / 64));
  k_node_cost_simt<<<grid, 256, 0, s>>>(n1, n2, L, ldr, R1, R2, d, ldx, X1h,
                                        X2h, alpha, C, ldc);
  FA_LAUNCHED("k_node_cost_simt");
  return FA_OK;
}

}  // namespace fa
