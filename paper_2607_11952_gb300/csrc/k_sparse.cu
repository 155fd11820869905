// Sparse x dense kernels of FastAlign (Section 3.3, "sparsity-aware"):
//   - RWR positional encoding, Algorithm 1 (SpMM with a tall-skinny dense R)
//   - SDDMM for the intra-network costs C1, C2, Algorithm 1
//   - the "SpMM on a wide dense matrix" pair  Z = P1 . D . P2^T
//     (Section 3.4; Algorithm 1 propagation, edge and neighbourhood costs), split into
//       left:  W  = P1 D   (row gathers of D, stored transposed as W^T)
//       right: Z  = W P2^T (row gathers of W^T), with a fused epilogue that
//              either stores Z (C_node propagation, Algorithm 1) or assembles
//              the cost (Algorithm 1 cost assembly, Eq. 2) and the log Gibbs kernel of the
//              proximal step.
// Storing the left product transposed turns both halves of the triple
// product into coalesced row gathers; the CTA order keeps one column panel
// of the gathered operand resident in L2 while every row tile uses it (the
// GPU form of the paper's column-blocked SpMM, Section 3.4).
#include <math.h>

#include <stdlib.h>

#include "fa_internal.cuh"

namespace fa {

// ------------------------------------------------------------ small helpers
__global__ void k_fill(float* p, int64_t n, float v) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < n; i += stride) p[i] = v;
}

fa_status launch_fill(float* p, int64_t n, float v, cudaStream_t s) {
  if (n <= 0) return FA_OK;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_fill<<<(unsigned)blocks, 256, 0, s>>>(p, n, v);
  FA_LAUNCHED("k_fill");
  return FA_OK;
}

__global__ void k_exp_vec(int n, const float* __restrict__ x, float* __restrict__ y) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = expf(x[i]);
}

fa_status launch_exp_vec(int n, const float* x, float* y, cudaStream_t s) {
  if (n <= 0) return FA_OK;
  k_exp_vec<<<(n + 255) / 256, 256, 0, s>>>(n, x, y);
  FA_LAUNCHED("k_exp_vec");
  return FA_OK;
}

// ------------------------------------------------------------ RWR (Algorithm 1)
// Rout[i,:] = (1-beta) sum_k Abar[i,k] Rin[k,:]; the beta R^(0) term is
// added afterwards by k_add_onehot.  Column panels of 128 (one float4 per
// lane), one warp per row, four neighbour gathers in flight; blockIdx.x runs
// over rows first, so one panel of Rin (n x 128 floats) stays in L2 while
// every row uses it instead of whole rows of Rin being re-read from HBM.
__global__ void __launch_bounds__(256) k_rwr_step(
    int n, int L, int64_t ldr, const int32_t* __restrict__ rp,
    const int32_t* __restrict__ ci, const float* __restrict__ val, float c,
    const float* __restrict__ Rin, float* __restrict__ Rout) {
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const int64_t nv = ldr / 4;
  const int64_t c4 = (int64_t)blockIdx.y * 32 + lane;
  if (row >= n || c4 >= nv) return;
  const int e0 = rp[row], e1 = rp[row + 1];
  const float4* Rv = reinterpret_cast<const float4*>(Rin) + c4;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  int e = e0;
  for (; e + 4 <= e1; e += 4) {
    float w[4];
    float4 r[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      w[u] = val[e + u];
      r[u] = __ldg(Rv + (int64_t)ci[e + u] * nv);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      acc.x = fmaf(w[u], r[u].x, acc.x); acc.y = fmaf(w[u], r[u].y, acc.y);
      acc.z = fmaf(w[u], r[u].z, acc.z); acc.w = fmaf(w[u], r[u].w, acc.w);
    }
  }
  for (; e < e1; ++e) {
    const float w = val[e];
    const float4 r = __ldg(Rv + (int64_t)ci[e] * nv);
    acc.x = fmaf(w, r.x, acc.x); acc.y = fmaf(w, r.y, acc.y);
    acc.z = fmaf(w, r.z, acc.z); acc.w = fmaf(w, r.w, acc.w);
  }
  acc.x *= c; acc.y *= c; acc.z *= c; acc.w *= c;
  reinterpret_cast<float4*>(Rout + (int64_t)row * ldr)[c4] = acc;
}

fa_status launch_rwr_step(const DevGraph& g, int L, int64_t ldr, float beta,
                          const float* Rin, float* Rout, cudaStream_t s) {
  if (g.n <= 0) return FA_OK;
  dim3 grid((unsigned)((g.n + 7) / 8), (unsigned)((ldr / 4 + 31) / 32));
  k_rwr_step<<<grid, 256, 0, s>>>(g.n, L, ldr, g.row_ptr, g.col, g.val_row, 1.0f - beta,
                                  Rin, Rout);
  FA_LAUNCHED("k_rwr_step");
  return FA_OK;
}

// R[nodes[l], l] += value  (the beta R^(0) term; R^(0) is one-hot, Algorithm 1)
__global__ void k_add_onehot(int L, int64_t ldr, const int32_t* __restrict__ nodes,
                             float value, float* __restrict__ R) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < L) R[(int64_t)nodes[l] * ldr + l] += value;
}

fa_status launch_add_onehot(int L, int64_t ldr, const int32_t* nodes,
                            float value, float* R, cudaStream_t s) {
  if (L <= 0) return FA_OK;
  k_add_onehot<<<(L + 255) / 256, 256, 0, s>>>(L, ldr, nodes, value, R);
  FA_LAUNCHED("k_add_onehot");
  return FA_OK;
}

fa_status launch_onehot(int n, int L, int64_t ldr, const int32_t* nodes,
                        float* R, cudaStream_t s) {
  FA_TRY(launch_fill(R, (int64_t)n * ldr, 0.0f, s));
  return launch_add_onehot(L, ldr, nodes, 1.0f, R, s);
}

// ------------------------------------------------------------ SDDMM (Algorithm 1)
// out[e] = w[e] * <R[i,:], R[k,:]> for every stored entry e = (i, k); w is
// Abar (1/deg i) for C1 = (R1 R1^T) .* Abar1 or Abar^T (1/deg k) for
// C2 = (R2 R2^T) .* Abar2^T.  One warp per row, lanes over the L columns.
__global__ void __launch_bounds__(256) k_sddmm(
    int n, int64_t ldr, const int32_t* __restrict__ rp,
    const int32_t* __restrict__ ci, const float* __restrict__ w,
    const float* __restrict__ R, float* __restrict__ out) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= n) return;
  const int nv = (int)(ldr / 4);
  const float4* ri = reinterpret_cast<const float4*>(R + (int64_t)warp * ldr);
  for (int e = rp[warp]; e < rp[warp + 1]; ++e) {
    const float4* rk = reinterpret_cast<const float4*>(R + (int64_t)ci[e] * ldr);
    float acc = 0.f;
    for (int c0 = lane; c0 < nv; c0 += 32) {
      float4 a = __ldg(ri + c0), b = __ldg(rk + c0);
      acc += a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[e] = w[e] * acc;
  }
}

// The dot products run over all ldr columns of R: the padding columns past
// the L anchors stay 0 through the RWR, so they add nothing.
fa_status launch_sddmm(const DevGraph& g, int /*L*/, int64_t ldr, const float* R,
                       bool weight_by_col, float* out, cudaStream_t s) {
  if (g.nnz == 0) return FA_OK;
  int64_t threads = (int64_t)g.n * 32;
  k_sddmm<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
      g.n, ldr, g.row_ptr, g.col, weight_by_col ? g.val_col : g.val_row, R, out);
  FA_LAUNCHED("k_sddmm");
  return FA_OK;
}

// ------------------------------------------------------------ attributes
// Xh[i,:] = X[i,:] / |X[i,:]|_2 (or a plain copy), zero rows stay zero,
// padding columns [d, ldx) set to 0.  One warp per row.
__global__ void k_normalize_rows(int n, int d, const float* __restrict__ X,
                                 int64_t ldx, int normalize,
                                 float* __restrict__ Xh) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= n) return;
  const float* x = X + (int64_t)warp * d;
  float ss = 0.f;
  for (int c = lane; c < d; c += 32) ss += x[c] * x[c];
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  float scale = 1.0f;
  if (normalize) scale = ss > 0.f ? 1.0f / sqrtf(ss) : 0.f;
  for (int c = lane; c < ldx; c += 32)
    Xh[(int64_t)warp * ldx + c] = c < d ? x[c] * scale : 0.f;
}

fa_status launch_normalize_rows(int n, int d, const float* X, int64_t ldx,
                                bool normalize, float* Xh, cudaStream_t s) {
  int64_t threads = (int64_t)n * 32;
  k_normalize_rows<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
      n, d, X, ldx, normalize ? 1 : 0, Xh);
  FA_LAUNCHED("k_normalize_rows");
  return FA_OK;
}

// ------------------------------------------------------------ left SpMM
// W^T[j, i] = sum_k P[i,k] s_k D[k, j]  for NV value sets P in {va, vb}.
// CTA tile: 32 rows i x 128 columns j.  The tile's neighbour lists are one
// contiguous CSR range [rp[i0], rp[i0+32]), split evenly over the 8 warps by
// edge count, so high-degree rows are shared and warps finish together.  A
// warp loads 32 edges at a time lane-parallel (neighbour k, weights times
// s_k, output row by binary search in the tile's row pointers), broadcasts
// them and keeps kGU row gathers of D[k, j0:j0+128] in flight (lane l:
// columns 4l..4l+3, 256 B per gather in BF16, 512 B in FP32).  A finished row
// goes to a shared-memory tile; a row split between warps (at most the first
// and the last row of a warp's range) leaves one partial per warp in that
// warp's head or tail slot, added in warp order afterwards, so the sums
// are formed in a fixed order without atomics.  The tile is then stored
// transposed, 32 consecutive i per column j (NV floats per element).  blockIdx.x runs over row tiles first, so all row
// tiles of one 128-column panel of D run back-to-back and the panel
// (n1 x 128 elements) stays in L2.
constexpr int kGU = 8;     // gathers in flight per warp

// Largest t in [0, n) with p[t] <= e, for p[0] <= e < p[n] (p nondecreasing).
template <int N>
__device__ __forceinline__ int seg_of(const int* p, int e) {
  int lo = 0, hi = N;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (p[mid] <= e) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ float4 load_quad(const float* p) {
  return __ldg(reinterpret_cast<const float4*>(p));
}
__device__ __forceinline__ float4 load_quad(const __nv_bfloat16* p) {
  const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
  return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                     __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
}

// One CSR edge as a warp stages it: neighbour (gathered row), output row or
// column within the tile, and the two weights times the neighbour's scaling.
struct EdgeRec {
  int nb, seg;
  float wa, wb;
};
__device__ __forceinline__ EdgeRec lds_edge(const EdgeRec* p) {
  const int4 v = *reinterpret_cast<const int4*>(p);
  return EdgeRec{v.x, v.y, __int_as_float(v.z), __int_as_float(v.w)};
}

template <typename TD, int NV>
__global__ void __launch_bounds__(256) k_spmm_left_T(
    int n1, int n2, int64_t ldd, int64_t ldw, const int32_t* __restrict__ rp,
    const int32_t* __restrict__ ci, const float* __restrict__ va,
    const float* __restrict__ vb, const float* __restrict__ scale,
    const TD* __restrict__ D, float* __restrict__ Wt) {
  constexpr int TI = 32, TJ = 128;
  // tile row stride (floats): a multiple of 4 so a lane's 4 columns are
  // 16-byte stores; the +4 (+2 words per 64-bit read) spreads the banks of
  // the transposed read over a half warp
  constexpr int RS = TJ * NV + 4;
  __shared__ __align__(16) float tile[TI * RS];
  __shared__ __align__(16) float split_s[8][2][TJ * NV];   // [warp][head/tail][columns]
  __shared__ int split_row[8][2];                          // row of each slot, -1 if unused
  __shared__ __align__(16) EdgeRec edges[8][32];
  __shared__ int rps[TI + 1];
  const int i0 = blockIdx.x * TI;
  const int j0 = blockIdx.y * TJ;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int t = threadIdx.x; t < TI * RS / 4; t += blockDim.x)
    reinterpret_cast<float4*>(tile)[t] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (threadIdx.x <= TI) rps[threadIdx.x] = rp[min(i0 + (int)threadIdx.x, n1)];
  if (threadIdx.x < 16) split_row[threadIdx.x >> 1][threadIdx.x & 1] = -1;
  __syncthreads();
  {
    const int E0 = rps[0], len = rps[TI] - E0;
    const int eb = E0 + (int)((int64_t)len * warp / 8);
    const int ee = E0 + (int)((int64_t)len * (warp + 1) / 8);
    const TD* dcol = D + j0 + 4 * lane;
    EdgeRec* my = edges[warp];
    int cur = -1;
    float acc[4][NV];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[c][v] = 0.f;
    auto flush = [&]() {
      if (cur >= 0) {
        float* dst = tile + cur * RS + 4 * lane * NV;
        const bool starts_before = rps[cur] < eb, ends_after = rps[cur + 1] > ee;
        if (starts_before || ends_after) {   // row split with another warp: a slot
          const int slot = starts_before ? 0 : 1;
          float* sp = &split_s[warp][slot][4 * lane * NV];
#pragma unroll
          for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int v = 0; v < NV; ++v) sp[c * NV + v] = acc[c][v];
          if (lane == 0) split_row[warp][slot] = cur;
        } else if constexpr (NV == 2) {
          reinterpret_cast<float4*>(dst)[0] = make_float4(acc[0][0], acc[0][1], acc[1][0], acc[1][1]);
          reinterpret_cast<float4*>(dst)[1] = make_float4(acc[2][0], acc[2][1], acc[3][0], acc[3][1]);
        } else {
          reinterpret_cast<float4*>(dst)[0] = make_float4(acc[0][0], acc[1][0], acc[2][0], acc[3][0]);
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[c][v] = 0.f;
    };
    for (int base = eb; base < ee; base += 32) {
      const int e = base + lane;
      if (e < ee) {
        const int k = ci[e];
        const float sk = scale ? scale[k] : 1.f;
        my[lane] = EdgeRec{k, seg_of<TI>(rps, e), va[e] * sk, NV == 2 ? vb[e] * sk : 0.f};
      }
      __syncwarp();
      const int cnt = min(32, ee - base);
      for (int u = 0; u < cnt; u += kGU) {
        float4 d[kGU];
#pragma unroll
        for (int g = 0; g < kGU; ++g)
          if (u + g < cnt) d[g] = load_quad(dcol + (int64_t)my[u + g].nb * ldd);
#pragma unroll
        for (int g = 0; g < kGU; ++g) {
          if (u + g < cnt) {
            const EdgeRec er = lds_edge(&my[u + g]);
            if (er.seg != cur) {
              flush();
              cur = er.seg;
            }
            const float dv[4] = {d[g].x, d[g].y, d[g].z, d[g].w};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              acc[c][0] = fmaf(er.wa, dv[c], acc[c][0]);
              if constexpr (NV == 2) acc[c][NV - 1] = fmaf(er.wb, dv[c], acc[c][NV - 1]);
            }
          }
        }
      }
      __syncwarp();
    }
    flush();
  }
  __syncthreads();
  // split rows: the warps' partials in warp order (head before tail)
  for (int k = threadIdx.x; k < TJ * NV; k += blockDim.x) {
    int row = -1;
    float z = 0.f;
    for (int w = 0; w < 8; ++w) {
#pragma unroll
      for (int sl = 0; sl < 2; ++sl) {
        const int r = split_row[w][sl];
        if (r < 0) continue;
        if (r != row) {
          if (row >= 0) tile[row * RS + k] = z;
          row = r;
          z = 0.f;
        }
        z += split_s[w][sl][k];
      }
    }
    if (row >= 0) tile[row * RS + k] = z;
  }
  __syncthreads();
  // transposed store: warp w writes columns c = w, w+8, ...; lane = row
  for (int c = warp; c < TJ; c += 8) {
    const int j = j0 + c;
    if (j >= n2) break;
    if constexpr (NV == 1) {
      Wt[(int64_t)j * ldw + i0 + lane] = tile[lane * RS + c];
    } else {
      reinterpret_cast<float2*>(Wt + ((int64_t)j * ldw + i0) * 2)[lane] =
          *reinterpret_cast<const float2*>(&tile[lane * RS + 2 * c]);
    }
  }
}

template <int NV> struct VecF;
template <> struct VecF<1> { using T = float; };
template <> struct VecF<2> { using T = float2; };

// Row form of the left product, transposed store: CTA tile of 32 rows i by
// 128 columns j; warp per row (4 rows per warp in turn), lane l covers
// columns 4l .. 4l+3 of the tile, and kRowGathers neighbour rows
// D[k, j0:j0+128] are in flight per warp (8 B per lane and gather in BF16,
// 16 B in FP32).  Each output sums its row's edges in CSR order, so the
// result does not depend on the tile shape.  Used for Pass A's two value
// sets; FA_PASSA_ROWS=1 selects it for one value set too.
constexpr int kRowGathers = 8;

template <typename TD, int NV, int MINB>
__global__ void __launch_bounds__(256, MINB) k_spmm_left_T_rows(
    int n1, int n2, int64_t ldd, int64_t ldw, const int32_t* __restrict__ rp,
    const int32_t* __restrict__ ci, const float* __restrict__ va,
    const float* __restrict__ vb, const float* __restrict__ scale,
    const TD* __restrict__ D, float* __restrict__ Wt) {
  constexpr int TI = 32, TJ = 128, PAD = (NV == 1) ? 1 : 2, NG = kRowGathers;
  __shared__ float tile[TI][TJ * NV + PAD];
  const int i0 = blockIdx.x * TI;
  const int j0 = blockIdx.y * TJ;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const TD* dcol = D + j0 + 4 * lane;
#pragma unroll 1
  for (int rr = 0; rr < 4; ++rr) {
    const int r = warp * 4 + rr;
    const int i = i0 + r;
    float acc[4][NV];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[c][v] = 0.f;
    if (i < n1) {
      const int e0 = rp[i], e1 = rp[i + 1];
      int e = e0;
      for (; e + NG <= e1; e += NG) {
        int k[NG];
        float4 d[NG];
        float w[NG], x[NG];
#pragma unroll
        for (int u = 0; u < NG; ++u) k[u] = ci[e + u];
#pragma unroll
        for (int u = 0; u < NG; ++u) d[u] = load_quad(dcol + (int64_t)k[u] * ldd);
#pragma unroll
        for (int u = 0; u < NG; ++u) {
          const float su = scale ? scale[k[u]] : 1.f;
          w[u] = va[e + u] * su;
          x[u] = NV == 2 ? vb[e + u] * su : 0.f;
        }
#pragma unroll
        for (int u = 0; u < NG; ++u) {
          const float dv[4] = {d[u].x, d[u].y, d[u].z, d[u].w};
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            acc[c][0] = fmaf(w[u], dv[c], acc[c][0]);
            if (NV == 2) acc[c][NV - 1] = fmaf(x[u], dv[c], acc[c][NV - 1]);
          }
        }
      }
      for (; e < e1; ++e) {
        const int k0 = ci[e];
        const float s0 = scale ? scale[k0] : 1.f;
        const float4 d0 = load_quad(dcol + (int64_t)k0 * ldd);
        const float dv[4] = {d0.x, d0.y, d0.z, d0.w};
        const float w0 = va[e] * s0;
        const float x0 = NV == 2 ? vb[e] * s0 : 0.f;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          acc[c][0] = fmaf(w0, dv[c], acc[c][0]);
          if (NV == 2) acc[c][NV - 1] = fmaf(x0, dv[c], acc[c][NV - 1]);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int v = 0; v < NV; ++v) tile[r][(4 * lane + c) * NV + v] = acc[c][v];
  }
  __syncthreads();
  // transposed store: warp w writes columns c = w, w+8, ...; lane = row
  using VT = typename VecF<NV>::T;
  for (int c = warp; c < TJ; c += 8) {
    const int j = j0 + c;
    if (j >= n2) break;
    VT* dst = reinterpret_cast<VT*>(Wt + ((int64_t)j * ldw + i0) * NV);
    if constexpr (NV == 1) {
      dst[lane] = tile[lane][c];
    } else {
      dst[lane] = make_float2(tile[lane][c * 2], tile[lane][c * 2 + 1]);
    }
  }
}

fa_status launch_spmm_left_T(const DevGraph& g1, int n2, int64_t ldd,
                             int64_t ldw, const float* va, const float* vb,
                             const float* scale, const void* D, bool d_bf16,
                             float* Wt, cudaStream_t s) {
  const bool two = vb != nullptr;
  // measured at 50k on GB300: the row-per-warp form is faster for the two
  // value sets of Pass A in BF16 (14 vs 22 ms) and takes them always; for
  // one value set (propagation) the forms were equal and FA_PASSA_ROWS=1
  // selects the row form
  static const int form = [] {
    const char* v = getenv("FA_PASSA_ROWS");
    return v ? atoi(v) : -1;
  }();
  if (form == 1 || two) {
    dim3 g2d((unsigned)((g1.n + 31) / 32), (unsigned)((n2 + 127) / 128));
    // 4 CTAs per SM (64 registers, a 32-byte spill in the BF16 two-set
    // form) measured 48.7 ms per 50k outer iteration against 49.4 ms for 3
    // (80 registers); FA_PASSA_MINB=3 selects 3 (tuning)
    const char* mb = getenv("FA_PASSA_MINB");
    const bool four = !(mb && atoi(mb) == 3);
#define FA_PA(T, NVV)                                                                      \
    if (four) k_spmm_left_T_rows<T, NVV, 4><<<g2d, 256, 0, s>>>(g1.n, n2, ldd, ldw, g1.row_ptr, \
                                                                g1.col, va, vb, scale, Dp, Wt); \
    else k_spmm_left_T_rows<T, NVV, 3><<<g2d, 256, 0, s>>>(g1.n, n2, ldd, ldw, g1.row_ptr,      \
                                                           g1.col, va, vb, scale, Dp, Wt);
    if (d_bf16) {
      auto* Dp = static_cast<const __nv_bfloat16*>(D);
      if (two) { FA_PA(__nv_bfloat16, 2) } else { FA_PA(__nv_bfloat16, 1) }
    } else {
      auto* Dp = static_cast<const float*>(D);
      if (two) { FA_PA(float, 2) } else { FA_PA(float, 1) }
    }
#undef FA_PA
    FA_LAUNCHED("k_spmm_left_T_rows");
    return FA_OK;
  }
  dim3 grid((unsigned)((g1.n + 31) / 32), (unsigned)((n2 + 127) / 128));
  if (d_bf16)
    k_spmm_left_T<__nv_bfloat16, 1><<<grid, 256, 0, s>>>(g1.n, n2, ldd, ldw, g1.row_ptr, g1.col, va, vb, scale,
                                                         static_cast<const __nv_bfloat16*>(D), Wt);
  else
    k_spmm_left_T<float, 1><<<grid, 256, 0, s>>>(g1.n, n2, ldd, ldw, g1.row_ptr, g1.col, va, vb, scale,
                                                 static_cast<const float*>(D), Wt);
  FA_LAUNCHED("k_spmm_left_T");
  return FA_OK;
}

// ------------------------------------------------------------ right SpMM
// Z[i, j] = sum_{l in N2(j)} Q[j,l] s_l W^T[l, i].  CTA tile: 64 columns j x
// 32 rows i; warp w owns columns j0+8w..j0+8w+7, lane = row offset, so each
// neighbour l is one coalesced 128/256-byte gather of W^T[l, i0:i0+32] and
// every lane ends up holding 8 consecutive outputs of its own row -- the
// epilogue needs no transpose.  blockIdx.x runs over column tiles first so
// the W^T panel of one row tile (n2 x 32 elements) stays in L2.
template <int NV>
__device__ __forceinline__ void right_accumulate(
    int j, int n2, int64_t ldw, int i0, int lane,
    const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
    const float* __restrict__ qa, const float* __restrict__ qb,
    const float* __restrict__ scale, const float* __restrict__ Wt,
    float& za, float& zb) {
  za = 0.f;
  zb = 0.f;
  if (j >= n2) return;
  const int e0 = rp[j], e1 = rp[j + 1];
  const float* base = Wt + (int64_t)(i0 + lane) * NV;
  int e = e0;
  for (; e + 2 <= e1; e += 2) {
    const int l0 = ci[e], l1 = ci[e + 1];
    const float s0 = scale ? scale[l0] : 1.f, s1 = scale ? scale[l1] : 1.f;
    if constexpr (NV == 1) {
      float w0 = __ldg(base + (int64_t)l0 * ldw);
      float w1 = __ldg(base + (int64_t)l1 * ldw);
      za += qa[e] * s0 * w0 + qa[e + 1] * s1 * w1;
    } else {
      float2 w0 = __ldg(reinterpret_cast<const float2*>(base + (int64_t)l0 * ldw * 2));
      float2 w1 = __ldg(reinterpret_cast<const float2*>(base + (int64_t)l1 * ldw * 2));
      za += qa[e] * s0 * w0.x + qa[e + 1] * s1 * w1.x;
      zb += qb[e] * s0 * w0.y + qb[e + 1] * s1 * w1.y;
    }
  }
  for (; e < e1; ++e) {
    const int l0 = ci[e];
    const float s0 = scale ? scale[l0] : 1.f;
    if constexpr (NV == 1) {
      za += qa[e] * s0 * __ldg(base + (int64_t)l0 * ldw);
    } else {
      float2 w0 = __ldg(reinterpret_cast<const float2*>(base + (int64_t)l0 * ldw * 2));
      za += qa[e] * s0 * w0.x;
      zb += qb[e] * s0 * w0.y;
    }
  }
}

// C_node propagation (Algorithm 1): plain store of Z.
__global__ void __launch_bounds__(256) k_spmm_right_prop(
    int n1, int n2, int64_t ldw, const int32_t* __restrict__ rp,
    const int32_t* __restrict__ ci, const float* __restrict__ qa,
    const float* __restrict__ Wt, float* __restrict__ C, int64_t ldc) {
  const int j0 = blockIdx.x * 64, i0 = blockIdx.y * 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int jb = j0 + warp * 8;
  float z[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    float zb;
    right_accumulate<1>(jb + q, n2, ldw, i0, lane, rp, ci, qa, nullptr,
                        nullptr, Wt, z[q], zb);
  }
  const int i = i0 + lane;
  if (i < n1) {
    float4* dst = reinterpret_cast<float4*>(C + (int64_t)i * ldc + jb);
    dst[0] = make_float4(z[0], z[1], z[2], z[3]);
    dst[1] = make_float4(z[4], z[5], z[6], z[7]);
  }
}

fa_status launch_spmm_right_prop(const DevGraph& g2, int n1, int64_t ldw,
                                 const float* qa, const float* Wt, float* C,
                                 int64_t ldc, cudaStream_t s) {
  dim3 grid((unsigned)(ldc / 64), (unsigned)((n1 + 31) / 32));
  k_spmm_right_prop<<<grid, 256, 0, s>>>(n1, g2.n, ldw, g2.row_ptr, g2.col,
                                         qa, Wt, C, ldc);
  FA_LAUNCHED("k_spmm_right_prop");
  return FA_OK;
}

// Cost assembly + log Gibbs kernel (Phase 2 of Algorithm 1, Eq. 2, proximal step):
//   C   = C_node + lam_e Z_e - lam_n log max(Z_n, delta) + lam_a C_anc
//   x   = -C/eps + (lam_p/eps) (log u_i + log K_prev_ij + log v_j)
// stored as float32, plus the per-(row, 64-column tile) maximum of x.
__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }

// CTA tile: 64 columns j x 64 rows i.  The tile's neighbour lists are one
// contiguous CSR range [rp[j0], rp[j0+64]); it is split evenly over the 8
// warps by edge count (not by column), so a hub column's gathers are shared
// and the warps of a CTA finish together.  A warp loads 32 edges at a time
// lane-parallel (column index, both weights times the scaling s_l, and the
// output column found by binary search in the tile's row pointers), then
// broadcasts them and keeps GU gathers of W^T[l, i0:i0+64] (one float4 per
// lane: rows 2 lane, 2 lane + 1, both value sets) in flight.  The sums are
// formed without atomics, in a fixed order: a column whose edges lie
// wholly in one warp's range is stored into the shared tile by that warp;
// a column split between warps (at most the first and the last column of a
// warp's range) leaves one partial per warp in that warp's head or tail
// slot, and the epilogue adds a split column's partials in warp order.  The
// epilogue walks rows, lanes over columns, so the C_node, K_prev and X rows
// are coalesced.  Shared tiles are XOR-swizzled by row so both the stores
// (lanes over rows) and the epilogue (lanes over columns) are free of bank
// conflicts up to 2 ways.  Two runs give bit-identical results.
constexpr int kRT = 64;    // rows per tile
constexpr int kCT = 64;    // columns per tile

__device__ __forceinline__ int sw_idx(int r, int c) { return r * kCT + (c ^ (r & 31)); }

template <typename TK, int MINB, int GU>
__global__ void __launch_bounds__(256, MINB) k_spmm_right_cost(
    int n1, int n2, int64_t ldw, int64_t ldo, const int32_t* __restrict__ rp,
    const int32_t* __restrict__ ci, const float* __restrict__ qa,
    const float* __restrict__ qb, const float* __restrict__ scale,
    const float* __restrict__ Wt, CostEpi ep) {
  __shared__ float ze_s[kRT * kCT];
  __shared__ float zn_s[kRT * kCT];
  __shared__ __align__(16) float4 split_s[8][2][kRT / 2];   // [warp][head/tail][lane]: a0 b0 a1 b1
  __shared__ int split_col[8][2];                            // column of each slot, -1 if unused
  __shared__ __align__(16) EdgeRec edges[8][32];
  __shared__ int rps[kCT + 1];
  const int j0 = blockIdx.x * kCT, i0 = blockIdx.y * kRT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int t = threadIdx.x; t < kRT * kCT; t += blockDim.x) {
    ze_s[t] = 0.f;
    zn_s[t] = 0.f;
  }
  if (threadIdx.x <= kCT) rps[threadIdx.x] = rp[min(j0 + (int)threadIdx.x, n2)];
  if (threadIdx.x < 16) split_col[threadIdx.x >> 1][threadIdx.x & 1] = -1;
  __syncthreads();

  // ---- gathers: Z_e[i, j] and Z_n[i, j] for rows 2 lane, 2 lane + 1
  {
    const int E0 = rps[0], len = rps[kCT] - E0;
    const int eb = E0 + (int)((int64_t)len * warp / 8);
    const int ee = E0 + (int)((int64_t)len * (warp + 1) / 8);
    const int r0 = 2 * lane, r1 = 2 * lane + 1;
    const float* wbase = Wt + (int64_t)(i0 + r0) * 2;
    int cur = -1;
    float a0 = 0.f, b0 = 0.f, a1 = 0.f, b1 = 0.f;
    auto flush = [&]() {
      if (cur >= 0) {
        const bool starts_before = rps[cur] < eb, ends_after = rps[cur + 1] > ee;
        if (!starts_before && !ends_after) {   // the whole column is this warp's
          ze_s[sw_idx(r0, cur)] = a0;
          zn_s[sw_idx(r0, cur)] = b0;
          ze_s[sw_idx(r1, cur)] = a1;
          zn_s[sw_idx(r1, cur)] = b1;
        } else {                               // split: head (first) or tail slot
          const int slot = starts_before ? 0 : 1;
          split_s[warp][slot][lane] = make_float4(a0, b0, a1, b1);
          if (lane == 0) split_col[warp][slot] = cur;
        }
      }
      a0 = b0 = a1 = b1 = 0.f;
    };
    EdgeRec* my = edges[warp];
    for (int base = eb; base < ee; base += 32) {
      const int e = base + lane;
      if (e < ee) {
        const int l = ci[e];
        const float sl = scale ? scale[l] : 1.f;
        my[lane] = EdgeRec{l, seg_of<kCT>(rps, e), qa[e] * sl, qb[e] * sl};
      }
      __syncwarp();
      const int cnt = min(32, ee - base);
      for (int u = 0; u < cnt; u += GU) {
        float4 w[GU];
#pragma unroll
        for (int k = 0; k < GU; ++k)
          if (u + k < cnt)
            w[k] = __ldg(reinterpret_cast<const float4*>(wbase + (int64_t)my[u + k].nb * ldw * 2));
#pragma unroll
        for (int k = 0; k < GU; ++k) {
          if (u + k < cnt) {
            const EdgeRec er = lds_edge(&my[u + k]);
            if (er.seg != cur) {
              flush();
              cur = er.seg;
            }
            a0 = fmaf(er.wa, w[k].x, a0);
            b0 = fmaf(er.wb, w[k].y, b0);
            a1 = fmaf(er.wa, w[k].z, a1);
            b1 = fmaf(er.wb, w[k].w, b1);
          }
        }
      }
      __syncwarp();
    }
    flush();
  }
  __syncthreads();
  // ---- split columns: the warps' partials in warp order (head before
  // tail within a warp: a warp's head column precedes its tail column)
  {
    if (threadIdx.x < kRT) {
      const int row = threadIdx.x, ln = row >> 1, hi = row & 1;
      int col = -1;
      float za = 0.f, zb = 0.f;
      for (int w = 0; w < 8; ++w) {
#pragma unroll
        for (int sl = 0; sl < 2; ++sl) {
          const int c = split_col[w][sl];
          if (c < 0) continue;
          if (c != col) {
            if (col >= 0) {
              ze_s[sw_idx(row, col)] = za;
              zn_s[sw_idx(row, col)] = zb;
            }
            col = c;
            za = zb = 0.f;
          }
          const float4 v = split_s[w][sl][ln];
          za += hi ? v.z : v.x;
          zb += hi ? v.w : v.y;
        }
      }
      if (col >= 0) {
        ze_s[sw_idx(row, col)] = za;
        zn_s[sw_idx(row, col)] = zb;
      }
    }
  }
  __syncthreads();

  // ---- epilogue: rows over warps, columns j0 + lane and j0 + 32 + lane
  const float inv_eps = 1.0f / ep.eps;
  const float prox = ep.lam_p * inv_eps;
  const float c_off = -logf(ep.eps_anc);          // C_anc off the anchors
  const float c_on = -logf(ep.eps_anc + 1.0f);    // C_anc on an anchor
  const TK* Kp = static_cast<const TK*>(ep.K_prev);
  for (int r = warp; r < kRT; r += 8) {
    const int i = i0 + r;
    if (i >= n1) break;
    const float lu = ep.log_u[i];
    const int a0 = ep.anc_ptr[i], a1 = ep.anc_ptr[i + 1];
    const int64_t row = (int64_t)i * ldo;
    float mx = -INFINITY;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = lane + 32 * h, j = j0 + c;
      float x = -INFINITY;
      if (j < n2) {
        const int si = sw_idx(r, c);
        float canc = c_off;
        for (int a = a0; a < a1; ++a)
          if (ep.anc_col[a] == j) canc = c_on;
        const float C = ep.C_node[row + j] + ep.lam_e * ze_s[si] -
                        ep.lam_n * logf(fmaxf(zn_s[si], ep.delta)) + ep.lam_a * canc;
        x = -C * inv_eps;
        if (prox != 0.f) x += prox * (lu + logf(to_f32(Kp[row + j])) + ep.log_v[j]);
        mx = fmaxf(mx, x);
      }
      ep.X[row + j] = x;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) ep.rowmax_part[(int64_t)blockIdx.x * n1 + i] = mx;
  }
}

fa_status launch_spmm_right_cost(const DevGraph& g2, int n1, int64_t ldw,
                                 int64_t ldo, const float* qa, const float* qb,
                                 const float* scale, const float* Wt,
                                 const CostEpi& ep, bool k_bf16,
                                 cudaStream_t s) {
  // resident CTAs per SM the register budget is sized for: 3 (80 registers)
  // measured faster than 2 (88) on GB300 at 10k and 50k
  // Resident CTAs per SM the register budget is sized for, and gathers in
  // flight per warp.  Measured on GB300 (one outer iteration, 50k BF16):
  // 5 CTAs x 4 gathers (48 registers; 5 x 45 KB of shared memory fit the
  // SM) 46.1 ms, 4 x 6 48.8 ms, 3 x 8 56.1 ms, 2 x 16 72.3 ms: the gathers'
  // latency is hidden by more warps, not by deeper warps.  FA_PASSB_MINB=4
  // or 3 selects those shapes (tuning).
  const char* mb = getenv("FA_PASSB_MINB");
  const int minb = (mb && atoi(mb) == 3) ? 3 : (mb && atoi(mb) == 4) ? 4 : 5;
  dim3 grid((unsigned)(ldo / kCT), (unsigned)((n1 + kRT - 1) / kRT));
#define FA_PB(T, M, GU) \
  k_spmm_right_cost<T, M, GU><<<grid, 256, 0, s>>>(n1, g2.n, ldw, ldo, g2.row_ptr, g2.col, qa, qb, scale, Wt, ep)
  if (k_bf16) {
    if (minb == 4) FA_PB(__nv_bfloat16, 4, 6); else if (minb == 5) FA_PB(__nv_bfloat16, 5, 4); else FA_PB(__nv_bfloat16, 3, 8);
  } else {
    if (minb == 4) FA_PB(float, 4, 6); else if (minb == 5) FA_PB(float, 5, 4); else FA_PB(float, 3, 8);
  }
#undef FA_PB
  FA_LAUNCHED("k_spmm_right_cost");
  return FA_OK;
}

// rowmax[i] = max over column tiles of the partial maxima.  An all -inf row
// (every entry underflowed) is reported and pinned to 0.
__global__ void k_rowmax_reduce(int n1, int ntiles, const float* __restrict__ part,
                                float* __restrict__ rowmax, int* status) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n1) return;
  float m = -INFINITY;
  for (int t = 0; t < ntiles; ++t) m = fmaxf(m, part[(int64_t)t * n1 + i]);
  if (!(m > -INFINITY) || isnan(m)) {
    atomicOr(status, ST_NUMERIC);
    m = 0.f;
  }
  rowmax[i] = m;
}

fa_status launch_rowmax_reduce(int n1, int ntiles, const float* part,
                               float* rowmax, int* status, cudaStream_t s) {
  k_rowmax_reduce<<<(n1 + 255) / 256, 256, 0, s>>>(n1, ntiles, part, rowmax, status);
  FA_LAUNCHED("k_rowmax_reduce");
  return FA_OK;
}

}  // namespace fa
