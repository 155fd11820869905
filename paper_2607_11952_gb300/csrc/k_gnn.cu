// Learned warm start for the Sinkhorn solves (not in the paper): a 2-layer
// graph network on the column graph G2 predicts the correction
// y = log v* - log v1 between the converged column scaling of a solve and
// its cold first column update, from per-node features.
//
//   AF = Abar F,  A1 = AF W1 + b1,  H = relu(A1),  z2 = H w2,
//   a  = Abar z2 + c
//   L  = 1/n sum_j ((a_j - mean a) - (y_j - mean y))^2     (gauge invariant)
//
// W1 and w2 are used in BF16 (FP32 master copies are updated by Adam); all
// accumulation is FP32.  Reductions over nodes are deterministic (per-block
// partials summed in a fixed order).  Parameter vector layout:
// W1 [FA_GNN_FIN x 64 row-major] | b1 [64] | w2 [64] | c.
#include <math.h>

#include "fa_internal.cuh"

namespace fa {

constexpr int kFin = FA_GNN_FIN;
constexpr int kHid = FA_GNN_HIDDEN;
constexpr int kNP = FA_GNN_NPARAMS;
constexpr int kOffB1 = kFin * kHid;
constexpr int kOffW2 = kOffB1 + kHid;
constexpr int kOffC = kOffW2 + kHid;

// workspace (floats): AF n*kFin | A1 n*64 | z2 n | g n | gz2 n | partials nb*kNP | scal 8
struct GnnWs {
  float *AF, *A1, *z2, *g, *gz2, *part, *scal;
  int nb;
};
constexpr int kGradThreads = 256;
static inline int grad_blocks(int n) {
  int nb = (n + 4 * (kGradThreads / 32) - 1) / (4 * (kGradThreads / 32));   // 4 nodes per warp
  return nb < 1 ? 1 : nb;
}
static GnnWs ws_layout(float* w, int n) {
  GnnWs s;
  s.AF = w;
  s.A1 = s.AF + (size_t)n * kFin;
  s.z2 = s.A1 + (size_t)n * kHid;
  s.g = s.z2 + n;
  s.gz2 = s.g + n;
  s.part = s.gz2 + n;
  s.nb = grad_blocks(n);
  s.scal = s.part + (size_t)s.nb * kNP;
  return s;
}
int64_t gnn_workspace_floats(int n) {
  return (int64_t)n * (kFin + kHid + 3) + (int64_t)grad_blocks(n) * kNP + 8;
}

// ------------------------------------------------------------ reductions
// one block: out[0] = mean of x; when y (z) != null, out[1] (out[2]) = mean
// of y (z)
__global__ void __launch_bounds__(1024) k_means(int n, const float* __restrict__ x,
                                                const float* __restrict__ y,
                                                const float* __restrict__ z, float* out) {
  __shared__ double sx[32], sy[32], sz[32];
  double ax = 0.0, ay = 0.0, az = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    ax += x[i];
    if (y) ay += y[i];
    if (z) az += z[i];
  }
  for (int o = 16; o > 0; o >>= 1) {
    ax += __shfl_xor_sync(0xffffffffu, ax, o);
    ay += __shfl_xor_sync(0xffffffffu, ay, o);
    az += __shfl_xor_sync(0xffffffffu, az, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sx[threadIdx.x >> 5] = ax;
    sy[threadIdx.x >> 5] = ay;
    sz[threadIdx.x >> 5] = az;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tx = 0.0, ty = 0.0, tz = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { tx += sx[w]; ty += sy[w]; tz += sz[w]; }
    out[0] = (float)(tx / n);
    if (y) out[1] = (float)(ty / n);
    if (z) out[2] = (float)(tz / n);
  }
}

// ------------------------------------------------------------ features
// F[j] = (log_v1_j - mean log_v1, corr_prev_j - mean corr_prev,
//         log(1 + deg_j), pot_prev_j - mean pot_prev, anchor_j, log(1 + t));
// the potentials are centred (they are defined up to a constant)
__global__ void k_gnn_features(int n, const int32_t* __restrict__ rp, const float* __restrict__ lv,
                               const float* __restrict__ corr, const float* __restrict__ pot,
                               const float* __restrict__ anc, float lt,
                               const float* __restrict__ mean, float* __restrict__ F) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  float* f = F + (size_t)j * kFin;
  f[0] = lv[j] - mean[0];
  f[1] = corr ? corr[j] - mean[1] : 0.f;
  f[2] = log1pf((float)(rp[j + 1] - rp[j]));
  f[3] = pot ? pot[j] - mean[2] : 0.f;
  f[4] = anc ? anc[j] : 0.f;
  f[5] = lt;
}

// ------------------------------------------------------------ forward
// AF[i] = sum_k Abar[i,k] F[k]  (thread per node)
__global__ void k_gnn_agg(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                          const float* __restrict__ val, const float* __restrict__ F,
                          float* __restrict__ AF) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float a[kFin];
#pragma unroll
  for (int f = 0; f < kFin; ++f) a[f] = 0.f;
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    const float w = val[e];
    const float* fk = F + (size_t)ci[e] * kFin;
#pragma unroll
    for (int f = 0; f < kFin; ++f) a[f] += w * fk[f];
  }
#pragma unroll
  for (int f = 0; f < kFin; ++f) AF[(size_t)i * kFin + f] = a[f];
}

// A1 = AF W1 + b1, z2 = relu(A1) w2  (warp per node, two hidden units per lane)
__global__ void __launch_bounds__(256) k_gnn_hidden(int n, const float* __restrict__ AF,
                                                    const __nv_bfloat16* __restrict__ W1,
                                                    const float* __restrict__ theta,
                                                    const __nv_bfloat16* __restrict__ w2,
                                                    float* __restrict__ A1, float* __restrict__ z2) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  float fi[kFin];
#pragma unroll
  for (int f = 0; f < kFin; ++f) fi[f] = AF[(size_t)i * kFin + f];
  float z = 0.f;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int h = lane + 32 * q;
    float a = theta[kOffB1 + h];
#pragma unroll
    for (int f = 0; f < kFin; ++f) a += fi[f] * __bfloat162float(W1[f * kHid + h]);
    A1[(size_t)i * kHid + h] = a;
    z += fmaxf(a, 0.f) * __bfloat162float(w2[h]);
  }
  for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
  if (lane == 0) z2[i] = z;
}

// out[i] = sum_k val[e] x[k] (+ theta[kOffC] when add_c)  (thread per node)
__global__ void k_gnn_spmv(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const float* __restrict__ val, const float* __restrict__ x,
                           const float* __restrict__ theta, int add_c, float* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.f;
  for (int e = rp[i]; e < rp[i + 1]; ++e) s += val[e] * x[ci[e]];
  out[i] = s + (add_c ? theta[kOffC] : 0.f);
}

// ------------------------------------------------------------ backward
// one block: residual r, g = 2 r / n, loss = mean r^2, dL/dc = sum g
__global__ void __launch_bounds__(1024) k_gnn_resid(int n, const float* __restrict__ a,
                                                    const float* __restrict__ y,
                                                    const float* __restrict__ means,
                                                    float* __restrict__ g, float* loss,
                                                    float* __restrict__ grad) {
  __shared__ double sl[32], sg[32];
  double al = 0.0, ag = 0.0;
  const float ma = means[0], my = means[1];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float r = (a[i] - ma) - (y[i] - my);
    const float gi = 2.f * r / (float)n;
    g[i] = gi;
    al += (double)r * r;
    ag += gi;
  }
  for (int o = 16; o > 0; o >>= 1) {
    al += __shfl_xor_sync(0xffffffffu, al, o);
    ag += __shfl_xor_sync(0xffffffffu, ag, o);
  }
  if ((threadIdx.x & 31) == 0) { sl[threadIdx.x >> 5] = al; sg[threadIdx.x >> 5] = ag; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tl = 0.0, tg = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { tl += sl[w]; tg += sg[w]; }
    if (loss) *loss = (float)(tl / n);
    grad[kOffC] = (float)tg;
  }
}

// per-block partial gradients of W1, b1, w2 (warp per node, 4 nodes per warp)
__global__ void __launch_bounds__(kGradThreads) k_gnn_grad_part(
    int n, const float* __restrict__ AF, const float* __restrict__ A1,
    const __nv_bfloat16* __restrict__ w2, const float* __restrict__ gz2, float* __restrict__ part) {
  __shared__ float red[kGradThreads / 32][kNP - 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float dW[kFin][2], db[2] = {0.f, 0.f}, dw[2] = {0.f, 0.f};
#pragma unroll
  for (int f = 0; f < kFin; ++f) dW[f][0] = dW[f][1] = 0.f;
  const float w2a = __bfloat162float(w2[lane]), w2b = __bfloat162float(w2[lane + 32]);
  const int base = (blockIdx.x * (kGradThreads / 32) + warp) * 4;
  for (int k = 0; k < 4; ++k) {
    const int i = base + k;
    if (i >= n) break;
    const float gi = gz2[i];
    float af[kFin];
#pragma unroll
    for (int f = 0; f < kFin; ++f) af[f] = AF[(size_t)i * kFin + f];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const float a = A1[(size_t)i * kHid + lane + 32 * q];
      const float h = fmaxf(a, 0.f);
      const float d = a > 0.f ? gi * (q == 0 ? w2a : w2b) : 0.f;
#pragma unroll
      for (int f = 0; f < kFin; ++f) dW[f][q] += af[f] * d;
      db[q] += d;
      dw[q] += gi * h;
    }
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int h = lane + 32 * q;
#pragma unroll
    for (int f = 0; f < kFin; ++f) red[warp][f * kHid + h] = dW[f][q];
    red[warp][kOffB1 + h] = db[q];
    red[warp][kOffW2 + h] = dw[q];
  }
  __syncthreads();
  for (int p = threadIdx.x; p < kNP - 1; p += blockDim.x) {
    float s = 0.f;
    for (int w = 0; w < kGradThreads / 32; ++w) s += red[w][p];
    part[(size_t)blockIdx.x * kNP + p] = s;
  }
}

__global__ void k_gnn_grad_reduce(int nb, const float* __restrict__ part, float* __restrict__ grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kNP - 1) return;
  float s = 0.f;
  for (int b = 0; b < nb; ++b) s += part[(size_t)b * kNP + p];
  grad[p] = s;
}

// ------------------------------------------------------------ optimiser
__global__ void k_gnn_adam(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ grad, float lr, float b1, float b2, float eps,
                           int step, __nv_bfloat16* __restrict__ W1,
                           __nv_bfloat16* __restrict__ w2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kNP) return;
  const float c1 = 1.f - powf(b1, (float)step);   // bias corrections
  const float c2 = 1.f - powf(b2, (float)step);
  const float g = grad[p];
  const float mp = b1 * m[p] + (1.f - b1) * g;
  const float vp = b2 * v[p] + (1.f - b2) * g * g;
  m[p] = mp;
  v[p] = vp;
  const float th = theta[p] - lr * (mp / c1) / (sqrtf(vp / c2) + eps);
  theta[p] = th;
  if (p < kOffB1) W1[p] = __float2bfloat16_rn(th);
  else if (p >= kOffW2 && p < kOffC) w2[p - kOffW2] = __float2bfloat16_rn(th);
}

__global__ void k_gnn_sync_bf16(const float* __restrict__ theta, __nv_bfloat16* __restrict__ W1,
                                __nv_bfloat16* __restrict__ w2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kOffB1) W1[p] = __float2bfloat16_rn(theta[p]);
  else if (p >= kOffW2 && p < kOffC) w2[p - kOffW2] = __float2bfloat16_rn(theta[p]);
}

__device__ __forceinline__ float clamp_pred(float p, float max_abs) {
  return isfinite(p) ? fminf(fmaxf(p, -max_abs), max_abs) : 0.f;
}

// warm start: out = log_v1 + scale * clamp(pred, -max_abs, max_abs); a
// non-finite prediction contributes 0 (the cold start for that column)
__global__ void k_gnn_warm(int n, const float* __restrict__ lv1, const float* __restrict__ pred,
                           float max_abs, const float* __restrict__ scale,
                           float* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = lv1[i] + (scale ? scale[0] : 1.f) * clamp_pred(pred[i], max_abs);
}

// one block: the centred least-squares scale of clamp(pred) against y,
// clipped to [0, 1] (two fixed-order passes: means, then moments)
__global__ void __launch_bounds__(1024) k_gnn_fit_scale(int n, const float* __restrict__ pred,
                                                        const float* __restrict__ y,
                                                        float max_abs, int shrink,
                                                        float* __restrict__ out) {
  __shared__ double s1[32], s2[32], s3[32];
  __shared__ double mp, my;
  double ap = 0.0, ay = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    ap += clamp_pred(pred[i], max_abs);
    ay += y[i];
  }
  for (int o = 16; o > 0; o >>= 1) {
    ap += __shfl_xor_sync(0xffffffffu, ap, o);
    ay += __shfl_xor_sync(0xffffffffu, ay, o);
  }
  if ((threadIdx.x & 31) == 0) { s1[threadIdx.x >> 5] = ap; s2[threadIdx.x >> 5] = ay; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tp = 0.0, ty = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { tp += s1[w]; ty += s2[w]; }
    mp = tp / n;
    my = ty / n;
  }
  __syncthreads();
  double cxy = 0.0, cxx = 0.0, cyy = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double dp = clamp_pred(pred[i], max_abs) - mp;
    const double dy = (double)y[i] - my;
    cxy += dp * dy;
    cxx += dp * dp;
    cyy += dy * dy;
  }
  for (int o = 16; o > 0; o >>= 1) {
    cxy += __shfl_xor_sync(0xffffffffu, cxy, o);
    cxx += __shfl_xor_sync(0xffffffffu, cxx, o);
    cyy += __shfl_xor_sync(0xffffffffu, cyy, o);
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    s1[threadIdx.x >> 5] = cxy;
    s2[threadIdx.x >> 5] = cxx;
    s3[threadIdx.x >> 5] = cyy;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double txy = 0.0, txx = 0.0, tyy = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { txy += s1[w]; txx += s2[w]; tyy += s3[w]; }
    double a = txx > 0.0 ? txy / txx : 0.0;
    a = a < 0.0 ? 0.0 : (a > 1.0 ? 1.0 : a);
    const double r2 = (txx > 0.0 && tyy > 0.0) ? (txy * txy) / (txx * tyy) : 0.0;
    if (shrink == 1) a *= r2;
    else if (shrink == 2) a *= sqrt(r2);
    out[0] = (float)a;
  }
}

__global__ void k_axpby(int n, float a, const float* __restrict__ x, float b,
                        const float* __restrict__ y, float* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a * x[i] + (y ? b * y[i] : 0.f);
}

}  // namespace fa

// ------------------------------------------------------------ C ABI
struct fa_gnn {
  float* theta = nullptr;           // FP32 master parameters (kNP)
  float* m = nullptr;               // Adam first moment
  float* v = nullptr;               // Adam second moment
  __nv_bfloat16* W1 = nullptr;      // BF16 copy used by the forward pass
  __nv_bfloat16* w2 = nullptr;
  int64_t step = 0;
};

using namespace fa;

extern "C" {

fa_status fa_gnn_create(fa_gnn** out) {
  if (!out) { set_error("fa_gnn_create: out is NULL"); return FA_ERR_ARG; }
  *out = nullptr;
  fa_gnn* g = new fa_gnn();
  cudaError_t e;
  if ((e = cudaMalloc(&g->theta, kNP * 4)) != cudaSuccess || (e = cudaMalloc(&g->m, kNP * 4)) != cudaSuccess ||
      (e = cudaMalloc(&g->v, kNP * 4)) != cudaSuccess || (e = cudaMalloc(&g->W1, kOffB1 * 2)) != cudaSuccess ||
      (e = cudaMalloc(&g->w2, kHid * 2)) != cudaSuccess) {
    cudaGetLastError();
    set_error("fa_gnn_create: %s", cudaGetErrorString(e));
    fa_gnn_destroy(g);
    return FA_ERR_OOM;
  }
  if (cudaMemset(g->theta, 0, kNP * 4) != cudaSuccess || cudaMemset(g->m, 0, kNP * 4) != cudaSuccess ||
      cudaMemset(g->v, 0, kNP * 4) != cudaSuccess || cudaMemset(g->W1, 0, kOffB1 * 2) != cudaSuccess ||
      cudaMemset(g->w2, 0, kHid * 2) != cudaSuccess) {
    set_error("fa_gnn_create: memset failed");
    fa_gnn_destroy(g);
    return FA_ERR_CUDA;
  }
  *out = g;
  return FA_OK;
}

fa_status fa_gnn_destroy(fa_gnn* g) {
  if (!g) return FA_OK;
  if (g->theta) cudaFree(g->theta);
  if (g->m) cudaFree(g->m);
  if (g->v) cudaFree(g->v);
  if (g->W1) cudaFree(g->W1);
  if (g->w2) cudaFree(g->w2);
  delete g;
  return FA_OK;
}

fa_status fa_gnn_set_params(fa_gnn* g, const float* host_theta) {
  if (!g || !host_theta) { set_error("fa_gnn_set_params: NULL argument"); return FA_ERR_ARG; }
  FA_CUDA(cudaMemcpy(g->theta, host_theta, kNP * 4, cudaMemcpyHostToDevice));
  FA_CUDA(cudaMemset(g->m, 0, kNP * 4));
  FA_CUDA(cudaMemset(g->v, 0, kNP * 4));
  g->step = 0;
  k_gnn_sync_bf16<<<(kNP + 255) / 256, 256>>>(g->theta, g->W1, g->w2);
  FA_LAUNCHED("k_gnn_sync_bf16");
  FA_CUDA(cudaDeviceSynchronize());
  return FA_OK;
}

fa_status fa_gnn_get_params(const fa_gnn* g, float* host_theta) {
  if (!g || !host_theta) { set_error("fa_gnn_get_params: NULL argument"); return FA_ERR_ARG; }
  FA_CUDA(cudaMemcpy(host_theta, g->theta, kNP * 4, cudaMemcpyDeviceToHost));
  return FA_OK;
}

int64_t fa_gnn_workspace_floats(int32_t n) { return n < 1 ? -1 : gnn_workspace_floats(n); }

fa_status fa_gnn_features(const fa_graph* g2, const float* log_v1, const float* corr_prev,
                          const float* pot_prev, const float* anchor_mask, int32_t outer_index,
                          float* F, float* ws, fa_stream_t stream) {
  if (!g2 || !log_v1 || !F || !ws) { set_error("fa_gnn_features: NULL argument"); return FA_ERR_ARG; }
  if (outer_index < 0) { set_error("fa_gnn_features: outer_index < 0"); return FA_ERR_ARG; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int n = g2->d.n;
  GnnWs w = ws_layout(ws, n);
  k_means<<<1, 1024, 0, s>>>(n, log_v1, corr_prev, pot_prev, w.scal);
  FA_LAUNCHED("k_means");
  k_gnn_features<<<(n + 255) / 256, 256, 0, s>>>(n, g2->d.row_ptr, log_v1, corr_prev, pot_prev,
                                                 anchor_mask, log1pf((float)outer_index), w.scal, F);
  FA_LAUNCHED("k_gnn_features");
  return FA_OK;
}

fa_status fa_gnn_forward(fa_gnn* g, const fa_graph* graph, const float* F, float* ws, float* a_out,
                         fa_stream_t stream) {
  if (!g || !graph || !F || !ws || !a_out) { set_error("fa_gnn_forward: NULL argument"); return FA_ERR_ARG; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const DevGraph& d = graph->d;
  const int n = d.n;
  GnnWs w = ws_layout(ws, n);
  k_gnn_agg<<<(n + 255) / 256, 256, 0, s>>>(n, d.row_ptr, d.col, d.val_row, F, w.AF);
  FA_LAUNCHED("k_gnn_agg");
  k_gnn_hidden<<<(unsigned)(((int64_t)n * 32 + 255) / 256), 256, 0, s>>>(n, w.AF, g->W1, g->theta,
                                                                          g->w2, w.A1, w.z2);
  FA_LAUNCHED("k_gnn_hidden");
  k_gnn_spmv<<<(n + 255) / 256, 256, 0, s>>>(n, d.row_ptr, d.col, d.val_row, w.z2, g->theta, 1, a_out);
  FA_LAUNCHED("k_gnn_spmv");
  return FA_OK;
}

fa_status fa_gnn_backward(fa_gnn* g, const fa_graph* graph, const float* ws_in, const float* a_pred,
                          const float* target, float* grad, float* loss, fa_stream_t stream) {
  if (!g || !graph || !ws_in || !a_pred || !target || !grad) {
    set_error("fa_gnn_backward: NULL argument");
    return FA_ERR_ARG;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const DevGraph& d = graph->d;
  const int n = d.n;
  GnnWs w = ws_layout(const_cast<float*>(ws_in), n);
  k_means<<<1, 1024, 0, s>>>(n, a_pred, target, nullptr, w.scal);
  FA_LAUNCHED("k_means");
  k_gnn_resid<<<1, 1024, 0, s>>>(n, a_pred, target, w.scal, w.g, loss, grad);
  FA_LAUNCHED("k_gnn_resid");
  // a = Abar z2 + c  =>  dL/dz2 = Abar^T g (Abar^T[i,k] = 1/deg k)
  k_gnn_spmv<<<(n + 255) / 256, 256, 0, s>>>(n, d.row_ptr, d.col, d.val_col, w.g, g->theta, 0, w.gz2);
  FA_LAUNCHED("k_gnn_spmv");
  k_gnn_grad_part<<<w.nb, kGradThreads, 0, s>>>(n, w.AF, w.A1, g->w2, w.gz2, w.part);
  FA_LAUNCHED("k_gnn_grad_part");
  k_gnn_grad_reduce<<<(kNP + 255) / 256, 256, 0, s>>>(w.nb, w.part, grad);
  FA_LAUNCHED("k_gnn_grad_reduce");
  return FA_OK;
}

fa_status fa_gnn_adam_step(fa_gnn* g, const float* grad, float lr, float beta1, float beta2,
                           float eps, fa_stream_t stream) {
  if (!g || !grad) { set_error("fa_gnn_adam_step: NULL argument"); return FA_ERR_ARG; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  g->step += 1;
  k_gnn_adam<<<(kNP + 255) / 256, 256, 0, s>>>(g->theta, g->m, g->v, grad, lr, beta1, beta2, eps,
                                               (int)g->step, g->W1, g->w2);
  FA_LAUNCHED("k_gnn_adam");
  return FA_OK;
}

fa_status fa_gnn_warm_start(int32_t n, const float* log_v1, const float* pred, float max_abs,
                            const float* scale, float* out, fa_stream_t stream) {
  if (n < 1 || !log_v1 || !pred || !out || !(max_abs > 0.f)) {
    set_error("fa_gnn_warm_start: bad argument");
    return FA_ERR_ARG;
  }
  k_gnn_warm<<<(n + 255) / 256, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      n, log_v1, pred, max_abs, scale, out);
  FA_LAUNCHED("k_gnn_warm");
  return FA_OK;
}

fa_status fa_gnn_fit_scale(int32_t n, const float* pred, const float* y, float max_abs,
                           int32_t shrink, float* scale, fa_stream_t stream) {
  if (n < 1 || !pred || !y || !scale || !(max_abs > 0.f)) {
    set_error("fa_gnn_fit_scale: bad argument");
    return FA_ERR_ARG;
  }
  k_gnn_fit_scale<<<1, 1024, 0, reinterpret_cast<cudaStream_t>(stream)>>>(n, pred, y, max_abs,
                                                                          shrink, scale);
  FA_LAUNCHED("k_gnn_fit_scale");
  return FA_OK;
}

fa_status fa_vec_axpby(int32_t n, float a, const float* x, float b, const float* y, float* out,
                       fa_stream_t stream) {
  if (n < 0 || (n > 0 && (!x || !out))) { set_error("fa_vec_axpby: bad argument"); return FA_ERR_ARG; }
  if (n == 0) return FA_OK;
  k_axpby<<<(n + 255) / 256, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(n, a, x, b, y, out);
  FA_LAUNCHED("k_axpby");
  return FA_OK;
}

}  // extern "C"
