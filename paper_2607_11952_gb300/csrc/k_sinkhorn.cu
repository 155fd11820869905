// Phase 3 of Algorithm 1 (Eq. 3): Sinkhorn on the row-stabilised Gibbs
// kernel K, in the scaling form u = exp(b/eps), v = exp(a/eps).
//
// The paper's GPU design (Section 3.6) runs one thread block per column with
// two streaming passes, and a tiled transpose for the other update, i.e.
// several reads of the n1 x n2 matrix per iteration.  Here one sweep reads K
// exactly once per full iteration:
//
//   for every row i:   r_i = sum_j K_ij v_j,  u_i = mu_i / r_i   (b update)
//                      colacc_j += K_ij u_i                       (same pass)
//   at the end:        v_j = nu_j / colacc_j                      (a update)
//
// The row sum must be complete before its column contributions are added,
// so every CTA needs whole rows.  A row of K is split over a thread-block
// cluster of Q CTAs: CTA q owns one column slab and keeps the matching
// slice of v and of the column accumulators in registers for the whole
// sweep.  Per step of R rows, each CTA reduces its slab's partial row sums,
// pushes them into every CTA of the cluster through distributed shared
// memory, and after one cluster barrier all CTAs hold identical row sums.
// K is streamed with 16-byte loads that bypass L1; HBM traffic per sweep is
// n1 x ld x sizeof(K) plus O((n1 + G ld) * 4) bytes of vectors/partials.
#include <cooperative_groups.h>
#include <math.h>
#include <stdlib.h>

#include "fa_internal.cuh"

namespace cg = cooperative_groups;

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
  __device__ static __forceinline__ void unpack(const uint4& u, float (&f)[8]) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float2 t = __bfloat1622float2(h[q]);
      f[2 * q] = t.x;
      f[2 * q + 1] = t.y;
    }
  }
};

__device__ __forceinline__ uint4 ld_stream(const void* p) {
  uint4 r;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "l"(p));
  return r;
}

// ------------------------------------------------------------ plan init
// T0 = mu nu^T (reading: independent coupling): K = 1, log u = log mu,
// log v = log nu.
template <typename TK>
__global__ void k_plan_init(int n1, int n2, int64_t ld, TK* K, float* log_u,
                            float* log_v, float lmu, float lnu) {
  int64_t total = (int64_t)n1 * ld;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t j = t % ld;
    K[t] = (TK)(j < n2 ? 1.0f : 0.0f);
  }
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n1) log_u[t] = lmu;
  if (t < n2) log_v[t] = lnu;
}

fa_status launch_plan_init(int n1, int n2, int64_t ld, void* K, bool bf16,
                           float* log_u, float* log_v, cudaStream_t s) {
  int64_t total = (int64_t)n1 * ld;
  int64_t blocks = (total + 255) / 256;
  int64_t need = ((n1 > n2 ? n1 : n2) + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  if (blocks < need) blocks = need;
  const float lmu = -logf((float)n1), lnu = -logf((float)n2);
  if (bf16)
    k_plan_init<__nv_bfloat16><<<(unsigned)blocks, 256, 0, s>>>(
        n1, n2, ld, static_cast<__nv_bfloat16*>(K), log_u, log_v, lmu, lnu);
  else
    k_plan_init<float><<<(unsigned)blocks, 256, 0, s>>>(
        n1, n2, ld, static_cast<float*>(K), log_u, log_v, lmu, lnu);
  FA_LAUNCHED("k_plan_init");
  return FA_OK;
}

// ------------------------------------------------------------ normalise
// K_ij = exp(x_ij - max_j x_ij) (row stabiliser, reading b0 = -eps m_i) in
// the storage type, and the column sums of the stored values (u = 1): the
// first a update.  Grid: (column slabs of 1024, G row groups).
__device__ __forceinline__ void store4(float* p, const float (&k)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(k[0], k[1], k[2], k[3]);
}
__device__ __forceinline__ void store4(__nv_bfloat16* p, float (&k)[4]) {
  __nv_bfloat162 a = __floats2bfloat162_rn(k[0], k[1]);
  __nv_bfloat162 b = __floats2bfloat162_rn(k[2], k[3]);
  float2 fa_ = __bfloat1622float2(a), fb = __bfloat1622float2(b);
  k[0] = fa_.x; k[1] = fa_.y; k[2] = fb.x; k[3] = fb.y;     // rounded values
  uint2 u;
  u.x = *reinterpret_cast<uint32_t*>(&a);
  u.y = *reinterpret_cast<uint32_t*>(&b);
  *reinterpret_cast<uint2*>(p) = u;
}

template <typename TK>
__global__ void __launch_bounds__(256) k_normalize(
    int n1, int64_t ld, const float* __restrict__ X,
    const float* __restrict__ rowmax, TK* __restrict__ K,
    float* __restrict__ colpart) {
  const int64_t col = (int64_t)blockIdx.x * 1024 + threadIdx.x * 4;
  if (col >= ld) return;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int i = blockIdx.y; i < n1; i += gridDim.y) {
    const float m = rowmax[i];
    float4 x = __ldcs(reinterpret_cast<const float4*>(X + (int64_t)i * ld + col));
    float k[4] = {expf(x.x - m), expf(x.y - m), expf(x.z - m), expf(x.w - m)};
    store4(K + (int64_t)i * ld + col, k);
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[e] += k[e];
  }
  *reinterpret_cast<float4*>(colpart + (int64_t)blockIdx.y * ld + col) =
      make_float4(acc[0], acc[1], acc[2], acc[3]);
}

fa_status launch_normalize_kernel(int n1, int n2, int64_t ld, const float* X,
                                  const float* rowmax, void* K, bool bf16,
                                  float* colpart, int G, cudaStream_t s) {
  (void)n2;
  dim3 grid((unsigned)((ld + 1023) / 1024), (unsigned)G);
  if (bf16)
    k_normalize<__nv_bfloat16><<<grid, 256, 0, s>>>(
        n1, ld, X, rowmax, static_cast<__nv_bfloat16*>(K), colpart);
  else
    k_normalize<float><<<grid, 256, 0, s>>>(n1, ld, X, rowmax,
                                            static_cast<float*>(K), colpart);
  FA_LAUNCHED("k_normalize");
  return FA_OK;
}

// ------------------------------------------------------------ fused sweep
constexpr int kSweepThreads = 256;
constexpr int kMaxQ = 16;

template <typename TK, int S, int R>
__global__ void __launch_bounds__(kSweepThreads, 2) k_sweep(
    const TK* __restrict__ K, int64_t ld, int n1, int n2,
    const float* __restrict__ log_v, float* __restrict__ log_u, float mu,
    float log_mu, float* __restrict__ colpart, int* __restrict__ status) {
  constexpr int V = KT<TK>::V;
  cg::cluster_group cluster = cg::this_cluster();
  const int Q = (int)cluster.num_blocks();
  const int q = (int)cluster.block_rank();
  const int g = blockIdx.x / Q;          // cluster index = row group
  const int G = gridDim.x / Q;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t nvec = ld / V;
  const int64_t vbase = (int64_t)q * S * kSweepThreads + tid;

  __shared__ float red[R][kSweepThreads / 32];
  __shared__ float xch[2][kMaxQ][R];

  float vv[S][V], acc[S][V];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int64_t vec = vbase + (int64_t)s * kSweepThreads;
#pragma unroll
    for (int e = 0; e < V; ++e) {
      const int64_t col = vec * V + e;
      vv[s][e] = (vec < nvec && col < n2) ? expf(log_v[col]) : 0.f;
      acc[s][e] = 0.f;
    }
  }

  int buf = 0;
  int bad = 0;
  for (int i0 = g * R; i0 < n1; i0 += G * R) {
    uint4 kk[R][S];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int row = i0 + r;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const int64_t vec = vbase + (int64_t)s * kSweepThreads;
        if (row < n1 && vec < nvec)
          kk[r][s] = ld_stream(K + (int64_t)row * ld + vec * V);
        else
          kk[r][s] = make_uint4(0u, 0u, 0u, 0u);
      }
    }
    float p[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float t = 0.f;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        float f[V];
        KT<TK>::unpack(kk[r][s], f);
#pragma unroll
        for (int e = 0; e < V; ++e) t += f[e] * vv[s][e];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      p[r] = t;
    }
    if (lane == 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) red[r][warp] = p[r];
    }
    __syncthreads();
    if (tid < R) {
      float t = 0.f;
#pragma unroll
      for (int w = 0; w < kSweepThreads / 32; ++w) t += red[tid][w];
      for (int dst = 0; dst < Q; ++dst) {
        float* rp = cluster.map_shared_rank(&xch[buf][q][tid], dst);
        *rp = t;
      }
    }
    cluster.sync();   // release the DSMEM stores, acquire the peers'
    float u[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float rs = 0.f;
      for (int qq = 0; qq < Q; ++qq) rs += xch[buf][qq][r];
      const int row = i0 + r;
      float ur = 0.f;
      if (row < n1) {
        if (rs > 0.f && isfinite(rs)) {
          ur = mu / rs;
          if (!isfinite(ur)) { ur = 0.f; bad = 1; }
        } else {
          bad = 1;
        }
        if (q == 0 && tid == r) log_u[row] = log_mu - logf(rs);
      }
      u[r] = ur;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
#pragma unroll
      for (int s = 0; s < S; ++s) {
        float f[V];
        KT<TK>::unpack(kk[r][s], f);
#pragma unroll
        for (int e = 0; e < V; ++e) acc[s][e] += u[r] * f[e];
      }
    }
    buf ^= 1;
  }
  if (bad && tid == 0) atomicOr(status, ST_NUMERIC);
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int64_t vec = vbase + (int64_t)s * kSweepThreads;
    if (vec < nvec) {
      float* dst = colpart + (int64_t)g * ld + vec * V;
#pragma unroll
      for (int e = 0; e < V; e += 4)
        *reinterpret_cast<float4*>(dst + e) =
            make_float4(acc[s][e], acc[s][e + 1], acc[s][e + 2], acc[s][e + 3]);
    }
  }
}

using SweepFn = void (*)(const void*, int64_t, int, int, const float*, float*,
                         float, float, float*, int*);

template <typename TK, int S, int R>
static void* sweep_ptr() {
  return reinterpret_cast<void*>(&k_sweep<TK, S, R>);
}

// Register budget (256 threads, 2 CTAs/SM): about 2*S*V + 4*R*S + 20 <= 128.
// Largest spill-free S per R (checked with -Xptxas -v).
static constexpr int kSmaxF32[3] = {0, 8, 6};    // index R
static constexpr int kSmaxBF16[3] = {0, 4, 3};

static void* sweep_kernel(bool bf16, int S, int R) {
#define FA_CASE_F32(SS, RR) if (!bf16 && S == SS && R == RR) return sweep_ptr<float, SS, RR>();
#define FA_CASE_B16(SS, RR) if (bf16 && S == SS && R == RR) return sweep_ptr<__nv_bfloat16, SS, RR>();
  FA_CASE_F32(1, 1) FA_CASE_F32(2, 1) FA_CASE_F32(3, 1) FA_CASE_F32(4, 1)
  FA_CASE_F32(5, 1) FA_CASE_F32(6, 1) FA_CASE_F32(7, 1) FA_CASE_F32(8, 1)
  FA_CASE_F32(1, 2) FA_CASE_F32(2, 2) FA_CASE_F32(3, 2) FA_CASE_F32(4, 2)
  FA_CASE_F32(5, 2) FA_CASE_F32(6, 2)
  FA_CASE_B16(1, 1) FA_CASE_B16(2, 1) FA_CASE_B16(3, 1) FA_CASE_B16(4, 1)
  FA_CASE_B16(1, 2) FA_CASE_B16(2, 2) FA_CASE_B16(3, 2)
#undef FA_CASE_F32
#undef FA_CASE_B16
  return nullptr;
}

static int env_int(const char* name, int dflt) {
  const char* v = getenv(name);
  if (!v || !*v) return dflt;
  return atoi(v);
}

SweepPlan plan_sweep(int n1, int64_t ld, bool bf16, int max_G) {
  SweepPlan sp;
  sp.Q = 0;
  const int V = bf16 ? 8 : 4;
  const int64_t nvec = ld / V;
  const int* smax = bf16 ? kSmaxBF16 : kSmaxF32;
  int Rwant = env_int("FA_SWEEP_R", 2);
  if (Rwant < 1 || Rwant > 2) Rwant = 2;
  int Qforce = env_int("FA_SWEEP_Q", 0);
  for (int Q = 1; Q <= kMaxQ; Q *= 2) {
    if (Qforce && Q != Qforce) continue;
    const int S = (int)((nvec + (int64_t)Q * kSweepThreads - 1) / ((int64_t)Q * kSweepThreads));
    int R = Rwant;
    if (S > smax[R]) R = 1;
    if (S <= smax[R]) {
      sp.Q = Q;
      sp.S = S < 1 ? 1 : S;
      sp.R = R;
      break;
    }
    sp.Q = 0;
  }
  int G = env_int("FA_SWEEP_G", 0);
  if (G <= 0) G = max_G;
  const int rows_needed = (n1 + sp.R - 1) / sp.R;
  if (G > rows_needed) G = rows_needed;
  if (G > max_G) G = max_G;
  if (G < 1) G = 1;
  sp.G = G;
  return sp;
}

fa_status launch_sweep(const SweepPlan& sp, int n1, int n2, int64_t ld,
                       const void* K, bool bf16, const float* log_v,
                       float* log_u, float mu, float* colpart, int* status,
                       cudaStream_t s) {
  if (sp.Q < 1) {
    set_error("fa_sinkhorn: n2=%d too wide for a %d-CTA cluster sweep", n2, kMaxQ);
    return FA_ERR_UNSUPPORTED;
  }
  void* fn = sweep_kernel(bf16, sp.S, sp.R);
  if (!fn) {
    set_error("fa_sinkhorn: no sweep kernel for S=%d R=%d", sp.S, sp.R);
    return FA_ERR_UNSUPPORTED;
  }
  if (sp.Q > 8) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) {
      set_error("cluster size %d not allowed: %s", sp.Q, cudaGetErrorString(e));
      return FA_ERR_UNSUPPORTED;
    }
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(sp.G * sp.Q));
  cfg.blockDim = dim3(kSweepThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)sp.Q;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const float log_mu = logf(mu);
  void* args[] = {(void*)&K, (void*)&ld, (void*)&n1, (void*)&n2,
                  (void*)&log_v, (void*)&log_u, (void*)&mu, (void*)&log_mu,
                  (void*)&colpart, (void*)&status};
  cudaError_t e = cudaLaunchKernelExC(&cfg, fn, args);
  if (e != cudaSuccess) {
    set_error("k_sweep launch (Q=%d S=%d R=%d G=%d): %s", sp.Q, sp.S, sp.R,
              sp.G, cudaGetErrorString(e));
    return FA_ERR_CUDA;
  }
  FA_LAUNCHED("k_sweep");
  return FA_OK;
}

// Number of clusters of the chosen shape that fit on the device at once.
int sweep_max_active_clusters(const SweepPlan& sp, bool bf16) {
  void* fn = sweep_kernel(bf16, sp.S, sp.R);
  if (!fn || sp.Q < 1) return 0;
  if (sp.Q > 8) cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(sp.Q * 64));
  cfg.blockDim = dim3(kSweepThreads);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)sp.Q;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

// ------------------------------------------------------------ finalize
// colsum_j = sum_g colpart[g][j] (fixed order), column marginal
// m_j = v_j colsum_j, err = sum_j |m_j - nu| in FP64 (deterministic two-level
// reduction: per-block partials, summed in index order by the last block),
// and the next column scaling log v_j = log nu - log colsum_j.
constexpr int kFinThreads = 256;

__global__ void __launch_bounds__(kFinThreads) k_col_finalize(
    int n2, int64_t ld, int G, const float* __restrict__ colpart,
    const float* __restrict__ log_v_cur, float nu, float log_nu,
    float* __restrict__ log_v_next, double* __restrict__ err_part,
    unsigned* __restrict__ ticket, double* __restrict__ err_out,
    int* __restrict__ status) {
  __shared__ double sred[kFinThreads / 32];
  __shared__ bool last;
  const int j = blockIdx.x * kFinThreads + threadIdx.x;
  double e = 0.0;
  if (j < n2) {
    float cs = 0.f;
    for (int g = 0; g < G; ++g) cs += colpart[(int64_t)g * ld + j];
    if (log_v_cur) {
      const double m = exp((double)log_v_cur[j]) * (double)cs;
      e = fabs(m - (double)nu);
    }
    float lv;
    if (cs > 0.f && isfinite(cs)) {
      lv = log_nu - logf(cs);
    } else {
      atomicOr(status, ST_NUMERIC);
      lv = log_nu + 87.0f;   // keep finite; the status word reports it
    }
    log_v_next[j] = lv;
  }
  for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
  if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kFinThreads / 32; ++w) t += sred[w];
    err_part[blockIdx.x] = t;
    __threadfence();
    unsigned prev = atomicAdd(ticket, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double t = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b)
      t += ((volatile double*)err_part)[b];
    *err_out = t;
    *ticket = 0u;
  }
}

fa_status launch_col_finalize(int n2, int64_t ld, int G, const float* colpart,
                              const float* log_v_cur, float nu,
                              float* log_v_next, double* err_part,
                              unsigned* ticket, double* err_out, int* status,
                              cudaStream_t s) {
  const int blocks = (n2 + kFinThreads - 1) / kFinThreads;
  k_col_finalize<<<blocks, kFinThreads, 0, s>>>(
      n2, ld, G, colpart, log_v_cur, nu, logf(nu), log_v_next, err_part,
      ticket, err_out, status);
  FA_LAUNCHED("k_col_finalize");
  return FA_OK;
}

}  // namespace fa
