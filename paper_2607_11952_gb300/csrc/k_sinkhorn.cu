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
// so a row is owned by one thread-block cluster of Q CTAs; CTA q owns a
// column slab (the row's 16-byte units split over the Q CTAs as evenly as
// possible, W the widest slab) and keeps the matching slice of v and of the
// column accumulators in registers for the whole sweep.  Rows arrive through
// a ring of NS shared-memory stages filled by TMA bulk copies (one producer
// thread, mbarrier completion), so HBM latency is hidden by the ring depth,
// not by registers.  Per step of R rows each CTA reduces its slab's partial
// row sums and stores them into every CTA of the cluster (distributed shared
// memory, st.async completing on the receiver's mbarrier, no fences); the
// column update of a step runs one step later, so the exchange latency
// overlaps the next step's partial sums.  With Q = 1 there is no exchange.
// HBM traffic per sweep: n1 x ld x sizeof(K) plus O(n1 + G ld) floats for
// the vectors and partial column sums.
#include <cooperative_groups.h>
#include <math.h>
#include <stdlib.h>

#include <algorithm>

#include "fa_internal.cuh"
#include "sweep_dev.cuh"

namespace cg = cooperative_groups;

namespace fa {

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


constexpr int kMaxQ = 16;           // largest cluster
constexpr int kNX = 4;              // exchange slots (step t uses t % kNX)
constexpr int kMaxNS = 8;           // largest ring
constexpr size_t kSmemBudget = 220 * 1024;

// Shared memory: ring[NS][R][W] of K | full[kMaxNS] + xbar[kNX] mbarriers |
// red[2][R][kNW] | xch[kNX][kMaxQ][R].
//
// Exchange protocol (Q > 1): the partial row sums of step t go to slot
// t % kNX of every CTA of the cluster by st.async, each store completing
// 4 transaction bytes on the receiver's xbar[t % kNX]; a receiver arms that
// barrier for Q*R*4 bytes (its own arrival) before the step can complete
// and re-arms it for step t + kNX once every thread has consumed step t.
// A CTA sends step t only after it has received everybody's step t-2, by
// which time each receiver has consumed step t-4 (the slot's previous user)
// and re-armed it, so kNX = 4 slots never alias.  One cluster barrier after
// the mbarrier initialisation and one before exit bracket all remote
// traffic; every mbarrier wait is bounded.
// CTAs per SM a launch shape is built for: 256-thread CTAs whose threads own
// at most 16 elements of a row run four to an SM, wider ones two.
__host__ __device__ constexpr int sweep_ctas_per_sm(int NT, int elems_per_thread) {
  return NT == 256 ? (elems_per_thread <= 16 ? 4 : 2) : 1;
}

// rs[r] = sum over CTAs c < QQ of xs[c * R + r], in CTA order
template <int R, int QQ>
__device__ __forceinline__ void sum_slots(const float* xs, float (&rs)[R]) {
  if constexpr (R == 2) {
    // both rows of a CTA's slot in one 8-byte load, summed as a pair
    f2_t a = *reinterpret_cast<const f2_t*>(xs);
#pragma unroll
    for (int c = 1; c < QQ; ++c) a = fadd2(a, *reinterpret_cast<const f2_t*>(xs + 2 * c));
    const float2 f = upk2(a);
    rs[0] = f.x;
    rs[1 % R] = f.y;
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float a = 0.f;
#pragma unroll
      for (int c = 0; c < QQ; ++c) a += xs[c * R + r];
      rs[r] = a;
    }
  }
}

template <typename TK, int S, int R, int NT>
__global__ void __launch_bounds__(NT, sweep_ctas_per_sm(NT, S * KT<TK>::V)) k_sweep(
    const TK* __restrict__ K, int64_t ld, int n1, int n2, int W, int NS,
    const float* __restrict__ log_v, float* __restrict__ log_u, float mu,
    float log_mu, float* __restrict__ colpart, int* __restrict__ status) {
  constexpr int V = KT<TK>::V;
  constexpr int NW = NT / 32;
  extern __shared__ __align__(128) unsigned char smem[];
  TK* ring = reinterpret_cast<TK*>(smem);
  const size_t ring_bytes = (size_t)NS * R * W * sizeof(TK);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + ring_bytes);
  uint64_t* xbar = full + kMaxNS;
  float* red = reinterpret_cast<float*>(xbar + kNX);
  float* xch = red + 2 * R * NW;
  __shared__ int s_timeout;

  const int Q = (int)cluster_size();
  const int q = (int)cluster_rank();
  const int g = blockIdx.x / Q;            // cluster = row-step group
  const int G = gridDim.x / Q;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nsteps = (n1 + R - 1) / R;
  const int T = g < nsteps ? (nsteps - 1 - g) / G + 1 : 0;   // cluster-uniform
  // column slab of CTA q: the row's ld / V 16-byte units split as evenly as
  // possible (the first ld/V mod Q slabs one unit wider); W, the widest
  // slab, is the ring's row pitch
  const int units = (int)(ld / V), ubase = units / Q, urem = units - ubase * Q;
  const int Wq = V * (ubase + (q < urem ? 1 : 0));
  const int64_t off = (int64_t)V * (q * ubase + min(q, urem));
  const TK* Kslab = K + off;
  const uint32_t row_bytes = (uint32_t)Wq * sizeof(TK);
  const uint32_t xch_bytes = (uint32_t)(Q * R * 4);

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) mbar_init(smem_u32(&full[s]), 1);
    for (int s = 0; s < kNX; ++s) mbar_init(smem_u32(&xbar[s]), 1);
    fence_mbar_init();
    s_timeout = 0;
    if (Q > 1)
      for (int t = 0; t < min(kNX, T); ++t) mbar_expect_tx(smem_u32(&xbar[t]), xch_bytes);
  }
  __syncthreads();
  if (Q > 1) {   // every CTA's barriers exist before any remote store
    cluster_arrive();
    cluster_wait();
  }

  // v and the column accumulators as packed pairs (columns 2k, 2k+1)
  constexpr int V2 = V / 2;
  f2_t vv[S][V2], acc[S][V2];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int e0 = (s * NT + tid) * V;
#pragma unroll
    for (int k = 0; k < V2; ++k) {
      const int64_t col = off + e0 + 2 * k;
      const float a = (e0 < Wq && col < n2) ? expf(log_v[col]) : 0.f;
      const float b = (e0 < Wq && col + 1 < n2) ? expf(log_v[col + 1]) : 0.f;
      vv[s][k] = pk2(a, b);
      acc[s][k] = pk2(0.f, 0.f);
    }
  }

  // 32-bit shared addresses of this thread's vectors in a ring row.  A
  // vector past the slab edge (e0 >= W) is read at the slab's last vector
  // instead: its v is 0, so it adds nothing to the row sums, and its column
  // accumulators are never stored -- so no per-vector branch is needed.
  uint32_t voff[S];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int e0 = (s * NT + tid) * V;
    voff[s] = (uint32_t)((e0 < Wq ? e0 : Wq - V) * (int)sizeof(TK));
  }
  const uint32_t ring_s = smem_u32(ring);
  const uint32_t rowb = (uint32_t)W * sizeof(TK);
  // vectors s < S-1 are inside the slab for every thread; the last one only
  // for the first warps: skip it warp-uniformly where no lane has one
  const bool last_ok = ((S - 1) * NT + warp * 32) * V < Wq;

  // producer: step t goes to stage t % NS
  int issued = 0;   // meaningful in thread 0 only
  auto issue = [&](int t, int stage) {
    const int row0 = (g + t * G) * R;
    const int nrows = min(R, n1 - row0);
    const uint32_t mb = smem_u32(&full[stage]);
    mbar_expect_tx(mb, (uint32_t)nrows * row_bytes);
    for (int r = 0; r < nrows; ++r)
      bulk_g2s(smem_u32(ring + ((size_t)stage * R + r) * W),
               Kslab + (int64_t)(row0 + r) * ld, row_bytes, mb);
  };
  if (tid == 0) {
    for (int t = 0; t < min(NS, T); ++t) issue(t, t);
    issued = min(NS, T);
  }

  bool dead = false;
  // ring stage and phase parity of step t, and the stage of step t-1
  // (kept incrementally: no runtime division by NS in the loop)
  int st_r = 0, st_c = 0;
  uint32_t ph_r = 0;
  for (int t = 0; t <= T; ++t) {
    if (t < T) {
      // -------- partial row sums of step t
      const int stage = st_r;
      if (!dead && !mbar_wait_bounded(smem_u32(&full[stage]), ph_r)) {
        atomicOr(status, ST_TIMEOUT);
        s_timeout = 1;
      }
      const int row0 = (g + t * G) * R;
      float* rb = red + (t & 1) * R * NW;
      // two independent paired accumulators per row (four FMA chains); the
      // R rows' shuffle trees are interleaved
      const uint32_t sb = ring_s + (uint32_t)(stage * R) * rowb;
      float p[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        f2_t pa[2] = {pk2(0.f, 0.f), pk2(0.f, 0.f)};
        if (row0 + r < n1) {
          const uint32_t rbase = sb + (uint32_t)r * rowb;
#pragma unroll
          for (int s = 0; s < S; ++s) {
            if (s + 1 < S || last_ok) {
              f2_t f[V2];
              pairs(lds128a(rbase + voff[s]), f, TK());
#pragma unroll
              for (int k = 0; k < V2; ++k) pa[k & 1] = ffma2(f[k], vv[s][k], pa[k & 1]);
            }
          }
        }
        const float2 a = upk2(pa[0]), b = upk2(pa[1]);
        p[r] = (a.x + a.y) + (b.x + b.y);
      }
      if constexpr (R == 2) {
        // the two rows' butterfly sums as one paired add per level
        f2_t pp = pk2(p[0], p[1]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float2 h = upk2(pp);
          pp = fadd2(pp, pk2(__shfl_xor_sync(0xffffffffu, h.x, o),
                             __shfl_xor_sync(0xffffffffu, h.y, o)));
        }
        const float2 h = upk2(pp);
        p[0] = h.x;
        p[1 % R] = h.y;
      } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
          for (int r = 0; r < R; ++r) p[r] += __shfl_xor_sync(0xffffffffu, p[r], o);
        }
      }
      if (lane == 0) {
#pragma unroll
        for (int r = 0; r < R; ++r) rb[r * NW + warp] = p[r];
      }
      __syncthreads();
      if (Q > 1 && tid < R) {
        float sum = 0.f;
#pragma unroll
        for (int w = 0; w < NW; ++w) sum += rb[tid * NW + w];
        const uint32_t slot = smem_u32(xch + ((t % kNX) * kMaxQ + q) * R + tid);
        const uint32_t bar = smem_u32(&xbar[t % kNX]);
        for (int dst = 0; dst < Q; ++dst)
          st_async_f32(map_cluster(slot, (uint32_t)dst), sum, map_cluster(bar, (uint32_t)dst));
      }
    }
    if (t > 0) {
      // -------- step t-1: full row sums, u, column accumulation
      const int tp = t - 1;
      if (Q > 1 && !dead &&
          !mbar_wait_bounded(smem_u32(&xbar[tp % kNX]), (uint32_t)((tp / kNX) & 1))) {
        atomicOr(status, ST_TIMEOUT);
        s_timeout = 1;
      }
      const int stage = st_c;
      const int row0 = (g + tp * G) * R;
      const uint32_t sb = ring_s + (uint32_t)(stage * R) * rowb;
      const float* rbp = red + (tp & 1) * R * NW;
      // full row sums: the Q CTA partials of the exchange slot, summed in
      // CTA order (fully unrolled per cluster size: independent loads at
      // constant offsets; the same order in every CTA, so u is identical
      // across the cluster)
      float rsum[R];
      if (Q > 1) {
        const float* xs = xch + (tp % kNX) * kMaxQ * R;
        switch (Q) {
          case 2: sum_slots<R, 2>(xs, rsum); break;
          case 3: sum_slots<R, 3>(xs, rsum); break;
          case 4: sum_slots<R, 4>(xs, rsum); break;
          case 5: sum_slots<R, 5>(xs, rsum); break;
          case 6: sum_slots<R, 6>(xs, rsum); break;
          case 7: sum_slots<R, 7>(xs, rsum); break;
          case 8: sum_slots<R, 8>(xs, rsum); break;
          case 9: sum_slots<R, 9>(xs, rsum); break;
          case 10: sum_slots<R, 10>(xs, rsum); break;
          case 11: sum_slots<R, 11>(xs, rsum); break;
          case 12: sum_slots<R, 12>(xs, rsum); break;
          case 13: sum_slots<R, 13>(xs, rsum); break;
          case 14: sum_slots<R, 14>(xs, rsum); break;
          case 15: sum_slots<R, 15>(xs, rsum); break;
          default: sum_slots<R, 16>(xs, rsum); break;   // Q = 16 (kMaxQ)
        }
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          rsum[r] = 0.f;
#pragma unroll
          for (int w = 0; w < NW; ++w) rsum[r] += rbp[r * NW + w];
        }
      }
      float u[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float rs = rsum[r];
        const int row = row0 + r;
        float ur = 0.f;
        if (row < n1) {
          if (rs > 0.f && isfinite(rs)) {
            ur = __fdividef(mu, rs);   // identical in every CTA of the cluster
            if (!isfinite(ur)) { ur = 0.f; atomicOr(status, ST_NUMERIC); }
          } else if (tid == 0) {
            atomicOr(status, ST_NUMERIC);
          }
          if (q == 0 && tid == r) log_u[row] = log_mu - logf(rs);
        }
        u[r] = ur;
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (row0 + r < n1) {
          const f2_t u2 = pk2(u[r], u[r]);
          const uint32_t rbase = sb + (uint32_t)r * rowb;
#pragma unroll
          for (int s = 0; s < S; ++s) {
            if (s + 1 < S || last_ok) {
              f2_t f[V2];
              pairs(lds128a(rbase + voff[s]), f, TK());
#pragma unroll
              for (int k = 0; k < V2; ++k) acc[s][k] = ffma2(u2, f[k], acc[s][k]);
            }
          }
        }
      }
      __syncthreads();   // stage tp, red[tp & 1] and slot tp % kNX consumed
      dead = s_timeout != 0;
      if (tid == 0) {
        if (Q > 1 && tp + kNX < T) mbar_expect_tx(smem_u32(&xbar[tp % kNX]), xch_bytes);
        if (!dead && tp + NS < T) {
          issue(tp + NS, stage);
          issued = tp + NS + 1;
        }
      }
    }
    st_c = st_r;
    if (++st_r == NS) {
      st_r = 0;
      ph_r ^= 1u;
    }
  }
  // after a timeout, wait (bounded) for copies still in flight into the ring
  if (tid == 0 && dead) {
    for (int t = max(0, issued - NS); t < issued; ++t)
      mbar_wait_bounded(smem_u32(&full[t % NS]), (uint32_t)((t / NS) & 1));
  }
  if (Q > 1) {   // no CTA leaves while a peer may still address its memory
    cluster_arrive();
    cluster_wait();
  }
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int e0 = (s * NT + tid) * V;
    if (e0 < Wq) {
      float* dst = colpart + (int64_t)g * ld + off + e0;
#pragma unroll
      for (int k = 0; k < V2; k += 2) {
        const float2 a = upk2(acc[s][k]), b = upk2(acc[s][k + 1]);
        *reinterpret_cast<float4*>(dst + 2 * k) = make_float4(a.x, a.y, b.x, b.y);
      }
    }
  }
}

template <typename TK, int S, int R>
static void* sweep_ptr(int NT) {
  if (NT == 1024) {   // 64 registers per thread: only small slabs per thread
    if constexpr (S <= (sizeof(TK) == 2 ? 3 : 6))
      return reinterpret_cast<void*>(&k_sweep<TK, S, R, 1024>);
    else
      return nullptr;
  }
  return NT == 256 ? reinterpret_cast<void*>(&k_sweep<TK, S, R, 256>)
                   : reinterpret_cast<void*>(&k_sweep<TK, S, R, 512>);
}

// Largest S (16-byte vectors per thread and row) kept in registers without
// spills at 512 threads: v and the column accumulators take 2*S*V floats.
static constexpr int kSmaxF32 = 12;
static constexpr int kSmaxBF16 = 6;

static void* sweep_kernel(bool bf16, int S, int R, int NT) {
#define FA_F(SS) \
  if (!bf16 && S == SS) return R == 2 ? sweep_ptr<float, SS, 2>(NT) : sweep_ptr<float, SS, 1>(NT);
#define FA_B(SS) \
  if (bf16 && S == SS)                                                         \
    return R == 4 ? sweep_ptr<__nv_bfloat16, SS, 4>(NT)                        \
                  : R == 2 ? sweep_ptr<__nv_bfloat16, SS, 2>(NT) : sweep_ptr<__nv_bfloat16, SS, 1>(NT);
  FA_F(1) FA_F(2) FA_F(3) FA_F(4) FA_F(5) FA_F(6) FA_F(7) FA_F(8) FA_F(9)
  FA_F(10) FA_F(11) FA_F(12)
  FA_B(1) FA_B(2) FA_B(3) FA_B(4) FA_B(5) FA_B(6) FA_B(7)
#undef FA_F
#undef FA_B
  return nullptr;
}

static int env_int(const char* name, int dflt) {
  const char* v = getenv(name);
  if (!v || !*v) return dflt;
  return atoi(v);
}

// warp-specialised sweep (k_sweep_ws.cu)
void* sweep_ws_kernel(bool bf16, int S, int R);
size_t sweep_ws_smem(int NS, int R, int W, bool bf16);
int sweep_ws_threads();
int sweep_ws_compute_threads();

static size_t sweep_smem(const SweepPlan& sp, bool bf16) {
  const size_t b = bf16 ? 2 : 4;
  return (size_t)sp.NS * sp.R * sp.W * b + (size_t)(kMaxNS + kNX) * 8 +
         (size_t)(2 * sp.R * (sp.NT / 32) + kNX * kMaxQ * sp.R) * sizeof(float);
}

// Pick the smallest cluster whose column slab fits the register budget and
// leaves at least 3 ring stages (2 for very wide rows); R = 2 rows per step
// when the ring still has >= 3 stages.  FA_SWEEP_{Q,R,NS} override (tuning).
// Warp-specialised sweep (k_sweep_ws.cu): 8 compute warps (256 threads own
// the slab), two CTAs per SM; smallest cluster whose slab fits the
// instantiated register shapes, R up to 4 (BF16) or 2 rows per step with
// Q R <= 32, and a ring of at least L + 2 stages (L + 1 for very wide rows).
static SweepPlan plan_sweep_ws(int64_t ld, bool bf16) {
  SweepPlan sp;
  sp.Q = 0;
  sp.kind = 1;
  const int V = bf16 ? 8 : 4;
  const size_t b = bf16 ? 2 : 4;
  int L = env_int("FA_SWEEP_L", 1);
  L = L < 1 ? 1 : (L > 2 ? 2 : L);
  const int Qforce = env_int("FA_SWEEP_Q", 0);
  const int Rforce = env_int("FA_SWEEP_R", 0);
  const int NSforce = env_int("FA_SWEEP_NS", 0);
  const int NTC = sweep_ws_compute_threads();
  const int smax = bf16 ? 4 : 8;   // register shapes that run without spills
  const size_t budget = kSmemBudget / 2;
  for (int pass = 0; pass < 2 && sp.Q == 0; ++pass) {
    const int min_ns = pass == 0 ? L + 2 : L + 1;
    for (int Q = 1; Q <= kMaxQ && sp.Q == 0; Q *= 2) {
      if (Qforce && Q != Qforce) continue;
      if (ld % Q) continue;
      const int64_t W = ld / Q;
      if ((W * (int64_t)b) % 16) continue;
      const int S = (int)((W + (int64_t)NTC * V - 1) / ((int64_t)NTC * V));
      if (S > smax) continue;
      for (int R = bf16 ? 4 : 2; R >= 1; R /= 2) {
        if (Rforce && R != Rforce) continue;
        if (Q * R > 32) continue;
        const size_t fixed = sweep_ws_smem(0, R, (int)W, bf16);
        int NS = (int)((budget - fixed) / ((size_t)R * W * b));
        if (NS > kMaxNS) NS = kMaxNS;
        if (NSforce) NS = NSforce < NS ? NSforce : NS;
        if (NS >= min_ns) {
          sp.Q = Q;
          sp.W = (int)W;
          sp.S = S;
          sp.R = R;
          sp.NS = NS;
          sp.NT = NTC;
          sp.L = L;
          break;
        }
      }
    }
  }
  return sp;
}

// tensor-core row-pass sweep (k_sweep_mma.cu)
void* sweep_mma_kernel(int S, int NW, int MINB);
size_t sweep_mma_smem(int NS, int R, int W, int NW);

// Shape of the tensor-core sweep: two stages of R rows (R <= 8; the MMA
// tile holds 8) per CTA, two 128-thread CTAs per SM when they fit, else one
// 256-thread CTA.  Larger R first (fewer steps, less per-step overhead),
// then the smaller cluster.  FA_SWEEP_MB / FA_SWEEP_Q / FA_SWEEP_R force
// the CTAs per SM, the cluster size and the rows per step (tuning).
static SweepPlan plan_sweep_mma(int64_t ld) {
  SweepPlan sp;
  sp.Q = 0;
  sp.kind = 2;
  const int MBforce = env_int("FA_SWEEP_MB", 0);
  const int Qforce = env_int("FA_SWEEP_Q", 0);
  const int Rforce = env_int("FA_SWEEP_R", 0);
  int NS = env_int("FA_SWEEP_NS", 2);
  NS = NS < 2 ? 2 : (NS > 4 ? 4 : NS);
  const size_t sm_bytes = 228 * 1024, reserved = 1024, cta_max = 227 * 1024;
  for (int MB = 2; MB >= 1 && sp.Q == 0; --MB) {
    if (MBforce && MB != MBforce) continue;
    const int NW = MB == 2 ? 4 : 8;
    const int smax = MB == 2 ? 6 : 8;         // instantiated register shapes
    const size_t budget = std::min(cta_max, sm_bytes / MB - reserved);
    const int rmin = MB == 2 ? 6 : 4;
    for (int R = 8; R >= rmin && sp.Q == 0; --R) {
      if (Rforce && R != Rforce) continue;
      for (int Q = 1; Q <= kMaxQ; Q *= 2) {
        if (Qforce && Q != Qforce) continue;
        if (ld % Q) continue;
        const int64_t W = ld / Q;
        if (W % 8) continue;
        const int64_t vecs = W / 8;
        const int S = (int)((vecs + NW * 32 - 1) / (NW * 32));
        if (S > smax) continue;
        if (sweep_mma_smem(NS, R, (int)W, NW) > budget) continue;
        sp.Q = Q;
        sp.W = (int)W;
        sp.S = S;
        sp.R = R;
        sp.NS = NS;
        sp.NT = NW * 32;
        sp.MB = MB;
        break;
      }
    }
  }
  return sp;
}

SweepPlan plan_sweep(int n1, int64_t ld, bool bf16, int max_G) {
  SweepPlan sp;
  sp.Q = 0;
  // FA_SWEEP_KIND selects the sweep: 0 (default) CTA-synchronous,
  // 1 warp-specialised, 2 tensor-core row pass (BF16 storage only)
  const int kind_env = env_int("FA_SWEEP_KIND", 0);
  if (bf16 && kind_env == 2) {
    sp = plan_sweep_mma(ld);
    if (sp.Q > 0) {
      int G = env_int("FA_SWEEP_G", 0);
      if (G <= 0) G = max_G;
      const int steps = (n1 + sp.R - 1) / sp.R;
      if (G > steps) G = steps;
      if (G > max_G) G = max_G;
      if (G < 1) G = 1;
      sp.G = G;
      return sp;
    }
    sp = SweepPlan();   // no tensor-core shape: fall back below
    sp.Q = 0;
  }
  if (kind_env == 1) {
    sp = plan_sweep_ws(ld, bf16);
    if (sp.Q > 0) {
      int G = env_int("FA_SWEEP_G", 0);
      if (G <= 0) G = max_G;
      const int steps = (n1 + sp.R - 1) / sp.R;
      if (G > steps) G = steps;
      if (G > max_G) G = max_G;
      if (G < 1) G = 1;
      sp.G = G;
      return sp;
    }
    sp = SweepPlan();   // no warp-specialised shape: fall back below
    sp.Q = 0;
  }
  sp.kind = 0;
  const int V = bf16 ? 8 : 4;
  const size_t b = bf16 ? 2 : 4;
  const int Qforce = env_int("FA_SWEEP_Q", 0);
  const int Rforce = env_int("FA_SWEEP_R", 0);
  const int NSforce = env_int("FA_SWEEP_NS", 0);
  // 512 threads and one CTA per SM, or 256 threads and two CTAs per SM
  // (half the shared memory each)
  // measured on GB300 (10k and 50k rows, FP32 and BF16): 256 threads with two
  // CTAs per SM is as fast or faster than 512 (one CTA) and 1024 threads
  const int nt_env = env_int("FA_SWEEP_NT", 256);
  const int NT = (nt_env == 256 || nt_env == 1024) ? nt_env : 512;
  int smax = NT == 1024 ? (bf16 ? 3 : 6) : (bf16 ? kSmaxBF16 : kSmaxF32);
  const int smax_env = env_int("FA_SWEEP_SMAX", 0);
  if (smax_env > 0 && (smax_env < smax || (bf16 && NT == 256 && smax_env == 7))) smax = smax_env;
  // The row's ld / V 16-byte units are split as evenly as possible over the
  // Q CTAs (slab widths differ by at most one unit), so Q need not divide
  // ld; W is the widest slab.  A step costs a fixed part (barriers, the
  // exchange) plus a part per round of NT vectors, so a shape should have
  // few rounds, a nearly full last round and, where the ring allows, two
  // rows per step.  BF16 default rule (measured on GB300, 50,000 rows and
  // 30k-110k columns: it picks the fastest of the rules below at every
  // width):
  //   1. the smallest power-of-two cluster up to 8 whose slab takes at most
  //      5 vectors per thread with the last round at least 80% full;
  //   2. else the smallest cluster up to 10 with at most 5 vectors;
  //   3. else the smallest cluster of any size that fits the register
  //      shapes.
  // FP32, already at the copy peak, keeps powers of two.  FA_SWEEP_ANYQ=0
  // forces powers of two, =1 the smallest cluster of any size.
  const int64_t units = ld / V;
  const int qrule = env_int("FA_SWEEP_ANYQ", bf16 ? 2 : 0);
  auto fit = [&](int Q, int min_ns, int s_cap, double min_fill) -> bool {
    if (Qforce && Q != Qforce) return false;
    if (units < Q) return false;
    const int64_t W = V * ((units + Q - 1) / Q);
    const int S = (int)((W + (int64_t)NT * V - 1) / ((int64_t)NT * V));
    if (S > s_cap) return false;
    if ((double)(W / V) < min_fill * (double)S * NT) return false;
    const size_t budget = kSmemBudget / sweep_ctas_per_sm(NT, S * V);
    for (int R = bf16 ? 4 : 2; R >= 1; R /= 2) {
      if (Rforce && R != Rforce) continue;
      const size_t fixed = (size_t)(kMaxNS + kNX) * 8 + (size_t)(2 * R * (NT / 32) + kNX * kMaxQ * R) * 4;
      int NS = (int)((budget - fixed) / ((size_t)R * W * b));
      if (NS > kMaxNS) NS = kMaxNS;
      if (NSforce) NS = NSforce < NS ? NSforce : NS;
      if (NS >= min_ns) {
        sp.Q = Q;
        sp.W = (int)W;
        sp.S = S;
        sp.R = R;
        sp.NS = NS;
        sp.NT = NT;
        return true;
      }
    }
    return false;
  };
  for (int pass = 0; pass < 2 && sp.Q == 0; ++pass) {
    const int min_ns = pass == 0 ? 3 : 2;
    if (qrule == 2) {
      const int s5 = smax < 5 ? smax : 5;
      for (int Q = 1; Q <= 8 && sp.Q == 0; Q *= 2) fit(Q, min_ns, s5, 0.8);
      for (int Q = 1; Q <= 10 && sp.Q == 0; ++Q) fit(Q, min_ns, s5, 0.0);
      for (int Q = 1; Q <= kMaxQ && sp.Q == 0; ++Q) fit(Q, min_ns, smax, 0.0);
    } else {
      for (int Q = 1; Q <= kMaxQ && sp.Q == 0; Q = qrule ? Q + 1 : 2 * Q)
        fit(Q, min_ns, smax, 0.0);
    }
  }
  if (sp.Q == 0) return sp;
  int G = env_int("FA_SWEEP_G", 0);
  if (G <= 0) G = max_G;
  const int steps = (n1 + sp.R - 1) / sp.R;
  if (G > steps) G = steps;
  if (G > max_G) G = max_G;
  if (G < 1) G = 1;
  sp.G = G;
  return sp;
}

static size_t sweep_dyn_smem(const SweepPlan& sp, bool bf16) {
  if (sp.kind == 2) return sweep_mma_smem(sp.NS, sp.R, sp.W, sp.NT / 32);
  return sp.kind ? sweep_ws_smem(sp.NS, sp.R, sp.W, bf16) : sweep_smem(sp, bf16);
}
static void* sweep_fn(const SweepPlan& sp, bool bf16) {
  if (sp.kind == 2) return bf16 ? sweep_mma_kernel(sp.S, sp.NT / 32, sp.MB) : nullptr;
  return sp.kind ? sweep_ws_kernel(bf16, sp.S, sp.R) : sweep_kernel(bf16, sp.S, sp.R, sp.NT);
}

static cudaLaunchConfig_t sweep_config(const SweepPlan& sp, bool bf16, unsigned grid,
                                       cudaLaunchAttribute* attr, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3((unsigned)(sp.kind == 1 ? sweep_ws_threads() : sp.NT));
  cfg.dynamicSmemBytes = sweep_dyn_smem(sp, bf16);
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)sp.Q;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

static cudaError_t prepare_sweep(void* fn, const SweepPlan& sp, bool bf16) {
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sweep_dyn_smem(sp, bf16));
  if (e != cudaSuccess) return e;
  if (sp.Q > 8) e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

fa_status launch_sweep(const SweepPlan& sp, int n1, int n2, int64_t ld,
                       const void* K, bool bf16, const float* log_v,
                       float* log_u, float mu, float* colpart, int* status,
                       cudaStream_t s) {
  if (sp.Q < 1) {
    set_error("fa_sinkhorn: no cluster shape fits a row of %lld elements", (long long)ld);
    return FA_ERR_UNSUPPORTED;
  }
  void* fn = sweep_fn(sp, bf16);
  if (!fn) {
    set_error("fa_sinkhorn: no sweep kernel for S=%d R=%d", sp.S, sp.R);
    return FA_ERR_UNSUPPORTED;
  }
  cudaError_t e = prepare_sweep(fn, sp, bf16);
  if (e != cudaSuccess) {
    set_error("k_sweep attributes: %s", cudaGetErrorString(e));
    return FA_ERR_UNSUPPORTED;
  }
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = sweep_config(sp, bf16, (unsigned)(sp.G * sp.Q), attr, s);
  const float log_mu = logf(mu);
  int W = sp.W, NS = sp.NS, L = sp.L;
  void* args[] = {(void*)&K, (void*)&ld, (void*)&n1, (void*)&n2, (void*)&W,
                  (void*)&NS, (void*)&log_v, (void*)&log_u, (void*)&mu,
                  (void*)&log_mu, (void*)&colpart, (void*)&status};
  void* args_ws[] = {(void*)&K, (void*)&ld, (void*)&n1, (void*)&n2, (void*)&W,
                     (void*)&NS, (void*)&L, (void*)&log_v, (void*)&log_u, (void*)&mu,
                     (void*)&log_mu, (void*)&colpart, (void*)&status};
  int R = sp.R;
  void* args_mma[] = {(void*)&K, (void*)&ld, (void*)&n1, (void*)&n2, (void*)&W,
                      (void*)&NS, (void*)&R, (void*)&log_v, (void*)&log_u, (void*)&mu,
                      (void*)&log_mu, (void*)&colpart, (void*)&status};
  e = cudaLaunchKernelExC(&cfg, fn, sp.kind == 2 ? args_mma : sp.kind ? args_ws : args);
  if (e != cudaSuccess) {
    set_error("k_sweep launch (kind=%d Q=%d S=%d R=%d NS=%d G=%d): %s", sp.kind, sp.Q, sp.S,
              sp.R, sp.NS, sp.G, cudaGetErrorString(e));
    return FA_ERR_CUDA;
  }
  if (sp.kind == 2) FA_LAUNCHED("k_sweep_mma");
  else if (sp.kind) FA_LAUNCHED("k_sweep_ws");
  else FA_LAUNCHED("k_sweep");
  return FA_OK;
}

// Number of clusters of the chosen shape that fit on the device at once.
int sweep_max_active_clusters(const SweepPlan& sp, bool bf16) {
  void* fn = sweep_fn(sp, bf16);
  if (!fn || sp.Q < 1) return 0;
  if (prepare_sweep(fn, sp, bf16) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = sweep_config(sp, bf16, (unsigned)(sp.Q * 64), attr, 0);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

// ------------------------------------------------------------ finalize
// colsum_j = sum_g colpart[g][j] (in the order g = 0, 1, ..., G-1), column
// marginal m_j = v_j colsum_j, err = sum_j |m_j - nu| in FP64 (deterministic
// two-level reduction: per-block partials, summed by the last block in a
// fixed order), and the next column scaling log v_j = log nu - log colsum_j.
// Four columns per thread: colpart rows are read as 16-byte vectors (ld and
// the column offsets passed in are multiples of 4); the log_v arrays are
// read and written element by element (no alignment assumed).  v_j enters
// the error through expf widened to FP64: the FP32 column sums already
// carry a relative error of about G 2^-24, far above expf's.
constexpr int kFinThreads = 256;
constexpr int kFinCols = 4;

__global__ void __launch_bounds__(kFinThreads) k_col_finalize(
    int n2, int64_t ld, int G, const float* __restrict__ colpart,
    const float* __restrict__ log_v_cur, float nu, float log_nu,
    float* __restrict__ log_v_next, double* __restrict__ err_part,
    unsigned* __restrict__ ticket, double* __restrict__ err_out,
    int* __restrict__ status) {
  __shared__ double sred[kFinThreads / 32];
  __shared__ bool last;
  const int j = (blockIdx.x * kFinThreads + threadIdx.x) * kFinCols;
  double e = 0.0;
  if (j < n2) {
    const float* p = colpart + j;
    float4 cs = make_float4(0.f, 0.f, 0.f, 0.f);
    int g = 0;
    for (; g + 4 <= G; g += 4) {   // four rows in flight, added in row order
      const float4 a0 = __ldcs(reinterpret_cast<const float4*>(p + (int64_t)g * ld));
      const float4 a1 = __ldcs(reinterpret_cast<const float4*>(p + (int64_t)(g + 1) * ld));
      const float4 a2 = __ldcs(reinterpret_cast<const float4*>(p + (int64_t)(g + 2) * ld));
      const float4 a3 = __ldcs(reinterpret_cast<const float4*>(p + (int64_t)(g + 3) * ld));
      cs.x += a0.x; cs.y += a0.y; cs.z += a0.z; cs.w += a0.w;
      cs.x += a1.x; cs.y += a1.y; cs.z += a1.z; cs.w += a1.w;
      cs.x += a2.x; cs.y += a2.y; cs.z += a2.z; cs.w += a2.w;
      cs.x += a3.x; cs.y += a3.y; cs.z += a3.z; cs.w += a3.w;
    }
    for (; g < G; ++g) {
      const float4 a = __ldcs(reinterpret_cast<const float4*>(p + (int64_t)g * ld));
      cs.x += a.x; cs.y += a.y; cs.z += a.z; cs.w += a.w;
    }
    const float c4[kFinCols] = {cs.x, cs.y, cs.z, cs.w};
#pragma unroll
    for (int k = 0; k < kFinCols; ++k) {
      const int jj = j + k;
      if (jj >= n2) break;
      const float c = c4[k];
      if (log_v_cur) {
        const double m = (double)expf(log_v_cur[jj]) * (double)c;
        e += fabs(m - (double)nu);
      }
      float lv;
      if (c > 0.f && isfinite(c)) {
        lv = log_nu - logf(c);
      } else {
        atomicOr(status, ST_NUMERIC);
        lv = log_nu + 87.0f;   // keep finite; the status word reports it
      }
      log_v_next[jj] = lv;
    }
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
  if (last) {
    // the last block sums the block partials: thread t takes blocks t,
    // t + 256, ... in order, then a fixed tree
    __threadfence();
    double t = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += kFinThreads)
      t += ((volatile double*)err_part)[b];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
      double u = 0.0;
      for (int w = 0; w < kFinThreads / 32; ++w) u += sred[w];
      *err_out = u;
      *ticket = 0u;
    }
  }
}

int col_finalize_blocks(int n2) {
  const int per = kFinThreads * kFinCols;
  return (n2 + per - 1) / per;
}

fa_status launch_col_finalize(int n2, int64_t ld, int G, const float* colpart,
                              const float* log_v_cur, float nu,
                              float* log_v_next, double* err_part,
                              unsigned* ticket, double* err_out, int* status,
                              cudaStream_t s) {
  if ((reinterpret_cast<uintptr_t>(colpart) & 15u) != 0 || (ld & 3) != 0) {
    set_error("column finalisation: partial sums not 16-byte aligned");
    return FA_ERR_ARG;
  }
  const int blocks = col_finalize_blocks(n2);
  k_col_finalize<<<blocks, kFinThreads, 0, s>>>(
      n2, ld, G, colpart, log_v_cur, nu, logf(nu), log_v_next, err_part,
      ticket, err_out, status);
  FA_LAUNCHED("k_col_finalize");
  return FA_OK;
}

}  // namespace fa
