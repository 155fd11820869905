// Fused Sinkhorn sweep, warp-specialised form (Phase 3 of Algorithm 1, Eq. 3).
//
// Same arithmetic and data flow as k_sweep (one read of K per full
// iteration; a thread-block cluster of Q CTAs owns a row, CTA q the column
// slab [q W, (q+1) W) with its slice of v and of the column accumulators in
// registers), but the CTA never synchronises as a whole inside the loop:
//
//   NC compute warps  row pass of step t on ring stage t % NS: partial row
//                     sums, reduced in the warp and left in shared memory
//                     (arrive on pbar); then the column pass of step t - L
//                     once the cluster's full row sums for it have arrived
//                     (wait on xbar), releasing the stage (arrive on empty).
//   producer warp     one lane keeps the ring full with bulk copies
//                     (waits on empty, completes on full).
//   reducer warp      sums the NC warp partials of a step and stores the
//                     CTA's partial row sums into every CTA of the cluster
//                     (st.async, completing on the receiver's xbar).
//
// Compute warps drift freely within the ring and the lag L, so the latency
// of the in-cluster exchange and of the per-step reductions is overlapped
// with other warps' row passes instead of being paid at CTA barriers.
//
// Exchange slots: step k uses slot k % kNXW of xch and xbar.  Before
// sending step k the reducer (a) waits until every local compute warp has
// read step k-2 (xcons), then re-arms that slot for step k+2, and (b) waits
// until its own xbar has received every CTA's step k-2, which each CTA sent
// only after re-arming its slot for step k: so no store of step k can reach
// a slot that still holds an unread step, or a barrier phase not yet armed.
// Every mbarrier wait is bounded; one cluster barrier after initialisation
// and one before exit bracket all remote traffic.
#include <math.h>

#include "fa_internal.cuh"
#include "sweep_dev.cuh"

namespace fa {

constexpr int kNXW = 4;       // exchange slots
constexpr int kMaxQW = 16;    // largest cluster
constexpr int kMaxNSW = 8;    // largest ring
constexpr int kNCW = 8;       // compute warps per CTA
constexpr int kThreadsW = (kNCW + 2) * 32;

__device__ __forceinline__ void mbar_arrive_local(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}

template <typename TK, int S, int R>
__global__ void __launch_bounds__(kThreadsW, 2) k_sweep_ws(
    const TK* __restrict__ K, int64_t ld, int n1, int n2, int W, int NS, int L,
    const float* __restrict__ log_v, float* __restrict__ log_u, float mu,
    float log_mu, float* __restrict__ colpart, int* __restrict__ status) {
  constexpr int V = KT<TK>::V;
  constexpr int V2 = V / 2;
  constexpr int NCT = kNCW * 32;
  extern __shared__ __align__(128) unsigned char smem[];
  TK* ring = reinterpret_cast<TK*>(smem);
  const size_t ring_bytes = (size_t)NS * R * W * sizeof(TK);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + ring_bytes);
  uint64_t* empty = full + kMaxNSW;
  uint64_t* pbar = empty + kMaxNSW;
  uint64_t* xbar = pbar + kMaxNSW;
  uint64_t* xcons = xbar + kNXW;
  float* part = reinterpret_cast<float*>(xcons + kNXW);   // [kMaxNSW][R][kNCW]
  float* xch = part + kMaxNSW * R * kNCW;                  // [kNXW][kMaxQW][R]
  __shared__ int s_dead;

  const int Q = (int)cluster_size();
  const int q = (int)cluster_rank();
  const int g = blockIdx.x / Q;
  const int G = gridDim.x / Q;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nsteps = (n1 + R - 1) / R;
  const int T = g < nsteps ? (nsteps - 1 - g) / G + 1 : 0;   // cluster-uniform
  const uint32_t xch_bytes = (uint32_t)(Q * R * 4);

  if (tid == 0) {
    for (int s = 0; s < kMaxNSW; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), kNCW);
      mbar_init(smem_u32(&pbar[s]), kNCW);
    }
    for (int s = 0; s < kNXW; ++s) {
      mbar_init(smem_u32(&xbar[s]), 1);
      mbar_init(smem_u32(&xcons[s]), kNCW);
    }
    fence_mbar_init();
    s_dead = 0;
    for (int k = 0; k < 2 && k < T; ++k) mbar_expect_tx(smem_u32(&xbar[k]), xch_bytes);
  }
  __syncthreads();
  cluster_arrive();   // every CTA's barriers exist before any remote store
  cluster_wait();

  volatile int* dead = &s_dead;
  auto give_up = [&](int bits) {
    atomicOr(status, bits);
    *dead = 1;
  };

  if (warp < kNCW) {
    // ---------------------------------------------------------- compute
    f2_t vv[S][V2], acc[S][V2];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const int e0 = (s * NCT + tid) * V;
#pragma unroll
      for (int k = 0; k < V2; ++k) {
        const int64_t col = (int64_t)q * W + e0 + 2 * k;
        const float a = (e0 < W && col < n2) ? expf(log_v[col]) : 0.f;
        const float b = (e0 < W && col + 1 < n2) ? expf(log_v[col + 1]) : 0.f;
        vv[s][k] = pk2(a, b);
        acc[s][k] = pk2(0.f, 0.f);
      }
    }
    for (int t = 0; t < T + L; ++t) {
      if (__any_sync(0xffffffffu, *dead)) break;
      if (t < T) {
        // -------- row pass of step t
        const int st = t % NS;
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(smem_u32(&full[st]), (uint32_t)((t / NS) & 1)))) {
          give_up(ST_TIMEOUT);
          break;
        }
        const TK* buf = ring + (size_t)st * R * W;
        const int row0 = (g + t * G) * R;
        float p[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          f2_t pa[2] = {pk2(0.f, 0.f), pk2(0.f, 0.f)};
          if (row0 + r < n1) {
#pragma unroll
            for (int s = 0; s < S; ++s) {
              const int e0 = (s * NCT + tid) * V;
              if (e0 < W) {
                f2_t f[V2];
                pairs(lds128(buf + (size_t)r * W + e0), f, TK());
#pragma unroll
                for (int k = 0; k < V2; ++k) pa[k & 1] = ffma2(f[k], vv[s][k], pa[k & 1]);
              }
            }
          }
          const float2 a = upk2(pa[0]), b = upk2(pa[1]);
          p[r] = (a.x + a.y) + (b.x + b.y);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
          for (int r = 0; r < R; ++r) p[r] += __shfl_xor_sync(0xffffffffu, p[r], o);
        }
        if (lane == 0) {
#pragma unroll
          for (int r = 0; r < R; ++r) part[(st * R + r) * kNCW + warp] = p[r];
          mbar_arrive_local(smem_u32(&pbar[st]));
        }
      }
      const int k = t - L;
      if (k >= 0) {
        // -------- column pass of step k
        const int sl = k % kNXW;
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(smem_u32(&xbar[sl]), (uint32_t)((k / kNXW) & 1)))) {
          give_up(ST_TIMEOUT);
          break;
        }
        // lane r*Q + qq holds CTA qq's partial of row r; sum each group of Q
        float x = lane < Q * R ? xch[(sl * kMaxQW + (lane % Q)) * R + lane / Q] : 0.f;
        for (int o = Q >> 1; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        float rs[R];
#pragma unroll
        for (int r = 0; r < R; ++r) rs[r] = __shfl_sync(0xffffffffu, x, r * Q);
        __syncwarp();
        if (lane == 0) mbar_arrive_local(smem_u32(&xcons[sl]));
        const int st = k % NS;
        const TK* buf = ring + (size_t)st * R * W;
        const int row0 = (g + k * G) * R;
        float u[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int row = row0 + r;
          float ur = 0.f;
          if (row < n1) {
            if (rs[r] > 0.f && isfinite(rs[r])) {
              ur = __fdividef(mu, rs[r]);
              if (!isfinite(ur)) {
                ur = 0.f;
                if (lane == 0) atomicOr(status, ST_NUMERIC);
              }
            } else if (lane == 0) {
              atomicOr(status, ST_NUMERIC);
            }
            if (q == 0 && warp == 0 && lane == r) log_u[row] = log_mu - logf(rs[r]);
          }
          u[r] = ur;
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if (row0 + r < n1) {
            const f2_t u2 = pk2(u[r], u[r]);
#pragma unroll
            for (int s = 0; s < S; ++s) {
              const int e0 = (s * NCT + tid) * V;
              if (e0 < W) {
                f2_t f[V2];
                pairs(lds128(buf + (size_t)r * W + e0), f, TK());
#pragma unroll
                for (int kk = 0; kk < V2; ++kk) acc[s][kk] = ffma2(u2, f[kk], acc[s][kk]);
              }
            }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive_local(smem_u32(&empty[st]));
      }
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const int e0 = (s * NCT + tid) * V;
      if (e0 < W) {
        float* dst = colpart + (int64_t)g * ld + (int64_t)q * W + e0;
#pragma unroll
        for (int k = 0; k < V2; k += 2) {
          const float2 a = upk2(acc[s][k]), b = upk2(acc[s][k + 1]);
          *reinterpret_cast<float4*>(dst + 2 * k) = make_float4(a.x, a.y, b.x, b.y);
        }
      }
    }
  } else if (warp == kNCW) {
    // ---------------------------------------------------------- producer
    if (lane == 0) {
      const TK* Kslab = K + (int64_t)q * W;
      const uint32_t row_bytes = (uint32_t)W * sizeof(TK);
      int issued = 0;
      for (int j = 0; j < T; ++j) {
        const int st = j % NS;
        if (j >= NS) {
          if (*dead) break;
          if (!mbar_wait_bounded(smem_u32(&empty[st]), (uint32_t)(((j - NS) / NS) & 1))) {
            give_up(ST_TIMEOUT);
            break;
          }
        }
        const int row0 = (g + j * G) * R;
        const int nrows = min(R, n1 - row0);
        const uint32_t mb = smem_u32(&full[st]);
        mbar_expect_tx(mb, (uint32_t)nrows * row_bytes);
        for (int r = 0; r < nrows; ++r)
          bulk_g2s(smem_u32(ring + ((size_t)st * R + r) * W), Kslab + (int64_t)(row0 + r) * ld,
                   row_bytes, mb);
        issued = j + 1;
      }
      // after a timeout, wait (bounded) for copies still in flight
      if (*dead) {
        for (int j = max(0, issued - NS); j < issued; ++j)
          mbar_wait_bounded(smem_u32(&full[j % NS]), (uint32_t)((j / NS) & 1));
      }
    }
  } else {
    // ---------------------------------------------------------- reducer
    for (int k = 0; k < T; ++k) {
      if (__any_sync(0xffffffffu, *dead)) break;
      const int st = k % NS;
      if (!__all_sync(0xffffffffu, mbar_wait_bounded(smem_u32(&pbar[st]), (uint32_t)((k / NS) & 1)))) {
        give_up(ST_TIMEOUT);
        break;
      }
      // lane r*NC + w holds warp w's partial of row r; sum each group of NC
      float x = lane < R * kNCW ? part[(st * R + lane / kNCW) * kNCW + lane % kNCW] : 0.f;
#pragma unroll
      for (int o = kNCW >> 1; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (k >= 2) {
        const int sp = (k - 2) % kNXW;
        const uint32_t par = (uint32_t)(((k - 2) / kNXW) & 1);
        bool ok = mbar_wait_bounded(smem_u32(&xcons[sp]), par);
        ok = ok && mbar_wait_bounded(smem_u32(&xbar[sp]), par);
        if (!__all_sync(0xffffffffu, ok)) {
          give_up(ST_TIMEOUT);
          break;
        }
      }
      if (lane == 0 && k + 2 < T) mbar_expect_tx(smem_u32(&xbar[(k + 2) % kNXW]), xch_bytes);
      // lane r*Q + dst sends row r's CTA partial to CTA dst
      const int r = lane / Q, dst = lane % Q;
      const float val = __shfl_sync(0xffffffffu, x, min(r, R - 1) * kNCW);
      if (lane < R * Q) {
        const int sl = k % kNXW;
        const uint32_t slot = smem_u32(xch + (sl * kMaxQW + q) * R + r);
        st_async_f32(map_cluster(slot, (uint32_t)dst), val,
                     map_cluster(smem_u32(&xbar[sl]), (uint32_t)dst));
      }
    }
  }
  __syncwarp();
  // no CTA leaves while a peer may still address its shared memory
  cluster_arrive();
  cluster_wait();
}

template <typename TK, int S, int R>
static void* ws_ptr() {
  return reinterpret_cast<void*>(&k_sweep_ws<TK, S, R>);
}

void* sweep_ws_kernel(bool bf16, int S, int R) {
#define FA_WF(SS) \
  if (!bf16 && S == SS) return R == 2 ? ws_ptr<float, SS, 2>() : ws_ptr<float, SS, 1>();
#define FA_WB(SS)                                                                    \
  if (bf16 && S == SS)                                                               \
    return R == 4 ? ws_ptr<__nv_bfloat16, SS, 4>()                                   \
                  : R == 2 ? ws_ptr<__nv_bfloat16, SS, 2>() : ws_ptr<__nv_bfloat16, SS, 1>();
  FA_WF(1) FA_WF(2) FA_WF(3) FA_WF(4) FA_WF(5) FA_WF(6) FA_WF(7) FA_WF(8)
  FA_WB(1) FA_WB(2) FA_WB(3) FA_WB(4)
#undef FA_WF
#undef FA_WB
  return nullptr;
}

size_t sweep_ws_smem(int NS, int R, int W, bool bf16) {
  const size_t b = bf16 ? 2 : 4;
  return (size_t)NS * R * W * b + (size_t)(3 * kMaxNSW + 2 * kNXW) * 8 +
         (size_t)(kMaxNSW * R * kNCW + kNXW * kMaxQW * R) * sizeof(float);
}

int sweep_ws_threads() { return kThreadsW; }
int sweep_ws_compute_threads() { return kNCW * 32; }

}  // namespace fa
